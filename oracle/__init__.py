"""Plain, slow FP64 CPU oracle of the bidomain time step.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA library and
its Python binding never do.  It shares no code with the CUDA path: its inputs
come from the seeded generators in ``workloads`` (geometry and parameters only).

Contents (paper sections in brackets):
  bidomain.py   P1 assembly of S_1, S_i, S_e, S_m, M, M_H [Sec. 3.1], the
                Mitchell-Schaeffer reaction term, the resolution algorithm's
                three steps [Sec. 3.2], the solve of Step 2 by pinned sparse
                direct factorisation, by plain CG or by dense pseudo-inverse
                [Prop. 1], the normalisation [proof of Prop. 1], and the
                block-LU preconditioner at its exact limit P_1 = S_1,
                P_K = K_m [Def. 5.1, eq. prec2, Sec. 5.2]; the Crank-Nicolson and
                Strang-splitting time schemes [Remark on the time discretisation]
                with Heun's method for the reaction half steps.
  algebra.py    dense matrices of Props. 2-3 and Remark K (tiny meshes only).

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
closed forms, textbook element matrices, invariants stated in the paper, or an
independent special case (see tests/test_oracle_*.py).  The Mitchell-Schaeffer
constants are not in the paper (it uses Luo-Rudy II); they are workload inputs.
"""
