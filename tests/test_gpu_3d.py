"""GPU parity of the 3D slab, precision form (factors in FP64, FP32 and BF16).

The 1 x 1 x 0.3 cm orthotropic slab with the fibre angle rotating from -60 to
+60 degrees through the depth, isolated heart (Pi = Id, N_H = N).  At
65 x 65 x 21 nodes every factor precision is compared with the oracle's FP64
solve (plain projected CG to relative residual 1e-14): U and V each agree
within 1e-9 of the oracle's, relative to the oracle block's largest entry,
whatever the factor storage, because PCG stops on the FP64 residual (1e-14 on
both sides; see test_gpu_parity for why not 1e-13).  At 161 x 161 x 49 nodes (N = 1 270 129) the BF16 form is
checked by properties: the true residual against the oracle's Lambda and the
normalisation.
"""
import numpy as np
import pytest

from oracle import bidomain as ob
from potentials import assert_potentials_close
from workloads import slab_3d, params_3d, stimulus_centre_ball

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def bid():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_08708_gb300 import bid as b
    return b


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def H(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def slab65(bid):
    mesh, p = slab_3d(65, 65, 21), params_3d(0.05)
    S = bid.System(mesh, p)
    o = ob.build_system(mesh, p)
    assert (S.perm == o.order).all() and o.N == o.NH == 88725
    rng = np.random.default_rng(31)
    V = p["v_rest"] + 100 * rng.random(o.NH)
    Y = ob.rhs(o, V, rng.random(o.NH), np.zeros(o.NH), 5.0, p["dt"])
    g = ob.gamma_of(p, p["dt"])
    X0 = np.concatenate([np.zeros(o.N), V])
    Xo, _ = ob.solve_cg(o, g, Y, X0, tol=1e-14, max_iter=40000)
    Xo = ob.normalise(o, Xo)
    return mesh, p, S, o, Y, Xo


@pytest.mark.parametrize("eps,prec", [(0.0, "fp64"), (1e-2, "fp64"), (1e-2, "fp32"),
                                      (1e-2, "bf16"), (1e-1, "bf16")])
def test_slab65_precision_forms_match_oracle(bid, slab65, eps, prec):
    mesh, p, S, o, Y, Xo = slab65
    P = bid.Precond(S, p["dt"], eps=eps, precision=prec)
    X = torch.zeros(o.N + o.NH, dtype=torch.float64, device=DEV)
    info = P.solve(T(Y), X, tol=1e-14, max_iter=800)
    Xg = H(X)
    assert_potentials_close(Xg, Xo, o.N, 1e-9, info)
    assert info["relres_true"] <= 1e-14
    # exact factors still leave the monodomain approximation K_m != K (the slab's
    # anisotropy ratios differ), so a few iterations remain
    assert 1 <= info["iters"] <= 200
    assert P.stats["levels1"] >= 5


def test_slab65_steps_match_oracle(bid, slab65):
    # five steps with the centre-ball stimulus, BF16 factors: per step the oracle
    # (plain CG, 1e-14) is fed the GPU's state
    mesh, p, S, o, _, _ = slab65
    P = bid.Precond(S, p["dt"], eps=1e-2, precision="bf16")
    ist = ob.heart_stimulus(o, stimulus_centre_ball(mesh))
    U0, V0, h0 = ob.initial_state(o)
    U, V, h, I = T(U0), T(V0), T(h0), T(ist)
    dt = p["dt"]
    for k in range(5):
        Ug, Vg, hg = H(U), H(V), H(h)
        its = P.step(U, V, h, I, k * dt, 1, tol=1e-14, max_iter=800)
        U1, V1, h1 = ob.time_step(o, Ug, Vg, hg, ist, k * dt, dt, solver="cg", tol=1e-14)
        X1 = np.concatenate([U1, V1])
        Xg = np.concatenate([H(U), H(V)])
        assert_potentials_close(Xg, X1, o.N, 1e-9, k)
        assert np.abs(H(h) - h1).max() <= 1e-13
        assert its[0] >= 1


def test_slab161_bf16_properties(bid):
    mesh, p = slab_3d(161, 161, 49), params_3d(0.05)
    S = bid.System(mesh, p)
    assert S.N == S.NH == 1270129
    P = bid.Precond(S, p["dt"], eps=1e-2, precision="bf16")
    assert P.stats["lowrank_blocks"] > 0
    o = ob.build_system(mesh, p)
    assert (S.perm == o.order).all()
    ist = ob.heart_stimulus(o, stimulus_centre_ball(mesh))
    U0, V0, h0 = ob.initial_state(o)
    U, V, h, I = T(U0), T(V0), T(h0), T(ist)
    L = ob.system_matrix(o, ob.gamma_of(p, p["dt"]))
    for k in range(2):
        Vb, hb = H(V), H(h)
        its = P.step(U, V, h, I, k * p["dt"], 1, tol=1e-8, max_iter=200)
        Y = ob.rhs(o, Vb, hb, ist, k * p["dt"], p["dt"])
        X = np.concatenate([H(U), H(V)])
        assert np.linalg.norm(L @ X - Y) <= 1.0001e-8 * np.linalg.norm(Y), k
        assert abs(H(U) @ o.M.diagonal()) <= 1e-10 * np.abs(X).max() * o.M.sum()
        assert 1 <= its[0] <= 60
