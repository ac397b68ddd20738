"""GPU parity of the multigrid alternative for P_1 and P_K (BID_ELLIPTIC_MG):
the V-cycle kernels against the host replay of the same cycle, and PCG with
the multigrid block-LU preconditioner against the oracle's solve.

The preconditioner changes only the iteration count, never the solution
(Prop. 1 fixes the normalised X): the solves are compared with the oracle's
sparse direct solve potential by potential within 1e-9 (solve tolerance
1e-14, as in test_gpu_parity).  The V-cycle itself is a fixed sequence of
FP64 sparse products; the GPU and host replays differ only in summation
rounding (fused multiply-adds), within 1e-12 of the result's largest entry.
"""
import numpy as np
import pytest

from oracle import bidomain as ob
from potentials import assert_potentials_close
from workloads import torso_square_2d, slab_3d, params_2d, params_3d, stimulus_left_apex

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


CASES = {
    "2d65": lambda: (torso_square_2d(65), params_2d(0.25)),
    "2d129": lambda: (torso_square_2d(129), params_2d(0.1)),
    "3d": lambda: (slab_3d(17, 15, 9), params_3d(0.05)),
}


@pytest.mark.parametrize("case,precision", [(c, "fp64") for c in CASES] + [("2d129", "fp32")])
def test_vcycle_matches_host_replay(bid, case, precision):
    # FP32 storage (matrices and work vectors, FP32 accumulation) against the
    # FP64 replay: within FP32 rounding of the cycle's few dozen passes
    tol = 1e-12 if precision == "fp64" else 2e-5
    mesh, p = CASES[case]()
    S = bid.System(mesh, p)
    P = bid.Precond(S, p["dt"], elliptic="mg", precision=precision)
    Hs = bid.HostSystem(mesh, p)
    g = ob.gamma_of(p, p["dt"])
    rng = np.random.default_rng(12)
    for which, n in ((1, S.N), (2, S.NH)):
        b = rng.normal(size=n)
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        P.apply_factor(which, T(b), x)
        xg = H(x)
        xh, levels = Hs.mg_solve(which, b, gamma=g)
        assert levels == (P.stats["levels1"] if which == 1 else P.stats["levelsk"])
        if which == 1:                       # defined up to a constant
            xg, xh = xg - xg.mean(), xh - xh.mean()
        assert np.abs(xg - xh).max() <= tol * np.abs(xh).max(), (case, which)


@pytest.mark.parametrize("case,precision", [(c, "fp64") for c in CASES] + [("2d129", "fp32"), ("3d", "fp32")])
def test_solve_with_multigrid_matches_oracle(bid, case, precision):
    mesh, p = CASES[case]()
    S = bid.System(mesh, p)
    P = bid.Precond(S, p["dt"], elliptic="mg", precision=precision)
    o = ob.build_system(mesh, p)
    assert (S.perm == o.order).all()
    rng = np.random.default_rng(5)
    V = p["v_rest"] + 100 * rng.random(o.NH)
    Y = ob.rhs(o, V, rng.random(o.NH), np.zeros(o.NH), 5.0, p["dt"])
    X = T(np.concatenate([np.zeros(o.N), V]))
    info = P.solve(T(Y), X, tol=1e-14, max_iter=800)
    Xo = ob.solve_direct(o, ob.gamma_of(p, p["dt"]), Y)
    assert_potentials_close(H(X), Xo, o.N, 1e-9, info)
    assert info["relres_true"] <= 1e-14


def test_steps_with_multigrid_match_oracle(bid):
    mesh, p = torso_square_2d(65), params_2d(0.25)
    S = bid.System(mesh, p)
    P = bid.Precond(S, p["dt"], elliptic="mg")
    o = ob.build_system(mesh, p)
    ist = ob.heart_stimulus(o, stimulus_left_apex(mesh))
    U0, V0, h0 = ob.initial_state(o)
    U, V, h, I = T(U0), T(V0), T(h0), T(ist)
    for k in range(6):
        Ug, Vg, hg = H(U), H(V), H(h)
        P.step(U, V, h, I, k * p["dt"], 1, tol=1e-14, max_iter=800)
        U1, V1, h1 = ob.time_step(o, Ug, Vg, hg, ist, k * p["dt"], p["dt"])
        assert_potentials_close(np.concatenate([H(U), H(V)]), np.concatenate([U1, V1]), o.N, 1e-9, k)
        assert np.abs(H(h) - h1).max() <= 1e-13


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_multigrid_iterations_stay_bounded(bid, precision):
    # the V-cycle's contraction does not depend on the mesh, so the PCG
    # iteration count at rel-res 1e-8 grows only slowly from 129^2 to 513^2
    its = []
    for n in (129, 257, 513):
        mesh, p = torso_square_2d(n), params_2d(0.1)
        S = bid.System(mesh, p)
        P = bid.Precond(S, p["dt"], elliptic="mg", precision=precision)
        o = ob.build_system(mesh, p)
        rng = np.random.default_rng(n)
        Y = ob.rhs(o, p["v_rest"] + 100 * rng.random(o.NH), rng.random(o.NH), np.zeros(o.NH), 5.0, p["dt"])
        X = torch.zeros(o.N + o.NH, dtype=torch.float64, device=DEV)
        info = P.solve(T(Y), X, tol=1e-8, max_iter=200)
        L = ob.system_matrix(o, ob.gamma_of(p, p["dt"]))
        assert np.linalg.norm(L @ H(X) - Y) <= 1.0001e-8 * np.linalg.norm(Y)
        its.append(info["iters"])
    assert its[-1] <= 20 and its[-1] <= its[0] + 8, its


def test_multigrid_rejections(bid):
    mesh, p = torso_square_2d(33), params_2d(0.1)
    S = bid.System(mesh, p)
    with pytest.raises(bid.BidError) as e:
        bid.Precond(S, 0.1, precision="bf16", elliptic="mg")
    assert e.value.code == bid.EINVAL
    P = bid.Precond(S, 0.1, elliptic="mg")
    b = torch.ones(S.N, dtype=torch.float64, device=DEV)
    x = torch.zeros_like(b)
    assert P.apply_factor_noalloc(1, b, x, check=False) == bid.EINVAL
    with pytest.raises(bid.BidError) as e:
        bid.Batch([S], 0.1, elliptic="mg")
    assert e.value.code == bid.EINVAL
