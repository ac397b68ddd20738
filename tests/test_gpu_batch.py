"""GPU parity of the batched form: many independent torso slices advanced by
one launch per phase (combined layout, forest factors, per-slice PCG scalars
and convergence) against the FP64 oracle slice by slice, and against the same
slices run one at a time through the single-system path.

Tolerances as in test_gpu_parity: solves to relative residual 1e-14 agree with
the oracle's direct solve within 1e-9 per slice, U and V each relative to the
oracle block's largest entry; the factor
applications of a slice inside the batch equal its applications alone (same
tree and blocks, possibly another summation order) to 1e-12 relative with FP64
factors and 1e-6 with FP32 factors.
"""
import numpy as np
import pytest

from oracle import bidomain as ob
from potentials import assert_potentials_close
from workloads import batched_slices, torso_square_2d, params_2d, stimulus_seeded_disc

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


def _slices(count, seed, min_k, max_k, step, dt):
    out = []
    for d in batched_slices(count, seed, min_k, max_k, step):
        m = torso_square_2d(d["n"], semi_axes=d["semi_axes"], fibre_deg=d["fibre_deg"])
        out.append((m, params_2d(dt), d["stim_seed"]))
    return out


def _state(bid, sl, systems, B, oracle_for=None):
    """Combined initial state (U = 0, V = v_rest, h = 1) and stimulus of the
    slices in the library numbering, plus oracle systems of the slices listed
    in oracle_for (all when None)."""
    X = np.zeros(B.n)
    h = np.ones(int(B.hoff[-1]))
    ist = np.zeros_like(h)
    os_ = {}
    for k, ((m, p, seed), S) in enumerate(zip(sl, systems)):
        a = int(B.off[k])
        X[a + S.N:B.off[k + 1]] = p["v_rest"]
        ist[B.hoff[k]:B.hoff[k + 1]] = stimulus_seeded_disc(m, seed=seed)[S.perm[:S.NH]]
        if oracle_for is None or k in oracle_for:
            o = ob.build_system(m, p)
            assert (o.order == S.perm).all()
            os_[k] = o
    return X, h, ist, os_


@pytest.fixture(scope="module")
def small(bid):
    sl = _slices(6, 21, 3, 9, 8, 0.1)
    systems = [bid.System(m, p) for m, p, _ in sl]
    return sl, systems


def test_batch_factor_equals_single(bid, small):
    sl, systems = small
    leaf = [8, 16, 32, 16, 8, 64]
    for prec, eps in (("fp64", 0.0), ("fp32", 1e-3)):
        B = bid.Batch(systems, 0.1, eps=eps, precision=prec, leaf=leaf)
        b = np.random.default_rng(3).normal(size=B.n)
        for which in (1, 2):
            x = torch.zeros(B.n, dtype=torch.float64, device=DEV)
            B.apply_factor(which, T(b), x)
            xb = H(x)
            for k, S in enumerate(systems):
                P = bid.Precond(S, 0.1, eps=eps, precision=prec, leaf=leaf[k])
                a, e = int(B.off[k]), int(B.off[k + 1])
                seg = slice(a, a + S.N) if which == 1 else slice(a + S.N, e)
                xs = torch.zeros(seg.stop - seg.start, dtype=torch.float64, device=DEV)
                P.apply_factor(which, T(b[seg]), xs)
                ref = H(xs)
                # same tree and blocks; the summation order can differ (the level
                # from which clusters take the large-cluster kernels is set by
                # the whole forest; P_1 also subtracts the slice mean, summed in
                # another order): FP64 to rounding, FP32 storage to FP32 rounding
                tol = 1e-12 if prec == "fp64" else 1e-6
                assert np.abs(xb[seg] - ref).max() <= tol * np.abs(ref).max(), (prec, which, k)


@pytest.mark.parametrize("prec,eps,tol", [("fp64", 0.0, 1e-12), ("fp32", 1e-3, 1e-6)])
def test_batch_precond_equals_single(bid, small, prec, eps, tol):
    # the P_1 input shift (slice mean) is summed in another order than alone;
    # with FP32 factors that rounding difference can flip the FP32 rounding of
    # an input, hence the FP32-level bound there
    sl, systems = small
    B = bid.Batch(systems, 0.1, eps=eps, precision=prec, leaf=16)
    r = np.random.default_rng(4).normal(size=B.n)
    z = torch.zeros(B.n, dtype=torch.float64, device=DEV)
    B.apply_precond(T(r), z)
    zb = H(z)
    for k, S in enumerate(systems):
        P = bid.Precond(S, 0.1, eps=eps, precision=prec, leaf=16)
        a, e = int(B.off[k]), int(B.off[k + 1])
        zs = torch.zeros(e - a, dtype=torch.float64, device=DEV)
        P.apply(T(r[a:e]), zs)
        ref = H(zs)
        d = zb[a:e] - ref
        d[:S.N] -= d[:S.N].mean()          # the U block is defined up to a constant
        assert np.abs(d).max() <= tol * np.abs(ref).max(), k


@pytest.mark.parametrize("kw", [dict(eps=0.0), dict(eps=1e-3, precision="fp32"),
                                dict(eps=1e-2, precision="bf16")])
def test_batch_solve_matches_oracle(bid, small, kw):
    sl, systems = small
    B = bid.Batch(systems, 0.1, **kw)
    rng = np.random.default_rng(9)
    Y = np.zeros(B.n)
    ref = []
    for k, (m, p, _) in enumerate(sl):
        o = ob.build_system(m, p)
        V = p["v_rest"] + 100 * rng.random(o.NH)
        Yk = ob.rhs(o, V, rng.random(o.NH), np.zeros(o.NH), 5.0, p["dt"])
        Y[B.off[k]:B.off[k + 1]] = Yk
        ref.append(ob.solve_direct(o, ob.gamma_of(p, p["dt"]), Yk))
    X = torch.zeros(B.n, dtype=torch.float64, device=DEV)
    info, _ = B.solve(T(Y), X, tol=1e-14, max_iter=600)
    Xg = H(X)
    for k, Xo in enumerate(ref):
        Xk = Xg[B.off[k]:B.off[k + 1]]
        assert_potentials_close(Xk, Xo, systems[k].N, 1e-9, (k, info[k]))
        assert info[k]["relres_true"] <= 1e-14


def test_batch_step_matches_oracle_and_single(bid, small):
    # 4 steps of every slice (stimulus on): the batch against the oracle fed
    # the batch's state, and the iteration counts against the same slice
    # stepped alone (per-slice convergence: a converged slice is frozen)
    sl, systems = small
    dt = 0.1
    B = bid.Batch(systems, dt, eps=1e-3, precision="fp32", leaf=16)
    X0, h0, ist, os_ = _state(bid, sl, systems, B)
    X, h, I = T(X0), T(h0), T(ist)
    singles = []
    for k, S in enumerate(systems):
        P = bid.Precond(S, dt, eps=1e-3, precision="fp32", leaf=16)
        a, o = int(B.off[k]), os_[k]
        singles.append((P, T(X0[a:a + o.N]), T(X0[a + o.N:B.off[k + 1]]),
                        T(h0[B.hoff[k]:B.hoff[k + 1]]), T(ist[B.hoff[k]:B.hoff[k + 1]])))
    for step in range(4):
        Xb, hb = H(X), H(h)
        its = B.step(X, h, I, step * dt, 1, tol=1e-14, max_iter=400)
        Xa, ha = H(X), H(h)
        for k, o in os_.items():
            a, e = int(B.off[k]), int(B.off[k + 1])
            hs, he = int(B.hoff[k]), int(B.hoff[k + 1])
            U1, V1, h1 = ob.time_step(o, Xb[a:a + o.N], Xb[a + o.N:e], hb[hs:he], ist[hs:he],
                                      step * dt, dt)
            X1 = np.concatenate([U1, V1])
            assert_potentials_close(Xa[a:e], X1, o.N, 1e-9, (step, k))
            assert np.abs(ha[hs:he] - h1).max() <= 1e-13
            P, U, V, hh, Ik = singles[k]
            it1 = P.step(U, V, hh, Ik, step * dt, 1, tol=1e-14, max_iter=400)
            # same iteration up to summation order: the counts agree unless a
            # residual sits within rounding of tol
            assert abs(int(it1[0]) - int(its[0, k])) <= 1, (step, k, it1, its[0])
            if it1[0] == its[0, k]:
                Xs = np.concatenate([H(U), H(V)])
                assert_potentials_close(Xa[a:e], Xs, o.N, 1e-9, (step, k))
            else:   # continue the single run from the batch's state
                U.copy_(T(Xa[a:a + o.N]))
                V.copy_(T(Xa[a + o.N:e]))
            hh.copy_(T(ha[hs:he]))


def test_batch_is_deterministic_and_errors(bid, small):
    sl, systems = small
    B = bid.Batch(systems, 0.1, eps=1e-3, precision="fp32")
    Y = np.zeros(B.n)
    rng = np.random.default_rng(10)
    for k, (m, p, _) in enumerate(sl):
        o = ob.build_system(m, p)
        Y[B.off[k]:B.off[k + 1]] = ob.rhs(o, p["v_rest"] + 100 * rng.random(o.NH),
                                           np.ones(o.NH), np.zeros(o.NH), 5.0, 0.1)
    outs = []
    for _ in range(2):
        X = torch.zeros(B.n, dtype=torch.float64, device=DEV)
        B.solve(T(Y), X, tol=1e-10)
        outs.append(H(X))
    assert np.array_equal(outs[0], outs[1])
    # one slice with a zero right-hand side: zero solution, the others solve
    Yz = Y.copy()
    Yz[B.off[2]:B.off[3]] = 0.0
    X = torch.ones(B.n, dtype=torch.float64, device=DEV)
    info, _ = B.solve(T(Yz), X, tol=1e-10)
    assert info[2]["iters"] == 0 and not H(X)[B.off[2]:B.off[3]].any()
    assert all(i["relres_true"] < 1e-10 for k, i in enumerate(info) if k != 2)
    # max_iter reached on every slice
    X = torch.zeros(B.n, dtype=torch.float64, device=DEV)
    info, rc = B.solve(T(Y), X, tol=1e-30, max_iter=2, check=False)
    assert rc == bid.ENOCONV and all(i["iters"] == 2 for i in info)
    # a NaN in one slice: that slice stagnates
    Yn = Y.copy()
    Yn[B.off[1] + 3] = np.nan
    info, rc = B.solve(T(Yn), X, check=False)
    assert rc == bid.ESTAGNATE and info[1]["status"] == bid.ESTAGNATE
    with pytest.raises(bid.BidError) as e:
        bid.Batch(systems, 0.1, leaf=[16] * (len(systems) - 1) + [2])
    assert e.value.code == bid.EINVAL
    p2 = dict(sl[0][1])
    p2["tau_in"] = 0.5
    S2 = bid.System(sl[0][0], p2)
    with pytest.raises(bid.BidError) as e:
        bid.Batch([systems[0], S2], 0.1)
    assert e.value.code == bid.EINVAL


def test_tune_leaf_picks_a_candidate_and_caches(bid):
    S = bid.System(torso_square_2d(129), params_2d(0.1))
    best, ms = bid.tune_leaf(S, 0.1, eps=1e-3, precision="fp32", candidates=(8, 16, 32), reps=3)
    assert best in (8, 16, 32) and ms[best] == min(ms.values()) and all(v > 0 for v in ms.values())
    best2, ms2 = bid.tune_leaf(S, 0.1, eps=1e-3, precision="fp32", candidates=(8, 16, 32), reps=3)
    assert best2 == best and ms2 == ms            # cached: same answer, no new timing


def test_full_size_batch_properties(bid):
    # the 64-slice workload (sides 129..1025, seeded geometry and stimulus),
    # chosen form, two steps: every slice's true residual below tol, its U
    # normalised, and a sample of slices equal to the same slice run alone
    dt = 0.1
    sl = _slices(64, 2026, 4, 32, 32, dt)
    systems = [bid.System(m, p) for m, p, _ in sl]
    B = bid.Batch(systems, dt, eps=1e-3, precision="fp32", leaf=16)
    sample = (0, 17, 40, 63)
    X0, h0, ist, os_ = _state(bid, sl, systems, B, oracle_for=sample)
    X, h, I = T(X0), T(h0), T(ist)
    for step in range(2):
        Xb, hb = H(X), H(h)
        its = B.step(X, h, I, step * dt, 1, tol=1e-8, max_iter=100)
        assert (its[0] >= 1).all()
        Xa = H(X)
        for k in sample:
            o, (m, p, _) = os_[k], sl[k]
            a, e = int(B.off[k]), int(B.off[k + 1])
            hs, he = int(B.hoff[k]), int(B.hoff[k + 1])
            g = ob.gamma_of(p, dt)
            Y = ob.rhs(o, Xb[a + o.N:e], hb[hs:he], ist[hs:he], step * dt, dt)
            L = ob.system_matrix(o, g)
            assert np.linalg.norm(L @ Xa[a:e] - Y) <= 1.0001e-8 * np.linalg.norm(Y), (step, k)
            assert abs(Xa[a:a + o.N] @ o.M.diagonal()) <= 1e-10 * np.abs(Xa[a:e]).max() * o.M.sum()


def test_tune_batch_leaf_per_size_class(bid, small):
    sl, systems = small
    leaf = bid.tune_batch_leaf(systems, 0.1, eps=1e-3, precision="fp32", candidates=(8, 16),
                               reps=2)
    assert len(leaf) == len(systems) and set(leaf) <= {8, 16}
    import math
    cls = {}
    for S, lf in zip(systems, leaf):
        cls.setdefault(math.floor(2 * math.log2(S.N)), set()).add(lf)
    assert all(len(v) == 1 for v in cls.values())   # one answer per size class
    B = bid.Batch(systems, 0.1, eps=1e-3, precision="fp32", leaf=leaf)
    assert B.leaf == leaf
