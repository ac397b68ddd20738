"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 element-wise results (Lambda product, Step 1 + Step 3) within
1e-13 relative to the largest entry (rounding order only).  Solves are
compared potential by potential: U and V each within 1e-9 of the oracle's,
relative to the largest entry of the oracle's block (tests/potentials.py).
The solution error is at most cond * (relative residual), and a run to
relative residual 1e-13 leaves errors of up to about 1e-9 in U (the oracle's
own CG at 1e-13 against its direct solve, 97^2 and 129^2 slices), so parity
solves run to 1e-14 on both sides, which leaves about 1e-10.  Every factor
precision (FP64, FP32, BF16, eps > 0) reaches the same bound because PCG stops
on the FP64 residual.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bidomain as ob
from potentials import assert_potentials_close
from workloads import (torso_square_2d, slab_3d, params_2d, params_3d, stimulus_left_apex,
                       stimulus_seeded_disc)

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
    "2d97": lambda: (torso_square_2d(97), params_2d(0.1)),
    "3d": lambda: (slab_3d(13, 11, 7), params_3d(0.05)),
}


def _setup(bid, case, **kw):
    mesh, p = CASES[case]()
    S = bid.System(mesh, p)
    P = bid.Precond(S, p["dt"], **kw)
    o = ob.build_system(mesh, p)
    assert (S.perm == o.order).all()
    return mesh, p, S, P, o


@pytest.mark.parametrize("case", list(CASES))
def test_lambda_matches_oracle(bid, case):
    mesh, p, S, P, o = _setup(bid, case)
    g = ob.gamma_of(p, p["dt"])
    x = np.random.default_rng(0).normal(size=o.N + o.NH)
    y = torch.zeros(o.N + o.NH, dtype=torch.float64, device=DEV)
    S.apply_lambda(g, T(x), y)
    ref = ob.system_matrix(o, g) @ x
    assert np.abs(H(y) - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("stim", [0, 1])
def test_rhs_gate_matches_oracle(bid, stim):
    mesh, p, S, P, o = _setup(bid, "2d65")
    rng = np.random.default_rng(1 + stim)
    V = rng.uniform(p["v_rest"] - 5, p["v_peak"] + 5, size=o.NH)
    w = (V - p["v_rest"]) / (p["v_peak"] - p["v_rest"])
    assert np.abs(w - p["v_gate"]).min() > 1e-9          # no gate decision at a tie
    h = rng.uniform(0, 1, size=o.NH)
    ist = ob.heart_stimulus(o, stimulus_left_apex(mesh))
    Yg = torch.zeros(o.N + o.NH, dtype=torch.float64, device=DEV)
    hg = T(h)
    P.rhs_gate(T(V), hg, T(ist), stim, Yg)
    t = 0.5 if stim else 5.0
    Yo = ob.rhs(o, V, h, ist, t, p["dt"])
    ho = ob.gate_update(o, V, h, p["dt"])
    assert np.abs(H(Yg) - Yo).max() <= 1e-13 * np.abs(Yo).max()
    assert np.abs(H(hg) - ho).max() <= 1e-15


@pytest.mark.parametrize("case", list(CASES))
def test_exact_factors_match_oracle(bid, case):
    mesh, p, S, P, o = _setup(bid, case, eps=0.0)
    g = ob.gamma_of(p, p["dt"])
    rng = np.random.default_rng(2)
    b = rng.normal(size=o.N)
    x = torch.zeros(o.N, dtype=torch.float64, device=DEV)
    P.apply_factor(1, T(b), x)
    xg = H(x)
    xg -= xg.mean()
    xo = ob.s1_pseudo_inverse_apply(o, b)
    assert np.abs(xg - xo).max() <= 1e-10 * np.abs(xo).max()
    b2 = rng.normal(size=o.NH)
    x2 = torch.zeros(o.NH, dtype=torch.float64, device=DEV)
    P.apply_factor(2, T(b2), x2)
    xo2 = spla.spsolve(ob.monodomain_matrix(o, g).tocsc(), b2)
    assert np.abs(H(x2) - xo2).max() <= 1e-12 * np.abs(xo2).max()


@pytest.mark.parametrize("case", ["2d65", "3d"])
def test_exact_preconditioner_matches_oracle(bid, case):
    mesh, p, S, P, o = _setup(bid, case, eps=0.0)
    g = ob.gamma_of(p, p["dt"])
    r = np.random.default_rng(3).normal(size=o.N + o.NH)
    r[:o.N] -= r[:o.N].mean()
    z = torch.zeros_like(T(r))
    P.apply(T(r), z)
    zg = H(z)
    zo = ob.precond_apply_exact(o, g, r)
    zg[:o.N] -= zg[:o.N].mean()
    zo[:o.N] -= zo[:o.N].mean()
    assert np.abs(zg - zo).max() <= 1e-10 * np.abs(zo).max()


def test_equal_anisotropy_converges_in_one_iteration(bid):
    # isolated heart, sigma_e = lam sigma_i: K_m = K, so exact P_1 and P_K make
    # P_Lambda = Lambda on its range (Sec. 5.2, P_Lambda exact as eps -> 0)
    mesh = slab_3d(13, 12, 7)
    p = params_3d(0.05)
    p["sigma_e"] = tuple(0.7 * np.array(p["sigma_i"]))
    S = bid.System(mesh, p)
    P = bid.Precond(S, p["dt"], eps=0.0)
    o = ob.build_system(mesh, p)
    V = p["v_rest"] + 100 * np.random.default_rng(4).random(o.NH)
    Y = np.concatenate([np.zeros(o.N), o.MH @ V])
    X = torch.zeros(o.N + o.NH, dtype=torch.float64, device=DEV)
    info = P.solve(T(Y), X, tol=1e-10, max_iter=20)
    assert info["iters"] == 1, info


SOLVE_FORMS = [("2d65", dict(eps=0.0)), ("2d97", dict(eps=0.0)), ("3d", dict(eps=0.0)),
               ("2d97", dict(eps=1e-3)), ("2d97", dict(eps=1e-2, precision="fp32")),
               ("2d97", dict(eps=1e-3, precision="bf16")), ("3d", dict(eps=1e-2, precision="bf16")),
               ("2d97", dict(eps=0.0, leaf=16, block=16))]


@pytest.mark.parametrize("case,kw", SOLVE_FORMS)
def test_solve_matches_oracle(bid, case, kw):
    mesh, p, S, P, o = _setup(bid, case, **kw)
    g = ob.gamma_of(p, p["dt"])
    rng = np.random.default_rng(5)
    V = p["v_rest"] + 100 * rng.random(o.NH)
    h = rng.random(o.NH)
    Y = ob.rhs(o, V, h, np.zeros(o.NH), 5.0, p["dt"])
    X = T(np.concatenate([np.zeros(o.N), V]))
    info = P.solve(T(Y), X, tol=1e-14, max_iter=600)
    Xo = ob.solve_direct(o, g, Y)
    Xg = H(X)
    assert_potentials_close(Xg, Xo, o.N, 1e-9, info)
    assert info["relres_true"] <= 1e-14
    assert abs(Xg[:o.N] @ o.M.diagonal()) <= 1e-12 * np.abs(Xg).max() * o.M.sum()


def test_step_trajectory_matches_oracle(bid):
    # 65^2 torso, 20 steps of 0.25 ms with the corner stimulus: per step, the
    # oracle is fed the GPU's state; at the end the two trajectories agree too
    mesh, p, S, P, o = _setup(bid, "2d65", eps=1e-3)
    ist = ob.heart_stimulus(o, stimulus_left_apex(mesh))
    U0, V0, h0 = ob.initial_state(o)
    U, V, h, I = T(U0), T(V0), T(h0), T(ist)
    Uo, Vo, ho = U0.copy(), V0.copy(), h0.copy()
    dt = p["dt"]
    for k in range(20):
        Ug, Vg, hg = H(U), H(V), H(h)
        its = P.step(U, V, h, I, k * dt, 1, tol=1e-14, max_iter=600)
        U1, V1, h1 = ob.time_step(o, Ug, Vg, hg, ist, k * dt, dt)
        Xg = np.concatenate([H(U), H(V)])
        X1 = np.concatenate([U1, V1])
        assert_potentials_close(Xg, X1, o.N, 1e-9, k)
        assert np.abs(H(h) - h1).max() <= 1e-13
        Uo, Vo, ho = ob.time_step(o, Uo, Vo, ho, ist, k * dt, dt)
        assert its[0] >= 1
    # the two trajectories, each run on its own, agree at the end as well (the
    # per-step errors do not grow: the oracle's CG trajectory at 1e-14 stays
    # within 1e-10 of its direct one over these 20 steps)
    Xo = np.concatenate([Uo, Vo])
    Xg = np.concatenate([H(U), H(V)])
    assert_potentials_close(Xg, Xo, o.N, 1e-9, "end")
    assert np.abs(H(h) - ho).max() <= 1e-12
    assert H(V).max() > -60.0                # the stimulus depolarised the site


def test_solve_is_deterministic(bid):
    mesh, p, S, P, o = _setup(bid, "2d97", eps=1e-3)
    Y = ob.rhs(o, p["v_rest"] + 100 * np.random.default_rng(6).random(o.NH), np.ones(o.NH),
               np.zeros(o.NH), 5.0, p["dt"])
    outs = []
    for _ in range(2):
        X = torch.zeros(o.N + o.NH, dtype=torch.float64, device=DEV)
        P.solve(T(Y), X, tol=1e-10)
        outs.append(H(X))
    assert np.array_equal(outs[0], outs[1])


def test_edge_cases(bid):
    mesh, p, S, P, o = _setup(bid, "2d65")
    n = o.N + o.NH
    X = torch.ones(n, dtype=torch.float64, device=DEV)
    info = P.solve(torch.zeros(n, dtype=torch.float64, device=DEV), X)
    assert info["iters"] == 0 and not H(X).any()
    Y = ob.rhs(o, p["v_rest"] + 50 * np.random.default_rng(7).random(o.NH), np.ones(o.NH),
               np.zeros(o.NH), 5.0, p["dt"])
    X = torch.zeros(n, dtype=torch.float64, device=DEV)
    info = P.solve(T(Y), X, tol=1e-30, max_iter=2, check=False)
    assert info["rc"] == bid.ENOCONV and info["iters"] == 2
    Yn = Y.copy()
    Yn[3] = np.nan
    info = P.solve(T(Yn), X, check=False)
    assert info["rc"] == bid.ESTAGNATE
    Yt = T(Y)
    with pytest.raises(bid.BidError) as e:
        P.solve(Yt, Yt)
    assert e.value.code == bid.EINVAL
    with pytest.raises(bid.BidError):
        bid.Precond(S, -1.0)


def _full_size_properties(bid, n, steps, eps, precision):
    mesh = torso_square_2d(n)
    p = params_2d(0.1)
    S = bid.System(mesh, p)
    P = bid.Precond(S, p["dt"], eps=eps, precision=precision)
    o = ob.build_system(mesh, p)
    assert (S.perm == o.order).all()
    ist = ob.heart_stimulus(o, stimulus_seeded_disc(mesh, seed=0))
    U0, V0, h0 = ob.initial_state(o)
    U, V, h, I = T(U0), T(V0), T(h0), T(ist)
    g = ob.gamma_of(p, p["dt"])
    L = ob.system_matrix(o, g)
    rng = np.random.default_rng(8)
    for k in range(steps):
        Vb, hb = H(V), H(h)
        P.step(U, V, h, I, k * p["dt"], 1, tol=1e-8, max_iter=100)
        Y = ob.rhs(o, Vb, hb, ist, k * p["dt"], p["dt"])
        X = np.concatenate([H(U), H(V)])
        assert np.linalg.norm(L @ X - Y) <= 1e-8 * np.linalg.norm(Y) * 1.0001
        assert abs(H(U) @ o.M.diagonal()) <= 1e-10 * np.abs(X).max() * o.M.sum()
        idx = rng.choice(o.NH, 2000, replace=False)
        _, gg = ob.ms_reaction(Vb[idx], hb[idx], p)
        np.testing.assert_allclose(H(h)[idx], hb[idx] + p["dt"] * gg, rtol=0, atol=1e-15)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_513_step_matches_oracle(bid, precision):
    # the 513^2 slice (N = 263 169, N_H = 49 925) in the bench's form (eps 1e-3,
    # leaf 32): low-rank groups accepted, several levels of large clusters and
    # the masked second P_1 solve all take part.  Five steps at rel-res 1e-8
    # bring the stimulated state away from rest; then one step at 1e-14 from
    # that state is compared with the oracle's step (sparse direct solve) from
    # the same state, U and V each to 1e-9, h exactly up to rounding
    mesh = torso_square_2d(513)
    p = params_2d(0.1)
    S = bid.System(mesh, p)
    assert (S.N, S.NH) == (263169, 49925)
    P = bid.Precond(S, p["dt"], eps=1e-3, precision=precision, leaf=32)
    st = P.stats
    assert st["lowrank_blocks"] > 0 and st["lowrank_entries"] > 0
    assert st["large_levels1"] >= 3 and st["large_levelsk"] >= 2, st
    assert 0 < st["masked_dead1"] < st["masked_clusters1"], st
    assert st["alg_bytes_p1_masked"] < st["alg_bytes_p1"]
    assert st["mid_clusters1"] > 0 and st["mid_clustersk"] > 0, st
    o = ob.build_system(mesh, p)
    assert (S.perm == o.order).all()
    ist = ob.heart_stimulus(o, stimulus_seeded_disc(mesh, seed=0))
    U0, V0, h0 = ob.initial_state(o)
    U, V, h, I = T(U0), T(V0), T(h0), T(ist)
    dt = p["dt"]
    P.step(U, V, h, I, 0.0, 5, tol=1e-8, max_iter=200)
    Ug, Vg, hg = H(U), H(V), H(h)
    assert Vg.max() > p["v_rest"] + 1.0       # the stimulus has moved the state
    its = P.step(U, V, h, I, 5 * dt, 1, tol=1e-14, max_iter=800)
    U1, V1, h1 = ob.time_step(o, Ug, Vg, hg, ist, 5 * dt, dt)
    assert_potentials_close(np.concatenate([H(U), H(V)]), np.concatenate([U1, V1]), o.N, 1e-9,
                            (precision, int(its[0])))
    assert np.abs(H(h) - h1).max() <= 1e-13
    assert abs(H(U) @ o.M.diagonal()) <= 1e-12 * np.abs(H(U)).max() * o.M.sum()


@pytest.mark.parametrize("precision,leaf", [("fp32", 32), ("bf16", 32), ("fp64", 16)])
def test_mid_clusters_equal_chunked_kernels(bid, monkeypatch, precision, leaf):
    # the large clusters whose block fits one CTA's shared memory (one CTA per
    # cluster, the default) against the chunked task kernels (BID_MID_BYTES=0)
    # on the 513^2 slice with eps 1e-3: the same P_1, P_K and P_Lambda^-1
    # applications up to the accumulation precision's rounding (FP32: 1e-5,
    # FP64: 1e-12 of the largest entry), and PCG solves to rel-res 1e-13 that
    # agree potential by potential to 1e-8 within one iteration of each other
    mesh, p = torso_square_2d(513), params_2d(0.1)
    S = bid.System(mesh, p)
    o = ob.build_system(mesh, p)
    rng = np.random.default_rng(513)
    b1, bk, r = T(rng.normal(size=S.N)), T(rng.normal(size=S.NH)), T(rng.normal(size=S.N + S.NH))
    Y = T(ob.rhs(o, p["v_rest"] + 100 * rng.random(o.NH), np.ones(o.NH), np.zeros(o.NH), 5.0, p["dt"]))
    monkeypatch.setenv("BID_ROOT_GRAM", "0")   # the same top levels in both runs
    out = {}
    for mb in ("0", None):
        if mb is None:
            monkeypatch.delenv("BID_MID_BYTES", raising=False)
        else:
            monkeypatch.setenv("BID_MID_BYTES", mb)
        P = bid.Precond(S, p["dt"], eps=1e-3, precision=precision, leaf=leaf)
        x1, xk, z = torch.zeros_like(b1), torch.zeros_like(bk), torch.zeros_like(r)
        P.apply_factor(1, b1, x1)
        P.apply_factor(2, bk, xk)
        P.apply(r, z)
        X = torch.zeros_like(r)
        info = P.solve(Y, X, tol=1e-13, max_iter=800)
        out[mb] = (H(x1), H(xk), H(z), H(X), info["iters"], P.stats["mid_clusters1"],
                   P.stats["mid_clustersk"])
        del P
    assert out["0"][5] == 0 and out[None][5] > 0 and out[None][6] > 0
    tol = 1e-12 if precision == "fp64" else 1e-5
    for a, c in zip(out["0"][:3], out[None][:3]):
        assert np.isfinite(c).all()
        assert np.abs(a - c).max() <= tol * np.abs(a).max()
    assert abs(out["0"][4] - out[None][4]) <= 1, (out["0"][4], out[None][4])
    assert_potentials_close(out[None][3], out["0"][3], o.N, 1e-8, precision)


@pytest.mark.parametrize("precision,leaf", [("fp32", 32), ("bf16", 32), ("fp64", 16)])
def test_wide_clusters_equal_chunked_kernels(bid, monkeypatch, precision, leaf):
    # the large clusters split in column slices over a thread-block cluster
    # (partial sums combined through distributed shared memory; the default)
    # against the chunked task kernels (BID_WIDE_BYTES=0) on the 513^2 slice
    # with eps 1e-3: the same P_1, P_K and P_Lambda^-1 applications up to the
    # accumulation precision's rounding, the same masked solve, and PCG solves
    # that agree potential by potential to 1e-8 within one iteration
    mesh, p = torso_square_2d(513), params_2d(0.1)
    S = bid.System(mesh, p)
    o = ob.build_system(mesh, p)
    rng = np.random.default_rng(514)
    b1, bk, r = T(rng.normal(size=S.N)), T(rng.normal(size=S.NH)), T(rng.normal(size=S.N + S.NH))
    Y = T(ob.rhs(o, p["v_rest"] + 100 * rng.random(o.NH), np.ones(o.NH), np.zeros(o.NH), 5.0, p["dt"]))
    monkeypatch.setenv("BID_ROOT_GRAM", "0")   # the root stays a wide cluster here
    out = {}
    for wb in ("0", None):
        if wb is None:
            monkeypatch.delenv("BID_WIDE_BYTES", raising=False)
        else:
            monkeypatch.setenv("BID_WIDE_BYTES", wb)
        P = bid.Precond(S, p["dt"], eps=1e-3, precision=precision, leaf=leaf)
        x1, xk, z = torch.zeros_like(b1), torch.zeros_like(bk), torch.zeros_like(r)
        P.apply_factor(1, b1, x1)
        P.apply_factor(2, bk, xk)
        P.apply(r, z)
        X = torch.zeros_like(r)
        info = P.solve(Y, X, tol=1e-13, max_iter=800)
        out[wb] = (H(x1), H(xk), H(z), H(X), info["iters"], P.stats["wide_clusters1"])
        del P
    assert out["0"][5] == 0 and out[None][5] > 0, (out["0"][5], out[None][5])
    tol = 1e-12 if precision == "fp64" else 1e-5
    for a, c in zip(out["0"][:3], out[None][:3]):
        assert np.isfinite(c).all()
        assert np.abs(a - c).max() <= tol * np.abs(a).max()
    assert abs(out["0"][4] - out[None][4]) <= 1, (out["0"][4], out[None][4])
    assert_potentials_close(out[None][3], out["0"][3], o.N, 1e-8, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_root_gram_equals_root_passes(bid, monkeypatch, precision):
    # the top block's passes (the root and its two children) replaced by one
    # product with G = M^T M (the default where the root has no boundary or
    # low-rank groups) against the passes themselves (BID_ROOT_GRAM=0), 1025^2
    # slice: the same P_1 and P_Lambda^-1 applications up to the storage
    # precision's rounding, and PCG solves within one iteration that agree
    # potential by potential to 1e-8
    mesh, p = torso_square_2d(1025), params_2d(0.1)
    S = bid.System(mesh, p)
    o = ob.build_system(mesh, p)
    rng = np.random.default_rng(1026)
    b1, r = T(rng.normal(size=S.N)), T(rng.normal(size=S.N + S.NH))
    Y = T(ob.rhs(o, p["v_rest"] + 100 * rng.random(o.NH), np.ones(o.NH), np.zeros(o.NH), 5.0, p["dt"]))
    out = {}
    for rg in ("0", None):
        if rg is None:
            monkeypatch.delenv("BID_ROOT_GRAM", raising=False)
        else:
            monkeypatch.setenv("BID_ROOT_GRAM", rg)
        P = bid.Precond(S, p["dt"], eps=1e-3 if precision == "fp32" else 0.0, precision=precision, leaf=32)
        x1, z = torch.zeros_like(b1), torch.zeros_like(r)
        P.apply_factor(1, b1, x1)
        P.apply(r, z)
        X = torch.zeros_like(r)
        info = P.solve(Y, X, tol=1e-13, max_iter=800)
        out[rg] = (H(x1), H(z), H(X), info["iters"], P.stats["gram_pivots1"])
        del P
    assert out["0"][4] == 0 and out[None][4] == 1025 + 2 * 512, (out["0"][4], out[None][4])
    tol = 1e-11 if precision == "fp64" else 1e-5
    for a, c in zip(out["0"][:2], out[None][:2]):
        assert np.isfinite(c).all()
        assert np.abs(a - c).max() <= tol * np.abs(a).max()
    assert abs(out["0"][3] - out[None][3]) <= 1, (out["0"][3], out[None][3])
    assert_potentials_close(out[None][2], out["0"][2], o.N, 1e-8, precision)


def test_full_size_513_properties(bid):
    _full_size_properties(bid, 513, 3, 1e-3, "fp64")


def test_full_size_2049_properties(bid):
    _full_size_properties(bid, 2049, 2, 1e-3, "fp32")


_HOST_LOOP_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1711_08708_gb300 import bid
from workloads import torso_square_2d, params_2d
from oracle import bidomain as ob
mesh, p = torso_square_2d(65), params_2d(0.25)
S = bid.System(mesh, p)
P = bid.Precond(S, p["dt"], eps=1e-3, precision="fp32")
o = ob.build_system(mesh, p)
Y = ob.rhs(o, p["v_rest"] + 100 * np.random.default_rng(5).random(o.NH), np.ones(o.NH),
           np.zeros(o.NH), 5.0, p["dt"])
X = torch.zeros(o.N + o.NH, dtype=torch.float64, device="cuda")
info = P.solve(torch.tensor(Y, device="cuda"), X, tol=1e-10)
S2 = bid.System(torso_square_2d(49, semi_axes=(2.0, 3.0)), p)
B = bid.Batch([S, S2], p["dt"], eps=1e-3, precision="fp32")
Yb = np.zeros(B.n)
Yb[:o.N + o.NH] = Y
Yb[o.N + o.NH + S2.N:] = 10.0 * S2.mH
Xb = torch.zeros(B.n, dtype=torch.float64, device="cuda")
binfo, _ = B.solve(torch.tensor(Yb, device="cuda"), Xb, tol=1e-10)
np.save(sys.argv[2], np.concatenate([X.cpu().numpy(), [info["iters"]], Xb.cpu().numpy(),
                                     [i["iters"] for i in binfo]]))
"""


@pytest.mark.parametrize("graph", ["1", "0"])
def test_host_driven_loop_equals_graph_loop(bid, tmp_path, graph):
    # BID_PCG_GRAPH=0 launches the graph's kernels from the host: the same
    # iterates, bit for bit
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "s.py"
    script.write_text(_HOST_LOOP_SCRIPT)
    out = {}
    for g in ("1", graph):
        f = tmp_path / f"x{g}.npy"
        env = dict(os.environ, BID_PCG_GRAPH=g)
        subprocess.run([sys.executable, str(script), root, str(f)], check=True, env=env,
                       timeout=600)
        out[g] = np.load(f)
    assert out["1"][-1] >= 1
    assert np.array_equal(out["1"], out[graph])


_DATAFLOW_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1711_08708_gb300 import bid
from workloads import torso_square_2d, params_2d
from oracle import bidomain as ob
p = params_2d(0.1)
out, levels = [], []
for prec, leaf in (("fp32", 32), ("fp64", 16), ("bf16", 32)):
    mesh = torso_square_2d(257)
    S = bid.System(mesh, p)
    P = bid.Precond(S, p["dt"], eps=1e-3, precision=prec, leaf=leaf)
    st = P.stats
    levels += [st["dataflow_levels1"], st["dataflow_levelsk"]]
    rng = np.random.default_rng(7)
    for which, n in ((1, S.N), (2, S.NH)):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        P.apply_factor(which, torch.tensor(rng.normal(size=n), device="cuda"), x)
        out.append(x.cpu().numpy())
o = ob.build_system(mesh, p)
Y = ob.rhs(o, p["v_rest"] + 100 * rng.random(o.NH), np.ones(o.NH), np.zeros(o.NH), 5.0, p["dt"])
X = torch.zeros(o.N + o.NH, dtype=torch.float64, device="cuda")
info = P.solve(torch.tensor(Y, device="cuda"), X, tol=1e-10)
out += [X.cpu().numpy(), [info["iters"]]]
S2 = bid.System(torso_square_2d(193, semi_axes=(2.0, 3.0)), p)
B = bid.Batch([S, S2], p["dt"], eps=1e-3, precision="fp32", leaf=32)
levels += [B.stats["dataflow_levels1"]]
Yb = np.zeros(B.n)
Yb[:o.N + o.NH] = Y
Yb[o.N + o.NH + S2.N:] = 10.0 * S2.mH
Xb = torch.zeros(B.n, dtype=torch.float64, device="cuda")
binfo, _ = B.solve(torch.tensor(Yb, device="cuda"), Xb, tol=1e-10)
out += [Xb.cpu().numpy(), [i["iters"] for i in binfo]]
np.save(sys.argv[2], np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in out]))
np.save(sys.argv[3], np.array(levels))
"""


@pytest.mark.parametrize("variant", ["on", "wide", "leaf"])
def test_dataflow_levels_equal_level_launches(bid, tmp_path, variant):
    # a range of flat levels in two dataflow launches per pass (BID_TREE=1),
    # over more levels (BID_TREE_SMEM=65536) or taking in the leaf level
    # (BID_TREE_FROM=0), gives the same factor solves, PCG iterates and
    # batched iterates, bit for bit, as one launch per level (the default)
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "s.py"
    script.write_text(_DATAFLOW_SCRIPT)
    envs = {"default": {}, "on": {"BID_TREE": "1"}, "wide": {"BID_TREE": "1", "BID_TREE_SMEM": "65536"},
            "leaf": {"BID_TREE": "1", "BID_TREE_FROM": "0"}}
    res = {}
    for name in ("default", variant):
        f, lv = tmp_path / f"x_{name}.npy", tmp_path / f"l_{name}.npy"
        env = {k: v for k, v in os.environ.items() if not k.startswith("BID_TREE")}
        env.update(envs[name])
        subprocess.run([sys.executable, str(script), root, str(f), str(lv)], check=True, env=env,
                       timeout=900)
        res[name] = (np.load(f), np.load(lv))
    x0, l0 = res["default"]
    x1, l1 = res[variant]
    assert (l0 == 0).all()
    assert (l1[[0, 2, 4, 6]] >= 2).all()            # P_1 of every precision and the batch forest
    assert np.array_equal(x0, x1)


_MASK_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1711_08708_gb300 import bid
from workloads import torso_square_2d, params_2d
from oracle import bidomain as ob
p = params_2d(0.1)
mesh = torso_square_2d(257)
S = bid.System(mesh, p)
o = ob.build_system(mesh, p)
out = {}
for prec in ("fp64", "fp32", "bf16"):
    P = bid.Precond(S, p["dt"], eps=1e-3, precision=prec, leaf=32)
    rng = np.random.default_rng(3)
    r = torch.tensor(rng.normal(size=S.N + S.NH), device="cuda")
    z = torch.zeros_like(r)
    P.apply(r, z)
    Y = ob.rhs(o, p["v_rest"] + 100 * rng.random(o.NH), np.ones(o.NH), np.zeros(o.NH), 5.0, p["dt"])
    X = torch.zeros(o.N + o.NH, dtype=torch.float64, device="cuda")
    info = P.solve(torch.tensor(Y, device="cuda"), X, tol=1e-10)
    out[prec + "_z"], out[prec + "_x"], out[prec + "_it"] = z.cpu().numpy(), X.cpu().numpy(), info["iters"]
S2 = bid.System(torso_square_2d(193, semi_axes=(2.0, 3.0)), p)
B = bid.Batch([S, S2], p["dt"], eps=1e-3, precision="fp32", leaf=32)
rng = np.random.default_rng(4)
rb = torch.tensor(rng.normal(size=B.n), device="cuda")
zb = torch.zeros_like(rb)
B.apply_precond(rb, zb)
Yb = np.zeros(B.n)
Yb[:o.N + o.NH] = ob.rhs(o, p["v_rest"] + 100 * rng.random(o.NH), np.ones(o.NH), np.zeros(o.NH), 5.0, p["dt"])
Yb[o.N + o.NH + S2.N:] = 10.0 * S2.mH
Xb = torch.zeros(B.n, dtype=torch.float64, device="cuda")
binfo, _ = B.solve(torch.tensor(Yb, device="cuda"), Xb, tol=1e-10)
out["batch_z"], out["batch_x"] = zb.cpu().numpy(), Xb.cpu().numpy()
out["batch_it"] = np.array([i["iters"] for i in binfo])
np.savez(sys.argv[2], **out)
"""


def test_masked_second_solve_matches_full_solve(bid, tmp_path):
    # the preconditioner's second P_1 solve takes the clusters without heart
    # nodes as scaled all-ones results (default) or computes them (BID_MASK=0):
    # the same P_Lambda^-1 r up to the factor's rounding, the same PCG
    # iteration counts and solutions within the solve tolerance, for one slice
    # (each factor precision) and for a two-slice batch (each tree its own shift)
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "s.py"
    script.write_text(_MASK_SCRIPT)
    res = {}
    for name, extra in (("masked", {}), ("full", {"BID_MASK": "0"})):
        f = tmp_path / f"x_{name}.npz"
        env = {k: v for k, v in os.environ.items() if k != "BID_MASK"}
        env.update(extra)
        subprocess.run([sys.executable, str(script), root, str(f)], check=True, env=env, timeout=900)
        res[name] = dict(np.load(f))
    a, b = res["masked"], res["full"]
    for key, tol in (("fp64", 1e-12), ("fp32", 1e-5), ("bf16", 1e-2), ("batch", 1e-5)):
        za, zb = a[key + "_z"], b[key + "_z"]
        assert np.abs(za - zb).max() <= tol * np.abs(zb).max(), key
        assert np.linalg.norm(a[key + "_x"] - b[key + "_x"]) <= 1e-7 * np.linalg.norm(b[key + "_x"]), key
        assert np.abs(np.asarray(a[key + "_it"]) - np.asarray(b[key + "_it"])).max() <= 1, key


_FLATP_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1711_08708_gb300 import bid
from workloads import torso_square_2d, params_2d
from oracle import bidomain as ob
p = params_2d(0.1)
mesh = torso_square_2d(1025)
S = bid.System(mesh, p)
o = ob.build_system(mesh, p)
out, levels = {}, []
for prec in ("fp64", "fp32", "bf16"):
    P = bid.Precond(S, p["dt"], eps=1e-3, precision=prec, leaf=32)
    levels += [P.stats["flatp_levels1"], P.stats["flatp_levelsk"]]
    rng = np.random.default_rng(9)
    for which, n in ((1, S.N), (2, S.NH)):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        P.apply_factor(which, torch.tensor(rng.normal(size=n), device="cuda"), x)
        out[f"{prec}_f{which}"] = x.cpu().numpy()
    r = torch.tensor(rng.normal(size=S.N + S.NH), device="cuda")
    z = torch.zeros_like(r)
    P.apply(r, z)
    out[prec + "_z"] = z.cpu().numpy()
    Y = ob.rhs(o, p["v_rest"] + 100 * rng.random(o.NH), np.ones(o.NH), np.zeros(o.NH), 5.0, p["dt"])
    X = torch.zeros(o.N + o.NH, dtype=torch.float64, device="cuda")
    info = P.solve(torch.tensor(Y, device="cuda"), X, tol=1e-10)
    out[prec + "_x"], out[prec + "_it"] = X.cpu().numpy(), np.array([info["iters"]])
    del P
np.savez(sys.argv[2], levels=np.array(levels), **out)
"""


def test_persistent_flat_levels_equal_one_cta_per_group(bid, tmp_path):
    # the persistent double-buffered flat launches (BID_FLATP=1, on the levels
    # with more groups than resident CTAs) and one CTA per group (the default)
    # give the same factor solves, masked preconditioner and PCG iterates, bit
    # for bit, in every storage precision
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "s.py"
    script.write_text(_FLATP_SCRIPT)
    res = {}
    for name, extra in (("pb", {"BID_FLATP": "1"}), ("plain", {})):
        f = tmp_path / f"x_{name}.npz"
        env = {k: v for k, v in os.environ.items() if k != "BID_FLATP"}
        env.update(extra)
        subprocess.run([sys.executable, str(script), root, str(f)], check=True, env=env, timeout=900)
        res[name] = dict(np.load(f))
    assert (res["pb"]["levels"][0::2] >= 1).all(), res["pb"]["levels"]    # P_1 of every precision
    assert (res["plain"]["levels"] == 0).all()
    for k in res["pb"]:
        if k != "levels":
            assert np.array_equal(res["pb"][k], res["plain"][k]), k
