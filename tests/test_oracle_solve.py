"""Pins of the oracle's Step-2 solvers and of the scheme (Sec. 3.2, Prop. 1)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bidomain as ob
from workloads import (torso_square_2d, slab_3d, params_2d, params_3d,
                       stimulus_left_apex)


def _random_rhs(s, seed):
    rng = np.random.default_rng(seed)
    Y = np.concatenate([np.zeros(s.N), rng.normal(size=s.NH)])
    return Y


def test_three_solvers_agree_and_normalise():
    m = torso_square_2d(13)
    s = ob.build_system(m, params_2d(0.25))
    g = ob.gamma_of(s.params, 0.25)
    Y = _random_rhs(s, 0)
    Y[:s.N] = np.random.default_rng(9).normal(size=s.N)
    Y[:s.N] -= Y[:s.N].mean()
    Xd = ob.solve_dense(s, g, Y)
    Xs = ob.solve_direct(s, g, Y)
    Xc, it = ob.solve_cg(s, g, Y, tol=1e-14)
    nrm = np.abs(Xd).max()
    assert np.abs(Xs - Xd).max() < 1e-10 * nrm
    assert np.abs(Xc - Xd).max() < 1e-10 * nrm
    assert it > 1
    for X in (Xd, Xs, Xc):
        assert abs((s.M @ X[:s.N]).sum()) < 1e-12 * nrm
        L = ob.system_matrix(s, g)
        assert np.linalg.norm(L @ X - Y) < 1e-10 * np.linalg.norm(Y)


def test_zero_rhs_gives_zero():
    m = torso_square_2d(9)
    s = ob.build_system(m, params_2d(0.25))
    X, it = ob.solve_cg(s, 4000.0, np.zeros(s.N + s.NH))
    assert it == 0 and not X.any()


def test_scheme_satisfies_discrete_equations():
    # the solution of Step 2 with Y from Step 1 satisfies eq. bid-disc-a as written
    m = torso_square_2d(17)
    p = params_2d(0.25)
    s = ob.build_system(m, p)
    U, V, h = ob.initial_state(s)
    rng = np.random.default_rng(5)
    V = V + 40 * rng.random(s.NH)
    h = rng.random(s.NH)
    ist = ob.heart_stimulus(s, stimulus_left_apex(m))
    dt = p["dt"]
    U1, V1, h1 = ob.time_step(s, U, V, h, ist, 0.0, dt)
    Pi = ob.restriction(s.N, s.NH)
    eq1 = s.S1 @ U1 + Pi.T @ (s.Si @ V1)
    i_ion, g = ob.ms_reaction(V, h, p)
    lhs2 = (p["chi"] * p["Cm"] * (s.MH @ (V1 - V)) / dt + p["chi"] * (s.MH @ (i_ion - ist)))
    rhs2 = -(s.Si @ (Pi @ U1)) - s.Si @ V1
    scale = np.abs(lhs2).max()
    assert np.abs(eq1).max() < 1e-9 * scale
    assert np.abs(lhs2 - rhs2).max() < 1e-9 * scale
    np.testing.assert_allclose(h1, h + dt * g, rtol=0, atol=0)


def test_rest_is_a_fixed_point():
    m = torso_square_2d(17)
    s = ob.build_system(m, params_2d(0.25))
    U, V, h = ob.initial_state(s)
    U1, V1, h1 = ob.time_step(s, U, V, h, np.zeros(s.NH), 5.0, 0.25)
    assert np.abs(U1).max() < 1e-9 and np.abs(V1 - V).max() < 1e-9
    assert np.abs(h1 - 1).max() == 0


def test_monodomain_reduction_equal_anisotropy():
    # isolated heart with sigma_e = lam sigma_i: the bidomain step's V equals the
    # monodomain step (gamma M + S_m) V = Y_2 and U = -V/(1+lam) + c (Sec. 1, 5.2)
    lam = 0.6
    m = slab_3d(7, 7, 4)
    p = params_3d(0.05)
    p["sigma_e"] = tuple(lam * np.array(p["sigma_i"]))
    s = ob.build_system(m, p)
    rng = np.random.default_rng(6)
    V = p["v_rest"] + 100 * rng.random(s.NH)
    h = rng.random(s.NH)
    ist = np.zeros(s.NH)
    U1, V1, _ = ob.time_step(s, np.zeros(s.N), V, h, ist, 3.0, 0.05)
    g = ob.gamma_of(p, 0.05)
    Y = ob.rhs(s, V, h, ist, 3.0, 0.05)
    Vm = spla.spsolve((g * s.MH + s.Sm).tocsc(), Y[s.N:])
    np.testing.assert_allclose(V1, Vm, rtol=1e-10, atol=1e-10 * np.abs(Vm).max())
    Um = -Vm / (1 + lam)
    Um -= (s.M @ Um).sum() / s.M.sum()
    np.testing.assert_allclose(U1, Um, atol=1e-9 * np.abs(Um).max())


def _poisson_error(n, sig):
    # pure-Neumann Poisson -div(sig grad u) = f on [0,L]^2, u* = cos(kx)cos(ky)
    L = 10.0
    m = torso_square_2d(n, length=L, semi_axes=(1e-9, 1e-9))
    assert m.region.sum() == 0
    k = np.pi / L
    x, y = m.coords[:, 0], m.coords[:, 1]
    u = np.cos(k * x) * np.cos(k * y)
    f = (sig[0] + sig[1]) * k * k * u
    X = m.coords[m.elems]
    S = ob.assemble(m.elems, ob.element_stiffness(X, np.broadcast_to(np.diag(sig), (m.n_elems, 2, 2))), m.n_nodes)
    M = ob.assemble(m.elems, ob.element_mass(X, lumped=False), m.n_nodes)
    b = M @ f
    b -= b.mean()
    keep = np.arange(m.n_nodes - 1)
    uh = np.zeros(m.n_nodes)
    uh[keep] = spla.spsolve(S[keep][:, keep].tocsc(), b[keep])
    uh -= (M @ uh).sum() / M.sum()
    e = uh - u
    return np.sqrt(e @ (M @ e))


@pytest.mark.parametrize("sig", [(2.0, 2.0), (3.0, 0.3)])
def test_manufactured_second_order(sig):
    errs = [_poisson_error(n, sig) for n in (9, 17, 33, 65)]
    rates = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.6 < r < 4.4 for r in rates[1:]), rates


def test_config_small_wave_is_excited():
    # 65^2 torso, 40 steps of 0.25 ms: the stimulated corner depolarises (the
    # 50 uA/cm^2, 1 ms stimulus is a workload reading; the paper gives no amplitude)
    m = torso_square_2d(65)
    p = params_2d(0.25)
    s = ob.build_system(m, p)
    ist = ob.heart_stimulus(s, stimulus_left_apex(m))
    U, V, h = ob.initial_state(s)
    t = 0.0
    for _ in range(40):
        U, V, h = ob.time_step(s, U, V, h, ist, t, p["dt"])
        t += p["dt"]
    assert V.max() > 0.0                 # upstroke reached
    assert (V > -40).sum() > (ist > 0).sum()  # the wave has spread past the site
    assert abs((s.M @ U).sum()) < 1e-9 * np.abs(U).max()
