"""Pins of the oracle's system matrix against Props. 1-3 and Remark K (dense,
tiny meshes), and of the exact-limit preconditioner against the equal-anisotropy
case where the monodomain approximation is exact (Sec. 1, Sec. 5.2)."""
import numpy as np
import pytest

from oracle import bidomain as ob
from oracle import algebra as oa
from workloads import torso_square_2d, slab_3d, params_2d, params_3d


@pytest.fixture(scope="module")
def tiny():
    m = torso_square_2d(13)
    s = ob.build_system(m, params_2d(0.25))
    g = ob.gamma_of(s.params, 0.25)
    return s, g, oa.dense_blocks(s, g)


def test_prop1_psd_and_kernel(tiny):
    s, g, B = tiny
    Lam = B["Lam"]
    assert s.NH > 10
    assert np.abs(Lam - Lam.T).max() < 1e-12 * np.abs(Lam).max()
    w, V = np.linalg.eigh(Lam)
    tol = 1e-12 * np.abs(w).max()
    assert np.sum(np.abs(w) <= tol) == 1
    assert w.min() > -tol
    k = np.argmin(np.abs(w))
    v = V[:, k] / V[0, k]
    np.testing.assert_allclose(v[:s.N], 1.0, atol=1e-9)
    np.testing.assert_allclose(v[s.N:], 0.0, atol=1e-9)


def test_range_u_block_sums_to_zero(tiny):
    s, g, B = tiny
    X = np.random.default_rng(1).normal(size=s.N + s.NH)
    Y = B["Lam"] @ X
    assert abs(Y[:s.N].sum()) < 1e-10 * np.abs(Y).max()


def test_prop2_lu(tiny):
    s, g, B = tiny
    np.testing.assert_allclose(B["L"] @ B["U"], B["Lam"], atol=1e-9 * np.abs(B["Lam"]).max())
    K = B["K"]
    assert np.abs(K - K.T).max() < 1e-9 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() > 0


def test_remark_k_harmonic_mean(tiny):
    _, _, B = tiny
    K0q, Aq = oa.harmonic_part_on_complement(B)
    np.testing.assert_allclose(K0q @ Aq, np.eye(K0q.shape[0]), atol=1e-7)


def test_prop3_pseudo_inverse_solves(tiny):
    s, g, B = tiny
    rng = np.random.default_rng(2)
    Y = rng.normal(size=s.N + s.NH)
    Y[:s.N] -= Y[:s.N].mean()              # Y in Ran(Lambda)
    X = B["Uinv"] @ B["Lp"] @ Y
    np.testing.assert_allclose(B["Lam"] @ X, Y, atol=1e-8 * np.abs(Y).max())


def _equal_anisotropy_slab(lam=0.7):
    m = slab_3d(5, 5, 4)
    p = params_3d(0.05)
    p["sigma_e"] = tuple(lam * np.array(p["sigma_i"]))
    return ob.build_system(m, p), ob.gamma_of(p, 0.05), lam


def test_monodomain_exact_for_equal_anisotropy():
    s, g, _ = _equal_anisotropy_slab()
    B = oa.dense_blocks(s, g)
    np.testing.assert_allclose(B["Km"], B["K"], atol=1e-9 * np.abs(B["K"]).max())


def test_exact_limit_preconditioner_is_exact_inverse_for_equal_anisotropy():
    s, g, _ = _equal_anisotropy_slab()
    rng = np.random.default_rng(3)
    r = rng.normal(size=s.N + s.NH)
    r[:s.N] -= r[:s.N].mean()
    z = ob.precond_apply_exact(s, g, r)
    Lam = ob.system_matrix(s, g)
    np.testing.assert_allclose(Lam @ z, r, atol=1e-9 * np.abs(r).max())


def test_exact_limit_preconditioner_matches_dense_lu_form(tiny):
    # eq. prec2 with P_1 = S_1 and P_K = K_m, built densely, vs the oracle routine
    s, g, B = tiny
    rng = np.random.default_rng(4)
    r = rng.normal(size=s.N + s.NH)
    r[:s.N] -= r[:s.N].mean()
    S1p, Si, Pi, Km = B["S1p"], B["Si"], B["Pi"], B["Km"]
    Kmi = np.linalg.inv(Km)
    Lp = np.block([[S1p, np.zeros((s.N, s.NH))], [-Kmi @ Si @ Pi @ S1p, Kmi]])
    Up = np.block([[np.eye(s.N), -S1p @ Pi.T @ Si], [np.zeros((s.NH, s.N)), np.eye(s.NH)]])
    z_dense = Up @ Lp @ r
    z = ob.precond_apply_exact(s, g, r)
    z[:s.N] -= z[:s.N].mean()
    z_dense[:s.N] -= z_dense[:s.N].mean()
    np.testing.assert_allclose(z, z_dense, atol=1e-8 * np.abs(z_dense).max())
