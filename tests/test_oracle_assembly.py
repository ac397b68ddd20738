"""Pins of the oracle's discretisation (Sec. 3.1) against textbook forms and the
invariants the paper states (H1, H2, masses summing to the domain measure)."""
import os

import numpy as np
import pytest

from oracle import bidomain as ob
from workloads import torso_square_2d, slab_3d, params_2d, params_3d

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "p1_element_matrices.txt")


def _golden():
    out, name, scale, rows = {}, None, 1.0, []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            if name:
                out[name] = scale * np.array(rows)
            name, rows = line[1:-1], []
        elif line.startswith("scale"):
            scale = float(line.split()[1])
        else:
            rows.append([float(v) for v in line.split()])
    out[name] = scale * np.array(rows)
    return out


@pytest.mark.parametrize("h", [1.0, 0.37])
def test_triangle_stiffness_textbook(h):
    X = np.array([[[0.0, 0.0], [h, 0.0], [0.0, h]]])
    K = ob.element_stiffness(X, np.eye(2)[None])[0]
    np.testing.assert_allclose(K, _golden()["triangle_right_angle_at_0"], atol=1e-14)


def test_tetrahedron_stiffness_textbook():
    X = np.array([[[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]])
    K = ob.element_stiffness(X, np.eye(3)[None])[0]
    np.testing.assert_allclose(K, _golden()["tetrahedron_reference"], atol=1e-14)


def test_stiffness_scales_with_conductivity_and_rotation():
    # rotating the element and the tensor together leaves K_e unchanged
    rng = np.random.default_rng(0)
    X = rng.normal(size=(1, 3, 2))
    A = rng.normal(size=(2, 2))
    sig = A @ A.T + np.eye(2)
    c, s = np.cos(0.7), np.sin(0.7)
    R = np.array([[c, -s], [s, c]])
    K1 = ob.element_stiffness(X, sig[None])
    K2 = ob.element_stiffness(X @ R.T, (R @ sig @ R.T)[None])
    np.testing.assert_allclose(K1, K2, atol=1e-12)


@pytest.fixture(scope="module")
def sys2d():
    m = torso_square_2d(33)
    return m, ob.build_system(m, params_2d(0.25))


@pytest.fixture(scope="module")
def sys3d():
    m = slab_3d(9, 9, 5)
    return m, ob.build_system(m, params_3d(0.05))


def test_h1_heart_first(sys2d):
    m, s = sys2d
    el = s.new_of_old[m.elems[m.region == 1]]
    assert el.max() < s.NH            # every heart element lives on the first N_H nodes
    assert s.NH == np.unique(m.elems[m.region == 1]).size


@pytest.mark.parametrize("which", ["sys2d", "sys3d"])
def test_h2_kernels_and_symmetry(which, request):
    _, s = request.getfixturevalue(which)
    for A, n in ((s.S1, s.N), (s.Se, s.N), (s.Si, s.NH), (s.Sm, s.NH)):
        assert abs(A - A.T).max() < 1e-13 * abs(A).max()
        assert np.abs(A @ np.ones(n)).max() < 1e-12 * abs(A).max()


def test_mass_totals_2d(sys2d):
    m, s = sys2d
    h = m.meta["h"]
    # brute force: count heart triangles, each of area h^2/2
    n_heart = sum(1 for r in m.region.tolist() if r == 1)
    for lumped in (True, False):
        ss = ob.build_system(m, params_2d(0.25), lumped=lumped)
        assert abs(ss.M.sum() - 100.0) < 1e-10
        assert abs(ss.MH.sum() - n_heart * h * h / 2) < 1e-10


def test_mass_totals_3d(sys3d):
    _, s = sys3d
    assert abs(s.M.sum() - 0.3) < 1e-13
    assert abs(s.MH.sum() - 0.3) < 1e-13


def test_lumped_is_row_sum_of_consistent(sys2d):
    m, _ = sys2d
    a = ob.build_system(m, params_2d(0.25), lumped=True)
    b = ob.build_system(m, params_2d(0.25), lumped=False)
    np.testing.assert_allclose(a.M.diagonal(), np.asarray(b.M.sum(axis=1)).ravel(), rtol=1e-13)


def test_fibre_frame_tensors():
    m = torso_square_2d(9)
    th = np.deg2rad(30.0)
    a = np.array([np.cos(th), np.sin(th)])
    t = np.array([-np.sin(th), np.cos(th)])
    sig = ob.fibre_tensor(m.fibre[:1], np.array([3.0, 0.3, 0.3]))[0]
    assert abs(a @ sig @ a - 3.0) < 1e-14 and abs(t @ sig @ t - 0.3) < 1e-14
    assert abs(a @ sig @ t) < 1e-14


def test_monodomain_tensor_harmonic_means():
    # sigma_m in the fibre frame = diag of harmonic means g_i g_e / (g_i + g_e)
    m = slab_3d(3, 3, 3)
    p = params_3d(0.05)
    sys = ob.build_system(m, p)
    F = m.fibre[0]
    si = ob.fibre_tensor(m.fibre[:1], np.array(p["sigma_i"]))[0]
    se = ob.fibre_tensor(m.fibre[:1], np.array(p["sigma_e"]))[0]
    sm = np.linalg.inv(np.linalg.inv(si) + np.linalg.inv(se))
    local = F.T @ sm @ F
    expect = np.array([1.2, 1.65 / 2.65, 0.24375])
    np.testing.assert_allclose(np.diag(local), expect, rtol=1e-13)
    assert np.abs(local - np.diag(np.diag(local))).max() < 1e-13
    assert sys.Sm.shape == (sys.NH, sys.NH)
