"""CPU checks of the multigrid alternative for P_1 and P_K (host replay of the
V-cycle the GPU kernels run, bid_host_mg_solve).

The paper leaves the preconditioners of S_1 and K open (Sec. 5.2: any good
preconditioner of each fits the block-LU form); a V-cycle of geometric
multigrid is one.  What pins it, without a reference implementation:
- it is a symmetric positive operator (Chebyshev smoothers with the same
  polynomial before and after the correction, Galerkin coarse operators), so
  conjugate gradients may use it: <V a, b> = <a, V b> on 1^perp to rounding;
- its error contraction as a stationary iteration x += V (b - A x) is small
  and does not grow with the mesh (the multigrid property): below 0.3 on the
  65^2 .. 257^2 slices and the 3D slab, for S_1 and for K_m;
- meshes that are not Kuhn lattices are refused.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import bidomain as ob
from workloads import torso_square_2d, slab_3d, params_2d, params_3d


@pytest.fixture(scope="module")
def bid():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_08708_gb300 import bid as b
    return b


def _host(bid, mesh, p):
    H = bid.HostSystem(mesh, p)
    ptr, col, val = H.csr(0)
    S1 = sp.csr_matrix((val, col, ptr))
    ptr, col, val = H.csr(2)
    Sm = sp.csr_matrix((val, col, ptr))
    _, m, mH = H.perm_and_mass()
    g = ob.gamma_of(p, p["dt"])
    return H, S1, (g * sp.diags(mH) + Sm).tocsr(), g


def _contraction(apply, A, b, project, its=3):
    # mean residual reduction per step over the first steps (later ones reach
    # the rounding floor when the cycle is nearly exact)
    x = np.zeros_like(b)
    res = []
    for _ in range(its + 1):
        r = b - A @ x
        if project:
            r -= r.mean()
        res.append(np.linalg.norm(r))
        x = x + apply(r)
    return (res[-1] / res[0]) ** (1.0 / its)


@pytest.mark.parametrize("n", [65, 129, 257])
def test_vcycle_contracts_independently_of_the_mesh(bid, n):
    mesh, p = torso_square_2d(n), params_2d(0.1)
    H, S1, Km, g = _host(bid, mesh, p)
    rng = np.random.default_rng(n)
    b = rng.normal(size=S1.shape[0])
    b -= b.mean()
    f1 = _contraction(lambda r: H.mg_solve(1, r)[0], S1, b, True)
    bk = rng.normal(size=Km.shape[0])
    fk = _contraction(lambda r: H.mg_solve(2, r, gamma=g)[0], Km, bk, False)
    assert f1 < 0.3 and fk < 0.3, (n, f1, fk)
    _, levels = H.mg_solve(1, b)
    assert levels >= 3 + (n > 65) + (n > 129)


def test_vcycle_contracts_on_the_slab(bid):
    mesh, p = slab_3d(33, 33, 11), params_3d(0.05)
    H, S1, Km, g = _host(bid, mesh, p)
    rng = np.random.default_rng(7)
    b = rng.normal(size=S1.shape[0])
    b -= b.mean()
    f1 = _contraction(lambda r: H.mg_solve(1, r)[0], S1, b, True)
    fk = _contraction(lambda r: H.mg_solve(2, r, gamma=g)[0], Km, rng.normal(size=Km.shape[0]), False)
    assert f1 < 0.35 and fk < 0.35, (f1, fk)


@pytest.mark.parametrize("which", [1, 2])
def test_vcycle_is_symmetric_positive(bid, which):
    mesh, p = torso_square_2d(65), params_2d(0.1)
    H, S1, Km, g = _host(bid, mesh, p)
    n = S1.shape[0] if which == 1 else Km.shape[0]
    rng = np.random.default_rng(3 + which)
    a, c = rng.normal(size=n), rng.normal(size=n)
    if which == 1:
        a -= a.mean()
        c -= c.mean()
    Va = H.mg_solve(which, a, gamma=g)[0]
    Vc = H.mg_solve(which, c, gamma=g)[0]
    if which == 1:               # the singular hierarchy's output is defined up to a constant
        Va -= Va.mean()
        Vc -= Vc.mean()
    assert abs(Va @ c - a @ Vc) <= 1e-12 * np.linalg.norm(Va) * np.linalg.norm(c)
    assert Va @ a > 0 and Vc @ c > 0


def test_refuses_meshes_that_are_not_kuhn_lattices(bid):
    p = params_2d(0.1)
    m = torso_square_2d(33)
    mirrored = m.__class__(**{**m.__dict__})
    mirrored.coords = m.coords.copy()
    mirrored.coords[:, 0] = 10.0 - mirrored.coords[:, 0]     # "/" cells become "\\" cells
    H = bid.HostSystem(mirrored, p)
    N, NH = H.csr(0)[0].size - 1, H.csr(1)[0].size - 1
    with pytest.raises(bid.BidError) as e:
        H.mg_solve(1, np.zeros(N))
    assert e.value.code == bid.EINVAL and b"Kuhn" in bid.lib.bid_last_error()
    jittered = m.__class__(**{**m.__dict__})
    jittered.coords = m.coords + 1e-3 * np.random.default_rng(1).random(m.coords.shape)
    H = bid.HostSystem(jittered, p)
    with pytest.raises(bid.BidError) as e:
        H.mg_solve(2, np.zeros(NH), gamma=1.0)
    assert e.value.code == bid.EINVAL and b"lattice" in bid.lib.bid_last_error()
