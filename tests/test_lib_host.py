"""CPU checks of the C-ABI library: it loads, exports every symbol include/bid.h
declares, and its host half (P1 assembly and the packed hierarchical factor,
replayed on the host over the very blocks and tiles the GPU kernels read)
agrees with the FP64 oracle."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import bidomain as ob
from workloads import torso_square_2d, slab_3d, params_2d, params_3d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bid():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_08708_gb300 import bid as b
    return b


def _declared():
    src = open(os.path.join(ROOT, "include", "bid.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bid_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(bid):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(bid.lib, n), n
        assert n in bid.SIGNATURES, n


def test_binding_arity_matches_header(bid):
    # every prototype's parameter count equals the binding's argument list
    src = open(os.path.join(ROOT, "include", "bid.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decls = {}
    for m in re.finditer(r"\b(bid_\w+)\s*\(([^;{]*?)\)\s*;", src):
        params = m.group(2).strip()
        decls[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    assert len(decls) >= 50
    for name, n in decls.items():
        assert len(bid.SIGNATURES[name][1]) == n, name


def test_library_is_the_in_tree_build(bid):
    assert os.path.dirname(bid.LIB_PATH) == os.path.join(ROOT, "paper_1711_08708_gb300")


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_host_assembly_matches_oracle(bid, case):
    if case == "2d":
        m, p = torso_square_2d(33), params_2d(0.25)
    else:
        m, p = slab_3d(9, 8, 5), params_3d(0.05)
    hs = bid.HostSystem(m, p)
    s = ob.build_system(m, p)
    perm, mm, mH = hs.perm_and_mass()
    assert (perm == s.order).all()
    np.testing.assert_allclose(mm, s.M.diagonal(), rtol=1e-13)
    np.testing.assert_allclose(mH, s.MH.diagonal(), rtol=1e-13)
    for which, A in ((0, s.S1), (1, s.Si), (2, s.Sm)):
        ptr, col, val = hs.csr(which)
        B = sp.csr_matrix((val, col, ptr), shape=A.shape)
        assert abs(B - A).max() <= 1e-14 * abs(A).max()


@pytest.mark.parametrize("leaf,block", [(64, 64), (16, 16), (24, 32)])
def test_host_factor_exact_equals_pseudo_inverse(bid, leaf, block):
    m, p = torso_square_2d(41), params_2d(0.25)
    hs = bid.HostSystem(m, p)
    s = ob.build_system(m, p)
    rng = np.random.default_rng(leaf)
    b = rng.normal(size=s.N)
    x, st = hs.factor_solve(1, b, leaf=leaf, block=block)
    xo = ob.s1_pseudo_inverse_apply(s, b)
    x -= x.mean()
    assert np.abs(x - xo).max() <= 1e-11 * np.abs(xo).max()
    g = ob.gamma_of(p, 0.25)
    b2 = rng.normal(size=s.NH)
    x2, _ = hs.factor_solve(2, b2, gamma=g, leaf=leaf, block=block)
    xo2 = spla.spsolve(ob.monodomain_matrix(s, g).tocsc(), b2)
    assert np.abs(x2 - xo2).max() <= 1e-12 * np.abs(xo2).max()
    assert st["levels1"] >= 1 and st["lowrank_blocks"] == 0


@pytest.mark.parametrize("n,leaf,block,precision", [(161, 16, 128, "fp64"), (129, 32, 64, "fp32"),
                                                   (129, 8, 16, "bf16"), (161, 16, 128, "bf16")])
def test_host_factor_exact_with_upper_levels(bid, n, leaf, block, precision):
    # large enough that clusters above the bottom subtrees exist (upper levels,
    # column-chunked row tasks); the layout padding of each storage precision
    # (16-byte vectors of 2, 4 or 8 entries) is replayed in FP64
    m, p = torso_square_2d(n), params_2d(0.1)
    hs = bid.HostSystem(m, p)
    s = ob.build_system(m, p)
    b = np.random.default_rng(n).normal(size=s.N)
    x, st = hs.factor_solve(1, b, leaf=leaf, block=block, precision=precision)
    x -= x.mean()
    xo = ob.s1_pseudo_inverse_apply(s, b)
    assert np.abs(x - xo).max() <= 1e-10 * np.abs(xo).max()
    assert st["levels1"] >= 3 and st["dense_blocks"] >= 1   # some large clusters


@pytest.mark.parametrize("n,leaf,precision,eps,cap,first", [(161, 16, "fp64", 0.0, 32768, 1),
                                                            (129, 32, "fp32", 1e-3, 32768, 0),
                                                            (161, 16, "bf16", 1e-3, 49152, 1),
                                                            (129, 8, "fp32", 0.0, 65536, 2)])
def test_dataflow_schedule_is_complete(bid, n, leaf, precision, eps, cap, first):
    # the bottom flat levels replayed in the order of the dataflow kernels'
    # signals, each group as early as its dependencies allow (forward the
    # highest-numbered ready group, backward the lowest): a missing
    # dependency would read an update slot or an x entry before it is
    # written, so bit equality with the level-by-level replay checks the
    # schedule
    m, p = torso_square_2d(n), params_2d(0.1)
    hs = bid.HostSystem(m, p)
    rng = np.random.default_rng(n + leaf)
    s = ob.build_system(m, p)
    g = ob.gamma_of(p, 0.1)
    for which, size, gam in ((1, s.N, 0.0), (2, s.NH, g)):
        b = rng.normal(size=size)
        x0, _ = hs.factor_solve(which, b, gamma=gam, eps=eps, leaf=leaf, precision=precision)
        x1, _, sch = hs.factor_solve_dataflow(which, b, smem_cap=cap, first=first, gamma=gam, eps=eps,
                                              leaf=leaf, precision=precision)
        assert sch["first"] == first and sch["levels"] >= 2 and sch["groups"] > 10
        assert sch["deps_fwd"] > 0 and sch["deps_bwd"] >= sch["deps_fwd"]
        assert np.array_equal(x0, x1)
    # a cap below any group: no schedule, plain level order
    _, _, sch = hs.factor_solve_dataflow(1, rng.normal(size=s.N), smem_cap=64, leaf=leaf, precision=precision)
    assert sch["levels"] == 0


@pytest.mark.parametrize("n,leaf,precision,eps", [(129, 16, "fp64", 0.0), (161, 32, "fp32", 1e-3),
                                                  (257, 32, "bf16", 1e-3)])
def test_masked_solve_equals_full_replay(bid, n, leaf, precision, eps):
    # P_1 applied to an input that is zero off the heart (the preconditioner's
    # second P_1 solve): the clusters whose subtree holds no heart node see the
    # constant -mean(b) alone and are replaced by scaled all-ones results;
    # equal to the full replay up to rounding.  A cluster wrongly taken as
    # dead (a live child missed) changes x at O(1).
    m, p = torso_square_2d(n), params_2d(0.1)
    hs = bid.HostSystem(m, p)
    o = ob.build_system(m, p)
    b = np.zeros(o.N)
    b[:o.NH] = np.random.default_rng(n).normal(size=o.NH)
    x0, _ = hs.factor_solve(1, b, eps=eps, leaf=leaf, precision=precision)
    x1, (dead, total) = hs.factor_solve_masked(b, eps=eps, leaf=leaf, precision=precision)
    assert dead > total // 2
    assert np.abs(x1 - x0).max() <= 1e-12 * np.abs(x0).max()
    b[-5] = 1.0
    with pytest.raises(bid.BidError):
        hs.factor_solve_masked(b, eps=eps, leaf=leaf, precision=precision)


@pytest.mark.parametrize("precision,leaf", [("fp32", 32), ("fp64", 16), ("bf16", 32)])
def test_mid_clusters_equal_chunked_replay(bid, monkeypatch, precision, leaf):
    # large clusters whose block fits one CTA's shared memory (BID_MID_BYTES,
    # default 96 KiB) are solved as one unit: every dense row, then each
    # low-rank group's V^T w and U t (backward U^T v, then the columns); the
    # chunked task replay (BID_MID_BYTES=0) gives the same P_1 and P_K solves
    # and the same masked solve up to rounding.  A dropped low-rank group or a
    # wrong row of the block changes x at O(1).
    m, p = torso_square_2d(257), params_2d(0.1)
    hs = bid.HostSystem(m, p)
    o = ob.build_system(m, p)
    rng = np.random.default_rng(257)
    b1, bk = rng.normal(size=o.N), rng.normal(size=o.NH)
    bm = np.zeros(o.N)
    bm[:o.NH] = rng.normal(size=o.NH)
    g = p["chi"] * p["Cm"] / p["dt"]
    monkeypatch.setenv("BID_ROOT_GRAM", "0")   # the same top levels in both runs
    out = {}
    for mb in ("0", None):
        if mb is None:
            monkeypatch.delenv("BID_MID_BYTES", raising=False)
        else:
            monkeypatch.setenv("BID_MID_BYTES", mb)
        x1, st = hs.factor_solve(1, b1, eps=1e-3, leaf=leaf, precision=precision)
        xk, _ = hs.factor_solve(2, bk, gamma=g, eps=1e-3, leaf=leaf, precision=precision)
        xm, _ = hs.factor_solve_masked(bm, eps=1e-3, leaf=leaf, precision=precision)
        out[mb] = (x1, xk, xm, st)
    assert out["0"][3]["mid_clusters1"] == 0
    assert out[None][3]["mid_clusters1"] >= 4 and out[None][3]["lowrank_blocks"] > 0
    for a, c in zip(out["0"][:3], out[None][:3]):
        assert np.abs(a - c).max() <= 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("precision,leaf", [("fp32", 32), ("fp64", 16), ("bf16", 32)])
def test_wide_clusters_equal_chunked_replay(bid, monkeypatch, precision, leaf):
    # large clusters split in column slices over a thread-block cluster: the
    # replay builds each CTA's shared-memory image from its bulk copies and
    # reads every factor entry through the kernels' index arithmetic (dense
    # columns, V rows of its slice, U of its groups), combining the partial
    # sums by rank; it equals the chunked task replay (BID_WIDE_BYTES=0) up to
    # rounding in the P_1, P_K and masked solves.  An entry read outside its
    # piece, a row or column covered twice or not at all fails the replay.
    m, p = torso_square_2d(513), params_2d(0.1)
    hs = bid.HostSystem(m, p)
    o = ob.build_system(m, p)
    rng = np.random.default_rng(513)
    b1, bk = rng.normal(size=o.N), rng.normal(size=o.NH)
    bm = np.zeros(o.N)
    bm[:o.NH] = rng.normal(size=o.NH)
    g = p["chi"] * p["Cm"] / p["dt"]
    monkeypatch.setenv("BID_ROOT_GRAM", "0")   # the root stays a wide cluster here
    out = {}
    for wb in ("0", None):
        if wb is None:
            monkeypatch.delenv("BID_WIDE_BYTES", raising=False)
        else:
            monkeypatch.setenv("BID_WIDE_BYTES", wb)
        x1, st = hs.factor_solve(1, b1, eps=1e-3, leaf=leaf, precision=precision)
        xk, stk = hs.factor_solve(2, bk, gamma=g, eps=1e-3, leaf=leaf, precision=precision)
        xm, _ = hs.factor_solve_masked(bm, eps=1e-3, leaf=leaf, precision=precision)
        out[wb] = (x1, xk, xm, st["wide_clusters1"] + stk["wide_clusters1"])
    assert out["0"][3] == 0 and out[None][3] >= 1
    for a, c in zip(out["0"][:3], out[None][:3]):
        assert np.abs(a - c).max() <= 1e-12 * np.abs(a).max()


def test_root_gram_equals_root_passes(bid, monkeypatch):
    # the top block (the root, without boundary or low-rank groups, and its two
    # children, whose boundary rows -- low-rank groups expanded -- lie on the
    # root) solved as one product x = G w with G = M^T M, M the inverse of the
    # block's Cholesky factor assembled at build, against the blocks' forward
    # and backward passes (BID_ROOT_GRAM=0): the same P_1 and masked P_1 solves
    # up to rounding on the 1025^2 slice (root separator of 1025 pivots,
    # children of 512)
    m, p = torso_square_2d(1025), params_2d(0.1)
    hs = bid.HostSystem(m, p)
    o = ob.build_system(m, p)
    rng = np.random.default_rng(1025)
    b1 = rng.normal(size=o.N)
    bm = np.zeros(o.N)
    bm[:o.NH] = rng.normal(size=o.NH)
    out = {}
    for rg in ("0", None):
        if rg is None:
            monkeypatch.delenv("BID_ROOT_GRAM", raising=False)
        else:
            monkeypatch.setenv("BID_ROOT_GRAM", rg)
        x1, st = hs.factor_solve(1, b1, eps=1e-3, leaf=32, precision="fp32")
        xm, _ = hs.factor_solve_masked(bm, eps=1e-3, leaf=32, precision="fp32")
        out[rg] = (x1, xm, st["gram_pivots1"])
    assert out["0"][2] == 0 and out[None][2] == 1025 + 2 * 512   # the root and its two children
    for a, c in zip(out["0"][:2], out[None][:2]):
        assert np.abs(a - c).max() <= 1e-12 * np.abs(a).max()


def test_host_factor_3d_exact():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_08708_gb300 import bid
    m, p = slab_3d(11, 10, 6), params_3d(0.05)
    hs = bid.HostSystem(m, p)
    s = ob.build_system(m, p)
    b = np.random.default_rng(7).normal(size=s.N)
    x, _ = hs.factor_solve(1, b, leaf=32, block=32)
    x -= x.mean()
    xo = ob.s1_pseudo_inverse_apply(s, b)
    assert np.abs(x - xo).max() <= 1e-11 * np.abs(xo).max()


@pytest.mark.parametrize("precision,eps,first", [("fp64", 0.0, 1), ("fp32", 1e-2, 0), ("bf16", 1e-2, 2)])
def test_3d_dataflow_schedule_and_masked_solve(bid, precision, eps, first):
    # 3D slab (isolated heart: every node is a heart node, deeper separators,
    # low-rank groups at eps > 0): the dataflow order equals the level order bit
    # for bit, and the masked replay has no dead cluster and equals the full one
    m, p = slab_3d(17, 17, 7), params_3d(0.05)
    hs = bid.HostSystem(m, p)
    s = ob.build_system(m, p)
    assert s.NH == s.N
    b = np.random.default_rng(31).normal(size=s.N)
    x0, _ = hs.factor_solve(1, b, eps=eps, leaf=16, precision=precision)
    x1, _, sch = hs.factor_solve_dataflow(1, b, smem_cap=65536, first=first, eps=eps, leaf=16,
                                          precision=precision)
    assert sch["levels"] >= 2 and sch["deps_fwd"] > 0
    assert np.array_equal(x0, x1)
    x2, (dead, total) = hs.factor_solve_masked(b, eps=eps, leaf=16, precision=precision)
    assert dead == 0 and total > 10
    assert np.array_equal(x0, x2)


def test_masked_solve_without_heart_input(bid):
    # b = 0 everywhere: mean 0, every result zero, on either path
    m, p = torso_square_2d(65), params_2d(0.1)
    hs = bid.HostSystem(m, p)
    s = ob.build_system(m, p)
    x, (dead, total) = hs.factor_solve_masked(np.zeros(s.N), eps=1e-3, leaf=16, precision="fp32")
    assert not x.any() and 0 < dead < total


def test_host_factor_truncation_error_tracks_eps(bid):
    m, p = torso_square_2d(257), params_2d(0.1)
    hs = bid.HostSystem(m, p)
    s = ob.build_system(m, p)
    b = np.random.default_rng(3).normal(size=s.N)
    x0, _ = hs.factor_solve(1, b)
    x0 -= x0.mean()
    errs = []
    for eps in (1e-2, 1e-4, 1e-6):
        x, st = hs.factor_solve(1, b, eps=eps, leaf=16, block=64)
        x -= x.mean()
        errs.append(np.abs(x - x0).max() / np.abs(x0).max())
        assert st["lowrank_blocks"] > 0
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-3


def test_host_errors(bid):
    m, p = torso_square_2d(9), params_2d(0.25)
    bad = dict(p)
    bad["sigma_T"] = -1.0
    with pytest.raises(bid.BidError) as e:
        bid.HostSystem(m, bad)
    assert e.value.code == bid.EINVAL
    m2 = torso_square_2d(9)
    m2.region[:] = 0
    with pytest.raises(bid.BidError) as e:
        bid.HostSystem(m2, p)
    assert e.value.code == bid.EINVAL
    m3 = torso_square_2d(9)
    m3.elems[0, 0] = 10 ** 6
    with pytest.raises(bid.BidError):
        bid.HostSystem(m3, p)
    hs = bid.HostSystem(m, p)
    with pytest.raises(bid.BidError):
        hs.factor_solve(1, np.zeros(hs.perm_and_mass()[0].size), block=4)


def test_host_factor_disconnected_heart(bid):
    # two separate heart blobs: K_m has two components, so nested dissection
    # meets halves that are already disconnected (no natural separator)
    m = torso_square_2d(65)
    c = m.coords[m.elems].mean(axis=1)
    blob = lambda cx: ((c[:, 0] - cx) / 1.5) ** 2 + ((c[:, 1] - 5) / 2) ** 2 <= 1
    m.region[:] = (blob(2.5) | blob(7.5)).astype(np.int32)
    p = params_2d(0.1)
    hs = bid.HostSystem(m, p)
    s = ob.build_system(m, p)
    g = ob.gamma_of(p, 0.1)
    b2 = np.random.default_rng(1).normal(size=s.NH)
    x2, _ = hs.factor_solve(2, b2, gamma=g, leaf=16)
    xo2 = spla.spsolve(ob.monodomain_matrix(s, g).tocsc(), b2)
    assert np.abs(x2 - xo2).max() <= 1e-12 * np.abs(xo2).max()
    b = np.random.default_rng(2).normal(size=s.N)
    x, _ = hs.factor_solve(1, b, leaf=16)
    x -= x.mean()
    xo = ob.s1_pseudo_inverse_apply(s, b)
    assert np.abs(x - xo).max() <= 1e-10 * np.abs(xo).max()


def _slices(count, seed, min_k, max_k, step, dt=0.1):
    from workloads import batched_slices
    out = []
    for d in batched_slices(count, seed, min_k, max_k, step):
        m = torso_square_2d(d["n"], semi_axes=d["semi_axes"], fibre_deg=d["fibre_deg"])
        out.append((m, params_2d(dt)))
    return out


@pytest.mark.parametrize("precision,leaf", [("fp64", 16), ("fp32", [8, 16, 32, 16]),
                                            ("bf16", [32, 8, 16, 64])])
def test_host_batch_factor_forest(bid, precision, leaf):
    # the forest factor of several slices (one tree per slice, its own leaf
    # size, vector indices in the combined layout, one pin per slice) replays
    # to each slice's own P_1 pseudo-inverse and K_m solve
    sl = _slices(4, 11, 3, 9, 8)
    hs = [bid.HostSystem(m, p) for m, p in sl]
    ss = [ob.build_system(m, p) for m, p in sl]
    off = np.cumsum([0] + [s.N + s.NH for s in ss])
    rng = np.random.default_rng(5)
    b = rng.normal(size=off[-1])
    g = ob.gamma_of(sl[0][1], 0.1)
    x1, st1 = bid.host_batch_factor_solve(hs, 1, b, gamma=g, leaf=leaf, precision=precision)
    x2, _ = bid.host_batch_factor_solve(hs, 2, b, gamma=g, leaf=leaf, precision=precision)
    assert st1["levels1"] >= 3
    for k, s in enumerate(ss):
        o = off[k]
        bu, bv = b[o:o + s.N], b[o + s.N:off[k + 1]]
        xu = x1[o:o + s.N] - x1[o:o + s.N].mean()
        xo = ob.s1_pseudo_inverse_apply(s, bu)
        assert np.abs(xu - xo).max() <= 1e-10 * np.abs(xo).max()
        assert not x1[o + s.N:off[k + 1]].any()          # V entries untouched
        xo2 = spla.spsolve(ob.monodomain_matrix(s, g).tocsc(), bv)
        assert np.abs(x2[o + s.N:off[k + 1]] - xo2).max() <= 1e-12 * np.abs(xo2).max()
        assert not x2[o:o + s.N].any()


@pytest.mark.parametrize("precision,cap,first", [("fp32", 32768, 1), ("fp64", 65536, 0),
                                                  ("bf16", 49152, 2)])
def test_host_batch_dataflow_schedule_is_complete(bid, precision, cap, first):
    # the forest's bottom flat levels in the dataflow order (vector indices of
    # the combined layout, one tree per slice) equal the level-by-level replay
    sl = _slices(3, 7, 6, 10, 16)
    hs = [bid.HostSystem(m, p) for m, p in sl]
    ss = [ob.build_system(m, p) for m, p in sl]
    n = sum(s.N + s.NH for s in ss)
    rng = np.random.default_rng(11)
    g = ob.gamma_of(sl[0][1], 0.1)
    for which in (1, 2):
        b = rng.normal(size=n)
        x0, _ = bid.host_batch_factor_solve(hs, which, b, gamma=g, eps=1e-3, leaf=[32, 16, 32],
                                            precision=precision)
        x1, _, sch = bid.host_batch_factor_solve(hs, which, b, gamma=g, eps=1e-3, leaf=[32, 16, 32],
                                                 precision=precision, smem_cap=cap, first=first,
                                                 schedule=True)
        assert sch["first"] == first and sch["levels"] >= 2
        assert sch["deps_fwd"] > 0 and sch["deps_bwd"] > 0
        assert np.array_equal(x0, x1)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_host_batch_masked_solve_equals_full_replay(bid, precision):
    # the batched preconditioner's second P_1 forest solve: input zero on
    # every slice's torso nodes, each tree shifted by its own mean; the dead
    # clusters take their tree's scaled all-ones results
    sl = _slices(3, 5, 6, 10, 16)
    hs = [bid.HostSystem(m, p) for m, p in sl]
    ss = [ob.build_system(m, p) for m, p in sl]
    off = np.cumsum([0] + [s.N + s.NH for s in ss])
    rng = np.random.default_rng(21)
    b = np.zeros(off[-1])
    for k, s in enumerate(ss):
        b[off[k]:off[k] + s.NH] = rng.normal(size=s.NH)
    kw = dict(eps=1e-3, leaf=[32, 16, 32], precision=precision)
    x0, _ = bid.host_batch_factor_solve(hs, 1, b, **kw)
    x1, _ = bid.host_batch_factor_solve(hs, 1, b, masked=True, **kw)
    assert np.abs(x1 - x0).max() <= 1e-12 * np.abs(x0).max()
    b2 = b.copy()
    b2[off[1] + ss[1].N - 1] = 1.0                   # a torso node of slice 1
    with pytest.raises(bid.BidError):
        bid.host_batch_factor_solve(hs, 1, b2, masked=True, **kw)


def test_host_batch_factor_errors(bid):
    sl = _slices(2, 3, 3, 4, 8)
    hs = [bid.HostSystem(m, p) for m, p in sl]
    n = sum(bid.HostSystem(m, p).perm_and_mass()[0].size + bid.HostSystem(m, p).perm_and_mass()[2].size
            for m, p in sl)
    with pytest.raises(bid.BidError) as e:
        bid.host_batch_factor_solve(hs, 1, np.zeros(n), leaf=[16, 2])
    assert e.value.code == bid.EINVAL
    with pytest.raises(bid.BidError):
        bid.host_batch_factor_solve(hs, 3, np.zeros(n))
