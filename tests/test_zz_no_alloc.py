"""The allocation-free factor solve (bid_apply_factor_noalloc) gives the same
result as bid_apply_factor, called twice in a row through the C ABI.

It exists for callers that cannot call cudaMalloc when they solve (a
real-time loop that must avoid the allocator's implicit synchronisation, or an
application that gives the library a fixed memory budget and forbids device
allocations afterwards), so its scratch lives in one static device array.  This file is collected last so that
a run stopping at the first failure has run every other test already; it
passes both alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

from workloads import torso_square_2d, params_2d

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


@pytest.mark.parametrize("precision,eps", [("fp64", 0.0), ("fp32", 1e-3)])
def test_noalloc_matches_allocating_entry_point(bid, precision, eps):
    mesh, p = torso_square_2d(97), params_2d(0.1)
    S = bid.System(mesh, p)
    P = bid.Precond(S, p["dt"], eps=eps, precision=precision)
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream().cuda_stream
    for which, n in ((1, S.N), (2, S.NH)):
        b = torch.tensor(rng.normal(size=n), dtype=torch.float64, device=DEV)
        ref = torch.zeros(n, dtype=torch.float64, device=DEV)
        P.apply_factor(which, b, ref)
        torch.cuda.synchronize()
        r = ref.cpu().numpy()
        for call in range(2):
            x = torch.full((n,), np.nan, dtype=torch.float64, device=DEV)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            rc = bid.lib.bid_apply_factor_noalloc(P.h, which, b.data_ptr(), x.data_ptr(), stream)
            assert rc == bid.OK, bid.lib.bid_last_error()
            torch.cuda.synchronize()
            if call > 0:
                # after the first call (which may load the module that holds the
                # static array) a call takes no device memory at all
                assert torch.cuda.mem_get_info()[0] == free0, which
            xn = x.cpu().numpy()
            assert np.isfinite(xn).all()
            assert np.abs(xn - r).max() <= 1e-12 * np.abs(r).max(), (which, call)


def test_noalloc_rejects_factor_larger_than_scratch(bid):
    mesh, p = torso_square_2d(1025), params_2d(0.1)
    S = bid.System(mesh, p)
    P = bid.Precond(S, p["dt"], eps=0.0, precision="fp32")
    b = torch.ones(S.N, dtype=torch.float64, device=DEV)
    x = torch.zeros_like(b)
    rc = P.apply_factor_noalloc(1, b, x, check=False)
    assert rc == bid.EINVAL
    assert b"static scratch" in bid.lib.bid_last_error()
