"""The allocation-free panel selection (prrp_panel_select_noalloc) against the existing
context-based entry point, through the C ABI, on two calls in a row.

It exists for callers that cannot allocate device memory (a fixed arena owned by another
allocator, latency budgets that cannot absorb cudaMalloc's synchronization, or no
prrp_ctx); its scratch lives in a static device array shared by all calls, so the second
call also checks that the previous call's leftovers do not leak into the result.  This
file is collected last so a run that stops at the first failure has run everything else.
"""
import numpy as np
import pytest

import prrp_inputs as pi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prrp():
    import paper_1208_2451_gb300 as P
    return P


def _compare(prrp, ctx, P, tau):
    dP = torch.from_numpy(P).cuda()
    order_ref, L21_ref, sw_ref = prrp.prrp_panel_select(ctx, dP, tau=tau)
    order, L21, sw = prrp.prrp_panel_select_noalloc(dP, tau=tau)
    torch.cuda.synchronize()
    assert np.array_equal(order.cpu().numpy(), order_ref)
    assert sw == sw_ref
    np.testing.assert_allclose(L21.cpu().numpy(), L21_ref.cpu().numpy(), atol=1e-10, rtol=1e-9)


def test_noalloc_matches_context_entry_point_twice(prrp):
    ctx = prrp.prrp_create(0)
    try:
        # first call: a tall panel that needs interchanges (tau close to 1)
        _compare(prrp, ctx, pi.randn(64, 7 + 8192, m=8192), 1.05)
        # second call in a row, a different shape: the static scratch keeps the first
        # call's contents, which must not affect this result
        _compare(prrp, ctx, pi.randn(16, 7 + 1000, m=1000), 2.0)
    finally:
        ctx.close()
