"""The allocation-free panel selection (prrp_panel_select_noalloc) against the existing
context-based entry point, through the C ABI, on calls in a row, and against the oracle's
strong RRQR (Algorithm 2).

It exists for callers that cannot allocate device memory (a fixed arena owned by another
allocator, latency budgets that cannot absorb cudaMalloc's synchronization, or no
prrp_ctx); its scratch lives in a static device array shared by all calls, so every call
after the first also checks that the previous call's leftovers do not leak into the
result.  Both entry points run the same kernel with the same grid, so their outputs must be
bit-identical.  This file is collected last so a run that stops at the first failure has
run everything else.
"""
import numpy as np
import pytest

import oracle
import prrp_inputs as pi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prrp():
    import paper_1208_2451_gb300 as P
    return P


def _compare(prrp, ctx, P, tau):
    m, w = P.shape
    dP = torch.from_numpy(P).cuda()
    order_ref, L21_ref, sw_ref = prrp.prrp_panel_select(ctx, dP, tau=tau)
    order, L21, sw = prrp.prrp_panel_select_noalloc(dP, tau=tau)
    torch.cuda.synchronize()
    order = order.cpu().numpy()
    assert np.array_equal(order, order_ref)
    assert sw == sw_ref
    assert np.array_equal(L21.cpu().numpy(), L21_ref.cpu().numpy())
    # the oracle's strong RRQR: the same selection where its decisions are not near-ties
    ref = oracle.strong_rrqr(P.T, tau=tau, max_swaps=64)
    margins = ref.qrcp_margins + ref.test_margins + ref.choice_margins
    if min(margins, default=np.inf) > 1e-8:
        assert list(order) == list(ref.order)
        assert sw == ref.swaps
        np.testing.assert_allclose(L21.cpu().numpy(), ref.M.T, atol=1e-10, rtol=1e-9)
    if m > w:
        Lx = np.linalg.solve(P[order[:w]].T, P[order[w:]].T).T
        assert np.max(np.abs(Lx)) <= tau * (1 + 1e-9)


def test_noalloc_matches_context_entry_point_in_a_row(prrp):
    ctx = prrp.prrp_create(0)
    try:
        # a tall panel that needs interchanges (tau close to 1): the cooperative grid
        _compare(prrp, ctx, pi.randn(64, 7 + 8192, m=8192), 1.05)
        # the next call, another shape: the static scratch keeps the first call's
        # contents, which must not affect this result
        _compare(prrp, ctx, pi.randn(16, 7 + 1000, m=1000), 2.0)
        # m <= 512: the thread-block-cluster form of the same kernel
        _compare(prrp, ctx, pi.randn(16, 7 + 300, m=300), 1.05)
        # the 128-wide class
        _compare(prrp, ctx, pi.randn(128, 7 + 3000, m=3000), 2.0)
    finally:
        ctx.close()
