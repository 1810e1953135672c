"""GPU parity of block parallel / block pairwise LU_PRRP (Section 5, Appendix E) against the
CPU oracle: identical permutations where the oracle's decisions are untied (margins above
1e-8), the same stored factors (pivot rows' L11\\U11 and U12, every eliminated row's D)
to rounding, the same growth factor, max |D| and interchange count."""
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


@pytest.fixture(scope="module")
def ctx(prrp):
    c = prrp.prrp_create(0)
    yield c
    c.close()


def _block(prrp, ctx, A, b, P, tree, tau=2.0):
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    F = prrp.prrp_factor_block(ctx, dA, P, tree=tree, b=b, tau=tau)
    torch.cuda.synchronize()
    out = dA.cpu().numpy(), F.perm().astype(np.int64), F.stats()
    F.close()
    return out


@pytest.mark.parametrize("tree", ["parallel", "pairwise"])
@pytest.mark.parametrize("n,b,P,tau", [(256, 16, 4, 2.0), (300, 8, 8, 2.0), (512, 16, 16, 2.0), (97, 5, 3, 1.05),
                                       (200, 16, 1, 2.0), (640, 32, 7, 1.1)])
def test_block_matches_oracle(prrp, ctx, tree, n, b, P, tau):
    A = pi.randn(n, 6000 + n + P)
    ref = oracle.block_lu_prrp(A, b=b, P=P, tau=tau, tree=tree, max_swaps=64)
    LU, perm, st = _block(prrp, ctx, A, b, P, tree, tau)
    assert sorted(perm) == list(range(n))
    assert ref.min_margin > 1e-8, "choose a case with untied decisions"
    assert np.array_equal(perm, ref.perm)
    scale = float(np.max(np.abs(ref.LU)))
    np.testing.assert_allclose(LU, ref.LU, rtol=1e-9, atol=1e-9 * scale)
    assert st["growth"] == pytest.approx(ref.growth, rel=1e-9)
    assert st["max_l21"] == pytest.approx(ref.max_D, rel=1e-9)
    assert st["swaps"] == ref.swaps


def test_one_block_is_lu_prrp(prrp, ctx):
    A = pi.randn(250, 6100)                 # one block of 250 rows: one CTA's node
    _, perm, st = _block(prrp, ctx, A, 16, 1, "parallel")
    dA = torch.from_numpy(A).cuda()
    F = prrp.prrp_factor(ctx, dA, b=16)
    assert np.array_equal(perm, F.perm().astype(np.int64))
    assert st["growth"] == pytest.approx(F.stats()["growth"], rel=1e-12)
    F.close()


def test_block_limits(prrp, ctx):
    A = torch.from_numpy(pi.randn(1024, 6200)).cuda()
    with pytest.raises(prrp.PrrpError) as e:          # a 512-row leaf does not fit one CTA
        prrp.prrp_factor_block(ctx, A.clone(), 2, tree="parallel", b=16)
    assert e.value.name == "PRRP_ERR_UNSUPPORTED"
    F = prrp.prrp_factor_block(ctx, A.clone(), 16, tree="pairwise", b=16)
    with pytest.raises(prrp.PrrpError) as e:          # a product form, not P A = L U
        prrp.prrp_solve(ctx, F, torch.zeros((1024, 1), dtype=torch.float64, device="cuda"))
    assert e.value.name == "PRRP_ERR_UNSUPPORTED"
    F.close()
