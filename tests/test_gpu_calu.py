"""GPU parity of CALU_PRRP (Section 3: tournament pivoting) against the CPU oracle.

Bar (as for LU_PRRP):
* the permutation is identical whenever the oracle's smallest decision margin (over every
  tree node's QRCP, interchange test and choice, and the diagonal-block GEPP) exceeds 1e-8;
* ||PA - LU||_F / ||A||_F <= 64 n 2^-53;
* statistics (growth, max |L21|, interchanges) equal the oracle's;
* the growth factor stays under Section 3.2's bound (1 + tau b)^((n/b)(H+1) - 1);
* element-wise factors within the first-order bounds of tests/test_gpu_parity.py.
"""
import numpy as np
import pytest

import oracle
import prrp_inputs as pi
from oracle import metrics as M
from tests.test_gpu_parity import factor_tolerances

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def prrp():
    import paper_1208_2451_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(prrp):
    c = prrp.prrp_create(0)
    yield c
    c.close()


def _calu(prrp, ctx, A, b, leaf, tau=2.0, prec=0):
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    F = prrp.prrp_factor_calu(ctx, dA, leaf, b=b, tau=tau, prec=prec)
    torch.cuda.synchronize()
    out = dA.cpu().numpy(), F.perm().astype(np.int64), F.stats()
    F.close()
    return out


@pytest.mark.parametrize("n,b,leaf,tau,seed", [
    (256, 16, 16, 2.0, 1), (300, 16, 32, 1.05, 2), (513, 32, 64, 2.0, 3), (200, 8, 24, 2.0, 4),
    (1000, 64, 128, 2.0, 5), (2048, 64, 64, 2.0, 6), (777, 16, 40, 1.05, 7), (129, 64, 64, 2.0, 8)])
def test_calu_matches_oracle(prrp, ctx, n, b, leaf, tau, seed):
    A = pi.randn(n, 4000 + seed)
    ref = oracle.calu_prrp(A, b=b, tau=tau, leaf_rows=leaf, max_swaps=64)
    LU, perm, st = _calu(prrp, ctx, A, b, leaf, tau)
    assert sorted(perm) == list(range(n))
    assert M.factor_residual(A, LU, perm) <= 64 * n * EPS
    if ref.min_margin > 1e-8:
        assert np.array_equal(perm, ref.perm), "tournament pivots differ with untied decisions"
        assert st["swaps"] == ref.swaps
        assert st["growth"] == pytest.approx(ref.growth, rel=1e-9)
        assert st["max_l21"] == pytest.approx(ref.max_L21, rel=1e-9)
        if n <= 1000:
            tL, tU = factor_tolerances(ref.LU)
            assert np.all(np.abs(np.tril(LU, -1) - np.tril(ref.LU, -1)) <= tL + 1e-300)
            assert np.all(np.abs(np.triu(LU) - np.triu(ref.LU)) <= tU + 1e-300)
    assert np.log10(st["growth"]) <= oracle.calu_growth_bound_log10(n, b, tau, ref.height)


def test_one_leaf_is_lu_prrp(prrp, ctx):
    """Panels of fewer than 2 leaf_rows rows are one leaf: the pivots of prrp_factor."""
    A = pi.randn(250, 41)
    LU, perm, st = _calu(prrp, ctx, A, 16, 128)
    dA = torch.from_numpy(A).cuda()
    F = prrp.prrp_factor(ctx, dA, b=16)
    assert np.array_equal(perm, F.perm().astype(np.int64))
    assert st["growth"] == pytest.approx(F.stats()["growth"], rel=1e-12)
    F.close()


def test_calu_mixed_refined_solve(prrp, ctx):
    """Tournament pivots (FP64) with the 3xBF16 tensor-core Schur update and FP64 refinement:
    FP64-level normwise backward error."""
    n = 1500
    A = pi.randn(n, 4100)
    B = pi.rhs(n, 3, 4100)
    dA = torch.from_numpy(A).cuda()
    F = prrp.prrp_factor_calu(ctx, dA, 64, b=64, prec=2)
    dB = torch.from_numpy(B).cuda()
    info = prrp.prrp_solve(ctx, F, dB, A_orig=torch.from_numpy(A).cuda(), refine_max_iter=30)
    F.close()
    X = dB.cpu().numpy()
    assert info["eta"] <= 1e-15
    for c in range(3):
        assert M.eta(A, X[:, c], B[:, c]) <= 1e-15


def test_calu_errors(prrp, ctx):
    A = torch.from_numpy(pi.randn(300, 42)).cuda()
    for leaf, b, name in ((8, 16, "PRRP_ERR_INVALID_ARG"), (256, 64, "PRRP_ERR_UNSUPPORTED"),
                          (128, 128, "PRRP_ERR_UNSUPPORTED"), (0, 16, "PRRP_ERR_INVALID_ARG")):
        with pytest.raises(prrp.PrrpError) as e:
            prrp.prrp_factor_calu(ctx, A.clone(), leaf, b=b)
        assert e.value.name == name
    # a zero first panel: SINGULAR (every candidate norm is exactly zero)
    Z = pi.randn(200, 43)
    Z[:, :16] = 0.0
    with pytest.raises(prrp.PrrpError) as e:
        prrp.prrp_factor_calu(ctx, torch.from_numpy(Z).cuda(), 32, b=16)
    assert e.value.name == "PRRP_ERR_SINGULAR"
