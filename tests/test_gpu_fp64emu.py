"""FP64-accurate Schur update on the BF16 tensor cores (prec = PRRP_FP64_EMU).

Each row of L and each column of U is scaled by a power of two 2^e (max |entry| < 2^e) and
cut into 8 signed base-128 digits, so an entry is represented to within 2^(e - 57), i.e. to
2^-56 of its line's largest magnitude.  All digit products with p + q <= 7 are accumulated
exactly; the dropped ones (p + q >= 8, at most 7 pairs per diagonal, digits up to 128 and
64) add at most K 2^-52 mrow mcol, and the FP64 assembly two roundings of the product and
one of the result.  Per entry, with mrow = max_k |L_ik| and mcol = max_k |U_kj|:
    |dC| <= K 2^-50 mrow mcol + 2^-52 |C_new|,
which for K = 64 is tighter than the worst case of an FP64 dot product, K^2 2^-53 mrow mcol.
"""
import numpy as np
import pytest

import oracle
import prrp_inputs as pi
from oracle import metrics as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53
EMU = 4


@pytest.fixture(scope="module")
def prrp():
    import paper_1208_2451_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(prrp):
    c = prrp.prrp_create(0)
    yield c
    c.close()


def _update(prrp, ctx, L, U, Cm):
    dC = torch.from_numpy(Cm).cuda()
    prrp.prrp_schur_update(ctx, torch.from_numpy(L).cuda(), torch.from_numpy(U).cuda(), dC, prec=EMU)
    return dC.cpu().numpy()


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (129, 65, 16), (300, 200, 50), (1, 1, 1), (257, 191, 64)])
def test_emulated_update_exact_reference(prrp, ctx, m, n, k):
    """Against the product in extended precision: within the derived bound, and far below
    any single-precision split (the worst entry stays under 2^-46 of mrow mcol)."""
    g = pi.rng(m * 31 + n * 7 + k)
    L = g.uniform(-2.0, 2.0, (m, k))
    U = g.standard_normal((k, n)) * np.exp(2.0 * g.standard_normal((1, n)))
    Cm = g.standard_normal((m, n))
    got = _update(prrp, ctx, L, U, Cm)
    exact = Cm.astype(np.longdouble) - L.astype(np.longdouble) @ U.astype(np.longdouble)
    err = np.abs(got.astype(np.longdouble) - exact).astype(np.float64)
    mrow = np.max(np.abs(L), axis=1, keepdims=True)
    mcol = np.max(np.abs(U), axis=0, keepdims=True)
    bound = k * 2.0 ** -50 * mrow * mcol + 2.0 ** -52 * np.abs(got)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert float(np.max(err / (mrow * mcol))) < 2.0 ** -46


@pytest.mark.parametrize("m,n,k", [(8128, 8064, 64), (5000, 31, 16)])
def test_emulated_update_large(prrp, ctx, m, n, k):
    """At the shape of the first update of the n = 8192 factorization: within the derived
    bound plus the FP64 product's own error against numpy's FP64 product."""
    g = pi.rng(m + n + k)
    L = g.uniform(-2.0, 2.0, (m, k))
    U = g.standard_normal((k, n))
    Cm = g.standard_normal((m, n))
    got = _update(prrp, ctx, L, U, Cm)
    want = Cm - L @ U
    S = np.abs(L) @ np.abs(U)
    mrow = np.max(np.abs(L), axis=1, keepdims=True)
    mcol = np.max(np.abs(U), axis=0, keepdims=True)
    bound = k * 2.0 ** -50 * mrow * mcol + k * EPS * S + 2.0 ** -51 * np.abs(want)
    assert np.all(np.abs(got - want) <= bound)


@pytest.mark.parametrize("n,b,seed,split", [(1000, 64, 3, None), (2048, 64, 5, None), (700, 32, 7, None),
                                            (513, 16, 11, None), (2048, 64, 13, (16, 8)), (2048, 64, 17, (8, 4))])
def test_emulated_factor_matches_oracle(prrp, ctx, n, b, seed, split):
    """The whole factorization with the emulated update: the oracle's pivots wherever its
    decisions are untied, the FP64 backward-error bound, the same statistics, and a solve
    without refinement as accurate as the plain FP64 path's on the same matrix.  The
    narrow SM splits put 128 to 256 rows on each panel CTA of the first panels (256: the
    one-lane-per-row form)."""
    A = pi.randn(n, seed)
    dA = torch.from_numpy(A).cuda()
    prrp.prrp_ctx_set_sm_split(ctx, *(split or (0, 0)))
    try:
        F = prrp.prrp_factor(ctx, dA, b=b, prec=EMU)
    finally:
        prrp.prrp_ctx_set_sm_split(ctx, 0, 0)
    st = F.stats()
    perm = F.perm().astype(np.int64)
    B = pi.rhs(n, 2, seed)
    dB = torch.from_numpy(B).cuda()
    prrp.prrp_solve(ctx, F, dB)
    F.close()
    LU = dA.cpu().numpy()
    ref = oracle.lu_prrp(A, b=b)
    assert sorted(perm) == list(range(n))
    assert M.factor_residual(A, LU, perm) <= 64 * n * EPS
    if ref.min_margin > 1e-8:
        assert np.array_equal(perm, ref.perm)
        assert st["swaps"] == ref.swaps
        assert st["growth"] == pytest.approx(ref.growth, rel=1e-9)
    assert st["max_l21"] <= 2.0 * (1 + 1e-12)
    X = dB.cpu().numpy()
    dA64 = torch.from_numpy(A).cuda()
    F64 = prrp.prrp_factor(ctx, dA64, b=b)
    dB64 = torch.from_numpy(B).cuda()
    prrp.prrp_solve(ctx, F64, dB64)
    F64.close()
    X64 = dB64.cpu().numpy()
    for c in range(2):
        e_emu, e64 = M.eta(A, X[:, c], B[:, c]), M.eta(A, X64[:, c], B[:, c])
        assert e_emu <= 3 * e64 + EPS, (e_emu, e64)
        assert e_emu <= 4e-15


def test_emulated_limits(prrp, ctx):
    """Panels wider than 64 (K > 64) are outside the exact split's range: UNSUPPORTED."""
    A = pi.randn(300, 1)
    with pytest.raises(prrp.PrrpError) as e:
        prrp.prrp_factor(ctx, torch.from_numpy(A).cuda(), b=128, prec=EMU)
    assert e.value.name == "PRRP_ERR_UNSUPPORTED"
    L = np.ones((10, 100))
    U = np.ones((100, 10))
    with pytest.raises(prrp.PrrpError) as e:
        _update(prrp, ctx, L, U, np.zeros((10, 10)))
    assert e.value.name == "PRRP_ERR_UNSUPPORTED"
