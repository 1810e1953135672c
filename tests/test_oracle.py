"""Pins for the CPU oracle: each test checks it against something other than itself.

* exact rational brute force on tiny integer matrices (Gram/Cramer determinants, no
  Householder): identical pivots, factors, growth and multipliers;
* strong RRQR stopping condition and swap monotonicity checked by determinants;
* b = 1 reduces to GEPP (LAPACK dgetrf through scipy); tau = inf reduces to QRCP (dgeqp3);
* closed forms: GEPP growth 2^(n-1) on Wilkinson's matrix and (2/3)(2^(n-1)-1) on Foster's;
* the paper's printed values: Table "upper_bound", Table "tab_foster", Appendix C counts;
* invariants at any size: P A = L U, |L21| <= tau, g_W <= (1 + tau b)^(n/b).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import prrp_inputs as pi
from oracle import metrics as M
from tests import exact_prrp as X

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = 2.0 ** -53


def _int_matrix(n, seed, lo=-5, hi=5):
    return pi.rng(seed).integers(lo, hi + 1, size=(n, n))


def _exact_cases():
    cases = []
    for seed in range(150):
        n = 2 + seed % 7
        b = 1 + seed % 3
        tau = [1.05, 1.1, 1.25, 1.5, 2.0][seed % 5]
        cases.append((n, b, tau, seed))
    for seed in range(150, 400):          # small tau, b >= 2: the interchange path
        cases.append((3 + seed % 6, 2 + seed % 2, [1.05, 1.1][seed % 2], seed))
    return cases


def test_exact_brute_force_agreement():
    """Oracle == exact rational LU_PRRP on tiny integer matrices (untied decisions)."""
    checked = with_swaps = 0
    for n, b, tau, seed in _exact_cases():
        A = _int_matrix(n, seed)
        try:
            ex = X.exact_lu_prrp(A.tolist(), b, Fraction(tau))
        except ZeroDivisionError:
            # exactly singular: floating point either meets the zero pivot or rounds it
            # to a pivot at the level of the rounding error.
            try:
                r = oracle.lu_prrp(A.astype(float), b=b, tau=tau)
            except oracle.SingularError:
                continue
            assert np.min(np.abs(np.diag(r.LU))) <= 1e-12 * np.max(np.abs(A))
            continue
        if any(m is not None and m == 0 for _, m in ex["margins"]):
            continue            # a genuine tie: any choice is valid
        r = oracle.lu_prrp(A.astype(float), b=b, tau=tau)
        if r.min_margin < 1e-8:
            continue
        checked += 1
        with_swaps += ex["swaps"] > 0
        assert list(r.perm) == ex["perm"], (n, b, tau, seed)
        assert r.swaps == ex["swaps"]
        LUx = np.array([[float(v) for v in row] for row in ex["LU"]])
        scale = max(1.0, np.max(np.abs(LUx)))
        np.testing.assert_allclose(r.LU, LUx, atol=1e-11 * scale, rtol=0)
        assert abs(r.growth - float(ex["growth"])) <= 1e-11 * float(ex["growth"])
        assert abs(r.growth_u - float(ex["growth_u"])) <= 1e-11 * float(ex["growth_u"])
        assert abs(r.max_L21 - float(ex["max_L21"])) <= 1e-12
    assert checked >= 80
    assert with_swaps >= 5, "the tau-swap path must be exercised"


def test_selection_is_tau_locally_maximal():
    """Each panel's chosen rows satisfy the strong RRQR condition, checked by brute-force
    determinants over every single interchange; the max-|det| subset passes too."""
    for seed in range(25):
        m, w = 4 + seed % 4, 1 + seed % 3
        P = pi.rng(100 + seed).integers(-6, 7, size=(m, w))
        Pf = [[Fraction(int(x)) for x in row] for row in P]
        if X.det([Pf[i] for i in X.max_det_subset(Pf, w)]) == 0:
            continue
        for tau in (1.25, 2.0):
            pr = oracle.strong_rrqr(P.T.astype(float), tau=tau)
            S = [int(i) for i in pr.order[:w]]
            assert X.locally_maximal(Pf, S, Fraction(tau)), (seed, tau)
            # M from R equals B_S^-1 B_rest by Cramer's rule.
            Bs = P.T[:, S].astype(float)
            Bm = P.T[:, pr.order[w:]].astype(float)
            np.testing.assert_allclose(pr.M, np.linalg.solve(Bs, Bm), atol=1e-12, rtol=1e-10)
        assert X.locally_maximal(Pf, X.max_det_subset(Pf, w), Fraction(1))


def test_swaps_grow_det_by_more_than_tau():
    """Every interchange multiplies |det R11| by |M_ij| > tau (Appendix A)."""
    seen = 0
    for seed in range(40):
        B = pi.randn(48, seed, m=6)
        pr = oracle.strong_rrqr(B, tau=1.05)
        for ratio in pr.det_ratios:
            assert ratio > 1.05
            seen += 1
        assert np.max(np.abs(pr.M)) <= 1.05 + 1e-12
    assert seen > 0


def test_b1_is_gepp():
    """b = 1: the panel is one column, QRCP picks its first largest entry, M = a/a_p with
    |M| <= 1, so LU_PRRP is GEPP (LAPACK dgetrf)."""
    for seed in range(6):
        n = 40 + 17 * seed
        A = pi.randn(n, seed)
        r = oracle.lu_prrp(A, b=1, tau=2.0)
        lu, piv = sl.lu_factor(A)
        perm = np.arange(n)
        for i, p in enumerate(piv):
            perm[[i, p]] = perm[[p, i]]
        assert r.min_margin > 1e-8
        assert np.array_equal(r.perm, perm)
        np.testing.assert_allclose(r.LU, lu, atol=1e-12 * n, rtol=0)
        assert r.swaps == 0


def test_tau_inf_is_qrcp():
    """tau = inf: no interchange, the selection is the first w pivots of QRCP (dgeqp3)."""
    for seed in range(8):
        w, p = 4 + seed, 60 + 11 * seed
        B = pi.randn(p, seed, m=w)
        pr = oracle.strong_rrqr(B, tau=np.inf)
        _, _, jpvt = sl.qr(B, mode="economic", pivoting=True)
        assert min(pr.qrcp_margins) > 1e-8
        assert list(pr.order[:w]) == list(jpvt[:w])
        assert pr.swaps == 0


@pytest.mark.parametrize("n", [2, 5, 17, 40, 60])
def test_wilkinson_b1_growth_is_2_pow_n_minus_1(n):
    """GEPP on Wilkinson's matrix grows exactly as 2^(n-1) (Section 2.2)."""
    r = oracle.lu_prrp(pi.wilkinson(n), b=1)
    assert r.growth == 2.0 ** (n - 1)
    assert r.growth_u == 2.0 ** (n - 1)


@pytest.mark.parametrize("n", [3, 10, 30, 50])
def test_foster_b1_growth(n):
    """GEPP on Foster's matrix with c = 1, kh = 2/3 grows as (2/3)(2^(n-1) - 1)."""
    r = oracle.lu_prrp(pi.foster(n), b=1)
    expect = (2.0 / 3.0) * (2.0 ** (n - 1) - 1.0)
    assert abs(r.growth - expect) <= 1e-13 * expect


@pytest.mark.parametrize("b", [16, 64])
def test_wilkinson_blocked_is_stable(b):
    """The matrix on which GEPP grows as 2^2047 factors stably with b >= 16."""
    n = 2048
    A = pi.wilkinson(n)
    r = oracle.lu_prrp(A, b=b, tau=2.0)
    assert M.factor_residual(A, r.LU, r.perm) <= 64 * n * EPS
    assert r.growth <= M.growth_bound(n, b, 2.0)
    assert r.growth < 10.0
    assert r.max_L21 <= 2.0


@pytest.mark.slow
def test_foster_table():
    """Table 'tab_foster': g_W = 2.66 and ||U^-1||_1 = 1.87 for b = 8..128, n = 2048."""
    g = json.load(open(os.path.join(GOLDEN, "foster_n2048.json")))
    A = pi.foster(g["n"], g["c"], g["h"], g["k"])
    for row in g["rows"]:
        r = oracle.lu_prrp(A, b=row["b"], tau=2.0)
        # within one unit of the last printed digit (8/3 is printed 2.66)
        assert abs(r.growth - row["gW"]) <= 0.01, (row, r.growth)
        U = np.triu(r.LU)
        ui1 = M.norm1(sl.solve_triangular(U, np.eye(g["n"])))
        assert abs(ui1 - row["U_inv_1"]) <= 0.01, (row, ui1)
        assert M.factor_residual(A, r.LU, r.perm) <= 64 * g["n"] * EPS


@pytest.mark.slow
def test_wright_table_growth():
    """Table 'tab_wright': g_W = 1 for b = 8..128 at n = 2048, h = 0.3 (both the exact
    exponential and the first-order block the paper displays give it)."""
    g = json.load(open(os.path.join(GOLDEN, "wright_n2048.json")))
    for exact in (True, False):
        A = pi.wright(g["n"], g["h"], exact)
        for row in g["rows"]:
            r = oracle.lu_prrp(A, b=row["b"], tau=2.0)
            assert abs(r.growth - row["gW"]) <= 0.01, (exact, row, r.growth)
            assert M.factor_residual(A, r.LU, r.perm) <= 64 * g["n"] * EPS


@pytest.mark.slow
def test_random_growth_context():
    """Section 2.3: g_W of LU_PRRP on randn(4096) with b = 64 is 'about 19' (statistical:
    one seed, a wide window; the max|U| variant of the definition gives ~55 and fails)."""
    r = oracle.lu_prrp(pi.randn(4096, 0), b=64, tau=2.0)
    assert 10.0 <= r.growth <= 40.0, r.growth
    assert r.growth_u > r.growth


def test_upper_bound_table():
    g = json.load(open(os.path.join(GOLDEN, "upper_bound_table.json")))
    for b, base in g["rows"]:
        # printed to 3 decimals, not always rounded (129^(1/64) = 1.07889 is printed 1.078,
        # 17^(1/8) = 1.42497 is printed 1.425): agreement within one unit of the last digit.
        x = M.bound_base(b, g["tau"])
        assert abs(x - base) < 1e-3, (b, x)


def test_flop_counts():
    """Appendix C: summing the per-step counts (QR 2m'b^2 - 2b^3/3, update 2b(m-kb)(n-kb),
    GEPP 2b^3/3 + (n-kb)b^2) gives m n^2 + m n b - n^3/3 - n^2 b/2 + 5 n b^2/6, checked in
    exact integer arithmetic. The printed closed form exceeds it by m n b + 7 n b^2 / 6 (an
    algebra slip in the paper); both share the 2n^3/3 leading term the metric uses."""
    for m, n, b in [(256, 256, 16), (1024, 1024, 64), (8192, 8192, 64), (96, 96, 8),
                    (300, 96, 8), (4096, 1024, 32)]:
        s = M.flops_lu_prrp_sum(m, n, b)
        c = M.flops_lu_prrp_closed(m, n, b)
        assert s == pytest.approx(c, rel=1e-13)
        exact = sum(Fraction(2 * (m - (k - 1) * b) * b * b) - Fraction(2, 3) * b ** 3
                    + 2 * b * (m - k * b) * (n - k * b) + Fraction(2, 3) * b ** 3
                    + (n - k * b) * b * b for k in range(1, n // b + 1))
        assert exact == (Fraction(m * n * n + m * n * b) - Fraction(n ** 3, 3)
                         - Fraction(n * n * b, 2) + Fraction(5 * n * b * b, 6))
        assert M.flops_lu_prrp_printed(m, n, b) - s == pytest.approx(m * n * b + 7 * n * b * b / 6,
                                                                     rel=1e-9)
    n = 8192
    assert M.flops_lu_prrp_sum(n, n, 64) / M.flops_metric(n) == pytest.approx(1.0, abs=0.02)


@pytest.mark.parametrize("n,b", [(256, 16), (300, 16), (129, 64), (64, 64), (50, 64), (1, 1)])
def test_invariants_random(n, b):
    for seed in range(3):
        A = pi.randn(n, seed)
        r = oracle.lu_prrp(A, b=b, tau=2.0)
        assert M.factor_residual(A, r.LU, r.perm) <= 64 * max(n, 1) * EPS
        assert r.max_L21 <= 2.0
        assert r.growth <= M.growth_bound(n, b, 2.0)
        assert sorted(r.perm) == list(range(n))


def test_l21_equals_a21_a11_inverse():
    """L21 from R (R11^-1 R12)^T equals A21 A11^-1 of the permuted panel (Section 2.1)."""
    A = pi.randn(200, 4)
    w = 16
    pr = oracle.strong_rrqr(A[:, :w].T, tau=2.0)
    P = A[pr.order, :w]
    np.testing.assert_allclose(pr.M.T, P[w:] @ np.linalg.inv(P[:w]), atol=1e-12, rtol=1e-10)


def test_solve_and_refine():
    n = 300
    A = pi.randn(n, 7)
    bv = pi.rhs(n, 1, 7)[:, 0]
    r = oracle.lu_prrp(A, b=16)
    x = oracle.lu_solve(r.LU, r.perm, bv)
    assert M.eta(A, x, bv) < 1e-15
    h1, h2, h3 = M.hpl(A, x, bv)
    assert max(h1, h2, h3) < 16
    x2, hist = oracle.refine(A, r.LU, r.perm, bv, max_iter=5)
    assert hist[-1] <= hist[0]
    np.testing.assert_allclose(x2, np.linalg.solve(A, bv), rtol=1e-9, atol=1e-10)


def test_errors():
    A = pi.randn(20, 1)
    A[3, 4] = np.nan
    with pytest.raises(oracle.NonFiniteError):
        oracle.lu_prrp(A, b=4)
    S = pi.randn(20, 2)
    S[:, 4:8] = 0.0              # the second panel is exactly zero
    with pytest.raises(oracle.SingularError) as e:
        oracle.lu_prrp(S, b=4)
    assert e.value.index == 5
    with pytest.raises(ValueError):
        oracle.strong_rrqr(pi.randn(8, 0, m=2), tau=0.5)
    for seed in range(40):
        B = pi.randn(48, seed, m=6)
        need = oracle.strong_rrqr(B, tau=1.05).swaps
        if need:
            with pytest.raises(oracle.SwapLimitError):
                oracle.strong_rrqr(B, tau=1.05, max_swaps=need - 1)
            break
    else:
        pytest.fail("no case needed an interchange")


def test_max_panels_prefix():
    """Stopping after k panels leaves exactly the first k panels of the full run."""
    A = pi.randn(200, 9)
    full = oracle.lu_prrp(A, b=16)
    part = oracle.lu_prrp(A, b=16, max_panels=3)
    assert part.panels == 3
    assert part.panel_transpositions == full.panel_transpositions[:3]


def test_selection_multipliers_validator():
    """The pivot validator used when a decision is a near-tie: on the oracle's own pivots it
    returns the oracle's block multipliers (<= tau); on a pivot sequence that keeps the
    natural order of a matrix needing pivoting it reports multipliers far above tau."""
    A = pi.randn(200, 11)
    r = oracle.lu_prrp(A, b=16, tau=2.0)
    mx = oracle.selection_multipliers(A, r.perm, 16)
    assert max(mx) == pytest.approx(r.max_L21, rel=1e-9)
    assert max(mx) <= 2.0
    bad = np.arange(200)
    assert max(oracle.selection_multipliers(A, bad, 16)) > 2.0
