"""GPU parity: the CUDA LU_PRRP path (through the C ABI) against the CPU oracle.

Bar:
* pivots: the permutation is identical whenever the oracle's smallest decision margin
  (QRCP top-two gap, swap-test distance to tau, swap-choice gap, GEPP gap) exceeds 1e-8;
  otherwise the GPU's own pivots must be a valid LU_PRRP selection, checked in FP64 on the
  oracle side (every panel's block multipliers |L21| <= tau);
* backward error of the GPU factors ||PA - LU||_F / ||A||_F <= 64 n 2^-53;
* factors element by element (n <= 2048): both sides are backward-stable factorizations of
  the same P A, L U = P A + E with |E| <= gamma_n |L||U| (gamma_n ~ n eps), so they differ
  like factors of a matrix perturbed by |dA| <= 2 gamma_n |L||U|.  To first order
  dL = L stril(L^-1 dA U^-1) and dU = triu(L^-1 dA U^-1) U, which gives the per-entry
  bounds |dL| <= |L| stril(|L^-1| |dA| |U^-1|), |dU| <= triu(|L^-1| |dA| |U^-1|) |U|,
  used with |dA| <= 4 n eps |L||U| (a factor 2 of slack for second-order terms).
"""
import numpy as np
import pytest

import oracle
import prrp_inputs as pi
from oracle import metrics as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


def factor_tolerances(LU):
    """Per-entry first-order bounds on |dL| and |dU| between two backward-stable
    factorizations with the same pivots (see the module docstring)."""
    from scipy.linalg import solve_triangular
    n = LU.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    Li = np.abs(solve_triangular(L, np.eye(n), lower=True, unit_diagonal=True))
    Ui = np.abs(solve_triangular(U, np.eye(n)))
    dA = 4 * n * EPS * (np.abs(L) @ np.abs(U))
    X = Li @ dA @ Ui
    return np.abs(L) @ np.tril(X, -1), np.triu(X) @ np.abs(U)


@pytest.fixture(scope="module")
def prrp():
    import paper_1208_2451_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(prrp):
    c = prrp.prrp_create(0)
    yield c
    c.close()


def gpu_factor(prrp, ctx, A, b, tau=2.0, max_swaps=64):
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    F = prrp.prrp_factor(ctx, dA, b=b, tau=tau, max_swaps=max_swaps)
    torch.cuda.synchronize()
    out = dA.cpu().numpy(), F.perm().astype(np.int64), F.stats()
    F.close()
    return out


def check_parity(prrp, ctx, A, b, tau=2.0, ref=None):
    n = A.shape[0]
    ref = ref if ref is not None else oracle.lu_prrp(A, b=b, tau=tau)
    LU, perm, st = gpu_factor(prrp, ctx, A, b, tau)
    assert sorted(perm) == list(range(n))
    res = M.factor_residual(A, LU, perm) if n else 0.0
    assert res <= 64 * max(n, 1) * EPS, res
    if ref.min_margin > 1e-8:
        assert np.array_equal(perm, ref.perm), "pivot sequence differs with untied decisions"
        if 0 < n <= 2048:
            tL, tU = factor_tolerances(ref.LU)
            dL = np.abs(np.tril(LU, -1) - np.tril(ref.LU, -1))
            dU = np.abs(np.triu(LU) - np.triu(ref.LU))
            assert np.all(dL <= tL + 1e-300), float(np.max(dL - tL))
            assert np.all(dU <= tU + 1e-300), float(np.max(dU - tU))
        assert st["swaps"] == ref.swaps
        assert st["growth"] == pytest.approx(ref.growth, rel=1e-9)
        assert st["growth_u"] == pytest.approx(ref.growth_u, rel=1e-9)
        assert st["max_l21"] == pytest.approx(ref.max_L21, rel=1e-9, abs=1e-300)
    else:
        mx = oracle.selection_multipliers(A, perm, b)
        assert max(mx, default=0.0) <= tau * (1 + 1e-10), "GPU pivots are not a valid selection"
    assert st["max_l21"] <= tau * (1 + 1e-12)
    assert st["growth"] <= M.growth_bound(n, b, tau) if n else True
    return ref, LU, perm, st


@pytest.mark.parametrize("seed", range(10))
def test_small_case_n256_b16(prrp, ctx, seed):
    """The small configuration: n = 256, b = 16, tau = 2, A iid N(0,1)."""
    check_parity(prrp, ctx, pi.randn(256, seed), 16)


@pytest.mark.parametrize("n,b", [(300, 16), (129, 64), (50, 64), (64, 64), (1, 1), (2, 1), (7, 3),
                                 (1000, 64), (513, 32), (200, 128), (77, 8), (640, 128), (33, 1)])
def test_ragged_sizes(prrp, ctx, n, b):
    check_parity(prrp, ctx, pi.randn(n, 1000 + n), b)


@pytest.mark.parametrize("seed", range(4))
def test_swap_path(prrp, ctx, seed):
    """tau close to 1 makes the strong RRQR interchanges fire on random panels."""
    A = pi.randn(256, 50 + seed)
    ref, _, _, st = check_parity(prrp, ctx, A, 16, tau=1.05)
    assert ref.swaps > 0 or ref.min_margin <= 1e-8


def test_empty(prrp, ctx):
    A = torch.empty((0, 0), dtype=torch.float64, device="cuda")
    F = prrp.prrp_factor(ctx, A, b=16)
    assert F.stats()["growth"] == 1.0


@pytest.mark.parametrize("m,w,tau", [(8192, 64, 2.0), (8192, 64, 1.05), (1000, 16, 1.05),
                                     (64, 64, 2.0), (65, 64, 2.0), (3000, 128, 2.0), (17, 5, 1.01)])
def test_panel_select(prrp, ctx, m, w, tau):
    """Rows a1-a3: strong RRQR of one tall panel, element by element against Algorithm 2."""
    P = pi.randn(w, 7 + m, m=m)
    ref = oracle.strong_rrqr(P.T, tau=tau, max_swaps=64)
    order, L21, swaps = prrp.prrp_panel_select(ctx, torch.from_numpy(P).cuda(), tau=tau)
    margins = ref.qrcp_margins + ref.test_margins + ref.choice_margins
    if min(margins, default=np.inf) > 1e-8:
        assert list(order) == list(ref.order)
        assert swaps == ref.swaps
        np.testing.assert_allclose(L21.cpu().numpy(), ref.M.T, atol=1e-10, rtol=1e-9)
    S = order[:w]
    Lx = np.linalg.solve(P[S].T, P[order[w:]].T).T if m > w else np.zeros((0, w))
    np.testing.assert_allclose(L21.cpu().numpy(), Lx, atol=1e-9, rtol=1e-8)
    assert np.max(np.abs(Lx), initial=0) <= tau * (1 + 1e-9)


@pytest.mark.parametrize("m,w,tau,cluster_rows", [(30000, 64, 2.0, 0), (30000, 32, 1.05, 0), (4096, 64, 2.0, 4096),
                                                  (3200, 16, 1.05, 4096), (30400, 16, 2.0, 0)])
def test_panel_select_many_rows(prrp, m, w, tau, cluster_rows):
    """Rows a1-a3 with 198 to 256 rows per CTA, the one-lane-per-row form of the panel
    kernel (grid form, and the cluster form with panels up to 4096 rows)."""
    c = prrp.prrp_create(0)
    try:
        prrp.prrp_ctx_set_panel_mode(c, cluster_rows)
        P = pi.randn(w, 11 + m + w, m=m)
        ref = oracle.strong_rrqr(P.T, tau=tau, max_swaps=64)
        order, L21, swaps = prrp.prrp_panel_select(c, torch.from_numpy(P).cuda(), tau=tau)
    finally:
        c.close()
    margins = ref.qrcp_margins + ref.test_margins + ref.choice_margins
    if min(margins, default=np.inf) > 1e-8:
        assert list(order) == list(ref.order)
        assert swaps == ref.swaps
        np.testing.assert_allclose(L21.cpu().numpy(), ref.M.T, atol=1e-10, rtol=1e-9)
    Lx = np.linalg.solve(P[order[:w]].T, P[order[w:]].T).T
    np.testing.assert_allclose(L21.cpu().numpy(), Lx, atol=1e-9, rtol=1e-8)
    assert np.max(np.abs(Lx)) <= tau * (1 + 1e-9)


def test_factor_cluster_panels_many_rows(prrp):
    """A whole factorization whose first panels run as 16-CTA clusters of up to 256 rows
    per CTA (cluster panels up to 4096 rows, as the serve loop can set)."""
    c = prrp.prrp_create(0)
    try:
        prrp.prrp_ctx_set_panel_mode(c, 4096)
        check_parity(prrp, c, pi.randn(4096, 77), 64)
    finally:
        c.close()


@pytest.mark.parametrize("m,n,k", [(8128, 8128, 64), (1000, 777, 64), (129, 65, 1), (300, 2000, 128),
                                   (64, 64, 100), (1, 1, 16), (5000, 31, 16)])
def test_schur_update(prrp, ctx, m, n, k):
    """Row a5 alone: C -= L U in FP64 against numpy's matmul."""
    g = pi.rng(m * 7 + n)
    L, U, Cm = g.standard_normal((m, k)), g.standard_normal((k, n)), g.standard_normal((m, n))
    dC = torch.from_numpy(Cm).cuda()
    prrp.prrp_schur_update(ctx, torch.from_numpy(L).cuda(), torch.from_numpy(U).cuda(), dC)
    want = Cm - L @ U
    err = np.max(np.abs(dC.cpu().numpy() - want))
    assert err <= 4 * k * EPS * np.max(np.abs(L)) * np.max(np.abs(U)) + 4 * EPS * np.max(np.abs(Cm))


@pytest.mark.parametrize("b", [16, 64])
def test_wilkinson_2048(prrp, ctx, b):
    """GEPP grows as 2^2047 on this matrix; LU_PRRP factors it stably."""
    A = pi.wilkinson(2048)
    _, LU, perm, st = check_parity(prrp, ctx, A, b)
    assert st["growth"] < 10


def test_foster_and_wright_2048(prrp, ctx):
    """Tables tab_foster and tab_wright: g_W = 2.66 and 1 (rows exactly tied: validity path)."""
    _, _, _, st = check_parity(prrp, ctx, pi.foster(2048), 64)
    assert abs(st["growth"] - 2.66) <= 0.01
    _, _, _, st = check_parity(prrp, ctx, pi.wright(2048, 0.3), 64)
    assert abs(st["growth"] - 1.0) <= 0.01


@pytest.mark.parametrize("name", ["foster", "wright", "gen_wilkinson"])
@pytest.mark.parametrize("b", [8, 32, 128])
def test_pathological_suite_2048(prrp, ctx, name, b):
    """Section 2.3 / Appendix F matrices at n = 2048 across panel widths: parity with the
    oracle (pivots, residual, statistics) and the paper's tie-independent growth figures
    (g_W = 2.66 for Foster, Table tab_foster, b from 8 to 128; 1 for Wright, Table
    tab_wright); the generalized Wilkinson matrix (random branch, rank 1) stays under the
    growth bound of Section 2.2."""
    A = {"foster": lambda: pi.foster(2048), "wright": lambda: pi.wright(2048, 0.3),
         "gen_wilkinson": lambda: pi.gen_wilkinson(2048, 1, 3)}[name]()
    _, _, _, st = check_parity(prrp, ctx, A, b)
    if name == "foster":
        assert abs(st["growth"] - 2.66) <= 0.01
    elif name == "wright":
        assert abs(st["growth"] - 1.0) <= 0.01
    else:
        assert st["growth"] <= M.growth_bound(2048, b, 2.0)


def test_full_size_n8192_b64(prrp, ctx):
    """The benchmark configuration (n = 8192, b = 64, tau = 2): whole factorization against
    the oracle, in the same launch configuration bench.py times."""
    A = pi.randn(8192, 0)
    ref = oracle.lu_prrp(A, b=64, tau=2.0)
    check_parity(prrp, ctx, A, 64, ref=ref)


def test_solve_and_refine(prrp, ctx):
    n = 1000
    A = pi.randn(n, 3)
    B = pi.rhs(n, 4, 3)
    dA = torch.from_numpy(A).cuda()
    F = prrp.prrp_factor(ctx, dA, b=64)
    dB = torch.from_numpy(B).cuda()
    info = prrp.prrp_solve(ctx, F, dB, A_orig=torch.from_numpy(A).cuda())
    X = dB.cpu().numpy()
    ref = oracle.lu_prrp(A, b=64)
    Xo = oracle.lu_solve(ref.LU, ref.perm, B)
    np.testing.assert_allclose(X, Xo, rtol=1e-10, atol=1e-11)
    assert info["eta"] <= 1e-15
    for c in range(4):
        assert M.eta(A, X[:, c], B[:, c]) <= 1e-15
    # without refinement: plain substitution
    dB2 = torch.from_numpy(B).cuda()
    info2 = prrp.prrp_solve(ctx, F, dB2)
    np.testing.assert_allclose(dB2.cpu().numpy(), Xo, rtol=1e-10, atol=1e-11)
    assert info2["eta"] == -1.0


@pytest.mark.parametrize("n,nrhs", [(1, 1), (63, 2), (64, 1), (65, 17), (200, 33), (700, 5), (1000, 16),
                                    (2100, 4)])
def test_substitution_shapes(prrp, ctx, n, nrhs):
    """Row a8 without refinement: blocked forward/back substitution with inverted 64 x 64
    diagonal blocks agrees with the oracle's substitution on the oracle's factors, for
    ragged block counts and right-hand-side counts on both sides of the one-launch limit
    (16) and across several staging passes.  The one-launch form takes its row blocks in
    whatever order the CTAs start, yet its arithmetic order is fixed: a second solve gives
    the same bits."""
    A = pi.randn(n, 40 + n)
    B = pi.rhs(n, nrhs, 40 + n)
    F = prrp.prrp_factor(ctx, torch.from_numpy(A).cuda(), b=64)
    dB = torch.from_numpy(B).cuda()
    prrp.prrp_solve(ctx, F, dB)
    dB2 = torch.from_numpy(B).cuda()
    prrp.prrp_solve(ctx, F, dB2)
    F.close()
    assert torch.equal(dB, dB2)
    ref = oracle.lu_prrp(A, b=64)
    Xo = oracle.lu_solve(ref.LU, ref.perm, B)
    np.testing.assert_allclose(dB.cpu().numpy(), Xo, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("n,b,tau", [(2000, 64, 2.0), (1500, 128, 2.0), (900, 32, 1.05)])
def test_cluster_panels_up_to_2048_rows(prrp, n, b, tau):
    """Rows a1-a3 in cluster mode with up to 128 rows per CTA (the serve loop's setting):
    the same parity bar as the default placement, and the same bits as the cooperative grid
    (identical arithmetic, only the exchange differs)."""
    A = pi.randn(n, 600 + n)
    c = prrp.prrp_create(0)
    try:
        prrp.prrp_ctx_set_panel_mode(c, 2048)
        check_parity(prrp, c, A, b, tau=tau)
        LU_c, perm_c, _ = gpu_factor(prrp, c, A, b, tau)
    finally:
        c.close()
    c = prrp.prrp_create(0)
    try:
        LU_g, perm_g, _ = gpu_factor(prrp, c, A, b, tau)
    finally:
        c.close()
    assert np.array_equal(perm_c, perm_g)
    assert np.array_equal(LU_c, LU_g)


def test_launch_timeline_and_panel_mode(prrp):
    """Timing level 2 keeps one (kind, start, end) interval per timed launch; the panel-mode
    knob validates its range."""
    c = prrp.prrp_create(0)
    try:
        A = pi.randn(300, 5)
        prrp.prrp_ctx_set_timing(c, 2)
        F = prrp.prrp_factor(c, torch.from_numpy(A).cuda(), b=64)
        F.close()
        tl = prrp.prrp_ctx_timeline(c)
        kinds = {k for k, _, _ in tl}
        assert {"scan", "panel", "permute", "update", "diag"} <= kinds
        assert all(t1 >= t0 >= 0.0 for _, t0, t1 in tl)
        assert sum(1 for k, _, _ in tl if k == "panel") == 5          # ceil(300 / 64) panels
        prrp.prrp_ctx_set_timing(c, 0)
        assert prrp.prrp_ctx_timeline(c) == []
        with pytest.raises(prrp.PrrpError):
            prrp.prrp_ctx_set_timing(c, 3)
        with pytest.raises(prrp.PrrpError):
            prrp.prrp_ctx_set_panel_mode(c, 5000)
        prrp.prrp_ctx_set_panel_mode(c, 0)
    finally:
        c.close()


def test_gesv_host(prrp, ctx):
    n = 700
    A = pi.randn(n, 8)
    B = pi.rhs(n, 2, 8)
    X, stats, info = prrp.prrp_gesv_host(ctx, A, B, b=64, refine_max_iter=5)
    np.testing.assert_allclose(X, np.linalg.solve(A, B), rtol=1e-9, atol=1e-10)
    assert info["eta"] <= 1e-15


def test_errors(prrp, ctx):
    A = pi.randn(64, 1)
    A[5, 9] = np.nan
    dA = torch.from_numpy(A).cuda()
    with pytest.raises(prrp.PrrpError) as e:
        prrp.prrp_factor(ctx, dA, b=16)
    assert e.value.name == "PRRP_ERR_NONFINITE"
    assert np.array_equal(np.isnan(dA.cpu().numpy()), np.isnan(A))
    assert np.array_equal(dA.cpu().numpy()[~np.isnan(A)], A[~np.isnan(A)]), "input written"
    S = pi.randn(40, 2)
    S[:, 8:16] = 0.0
    F = prrp.prrp_factor(ctx, torch.from_numpy(S).cuda(), b=8, allow=(prrp.binding.PRRP_ERR_SINGULAR,))
    assert F.status == prrp.binding.PRRP_ERR_SINGULAR and F.stats()["info"] == 9
    F.close()
    for kw in ({"b": 0}, {"b": 129}, {"tau": 0.5}, {"max_swaps": -1}):
        with pytest.raises(prrp.PrrpError) as e:
            prrp.prrp_factor(ctx, torch.from_numpy(pi.randn(8, 0)).cuda(), **kw)
        assert e.value.name == "PRRP_ERR_INVALID_ARG"
    # a case that needs interchanges fails cleanly when none are allowed
    A = pi.randn(256, 50)
    need = oracle.lu_prrp(A, b=16, tau=1.05).swaps
    assert need > 0
    with pytest.raises(prrp.PrrpError) as e:
        prrp.prrp_factor(ctx, torch.from_numpy(A).cuda(), b=16, tau=1.05, max_swaps=0)
    assert e.value.name == "PRRP_ERR_SWAP_LIMIT"
    # the context stays usable after every error
    check_parity(prrp, ctx, pi.randn(100, 5), 16)


def test_bounded_wait_times_out(prrp, ctx):
    """A grid barrier that one CTA never reaches gives up and reports PRRP_ERR_TIMEOUT; the
    context then still factors correctly."""
    assert prrp.prrp_selftest_wait(ctx, 20000) == prrp.binding.PRRP_ERR_TIMEOUT
    check_parity(prrp, ctx, pi.randn(128, 9), 16)


def test_solve_modes_agree(prrp, ctx):
    """The two substitution forms (one launch per triangle; one launch per 64-row block)
    compute the same solution up to the order of rounding, for FP64 factors and for the
    FP32 correction solves of a low-precision factorization."""
    n = 1100
    A = pi.randn(n, 46)
    B = pi.rhs(n, 3, 46)
    out = {}
    for prec in (prrp.binding.PRRP_FP64, prrp.binding.PRRP_TF32):
        for mode in (0, 1):
            c = prrp.prrp_create(0)
            try:
                prrp.prrp_ctx_set_solve_mode(c, mode)
                F = prrp.prrp_factor(c, torch.from_numpy(A).cuda(), b=64, prec=prec)
                dB = torch.from_numpy(B).cuda()
                info = prrp.prrp_solve(c, F, dB, A_orig=torch.from_numpy(A).cuda() if prec else None)
                F.close()
            finally:
                c.close()
            out[prec, mode] = dB.cpu().numpy()
            if prec:
                assert info["eta"] <= 1e-15, info
        np.testing.assert_allclose(out[prec, 0], out[prec, 1], rtol=1e-9, atol=1e-10)
    with pytest.raises(prrp.PrrpError):
        prrp.prrp_ctx_set_solve_mode(ctx, 2)


def test_substitution_wait_times_out(prrp, ctx):
    """The one-launch substitution's wait for an earlier row block gives up when that block
    never becomes final, reports PRRP_ERR_TIMEOUT through the host, and the next solve on
    the context is correct."""
    assert prrp.prrp_selftest_chain_wait(ctx, 20000) == prrp.binding.PRRP_ERR_TIMEOUT
    n = 300
    A = pi.randn(n, 44)
    B = pi.rhs(n, 2, 44)
    F = prrp.prrp_factor(ctx, torch.from_numpy(A).cuda(), b=32)
    dB = torch.from_numpy(B).cuda()
    prrp.prrp_solve(ctx, F, dB)
    F.close()
    ref = oracle.lu_prrp(A, b=32)
    np.testing.assert_allclose(dB.cpu().numpy(), oracle.lu_solve(ref.LU, ref.perm, B), rtol=1e-9, atol=1e-10)
