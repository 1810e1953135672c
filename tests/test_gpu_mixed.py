"""Mixed-precision forms on GB300: the Schur update on tcgen05 tensor cores (TF32, or the
3-term BF16 split with six products), FP64 pivoting, and FP64 iterative refinement of the
solve back to FP64-level backward error.

Error bounds for C -= L U computed this way (per entry, S = sum_k |L_ik| |U_kj|):
* TF32: each operand rounded to 11 significant bits (relative error <= 2^-11), FP32
  accumulation of K terms: |dC| <= (2^-10 + 2^-22 + K 2^-24) S;
* 3 x BF16: each operand represented by hi + mid + lo to 2^-24 relative, the three dropped
  cross products are below 3 * 2^-24, FP32 accumulation of 6K terms:
  |dC| <= (5 * 2^-24 + 6 K 2^-24) S.
"""
import numpy as np
import pytest

import oracle
import prrp_inputs as pi
from oracle import metrics as M

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


def _bound(prec, K, S):
    if prec == 1:    # TF32
        return (2.0 ** -10 + 2.0 ** -22 + K * 2.0 ** -24) * S
    return (5 * 2.0 ** -24 + 6 * K * 2.0 ** -24) * S


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (1000, 777, 64), (129, 65, 16), (300, 2000, 128),
                                   (64, 64, 100), (1, 1, 1), (5000, 31, 16), (8128, 8128, 64)])
def test_schur_update_tensor_cores(prrp, ctx, prec, m, n, k):
    """Row a5 in the low-precision forms against the exact FP64 product."""
    g = pi.rng(m * 13 + n * 7 + k)
    L, U, Cm = g.standard_normal((m, k)), g.standard_normal((k, n)), g.standard_normal((m, n))
    dC = torch.from_numpy(Cm).cuda()
    prrp.prrp_schur_update(ctx, torch.from_numpy(L).cuda(), torch.from_numpy(U).cuda(), dC, prec=prec)
    got = dC.cpu().numpy()
    want = Cm - L @ U
    S = np.abs(L) @ np.abs(U)
    assert np.all(np.abs(got - want) <= _bound(prec, k, S) + 4 * EPS * np.abs(Cm)), \
        float(np.max(np.abs(got - want) / S))
    # the tensor cores really computed something: the error is below the TF32/BF16 input
    # rounding of a single operand, not just the difference of magnitudes
    rel = np.max(np.abs(got - want)) / np.max(S)
    assert rel < (2e-3 if prec == 1 else 1e-5)


@pytest.mark.parametrize("prec", [1, 2])
def test_a7_forms_with_aliased_operand(prrp, ctx, prec):
    """Row a7 in the low-precision modes runs on the tensor-core update in its form
    C -= L U with C aliasing an operand (both operands are split before C is written):
    U12 = X - (I - L11^-1) X and the final multipliers Y L11 = Y - Y (I - L11).  Both agree
    with the FP64 triangular solve / product within the update's error bound."""
    import scipy.linalg as sl
    w, nc, rows = 64, 1000, 777
    g = pi.rng(7000 + prec)
    _, L11, _ = sl.lu(g.standard_normal((w, w)))        # unit lower, |l| <= 1, as from GEPP
    X = g.standard_normal((w, nc))
    Y = g.uniform(-2.0, 2.0, (rows, w))
    E1 = np.eye(w) - np.linalg.inv(L11)
    E2 = np.eye(w) - L11
    dX = torch.from_numpy(X).cuda()
    prrp.prrp_schur_update(ctx, torch.from_numpy(E1).cuda(), dX, dX, prec=prec)
    want = sl.solve_triangular(L11, X, lower=True, unit_diagonal=True)
    S = np.abs(E1) @ np.abs(X)
    err = np.abs(dX.cpu().numpy() - want)
    assert np.all(err <= _bound(prec, w, S) + 64 * EPS * (np.abs(np.linalg.inv(L11)) @ np.abs(X))), \
        float(np.max(err / S))
    dY = torch.from_numpy(Y).cuda()
    prrp.prrp_schur_update(ctx, dY, torch.from_numpy(E2).cuda(), dY, prec=prec)
    want = Y @ L11
    S = np.abs(Y) @ np.abs(E2)
    err = np.abs(dY.cpu().numpy() - want)
    assert np.all(err <= _bound(prec, w, S) + 4 * EPS * (np.abs(Y) @ np.abs(L11))), float(np.max(err / S))


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("r0,c0,ld,n", [(3, 2, 1000, 302), (3, 2, 1000, 301), (1, 1, 1000, 302),
                                        (0, 0, 777, 301), (5, 64, 900, 302), (2, 0, 1000, 302)])
def test_schur_update_inside_larger_matrix(prrp, ctx, prec, r0, c0, ld, n):
    """C as a block of a larger row-major matrix: 16-byte aligned blocks with an even
    leading dimension and column count move through shared memory by TMA, the others
    through registers; either way only the block changes, including along ragged tile
    edges."""
    m, k = 389, 64
    g = pi.rng(r0 * 31 + c0 * 7 + ld)
    L, U = g.standard_normal((m, k)), g.standard_normal((k, n))
    big = g.standard_normal((r0 + m + 7, ld))
    dbig = torch.from_numpy(big).cuda()
    prrp.prrp_schur_update(ctx, torch.from_numpy(L).cuda(), torch.from_numpy(U).cuda(),
                           dbig[r0:r0 + m, c0:c0 + n], prec=prec)
    got = dbig.cpu().numpy()
    want = big.copy()
    want[r0:r0 + m, c0:c0 + n] -= L @ U
    outside = np.ones(big.shape, dtype=bool)
    outside[r0:r0 + m, c0:c0 + n] = False
    assert np.array_equal(got[outside], big[outside])
    S = np.abs(L) @ np.abs(U)
    blk = got[r0:r0 + m, c0:c0 + n]
    assert np.all(np.abs(blk - want[r0:r0 + m, c0:c0 + n]) <= _bound(prec, k, S)
                  + 4 * EPS * np.abs(big[r0:r0 + m, c0:c0 + n]))


def _mixed_solve(prrp, ctx, A, B, prec, b):
    dA = torch.from_numpy(A).cuda()
    F = prrp.prrp_factor(ctx, dA, b=b, prec=prec)
    st = F.stats()
    LU = dA.cpu().numpy()
    perm = F.perm().astype(np.int64)
    dB = torch.from_numpy(B).cuda()
    info = prrp.prrp_solve(ctx, F, dB, A_orig=torch.from_numpy(A).cuda(), refine_max_iter=30)
    F.close()
    return LU, perm, st, dB.cpu().numpy(), info


@pytest.mark.parametrize("nb", [0, 256, 128])
@pytest.mark.parametrize("prec,n,kappa", [(1, 2048, None), (1, 1500, 1e4), (2, 1500, 1e6), (2, 400, 1e8)])
def test_gmres_refinement_reaches_fp64(prrp, ctx, prec, n, kappa, nb):
    """Where the factors' precision times the conditioning leaves classic refinement slow or
    divergent (TF32 on larger random matrices and at kappa = 1e4, where kappa u_TF32 > 1;
    3xBF16 up to kappa = 1e8 at n = 400), refinement continues with GMRES preconditioned by
    the factors and still reaches FP64-level backward error -- with the per-panel update
    (nb = 0) and with the rank-NB aggregated one (blocks of 4 and 2 panels)."""
    A = pi.randn(n, 31) if kappa is None else pi.conditioned(n, kappa, 31)
    B = pi.rhs(n, 3, 31)
    prrp.prrp_ctx_set_update_block(ctx, nb)
    try:
        LU, perm, st, X, info = _mixed_solve(prrp, ctx, A, B, prec, 64)
    finally:
        prrp.prrp_ctx_set_update_block(ctx, 0)
    assert info["eta"] <= 1e-15, info
    for c in range(3):
        assert M.eta(A, X[:, c], B[:, c]) <= 1e-15


def test_gmres_refinement_beyond_reach_keeps_best(prrp, ctx):
    """At kappa = 1e8 and n = 1500 the FP32-accurate factors are too weak a preconditioner
    for restarted GMRES(30) (kappa u_FP32 is about 6): refinement stops after two cycles
    without a new best and returns the best iterate it met, never one worse than the first
    solve, with the reported eta that of the returned X."""
    n = 1500
    A = pi.conditioned(n, 1e8, 31)
    B = pi.rhs(n, 3, 31)
    LU, perm, st, X, info = _mixed_solve(prrp, ctx, A, B, 2, 64)
    assert info["eta"] <= info["eta0"], info
    worst = max(M.eta(A, X[:, c], B[:, c]) for c in range(3))
    assert abs(worst - info["eta"]) <= 1e-3 * info["eta"], (worst, info)


@pytest.mark.parametrize("prec,n,b,kappa", [(2, 256, 16, None), (2, 1024, 64, None), (2, 1000, 64, 1e6),
                                            (1, 1024, 64, 1e2), (1, 700, 32, 1e2)])
def test_mixed_factor_and_refine(prrp, ctx, prec, n, b, kappa):
    """FP64 pivots on a low-precision Schur update, then FP64 refinement: eta <= 1e-15."""
    A = pi.randn(n, 21) if kappa is None else pi.conditioned(n, kappa, 21)
    B = pi.rhs(n, 4, 21)
    LU, perm, st, X, info = _mixed_solve(prrp, ctx, A, B, prec, b)
    assert sorted(perm) == list(range(n))
    res = M.factor_residual(A, LU, perm)
    assert res <= (1e-2 if prec == 1 else 1e-5) * max(1.0, st["growth"]), res
    # the pivots are a valid LU_PRRP selection of the exact matrix up to the update's error
    mx = oracle.selection_multipliers(A, perm, b)
    assert max(mx) <= 2.0 * (1 + (0.5 if prec == 1 else 1e-3)), max(mx)
    assert info["eta"] <= 1e-15, info
    for c in range(B.shape[1]):
        assert M.eta(A, X[:, c], B[:, c]) <= 1e-15


def _factor(prrp, ctx, A, prec, b, tau, nb):
    prrp.prrp_ctx_set_update_block(ctx, nb)
    try:
        dA = torch.from_numpy(A).cuda()
        F = prrp.prrp_factor(ctx, dA, b=b, tau=tau, prec=prec)
        out = dA.cpu().numpy(), F.perm().astype(np.int64), F.stats()
        F.close()
    finally:
        prrp.prrp_ctx_set_update_block(ctx, 0)
    return out


@pytest.mark.parametrize("prec,n,b,nb,tau", [(2, 1024, 64, 256, 2.0), (1, 1024, 64, 256, 2.0), (2, 1000, 64, 128, 2.0),
                                             (2, 900, 16, 256, 1.05), (2, 777, 32, 96, 1.1), (1, 700, 64, 192, 2.0),
                                             (2, 1500, 48, 200, 1.2)])
def test_aggregated_update(prrp, ctx, prec, n, b, nb, tau):
    """The rank-NB form of the update (blocks of floor(nb / b) panels; the columns right of a
    block moved, solved and updated once at the block's end): P A = L U to the mode's
    accuracy, every panel's pivots a valid LU_PRRP selection of the exact A, and, beside the
    per-panel form of the same mode, the same factors to that accuracy wherever both chose
    the same pivots."""
    A = pi.randn(n, 31 + n + b)
    LU, perm, st = _factor(prrp, ctx, A, prec, b, tau, nb)
    assert sorted(perm) == list(range(n))
    tol = 1e-2 if prec == 1 else 1e-5
    res = M.factor_residual(A, LU, perm)
    assert res <= tol * max(1.0, st["growth"]), res
    mx = oracle.selection_multipliers(A, perm, b)
    assert max(mx) <= tau * (1 + (0.5 if prec == 1 else 1e-3)), max(mx)
    assert st["max_l21"] <= tau * (1 + 1e-12)
    LU1, perm1, st1 = _factor(prrp, ctx, A, prec, b, tau, 0)
    assert M.factor_residual(A, LU1, perm1) <= tol * max(1.0, st1["growth"])
    if np.array_equal(perm, perm1):
        scale = float(np.max(np.abs(LU1)))
        assert np.max(np.abs(LU - LU1)) <= 50 * tol * scale, float(np.max(np.abs(LU - LU1)) / scale)
        assert st["growth"] == pytest.approx(st1["growth"], rel=0.5)


def test_aggregated_update_refines_to_fp64(prrp, ctx):
    """A factorization of several blocks from the rank-NB form preconditions FP64
    refinement to eta <= 1e-15, like the per-panel form."""
    n, b = 1200, 64
    A = pi.conditioned(n, 1e4, 33)
    B = pi.rhs(n, 2, 33)
    prrp.prrp_ctx_set_update_block(ctx, 256)
    try:
        LU, perm, st, X, info = _mixed_solve(prrp, ctx, A, B, 2, b)
    finally:
        prrp.prrp_ctx_set_update_block(ctx, 0)
    assert info["eta"] <= 1e-15, info
    for c in range(B.shape[1]):
        assert M.eta(A, X[:, c], B[:, c]) <= 1e-15


def test_update_block_limits(prrp, ctx):
    for bad in (-1, 257):
        with pytest.raises(prrp.PrrpError) as e:
            prrp.prrp_ctx_set_update_block(ctx, bad)
        assert e.value.name == "PRRP_ERR_INVALID_ARG"
    prrp.prrp_ctx_set_update_block(ctx, 0)


@pytest.mark.parametrize("prec", [1, 2])
def test_sm_split_changes_no_result(prrp, ctx, prec):
    """The SM split is a tuning knob: every tile of the update and every panel compute the
    same arithmetic whichever CTAs run them, so the factors are bit-identical."""
    n, b = 1536, 64
    A = pi.randn(n, 41)
    outs = []
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for split in ((0, 0), (40, 8), (96, 16), (sms, 0)):          # (sms, 0): no split
        prrp.prrp_ctx_set_sm_split(ctx, *split)
        try:
            dA = torch.from_numpy(A).cuda()
            F = prrp.prrp_factor(ctx, dA, b=b, prec=prec)
            outs.append((dA.cpu().numpy(), F.perm().astype(np.int64)))
            F.close()
        finally:
            prrp.prrp_ctx_set_sm_split(ctx, 0, 0)
    for LU, perm in outs[1:]:
        assert np.array_equal(perm, outs[0][1])
        assert np.array_equal(LU, outs[0][0])
