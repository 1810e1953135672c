"""Accuracy metrics and closed forms for LU_PRRP (oracle side).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's CPU
legs, never by the product package.

* ``growth_bound``     g_W <= (1 + tau b)^(n/b) (Section 2.2, end of the induction).
* ``bound_base``       the per-row base (1 + tau b)^(1/b) printed in Table "upper_bound".
* ``flops_lu_prrp``    the operation count of Appendix C, summed per step and in closed form.
* ``hpl``              HPL1, HPL2, HPL3 of Section 2.3.
* ``eta``, ``componentwise``   normwise (1-norm) and componentwise backward errors
                       (eq. "eta" and eq. "comp").
* ``factor_residual``  ||PA - LU||_F / ||A||_F.

Pins (tests/test_oracle_metrics.py): hand-computed exact values, the Rigal-Gaches and
Oettli-Prager perturbations that attain eta and w, and planted-mistake mutants.
"""
from __future__ import annotations

import numpy as np

EPS = 2.0 ** -53     # the unit roundoff the paper's HPL tests divide by


def growth_bound(n: int, b: int, tau: float = 2.0) -> float:
    """(1 + tau b)^(n/b); inf when the value exceeds the double range (e.g. b = 8, n = 2048:
    17^256), where every finite growth factor satisfies it."""
    try:
        return float((1.0 + tau * b) ** (n / b))
    except OverflowError:
        return float("inf")


def bound_base(b: int, tau: float = 2.0) -> float:
    return float((1.0 + tau * b) ** (1.0 / b))


def flops_step(m: int, n: int, b: int, k: int) -> float:
    """Appendix C, step k (1-based): strong RRQR + update + GEPP flops."""
    srrqr = 2.0 * (m - (k - 1) * b) * b * b - 2.0 / 3.0 * b ** 3
    update = 2.0 * b * (m - k * b) * (n - k * b)
    gepp = 2.0 / 3.0 * b ** 3 + (n - k * b) * b * b
    return srrqr + update + gepp


def flops_lu_prrp_sum(m: int, n: int, b: int) -> float:
    return float(sum(flops_step(m, n, b, k) for k in range(1, n // b + 1)))


def flops_lu_prrp_closed(m: int, n: int, b: int) -> float:
    """Closed form of the Appendix C per-step sum (n a multiple of b), summed by hand:
    m n^2 + m n b - n^3/3 - n^2 b/2 + 5 n b^2 / 6; for m = n, 2n^3/3 + n^2 b/2 + 5 n b^2/6."""
    return float(m * n * n + m * n * b - n ** 3 / 3.0 - 0.5 * n * n * b + 5.0 * n * b * b / 6.0)


def flops_lu_prrp_printed(m: int, n: int, b: int) -> float:
    """The closed form as printed in Appendix C, m n^2 + 2 m n b + 2 n b^2 - n^2 b/2 - n^3/3.
    It exceeds the sum of the printed per-step counts by m n b + 7 n b^2 / 6."""
    return float(m * n * n + 2.0 * m * n * b + 2.0 * n * b * b - 0.5 * n * n * b - n ** 3 / 3.0)


def flops_metric(n: int) -> float:
    """The throughput denominator: 2 n^3 / 3."""
    return 2.0 * n ** 3 / 3.0


def factor_residual(A: np.ndarray, LU: np.ndarray, perm: np.ndarray) -> float:
    n = A.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    return float(np.linalg.norm(A[perm] - L @ U) / np.linalg.norm(A))


def norm1(A: np.ndarray) -> float:
    return float(np.max(np.sum(np.abs(A), axis=0))) if A.size else 0.0


def norminf(A: np.ndarray) -> float:
    return float(np.max(np.sum(np.abs(A), axis=1))) if A.size else 0.0


def eta(A, x, b) -> float:
    r = b - A @ x
    return float(np.sum(np.abs(r)) / (norm1(A) * np.sum(np.abs(x)) + np.sum(np.abs(b))))


def componentwise(A, x, b) -> float:
    r = b - A @ x
    den = np.abs(A) @ np.abs(x) + np.abs(b)
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(den > 0, np.abs(r) / den, np.where(r == 0, 0.0, np.inf))
    return float(np.max(q))


def hpl(A, x, b):
    """(HPL1, HPL2, HPL3) for one right-hand side."""
    n = A.shape[0]
    r = np.max(np.abs(b - A @ x))
    return (float(r / (EPS * norm1(A) * n)),
            float(r / (EPS * norm1(A) * np.sum(np.abs(x)))),
            float(r / (EPS * norminf(A) * np.max(np.abs(x)) * n)))


def factor_norms(LU: np.ndarray):
    """(||U||_1, ||U^-1||_1, ||L||_1, ||L^-1||_1) as in the paper's tables."""
    n = LU.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    I = np.eye(n)
    from scipy.linalg import solve_triangular
    Ui = solve_triangular(U, I, lower=False)
    Li = solve_triangular(L, I, lower=True, unit_diagonal=True)
    return norm1(U), norm1(Ui), norm1(L), norm1(Li)
