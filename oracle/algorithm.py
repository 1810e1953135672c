"""Plain FP64 CPU oracle for LU_PRRP (LU factorization with panel rank revealing pivoting).

TEST INFRASTRUCTURE ONLY. This module is the slow, obviously correct restatement of the
paper's method that the CUDA path is checked against. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` (``cpu_baseline`` and
``--impl reference``) may import it; the product package never does, and the two share no
code (the only shared module is ``prrp_inputs``, which builds input matrices).

What it computes, in the paper's order:

* ``strong_rrqr``   Algorithm 2 (Appendix A): QR with column pivoting of B^T's panel, then
                    tau-bounded column interchanges until every |(R11^-1 R12)_ij| <= tau.
* ``lu_prrp``       Algorithm 1 (Section 2.1): for each panel, strong RRQR of its transpose
                    picks b pivot rows, L21 = (R11^-1 R12)^T, the permutation is applied to
                    the whole matrix, A22 -= L21 * A12 (eq. "update"), then GEPP on the b x b
                    diagonal block and U12 = L11^-1 Pi_jj^T A12. The in-place result is the
                    ordinary unit-lower L and upper U with P A = L U, where the rows under
                    each diagonal block carry L21 * Pi_jj * L11 (the decomposition displayed
                    after eq. "update_noperm").
* ``lu_solve``, ``refine``   forward/back substitution and FP64 iterative refinement
                    (Section 2.3 solver tests; Section 3.3 refinement).

Readings where the paper is silent:
  g_W is the largest entry of A and of the block Schur complements A^(k) after each panel
  update, over max|A|: the a^(k)_ij of Section 2.2 are the entries after k block steps,
  whose induction gives (1 + tau b)^(n/b); the diagonal-block GEPP is bounded separately
  there and is reported here as max|U| / max|A|.  This reading reproduces the paper's
  g_W = 1 (Wright), 2.66 (Foster) and about 19 (randn, n = 4096, b = 64).
  QRCP norms are recomputed from scratch at every step, ties go to the first column; the
  swap pair is the largest |M_ij|, ties to the smallest j then smallest i; after a swap the
  unpivoted Householder QR of the permuted B is recomputed; Pi_j is the product of the
  recorded transpositions in order; GEPP takes the first maximal |a|; tau >= 1.

Every decision records its margin (relative gap to the runner-up or to tau) so a
different-but-valid choice by another implementation can be told apart from a wrong one.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.linalg import solve_triangular


class SingularError(ArithmeticError):
    """A zero pivot: the panel (or diagonal block) is rank deficient.

    ``index`` is the LAPACK-style 1-based global column of the first zero pivot."""

    def __init__(self, index: int):
        super().__init__(f"singular at column {index}")
        self.index = index


class SwapLimitError(RuntimeError):
    """Strong RRQR needed more than ``max_swaps`` interchanges on one panel."""


class NonFiniteError(ValueError):
    """NaN or Inf in the input."""


@dataclass
class PanelResult:
    transpositions: list          # [(a, c)] position pairs, applied in order
    order: np.ndarray             # order[i] = original column of B at position i
    M: np.ndarray                 # R11^-1 R12, h x (p-h)
    R: np.ndarray                 # the final R (h x p) of the permuted B
    swaps: int
    qrcp_margins: list = field(default_factory=list)
    test_margins: list = field(default_factory=list)
    choice_margins: list = field(default_factory=list)
    det_ratios: list = field(default_factory=list)   # |det R11| after / before each swap


def _householder(x: np.ndarray):
    """Reflector H = I - beta v v^T with H x = alpha e_1, alpha = -sign(x_1) ||x||."""
    normx = np.sqrt(np.sum(x * x))
    alpha = -normx if x[0] >= 0 else normx
    v = x.copy()
    v[0] -= alpha
    vv = np.sum(v * v)
    beta = 0.0 if vv == 0.0 else 2.0 / vv
    return v, beta, alpha


def householder_qr(B: np.ndarray) -> np.ndarray:
    """R of the unpivoted Householder QR of B (h x p, h <= p), h reflectors."""
    R = np.array(B, dtype=np.float64, copy=True)
    h = R.shape[0]
    for t in range(h):
        v, beta, alpha = _householder(R[t:, t])
        R[t:, t:] -= beta * np.outer(v, v @ R[t:, t:])
        R[t, t] = alpha
        R[t + 1:, t] = 0.0
    return R


def _gap(values: np.ndarray, best: int) -> float:
    """Relative gap between the largest entry (at ``best``) and the runner-up."""
    if values.size < 2:
        return np.inf
    top = values[best]
    rest = np.delete(values, best)
    second = np.max(rest)
    return np.inf if top == 0 else float((top - second) / top)


def qrcp(B: np.ndarray, col_offset: int = 0):
    """Householder QR with column pivoting (Algorithm 2, step 1) of B (h x p, h <= p).

    Step t moves the column of largest 2-norm over rows t..h-1 (recomputed, first index on
    ties) to position t and annihilates it below row t. Returns (R, order, transpositions,
    margins). ``col_offset`` only shifts the column index reported by SingularError."""
    R = np.array(B, dtype=np.float64, copy=True)
    h, p = R.shape
    order = np.arange(p)
    transpositions, margins = [], []
    for t in range(h):
        norms = np.sqrt(np.sum(R[t:, t:] ** 2, axis=0))
        q = int(np.argmax(norms))
        if norms[q] == 0.0:
            raise SingularError(col_offset + t + 1)
        margins.append(_gap(norms, q))
        c = t + q
        transpositions.append((t, c))
        if c != t:
            R[:, [t, c]] = R[:, [c, t]]
            order[[t, c]] = order[[c, t]]
        v, beta, alpha = _householder(R[t:, t])
        R[t:, t + 1:] -= beta * np.outer(v, v @ R[t:, t + 1:])
        R[t, t] = alpha
        R[t + 1:, t] = 0.0
    return R, order, transpositions, margins


def strong_rrqr(B: np.ndarray, tau: float = 2.0, max_swaps: int | None = None,
                col_offset: int = 0) -> PanelResult:
    """Strong RRQR of B (h x p, h <= p), Algorithm 2 of Appendix A.

    QRCP, then while some |(R11^-1 R12)_ij| > tau: interchange selected column i with
    remaining column j (the largest |M_ij|; ties to smallest j, then i) and recompute the QR
    of the permuted B. Each interchange multiplies |det R11| by |M_ij| > tau."""
    if tau < 1.0:
        raise ValueError("tau must be >= 1")
    B = np.asarray(B, dtype=np.float64)
    h, p = B.shape
    R, order, transpositions, qm = qrcp(B, col_offset)
    res = PanelResult(transpositions=transpositions, order=order, M=np.zeros((h, p - h)),
                      R=R, swaps=0, qrcp_margins=qm)
    if p == h:
        return res
    while True:
        M = solve_triangular(R[:, :h], R[:, h:], lower=False)
        absM = np.abs(M)
        flat = absM.ravel(order="F")       # column-major: smallest j first, then i
        k = int(np.argmax(flat))
        i, j = k % h, k // h
        mu = float(flat[k])
        res.test_margins.append(abs(mu - tau) / tau)
        if mu <= tau:
            res.M = M
            res.R = R
            return res
        res.choice_margins.append(_gap(flat, k))
        if max_swaps is not None and res.swaps >= max_swaps:
            raise SwapLimitError(f"panel needs more than {max_swaps} swaps")
        det_before = np.prod(np.abs(np.diag(R[:, :h])))
        order[[i, h + j]] = order[[h + j, i]]
        transpositions.append((i, h + j))
        res.swaps += 1
        R = householder_qr(B[:, order])
        det_after = np.prod(np.abs(np.diag(R[:, :h])))
        res.det_ratios.append(det_after / det_before)


@dataclass
class LUResult:
    LU: np.ndarray            # in-place L\U, row-major n x n
    perm: np.ndarray          # perm[i] = original row at position i: (PA)[i,:] = A[perm[i],:]
    growth: float             # g_W = max(|A|, every block Schur complement) / max|A|
    growth_u: float           # max |U| / max |A| (includes the diagonal-block GEPP)
    max_L21: float            # largest |block multiplier| over all panels (<= tau)
    swaps: int                # strong RRQR interchanges over all panels
    min_margin: float         # smallest decision margin over every pivot choice
    panels: int               # panels processed
    margins: dict = field(default_factory=dict)
    panel_transpositions: list = field(default_factory=list)
    gepp_pivots: list = field(default_factory=list)
    det_ratios: list = field(default_factory=list)


def lu_prrp(A: np.ndarray, b: int = 64, tau: float = 2.0, max_swaps: int | None = None,
            max_panels: int | None = None) -> LUResult:
    """LU_PRRP of the n x n matrix A (Algorithm 1), FP64, returns P A = L U in place.

    ``max_panels`` stops after that many panels (the trailing block is then the Schur
    complement still to be factored); used to time a bounded sample of a large case."""
    A = np.array(A, dtype=np.float64, copy=True, order="C")
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("square matrix expected")
    if b < 1:
        raise ValueError("b must be >= 1")
    if not np.all(np.isfinite(A)):
        raise NonFiniteError("input has NaN or Inf")
    perm = np.arange(n)
    amax = float(np.max(np.abs(A))) if n else 0.0
    gmax = amax          # over A and the block Schur complements A^(k) (Section 2.2)
    umax = 0.0
    max_l21 = 0.0
    swaps = 0
    margins = {"qrcp": [], "test": [], "choice": [], "gepp": []}
    panel_trans, gepp_piv, det_ratios = [], [], []
    panels = 0
    for k0 in range(0, n, b):
        if max_panels is not None and panels >= max_panels:
            break
        w = min(b, n - k0)
        # Alg 1 l.3: strong RRQR of the transposed panel A(k0:n, k0:k0+w)^T.
        B = A[k0:, k0:k0 + w].T
        pr = strong_rrqr(B, tau, max_swaps, col_offset=k0)
        margins["qrcp"] += pr.qrcp_margins
        margins["test"] += pr.test_margins
        margins["choice"] += pr.choice_margins
        det_ratios += pr.det_ratios
        swaps += pr.swaps
        panel_trans.append(list(pr.transpositions))
        # Alg 1 l.5: apply Pi_j^T to whole rows of A (all n columns) and to perm.
        for (a, c) in pr.transpositions:
            if a != c:
                A[[k0 + a, k0 + c], :] = A[[k0 + c, k0 + a], :]
                perm[[k0 + a, k0 + c]] = perm[[k0 + c, k0 + a]]
        # Alg 1 l.4: L21 = (R11^-1 R12)^T, stored under the diagonal block.
        L21 = pr.M.T
        A[k0 + w:, k0:k0 + w] = L21
        if L21.size:
            max_l21 = max(max_l21, float(np.max(np.abs(L21))))
        # Alg 1 l.7 / eq. "update": A22 -= L21 * A12 (A12 not yet reduced by L11).
        if k0 + w < n:
            A[k0 + w:, k0 + w:] -= L21 @ A[k0:k0 + w, k0 + w:]
            gmax = max(gmax, float(np.max(np.abs(A[k0 + w:, k0 + w:]))))
        # Alg 1 l.10: GEPP on the w x w diagonal block; each interchange moves whole rows
        # of A and perm, and the matching columns of L21 (L21 * Pi_jj).
        piv = []
        for t in range(w):
            col = np.abs(A[k0 + t:k0 + w, k0 + t])
            q = int(np.argmax(col))
            if col[q] == 0.0:
                raise SingularError(k0 + t + 1)
            margins["gepp"].append(_gap(col, q))
            p = t + q
            piv.append(p)
            if p != t:
                A[[k0 + t, k0 + p], :] = A[[k0 + p, k0 + t], :]
                perm[[k0 + t, k0 + p]] = perm[[k0 + p, k0 + t]]
                A[k0 + w:, [k0 + t, k0 + p]] = A[k0 + w:, [k0 + p, k0 + t]]
            r0, r1 = k0 + t + 1, k0 + w
            A[r0:r1, k0 + t] /= A[k0 + t, k0 + t]
            A[r0:r1, k0 + t + 1:k0 + w] -= np.outer(A[r0:r1, k0 + t], A[k0 + t, k0 + t + 1:k0 + w])
        gepp_piv.append(piv)
        L11 = np.tril(A[k0:k0 + w, k0:k0 + w], -1) + np.eye(w)
        # Alg 1 l.11: U12 = L11^-1 Pi_jj^T A12 (the rows were interchanged above).
        if k0 + w < n:
            A[k0:k0 + w, k0 + w:] = solve_triangular(L11, A[k0:k0 + w, k0 + w:], lower=True,
                                                     unit_diagonal=True)
            # Final L under the block: L21 * Pi_jj * L11.
            A[k0 + w:, k0:k0 + w] = A[k0 + w:, k0:k0 + w] @ L11
        umax = max(umax, float(np.max(np.abs(np.triu(A[k0:k0 + w, k0:])))))
        panels += 1
    all_m = [m for v in margins.values() for m in v]
    return LUResult(LU=A, perm=perm, growth=(gmax / amax if amax > 0 else 1.0),
                    growth_u=(umax / amax if amax > 0 else 1.0),
                    max_L21=max_l21, swaps=swaps,
                    min_margin=(float(min(all_m)) if all_m else np.inf), panels=panels,
                    margins=margins, panel_transpositions=panel_trans, gepp_pivots=gepp_piv,
                    det_ratios=det_ratios)


def unpack(LU: np.ndarray):
    """Split an in-place L\\U into unit-lower L and upper U."""
    n = LU.shape[0]
    return np.tril(LU, -1) + np.eye(n), np.triu(LU)


def lu_solve(LU: np.ndarray, perm: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = U^-1 L^-1 P B by forward then back substitution."""
    B = np.asarray(B, dtype=np.float64)
    Y = solve_triangular(LU, B[perm], lower=True, unit_diagonal=True)
    return solve_triangular(LU, Y, lower=False)


def eta(A: np.ndarray, x: np.ndarray, bvec: np.ndarray) -> float:
    """Normwise backward error in the 1-norm, eq. (eta): ||r|| / (||A|| ||x|| + ||b||)."""
    r = bvec - A @ x
    return float(np.sum(np.abs(r)) / (np.max(np.sum(np.abs(A), axis=0)) * np.sum(np.abs(x))
                                      + np.sum(np.abs(bvec))))


def refine(A: np.ndarray, LU: np.ndarray, perm: np.ndarray, bvec: np.ndarray,
           max_iter: int = 10, target: float = 2.0 ** -53):
    """FP64 iterative refinement x <- x + (LU)^-1 P (b - A x) (Section 3.3): stops when
    eta <= target, when eta stops halving, or after max_iter corrections.
    Returns (x, eta history)."""
    x = lu_solve(LU, perm, bvec)
    hist = [eta(A, x, bvec)]
    for _ in range(max_iter):
        if hist[-1] <= target:
            break
        r = bvec - A @ x
        x_new = x + lu_solve(LU, perm, r)
        e = eta(A, x_new, bvec)
        if e > hist[-1] / 2:
            if e < hist[-1]:
                x, hist = x_new, hist + [e]
            break
        x, hist = x_new, hist + [e]
    return x, hist


def selection_multipliers(A: np.ndarray, perm: np.ndarray, b: int) -> list:
    """For a permutation produced by some LU_PRRP run, recompute in FP64 each panel's block
    multipliers L21 = A21 A11^-1 (Section 2.1, the product that equals (R11^-1 R12)^T) from
    the row sets it implies: panel j selects rows perm[k0:k0+w] (their order inside the
    block is GEPP's business and does not change L21's row set), and its Schur complement
    is taken with exactly those rows eliminated.  Returns max |L21| per panel, so a
    different-but-valid pivot sequence can be checked against tau."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    S = A[np.asarray(perm)]              # rows in the given final order
    out = []
    for k0 in range(0, n, b):
        w = min(b, n - k0)
        if k0 + w >= n:
            break
        A11 = S[k0:k0 + w, k0:k0 + w]
        A21 = S[k0 + w:, k0:k0 + w]
        L21 = np.linalg.solve(A11.T, A21.T).T
        out.append(float(np.max(np.abs(L21))))
        S[k0 + w:, k0 + w:] -= L21 @ S[k0:k0 + w, k0 + w:]
    return out
