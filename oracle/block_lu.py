"""Plain FP64 CPU oracle for block parallel and block pairwise LU_PRRP (Section 5, the
algebra of Appendix E): TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

Per panel (columns k0 .. k0+w-1 of the active rows), in the order of Section 5 and
Appendix E:

1. The active rows are cut into P block-rows A_0 .. A_{P-1} (each of at least w + 1
   rows, Appendix E's m/p >= b + 1).
2. A tree of nodes over the blocks.  The strong RRQR of a node's transposed panel columns
   (Algorithm 2) selects w rows, and its permutation acts on the node's rows (Appendix
   E's block-diagonal Pi_0 and the extended Pi_01, Pi_11, ...), so the selected rows take
   the node's first w positions; every other row e of the node is eliminated at once with
   D = (R11^-1 R12)^T (Appendix E's D_i = Rbarbar^T Rbar^-T): its trailing columns become
   A_e - D_e A_sel, its panel columns are no longer used (they store D_e).
   * block parallel LU_PRRP: a binary tree; a leaf's rows are its block, a merge node's
     rows are the first w positions of its left child then of its right child (the
     children's selections); an unpaired node goes up unchanged;
   * block pairwise LU_PRRP: a flat tree; block 0 is the leaf, node i's rows are the first
     w positions of block 0 (the running selection) then all rows of block i.
   The levels run bottom-up, so every elimination uses rows not yet updated in this panel
   (Section 5: "original rows of the active matrix"), and every row is updated once.
3. The root's w rows, now at the top of the active rows, are the pivot rows: GEPP on their
   w x w diagonal block, U12 = L11^-1 Pi_jj^T A12 (Appendix E: "an additional GEPP should
   be performed on this block").

The result is a product of lower triangular factors and U (not a classic L U), so the
record of every elimination is kept for ``block_solve``.  The growth factor g_W is the
largest entry of A and of every updated trailing row, over max|A| (as for LU_PRRP); since
|D| <= tau and a row is updated once per panel, it is at most (1 + tau b)^(n/b)
(Section 5).

Readings where the paper is silent (listed in the design notes): a panel of m active rows
has P' = max(1, min(P, m // (w + 1))) blocks of m // P' rows, the last taking the
remainder; a node's permutation is the product of its strong RRQR's transpositions, in
order, applied to whole rows at the node's positions; D is stored in the eliminated row's
panel columns.  Appendix E's D_11 = Rbarbar_11^T Rbar_01^-T is read as Rbar_11^-T (a typo: each
node's D uses its own R).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.linalg import solve_triangular

from .algorithm import NonFiniteError, SingularError, _gap, strong_rrqr


@dataclass
class BlockNode:
    level: int
    sel: np.ndarray           # original row ids of the selected rows, in selection order
    elim: np.ndarray          # original row ids of the rows eliminated by this node
    D: np.ndarray             # len(elim) x w multipliers: A_e <- A_e - D A_sel


@dataclass
class BlockLUResult:
    LU: np.ndarray            # pivot rows: L11 \ U11 and U12; eliminated rows' panel columns: D
    perm: np.ndarray          # perm[i] = original row at position i (pivot rows in order)
    growth: float             # g_W
    max_D: float              # largest |D| (<= tau)
    swaps: int                # strong RRQR interchanges over every node
    min_margin: float         # smallest decision margin (node QRCP / interchanges, GEPP)
    panels: list = field(default_factory=list)   # per panel: list of BlockNode, bottom-up


def _blocks(m: int, w: int, P: int):
    parts = max(1, min(P, m // (w + 1)))
    q = m // parts
    return [(i * q, m if i == parts - 1 else (i + 1) * q) for i in range(parts)]


def block_lu_prrp(A: np.ndarray, b: int = 16, P: int = 4, tau: float = 2.0, tree: str = "parallel",
                  max_swaps: int | None = None) -> BlockLUResult:
    """Block parallel (tree="parallel", binary tree) or block pairwise (tree="pairwise",
    flat tree) LU_PRRP of the n x n matrix A with panels of b columns and P block-rows."""
    if tree not in ("parallel", "pairwise"):
        raise ValueError("tree must be 'parallel' or 'pairwise'")
    A = np.array(A, dtype=np.float64, copy=True, order="C")
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("square matrix expected")
    if b < 1 or P < 1:
        raise ValueError("need b >= 1 and P >= 1")
    if not np.all(np.isfinite(A)):
        raise NonFiniteError("input has NaN or Inf")
    perm = np.arange(n)
    amax = float(np.max(np.abs(A))) if n else 0.0
    gmax, max_d, swaps = amax, 0.0, 0
    margins: list = []
    panels: list = []
    for k0 in range(0, n, b):
        w = min(b, n - k0)
        m = n - k0
        nodes: list = []

        def node(cpos, level):
            """Strong RRQR of the rows at active positions cpos (k0-relative); its
            transpositions move whole rows, so the selected rows take cpos[:w]; the rows
            left at cpos[w:] are eliminated.  Returns cpos[:w]."""
            nonlocal swaps, gmax, max_d
            cpos = list(cpos)
            B = A[k0 + np.asarray(cpos), k0:k0 + w].T
            pr = strong_rrqr(B, tau, max_swaps, col_offset=k0)
            margins.extend(pr.qrcp_margins + pr.test_margins + pr.choice_margins)
            swaps += pr.swaps
            for (a, c) in pr.transpositions:
                if a != c:
                    ra, rc = k0 + cpos[a], k0 + cpos[c]
                    A[[ra, rc], :] = A[[rc, ra], :]
                    perm[[ra, rc]] = perm[[rc, ra]]
            rs = k0 + np.asarray(cpos[:w])
            re = k0 + np.asarray(cpos[w:], dtype=int)
            D = pr.M.T.copy()
            if len(re):
                A[re, k0 + w:] -= D @ A[rs, k0 + w:]
                A[re, k0:k0 + w] = D
                max_d = max(max_d, float(np.max(np.abs(D))))
                if k0 + w < n:
                    gmax = max(gmax, float(np.max(np.abs(A[re, k0 + w:]))))
            nodes.append(BlockNode(level, perm[rs].copy(), perm[re].copy(), D))
            return cpos[:w]

        blocks = _blocks(m, w, P)
        if tree == "parallel":
            level = [node(range(r0, r1), 0) for r0, r1 in blocks]
            h = 0
            while len(level) > 1:
                h += 1
                nxt = [node(level[i] + level[i + 1], h) for i in range(0, len(level) - 1, 2)]
                if len(level) % 2:
                    nxt.append(level[-1])
                level = nxt
            root = level[0]
        else:
            # the flat tree: block 0 is the only leaf; node i merges the running selection
            # with all rows of block i
            root = node(range(*blocks[0]), 0)
            for i in range(1, len(blocks)):
                root = node(root + list(range(*blocks[i])), i)
        panels.append(nodes)
        assert list(root) == list(range(w))        # the root's rows lead the active rows
        # GEPP on the w x w diagonal block (first maximal |a|), rows moved whole
        for t in range(w):
            col = np.abs(A[k0 + t:k0 + w, k0 + t])
            q = int(np.argmax(col))
            if col[q] == 0.0:
                raise SingularError(k0 + t + 1)
            margins.append(_gap(col, q))
            p = t + q
            if p != t:
                A[[k0 + t, k0 + p], :] = A[[k0 + p, k0 + t], :]
                perm[[k0 + t, k0 + p]] = perm[[k0 + p, k0 + t]]
            r0, r1 = k0 + t + 1, k0 + w
            A[r0:r1, k0 + t] /= A[k0 + t, k0 + t]
            A[r0:r1, k0 + t + 1:k0 + w] -= np.outer(A[r0:r1, k0 + t], A[k0 + t, k0 + t + 1:k0 + w])
        if k0 + w < n:
            L11 = np.tril(A[k0:k0 + w, k0:k0 + w], -1) + np.eye(w)
            A[k0:k0 + w, k0 + w:] = solve_triangular(L11, A[k0:k0 + w, k0 + w:], lower=True,
                                                     unit_diagonal=True)
    return BlockLUResult(LU=A, perm=perm, growth=(gmax / amax if amax > 0 else 1.0), max_D=max_d,
                         swaps=swaps, min_margin=(float(min(margins)) if margins else np.inf),
                         panels=panels)


def block_solve(res: BlockLUResult, rhs: np.ndarray, b: int) -> np.ndarray:
    """x with A x = rhs from the block factorization: every recorded elimination applied to
    the right-hand side in the factorization's order (y_e <- y_e - D_e y_sel, rows by
    original id), the pivot rows' L11^-1 per panel, then back substitution with U."""
    LU, perm = res.LU, res.perm
    n = LU.shape[0]
    y = np.array(rhs, dtype=np.float64, copy=True)
    vec = y.ndim == 1
    if vec:
        y = y[:, None]
    for j, nodes in enumerate(res.panels):
        k0 = j * b
        w = min(b, n - k0)
        for nd in nodes:
            if len(nd.elim):
                y[nd.elim] -= nd.D @ y[nd.sel]
        ids = perm[k0:k0 + w]
        L11 = np.tril(LU[k0:k0 + w, k0:k0 + w], -1) + np.eye(w)
        y[ids] = solve_triangular(L11, y[ids], lower=True, unit_diagonal=True)
    x = solve_triangular(np.triu(LU), y[perm], lower=False)
    return x[:, 0] if vec else x
