"""Plain FP64 CPU oracle for CALU_PRRP: LU_PRRP whose panel pivots come from tournament
pivoting (Section 3).  TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

Per panel (m rows x w columns), in the order of Section 3.1:

1. Leaves: the panel's rows are cut into contiguous blocks; the strong RRQR of each block's
   transpose (Algorithm 2) selects w candidate rows, and its permutation is applied to the
   block's rows (whole rows of A), so the candidates lead their block.
2. Binary reduction tree: consecutive nodes are merged in pairs.  The node matrix is the left
   node's w candidates followed by the right node's; its strong RRQR selects w rows, and its
   permutation acts on the positions of those 2w rows (the matrices written Pi-bar_i1 and
   Pi-bar_2 in Section 3.1).  The root's selection then sits at the top of the panel.
3. QR without pivoting of the transposed panel, [R11 R12]: L21 = (R11^-1 R12)^T, which is
   A21 A11^-1 for the selected A11 (no longer bounded by tau).
4. As in LU_PRRP (Algorithm 1): A22 -= L21 A12, GEPP on the diagonal block, U12 = L11^-1
   Pi_jj^T A12, and the rows below the block receive L21 Pi_jj L11.

Section 3.2 bounds the growth of the first step by (1 + tau b)^(H+1) and that of the whole
factorization by (1 + tau b)^((n/b)(H+1) - 1), H the height of the reduction tree.

Readings where the paper is silent: a leaf holds at least w rows (a smaller block could not
offer w candidates), so a panel of m rows has max(1, floor(m / leaf_rows)) leaves and the last
one takes the remainder; in a level with an odd number of nodes the last node goes up
unpaired; the height H is the number of merge levels.  With one leaf the tournament is the
strong RRQR of the whole panel and CALU_PRRP is LU_PRRP.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.linalg import solve_triangular

from .algorithm import NonFiniteError, SingularError, _gap, householder_qr, strong_rrqr


@dataclass
class CALUResult:
    LU: np.ndarray            # in-place L\U, P A = L U
    perm: np.ndarray          # perm[i] = original row at position i
    growth: float             # max(|A|, every block Schur complement) / max|A|
    growth_u: float           # max |U| / max |A|
    max_L21: float            # largest |block multiplier| (not bounded by tau here)
    swaps: int                # strong RRQR interchanges over every tree node
    min_margin: float         # smallest decision margin over every pivot choice
    height: int               # largest reduction-tree height over the panels
    first_growth: float       # max |A^(1)| / max |A| after the first panel
    panel_l21: list = field(default_factory=list)   # max |L21| per panel
    nodes: list = field(default_factory=list)   # per node: (panel, level, B = node matrix, selected)


def calu_prrp(A: np.ndarray, b: int = 64, tau: float = 2.0, leaf_rows: int = 256,
              max_swaps: int | None = None, keep_nodes: bool = False) -> CALUResult:
    """CALU_PRRP with a binary reduction tree over leaves of ``leaf_rows`` (>= b) rows."""
    A = np.array(A, dtype=np.float64, copy=True, order="C")
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("square matrix expected")
    if b < 1 or leaf_rows < b:
        raise ValueError("need 1 <= b <= leaf_rows")
    if not np.all(np.isfinite(A)):
        raise NonFiniteError("input has NaN or Inf")
    perm = np.arange(n)
    amax = float(np.max(np.abs(A))) if n else 0.0
    gmax, umax, max_l21, first_growth = amax, 0.0, 0.0, 1.0
    swaps, height = 0, 0
    margins: list = []
    nodes_out: list = []
    panel_l21: list = []

    for k0 in range(0, n, b):
        w = min(b, n - k0)
        m = n - k0

        def node(cpos, level_no):
            """Strong RRQR of the node matrix (the rows at panel positions cpos); its
            transpositions move whole rows, so the selected rows take cpos[:w]."""
            nonlocal swaps
            B = A[k0 + np.asarray(cpos), k0:k0 + w].T.copy()
            pr = strong_rrqr(B, tau, max_swaps, col_offset=k0)
            margins.extend(pr.qrcp_margins + pr.test_margins + pr.choice_margins)
            swaps += pr.swaps
            if keep_nodes:
                nodes_out.append((k0 // b, level_no, B, np.array(pr.order[:w])))
            for (a, c) in pr.transpositions:
                if a != c:
                    ra, rc = k0 + cpos[a], k0 + cpos[c]
                    A[[ra, rc], :] = A[[rc, ra], :]
                    perm[[ra, rc]] = perm[[rc, ra]]
            return list(cpos[:w])

        # 1. leaves
        nleaf = max(1, m // leaf_rows)
        level = []
        for i in range(nleaf):
            r0 = i * leaf_rows
            r1 = m if i == nleaf - 1 else (i + 1) * leaf_rows
            level.append(node(list(range(r0, r1)), 0))
        # 2. binary reduction tree
        h = 0
        while len(level) > 1:
            h += 1
            nxt = [node(level[i] + level[i + 1], h) for i in range(0, len(level) - 1, 2)]
            if len(level) % 2:
                nxt.append(level[-1])
            level = nxt
        height = max(height, h)
        assert level[0] == list(range(w))          # the root's rows lead the panel
        # 3. QR without pivoting of the transposed panel: L21 = (R11^-1 R12)^T
        R = householder_qr(A[k0:, k0:k0 + w].T)
        if np.any(np.diag(R[:, :w]) == 0.0):
            raise SingularError(k0 + int(np.argmin(np.abs(np.diag(R[:, :w])))) + 1)
        L21 = solve_triangular(R[:, :w], R[:, w:], lower=False).T
        A[k0 + w:, k0:k0 + w] = L21
        if L21.size:
            max_l21 = max(max_l21, float(np.max(np.abs(L21))))
            panel_l21.append(float(np.max(np.abs(L21))))
        # 4. as LU_PRRP: Schur update with the unreduced A12, GEPP, U12, final L
        if k0 + w < n:
            A[k0 + w:, k0 + w:] -= L21 @ A[k0:k0 + w, k0 + w:]
            step = float(np.max(np.abs(A[k0 + w:, k0 + w:])))
            gmax = max(gmax, step)
            if k0 == 0 and amax > 0:
                first_growth = max(amax, step) / amax
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
                A[k0 + w:, [k0 + t, k0 + p]] = A[k0 + w:, [k0 + p, k0 + t]]
            r0, r1 = k0 + t + 1, k0 + w
            A[r0:r1, k0 + t] /= A[k0 + t, k0 + t]
            A[r0:r1, k0 + t + 1:k0 + w] -= np.outer(A[r0:r1, k0 + t], A[k0 + t, k0 + t + 1:k0 + w])
        L11 = np.tril(A[k0:k0 + w, k0:k0 + w], -1) + np.eye(w)
        if k0 + w < n:
            A[k0:k0 + w, k0 + w:] = solve_triangular(L11, A[k0:k0 + w, k0 + w:], lower=True,
                                                     unit_diagonal=True)
            A[k0 + w:, k0:k0 + w] = A[k0 + w:, k0:k0 + w] @ L11
        umax = max(umax, float(np.max(np.abs(np.triu(A[k0:k0 + w, k0:])))))

    return CALUResult(LU=A, perm=perm, growth=(gmax / amax if amax > 0 else 1.0),
                      growth_u=(umax / amax if amax > 0 else 1.0), max_L21=max_l21, swaps=swaps,
                      min_margin=(float(min(margins)) if margins else np.inf), height=height,
                      first_growth=first_growth, panel_l21=panel_l21, nodes=nodes_out)


def calu_growth_bound_log10(n: int, b: int, tau: float, height: int) -> float:
    """log10 of (1 + tau b)^((n/b)(H+1) - 1), Section 3.2."""
    return ((n / b) * (height + 1) - 1) * float(np.log10(1.0 + tau * b))
