"""Exact rational LU_PRRP for tiny integer matrices: the oracle's independent pin.

This restates the same selection rules as the oracle through different mathematics, in
exact arithmetic (``fractions.Fraction``), with no Householder reflector anywhere:

* QR with column pivoting picks, at step t, the panel row farthest from the span of the rows
  already chosen. Its squared distance is det(G(S+q)) / det(G(S)) with G the Gram matrix of
  the panel rows (Gram-Schmidt), which equals the squared remaining column norm that
  Algorithm 2 maximizes.
* M = R11^-1 R12 is computed by Cramer's rule: M_ij = det(P_S with selected row i replaced by
  remaining row j) / det(P_S). It does not depend on how the QR was taken.
* Schur update, GEPP, U12 and the final L are exact rational row operations.

Exact margins (relative gaps) are returned so a test can skip genuinely tied decisions.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import combinations


def det(M):
    """Exact determinant by fraction-valued Gaussian elimination."""
    n = len(M)
    if n == 0:
        return Fraction(1)
    a = [list(r) for r in M]
    d = Fraction(1)
    for c in range(n):
        p = next((r for r in range(c, n) if a[r][c] != 0), None)
        if p is None:
            return Fraction(0)
        if p != c:
            a[c], a[p] = a[p], a[c]
            d = -d
        d *= a[c][c]
        for r in range(c + 1, n):
            f = a[r][c] / a[c][c]
            if f:
                for k in range(c, n):
                    a[r][k] -= f * a[c][k]
    return d


def gram_det(rows):
    return det([[sum(x * y for x, y in zip(u, v)) for v in rows] for u in rows])


def _first_max(vals):
    """Index of the first largest value."""
    k = 0
    for i, v in enumerate(vals):
        if v > vals[k]:
            k = i
    return k


def _rel_gap(best, second):
    if second is None:
        return None
    return (best - second) / best if best != 0 else Fraction(0)


def exact_select(P, w, tau):
    """Panel selection on panel rows P (m lists of w Fractions) with Algorithm 2's rules.

    Returns (transpositions, order, M as w x (m-w) Fractions, margins)."""
    m = len(P)
    order = list(range(m))
    trans, margins = [], []
    chosen = []
    g_prev = Fraction(1)
    for t in range(w):
        ds = [gram_det([P[r] for r in chosen] + [P[order[pos]]]) / g_prev
              for pos in range(t, m)]
        q = _first_max(ds)
        best_pos, best_d = t + q, ds[q]
        second = max((d for i, d in enumerate(ds) if i != q), default=None)
        if best_d == 0:
            raise ZeroDivisionError(f"singular panel at step {t}")
        # margin on the norms (square roots of d), as the oracle measures: monotone in d,
        # so only zero-vs-nonzero matters for tie detection.
        margins.append(("qrcp", _rel_gap(best_d, second)))
        trans.append((t, best_pos))
        order[t], order[best_pos] = order[best_pos], order[t]
        chosen.append(order[t])
        g_prev = gram_det([P[r] for r in chosen])
    swaps = 0
    while True:
        S = [P[order[i]] for i in range(w)]
        dS = det(S)
        M = [[Fraction(0)] * (m - w) for _ in range(w)]
        flat = []                      # column-major: smallest j first, then i
        for j in range(m - w):
            for i in range(w):
                Si = list(S)
                Si[i] = P[order[w + j]]
                M[i][j] = det(Si) / dS
                flat.append((abs(M[i][j]), i, j))
        best = bi = bj = second = None
        if flat:
            k = _first_max([f[0] for f in flat])
            best, bi, bj = flat[k]
            second = max((f[0] for x, f in enumerate(flat) if x != k), default=None)
        if best is None or best <= tau:
            if best is not None:
                margins.append(("test", abs(best - tau) / tau))
            return trans, order, M, margins, swaps
        margins.append(("test", abs(best - tau) / tau))
        margins.append(("choice", _rel_gap(best, second)))
        order[bi], order[w + bj] = order[w + bj], order[bi]
        trans.append((bi, w + bj))
        swaps += 1
        if swaps > 64:
            raise RuntimeError("swap limit")


def exact_lu_prrp(A_int, b, tau):
    """Exact LU_PRRP (Algorithm 1) of a small integer matrix. Returns a dict with the
    in-place L\\U (Fractions), perm, growth, max_L21, swaps and the list of exact margins."""
    tau = Fraction(tau)
    n = len(A_int)
    A = [[Fraction(int(x)) for x in row] for row in A_int]
    perm = list(range(n))
    amax = max(abs(x) for row in A for x in row)
    gmax = amax                 # A and the block Schur complements
    umax = Fraction(0)
    max_l21 = Fraction(0)
    margins = []
    swaps = 0
    for k0 in range(0, n, b):
        w = min(b, n - k0)
        m = n - k0
        P = [A[k0 + i][k0:k0 + w] for i in range(m)]
        trans, order, M, mg, sw = exact_select(P, w, tau)
        margins += mg
        swaps += sw
        for (a, c) in trans:
            A[k0 + a], A[k0 + c] = A[k0 + c], A[k0 + a]
            perm[k0 + a], perm[k0 + c] = perm[k0 + c], perm[k0 + a]
        for j in range(m - w):
            for i in range(w):
                A[k0 + w + j][k0 + i] = M[i][j]
                max_l21 = max(max_l21, abs(M[i][j]))
        for r in range(k0 + w, n):
            for c in range(k0 + w, n):
                A[r][c] -= sum(A[r][k0 + i] * A[k0 + i][c] for i in range(w))
                gmax = max(gmax, abs(A[r][c]))
        # GEPP on the diagonal block with whole-row interchanges and L21 column swaps.
        for t in range(w):
            col = [abs(A[k0 + r][k0 + t]) for r in range(t, w)]
            q = max(range(len(col)), key=lambda i: (col[i], -i))
            best = col[q]
            if best == 0:
                raise ZeroDivisionError(f"singular block at column {k0 + t + 1}")
            rest = [col[i] for i in range(len(col)) if i != q]
            margins.append(("gepp", _rel_gap(best, max(rest)) if rest else None))
            p = t + q
            if p != t:
                A[k0 + t], A[k0 + p] = A[k0 + p], A[k0 + t]
                perm[k0 + t], perm[k0 + p] = perm[k0 + p], perm[k0 + t]
                for r in range(k0 + w, n):
                    A[r][k0 + t], A[r][k0 + p] = A[r][k0 + p], A[r][k0 + t]
            for r in range(k0 + t + 1, k0 + w):
                A[r][k0 + t] /= A[k0 + t][k0 + t]
                for c in range(k0 + t + 1, k0 + w):
                    A[r][c] -= A[r][k0 + t] * A[k0 + t][c]
        L11 = [[(A[k0 + r][k0 + c] if c < r else Fraction(int(c == r))) for c in range(w)]
               for r in range(w)]
        for c in range(k0 + w, n):                 # U12 = L11^-1 A12 (forward substitution)
            for r in range(w):
                A[k0 + r][c] -= sum(L11[r][i] * A[k0 + i][c] for i in range(r))
        for r in range(k0 + w, n):                 # L21 <- L21 * L11
            row = [A[r][k0 + i] for i in range(w)]
            for c in range(w):
                A[r][k0 + c] = sum(row[i] * L11[i][c] for i in range(c, w))
        for r in range(k0, k0 + w):
            for c in range(r, n):
                umax = max(umax, abs(A[r][c]))
    return {"LU": A, "perm": perm, "growth": gmax / amax if amax else Fraction(1),
            "growth_u": umax / amax if amax else Fraction(1),
            "max_L21": max_l21, "swaps": swaps, "margins": margins}


def locally_maximal(P, S, tau):
    """True when no single interchange of a row in S with a row outside it raises
    |det(P_S)| by more than a factor tau (the strong RRQR stopping condition)."""
    tau = Fraction(tau)
    dS = abs(det([P[i] for i in S]))
    rest = [r for r in range(len(P)) if r not in S]
    for i in range(len(S)):
        for j in rest:
            T = list(S)
            T[i] = j
            if abs(det([P[k] for k in T])) > tau * dS:
                return False
    return True


def max_det_subset(P, w):
    """The w-subset of panel rows of largest |det| (brute force over all subsets)."""
    best, best_S = Fraction(-1), None
    for S in combinations(range(len(P)), w):
        d = abs(det([P[i] for i in S]))
        if d > best:
            best, best_S = d, list(S)
    return best_S
