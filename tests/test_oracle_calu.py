"""Pins of the CALU_PRRP oracle (Section 3): what the paper and the mathematics fix, by
routes independent of the oracle's own steps."""
import itertools

import numpy as np
import pytest

import oracle
import prrp_inputs as pi
from oracle import metrics as M

EPS = 2.0 ** -53


@pytest.mark.parametrize("n,b,seed", [(64, 8, 3), (100, 16, 5), (37, 4, 9)])
def test_one_leaf_is_lu_prrp(n, b, seed):
    """With one leaf the tournament is the strong RRQR of the whole panel, so CALU_PRRP is
    LU_PRRP: the same pivots, the same factors up to rounding (L21 comes from an unpivoted QR
    of the permuted panel instead of the pivoted one)."""
    A = pi.randn(n, seed)
    r1 = oracle.lu_prrp(A, b=b)
    r2 = oracle.calu_prrp(A, b=b, leaf_rows=n)
    assert r2.height == 0
    assert np.array_equal(r1.perm, r2.perm)
    assert np.allclose(r1.LU, r2.LU, rtol=1e-10, atol=1e-12 * np.max(np.abs(r1.LU)))
    assert r2.growth == pytest.approx(r1.growth, rel=1e-10)


@pytest.mark.parametrize("n,b,leaf,seed", [(256, 16, 16, 1), (256, 16, 32, 2), (200, 8, 24, 3),
                                           (128, 4, 4, 4)])
def test_reconstructs_within_growth_bounds(n, b, leaf, seed):
    """P A = L U to the backward-error bar; the first step's growth within (1 + tau b)^(H+1)
    and the whole factorization's within (1 + tau b)^((n/b)(H+1) - 1) (Section 3.2)."""
    A = pi.randn(n, seed)
    r = oracle.calu_prrp(A, b=b, leaf_rows=leaf)
    H = r.height
    assert H == int(np.ceil(np.log2(max(1, n // leaf))))
    assert M.factor_residual(A, r.LU, r.perm) <= 64 * n * EPS
    assert np.log10(r.first_growth) <= (H + 1) * np.log10(1 + 2.0 * b)
    assert np.log10(r.growth) <= oracle.calu_growth_bound_log10(n, b, 2.0, H)


@pytest.mark.parametrize("n,b,leaf", [(96, 8, 16), (150, 16, 32)])
def test_multipliers_are_a21_a11_inverse(n, b, leaf):
    """Each panel's block multipliers, recomputed in FP64 as A21 A11^-1 from the row sets the
    final permutation implies (an independent route: a linear solve, no QR), have the
    oracle's largest magnitude; and unlike LU_PRRP they are not bounded by tau."""
    A = pi.randn(n, 17)
    r = oracle.calu_prrp(A, b=b, leaf_rows=leaf)
    again = oracle.selection_multipliers(A, r.perm, b)
    assert np.allclose(again, r.panel_l21, rtol=1e-9)


def _det_ratio_ok(B, sel, tau):
    """Every interchange of a selected column with an unselected one changes |det| of the
    selected w x w block by a factor <= tau (by Cramer's rule that ratio is |M_ij|)."""
    w = B.shape[0]
    base = abs(np.linalg.det(B[:, sel]))
    rest = [j for j in range(B.shape[1]) if j not in set(sel)]
    for i, j in itertools.product(range(w), rest):
        trial = list(sel)
        trial[i] = j
        if abs(np.linalg.det(B[:, trial])) > tau * base * (1 + 1e-9):
            return False
    return True


@pytest.mark.parametrize("n,b,leaf,tau,seed", [(8, 2, 2, 2.0, 1), (12, 2, 3, 1.05, 2), (10, 3, 3, 1.2, 3)])
def test_every_node_is_locally_maximal(n, b, leaf, tau, seed):
    """Brute force on tiny inputs: the selection at every node of every panel's tournament
    is tau-locally maximal among that node's candidates (the strong RRQR condition)."""
    A = pi.randn(n, 70 + seed)
    r = oracle.calu_prrp(A, b=b, tau=tau, leaf_rows=leaf, keep_nodes=True)
    assert r.nodes
    for _, _, B, sel in r.nodes:
        assert _det_ratio_ok(B, list(sel), tau)


def test_singular_panel_raises():
    A = pi.randn(40, 5)
    A[:, 3] = A[:, 2]
    with pytest.raises(oracle.SingularError):
        oracle.calu_prrp(A, b=8, leaf_rows=8)


@pytest.mark.parametrize("n,b,leaf", [(100, 8, 24), (75, 5, 10), (64, 8, 8)])
def test_tree_structure(n, b, leaf):
    """The tournament's shape, from its definition: per panel the leaves partition the panel's
    rows, a binary tree over P leaves has P - 1 merge nodes, and every merge node sees the
    2b candidates of its two children."""
    A = pi.randn(n, 31)
    r = oracle.calu_prrp(A, b=b, leaf_rows=leaf, keep_nodes=True)
    for j, k0 in enumerate(range(0, n, b)):
        w, m = min(b, n - k0), n - k0
        mine = [(lv, B) for (pj, lv, B, _) in r.nodes if pj == j]
        leaves = [B for lv, B in mine if lv == 0]
        merges = [B for lv, B in mine if lv > 0]
        assert len(leaves) == max(1, m // leaf)
        assert sum(B.shape[1] for B in leaves) == m
        assert len(merges) == len(leaves) - 1
        assert all(B.shape == (w, 2 * w) for B in merges)
