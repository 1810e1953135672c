"""Pins of the block parallel / block pairwise LU_PRRP oracle (Section 5, Appendix E), by
routes independent of the oracle's own steps:

* P = 1 is LU_PRRP (the one block is the whole panel): the same permutation, U and growth
  as the LU_PRRP oracle, which is pinned by exact arithmetic and the paper's tables;
* a replay of the recorded eliminations from A: every node's D equals A_e A_sel^-1 on the
  panel columns (a linear solve instead of the strong RRQR's back substitution), the
  eliminated rows' panel columns vanish, and the pivot rows' U matches the replayed rows;
* every node's selection is tau-locally maximal, by exact determinants over every single
  interchange (small integer matrices);
* |D| <= tau, and g_W <= (1 + tau b)^(n/b) (Section 5: a row is updated once per panel);
* the product-form solver inverts the factorization: block_solve(A) = I;
* Section 5's observations on random matrices: the block parallel growth rises with P
  once the leaves hold more than 2b rows, and block pairwise LU_PRRP stays below n.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy.linalg import solve_triangular

import oracle
import prrp_inputs as pi
from oracle import metrics as M
from tests import exact_prrp as X

EPS = 2.0 ** -53
TREES = ("parallel", "pairwise")


@pytest.mark.parametrize("tree", TREES)
@pytest.mark.parametrize("n,b", [(64, 8), (200, 16), (130, 32), (97, 5)])
def test_one_block_is_lu_prrp(tree, n, b):
    A = pi.randn(n, 300 + n + b)
    r = oracle.block_lu_prrp(A, b=b, P=1, tree=tree)
    ref = oracle.lu_prrp(A, b=b)
    assert np.array_equal(r.perm, ref.perm)
    assert np.allclose(np.triu(r.LU), np.triu(ref.LU), rtol=1e-12, atol=1e-12 * np.max(np.abs(ref.LU)))
    assert r.growth == pytest.approx(ref.growth, rel=1e-12)


def _replay(A, r, b, tol=1e-9):
    """Apply the recorded eliminations to A (rows by original id) and check each node's D,
    the vanishing panel columns and the pivot rows' U; returns the largest |D|."""
    W = np.array(A, dtype=np.float64, copy=True)
    n = W.shape[0]
    scale = np.max(np.abs(A))
    dmax = 0.0
    for j, nodes in enumerate(r.panels):
        k0 = j * b
        w = min(b, n - k0)
        for nd in nodes:
            if not len(nd.elim):
                continue
            As = W[nd.sel, k0:k0 + w]
            Ae = W[nd.elim, k0:k0 + w]
            Dx = np.linalg.solve(As.T, Ae.T).T
            np.testing.assert_allclose(nd.D, Dx, rtol=tol, atol=tol * max(1.0, float(np.max(np.abs(Dx)))))
            assert np.max(np.abs(Ae - nd.D @ As)) <= 1e3 * w * EPS * scale * max(1.0, np.max(np.abs(nd.D)))
            W[nd.elim, k0 + w:] -= nd.D @ W[nd.sel, k0 + w:]
            W[nd.elim, k0:k0 + w] = 0.0
            dmax = max(dmax, float(np.max(np.abs(nd.D))))
        # the pivot rows: GEPP of their diagonal block, then U12 = L11^-1 (their rows)
        ids = r.perm[k0:k0 + w]
        L11 = np.tril(r.LU[k0:k0 + w, k0:k0 + w], -1) + np.eye(w)
        U11 = np.triu(r.LU[k0:k0 + w, k0:k0 + w])
        np.testing.assert_allclose(L11 @ U11, W[ids, k0:k0 + w], rtol=1e-10, atol=1e-10 * scale)
        if k0 + w < n:
            U12 = solve_triangular(L11, W[ids, k0 + w:], lower=True, unit_diagonal=True)
            np.testing.assert_allclose(r.LU[k0:k0 + w, k0 + w:], U12, rtol=1e-9, atol=1e-9 * scale)
    return dmax


@pytest.mark.parametrize("tree", TREES)
@pytest.mark.parametrize("n,b,P,tau", [(96, 8, 4, 2.0), (150, 16, 3, 1.1), (200, 8, 8, 2.0), (64, 4, 16, 1.05)])
def test_replay_reproduces_the_factorization(tree, n, b, P, tau):
    A = pi.randn(n, 400 + n + P)
    r = oracle.block_lu_prrp(A, b=b, P=P, tau=tau, tree=tree)
    dmax = _replay(A, r, b)
    assert dmax <= tau * (1 + 1e-12)
    assert r.max_D == pytest.approx(dmax, rel=1e-12)
    assert r.growth <= M.growth_bound(n, b, tau)


@pytest.mark.parametrize("tree", TREES)
def test_nodes_are_tau_locally_maximal(tree):
    """Exact determinants over every single interchange of every node (small integer A)."""
    checked = 0
    for seed in range(12):
        n, b, P = 12, 2, 3
        A = pi.rng(700 + seed).integers(-5, 6, size=(n, n)).astype(float)
        try:
            r = oracle.block_lu_prrp(A, b=b, P=P, tau=1.25, tree=tree)
        except oracle.SingularError:
            continue
        W = A.copy()
        for j, nodes in enumerate(r.panels):
            k0 = j * b
            w = min(b, n - k0)
            for nd in nodes:
                rows = list(nd.sel) + list(nd.elim)
                if len(rows) > w:
                    Pf = [[Fraction(float(x)) for x in W[i, k0:k0 + w]] for i in rows]
                    if X.det(Pf[:w]) != 0:
                        assert X.locally_maximal(Pf, list(range(w)), Fraction(1.25) * (1 + Fraction(1, 10 ** 9)))
                        checked += 1
                if len(nd.elim):
                    W[nd.elim, k0 + w:] -= nd.D @ W[nd.sel, k0 + w:]
    assert checked >= 20


@pytest.mark.parametrize("tree", TREES)
@pytest.mark.parametrize("n,b,P", [(80, 8, 4), (123, 16, 5)])
def test_solver_inverts_the_factorization(tree, n, b, P):
    A = pi.randn(n, 500 + n)
    r = oracle.block_lu_prrp(A, b=b, P=P, tree=tree)
    Xs = oracle.block_solve(r, A, b)
    assert np.max(np.abs(Xs - np.eye(n))) <= 1e-8
    rhs = pi.rhs(n, 1, 9)[:, 0]
    x = oracle.block_solve(r, rhs, b)
    assert M.eta(A, x, rhs) <= 1e-13


def _mean_growth(tree, n, b, P, seeds):
    return float(np.mean([oracle.block_lu_prrp(pi.randn(n, 900 + s), b=b, P=P, tree=tree).growth for s in seeds]))


def test_block_parallel_growth_rises_with_p():
    """Section 5 (Figure fig:bluprrp): with leaves of more than 2b rows, the block parallel
    growth factor increases with the number of blocks P."""
    g = [_mean_growth("parallel", 512, 8, P, range(3)) for P in (2, 8, 32)]
    assert g[0] < g[1] < g[2], g


def test_block_pairwise_growth_below_n():
    """Section 5 (Figure fig:fluprrp): the block pairwise growth factor stays below n."""
    for n, b in ((256, 8), (512, 16)):
        for P in (4, 16):
            g = oracle.block_lu_prrp(pi.randn(n, 950 + P), b=b, P=P, tree="pairwise").growth
            assert g < n, (n, b, P, g)
