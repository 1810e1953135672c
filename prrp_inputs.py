"""Seeded synthetic inputs for LU_PRRP, shared by the oracle tests, the GPU tests and bench.py.

This module holds no arithmetic of the factorization itself: it only builds test matrices and
right-hand sides from a seed, so the CPU oracle and the CUDA path can be fed identical inputs
without sharing any code.

Matrices (row-major numpy float64, C-contiguous):

* ``randn``            iid N(0,1) entries, the paper's random workload (Section 2.3 and 3.3,
                       ``randn(n,n)`` with a N(0,1) right-hand side).
* ``wilkinson``        1 on the diagonal, -1 strictly below it, 1 in the last column: the matrix
                       on which GEPP grows as 2^(n-1) (Section 2.3, the GEPP-growth form with
                       diag(+-1) = I and T = I).
* ``foster``           the Volterra quadrature matrix of Foster (Section 2.3, parameters c, h, k).
* ``wright``           the multiple-shooting two-point boundary value matrix of Wright
                       (Section 2.3, 2x2 blocks, M = [[-1/6, 1], [1, -1/6]]).
* ``gen_wilkinson``    the generalized Wilkinson matrix of Appendix F (random semi-separable
                       strictly-lower part, unit diagonal, ones in the last column).
* ``conditioned``      Q1 diag(sigma) Q2^T with geometric singular values (cond kappa).
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    """Counter-free PCG64 stream for a seed (numpy's published PCG64 definition)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def randn(n: int, seed: int, m: int | None = None) -> np.ndarray:
    """m x n (default n x n) matrix of iid N(0,1) entries from ``seed``."""
    m = n if m is None else m
    return np.ascontiguousarray(rng(seed).standard_normal((m, n)))


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """n x nrhs right-hand sides, iid N(0,1); stream offset from the matrix seed."""
    return np.ascontiguousarray(rng(seed + 1_000_003).standard_normal((n, nrhs)))


def wilkinson(n: int) -> np.ndarray:
    """1 on the diagonal, -1 strictly below, 1 in the last column."""
    A = -np.tril(np.ones((n, n)), -1) + np.eye(n)
    if n > 0:
        A[:, n - 1] = 1.0
    return np.ascontiguousarray(A)


def foster(n: int, c: float = 1.0, h: float = 1.0, k: float = 2.0 / 3.0) -> np.ndarray:
    """Foster's matrix: first row e_1^T - e_n^T/c; row i>0 has -kh/2 in column 0, -kh in
    columns 1..i-1, 1-kh/2 on the diagonal and -1/c in the last column (which on the last row
    adds to the diagonal: 1 - 1/c - kh/2)."""
    kh = k * h
    A = np.zeros((n, n))
    if n == 0:
        return A
    A[1:, 0] = -kh / 2.0
    for i in range(1, n):
        A[i, 1:i] = -kh
        A[i, i] = 1.0 - kh / 2.0
    A[0, 0] = 1.0
    A[:, n - 1] += -1.0 / c
    if n == 1:
        A[0, 0] = 1.0 - 1.0 / c
    return np.ascontiguousarray(A)


def wright_block(h: float = 0.3, exact: bool = True) -> np.ndarray:
    """The 2x2 block e^{Mh} for M = [[-1/6, 1], [1, -1/6]].

    ``exact``: the matrix exponential, written through the eigen-decomposition of the symmetric
    M (eigenvalues 5/6 on (1,1)/sqrt2 and -7/6 on (1,-1)/sqrt2). Otherwise the first-order form
    I + Mh that the paper displays."""
    if exact:
        ep, em = math.exp(5.0 * h / 6.0), math.exp(-7.0 * h / 6.0)
        return np.array([[(ep + em) / 2, (ep - em) / 2], [(ep - em) / 2, (ep + em) / 2]])
    return np.array([[1.0 - h / 6.0, h], [h, 1.0 - h / 6.0]])


def wright(n: int, h: float = 0.3, exact: bool = True) -> np.ndarray:
    """Wright's block matrix (n even): I on the block diagonal, -e^{Mh} on the block
    subdiagonal, I in the top-right block."""
    if n % 2:
        raise ValueError("Wright matrix needs even n")
    E = wright_block(h, exact)
    A = np.eye(n)
    nb = n // 2
    for i in range(1, nb):
        A[2 * i:2 * i + 2, 2 * (i - 1):2 * i] = -E
    if nb > 1:
        A[0:2, n - 2:n] += np.eye(2)
    return np.ascontiguousarray(A)


def gen_wilkinson(n: int, r: int = 1, seed: int = 0) -> np.ndarray:
    """Generalized Wilkinson matrix of Appendix F (the random branch): a negative random
    rank-r upper-triangular part, each row rescaled so its off-diagonal max is n/(n+1),
    transposed to the strictly lower part, unit diagonal, ones in the last column."""
    g = rng(seed)
    u = g.random((n, r))
    v = g.random((n, r))
    T = -np.triu(u @ v.T)
    for k in range(1, n):
        umax = np.max(np.abs(T[k - 1, k:n])) * (1.0 + 1.0 / n)
        T[k - 1, k:n] /= umax
    T = T - np.diag(np.diag(T))
    A = T.T + np.eye(n)
    A[: n - 1, n - 1] = 1.0
    return np.ascontiguousarray(A)


def conditioned(n: int, kappa: float, seed: int) -> np.ndarray:
    """Q1 diag(sigma) Q2^T with Q from QR of seeded Gaussians and
    sigma_i = kappa^(-(i-1)/(n-1)) (2-norm condition number kappa)."""
    g = rng(seed)
    Q1, _ = np.linalg.qr(g.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(g.standard_normal((n, n)))
    sigma = kappa ** (-np.arange(n) / max(n - 1, 1))
    return np.ascontiguousarray((Q1 * sigma) @ Q2.T)


def batch_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """``count`` integer sizes uniform in [lo, hi] (the uneven-size batch workload)."""
    return rng(seed + 77).integers(lo, hi + 1, size=count).astype(np.int64)


def serve_requests(count: int, rate: float, nlo: int, nhi: int, rhs_hi: int, seed: int):
    """Poisson arrivals at ``rate`` requests/s: (arrival_s, n log-uniform in [nlo, nhi],
    nrhs uniform in 1..rhs_hi) per request."""
    g = rng(seed + 991)
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    ln = g.uniform(math.log(nlo), math.log(nhi + 1), size=count)
    ns = np.minimum(np.floor(np.exp(ln)).astype(np.int64), nhi)
    nr = g.integers(1, rhs_hi + 1, size=count).astype(np.int64)
    return t, ns, nr
