"""Pins for the oracle's backward-error metrics (Section 2.3: HPL1-HPL3, eq. "eta" and
eq. "comp"), each checked against something other than its own formula:

* hand-computed exact values on a 2 x 2 and a 3 x 3 system (fractions worked out by hand
  below, chosen so that the 1-norm and the infinity-norm of A, x and r all differ);
* Rigal-Gaches: eta is attained by the rank-one perturbation
  dA = (||A||_1 / d) r sign(x)^T, db = -(||b||_1 / d) r with d = ||A||_1 ||x||_1 + ||b||_1,
  which makes x an exact solution of (A + dA) x = b + db, and no feasible perturbation is
  smaller;
* Oettli-Prager: w is attained by dA = D1 |A| D2, db = -D1 |b| with
  D1 = diag(r_i / (|A||x| + |b|)_i) and D2 = diag(sign(x_j)), |dA| <= w |A|, |db| <= w |b|;
* a mutation test: plausible mistakes planted in a copy of the metrics source (and of the
  refinement's own eta) are each caught by these pins.
"""
import os
import sys
import types
from fractions import Fraction

import numpy as np
import pytest

import oracle
import prrp_inputs as pi
from oracle import metrics as M

EPS = 2.0 ** -53
ROOT = os.path.dirname(os.path.dirname(__file__))

# ---- exact cases, worked out by hand -------------------------------------------------
# 2 x 2:  A = [[2, -1], [1, 3]], x = [1, 2], b = [1, 6]
#   A x = [0, 7], r = b - A x = [1, -1]; ||r||_1 = 2, ||r||_inf = 1
#   ||A||_1 = max(3, 4) = 4, ||A||_inf = max(3, 4) = 4, ||x||_1 = 3, ||x||_inf = 2, ||b||_1 = 7
#   eta = 2 / (4*3 + 7) = 2/19
#   |A||x| + |b| = [4 + 1, 7 + 6] = [5, 13]  ->  w = max(1/5, 1/13) = 1/5
#   HPL1 = 1 / (eps 4 2), HPL2 = 1 / (eps 4 3), HPL3 = 1 / (eps 4 2 2)
# 3 x 3:  A = [[1, 2, 0], [0, 1, -3], [4, 0, 2]], x = [1, -1, 2], b = [0, -7, 9]
#   A x = [-1, -7, 8], r = [1, 0, 1]; ||r||_1 = 2, ||r||_inf = 1
#   ||A||_1 = max(5, 3, 5) = 5, ||A||_inf = max(3, 4, 6) = 6, ||x||_1 = 4, ||x||_inf = 2,
#   ||b||_1 = 16
#   eta = 2 / (5*4 + 16) = 1/18
#   |A||x| + |b| = [3 + 0, 7 + 7, 8 + 9] = [3, 14, 17]  ->  w = max(1/3, 0, 1/17) = 1/3
#   HPL1 = 1 / (eps 5 3), HPL2 = 1 / (eps 5 4), HPL3 = 1 / (eps 6 2 3)
EXACT = [
    dict(A=[[2, -1], [1, 3]], x=[1, 2], b=[1, 6],
         eta=Fraction(2, 19), w=Fraction(1, 5), hpl=(Fraction(1, 8), Fraction(1, 12), Fraction(1, 16))),
    dict(A=[[1, 2, 0], [0, 1, -3], [4, 0, 2]], x=[1, -1, 2], b=[0, -7, 9],
         eta=Fraction(1, 18), w=Fraction(1, 3), hpl=(Fraction(1, 15), Fraction(1, 20), Fraction(1, 36))),
]


def _close(got, want, rel=4 * EPS):
    want = float(want)
    return abs(got - want) <= rel * abs(want)


def _random_system(n, seed, noise=1e-6):
    A = pi.randn(n, seed)
    b = pi.rng(seed + 7).standard_normal(n)
    x = np.linalg.solve(A, b) + noise * pi.rng(seed + 11).standard_normal(n)
    return A, x, b


def _exact_pins(mod_metrics, eta_fns) -> bool:
    for c in EXACT:
        A = np.array(c["A"], dtype=np.float64)
        x = np.array(c["x"], dtype=np.float64)
        b = np.array(c["b"], dtype=np.float64)
        for f in eta_fns:
            if not _close(f(A, x, b), c["eta"]):
                return False
        if not _close(mod_metrics.componentwise(A, x, b), c["w"]):
            return False
        h = mod_metrics.hpl(A, x, b)
        for got, want in zip(h, c["hpl"]):
            if not _close(got * EPS, want):
                return False
    return True


def _rigal_gaches(eta_fn, A, x, b) -> bool:
    """eta is attained by the rank-one perturbation and x solves the perturbed system."""
    r = b - A @ x
    nA, nx, nb = M.norm1(A), float(np.sum(np.abs(x))), float(np.sum(np.abs(b)))
    d = nA * nx + nb
    dA = (nA / d) * np.outer(r, np.sign(x))
    db = -(nb / d) * r
    e = eta_fn(A, x, b)
    scale = M.norm1(A) * nx + nb
    if np.max(np.abs((A + dA) @ x - (b + db))) > 64 * EPS * scale:
        return False
    return (_close(M.norm1(dA) / nA, e, 1e-12) and _close(float(np.sum(np.abs(db))) / nb, e, 1e-12))


def _oettli_prager(mod_metrics, A, x, b) -> bool:
    r = b - A @ x
    den = np.abs(A) @ np.abs(x) + np.abs(b)
    d1 = r / den
    dA = (d1[:, None] * np.abs(A)) * np.sign(x)[None, :]
    db = -d1 * np.abs(b)
    w = mod_metrics.componentwise(A, x, b)
    if np.max(np.abs((A + dA) @ x - (b + db))) > 64 * EPS * float(np.max(den)):
        return False
    if not _close(float(np.max(np.abs(d1))), w, 1e-12):
        return False
    return bool(np.all(np.abs(dA) <= w * np.abs(A) * (1 + 1e-12)) and
                np.all(np.abs(db) <= w * np.abs(b) * (1 + 1e-12)))


def _all_pins(mod_metrics, eta_fns) -> bool:
    try:
        if not _exact_pins(mod_metrics, eta_fns):
            return False
        for n, seed in ((5, 1), (40, 2), (64, 3)):
            A, x, b = _random_system(n, seed)
            for f in eta_fns:
                if not _rigal_gaches(f, A, x, b):
                    return False
            if not _oettli_prager(mod_metrics, A, x, b):
                return False
    except Exception:
        return False
    return True


def test_exact_values_by_hand():
    assert _exact_pins(M, [M.eta, oracle.eta])


@pytest.mark.parametrize("n,seed,noise", [(3, 0, 1e-3), (17, 1, 1e-8), (64, 2, 1e-12), (200, 3, 1e-5)])
def test_eta_rigal_gaches(n, seed, noise):
    """The computed eta is the smallest relative perturbation that makes x exact
    (Rigal-Gaches): the rank-one pair attains it, and random feasible pairs never beat it."""
    A, x, b = _random_system(n, seed, noise)
    for f in (M.eta, oracle.eta):
        assert _rigal_gaches(f, A, x, b)
    e = M.eta(A, x, b)
    rng = pi.rng(seed + 99)
    nA, nb = M.norm1(A), float(np.sum(np.abs(b)))
    for _ in range(20):
        dA = rng.standard_normal((n, n)) * rng.uniform(0, 2) * e * nA / n
        db = (A + dA) @ x - b                      # makes (A + dA) x = b + db hold
        eps_pair = max(M.norm1(dA) / nA, float(np.sum(np.abs(db))) / nb)
        assert eps_pair >= e * (1 - 1e-9)


@pytest.mark.parametrize("n,seed", [(4, 5), (30, 6), (128, 7)])
def test_componentwise_oettli_prager(n, seed):
    A, x, b = _random_system(n, seed, 1e-7)
    assert _oettli_prager(M, A, x, b)


def test_componentwise_zero_denominator():
    """A row with |A||x| + |b| = 0 contributes 0 when its residual is 0 (reading: the paper
    leaves 0/0 open) and makes w infinite otherwise (no componentwise perturbation exists)."""
    A = np.array([[0.0, 0.0], [1.0, 2.0]])
    x = np.array([1.0, 1.0])
    assert M.componentwise(A, x, np.array([0.0, 3.0])) == 0.0
    A2 = np.array([[1.0, 0.0], [0.0, 1.0]])
    assert M.componentwise(A2, np.array([0.0, 1.0]), np.array([0.0, 1.0])) == 0.0


def test_hpl_scaling():
    """HPL1-3 are invariant when A and b are scaled by the same power of two (x unchanged),
    and scale as 1/eps: checks the formula's homogeneity, not its text."""
    A, x, b = _random_system(50, 8, 1e-9)
    h = M.hpl(A, x, b)
    h2 = M.hpl(8.0 * A, x, 8.0 * b)
    for u, v in zip(h, h2):
        assert _close(u, v, 1e-12)


def test_the_two_etas_agree():
    """The refinement's stopping test and the metrics module compute the same eta."""
    for n, seed in ((1, 0), (9, 1), (100, 2)):
        A, x, b = _random_system(n, seed, 1e-9)
        assert oracle.eta(A, x, b) == M.eta(A, x, b)


# ---- mutation test ------------------------------------------------------------------
MSRC = open(os.path.join(ROOT, "oracle", "metrics.py")).read()
ASRC = open(os.path.join(ROOT, "oracle", "algorithm.py")).read()

METRIC_MUTANTS = {
    "eta_inf_norm_of_A": ("return float(np.sum(np.abs(r)) / (norm1(A) * np.sum",
                          "return float(np.sum(np.abs(r)) / (norminf(A) * np.sum"),
    "eta_drops_b": ("* np.sum(np.abs(x)) + np.sum(np.abs(b))))", "* np.sum(np.abs(x))))"),
    "eta_inf_norm_of_r": ("return float(np.sum(np.abs(r)) / (norm1(A)", "return float(np.max(np.abs(r)) / (norm1(A)"),
    "comp_drops_b": ("den = np.abs(A) @ np.abs(x) + np.abs(b)", "den = np.abs(A) @ np.abs(x)"),
    "comp_signed_A": ("den = np.abs(A) @ np.abs(x)", "den = np.abs(A @ x)"),
    "hpl1_n_misplaced": ("float(r / (EPS * norm1(A) * n)),", "float(r * n / (EPS * norm1(A))),"),
    "hpl2_inf_norm_of_x": ("float(r / (EPS * norm1(A) * np.sum(np.abs(x)))),",
                           "float(r / (EPS * norm1(A) * np.max(np.abs(x)))),"),
    "hpl3_1_norm_of_A": ("float(r / (EPS * norminf(A) * np.max", "float(r / (EPS * norm1(A) * np.max"),
    "hpl3_drops_n": ("np.max(np.abs(x)) * n)))", "np.max(np.abs(x)))))"),
}
ALG_MUTANTS = {
    "refine_eta_row_sums": ("(np.max(np.sum(np.abs(A), axis=0)) * np.sum(np.abs(x))",
                            "(np.max(np.sum(np.abs(A), axis=1)) * np.sum(np.abs(x))"),
    "refine_eta_drops_b": ("+ np.sum(np.abs(bvec))))", "))"),
}


def _load(src, tag):
    name = f"oracle_{tag}_mutant_{abs(hash(src))}"
    mod = types.ModuleType(name)
    sys.modules[name] = mod
    exec(compile(src, name, "exec"), mod.__dict__)
    return mod


def test_unmodified_metrics_pass():
    assert _all_pins(_load(MSRC, "metrics"), [_load(MSRC, "metrics").eta, _load(ASRC, "alg").eta])


@pytest.mark.parametrize("name", sorted(METRIC_MUTANTS))
def test_metric_mutant_is_caught(name):
    old, new = METRIC_MUTANTS[name]
    assert MSRC.count(old) == 1, f"mutation anchor for {name} not unique"
    mod = _load(MSRC.replace(old, new), "metrics")
    assert not _all_pins(mod, [mod.eta]), f"pins did not catch {name}"


@pytest.mark.parametrize("name", sorted(ALG_MUTANTS))
def test_refinement_eta_mutant_is_caught(name):
    old, new = ALG_MUTANTS[name]
    assert ASRC.count(old) == 1, f"mutation anchor for {name} not unique"
    mod = _load(ASRC.replace(old, new), "alg")
    assert not _all_pins(M, [mod.eta]), f"pins did not catch {name}"
