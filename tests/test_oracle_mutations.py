"""The oracle's pins catch plausible mistakes: each mutant below is the oracle's own source
with one planted error (on the CPU, in a private module object), and the pin checks must
reject every one of them while accepting the unmodified source."""
import os
import sys
import types
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl

import prrp_inputs as pi
from tests import exact_prrp as X
from tests.test_oracle import _exact_cases, _int_matrix

SRC_PATH = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "algorithm.py")
SRC = open(SRC_PATH).read()

MUTANTS = {
    "qrcp_min_instead_of_max": ("q = int(np.argmax(norms))", "q = int(np.argmin(norms))"),
    "swap_test_never_fires": ("if mu <= tau:", "if mu <= 2 * tau + 1:"),
    "swap_choice_row_major": ('flat = absM.ravel(order="F")', 'flat = absM.ravel(order="C")'),
    "l21_not_transposed_back": ("L21 = pr.M.T\n", "L21 = pr.M.T[::-1]\n"),
    "schur_update_sign": ("A[k0 + w:, k0 + w:] -= L21 @", "A[k0 + w:, k0 + w:] += L21 @"),
    "gepp_no_pivoting": ("            q = int(np.argmax(col))\n", "            q = 0\n"),
    "gepp_forgets_l21_columns": ("                A[k0 + w:, [k0 + t, k0 + p]] = A[k0 + w:, [k0 + p, k0 + t]]\n", ""),
    "gepp_forgets_perm": ("                perm[[k0 + t, k0 + p]] = perm[[k0 + p, k0 + t]]\n", ""),
    "missing_final_l_fixup": ("            A[k0 + w:, k0:k0 + w] = A[k0 + w:, k0:k0 + w] @ L11\n", ""),
    "growth_ignores_schur": ("            gmax = max(gmax, float(np.max(np.abs(A[k0 + w:, k0 + w:]))))\n", ""),
    "householder_drops_beta": ("R[t:, t + 1:] -= beta * np.outer", "R[t:, t + 1:] -= np.outer"),
    "u12_not_solved": ("solve_triangular(L11, A[k0:k0 + w, k0 + w:], lower=True,\n                                                     unit_diagonal=True)",
                       "A[k0:k0 + w, k0 + w:]"),
}


def _load(src):
    name = f"oracle_mutant_{abs(hash(src))}"
    mod = types.ModuleType(name)
    sys.modules[name] = mod          # dataclasses resolve annotations through sys.modules
    exec(compile(src, name, "exec"), mod.__dict__)
    return mod


_EXACT = {}


def _exact(n, b, tau, seed):
    key = (n, b, tau, seed)
    if key not in _EXACT:
        A = _int_matrix(n, seed)
        try:
            _EXACT[key] = X.exact_lu_prrp(A.tolist(), b, Fraction(tau))
        except ZeroDivisionError:
            _EXACT[key] = None
    return _EXACT[key]


def _pins_pass(mod) -> bool:
    """A compact run of the pins of test_oracle.py against module ``mod``."""
    try:
        for n, b, tau, seed in _exact_cases()[::3]:
            ex = _exact(n, b, tau, seed)
            if ex is None or any(m is not None and m == 0 for _, m in ex["margins"]):
                continue
            r = mod.lu_prrp(_int_matrix(n, seed).astype(float), b=b, tau=tau, max_swaps=64)
            if r.min_margin < 1e-8:
                continue
            if list(r.perm) != ex["perm"] or r.swaps != ex["swaps"]:
                return False
            LUx = np.array([[float(v) for v in row] for row in ex["LU"]])
            if np.max(np.abs(r.LU - LUx)) > 1e-11 * max(1.0, np.max(np.abs(LUx))):
                return False
            if abs(r.growth - float(ex["growth"])) > 1e-11 * float(ex["growth"]):
                return False
        for seed in range(2):                       # b = 1 is GEPP
            A = pi.randn(40, seed)
            r = mod.lu_prrp(A, b=1, max_swaps=64)
            lu, _ = sl.lu_factor(A)
            if np.max(np.abs(r.LU - lu)) > 1e-10:
                return False
        A = pi.randn(120, 5)                        # P A = L U at a blocked size
        r = mod.lu_prrp(A, b=16, max_swaps=64)
        L = np.tril(r.LU, -1) + np.eye(120)
        if np.linalg.norm(A[r.perm] - L @ np.triu(r.LU)) > 1e-12 * np.linalg.norm(A) * 120:
            return False
    except Exception:
        return False
    return True


def test_unmodified_source_passes():
    assert _pins_pass(_load(SRC))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    assert SRC.count(old) == 1, f"mutation anchor for {name} not unique in the oracle source"
    assert not _pins_pass(_load(SRC.replace(old, new))), f"pins did not catch {name}"
