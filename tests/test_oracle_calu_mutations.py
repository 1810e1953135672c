"""The CALU_PRRP oracle's pins catch plausible mistakes: each mutant is the oracle's own
source with one planted error (on the CPU, in a private module object); the pins of
test_oracle_calu.py must reject every one while accepting the unmodified source."""
import os
import sys
import types

import numpy as np
import pytest

import oracle
import prrp_inputs as pi
from oracle import metrics as M
from tests.test_oracle_calu import _det_ratio_ok

SRC = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "calu.py")).read()

MUTANTS = {
    "merge_right_then_left": ("node(level[i] + level[i + 1], h)", "node(level[i + 1] + level[i], h)"),
    "odd_node_dropped": ("            if len(level) % 2:\n                nxt.append(level[-1])\n", ""),
    "leaf_skips_a_row": ("r1 = m if i == nleaf - 1 else (i + 1) * leaf_rows",
                         "r1 = m - 1 if i == nleaf - 1 else (i + 1) * leaf_rows"),
    "node_moves_not_applied": ("                    A[[ra, rc], :] = A[[rc, ra], :]\n", ""),
    "l21_from_pivoted_qr": ("R = householder_qr(A[k0:, k0:k0 + w].T)",
                            "R = householder_qr(A[k0:, k0:k0 + w][::-1].T)"),
    "schur_update_sign": ("A[k0 + w:, k0 + w:] -= L21 @", "A[k0 + w:, k0 + w:] += L21 @"),
    "selects_last_candidates": ("            return list(cpos[:w])\n", "            return list(cpos[-w:])\n"),
    "tau_ignored_at_nodes": ("pr = strong_rrqr(B, tau, max_swaps", "pr = strong_rrqr(B, 1e300, max_swaps"),
}


def _load(src):
    src = src.replace("from .algorithm import", "from oracle.algorithm import")
    name = f"calu_mutant_{abs(hash(src))}"
    mod = types.ModuleType(name)
    sys.modules[name] = mod
    exec(compile(src, name, "exec"), mod.__dict__)
    return mod


def _pins_pass(mod) -> bool:
    try:
        for n, b, seed in [(64, 8, 3), (37, 4, 9)]:               # one leaf = LU_PRRP
            A = pi.randn(n, seed)
            r1, r2 = oracle.lu_prrp(A, b=b), mod.calu_prrp(A, b=b, leaf_rows=n)
            if not np.array_equal(r1.perm, r2.perm):
                return False
        for n, b, leaf, seed in [(256, 16, 32, 2), (200, 8, 24, 3)]:   # reconstruction, bounds
            A = pi.randn(n, seed)
            r = mod.calu_prrp(A, b=b, leaf_rows=leaf)
            if M.factor_residual(A, r.LU, r.perm) > 64 * n * 2.0 ** -53:
                return False
            if np.log10(r.growth) > oracle.calu_growth_bound_log10(n, b, 2.0, r.height):
                return False
            if not np.allclose(oracle.selection_multipliers(A, r.perm, b), r.panel_l21, rtol=1e-9):
                return False
        for n, b, leaf, tau, seed in [(12, 2, 3, 1.05, 2), (10, 3, 3, 1.2, 3)]:   # brute force
            r = mod.calu_prrp(pi.randn(n, 70 + seed), b=b, tau=tau, leaf_rows=leaf, keep_nodes=True)
            if not all(_det_ratio_ok(B, list(sel), tau) for _, _, B, sel in r.nodes):
                return False
        for n, b, leaf in [(100, 8, 24), (75, 5, 10)]:            # tree structure
            r = mod.calu_prrp(pi.randn(n, 31), b=b, leaf_rows=leaf, keep_nodes=True)
            for j, k0 in enumerate(range(0, n, b)):
                w, m = min(b, n - k0), n - k0
                mine = [(lv, B) for (pj, lv, B, _) in r.nodes if pj == j]
                leaves = [B for lv, B in mine if lv == 0]
                merges = [B for lv, B in mine if lv > 0]
                if (len(leaves) != max(1, m // leaf) or sum(B.shape[1] for B in leaves) != m
                        or len(merges) != len(leaves) - 1 or any(B.shape != (w, 2 * w) for B in merges)):
                    return False
    except Exception:
        return False
    return True


def test_unmodified_source_passes():
    assert _pins_pass(_load(SRC))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    assert SRC.count(old) == 1, name
    assert not _pins_pass(_load(SRC.replace(old, new)))
