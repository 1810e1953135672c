"""The block LU_PRRP oracle's pins catch plausible mistakes: each mutant is the oracle's
source with one planted error (loaded on the CPU into a private module whose imports
resolve against the real oracle package); the pins must reject every one of them and
accept the unmodified source."""
import os
import sys
import types

import numpy as np
import pytest

import oracle
import prrp_inputs as pi
from tests.test_oracle_block import _replay

SRC_PATH = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "block_lu.py")
SRC = open(SRC_PATH).read()

MUTANTS = {
    "elimination_adds": ("A[re, k0 + w:] -= D @ A[rs, k0 + w:]", "A[re, k0 + w:] += D @ A[rs, k0 + w:]"),
    "d_rows_reversed": ("D = pr.M.T.copy()", "D = pr.M.T.copy()[::-1]"),
    "node_rows_not_moved": ("                if a != c:\n                    ra, rc", "                if False:\n                    ra, rc"),
    "blocks_drop_remainder": ("m if i == parts - 1 else (i + 1) * q", "(i + 1) * q"),
    "u12_not_solved": ("            A[k0:k0 + w, k0 + w:] = solve_triangular(", "            _ = solve_triangular("),
    "gepp_no_pivoting": ("            q = int(np.argmax(col))\n", "            q = 0\n"),
    "binary_tree_drops_unpaired": ("                    nxt.append(level[-1])\n", "                    pass\n"),
    "flat_tree_selection_only": ("root = node(root + list(range(*blocks[i])), i)",
                                 "root = node(root + list(range(*blocks[i]))[:w], i)"),
    "solver_skips_l11": ("        y[ids] = solve_triangular(L11, y[ids], lower=True, unit_diagonal=True)\n", ""),
}


def _load(src):
    name = f"oracle.block_lu_mutant_{abs(hash(src))}"
    mod = types.ModuleType(name)
    mod.__package__ = "oracle"
    sys.modules[name] = mod
    exec(compile(src, name, "exec"), mod.__dict__)
    return mod


def _pins_pass(mod) -> bool:
    try:
        for n, b in ((64, 8), (97, 5)):
            A = pi.randn(n, 300 + n + b)
            ref = oracle.lu_prrp(A, b=b)
            for tree in ("parallel", "pairwise"):
                r = mod.block_lu_prrp(A, b=b, P=1, tree=tree)
                if not np.array_equal(r.perm, ref.perm):
                    return False
                if not np.allclose(np.triu(r.LU), np.triu(ref.LU), rtol=1e-12, atol=1e-12 * np.max(np.abs(ref.LU))):
                    return False
        for tree in ("parallel", "pairwise"):
            for n, b, P in ((96, 8, 4), (150, 16, 3), (93, 8, 5)):
                A = pi.randn(n, 400 + n + P)
                r = mod.block_lu_prrp(A, b=b, P=P, tree=tree)
                _replay(A, r, b)
                if np.max(np.abs(mod.block_solve(r, A, b) - np.eye(n))) > 1e-8:
                    return False
                # the tree shape: the nodes of a panel follow the blocks of Section 5
                blocks = mod._blocks(n, min(b, n), P)
                expect = (2 * len(blocks) - 1) if tree == "parallel" else len(blocks)
                if len(r.panels[0]) != expect:
                    return False
                if tree == "parallel" and len(blocks) > 1:
                    # the first merge node holds the first two leaves' selections
                    first_merge = r.panels[0][len(blocks)]
                    both = set(r.panels[0][0].sel) | set(r.panels[0][1].sel)
                    if set(first_merge.sel) | set(first_merge.elim) != both:
                        return False
    except Exception:
        return False
    return True


def test_unmodified_source_passes():
    assert _pins_pass(_load(SRC))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    assert SRC.count(old) == 1, f"mutation anchor for {name} not unique"
    assert not _pins_pass(_load(SRC.replace(old, new))), f"pins did not catch {name}"
