"""Batched solves (prrp_batch_solve) on GB300 against the oracle.

* FP64 form: the whole of Algorithm 1 runs per system in one CTA in FP64, so pivots must
  equal the oracle's wherever its decision margins exceed 1e-8 (otherwise the GPU's
  selection must be valid: every panel's |L21| <= tau, recomputed in FP64).
* FP32 form (FP32 working copy and Schur update, FP64 pivot selection and refinement):
  pivots are a valid selection of the exact matrix up to the FP32 update error, and the
  refined solutions reach FP64-level normwise backward error, eta <= 1e-15.
* Each system is computed by one CTA independently of the others, so a system gives the
  same bits alone and inside any batch.
"""
import numpy as np
import pytest

import oracle
import prrp_inputs as pi
from oracle import metrics as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prrp():
    import paper_1208_2451_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(prrp):
    c = prrp.prrp_create(0)
    yield c
    c.close()


def _systems(sizes, seed, nrhs=1):
    As = [pi.randn(int(n), seed + i) for i, n in enumerate(sizes)]
    Bs = [pi.rhs(int(n), nrhs, seed + i) for i, n in enumerate(sizes)]
    return As, Bs


def _run(prrp, ctx, As, Bs, prec, b=16, tau=2.0, refine=10):
    dA = [torch.from_numpy(A).cuda() for A in As]
    dB = [torch.from_numpy(B).cuda() for B in Bs]
    dP = [torch.empty(A.shape[0], dtype=torch.int32, device="cuda") for A in As]
    st, info = prrp.prrp_batch_solve(ctx, dA, dB, b=b, tau=tau, prec=prec, refine_max_iter=refine,
                                     perms=dP)
    torch.cuda.synchronize()
    return st, info, [x.cpu().numpy() for x in dB], [p.cpu().numpy().astype(np.int64) for p in dP]


@pytest.mark.parametrize("sizes,seed", [([32, 47, 64, 100, 129, 200, 256, 300], 500),
                                        ([512, 1024, 511, 777], 510)])
def test_fp64_batch_pivots_match_oracle(prrp, ctx, sizes, seed):
    """FP64 batched factors: the oracle's pivots where its decisions are untied (sizes up to
    the kernel's limit, n = 1024), else a valid selection; refined to eta <= 1e-15."""
    As, Bs = _systems(sizes, seed)
    st, info, X, P = _run(prrp, ctx, As, Bs, prec=0)
    assert all(s == 0 for s in st)
    for A, B, x, p in zip(As, Bs, X, P):
        ref = oracle.lu_prrp(A, b=16, tau=2.0)
        if ref.min_margin > 1e-8:
            assert np.array_equal(p, ref.perm)
        else:
            assert max(oracle.selection_multipliers(A, p, 16)) <= 2.0 * (1 + 1e-10)
        assert M.eta(A, x[:, 0], B[:, 0]) <= 1e-15


def test_fp32_batch_valid_and_refined(prrp, ctx):
    sizes = list(pi.batch_sizes(64, 32, 512, 3))
    As, Bs = _systems(sizes, 900)
    st, info, X, P = _run(prrp, ctx, As, Bs, prec=3)
    assert all(s == 0 for s in st), st
    for A, B, x, p, inf in zip(As, Bs, X, P, info):
        assert sorted(p) == list(range(A.shape[0]))
        assert max(oracle.selection_multipliers(A, p, 16)) <= 2.0 * (1 + 1e-3)
        assert M.eta(A, x[:, 0], B[:, 0]) <= 1e-15
        assert inf["eta"] <= 1e-15 and inf["eta0"] > inf["eta"] * 0.999


def test_batch_multiple_rhs_and_tau_swaps(prrp, ctx):
    sizes = [40, 96, 250]
    As, _ = _systems(sizes, 77)
    Bs = [pi.rhs(A.shape[0], k, 3) for A, k in zip(As, (1, 4, 16))]
    st, info, X, P = _run(prrp, ctx, As, Bs, prec=0, tau=1.05)
    assert all(s == 0 for s in st)
    for A, B, x, p in zip(As, Bs, X, P):
        ref = oracle.lu_prrp(A, b=16, tau=1.05)
        assert ref.swaps > 0
        if ref.min_margin > 1e-8:
            assert np.array_equal(p, ref.perm)
        for c in range(B.shape[1]):
            assert M.eta(A, x[:, c], B[:, c]) <= 1e-15


def test_batch_per_system_failures(prrp, ctx):
    good, sing, bad = pi.randn(64, 1), pi.randn(64, 2), pi.randn(64, 3)
    sing[:, 16:32] = 0.0
    bad[3, 7] = np.inf
    Bs = [pi.rhs(64, 1, k) for k in range(3)]
    st, info, X, _ = _run(prrp, ctx, [good, sing, bad], Bs, prec=3)
    assert st[0] == 0 and st[1] == prrp.binding.PRRP_ERR_SINGULAR
    assert st[2] == prrp.binding.PRRP_ERR_NONFINITE
    assert M.eta(good, X[0][:, 0], Bs[0][:, 0]) <= 1e-15


def test_batch_result_same_alone_and_in_mix(prrp, ctx):
    """Per-system determinism: identical bits alone, in a small mix and in a large mix."""
    target = pi.randn(200, 4242)
    bt = pi.rhs(200, 2, 4242)
    alone = _run(prrp, ctx, [target], [bt], prec=3)[2][0]
    sizes = list(pi.batch_sizes(300, 32, 512, 8))
    As, Bs = _systems(sizes, 10_000)
    As.insert(137, target)
    Bs.insert(137, bt)
    mixed = _run(prrp, ctx, As, Bs, prec=3)[2][137]
    assert np.array_equal(alone, mixed)


def test_batch_4096_uneven(prrp, ctx):
    """The batched configuration: 4096 systems, n uniform in [32, 512], b = 16, one RHS,
    FP32 factor + FP64 refinement; every system refined to eta <= 1e-15 (checked on the
    GPU in FP64 to keep the test short)."""
    sizes = pi.batch_sizes(4096, 32, 512, 0)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    dA = [torch.randn(int(n), int(n), dtype=torch.float64, device="cuda", generator=g) for n in sizes]
    dB0 = [torch.randn(int(n), 1, dtype=torch.float64, device="cuda", generator=g) for n in sizes]
    dB = [b.clone() for b in dB0]
    st, info = prrp.prrp_batch_solve(ctx, dA, dB, b=16, prec=3)
    assert all(s == 0 for s in st)
    worst = 0.0
    for A, b0, x in zip(dA, dB0, dB):
        r = b0 - A @ x
        eta = float(r.abs().sum() / (A.abs().sum(0).max() * x.abs().sum() + b0.abs().sum()))
        worst = max(worst, eta)
    assert worst <= 1e-15, worst


def test_batch_tune_ahead_and_shared(prrp):
    """prrp_batch_tune fixes the launch shapes before any batch: a second call, from another
    context, finds them tuned for the process and returns at once, and batches solved
    afterwards through either context are correct."""
    import time
    c1, c2 = prrp.prrp_create(0), prrp.prrp_create(0)
    try:
        prrp.prrp_batch_tune(c1, 300, prec=3)
        t0 = time.perf_counter()
        prrp.prrp_batch_tune(c2, 300, prec=3)
        assert time.perf_counter() - t0 < 0.5
        sizes = [40, 130, 257, 300]
        As, Bs = _systems(sizes, 4400)
        for c in (c1, c2):
            st, info, X, P = _run(prrp, c, As, Bs, prec=3)
            assert all(s == 0 for s in st), st
            for A, B, x in zip(As, Bs, X):
                assert M.eta(A, x[:, 0], B[:, 0]) <= 1e-15
        with pytest.raises(prrp.PrrpError):
            prrp.prrp_batch_tune(c1, 2000)
    finally:
        c1.close()
        c2.close()
