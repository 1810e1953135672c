"""ctypes binding of libprrp.so: the C entry points under the same names, taking torch
tensors (device memory) or numpy arrays (host memory).  Only argument marshalling happens
here; every step of the factorization and solve runs in the library's CUDA kernels.

There is no CPU fallback: importing this module raises ImportError when libprrp.so has
not been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libprrp.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libprrp.so is not built ({_LIB_PATH} missing); run "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
_lib = C.CDLL(_LIB_PATH)

STATUS = {0: "PRRP_OK", 1: "PRRP_ERR_INVALID_ARG", 2: "PRRP_ERR_SINGULAR", 3: "PRRP_ERR_NONFINITE",
          4: "PRRP_ERR_OOM", 5: "PRRP_ERR_CUDA", 6: "PRRP_ERR_TIMEOUT", 7: "PRRP_ERR_SWAP_LIMIT",
          8: "PRRP_ERR_NOT_CONVERGED", 9: "PRRP_ERR_BUSY", 10: "PRRP_ERR_UNSUPPORTED"}
PRRP_OK, PRRP_ERR_INVALID_ARG, PRRP_ERR_SINGULAR, PRRP_ERR_NONFINITE = 0, 1, 2, 3
PRRP_ERR_OOM, PRRP_ERR_CUDA, PRRP_ERR_TIMEOUT, PRRP_ERR_SWAP_LIMIT = 4, 5, 6, 7
PRRP_ERR_NOT_CONVERGED, PRRP_ERR_BUSY, PRRP_ERR_UNSUPPORTED = 8, 9, 10
PRRP_FP64, PRRP_TF32, PRRP_BF16X3, PRRP_FP32, PRRP_FP64_EMU = 0, 1, 2, 3, 4


class prrp_opts(C.Structure):
    _fields_ = [("b", C.c_int), ("tau", C.c_double), ("prec", C.c_int), ("max_swaps", C.c_int),
                ("refine_max_iter", C.c_int), ("refine_target", C.c_double)]


class prrp_factor_stats(C.Structure):
    _fields_ = [("growth", C.c_double), ("growth_u", C.c_double), ("max_l21", C.c_double),
                ("amax", C.c_double),
                ("swaps", C.c_int), ("info", C.c_int), ("panels", C.c_int)]


class prrp_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("eta0", C.c_double), ("eta", C.c_double)]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_SIGS = {
    "prrp_opts_default": (None, [C.POINTER(prrp_opts)]),
    "prrp_status_string": (C.c_char_p, [_I]),
    "prrp_version": (C.c_char_p, []),
    "prrp_ctx_last_error": (C.c_char_p, [_P]),
    "prrp_create": (_I, [C.POINTER(_P), _I]),
    "prrp_destroy": (_I, [_P]),
    "prrp_factor": (_I, [_P, _I, _P, _I, C.POINTER(prrp_opts), _P, C.POINTER(_P)]),
    "prrp_factor_calu": (_I, [_P, _I, _P, _I, C.POINTER(prrp_opts), _I, _P, C.POINTER(_P)]),
    "prrp_factor_block": (_I, [_P, _I, _P, _I, C.POINTER(prrp_opts), _I, _I, _P, C.POINTER(_P)]),
    "prrp_factors_get": (_I, [_P, _P, C.POINTER(prrp_factor_stats)]),
    "prrp_factors_perm_device": (_P, [_P]),
    "prrp_factors_destroy": (None, [_P]),
    "prrp_solve": (_I, [_P, _P, _P, _I, _P, _I, C.POINTER(prrp_opts), _P, C.POINTER(prrp_solve_info)]),
    "prrp_gesv_host": (_I, [_P, _I, _P, _I, _I, _P, _I, _P, C.POINTER(prrp_opts), _P,
                            C.POINTER(prrp_factor_stats), C.POINTER(prrp_solve_info)]),
    "prrp_panel_select": (_I, [_P, _I, _I, _P, _I, _D, _I, _P, _P, C.POINTER(_I), _P]),
    "prrp_schur_update": (_I, [_P, _I, _I, _I, _P, _I, _P, _I, _P, _I, _I, _P]),
    "prrp_selftest_wait": (_I, [_P, C.c_uint, _P]),
    "prrp_selftest_chain_wait": (_I, [_P, C.c_uint, _P]),
    "prrp_ctx_set_solve_mode": (_I, [_P, C.c_int]),
    "prrp_batch_tune": (_I, [_P, C.c_int, _P, _P]),
    "prrp_panel_select_noalloc": (_I, [_I, _I, _P, _I, _D, _I, _P, _P, C.POINTER(_I), _P]),
    "prrp_ctx_set_timing": (_I, [_P, _I]),
    "prrp_ctx_kernel_stats": (_I, [_P, _P, _P, _P, _I]),
    "prrp_ctx_timeline": (_I, [_P, _I, _P, _P, _P, C.POINTER(_I)]),
    "prrp_ctx_set_panel_mode": (_I, [_P, _I]),
    "prrp_ctx_set_sm_split": (_I, [_P, _I, _I]),
    "prrp_ctx_set_update_block": (_I, [_P, _I]),
    "prrp_server_create": (_I, [_P, C.c_size_t, C.POINTER(prrp_opts), _I, C.POINTER(_P)]),
    "prrp_server_submit": (_I, [_P, _P, C.POINTER(C.c_uint64)]),
    "prrp_server_wait": (_I, [_P, C.c_uint64, C.c_int64, _P]),
    "prrp_server_stats": (_I, [_P, _P]),
    "prrp_server_destroy": (_I, [_P]),
    "prrp_ctx_device": (_I, [_P, C.POINTER(_I)]),
    "prrp_batch_solve": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, C.POINTER(prrp_opts), _P, _P, _P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def exported_symbols() -> list[str]:
    """Names this binding resolves in libprrp.so (all declared in include/prrp.h)."""
    return sorted(_SIGS)


class PrrpError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        self.name = STATUS.get(status, f"status {status}")
        msg = f"{where}: {self.name}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


def _check(status: int, where: str, ctx=None, allow=()):
    if status != PRRP_OK and status not in allow:
        detail = ""
        if ctx is not None and status == PRRP_ERR_CUDA:
            detail = (_lib.prrp_ctx_last_error(ctx) or b"").decode()
        raise PrrpError(status, where, detail)
    return status


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev_matrix(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda or t.dim() != 2:
        raise TypeError(f"{name}: a 2-D float64 CUDA tensor is expected")
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError(f"{name}: rows must be contiguous (row-major)")
    return max(t.stride(0), t.shape[1], 1)


def default_opts(b=64, tau=2.0, prec=PRRP_FP64, max_swaps=64, refine_max_iter=10,
                 refine_target=2.0 ** -53) -> prrp_opts:
    o = prrp_opts()
    _lib.prrp_opts_default(C.byref(o))
    o.b, o.tau, o.prec, o.max_swaps = int(b), float(tau), int(prec), int(max_swaps)
    o.refine_max_iter, o.refine_target = int(refine_max_iter), float(refine_target)
    return o


def prrp_version() -> str:
    return _lib.prrp_version().decode()


def prrp_status_string(status: int) -> str:
    return _lib.prrp_status_string(int(status)).decode()


class Context:
    """Owns a prrp_ctx* bound to one CUDA device."""

    def __init__(self, device: int = 0):
        h = C.c_void_p()
        _check(_lib.prrp_create(C.byref(h), int(device)), "prrp_create")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            _lib.prrp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Factors:
    """Owns a prrp_factors* (the permutation and statistics of one factorization; L\\U stay
    in the caller's tensor)."""

    def __init__(self, handle, n, A):
        self.handle = handle
        self.n = n
        self.A = A          # keeps the factored tensor alive

    def perm(self) -> np.ndarray:
        p = np.empty(self.n, dtype=np.int32)
        _check(_lib.prrp_factors_get(self.handle, p.ctypes.data_as(C.c_void_p), None),
               "prrp_factors_get")
        return p

    def stats(self) -> dict:
        s = prrp_factor_stats()
        _check(_lib.prrp_factors_get(self.handle, None, C.byref(s)), "prrp_factors_get")
        return {"growth": s.growth, "growth_u": s.growth_u, "max_l21": s.max_l21, "amax": s.amax,
                "swaps": s.swaps,
                "info": s.info, "panels": s.panels}

    def close(self):
        if getattr(self, "handle", None):
            _lib.prrp_factors_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prrp_create(device: int = 0) -> Context:
    return Context(device)


def prrp_destroy(ctx: Context) -> None:
    ctx.close()


def prrp_factor(ctx: Context, A, b=64, tau=2.0, prec=PRRP_FP64, max_swaps=64, stream=None,
                allow=()) -> Factors:
    """LU_PRRP of the square float64 CUDA tensor A in place (row-major L\\U on return)."""
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("square matrix expected")
    lda = _dev_matrix(A, "A") if n else 1
    o = default_opts(b, tau, prec, max_swaps)
    h = C.c_void_p()
    st = _lib.prrp_factor(ctx.handle, n, C.c_void_p(A.data_ptr() if n else 0), lda, C.byref(o),
                          _stream_ptr(stream), C.byref(h))
    F = Factors(h, n, A) if h.value else None
    if st != PRRP_OK and st not in allow:
        if F is not None:
            F.close()
        _check(st, "prrp_factor", ctx.handle)
    if F is not None:
        F.status = st
    return F


def prrp_factor_calu(ctx: Context, A, leaf_rows: int, b=64, tau=2.0, prec=PRRP_FP64, max_swaps=64,
                     stream=None, allow=()) -> Factors:
    """CALU_PRRP (tournament pivoting over leaves of leaf_rows rows) of the square float64
    CUDA tensor A in place."""
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("square matrix expected")
    lda = _dev_matrix(A, "A") if n else 1
    o = default_opts(b, tau, prec, max_swaps)
    h = C.c_void_p()
    st = _lib.prrp_factor_calu(ctx.handle, n, C.c_void_p(A.data_ptr() if n else 0), lda, C.byref(o),
                               int(leaf_rows), _stream_ptr(stream), C.byref(h))
    F = Factors(h, n, A) if h.value else None
    if st != PRRP_OK and st not in allow:
        if F is not None:
            F.close()
        _check(st, "prrp_factor_calu", ctx.handle)
    if F is not None:
        F.status = st
    return F


def prrp_factor_block(ctx: Context, A, blocks: int, tree: str = "parallel", b=16, tau=2.0, max_swaps=64,
                      stream=None) -> Factors:
    """Block parallel (tree="parallel") or block pairwise (tree="pairwise") LU_PRRP of the
    square float64 CUDA tensor A in place, for stability studies (product form: no solve)."""
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("square matrix expected")
    t = {"parallel": 0, "pairwise": 1}[tree]
    lda = _dev_matrix(A, "A") if n else 1
    o = default_opts(b, tau, PRRP_FP64, max_swaps)
    h = C.c_void_p()
    st = _lib.prrp_factor_block(ctx.handle, n, C.c_void_p(A.data_ptr() if n else 0), lda, C.byref(o),
                                int(blocks), t, _stream_ptr(stream), C.byref(h))
    F = Factors(h, n, A) if h.value else None
    if st != PRRP_OK:
        if F is not None:
            F.close()
        _check(st, "prrp_factor_block", ctx.handle)
    return F


def prrp_solve(ctx: Context, F: Factors, B, A_orig=None, refine_max_iter=10,
               refine_target=2.0 ** -53, stream=None) -> dict:
    """Overwrite the float64 CUDA tensor B (n x nrhs) with A^-1 B; refine in FP64 against
    A_orig when given."""
    ldb = _dev_matrix(B, "B")
    if B.shape[0] != F.n:
        raise ValueError(f"B: {F.n} rows are expected")
    a0 = None
    if A_orig is not None:
        # read by the library as n x n with the factored matrix's leading dimension
        lda0 = _dev_matrix(A_orig, "A_orig")
        if tuple(A_orig.shape) != (F.n, F.n) or (F.n > 0 and lda0 != _dev_matrix(F.A, "A")):
            raise ValueError("A_orig: the unfactored n x n matrix, with the factored matrix's row stride, "
                             "is expected")
        a0 = C.c_void_p(A_orig.data_ptr())
    o = default_opts(refine_max_iter=refine_max_iter, refine_target=refine_target)
    info = prrp_solve_info()
    st = _lib.prrp_solve(ctx.handle, F.handle, a0, B.shape[1], C.c_void_p(B.data_ptr()), ldb,
                         C.byref(o), _stream_ptr(stream), C.byref(info))
    _check(st, "prrp_solve", ctx.handle, allow=(PRRP_ERR_NOT_CONVERGED,))
    return {"iterations": info.iterations, "eta0": info.eta0, "eta": info.eta,
            "converged": st == PRRP_OK}


def prrp_gesv_host(ctx: Context, A: np.ndarray, B: np.ndarray, b=64, tau=2.0, prec=PRRP_FP64,
                   max_swaps=64, refine_max_iter=0, refine_target=2.0 ** -53, stream=None,
                   X: np.ndarray | None = None):
    """Solve A X = B from host arrays (copies in and out inside the call)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    n, nrhs = A.shape[0], B.shape[1]
    if X is None:
        X = np.empty((n, nrhs))
    o = default_opts(b, tau, prec, max_swaps, refine_max_iter, refine_target)
    stats, info = prrp_factor_stats(), prrp_solve_info()
    st = _lib.prrp_gesv_host(ctx.handle, n, A.ctypes.data_as(C.c_void_p), n, nrhs,
                             B.ctypes.data_as(C.c_void_p), nrhs, X.ctypes.data_as(C.c_void_p),
                             C.byref(o), _stream_ptr(stream), C.byref(stats), C.byref(info))
    _check(st, "prrp_gesv_host", ctx.handle, allow=(PRRP_ERR_NOT_CONVERGED,))
    return X, {"growth": stats.growth, "swaps": stats.swaps, "max_l21": stats.max_l21}, \
        {"iterations": info.iterations, "eta0": info.eta0, "eta": info.eta}


def prrp_panel_select(ctx: Context, P, tau=2.0, max_swaps=64, stream=None):
    """Strong RRQR selection on the m x w float64 CUDA tensor P: returns (order, L21, swaps)
    with order[i] the panel row at position i and L21 an (m - w) x w CUDA tensor."""
    import torch
    m, w = P.shape
    ldp = _dev_matrix(P, "P")
    L21 = torch.empty((max(m - w, 0), w), dtype=torch.float64, device=P.device)
    order = np.empty(m, dtype=np.int32)
    sw = C.c_int(0)
    st = _lib.prrp_panel_select(ctx.handle, m, w, C.c_void_p(P.data_ptr()), ldp, float(tau),
                                int(max_swaps), order.ctypes.data_as(C.c_void_p),
                                C.c_void_p(L21.data_ptr() if L21.numel() else 0), C.byref(sw),
                                _stream_ptr(stream))
    _check(st, "prrp_panel_select", ctx.handle)
    return order, L21, sw.value


def prrp_schur_update(ctx: Context, L, U, Cm, prec=PRRP_FP64, stream=None) -> None:
    """Cm -= L @ U on float64 CUDA tensors (k = L.shape[1] <= 128)."""
    ldl, ldu, ldc = _dev_matrix(L, "L"), _dev_matrix(U, "U"), _dev_matrix(Cm, "C")
    m, k = L.shape
    n = U.shape[1]
    if U.shape[0] != k or tuple(Cm.shape) != (m, n):
        raise ValueError("L (m x k), U (k x n) and C (m x n) are expected")
    st = _lib.prrp_schur_update(ctx.handle, m, n, k, C.c_void_p(L.data_ptr()), ldl,
                                C.c_void_p(U.data_ptr()), ldu, C.c_void_p(Cm.data_ptr()), ldc, int(prec),
                                _stream_ptr(stream))
    _check(st, "prrp_schur_update", ctx.handle)


def prrp_selftest_wait(ctx: Context, spin_limit: int = 20000, stream=None) -> int:
    """Run the bounded-wait self-test; returns the status (PRRP_ERR_TIMEOUT expected)."""
    return _lib.prrp_selftest_wait(ctx.handle, int(spin_limit), _stream_ptr(stream))


def prrp_selftest_chain_wait(ctx: Context, spin_limit: int = 20000, stream=None) -> int:
    """Run the substitution's bounded-wait self-test; returns the status (PRRP_ERR_TIMEOUT
    expected)."""
    return _lib.prrp_selftest_chain_wait(ctx.handle, int(spin_limit), _stream_ptr(stream))


KINDS = ["scan", "panel", "permute", "update", "diag", "u12", "lfix", "solve", "batch"]


def prrp_ctx_set_timing(ctx: Context, enable=True) -> None:
    """enable: False/0 off, True/1 per-class totals, 2 also a launch timeline."""
    _check(_lib.prrp_ctx_set_timing(ctx.handle, int(enable)), "prrp_ctx_set_timing")


def prrp_ctx_set_panel_mode(ctx: Context, cluster_max_rows: int = 0) -> None:
    """Panels of at most cluster_max_rows rows run as one thread-block cluster (0: default)."""
    _check(_lib.prrp_ctx_set_panel_mode(ctx.handle, int(cluster_max_rows)), "prrp_ctx_set_panel_mode")


def prrp_ctx_set_sm_split(ctx: Context, panel_ctas: int = 0, block_ctas: int = 0) -> None:
    """SMs for the panels and the diagonal-block work in the tensor-core modes (0: default)."""
    _check(_lib.prrp_ctx_set_sm_split(ctx.handle, int(panel_ctas), int(block_ctas)), "prrp_ctx_set_sm_split")


def prrp_ctx_set_update_block(ctx: Context, nb: int = 0) -> None:
    """Aggregated trailing update in the TF32 / BF16X3 modes: blocks of floor(nb / b)
    panels, nb <= 256 (0, the default, or nb < 2 b: the per-panel update)."""
    _check(_lib.prrp_ctx_set_update_block(ctx.handle, int(nb)), "prrp_ctx_set_update_block")


def prrp_ctx_set_solve_mode(ctx: Context, mode: int) -> None:
    """0: one launch per triangle for up to 16 right-hand sides (default); 1: one launch per
    64-row block (holds no SM while waiting; for contexts sharing the GPU)."""
    _check(_lib.prrp_ctx_set_solve_mode(ctx.handle, int(mode)), "prrp_ctx_set_solve_mode", ctx.handle)


def prrp_ctx_timeline(ctx: Context) -> list:
    """Launch timeline kept under timing level 2: [(kind name, start ms, end ms), ...]."""
    cnt = C.c_int(0)
    _check(_lib.prrp_ctx_timeline(ctx.handle, 0, None, None, None, C.byref(cnt)), "prrp_ctx_timeline")
    n = cnt.value
    if n == 0:
        return []
    k = (C.c_int * n)()
    a = (C.c_double * n)()
    b = (C.c_double * n)()
    _check(_lib.prrp_ctx_timeline(ctx.handle, n, k, a, b, C.byref(cnt)), "prrp_ctx_timeline")
    return [(KINDS[k[i]], a[i], b[i]) for i in range(min(n, cnt.value))]


def prrp_ctx_kernel_stats(ctx: Context, reset: bool = False) -> dict:
    """Per kernel class: {"ms", "launches", "flops"} since the last reset."""
    ms = (C.c_double * len(KINDS))()
    ln = (C.c_longlong * len(KINDS))()
    fl = (C.c_longlong * len(KINDS))()
    _check(_lib.prrp_ctx_kernel_stats(ctx.handle, ms, ln, fl, int(bool(reset))),
           "prrp_ctx_kernel_stats")
    return {k: {"ms": ms[i], "launches": ln[i], "flops": fl[i]} for i, k in enumerate(KINDS)}


def prrp_panel_select_noalloc(P, tau=2.0, max_swaps=64, stream=None):
    """prrp_panel_select without a context or any allocation inside the library (scratch in
    a static device array).  The outputs are allocated here, by the caller side: returns
    (order as a device int32 tensor, L21 device tensor, swaps)."""
    import torch
    m, w = P.shape
    ldp = _dev_matrix(P, "P")
    order = torch.empty(m, dtype=torch.int32, device=P.device)
    L21 = torch.empty((max(m - w, 0), w), dtype=torch.float64, device=P.device)
    sw = C.c_int(0)
    with torch.cuda.device(P.device):     # the C side runs on the current device
        if stream is None:
            stream = torch.cuda.current_stream(P.device)
        st = _lib.prrp_panel_select_noalloc(m, w, C.c_void_p(P.data_ptr()), ldp, float(tau),
                                            int(max_swaps), C.c_void_p(order.data_ptr()),
                                            C.c_void_p(L21.data_ptr() if L21.numel() else 0),
                                            C.byref(sw), _stream_ptr(stream))
    _check(st, "prrp_panel_select_noalloc")
    return order, L21, sw.value


def prrp_batch_tune(ctx: Context, nmax: int, b=16, prec=PRRP_FP32, stream=None) -> None:
    """Tune prrp_batch_solve's launch shape for sizes up to nmax ahead of use."""
    o = default_opts(b=b, prec=prec)
    _check(_lib.prrp_batch_tune(ctx.handle, int(nmax), C.byref(o), _stream_ptr(stream)), "prrp_batch_tune",
           ctx.handle)


def _dev_matrices(ts, name):
    """One pass over a list of 2-D float64 CUDA tensors with contiguous rows: an int64 array
    of (data pointer, rows, columns, leading dimension) per tensor."""
    import torch
    f64 = torch.float64
    if len(ts) == 0:
        return np.zeros((0, 4), dtype=np.int64)
    try:
        m = np.array([(t.data_ptr(), *t.shape, *t.stride(), t.dtype is f64 and t.is_cuda) for t in ts],
                     dtype=np.int64)
    except (AttributeError, TypeError, ValueError):     # not tensors, or of mixed dimensions
        m = None
    if m is None or m.ndim != 2 or m.shape[1] != 6 or not m[:, 5].all():
        raise TypeError(f"{name}: 2-D float64 CUDA tensors are expected")
    if np.any((m[:, 2] > 1) & (m[:, 4] != 1)):
        raise ValueError(f"{name}: rows must be contiguous (row-major)")
    m[:, 4] = np.maximum(np.maximum(m[:, 3], m[:, 2]), 1)
    return m[:, [0, 1, 2, 4]]


def _dev_perms(perms, n):
    """Device pointers of the permutation outputs: contiguous int32 CUDA tensors of at least
    n[i] elements (checked here, so the kernel never writes through a host pointer)."""
    import torch
    i32 = torch.int32
    if len(perms) != len(n) or not all(
            isinstance(p, torch.Tensor) and p.dtype is i32 and p.is_cuda and p.is_contiguous() and p.numel() >= int(k)
            for p, k in zip(perms, n)):
        raise TypeError("perms: one contiguous int32 CUDA tensor of at least n_i elements per system is expected")
    return np.array([p.data_ptr() for p in perms], dtype=np.int64)


_INFO_DTYPE = np.dtype({"names": ["iterations", "eta0", "eta"], "formats": ["<i4", "<f8", "<f8"],
                        "offsets": [prrp_solve_info.iterations.offset, prrp_solve_info.eta0.offset,
                                    prrp_solve_info.eta.offset],
                        "itemsize": C.sizeof(prrp_solve_info)})


def prrp_batch_solve(ctx: Context, As, Bs, b=16, tau=2.0, prec=PRRP_FP32, max_swaps=64,
                     refine_max_iter=10, refine_target=2.0 ** -53, stream=None, perms=None):
    """Solve the independent systems As[i] X_i = Bs[i] (float64 CUDA tensors, n_i <= 1024)
    in one batched launch; Bs[i] is overwritten by X_i.  perms (optional): int32 CUDA
    tensors receiving each system's row permutation.  Returns (statuses, infos)."""
    count = len(As)
    if len(Bs) != count or (perms is not None and len(perms) != count):
        raise ValueError("As, Bs (and perms) must have one entry per system")
    ma = _dev_matrices(As, "A")
    mb = _dev_matrices(Bs, "B")
    if np.any(ma[:, 1] != ma[:, 2]) or np.any(mb[:, 1] != ma[:, 1]):
        raise ValueError("each A must be square and each B must have as many rows as its A")
    n = np.ascontiguousarray(ma[:, 1], dtype=np.int32)
    lda = np.ascontiguousarray(ma[:, 3], dtype=np.int32)
    nrhs = np.ascontiguousarray(mb[:, 2], dtype=np.int32)
    ldb = np.ascontiguousarray(mb[:, 3], dtype=np.int32)
    pa = np.ascontiguousarray(ma[:, 0])
    pb = np.ascontiguousarray(mb[:, 0])
    pp = _dev_perms(perms, n) if perms is not None else None
    st = np.zeros(count, dtype=np.int32)
    infos = np.zeros(count, dtype=_INFO_DTYPE)
    o = default_opts(b, tau, prec, max_swaps, refine_max_iter, refine_target)
    rc = _lib.prrp_batch_solve(ctx.handle, count, n.ctypes.data, pa.ctypes.data, lda.ctypes.data,
                               nrhs.ctypes.data, pb.ctypes.data, ldb.ctypes.data,
                               pp.ctypes.data if pp is not None else None, C.byref(o),
                               _stream_ptr(stream), st.ctypes.data, infos.ctypes.data)
    # outcomes of individual systems are reported per system; anything else raises
    _check(rc, "prrp_batch_solve", ctx.handle,
           allow=(PRRP_ERR_SINGULAR, PRRP_ERR_NONFINITE, PRRP_ERR_SWAP_LIMIT, PRRP_ERR_NOT_CONVERGED))
    return st.tolist(), [{"iterations": i, "eta0": e0, "eta": e} for i, e0, e in infos.tolist()]



class prrp_request(C.Structure):
    _fields_ = [("n", C.c_int), ("nrhs", C.c_int), ("hA", C.c_void_p), ("lda", C.c_int),
                ("hB", C.c_void_p), ("ldb", C.c_int), ("hX", C.c_void_p), ("ldx", C.c_int)]


class prrp_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("eta", C.c_double),
                ("latency_us", C.c_double), ("queue_us", C.c_double)]


class prrp_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("units", C.c_uint64), ("p50_us", C.c_double), ("p99_us", C.c_double),
                ("mean_us", C.c_double), ("solves_per_s", C.c_double),
                ("peak_bytes_in_use", C.c_uint64), ("peak_busy_lanes", C.c_int)]


class Server:
    """Owns a prrp_server* (continuous-batching solve loop)."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int, lanes: int = 4, prec=PRRP_FP32, b=64,
                 tau=2.0, refine_max_iter=10, refine_target=2.0 ** -53):
        o = default_opts(b, tau, prec, 64, refine_max_iter, refine_target)
        h = C.c_void_p()
        _check(_lib.prrp_server_create(ctx.handle, C.c_size_t(int(hbm_budget_bytes)), C.byref(o),
                                       int(lanes), C.byref(h)), "prrp_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, A: np.ndarray, B: np.ndarray, X: np.ndarray) -> int:
        """Queue A X = B (host float64 arrays, row-major, kept alive until wait)."""
        for name, M in (("A", A), ("B", B), ("X", X)):
            if not isinstance(M, np.ndarray) or M.dtype != np.float64 or M.ndim != 2 or \
                    (M.shape[1] > 1 and M.strides[1] != 8) or M.strides[0] % 8:
                raise TypeError(f"{name}: a 2-D float64 host array with contiguous rows is expected")
        n = A.shape[0]
        nrhs = B.shape[1]
        if A.shape[1] != n or B.shape[0] != n or X.shape != (n, nrhs) or not X.flags.writeable:
            raise ValueError("A (n x n), B (n x nrhs) and a writable X (n x nrhs) are expected")
        r = prrp_request(n, nrhs, A.ctypes.data, A.strides[0] // 8, B.ctypes.data,
                         max(B.strides[0] // 8, nrhs), X.ctypes.data, max(X.strides[0] // 8, nrhs))
        t = C.c_uint64(0)
        _check(_lib.prrp_server_submit(self.handle, C.byref(r), C.byref(t)), "prrp_server_submit")
        self._keep[t.value] = (A, B, X)
        return t.value

    def wait(self, ticket: int, timeout_us: int = -1) -> dict:
        res = prrp_result()
        _check(_lib.prrp_server_wait(self.handle, C.c_uint64(ticket), C.c_int64(timeout_us),
                                     C.byref(res)), "prrp_server_wait")
        self._keep.pop(ticket, None)
        return {"status": res.status, "iterations": res.iterations, "eta": res.eta,
                "latency_us": res.latency_us, "queue_us": res.queue_us}

    def stats(self) -> dict:
        st = prrp_serve_stats()
        _check(_lib.prrp_server_stats(self.handle, C.byref(st)), "prrp_server_stats")
        return {f: getattr(st, f) for f, _ in prrp_serve_stats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            _check(_lib.prrp_server_destroy(self.handle), "prrp_server_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def partition_systems(sizes, parts: int) -> list:
    """Split independent systems over `parts` GPUs for the batched and served forms: largest
    first, each to the part with the least work so far (work = n^3, the factorization's
    order), ties to the lower part.  Returns one list of system indices per part (each in
    ascending order).  Host logic only; every part then runs prrp_batch_solve on its own
    systems, with no collective on the data path."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0.0] * parts
    out = [[] for _ in range(parts)]
    for i in order:
        k = min(range(parts), key=lambda p: (load[p], p))
        out[k].append(i)
        load[k] += float(sizes[i]) ** 3
    return [sorted(x) for x in out]


def prrp_server_create(ctx: Context, hbm_budget_bytes: int, lanes: int = 4, **kw) -> Server:
    return Server(ctx, hbm_budget_bytes, lanes, **kw)
