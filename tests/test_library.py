"""CPU checks of the C ABI boundary: libprrp.so builds for sm_103a, loads without a GPU,
exports every function include/prrp.h declares, and the binding covers them all."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "prrp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(prrp_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("prrp_factor", "prrp_solve", "prrp_create", "prrp_destroy",
                     "prrp_factors_get", "prrp_panel_select", "prrp_schur_update"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    lib = ctypes.CDLL(g._build_module().build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_1208_2451_gb300 as P
    assert set(P.exported_symbols()) == set(declared_functions())
    for required in ("prrp_batch_solve", "prrp_server_create", "prrp_server_submit",
                     "prrp_server_wait", "prrp_server_stats", "prrp_server_destroy"):
        assert required in declared_functions()
    assert P.prrp_version().startswith("prrp")
    assert P.prrp_status_string(2).startswith("singular")


def test_no_device_is_an_error_code_not_a_crash():
    """Without a usable GPU prrp_create reports an error status."""
    import torch
    import paper_1208_2451_gb300 as P
    if torch.cuda.is_available():
        return
    try:
        P.prrp_create(0)
    except P.PrrpError as e:
        assert e.name in ("PRRP_ERR_INVALID_ARG", "PRRP_ERR_CUDA")
    else:
        raise AssertionError("prrp_create succeeded without a device")


def test_product_package_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_1208_2451_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def _prototype_arity():
    """Parameter count of every prototype in the header (comments stripped)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for name in declared_functions():
        m = re.search(r"\b" + name + r"\s*\(", text)
        i, depth, j = m.end(), 1, m.end()
        while depth:
            depth += {"(": 1, ")": -1}.get(text[j], 0)
            j += 1
        params = " ".join(text[i:j - 1].split())
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_header():
    """Every ctypes signature in the binding takes as many arguments as the header's
    prototype, so a changed entry point cannot be called with a stale argument list."""
    import paper_1208_2451_gb300.binding as B
    arity = _prototype_arity()
    wrong = {n: (len(B._SIGS[n][1]), arity[n]) for n in arity if len(B._SIGS[n][1]) != arity[n]}
    assert not wrong, wrong


def test_batch_marshalling_host_logic():
    """prrp_batch_solve's argument marshalling: host tensors are refused before any call,
    and the per-system results are read back with the C struct's layout."""
    import numpy as np
    import torch
    import paper_1208_2451_gb300 as P
    B = P.binding
    try:
        B._dev_matrices([torch.zeros(4, 4, dtype=torch.float64)], "A")
    except TypeError:
        pass
    else:
        raise AssertionError("a host tensor was accepted")
    arr = (B.prrp_solve_info * 3)()
    for i in range(3):
        arr[i].iterations, arr[i].eta0, arr[i].eta = i + 1, 10.0 ** -i, 2.0 ** -(50 + i)
    view = np.frombuffer(arr, dtype=B._INFO_DTYPE)
    assert view.tolist() == [(i + 1, 10.0 ** -i, 2.0 ** -(50 + i)) for i in range(3)]
    for perms in ([torch.zeros(8, dtype=torch.int32)],          # host memory
                  [torch.zeros(8, dtype=torch.int64)],          # wrong type
                  [torch.zeros(8, dtype=torch.int32)] * 2):     # one per system
        try:
            B._dev_perms(perms, np.array([8], dtype=np.int32))
        except TypeError:
            pass
        else:
            raise AssertionError("a permutation output that the kernel cannot write was accepted")
