"""The C-ABI library builds, loads and exports every entry point declared in
include/pencil_he.h; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pencil_he.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2403_11166_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared():
    text = open(HEADER).read()
    return re.findall(r"^int\s+(\w+)\s*\(", text, flags=re.M)


def test_header_declares_the_boundary():
    names = set(declared())
    for n in ("encode_weights", "encrypt_share", "he_linear_forward", "he_linear_backward", "decrypt_to_share",
              "pencil_ntt_batch"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    names = set(declared())
    src = open(os.path.join(ROOT, "paper_2403_11166_gb300", "he.py")).read()
    listed = set(re.findall(r'"(\w+)"', src.split("EXPORTS = (")[1].split(")")[0]))
    assert listed == names


def test_bad_params_rejected_on_host(lib):
    class Params(ctypes.Structure):
        _fields_ = [("log_n", ctypes.c_int32), ("num_primes", ctypes.c_int32),
                    ("prime_bits", ctypes.c_int32), ("t_bits", ctypes.c_int32)]
    lib.pencil_ctx_create.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    for bad in [(11, 2, 54, 41), (13, 0, 60, 41), (13, 5, 60, 41), (13, 3, 61, 41), (13, 3, 60, 7),
                (12, 2, 40, 41)]:
        assert lib.pencil_ctx_create(ctypes.byref(Params(*bad)), 0, ctypes.byref(h)) == -3, bad
    assert lib.pencil_ctx_create(None, 0, ctypes.byref(h)) == -1
    lib.pencil_sync_status.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.pencil_sync_status(None, None) == -1


def test_binding_status_checks_are_well_formed():
    """Every status check in the binding passes exactly (code, call name)."""
    import ast
    src = open(os.path.join(ROOT, "paper_2403_11166_gb300", "he.py")).read()
    calls = [n for n in ast.walk(ast.parse(src)) if isinstance(n, ast.Call) and getattr(n.func, "id", None) == "_check"]
    assert calls and all(len(c.args) == 2 and isinstance(c.args[1], ast.Constant) for c in calls)


def test_profiler_ids_match_binding_names():
    """PENCIL_K_* of the header, in order, are the binding's KERNEL_NAMES."""
    text = open(HEADER).read()
    body = re.search(r"PENCIL_K_NTT_RAW = 0,(.*?)PENCIL_K_COUNT", text, flags=re.S).group(1)
    ids = ["PENCIL_K_NTT_RAW"] + [x.strip() for x in body.split(",") if x.strip()]
    src = open(os.path.join(ROOT, "paper_2403_11166_gb300", "he.py")).read()
    names = re.findall(r'"(\w+)"', re.search(r"KERNEL_NAMES = \((.*?)\)", src, flags=re.S).group(1))
    assert [i[len("PENCIL_K_"):].lower() for i in ids] == names
