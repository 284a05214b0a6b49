"""The C ABI builds, loads without a GPU, and exports every entry point that
include/tn.h declares; host-side marshalling layouts match the header."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tn_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1905_01330_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("tn_contract", "tn_group_plan_create", "tn_group_plan_run", "tn_sync_status"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(tn_\w+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(lib, n)
    lib.tn_status_string.restype = ctypes.c_char_p
    assert lib.tn_status_string(2) == b"shape mismatch"


def test_struct_layouts_match_header():
    from paper_1905_01330_gb300 import tn
    assert ctypes.sizeof(tn.TnTensor) == 8 + 4 + 4 + 8 * 8 + 8 * 8
    assert ctypes.sizeof(tn.TnContractSpec) == 3 * ctypes.sizeof(tn.TnTensor) + 4 + 32 + 32 + 4  # tail pad


def test_validation_errors_without_gpu(libpath):
    # argument checks run on the host before any CUDA call
    from paper_1905_01330_gb300 import tn
    lib = ctypes.CDLL(libpath)
    lib.tn_contract.restype = ctypes.c_int
    a, b, c = tn.TnTensor(), tn.TnTensor(), tn.TnTensor()
    for t, shape in ((a, (3, 4)), (b, (5, 6)), (c, (3, 6))):
        t.data = 0x1000
        t.rank = 2
        for i, n in enumerate(shape):
            t.shape[i] = n
    la = (ctypes.c_int * 1)(1)
    lb = (ctypes.c_int * 1)(0)
    assert lib.tn_contract(ctypes.byref(a), la, ctypes.byref(b), lb, 1, ctypes.byref(c), 0, None) == 2
    la2 = (ctypes.c_int * 1)(7)
    assert lib.tn_contract(ctypes.byref(a), la2, ctypes.byref(b), lb, 1, ctypes.byref(c), 0, None) == 1
    assert lib.tn_contract(None, la, ctypes.byref(b), lb, 1, ctypes.byref(c), 0, None) == 1
    assert lib.tn_contract(ctypes.byref(a), la, ctypes.byref(b), lb, 1, ctypes.byref(c), 9, None) == 1
