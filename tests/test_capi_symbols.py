"""The C-ABI library builds, loads, and exports every symbol include/nop.h declares.

Runs without a GPU: loading libnop.so makes no CUDA call.
"""
import ctypes
import os
import re

from paper_2509_01416_gb300 import build as B
from paper_2509_01416_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(nop_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    B.build()
    L = ctypes.CDLL(capi.LIB_PATH)
    declared = _declared()
    assert "nop_solve_fixed_source" in declared
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    # the binding knows every declared symbol too
    assert declared <= set(capi.SIGNATURES), declared - set(capi.SIGNATURES)


def test_status_strings_without_gpu():
    L = capi.lib()
    assert L.nop_status_str(0) == b"ok"
    assert L.nop_status_str(capi.NOP_ENOCONV) == b"iteration cap reached"


def test_create_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        return
    h = ctypes.c_void_p()
    assert capi.lib().nop_create(ctypes.byref(h), 0) == capi.NOP_ECUDA
    assert capi.lib().nop_destroy(None) == 0
