"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tc_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1706_05151_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for required in ["tc_orient", "tc_count", "tc_count_local", "tc_list", "tc_sparsify_count"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    import paper_1706_05151_gb300 as tc
    assert set(declared_functions()) <= set(tc.EXPORTS) | {"tc_batch", "tc_serve"}


def test_host_only_calls(lib):
    lib.tc_status_string.restype = ctypes.c_char_p
    assert lib.tc_status_string(0) == b"ok"
    assert lib.tc_status_string(2) == b"invalid graph"
    lib.tc_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.tc_version()
    size = ctypes.c_size_t(0)
    lib.tc_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]
    assert lib.tc_workspace_size(0, 1000, 5000, ctypes.byref(size)) == 0 and size.value > 0
    assert lib.tc_workspace_size(3, 1000, 5000, ctypes.byref(size)) == 0 and size.value >= 5000 * 5
    assert lib.tc_workspace_size(0, -1, 5, ctypes.byref(size)) == 1
    assert lib.tc_workspace_size(9, 10, 5, ctypes.byref(size)) == 1


def test_null_context_is_rejected(lib):
    lib.tc_count.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_size_t, ctypes.c_void_p]
    assert lib.tc_count(None, None, None, None, 0, None) == 1


def test_library_refuses_without_gpu():
    import torch
    import paper_1706_05151_gb300 as tc
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        tc.Context(0)
