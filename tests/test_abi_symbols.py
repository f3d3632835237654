"""The C-ABI library loads without a GPU and exports every function include/glim_lin.h
declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(glim_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2407_10344_b300 import build, _abi
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding declares exactly the functions of the header
    assert set(_abi.SIGNATURES) == names


def test_binding_refuses_to_run_without_a_gpu():
    import pytest
    import torch
    import paper_2407_10344_b300 as G
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="CUDA device is required"):
        G.Context(0)


def test_struct_layouts_match_header():
    from paper_2407_10344_b300 import _abi
    assert ctypes.sizeof(_abi.Frame) == 32
    assert ctypes.sizeof(_abi.Pair) == 16
    assert ctypes.sizeof(_abi.LinOpts) == 32
