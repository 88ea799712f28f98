"""The C-ABI library builds, loads without a GPU, and exports every entry
point declared in include/ifac.h (no compute calls here)."""
import ctypes
import os
import re

from paper_1901_07993_gb300 import build as libbuild
from paper_1901_07993_gb300 import ifac

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ifac.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+\**(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("bsr_gemm_trunc", "inv_factor_refine", "inv_factor_localized"):
        assert must in names
    assert set(names) == set(ifac.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = libbuild.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_opts_default_without_gpu():
    libbuild.build()
    o = ifac.opts()
    assert (o.m, o.max_iter, o.leaf_size, o.prec) == (2, 50, 512, ifac.FP64)
