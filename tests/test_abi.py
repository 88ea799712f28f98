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


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of ifac_bsr, ifac_opts and ifac_report have the C
    structs' sizes and field offsets (compiled against the header with gcc)."""
    import shutil
    import subprocess
    import pytest
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    mirrors = {"ifac_bsr": ifac._Bsr, "ifac_opts": ifac._Opts, "ifac_report": ifac._Report,
               "ifac_tune_result": ifac._TuneResult}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ifac.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_context_setters_reject_a_null_context():
    """The context switches validate their arguments before touching a
    device, so they can be called (and fail cleanly) without a GPU."""
    lib = ctypes.CDLL(libbuild.build())
    for name, args in (("ifac_set_split_slices", (None, 5)), ("ifac_set_fp32_intermediates", (None, 1)),
                       ("ifac_set_schedule", (None, -1, -1))):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        assert fn(*args) == ifac.ERR_INVALID, name
