"""The C ABI library builds, loads and exports every symbol of include/rsc.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_16635_gb300 import load_library
    return load_library()


def _header_functions():
    text = open(os.path.join(ROOT, "include", "rsc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rsc_[a-z0-9_]+)\s*\(", text)))


def test_every_header_symbol_is_exported(lib):
    names = _header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2508_16635_gb300.rsc import EXPORTS
    assert sorted(EXPORTS) == _header_functions()


def test_version_and_status_strings(lib):
    assert lib.rsc_abi_version() == 9
    assert lib.rsc_status_string(0) == b"RSC_OK"
    assert lib.rsc_status_string(6) == b"RSC_ESINGULAR"


def test_create_rejects_bad_parameters_without_touching_the_gpu(lib):
    from paper_2508_16635_gb300.rsc import Params
    ctx = ctypes.c_void_p()
    bad = [Params(100.0, 1e-3, 1.0, 0.35, 0, 4, 24, 0),     # L = 0
           Params(100.0, 1e-3, 1.0, 0.35, 31, 4, 3, 0),     # Nr too small
           Params(100.0, -1.0, 1.0, 0.35, 31, 4, 24, 0),    # Ek <= 0
           Params(100.0, 1e-3, 1.0, 1.5, 31, 4, 24, 0),     # eta >= 1
           Params(100.0, 1e-3, 1.0, 0.35, 31, 4, 24, 7)]    # unknown precision
    for p in bad:
        assert lib.rsc_create(ctypes.byref(p), None, ctypes.byref(ctx)) == 1
    assert lib.rsc_create(None, None, ctypes.byref(ctx)) == 1
    assert lib.rsc_destroy(None) == 1
    assert lib.rsc_last_error(None) == b"null context"


STRUCTS = [("rsc_params", "Params"), ("rsc_newton_opts", "NewtonOpts"),
           ("rsc_newton_report", "NewtonReport"), ("rsc_tuning", "Tuning"),
           ("rsc_continuation_opts", "ContinuationOpts"),
           ("rsc_continuation_point", "ContinuationPoint"),
           ("rsc_ek_continuation_opts", "EkContinuationOpts"), ("rsc_ek_point", "EkPoint")]


def test_binding_struct_layouts_match_the_header(tmp_path):
    """Size and every field offset of the ctypes mirrors equal the C compiler's layout of the
    structs in include/rsc.h (compiled here as plain C)."""
    import shutil
    import subprocess
    from paper_2508_16635_gb300 import rsc as b
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rsc.h"', 'int main(void) {']
    for cname, pyname in STRUCTS:
        lines.append(f'  printf("{pyname} size %zu\\n", sizeof({cname}));')
        for f, _ in getattr(b, pyname)._fields_:
            lines.append(f'  printf("{pyname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            py, f, v = line.split()
            got[(py, f)] = int(v)
    for _, pyname in STRUCTS:
        cls = getattr(b, pyname)
        assert got[(pyname, "size")] == ctypes.sizeof(cls), pyname
        for f, _ in cls._fields_:
            assert got[(pyname, f)] == getattr(cls, f).offset, (pyname, f)
