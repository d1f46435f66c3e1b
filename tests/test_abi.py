"""The C-ABI library builds, loads and exports every entry point declared in include/*.h, and
the ctypes binding's structs match the header's layout.  CPU only: no compute call."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_10031_gb300 import build, native
    build.build()
    return native.load()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:[A-Za-z_][\w ]*\*?\s*)\b(am_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    from paper_2106_10031_gb300 import native
    names = declared_functions()
    assert "am_march" in names and "am_load_mlp" in names and "am_seed" in names and "am_get_mesh" in names
    bound = {n for n, _, _ in native.ENTRY_POINTS}
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"
        assert n in bound, f"{n} has no binding"
    out = subprocess.run(["nm", "-D", "--defined-only", native.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (am_\w+)", out))
    assert set(names) <= exported


STRUCTS = ["am_ctx_opts", "am_mlp_desc", "am_march_opts", "am_stats_t", "am_mesh", "am_tuning", "am_tune_point", "am_march_point"]


def test_struct_layout_matches_header(tmp_path):
    from paper_2106_10031_gb300 import native
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "analytic_marching.h"', "int main(void){"]
    for s in STRUCTS:
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in getattr(native, s)._fields_:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for s in STRUCTS:
        cls = getattr(native, s)
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2106_10031_gb300 import AMError, Mesher
    with pytest.raises(AMError) as e:
        Mesher()
    assert e.value.status == 2   # AM_ERR_CUDA, no CPU fallback
