"""The product path and the oracle share no code: nothing in the package imports, includes or
loads anything under oracle/, and the oracle imports nothing of the package.  Static checks of
the sources; CPU only."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2106_10031_gb300")
ORC = os.path.join(ROOT, "oracle")


def _sources(folder, exts):
    out = []
    for e in exts:
        out += glob.glob(os.path.join(folder, "**", f"*{e}"), recursive=True)
    return [p for p in out if "_build" not in p]


def test_package_never_reaches_the_oracle():
    bad = []
    for p in _sources(PKG, (".py",)):
        src = open(p).read()
        if re.search(r"^\s*(from\s+oracle\b|import\s+oracle\b)", src, flags=re.M) or "liborc" in src:
            bad.append(p)
    for p in _sources(PKG, (".cu", ".cuh", ".h", ".cpp", ".c")):
        src = open(p).read()
        if re.search(r'#\s*include\s*[<"][^>"]*oracle', src) or "am_oracle" in src or "liborc" in src:
            bad.append(p)
    for p in glob.glob(os.path.join(ROOT, "include", "*.h")):
        if "oracle" in re.sub(r"/\*.*?\*/", "", open(p).read(), flags=re.S):
            bad.append(p)
    assert not bad, f"product sources that reach the oracle: {bad}"


def test_oracle_never_uses_the_package():
    bad = []
    for p in _sources(ORC, (".py", ".c", ".h")):
        src = open(p).read()
        if "paper_2106_10031_gb300" in src or "libam_gb300" in src or "analytic_marching.h" in src:
            bad.append(p)
    assert not bad, f"oracle sources that use the product: {bad}"
