"""The CUDA path and the oracle share no code: no source file of the library
package imports, includes or links anything of the oracle, and the oracle
imports nothing of the package.  The package fails loudly without its
compiled library (no CPU fallback)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2208_05683_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def sources(top, exts):
    for d, _, files in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_does_not_use_the_oracle():
    for path in sources(PKG, (".py", ".cu", ".cuh", ".cpp", ".h")):
        text = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), path
        assert "psf_oracle" not in text, path
        assert not re.search(r'#include\s+"[^"]*oracle', text), path


def test_oracle_does_not_use_the_package():
    for path in sources(ORACLE, (".py", ".c", ".h")):
        text = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+paper_2208_05683_gb300\b", text, re.M), path
        assert not re.search(r'#include\s+"[^"]*psf(_[a-z]+)?\.(h|cuh)"', text), path
        assert "libpsf.so" not in text, path


def test_package_has_no_cpu_fallback():
    # every compute entry point goes through the compiled library: the
    # binding holds no numpy/scipy arithmetic of the method
    text = open(os.path.join(PKG, "__init__.py")).read()
    assert not re.search(r"^\s*(import|from)\s+(scipy|oracle)\b", text, re.M)
    assert "matmul" not in text and "expm" not in text
