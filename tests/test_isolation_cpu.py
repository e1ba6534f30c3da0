"""Static checks that the FP64 oracle and the CUDA path stay independent: the product
package never imports the oracle, the CUDA sources never include anything from it, and
the oracle never imports the product (the seeded input generators, which hold none of the
method's arithmetic, are passed in by the tests)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2211_03516_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def test_product_never_imports_the_oracle():
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)", re.M)
    bad = [p for p in files(PKG, (".py",)) if pat.search(open(p).read())]
    assert bad == []


def test_cuda_sources_include_nothing_from_the_oracle():
    pat = re.compile(r'#include\s*[<"][^>"]*oracle', re.I)
    bad = [p for p in files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h")) if pat.search(open(p).read())]
    assert bad == []


def test_oracle_never_imports_the_product():
    pat = re.compile(r"paper_2211_03516_gb300")
    bad = [p for p in files(ORACLE, (".py", ".c", ".h")) if pat.search(open(p).read())]
    assert bad == []
