"""Host-side checks of the CUDA library that need no GPU: it loads, exports
every function include/fhe.h declares, and its modular arithmetic (the same
source the kernels compile) agrees with 128-bit reference arithmetic."""
import os
import re

import pytest

from tests.params import CHAIN36, CHAIN50

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fhe():
    from paper_2407_07308_gb300 import build

    build.build()
    from paper_2407_07308_gb300 import fhe as f

    return f


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(fhe_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(fhe):
    L = fhe.lib()
    names = declared_functions()
    assert len(names) > 40
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("chain,n", [(CHAIN50, 24), (CHAIN36, 5)])
def test_modarith_selftest(fhe, chain, n):
    assert fhe.fhe_selftest_modarith(chain["U"], chain["lo"], chain["hi"], n, 20000) == 0
