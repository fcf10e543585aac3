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


def test_slot_plan_matches_oracle(fhe):
    """The library's slot manager (host code) places every useful slot where
    the oracle's does and asks for the same rotation keys: structured masks
    (leading blocks, every fourth slot, full inputs) and random ones."""
    import random

    import numpy as np

    from oracle.circuits import slot_galois, slot_plan

    rnd = random.Random(5)
    for ns, N in ((2, 1 << 14), (8, 1 << 14), (16, 1 << 12), (128, 1 << 15)):
        cases = [[list(range(u))] * (ns // u) for u in (1, 2, 4) if ns % u == 0]
        if ns >= 8:
            cases.append([[i for i in range(ns) if i % 4 == 3]] * 4)
        cases.append([list(range(ns))] * 2)
        cases += [[sorted(rnd.sample(range(ns), rnd.randrange(0, ns + 1))) for _ in range(rnd.randrange(1, 7))]
                  for _ in range(12)]
        for useful in cases:
            mask = np.zeros((len(useful), ns), dtype=bool)
            for j, u_j in enumerate(useful):
                mask[j, u_j] = True
            n_out, dest, gal = fhe.fhe_slot_plan(ns, N, mask)
            o_out, pieces, o_dest = slot_plan(ns, useful)
            assert n_out == o_out
            assert dest.tolist() == o_dest
            assert gal == slot_galois(ns, N, pieces)
    for slots, ring_n in ((3, 1 << 12), (8, 1000), (16, 8)):  # odd slot count, N not a power of two, N < n_s
        with pytest.raises(fhe.FheError):
            fhe.fhe_slot_plan(slots, ring_n, np.zeros((1, slots), dtype=bool))
