"""Pins of the oracle's tournament max/min: the round depth and rotation
schedule, and decryption against plaintext max/min (with refreshes)."""
import random

import numpy as np

from oracle.circuits import Tournament, galois_schedule, round_depth
from oracle.philox import philox4x32_10
from paper_2407_07308_gb300 import synth
from tests.oracle_setup import OracleSetup
from tests.params import CHAIN50


def test_philox_known_answers():
    # the generator's published known-answer vectors (Random123 distribution)
    assert philox4x32_10((0, 0, 0, 0), (0, 0)) == (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)
    assert philox4x32_10((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2) == (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)
    assert philox4x32_10((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0)) == (
        0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)


def test_round_depth_and_schedule():
    assert round_depth(257, 2) == 8 + 1 + 1
    assert round_depth(17, 1) == 4 + 0 + 1
    N = 1 << 15
    g = galois_schedule(128, N)
    assert g == [pow(5, s, 2 * N) for s in (32, 16, 8, 4, 2, 1)] + [2 * N - 1]
    assert galois_schedule(8, 1024) == [25, 5, 2047]


def test_tournament_small_ring_with_refresh():
    p, d = 17, 2
    galois = galois_schedule(8, 256)
    st = OracleSetup(logN=8, p=p, L=8, K=2, seed=51, galois=galois, **CHAIN50)
    b = (p + 1) // 2
    rnd = random.Random(4)
    n = 3  # odd: the last ciphertext passes through the first cross round
    vals = [[rnd.randrange(b ** d) for _ in range(st.ss.ns)] for _ in range(n)]
    vals[2][3] = vals[0][1]  # a duplicate
    digits = [st.encrypt_slots([[(v // b ** k) % b for v in row] for row in vals], seed=60 + k) for k in range(d)]
    counter = [0]

    def refresh(cts):
        counter[0] += 1
        r = synth.EncRandomness(900 + counter[0], len(cts), st.N)
        return [st.o.encrypt(st.pk, st.o.decrypt_coeffs(c, st.s), r.u[i], r.e0[i], r.e1[i]) for i, c in enumerate(cts)]

    t = Tournament(st.evaluator(), d, st.ss.ns, st.N, refresh)
    out = t.run(digits, True, True)
    flat = [v for row in vals for v in row]
    for kind, want in (("max", max(flat)), ("min", min(flat))):
        got = [sum(st.decrypt_slots(out[kind][k])[s] * b ** k for k in range(d)) for s in range(st.ss.ns)]
        assert got == [want] * st.ss.ns, kind
    assert t.refreshes > 0
