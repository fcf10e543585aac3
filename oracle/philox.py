"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), written from its
published definition.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Used to check the
library's device generator word for word; the known-answer vectors of the
generator's reference distribution pin this implementation
(tests/test_oracle_tournament.py, test_philox_known_answers).

One round maps (c0, c1, c2, c3) with key (k0, k1) to
  (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
and the key is bumped by the Weyl constants between rounds.
"""
MASK = 0xFFFFFFFF
M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(ctr, key):
    c0, c1, c2, c3 = ctr
    k0, k1 = key
    for _ in range(10):
        p0, p1 = M0 * c0, M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & MASK, p1 & MASK, ((p0 >> 32) ^ c3 ^ k1) & MASK, p0 & MASK
        k0, k1 = (k0 + W0) & MASK, (k1 + W1) & MASK
    return c0, c1, c2, c3


def block(seed: int, tag: int, n: int):
    """Block n of stream `tag` under `seed`: counter (n, n >> 32, tag, 0),
    key (seed, seed >> 32) -- the library's stream layout."""
    return philox4x32_10((n & MASK, (n >> 32) & MASK, tag & MASK, 0), (seed & MASK, (seed >> 32) & MASK))
