"""Seeded synthetic inputs for BGV comparison workloads.

This module is the only code that the CUDA path's tests, the benchmark and the
CPU oracle share.  It draws random numbers and nothing else: it holds none of
the method's arithmetic (no NTT, no modular products, no key or ciphertext
formulas).  Every random quantity the scheme consumes -- the secret, the
uniform masks, the Gaussian errors, the encryption randomness -- is drawn here
and passed to both sides as an explicit input.

Distributions (BGV over X^N+1, the usual RLWE choices):
  * secret s and encryption mask u: uniform ternary {-1, 0, 1};
  * errors e: rounded normal with sigma = 3.2, cut at |e| <= ceil(6 sigma) = 20;
  * uniform masks a: independent uniform residues in [0, q_i) per prime;
  * plaintext values: uniform integers in [0, b^d), split into d digits of
    base b, least significant digit first.
"""
from __future__ import annotations

import math

import numpy as np

SIGMA = 3.2
TAIL = math.ceil(6 * SIGMA)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def ternary(g: np.random.Generator, n: int) -> np.ndarray:
    """n values uniform in {-1, 0, 1} (int64)."""
    return g.integers(-1, 2, size=n, dtype=np.int64)


def gaussian(g: np.random.Generator, n: int, sigma: float = SIGMA) -> np.ndarray:
    """n rounded-normal integers, |e| <= ceil(6 sigma) (int64)."""
    e = np.rint(g.normal(0.0, sigma, size=n)).astype(np.int64)
    return np.clip(e, -TAIL, TAIL)


def uniform_mod(g: np.random.Generator, moduli, n: int) -> np.ndarray:
    """Array [len(moduli)][n] of uint64, row i uniform in [0, moduli[i])."""
    out = np.empty((len(moduli), n), dtype=np.uint64)
    for i, q in enumerate(moduli):
        out[i] = g.integers(0, int(q), size=n, dtype=np.uint64)
    return out


def values(g: np.random.Generator, count: int, hi: int) -> np.ndarray:
    """count integers uniform in [0, hi) (int64)."""
    return g.integers(0, hi, size=count, dtype=np.int64)


def values_with_duplicates(g: np.random.Generator, count: int, hi: int, dup_frac: float) -> np.ndarray:
    """count integers: round(count*(1-dup_frac)) fresh draws from [0,hi), the
    rest copies of earlier draws, then shuffled."""
    fresh = int(round(count * (1.0 - dup_frac)))
    v = g.integers(0, hi, size=fresh, dtype=np.int64)
    dups = v[g.integers(0, fresh, size=count - fresh)]
    out = np.concatenate([v, dups])
    g.shuffle(out)
    return out


def to_digits(v: np.ndarray, base: int, d: int) -> np.ndarray:
    """Split integers into d base-`base` digits, least significant first:
    returns int64 [d][len(v)]."""
    v = np.asarray(v, dtype=np.int64).copy()
    out = np.empty((d, v.size), dtype=np.int64)
    for k in range(d):
        out[k] = v % base
        v //= base
    return out


class KeyMaterial:
    """Every random draw that key generation consumes, for L data primes and
    K special primes, ring degree N, and `n_galois` rotation keys.

    s        ternary secret [N]
    a_pk, e_pk   public-key mask [L][N] (uniform mod q_i) and error [N]
    a_ksk, e_ksk switching-key masks [nkeys][dnum][L+K][N] and errors
                 [nkeys][dnum][N]; key 0 is relinearisation, keys 1.. are the
                 Galois keys in the order requested.
    """

    def __init__(self, seed: int, primes, L: int, K: int, N: int, n_galois: int = 0):
        g = rng(seed)
        dnum = -(-L // K)
        self.s = ternary(g, N)
        self.a_pk = uniform_mod(g, primes[:L], N)
        self.e_pk = gaussian(g, N)
        nkeys = 1 + n_galois
        self.a_ksk = np.empty((nkeys, dnum, L + K, N), dtype=np.uint64)
        self.e_ksk = np.empty((nkeys, dnum, N), dtype=np.int64)
        for k in range(nkeys):
            for j in range(dnum):
                self.a_ksk[k, j] = uniform_mod(g, primes[: L + K], N)
                self.e_ksk[k, j] = gaussian(g, N)


class EncRandomness:
    """Encryption randomness for `count` ciphertexts of degree N:
    u [count][N] ternary, e0 and e1 [count][N] Gaussian."""

    def __init__(self, seed: int, count: int, N: int):
        g = rng(seed)
        self.u = np.stack([ternary(g, N) for _ in range(count)])
        self.e0 = np.stack([gaussian(g, N) for _ in range(count)])
        self.e1 = np.stack([gaussian(g, N) for _ in range(count)])
