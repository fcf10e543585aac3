"""ctypes wrapper of bgv_oracle.c plus level bookkeeping.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A ciphertext is ``Ct(data, level)`` with ``data`` a uint64 array
[npoly][level][N] of coefficient-domain residues: limb i is reduced mod q_i.
The BGV scheme over R_Q = Z_Q[X]/(X^N+1) with Q held in RNS follows BoostCom
Sec. 2.1 ("Basics and arithmetic ops") and Sec. 2.2 ("Efficient Polynomial and
NTT"); the formulas of each step are in bgv_oracle.c.

Pins (tests/test_oracle_ring.py, tests/test_oracle_bgv.py): primes against an
independent primality test and the printed first primes; the NTT against its
O(N^2) definition in pure Python; products against the schoolbook negacyclic
product; INTT(NTT(a)) = a; FBC against exact big-integer CRT; ModDown and
modswitch by exact divisibility and unchanged plaintext; decryption of every
operation against the plaintext result.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import lib as _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Ct:
    data: np.ndarray  # uint64 [npoly][level][N]
    level: int

    @property
    def npoly(self) -> int:
        return self.data.shape[0]


class Oracle:
    """BGV context: ring degree 2^logN, plaintext modulus p, L data primes and
    K special primes, the smallest primes q = 1 (mod U) in [lo, hi)."""

    def __init__(self, logN: int, p: int, L: int, K: int, U: int, lo: int, hi: int):
        self.L_ = _lib()
        self.logN, self.N, self.p, self.L, self.K = logN, 1 << logN, p, L, K
        self.h = self.L_.orc_ctx_new(logN, p, L, K, U, lo, hi)
        if not self.h:
            raise ValueError("not enough primes for this chain")
        q = np.zeros(L + K, dtype=np.uint64)
        self.L_.orc_ctx_primes(self.h, _p(q))
        self.primes = [int(x) for x in q]

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L_.orc_ctx_free(h)
            self.h = None

    def dnum(self, level: int) -> int:
        return self.L_.orc_dnum(self.h, level)

    def psi(self, i: int) -> int:
        return int(self.L_.orc_ctx_psi(self.h, i))

    # ---- single-limb transforms -------------------------------------------
    def ntt(self, i: int, a) -> np.ndarray:
        x = np.array(a, dtype=np.uint64)
        self.L_.orc_ntt(self.h, i, _p(x))
        return x

    def intt(self, i: int, a) -> np.ndarray:
        x = np.array(a, dtype=np.uint64)
        self.L_.orc_intt(self.h, i, _p(x))
        return x

    def ntt_direct(self, i: int, a) -> np.ndarray:
        x = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.empty_like(x)
        self.L_.orc_ntt_direct(self.h, i, _p(x), _p(out))
        return out

    def polymul(self, i: int, a, b) -> np.ndarray:
        x = np.ascontiguousarray(a, dtype=np.uint64)
        y = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.empty_like(x)
        self.L_.orc_polymul(self.h, i, _p(x), _p(y), _p(out))
        return out

    def polymul_int(self, a, b) -> np.ndarray:
        x = np.ascontiguousarray(a, dtype=np.int64)
        y = np.ascontiguousarray(b, dtype=np.int64)
        out = np.empty_like(x)
        self.L_.orc_polymul_int(self.h, _p(x), _p(y), _p(out))
        return out

    def automorphism_int(self, a, g: int) -> np.ndarray:
        x = np.ascontiguousarray(a, dtype=np.int64)
        out = np.empty_like(x)
        self.L_.orc_automorphism_int(self.h, _p(x), g, _p(out))
        return out

    def fbc(self, x: np.ndarray, src, dst) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.uint64)
        s = np.array(src, dtype=np.int32)
        d = np.array(dst, dtype=np.int32)
        y = np.empty((len(dst), self.N), dtype=np.uint64)
        self.L_.orc_fbc(self.h, _p(x), _p(s), len(src), _p(d), len(dst), _p(y))
        return y

    # ---- keys --------------------------------------------------------------
    def keygen(self, s, a, e) -> np.ndarray:
        """pk [2][L][N] from the secret s, masks a [L][N] and error e."""
        s = np.ascontiguousarray(s, dtype=np.int64)
        a = np.ascontiguousarray(a, dtype=np.uint64)
        e = np.ascontiguousarray(e, dtype=np.int64)
        pk = np.empty((2, self.L, self.N), dtype=np.uint64)
        self.L_.orc_keygen(self.h, _p(s), _p(a), _p(e), _p(pk))
        return pk

    def ksk(self, s, sprime, a, e) -> np.ndarray:
        """Switching key s' -> s, [dnum][2][L+K][N]."""
        s = np.ascontiguousarray(s, dtype=np.int64)
        sp = np.ascontiguousarray(sprime, dtype=np.int64)
        a = np.ascontiguousarray(a, dtype=np.uint64)
        e = np.ascontiguousarray(e, dtype=np.int64)
        dn = self.dnum(self.L)
        assert a.shape == (dn, self.L + self.K, self.N) and e.shape == (dn, self.N)
        out = np.empty((dn, 2, self.L + self.K, self.N), dtype=np.uint64)
        self.L_.orc_ksk_gen(self.h, _p(s), _p(sp), _p(a), _p(e), _p(out))
        return out

    def relin_key(self, s, a, e) -> np.ndarray:
        return self.ksk(s, self.polymul_int(s, s), a, e)

    def galois_key(self, s, g: int, a, e) -> np.ndarray:
        return self.ksk(s, self.automorphism_int(s, g), a, e)

    # ---- encryption --------------------------------------------------------
    def encrypt(self, pk, m, u, e0, e1) -> Ct:
        """Encrypt the plaintext coefficient vector m (integers) at level L."""
        m = np.ascontiguousarray(m, dtype=np.int64)
        u = np.ascontiguousarray(u, dtype=np.int64)
        e0 = np.ascontiguousarray(e0, dtype=np.int64)
        e1 = np.ascontiguousarray(e1, dtype=np.int64)
        ct = np.empty((2, self.L, self.N), dtype=np.uint64)
        self.L_.orc_encrypt(self.h, _p(pk), _p(m), _p(u), _p(e0), _p(e1), _p(ct))
        return Ct(ct, self.L)

    def dot_sk(self, ct: Ct, s) -> np.ndarray:
        """Residues [level][N] of c0 + c1 s mod q_i."""
        s = np.ascontiguousarray(s, dtype=np.int64)
        out = np.empty((ct.level, self.N), dtype=np.uint64)
        self.L_.orc_dot_sk(self.h, _p(ct.data), ct.level, _p(s), _p(out))
        return out

    def decrypt_coeffs(self, ct: Ct, s) -> np.ndarray:
        """Plaintext coefficients in [0,p): modulus-switch a copy to one limb,
        take [c0 + c1 s]_{q0} centred, reduce mod p."""
        c = ct
        while c.level > 1:
            c = self.modswitch(c)
        t = self.dot_sk(c, s)[0].astype(object)
        q0 = self.primes[0]
        t = np.where(t > q0 // 2, t - q0, t)
        return np.array([int(v) % self.p for v in t], dtype=np.int64)

    def noise_bits(self, ct: Ct, s) -> float:
        """log2 of || [c0 + c1 s]_{Q_l} ||_inf (centred), by exact CRT."""
        r = self.dot_sk(ct, s)
        qs = self.primes[: ct.level]
        Q = 1
        for q in qs:
            Q *= q
        coefs = [0] * self.N
        for i, q in enumerate(qs):
            Qi = Q // q
            f = Qi * pow(Qi % q, -1, q)
            row = r[i]
            for n in range(self.N):
                coefs[n] += int(row[n]) * f
        mx = 0
        for v in coefs:
            v %= Q
            if v > Q // 2:
                v -= Q
            mx = max(mx, abs(v))
        import math

        return math.log2(mx) if mx else 0.0

    # ---- ciphertext arithmetic ----------------------------------------------
    def _new(self, npoly, level):
        return np.empty((npoly, level, self.N), dtype=np.uint64)

    def add(self, a: Ct, b: Ct) -> Ct:
        assert a.level == b.level and a.npoly == b.npoly
        out = self._new(a.npoly, a.level)
        self.L_.orc_add(self.h, _p(a.data), _p(b.data), a.level, a.npoly, _p(out))
        return Ct(out, a.level)

    def sub(self, a: Ct, b: Ct) -> Ct:
        assert a.level == b.level and a.npoly == b.npoly
        out = self._new(a.npoly, a.level)
        self.L_.orc_sub(self.h, _p(a.data), _p(b.data), a.level, a.npoly, _p(out))
        return Ct(out, a.level)

    def neg(self, a: Ct) -> Ct:
        out = self._new(a.npoly, a.level)
        self.L_.orc_neg(self.h, _p(a.data), a.level, a.npoly, _p(out))
        return Ct(out, a.level)

    def mul_const(self, a: Ct, k: int) -> Ct:
        out = self._new(a.npoly, a.level)
        self.L_.orc_mul_const(self.h, _p(a.data), int(k), a.level, a.npoly, _p(out))
        return Ct(out, a.level)

    def add_const(self, a: Ct, k: int) -> Ct:
        assert a.npoly == 2
        out = self._new(2, a.level)
        self.L_.orc_add_const(self.h, _p(a.data), int(k), a.level, _p(out))
        return Ct(out, a.level)

    # ---- plaintext operands (slot vectors encoded as polynomials) ---------------
    def _plain_limbs(self, m, level: int):
        """The plaintext coefficients (integers), centred into (-p/2, p/2],
        reduced mod every q_i of the level."""
        mc = [int(v) % self.p for v in m]
        mc = [v - self.p if v > self.p // 2 else v for v in mc]
        return [np.array([v % q for v in mc], dtype=np.uint64) for q in self.primes[:level]]

    def add_plain(self, a: Ct, m, sign: int = 1) -> Ct:
        """c0 +- m (m the plaintext coefficients)."""
        assert a.npoly == 2
        out = a.data.copy()
        for i, mi in enumerate(self._plain_limbs(m, a.level)):
            q = int(self.primes[i])
            c0 = out[0, i].astype(object)
            out[0, i] = np.array([(int(x) + sign * int(y)) % q for x, y in zip(c0, mi)], dtype=np.uint64)
        return Ct(out, a.level)

    def mul_plain(self, a: Ct, m) -> Ct:
        """Every polynomial times m in R_q (negacyclic product per limb)."""
        out = self._new(a.npoly, a.level)
        limbs = self._plain_limbs(m, a.level)
        for j in range(a.npoly):
            for i in range(a.level):
                out[j, i] = self.polymul(i, a.data[j, i], limbs[i])
        return Ct(out, a.level)

    def tensor(self, a: Ct, b: Ct) -> Ct:
        assert a.level == b.level and a.npoly == 2 and b.npoly == 2
        out = self._new(3, a.level)
        self.L_.orc_tensor(self.h, _p(a.data), _p(b.data), a.level, _p(out))
        return Ct(out, a.level)

    def keyswitch(self, x: np.ndarray, level: int, ksk: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.uint64)
        out = self._new(2, level)
        self.L_.orc_keyswitch(self.h, _p(x), level, _p(ksk), _p(out))
        return out

    def relin(self, d: Ct, rlk: np.ndarray) -> Ct:
        assert d.npoly == 3
        out = self._new(2, d.level)
        self.L_.orc_relin(self.h, _p(d.data), d.level, _p(rlk), _p(out))
        return Ct(out, d.level)

    def modswitch(self, a: Ct) -> Ct:
        assert a.level > 1
        out = self._new(a.npoly, a.level - 1)
        self.L_.orc_modswitch(self.h, _p(a.data), a.level, a.npoly, _p(out))
        return Ct(out, a.level - 1)

    def automorphism(self, a: Ct, g: int) -> Ct:
        out = self._new(a.npoly, a.level)
        self.L_.orc_automorphism(self.h, _p(a.data), a.level, a.npoly, g, _p(out))
        return Ct(out, a.level)

    def rotate(self, a: Ct, g: int, gk: np.ndarray) -> Ct:
        assert a.npoly == 2
        out = self._new(2, a.level)
        self.L_.orc_rotate(self.h, _p(a.data), a.level, g, _p(gk), _p(out))
        return Ct(out, a.level)
