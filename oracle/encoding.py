"""Slot structure of F_p-valued plaintexts in Z_p[X]/(X^N+1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

BoostCom Sec. 2.1 ("Basics and arithmetic ops") packs many values into one
ciphertext through the ring isomorphism of the plaintext ring ("SIMD slots").
The paper uses non-power-of-two m; with m = 2N a power of two, X^N+1 splits
mod p into n_s = N / ord_{2N}(p) irreducible factors.  Each slot holds one
value of F_p (a constant of its slot field), which is all the comparison of
base-b digits needs.  Such plaintexts lie in the subring generated by
Y = X^(N/M), where
  * p = 1 (mod 4):  M = 2^(v2(p-1)-1) (= n_s) and Y^M+1 splits into linear
    factors Y - zeta^e, e odd mod 2M, zeta = g^((p-1)/2M), g the smallest
    primitive root mod p;  slot s = r*(M/2) + c holds m(zeta^e) with
    e = (-1)^r 5^c mod 2M, so sigma_5 rotates each row left by one and
    sigma_{2N-1} swaps the two rows;
  * p = 3 (mod 8):  M = 4, n_s = 2 and Y^4+1 = (Y^2+gY-1)(Y^2-gY-1) with
    g^2 = -2 (g the smaller root); slot k holds m mod the k-th factor.
Decoding checks that every coefficient outside the subring is zero.

Pins (tests/test_oracle_encoding.py): decode(encode(v)) = v; decode of a ring
product (schoolbook, mod p) is the slot-wise product; decode(sigma_5 m) is the
row rotation; n_s equals N / ord_{2N}(p) computed by brute force.
"""
from __future__ import annotations

import numpy as np


def _v2(x: int) -> int:
    v = 0
    while x % 2 == 0:
        x //= 2
        v += 1
    return v


def _smallest_primitive_root(p: int) -> int:
    fac, m, f = [], p - 1, 2
    while f * f <= m:
        if m % f == 0:
            fac.append(f)
            while m % f == 0:
                m //= f
        f += 1
    if m > 1:
        fac.append(m)
    g = 2
    while any(pow(g, (p - 1) // r, p) == 1 for r in fac):
        g += 1
    return g


class SlotStructure:
    def __init__(self, p: int, N: int):
        self.p, self.N = p, N
        if p % 4 == 1:
            self.kind = "linear"
            self.M = min(2 ** (_v2(p - 1) - 1), N)
            self.ns = self.M
            self.zeta = pow(_smallest_primitive_root(p), (p - 1) // (2 * self.M), p)
            half = self.M // 2 if self.M > 1 else 1
            rows = 2 if self.M > 1 else 1
            self.exps = []
            for r in range(rows):
                for c in range(half):
                    e = pow(5, c, 2 * self.M)
                    self.exps.append(e if r == 0 else (2 * self.M - e) % (2 * self.M))
        elif p % 8 == 3:
            self.kind = "quadratic"
            self.M, self.ns = 4, 2
            roots = sorted(x for x in range(p) if (x * x) % p == (p - 2) % p)
            self.gamma = roots[0]
        else:
            raise NotImplementedError("slot structure for p = 7 (mod 8) not provided")
        assert N % self.M == 0
        self.stride = N // self.M

    # -- F_p[Y]/(Y^M+1) <-> slots -------------------------------------------
    def decode_y(self, my) -> list:
        p, M = self.p, self.M
        my = [int(v) % p for v in my]
        if self.kind == "linear":
            out = []
            for e in self.exps:
                z = pow(self.zeta, e, p)
                acc, zz = 0, 1
                for j in range(M):
                    acc = (acc + my[j] * zz) % p
                    zz = zz * z % p
                out.append(acc)
            return out
        # quadratic: reduce m(Y) modulo Y^2 + sg*Y - 1 by Y^2 = 1 - sg*Y
        out = []
        for sg in (self.gamma, p - self.gamma):
            a0, a1 = 0, 0  # residue a0 + a1 Y
            pw0, pw1 = 1, 0  # Y^j mod the factor
            for j in range(M):
                a0 = (a0 + my[j] * pw0) % p
                a1 = (a1 + my[j] * pw1) % p
                # multiply (pw0 + pw1 Y) by Y: pw1 Y^2 + pw0 Y = pw1 (1 - sg Y) + pw0 Y
                pw0, pw1 = pw1 % p, (pw0 - sg * pw1) % p
            if a1 != 0:
                raise ValueError("plaintext is not a slot constant")
            out.append(a0)
        return out

    def encode_y(self, vals) -> list:
        p, M = self.p, self.M
        v = [int(x) % p for x in vals]
        assert len(v) == self.ns
        if self.kind == "linear":
            Minv = pow(M, -1, p)
            out = []
            for j in range(M):
                acc = 0
                for s, e in enumerate(self.exps):
                    acc = (acc + v[s] * pow(self.zeta, (-(e * j)) % (2 * M), p)) % p
                out.append(acc * Minv % p)
            return out
        # m = (v0+v1)/2 + (v0-v1)/2 * h,  h = -(Y + Y^3)/gamma  (1 mod f0, -1 mod f1)
        inv2, ig = pow(2, -1, p), pow(self.gamma, -1, p)
        c0 = (v[0] + v[1]) * inv2 % p
        c1 = (v[0] - v[1]) * inv2 % p
        h1 = (-ig) % p
        return [c0, c1 * h1 % p, 0, c1 * h1 % p]

    # -- full ring ------------------------------------------------------------
    def encode(self, vals) -> np.ndarray:
        """Plaintext coefficients (int64 [N], values in [0,p))."""
        my = self.encode_y(vals)
        m = np.zeros(self.N, dtype=np.int64)
        m[:: self.stride] = my
        return m

    def decode(self, coeffs) -> list:
        c = np.asarray(coeffs, dtype=np.int64) % self.p
        mask = np.ones(self.N, dtype=bool)
        mask[:: self.stride] = False
        if np.any(c[mask] != 0):
            raise ValueError("coefficients outside the slot subring are not zero")
        return self.decode_y(c[:: self.stride])
