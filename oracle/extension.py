"""F_{p^d}-valued slots and digit extraction ("mod extract").

TEST INFRASTRUCTURE ONLY (see the package docstring).

BoostCom Sec. 2.1 ("Non-arithmetic Comparison of uFHE-based BGV"): a wide
operand is decomposed into slots that each hold an element of the extension
field F_{p^d}; the mod-extract step then splits every slot element into its d
digits in F_p, each digit in a ciphertext of its own, before LT and EQ run per
digit.  The paper states what the step produces, not how it is evaluated; the
readings fixed here are:

  * slot fields: the F_p-slot structure (encoding.SlotStructure) has slot
    factors g_s of Y^M+1 (Y - zeta^e_s for p = 1 mod 4, Y^2 +- gamma Y - 1
    for p = 3 mod 8).  With e = d / deg(g_s) (a power of two) and
    Y' = X^(N/(M e)), the factors of Y'^(M e)+1 are f_s(Y') = g_s(Y'^e), one
    per slot and in the same slot order, each irreducible of degree d;
  * a d-digit value (a_0, .., a_{d-1}) is the slot element
    a_0 + a_1 Y' + .. + a_{d-1} Y'^(d-1) of F_p[Y']/(f_s); plaintexts are
    assembled by the Chinese remainder theorem over the f_s;
  * the automorphism sigma_p (X -> X^p) acts on every slot field as the
    Frobenius x -> x^p (p = p mod 2M e on Y'), so sigma_{p^t} raises to p^t;
  * digit k = Tr(lambda_k x) = sum_{t<d} lambda_k^(p^t) sigma_{p^t}(x), where
    lambda_0 .. lambda_{d-1} is the trace-dual basis of 1, Y', .., Y'^(d-1)
    (Tr(lambda_k Y'^j) = [k = j]); the result is an F_p constant in every
    slot, i.e. the ordinary F_p-slot encoding that the comparison takes.

Pins (tests/test_oracle_extension.py): the product of the f_s is Y'^(M e)+1
and each is irreducible (no factor of lower degree, by brute force over F_p for
small degrees); decode(encode(a)) = a; an encoding of F_p constants equals
SlotStructure.encode; the ring product of two encodings (schoolbook mod
X^N+1) decodes to the slot-wise field product; decode(sigma_p m) is the
slot-wise p-th power; Tr(lambda_k Y'^j) = [k = j]; and extraction on
ciphertexts decrypts to the digits.
"""
from __future__ import annotations

import numpy as np

from .encoding import SlotStructure


# -- polynomials over F_p: coefficient lists, lowest degree first ---------------
def _trim(a):
    a = list(a)
    while a and a[-1] == 0:
        a.pop()
    return a


def poly_mul(a, b, p):
    if not a or not b:
        return []
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] = (out[i + j] + x * y) % p
    return _trim(out)


def poly_divmod(a, f, p):
    """(quotient, remainder) of a by f (f's leading coefficient invertible)."""
    a = [v % p for v in a]
    f = _trim([v % p for v in f])
    inv_lead = pow(f[-1], -1, p)
    q = [0] * max(len(a) - len(f) + 1, 1)
    for i in range(len(a) - len(f), -1, -1):
        c = a[i + len(f) - 1] * inv_lead % p
        q[i] = c
        if c:
            for j, fj in enumerate(f):
                a[i + j] = (a[i + j] - c * fj) % p
    return _trim(q), _trim(a[: len(f) - 1])


def poly_mod(a, f, p):
    return poly_divmod(a, f, p)[1]


def poly_inv_mod(a, f, p):
    """a^-1 mod f by the extended Euclidean algorithm (gcd(a, f) = 1)."""
    r0, r1 = _trim([v % p for v in f]), poly_mod(a, f, p)
    s0, s1 = [], [1]
    while r1:
        q, r = poly_divmod(r0, r1, p)
        r0, r1 = r1, r
        qs = poly_mul(q, s1, p)
        n = max(len(s0), len(qs))
        s0, s1 = s1, _trim([((s0[i] if i < len(s0) else 0) - (qs[i] if i < len(qs) else 0)) % p
                            for i in range(n)])
    assert len(r0) == 1, "not invertible"
    c = pow(r0[0], -1, p)
    return poly_mod([v * c % p for v in s0], f, p)


class ExtSlots:
    """Slots holding F_{p^d} elements in the subring generated by
    Y' = X^(N/(M e))."""

    def __init__(self, p: int, N: int, d: int):
        self.ss = SlotStructure(p, N)
        self.p, self.N, self.d = p, N, d
        d0 = 1 if self.ss.kind == "linear" else 2
        e = d // d0
        if d < d0 or d % d0 or e & (e - 1) or self.ss.M * e > N:
            raise ValueError(f"no F_(p^{d}) slots for p = {p}, N = {N}")
        self.e, self.Me, self.ns = e, self.ss.M * e, self.ss.ns
        self.stride = N // self.Me
        if self.ss.kind == "linear":
            roots = [pow(self.ss.zeta, x, p) for x in self.ss.exps]
            self.factors = [[(-b) % p] + [0] * (e - 1) + [1] for b in roots]
        else:
            g = self.ss.gamma
            self.factors = [[p - 1] + [0] * (e - 1) + [sg] + [0] * (e - 1) + [1] for sg in (g, p - g)]
        self.F = [1] + [0] * (self.Me - 1) + [1]
        self.idem = []
        for f in self.factors:
            cof, r = poly_divmod(self.F, f, p)
            assert not r
            self.idem.append(poly_mod(poly_mul(cof, poly_inv_mod(cof, f, p), p), self.F, p))

    # -- one slot field ---------------------------------------------------------
    def fmul(self, s, a, b):
        return poly_mod(poly_mul(a, b, self.p), self.factors[s], self.p)

    def fpow(self, s, a, n):
        out, base = [1], poly_mod(a, self.factors[s], self.p)
        while n:
            if n & 1:
                out = self.fmul(s, out, base)
            base = self.fmul(s, base, base)
            n >>= 1
        return out

    def trace(self, s, a) -> int:
        acc = []
        for t in range(self.d):
            x = self.fpow(s, a, self.p ** t)
            acc = _trim([((acc[i] if i < len(acc) else 0) + (x[i] if i < len(x) else 0)) % self.p
                         for i in range(max(len(acc), len(x)))])
        assert len(acc) <= 1, "trace is not in F_p"
        return acc[0] if acc else 0

    def dual_basis(self, s):
        """lambda_k as coefficient lists: the inverse of the trace matrix
        T[i][j] = Tr(Y'^(i+j)) applied to the power basis."""
        p, d = self.p, self.d
        T = [[self.trace(s, [0] * (i + j) + [1]) for j in range(d)] for i in range(d)]
        # Gauss-Jordan inverse mod p
        A = [row[:] + [1 if i == k else 0 for k in range(d)] for i, row in enumerate(T)]
        for c in range(d):
            piv = next(r for r in range(c, d) if A[r][c])
            A[c], A[piv] = A[piv], A[c]
            iv = pow(A[c][c], -1, p)
            A[c] = [v * iv % p for v in A[c]]
            for r in range(d):
                if r != c and A[r][c]:
                    f = A[r][c]
                    A[r] = [(x - f * y) % p for x, y in zip(A[r], A[c])]
        Tinv = [row[d:] for row in A]
        return [_trim(Tinv[k]) for k in range(d)]

    # -- plaintexts ---------------------------------------------------------------
    def encode(self, elems) -> np.ndarray:
        """elems[s] = the d coordinates of slot s -> plaintext coefficients
        (int64 [N], values in [0, p))."""
        assert len(elems) == self.ns
        acc = [0] * self.Me
        for s, a in enumerate(elems):
            t = poly_mod(poly_mul(_trim([int(v) % self.p for v in a]), self.idem[s], self.p), self.F, self.p)
            for i, v in enumerate(t):
                acc[i] = (acc[i] + v) % self.p
        m = np.zeros(self.N, dtype=np.int64)
        m[:: self.stride] = acc
        return m

    def decode(self, coeffs):
        c = np.asarray(coeffs, dtype=np.int64) % self.p
        mask = np.ones(self.N, dtype=bool)
        mask[:: self.stride] = False
        if np.any(c[mask] != 0):
            raise ValueError("coefficients outside the extension-slot subring are not zero")
        my = [int(v) for v in c[:: self.stride]]
        out = []
        for f in self.factors:
            r = poly_mod(my, f, self.p)
            out.append(r + [0] * (self.d - len(r)))
        return out

    def galois(self) -> list:
        """sigma_{p^t} for t = 1 .. d-1."""
        return [pow(self.p, t, 2 * self.N) for t in range(1, self.d)]

    def extraction_plaintexts(self):
        """L[k][t]: plaintext whose slot s holds lambda_{k,s}^(p^t)."""
        duals = [self.dual_basis(s) for s in range(self.ns)]
        return [[self.encode([self.fpow(s, duals[s][k], self.p ** t) for s in range(self.ns)])
                 for t in range(self.d)] for k in range(self.d)]
