"""The univariate less-than polynomial over Z_p.

TEST INFRASTRUCTURE ONLY (see the package docstring).

BoostCom Sec. 2.1 ("Non-arithmetic Comparison of uFHE-based BGV") compares
digits with the univariate circuit of the BGV comparison work it builds on:
for digits x, y in [0, (p-1)/2], x < y exactly when z = x - y (mod p) lies in
[(p+1)/2, p-1].  LT is therefore the function f(z) = [z >= (p+1)/2] on Z_p,
and as every function Z_p -> Z_p it is a unique polynomial of degree <= p-1.
The oracle computes it by Lagrange interpolation over the p points.
EQ = 1 - z^(p-1) (Fermat).

Pins (tests/test_oracle_ltpoly.py): f evaluated at every z in Z_p equals the
indicator; the only non-zero even coefficient is that of z^(p-1) and it equals
(p+1)/2; the coefficients for p = 17 match tests/golden/ltpoly_p17.txt.
"""
from __future__ import annotations


def lt_coefficients(p: int) -> list:
    """c_0 .. c_{p-1} of the interpolating polynomial of [z >= (p+1)/2]."""
    coeffs = [0] * p
    for a in range((p + 1) // 2, p):  # the points where f = 1
        basis, den = [1], 1  # prod_{b != a} (z - b), and prod (a - b)
        for b in range(p):
            if b == a:
                continue
            nxt = [0] * (len(basis) + 1)
            for i, c in enumerate(basis):
                nxt[i + 1] = (nxt[i + 1] + c) % p
                nxt[i] = (nxt[i] - b * c) % p
            basis = nxt
            den = den * (a - b) % p
        inv = pow(den, p - 2, p)
        for i in range(p):
            coeffs[i] = (coeffs[i] + basis[i] * inv) % p
    return coeffs


def evaluate(coeffs, z: int, p: int) -> int:
    acc = 0
    for c in reversed(coeffs):
        acc = (acc * z + c) % p
    return acc
