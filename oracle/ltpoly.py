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

The bivariate circuit (Sec. 2.1; the univariate one needs digits below
(p+1)/2, the bivariate one works on full digits in [0, p)): LT(X, Y) =
sum_{a,b} c[a][b] X^a Y^b, the unique polynomial of degree <= p-1 in each
variable with LT(x, y) = [x < y] on Z_p x Z_p, i.e. sum over x < y of
L_x(X) L_y(Y) with L_v the Lagrange basis polynomial of the point v.  Pinned
by evaluation at every pair (x, y) for small p and at sampled pairs for large p.
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


def lagrange_basis(p: int, v: int) -> list:
    """Coefficients of L_v(Z) = prod_{u != v} (Z - u) / (v - u) over Z_p."""
    basis, den = [1], 1
    for u in range(p):
        if u == v:
            continue
        nxt = [0] * (len(basis) + 1)
        for i, c in enumerate(basis):
            nxt[i + 1] = (nxt[i + 1] + c) % p
            nxt[i] = (nxt[i] - u * c) % p
        basis = nxt
        den = den * (v - u) % p
    inv = pow(den, p - 2, p)
    return [c * inv % p for c in basis] + [0] * (p - len(basis))


def lt_bivariate_coefficients(p: int) -> list:
    """c[a][b] with sum c[a][b] x^a y^b = [x < y] for x, y in Z_p (as 0..p-1)."""
    L = [lagrange_basis(p, v) for v in range(p)]
    # sum_{x<y} L_x (X) L_y (Y) = sum_x L_x(X) (sum_{y>x} L_y(Y))
    suffix = [0] * p
    c = [[0] * p for _ in range(p)]
    for x in range(p - 1, -1, -1):
        for a in range(p):
            if L[x][a]:
                for b in range(p):
                    if suffix[b]:
                        c[a][b] = (c[a][b] + L[x][a] * suffix[b]) % p
        for b in range(p):
            suffix[b] = (suffix[b] + L[x][b]) % p
    return c


def evaluate_bivariate(c, x: int, y: int, p: int) -> int:
    acc = 0
    for a in reversed(range(p)):
        inner = 0
        for b in reversed(range(p)):
            inner = (inner * y + c[a][b]) % p
        acc = (acc * x + inner) % p
    return acc
