"""Pins of the less-than polynomial: brute force over Z_p, its structure, an
independent power-sum formula for its coefficients, and the digit base that
Table 3 of the paper fixes for the univariate circuit."""
import os

import pytest

from oracle.ltpoly import evaluate, lt_coefficients

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("p", [5, 17, 131, 257])
def test_lt_brute_force(p):
    c = lt_coefficients(p)
    assert len(c) == p
    for z in range(p):
        assert evaluate(c, z, p) == (1 if z >= (p + 1) // 2 else 0)
    # as a digit comparison: for x, y in [0,(p-1)/2], f(x-y) = [x < y]
    h = (p - 1) // 2
    for x in range(0, h + 1, max(1, h // 16)):
        for y in range(0, h + 1):
            assert evaluate(c, (x - y) % p, p) == int(x < y)


@pytest.mark.parametrize("p", [5, 17, 131, 257])
def test_lt_structure(p):
    c = lt_coefficients(p)
    even = [i for i in range(0, p, 2) if c[i]]
    assert even == [p - 1]
    assert c[p - 1] == (p + 1) // 2


@pytest.mark.parametrize("p", [5, 17, 131])
def test_eq_by_fermat(p):
    for z in range(p):
        assert (1 - pow(z, p - 1, p)) % p == (1 if z == 0 else 0)


@pytest.mark.parametrize("p", [5, 17, 131, 257])
def test_lt_coefficients_by_power_sums(p):
    # Over F_p, sum_{z != 0} z^k = -1 if (p-1) | k else 0, so a function f
    # with f(0) = 0 has c_j = -sum_{z != 0} f(z) z^(p-1-j) for 1 <= j <= p-1.
    f = [1 if z >= (p + 1) // 2 else 0 for z in range(p)]
    want = [f[0]] + [(-sum(f[z] * pow(z, p - 1 - j, p) for z in range(1, p))) % p for j in range(1, p)]
    assert lt_coefficients(p) == want


def _table3():
    rows = []
    with open(os.path.join(HERE, "golden", "table3_params.txt")) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                name, p, m, N, circ, d, l, logq, lam, ints = ln.split()
                rows.append((name, int(p), circ, int(d), int(l)))
    return rows


def test_table3_digit_bases():
    # Every configuration compares 64-bit integers with d*l digits.  The
    # univariate rows reach 64 bits only with base (p+1)/2 digits -- the
    # domain [0,(p-1)/2] on which the univariate LT polynomial is exact -- and
    # the bivariate rows need the full base p.
    rows = _table3()
    assert len(rows) == 20
    for name, p, circ, d, l in rows:
        b = (p + 1) // 2
        if circ == "U":
            assert b ** (d * l) >= 2 ** 64, name
        else:
            assert p ** (d * l) >= 2 ** 64, name
            assert b ** (d * l) < 2 ** 64, name


@pytest.mark.parametrize("p", [3, 5, 7, 17])
def test_lt_bivariate_brute_force(p):
    """sum c[a][b] x^a y^b = [x < y] at every pair of Z_p (as 0..p-1)."""
    from oracle.ltpoly import evaluate_bivariate, lt_bivariate_coefficients

    c = lt_bivariate_coefficients(p)
    for x in range(p):
        for y in range(p):
            assert evaluate_bivariate(c, x, y, p) == int(x < y)


def test_lt_bivariate_sampled_large_p():
    import random

    from oracle.ltpoly import evaluate_bivariate, lt_bivariate_coefficients

    p = 131
    c = lt_bivariate_coefficients(p)
    rnd = random.Random(5)
    for _ in range(400):
        x, y = rnd.randrange(p), rnd.randrange(p)
        assert evaluate_bivariate(c, x, y, p) == int(x < y)
    for v in (0, 1, 64, 65, 129, 130):  # the edges of the order
        assert evaluate_bivariate(c, v, v, p) == 0
        assert evaluate_bivariate(c, v, (v + 1) % p, p) == int(v + 1 < p)


def test_lt_bivariate_by_indicator_expansion():
    """An independent construction: the point indicator at i is
    1 - (Z - i)^(p-1) (Fermat), expanded by the binomial theorem, and
    LT = sum_{i<j} 1_i(X) 1_j(Y).  Both constructions agree, the constant
    terms vanish and the a = 0 row is Y^(p-1)."""
    from math import comb

    from oracle.ltpoly import lt_bivariate_coefficients

    p = 17
    ind = []
    for i in range(p):
        # (Z - i)^(p-1) = sum_a C(p-1, a) Z^a (-i)^(p-1-a)
        row = [-(comb(p - 1, a) * pow(-i, p - 1 - a, p)) % p for a in range(p)]
        row[0] = (row[0] + 1) % p
        ind.append(row)
    want = [[0] * p for _ in range(p)]
    for i in range(p):
        for j in range(i + 1, p):
            for a in range(p):
                for b in range(p):
                    want[a][b] = (want[a][b] + ind[i][a] * ind[j][b]) % p
    c = lt_bivariate_coefficients(p)
    assert c == want
    assert all(c[a][0] == 0 for a in range(p))
    assert c[0] == [0] * (p - 1) + [1]


def _golden(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return [int(s) for s in (line.split("#")[0].strip() for line in f) if s]


def test_lt_p17_worked_example():
    """The hand-worked p = 17 coefficients: first checked on their own (at
    every z in Z_17, and the structure the leading term fixes), then the
    oracle must reproduce them exactly."""
    want = _golden("ltpoly_p17.txt")
    p = 17
    assert len(want) == p
    for z in range(p):
        assert evaluate(want, z, p) == (1 if z >= (p + 1) // 2 else 0)
    assert want[p - 1] == (p + 1) // 2
    assert lt_coefficients(p) == want
