"""Pins of the oracle's BGV operations.

Checked against properties computed here with Python big integers (CRT), not
against the oracle's own formulas: basis conversion gives X + u Q with small
u; modulus switching and ModDown divide exactly and keep the plaintext; key
switching gives x s' + p * (small); every operation decrypts to the plaintext
result; the noise stays below q_0 / 2.
"""
import random

import numpy as np
import pytest

from oracle.circuits import Evaluator
from tests.oracle_setup import OracleSetup
from tests.params import CHAIN36, CHAIN50


def crt(residues, primes):
    Q = 1
    for q in primes:
        Q *= q
    x = 0
    for r, q in zip(residues, primes):
        Qi = Q // q
        x += int(r) * Qi * pow(Qi % q, -1, q)
    return x % Q, Q


def centred(x, Q):
    x %= Q
    return x - Q if x > Q // 2 else x


@pytest.fixture(scope="module")
def small17():
    return OracleSetup(logN=6, p=17, L=4, K=2, seed=11, galois=(5, 127), **CHAIN50)


def test_fbc_is_crt_plus_small_multiple(small17):
    o = small17.o
    g = np.random.default_rng(1)
    src, dst = [1, 2], [0, 3, 4, 5]
    x = np.stack([g.integers(0, o.primes[i], size=o.N, dtype=np.uint64) for i in src])
    y = o.fbc(x, src, dst)
    qs = [o.primes[i] for i in src]
    qd = [o.primes[i] for i in dst]
    QS = qs[0] * qs[1]
    us = set()
    for n in range(o.N):
        X, _ = crt([x[a][n] for a in range(2)], qs)
        Y, T = crt([y[b][n] for b in range(4)], qd)
        assert T > 2 * QS
        assert (Y - X) % QS == 0
        u = (Y - X) // QS
        assert 0 <= u < 2
        us.add(u)
    assert us == {0, 1}  # both overflow counts occur on random inputs


def test_encrypt_decrypt(small17):
    st = small17
    rnd = random.Random(2)
    vals = [[rnd.randrange(17) for _ in range(st.ss.ns)] for _ in range(3)]
    for v, ct in zip(vals, st.encrypt_slots(vals, seed=5)):
        assert st.decrypt_slots(ct) == v
        assert st.o.noise_bits(ct, st.s) < 30


def test_modswitch_divides_exactly_and_keeps_plaintext(small17):
    st, o = small17, small17.o
    ct = st.encrypt_slots([[3] * st.ss.ns], seed=6)[0]
    out = o.modswitch(ct)
    ql = o.primes[ct.level - 1]
    for k in range(2):
        for n in range(0, o.N, 7):
            X, Q = crt([ct.data[k, i, n] for i in range(ct.level)], o.primes[: ct.level])
            Xp, _ = crt([out.data[k, i, n] for i in range(out.level)], o.primes[: out.level])
            D = (X - Xp * ql) % Q  # the integer delta that was removed
            assert D % st.p == 0 and D % ql == X % ql and 0 <= D < st.p * ql
    assert st.decrypt_slots(out) == [3] * st.ss.ns
    # decryption residues at the new level are those of the old level
    # divided by q_l, up to the removed delta (same message mod p)
    assert st.o.decrypt_coeffs(out, st.s).tolist() == st.o.decrypt_coeffs(ct, st.s).tolist()


def test_keyswitch_gives_x_sprime_plus_p_small(small17):
    st, o = small17, small17.o
    g = np.random.default_rng(3)
    for level in (4, 3, 1):
        x = np.stack([g.integers(0, o.primes[i], size=o.N, dtype=np.uint64) for i in range(level)])
        out = o.keyswitch(x, level, st.rlk)
        s2 = o.polymul_int(st.s, st.s)
        res = []
        for i in range(level):
            q = o.primes[i]
            sq = np.array([v % q for v in st.s.tolist()], dtype=np.uint64)
            s2q = np.array([v % q for v in s2.tolist()], dtype=np.uint64)
            t = (o.polymul(i, out[1, i], sq).astype(object) + out[0, i].astype(object)
                 - o.polymul(i, x[i], s2q).astype(object)) % q
            res.append(t)
        for n in range(o.N):
            E, Q = crt([res[i][n] for i in range(level)], o.primes[:level])
            e = centred(E, Q)
            assert e % st.p == 0
            assert abs(e) < 2 ** 40


def test_tensor_relin_mul_decrypt(small17):
    st = small17
    ev = st.evaluator()
    rnd = random.Random(4)
    a = [rnd.randrange(17) for _ in range(st.ss.ns)]
    b = [rnd.randrange(17) for _ in range(st.ss.ns)]
    ca, cb = st.encrypt_slots([a, b], seed=7)
    c = ev.mul(ca, cb)
    assert c.level == 3
    assert st.decrypt_slots(c) == [(x * y) % 17 for x, y in zip(a, b)]
    assert st.decrypt_slots(ev.add(c, ca)) == [(x * y + x) % 17 for x, y in zip(a, b)]
    assert st.decrypt_slots(ev.sub(ca, cb)) == [(x - y) % 17 for x, y in zip(a, b)]
    assert st.decrypt_slots(ev.mul_const(ca, 16)) == [(16 * x) % 17 for x in a]
    assert st.decrypt_slots(ev.add_const(ca, 5)) == [(x + 5) % 17 for x in a]
    assert st.decrypt_slots(ev.neg(cb)) == [(-x) % 17 for x in b]


def test_rotation_decrypts_to_rotated_slots(small17):
    st = small17
    ev = st.evaluator()
    v = list(range(1, st.ss.ns + 1))
    ct = st.encrypt_slots([v], seed=8)[0]
    cols = st.ss.M // 2
    r5 = st.decrypt_slots(ev.rotate(ct, 5))
    assert r5 == [v[r * cols + (c + 1) % cols] for r in range(2) for c in range(cols)]
    rs = st.decrypt_slots(ev.rotate(ct, 2 * st.N - 1))
    assert rs == v[cols:] + v[:cols]


class _Lv:
    def __init__(self, level, npoly=2):
        self.level, self.npoly = level, npoly


class LevelOnly:
    """Stand-in backend that tracks levels only (for schedule counting)."""

    def __init__(self, p, L):
        self.p, self.L = p, L

    def modswitch(self, a):
        assert a.level > 1
        return _Lv(a.level - 1, a.npoly)

    def tensor(self, a, b):
        assert a.level == b.level
        return _Lv(a.level, 3)

    def relin(self, d, rlk):
        return _Lv(d.level, 2)

    def add(self, a, b):
        assert a.level == b.level
        return _Lv(a.level)

    sub = add

    def neg(self, a):
        return _Lv(a.level)

    def mul_const(self, a, c):
        return _Lv(a.level)

    def add_const(self, a, c):
        return _Lv(a.level)


@pytest.mark.parametrize("p,mults,depth", [(17, 8, 4), (131, 23, 8), (257, 30, 8)])
def test_ps_schedule_counts(p, mults, depth):
    L = 30
    ev = Evaluator(LevelOnly(p, L), None)
    lt, eq = ev.digit(_Lv(L), _Lv(L), True, True)
    assert ev.mul_count() == mults
    assert L - lt.level == depth and L - eq.level == depth
    # order of the univariate cost sqrt(p-3) + O(log p) (Sec. 1): well below
    # the bivariate 2p - 6 for the larger p
    assert mults < 2 * p - 6 or p < 20


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_merge_counts(d):
    # d-1 pair nodes; each computes L_hi + E_hi L_lo and, except at the root
    # when EQ is not wanted, E_hi E_lo
    p, L = 17, 40
    ev = Evaluator(LevelOnly(p, L), None)
    xs = [_Lv(L) for _ in range(d)]
    ev.compare(xs, xs, True, False)
    assert ev.mul_count() == 8 * d + max(0, 2 * (d - 1) - 1)
    ev2 = Evaluator(LevelOnly(p, L), None)
    ev2.compare(xs, xs, True, True)
    assert ev2.mul_count() == 8 * d + 2 * (d - 1)
    ev3 = Evaluator(LevelOnly(p, L), None)
    ev3.compare(xs, xs, False, True)
    assert ev3.mul_count() == 4 * d + (d - 1)  # z^16 by four squarings per digit


def _compare_case(st, d, count, seed):
    rnd = random.Random(seed)
    b = (st.p + 1) // 2
    ns = st.ss.ns
    xs_v = [[rnd.randrange(b ** d) for _ in range(ns)] for _ in range(count)]
    ys_v = [[rnd.randrange(b ** d) if rnd.random() < 0.7 else xs_v[c][s] for s in range(ns)] for c in range(count)]
    return xs_v, ys_v


def _digits(vals, b, d):
    return [[(v // b ** k) % b for v in vals] for k in range(d)]


@pytest.mark.parametrize("p,d,L", [(17, 2, 6), (131, 1, 9)])
def test_compare_lt_eq_small_ring(p, d, L):
    st = OracleSetup(logN=8, p=p, L=L, K=2, seed=21, **CHAIN50)
    b = (p + 1) // 2
    xs_v, ys_v = _compare_case(st, d, 1, seed=p)
    x = st.encrypt_slots(_digits(xs_v[0], b, d), seed=30)
    y = st.encrypt_slots(_digits(ys_v[0], b, d), seed=31)
    ev = st.evaluator()
    lt, eq = ev.compare(x, y, True, True)
    assert st.decrypt_slots(lt) == [int(a < c) for a, c in zip(xs_v[0], ys_v[0])]
    assert st.decrypt_slots(eq) == [int(a == c) for a, c in zip(xs_v[0], ys_v[0])]
    assert st.o.noise_bits(lt, st.s) < np.log2(st.o.primes[0]) - 1


def test_max_min_small_ring():
    p, d = 17, 2
    st = OracleSetup(logN=8, p=p, L=8, K=2, seed=22, **CHAIN50)
    b = (p + 1) // 2
    xs_v, ys_v = _compare_case(st, d, 1, seed=3)
    x = st.encrypt_slots(_digits(xs_v[0], b, d), seed=40)
    y = st.encrypt_slots(_digits(ys_v[0], b, d), seed=41)
    ev = st.evaluator()
    mx, mn = ev.max_min(x, y)
    got_max = [sum(st.decrypt_slots(mx[k])[s] * b ** k for k in range(d)) for s in range(st.ss.ns)]
    got_min = [sum(st.decrypt_slots(mn[k])[s] * b ** k for k in range(d)) for s in range(st.ss.ns)]
    assert got_max == [max(a, c) for a, c in zip(xs_v[0], ys_v[0])]
    assert got_min == [min(a, c) for a, c in zip(xs_v[0], ys_v[0])]


def test_small_config_full_size_lt():
    """N=2^12, p=17, d=1, 4 x 36-bit primes + 1 special: one encrypted LT of
    two packed ciphertexts, decrypted against plaintext, noise below q0/2."""
    st = OracleSetup(logN=12, p=17, L=4, K=1, seed=1, **CHAIN36)
    rnd = random.Random(1)
    xv = [rnd.randrange(9) for _ in range(st.ss.ns)]
    yv = [rnd.randrange(9) for _ in range(st.ss.ns)]
    x = st.encrypt_slots([xv], seed=2)
    y = st.encrypt_slots([yv], seed=3)
    ev = st.evaluator()
    lt = ev.compare_lt(x, y)
    assert st.decrypt_slots(lt) == [int(a < c) for a, c in zip(xv, yv)]
    nb = st.o.noise_bits(lt, st.s)
    assert nb < np.log2(st.o.primes[0]) - 1, nb


def test_compare_bivariate_full_digits_small_ring():
    """Full digits in [0, p): the bivariate circuit's LT and EQ decrypt to
    the plaintext comparison of values in [0, p^d), with noise below q0/2;
    the product count follows the schedule (x and y powers 2..p-1, one
    product per row a >= 1 with y terms, the EQ power, the merge)."""
    from oracle.ltpoly import lt_bivariate_coefficients

    p, d = 17, 2
    st = OracleSetup(logN=8, p=p, L=8, K=2, seed=23, **CHAIN50)
    rnd = random.Random(17)
    ns = st.ss.ns
    xs_v = [rnd.randrange(p ** d) for _ in range(ns)]
    ys_v = [rnd.randrange(p ** d) if rnd.random() < 0.7 else xs_v[s] for s in range(ns)]
    x = st.encrypt_slots(_digits(xs_v, p, d), seed=50)
    y = st.encrypt_slots(_digits(ys_v, p, d), seed=51)
    ev = st.evaluator()
    lt, eq = ev.compare(x, y, True, True, bivariate=True)
    assert st.decrypt_slots(lt) == [int(a < c) for a, c in zip(xs_v, ys_v)]
    assert st.decrypt_slots(eq) == [int(a == c) for a, c in zip(xs_v, ys_v)]
    assert st.o.noise_bits(lt, st.s) < np.log2(st.o.primes[0]) - 1
    c = lt_bivariate_coefficients(p)
    rows = sum(1 for a in range(1, p) if any(c[a][1:]))
    per_digit = 2 * (p - 2) + rows + 4  # powers of x and y, row products, z^16 by four squarings
    assert ev.mul_count() == d * per_digit + 2 * (d - 1)


def test_plaintext_operands():
    """ct + pt, ct - pt and ct * pt decrypt to the slot-wise sum, difference
    and product mod p."""
    p = 17
    st = OracleSetup(logN=8, p=p, L=3, K=2, seed=24, **CHAIN50)
    ns = st.ss.ns
    rnd = random.Random(2)
    a = [rnd.randrange(p) for _ in range(ns)]
    v = [rnd.randrange(p) for _ in range(ns)]
    x = st.encrypt_slots([a], seed=60)[0]
    ev = st.evaluator()
    assert st.decrypt_slots(ev.add_plain(x, v)) == [(u + w) % p for u, w in zip(a, v)]
    assert st.decrypt_slots(ev.sub_plain(x, v)) == [(u - w) % p for u, w in zip(a, v)]
    assert st.decrypt_slots(ev.mul_plain(x, v)) == [(u * w) % p for u, w in zip(a, v)]
    assert [t[0] for t in ev.trace] == ["padd", "psub", "pmul"]


def test_sort_rows_small_ring():
    """Every row of cols = 4 values (2 digits of base 9, ties included)
    comes out in increasing order."""
    from oracle.circuits import sort_galois, sort_rows

    p, d = 17, 2
    N = 2 ** 8
    st = OracleSetup(logN=8, p=p, L=11, K=2, seed=25, galois=sort_galois(p, N), **CHAIN50)
    ns = st.ss.ns
    b = (p + 1) // 2
    rnd = random.Random(4)
    vals = [rnd.randrange(b ** d) for _ in range(ns)]
    vals[1] = vals[2]  # a tie in row 0
    x = [st.encrypt_slots([dg], seed=70 + k)[0] for k, dg in enumerate(_digits(vals, b, d))]
    ev = st.evaluator()
    out = sort_rows(ev, x)
    got = [sum(st.decrypt_slots(out[k])[s] * b ** k for k in range(d)) for s in range(ns)]
    cols = ns // 2
    assert got == sorted(vals[:cols]) + sorted(vals[cols:])
    assert st.o.noise_bits(out[0], st.s) < np.log2(st.o.primes[0]) - 1


def test_sort_joint_sixteen_values():
    """Sixteen values (the paper's sort size) in row 0 of four ciphertexts of
    the p = 17 ring (4 columns each), ties across ciphertexts included: row r
    of the outputs, read in ciphertext order, is the sorted sequence of row r
    of the inputs; and one ciphertext reduces to the row sort."""
    from oracle.circuits import sort_galois, sort_joint, sort_rows

    p, d = 17, 2
    N = 2 ** 8
    st = OracleSetup(logN=8, p=p, L=11, K=2, seed=27, galois=sort_galois(p, N), **CHAIN50)
    ns = st.ss.ns
    cols = ns // 2
    b = (p + 1) // 2
    rnd = random.Random(6)
    K = 4
    vals = [[rnd.randrange(b ** d) for _ in range(ns)] for _ in range(K)]
    vals[3][0] = vals[0][2]  # ties across ciphertexts, in both rows
    vals[2][5] = vals[1][4] = vals[0][7]
    cts = [[st.encrypt_slots([dg], seed=90 + 10 * a + k)[0] for k, dg in enumerate(_digits(vals[a], b, d))]
           for a in range(K)]
    ev = st.evaluator()
    out = sort_joint(ev, cts)
    dec = [[sum(st.decrypt_slots(out[t][k])[s] * b ** k for k in range(d)) for s in range(ns)] for t in range(K)]
    for r in range(2):
        seq = [vals[a][r * cols + c] for a in range(K) for c in range(cols)]
        got = [dec[t][r * cols + c] for t in range(K) for c in range(cols)]
        assert got == sorted(seq)
    one = sort_rows(st.evaluator(), cts[0])
    assert [st.decrypt_slots(x) for x in one] == [st.decrypt_slots(x) for x in sort_joint(st.evaluator(), [cts[0]])[0]]


def test_sort_ranks_longer_than_p():
    """Sequences longer than p (24 values per row at p = 17: six ciphertexts
    of 4 columns, ties included): the rank of every value (the number of
    values below it plus those equal to it at a lower index) decrypts to its
    plaintext rank mod p, and every entry of the comparison matrix to the
    plaintext comparison of its two values."""
    from oracle.circuits import sort_galois, sort_ranks

    p, d = 17, 1
    N = 2 ** 8
    st = OracleSetup(logN=8, p=p, L=8, K=2, seed=29, galois=sort_galois(p, N), **CHAIN50)
    ns = st.ss.ns
    cols = ns // 2
    b = (p + 1) // 2
    rnd = random.Random(8)
    K = 6
    vals = [[rnd.randrange(b) for _ in range(ns)] for _ in range(K)]
    vals[5][1] = vals[0][2]
    cts = [[st.encrypt_slots([vals[a]], seed=120 + a)[0]] for a in range(K)]
    ranks, matrix = sort_ranks(st.evaluator(), cts)
    assert len(matrix) == K * K * cols - K
    for r in range(2):
        seq = [vals[a][r * cols + c] for a in range(K) for c in range(cols)]
        assert len(seq) > p
        for a in range(K):
            got = st.decrypt_slots(ranks[a])
            for c in range(cols):
                i = a * cols + c
                want = sum(1 for j, v in enumerate(seq) if v < seq[i] or (v == seq[i] and j < i)) % p
                assert got[r * cols + c] == want
        for (a, bb, sh), lt in list(matrix.items())[:: 7]:
            got = st.decrypt_slots(lt)
            for c in range(cols):
                i, j = a * cols + c, bb * cols + (c + sh) % cols
                assert got[r * cols + c] == int(seq[j] < seq[i])


def _check_plan(ns, useful, n_out, pieces, dest):
    """The plan is a valid compaction: every useful slot lands exactly once,
    no two land on one output slot, and each piece moves its slots by one
    slot rotation (a column shift and an optional row swap)."""
    cols = ns // 2 if ns >= 2 else 1
    landed = [d for j, u_j in enumerate(useful) for d in (dest[j][u] for u in u_j)]
    assert -1 not in landed and len(set(landed)) == len(landed) and all(d < n_out * ns for d in landed)
    for j, o, src, s, b in pieces:
        for u in src:
            r, c = divmod(u, cols)
            assert dest[j][u] == o * ns + (r ^ b) * cols + (c + s) % cols


@pytest.mark.parametrize("ns", [2, 8, 128])
def test_slot_plan_structured_cases(ns):
    """Brute-force facts about the slot manager's placement: leading blocks
    concatenate in input order (one rotation each), strided inputs interleave
    (the convolution example, results in every fourth slot), full inputs
    stay where they are, and the output count is the fewest possible."""
    from oracle.circuits import slot_plan

    cols = ns // 2
    for used in [u for u in (1, 2, 4, cols, ns) if u <= ns and ns % u == 0]:
        k = ns // used
        useful = [list(range(used))] * k
        n_out, pieces, dest = slot_plan(ns, useful)
        _check_plan(ns, useful, n_out, pieces, dest)
        assert n_out == 1 and len(pieces) == k
        assert [dest[j][t] for j in range(k) for t in range(used)] == list(range(ns))
    if ns >= 8:
        useful = [[i for i in range(ns) if i % 4 == 3]] * 4
        n_out, pieces, dest = slot_plan(ns, useful)
        _check_plan(ns, useful, n_out, pieces, dest)
        assert n_out == 1 and len(pieces) == 4 and [pc[3] for pc in pieces] == [0, 1, 2, 3]
    useful = [list(range(ns))] * 3
    n_out, pieces, dest = slot_plan(ns, useful)
    assert n_out == 3 and all(pc[3] == 0 and pc[4] == 0 for pc in pieces)


def test_slot_plan_random_masks():
    """Random useful sets: the plan is valid and no output beyond the first
    opens while an earlier one could take a slot under some rotation."""
    from oracle.circuits import slot_plan

    rnd = random.Random(3)
    for ns in (2, 8, 16):
        for _ in range(30):
            useful = [sorted(rnd.sample(range(ns), rnd.randrange(0, ns + 1))) for _ in range(rnd.randrange(1, 6))]
            n_out, pieces, dest = slot_plan(ns, useful)
            _check_plan(ns, useful, n_out, pieces, dest)
            total = sum(len(u) for u in useful)
            assert (total + ns - 1) // ns <= n_out <= max(1, total) or total == 0
            for o in range(n_out - 1):  # every output but the last is full
                assert sum(1 for j, u_j in enumerate(useful) for u in u_j if dest[j][u] // ns == o) == ns


@pytest.mark.parametrize("p,kind", [(17, "lead1"), (17, "lead2"), (17, "stride4"), (17, "random"), (131, "lead1")])
def test_slot_pack_decrypts(p, kind):
    """Slot compaction on ciphertexts: the useful values (garbage elsewhere)
    decrypt at the slots the plan assigns them."""
    from oracle.circuits import slot_galois, slot_pack, slot_plan
    from oracle.encoding import SlotStructure

    N = 2 ** 8
    ns = SlotStructure(p, N).ns
    rnd = random.Random(p + len(kind))
    if kind.startswith("lead"):
        used = int(kind[4:])
        useful = [list(range(used))] * (ns // used)
    elif kind == "stride4":
        useful = [[i for i in range(ns) if i % 4 == 3]] * 4
    else:
        useful = [sorted(rnd.sample(range(ns), rnd.randrange(1, ns))) for _ in range(4)]
    n_out, pieces, dest = slot_plan(ns, useful)
    st = OracleSetup(logN=8, p=p, L=3, K=2, seed=26, galois=slot_galois(ns, N, pieces), **CHAIN50)
    rows = [[rnd.randrange(p) for _ in range(ns)] for _ in useful]
    cts = [st.encrypt_slots([r], seed=80 + j)[0] for j, r in enumerate(rows)]
    ev = st.evaluator()
    outs = slot_pack(ev, cts, useful)
    assert len(outs) == n_out
    got = [st.decrypt_slots(c) for c in outs]
    for j, u_j in enumerate(useful):
        for u in u_j:
            o, t = divmod(dest[j][u], ns)
            assert got[o][t] == rows[j][u]

def test_private_query_decrypts():
    """Straight-lined private query (Sec. 5.3): per slot, the answer is
    data + op1, data * op1 or data^3 as the encrypted query type selects
    (codes 1, 2, 3), and 0 for any other type."""
    from oracle.circuits import eq_const, private_query

    p = 17
    st = OracleSetup(logN=8, p=p, L=8, K=2, seed=51, **CHAIN50)
    ns = st.ss.ns
    rnd = random.Random(4)
    qv = [rnd.randrange(5) for _ in range(ns)]
    qv[:4] = [0, 1, 2, 3]
    dv = [rnd.randrange(p) for _ in range(ns)]
    ov = [rnd.randrange(p) for _ in range(ns)]
    q, data, op1 = (st.encrypt_slots([v], seed=60 + i)[0] for i, v in enumerate((qv, dv, ov)))
    ev = st.evaluator()
    assert st.decrypt_slots(eq_const(ev, q, 2)) == [int(v == 2) for v in qv]
    out = private_query(ev, q, data, op1, 3, (1, 2, 3))
    want = [((d + o) if t == 1 else (d * o) if t == 2 else d ** 3 if t == 3 else 0) % p
            for t, d, o in zip(qv, dv, ov)]
    assert st.decrypt_slots(out) == want
