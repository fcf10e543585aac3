"""Comparison circuits over the oracle's BGV operations.

TEST INFRASTRUCTURE ONLY (see the package docstring).

BoostCom Sec. 2.1 ("Non-arithmetic Comparison of uFHE-based BGV"): operands
are split into digits; LT and EQ are computed for every digit independently
("the computation of LT and EQ for each digit is independent"), and the digit
results are combined in lexicographic order into an encryption of 1 when
a < b and 0 otherwise.  The univariate circuit is used (Table 3 lists both;
its digit bases (p+1)/2 are what make 64-bit operands out of the listed
(d, l) pairs).  The paper gives no evaluation schedule; the readings fixed here
(and mirrored exactly by the CUDA path, since bit-exact agreement depends on
them) are:

  * levels: every ciphertext product is tensor -> relinearise -> modulus
    switch by one prime when the level is > 1; an operand at a higher level is
    first switched down, one prime at a time, to the other operand's level
    (lowered copies are cached); additions align the same way;
  * scalar constants c in Z_p are lifted to the centred representative in
    (-p/2, p/2];
  * powers z^n: n = 1 is z; n a power of two squares z^(n/2); otherwise
    z^(2^a) * z^(n-2^a) with 2^a the largest power of two below n;
  * Paterson-Stockmeyer for f(z) = c_{p-1} z^(p-1) + O(z), O odd: baby odd
    powers z^1 .. z^(B-1), B = 2^b, b = ceil(log2(p-1) / 2); block k of O is
    the leaf L_k(z) = sum_{odd r < B} c_{Bk+r} z^r (terms with c = 0
    skipped); blocks are combined by  E(k0,t) = E(k0,t-1) + z^(B 2^(t-1)) *
    E(k0 + 2^(t-1), t-1), an empty half dropping its product or sum;
  * per digit: z = x_k - y_k; LT_k = f(z); EQ_k = 1 - z^(p-1);
  * merge: digits (least significant first) are paired (2i+1, 2i) ->
    (L_hi + E_hi L_lo, E_hi E_lo), an odd last node passes up unchanged, and
    the root computes the E product only when EQ is wanted;
  * max/min: L = LT(x, y); t_k = L (y_k - x_k); max_k = x_k + t_k,
    min_k = y_k - t_k (equal operands give the common value);
  * tournament over n ciphertexts (each digit a list of n): cross rounds
    pair ciphertexts [0, h) with [h, 2h), h = n // 2, an odd last one
    passing on after the winners; then in-slot rounds x <- sel(x, rot(x))
    with the column rotations sigma_{5^(2^i)} for 2^i = cols/2, .., 1
    (cols = n_s / 2), then the row swap sigma_{2N-1}.  When max and min
    are both wanted the first cross round shares one LT; afterwards the two
    tournaments run separately.  Before a round whose depth
    (ceil(log2(p-1)) + ceil(log2 d) + 1) would leave less than one level,
    every ciphertext is refreshed (a stand-in for bootstrapping).

  * bivariate digits (full range [0, p)): powers x^n, y^n by the same rule,
    computed when first needed; for a = 0 .. p-1 in order, rows with a
    non-zero c[a][b] give h_a = sum_b c[a][b] y^b (b >= 1; the coefficients
    have no constant terms) at the level of the lowest power used, and the
    term x^a h_a (for a = 0 the term is h_a), accumulated in order of a;
    EQ_k = 1 - (x - y)^(p-1);

  * plaintext operands (slot vectors) are encoded and their coefficients
    lifted to (-p/2, p/2] before reduction mod q_i; ct + pt and ct - pt touch
    c0 only, ct * pt multiplies both polynomials; no level is consumed;
  * sorting (p = 1 mod 4, the rows of cols = n_s / 2 columns sorted
    independently): rank_i = sum_{s=1}^{cols-1} (LT(x_{i+s}, x_i) +
    w_s[i] EQ(x_{i+s}, x_i)) with x_{i+s} = sigma_{5^s}(x) and the tie-break
    mask w_s[i] = [i + s >= cols] (equal values keep their order); then
    out = sum_{s=0}^{cols-1} EQ(sigma_{5^s}(rank) - idx) sigma_{5^s}(x) per
    digit (idx[i] = i, EQ(u) = 1 - u^(p-1)), shifts in increasing order;

  * slot compaction (the slot manager): each input comes with the list of
    its useful slots (index r cols + c, cols = n_s / 2 columns per row; the
    two single-slot rows of p = 3 mod 8 have cols = 1).  Inputs are placed in
    order; the slots still to place go, under the slot rotation (column
    shift right by s, rows swapped when b) and into the output that takes
    the most of them, the first such (output, b, s) in that order winning a
    tie; a new output opens when none has room.  A piece is evaluated as
    mask (a plaintext product), sigma_{5^(cols - s)} when s > 0,
    sigma_{2N-1} when b, and an addition into its output, pieces in plan
    order;

  * digit extraction from F_{p^d} slots: extension.py states the reading;
    the ciphertext's Frobenius images sigma_{p^t}(ct), t = 1 .. d-1, are
    taken first, in order of t; digit k is then the sum over t (ascending)
    of their products with the plaintexts lambda_k^(p^t);

  * private query (non-blocking comparison application): EQ(q, k) for a
    public code k is 1 - (q - k)^(p-1) with z = q + (-k) (a constant
    addition) and the power rule above; the three EQs come first, in code
    order, then data + op1, data * op1, data^op2 (power rule), then
    ((r1 c1 + r2 c2) + r3 c3);

Every operation appends (name, level) to ``trace``; the CUDA path emits the
same trace, and a test compares them.  The multiplication count is pinned
against the Paterson-Stockmeyer count (8 / 23 / 30 for p = 17 / 131 / 257) and
the depth against ceil(log2(p-1)).
"""
from __future__ import annotations

from .bgv import Ct, Oracle
from .encoding import SlotStructure
from .ltpoly import lt_bivariate_coefficients, lt_coefficients


def centred(c: int, p: int) -> int:
    c %= p
    return c - p if c > p // 2 else c


def baby_log(p: int) -> int:
    """b = ceil(log2(p-1) / 2)."""
    lg = (p - 2).bit_length()  # ceil(log2(p-1)) for p >= 3
    return (lg + 1) // 2


class Evaluator:
    def __init__(self, orc: Oracle, rlk, galois_keys=None):
        self.o = orc
        self.p = orc.p
        self.rlk = rlk
        self.gk = dict(galois_keys or {})
        self.trace = []
        self._lowered = {}

    # ---- level alignment -----------------------------------------------------
    def lower(self, ct: Ct, level: int) -> Ct:
        if ct.level == level:
            return ct
        assert ct.level > level >= 1
        key = (id(ct), level)
        hit = self._lowered.get(key)
        if hit is not None:
            return hit[1]
        above = self.lower(ct, level + 1)
        out = self.o.modswitch(above)
        self._lowered[key] = (ct, out)  # keep ct alive so id() stays unique
        return out

    def _align(self, a: Ct, b: Ct):
        lv = min(a.level, b.level)
        return self.lower(a, lv), self.lower(b, lv), lv

    # ---- traced operations ---------------------------------------------------
    def mul(self, a: Ct, b: Ct) -> Ct:
        a2, b2, lv = self._align(a, b)
        c = self.o.relin(self.o.tensor(a2, b2), self.rlk)
        if lv > 1:
            c = self.o.modswitch(c)
        self.trace.append(("mul", lv))
        return c

    def add(self, a: Ct, b: Ct) -> Ct:
        a2, b2, lv = self._align(a, b)
        self.trace.append(("add", lv))
        return self.o.add(a2, b2)

    def sub(self, a: Ct, b: Ct) -> Ct:
        a2, b2, lv = self._align(a, b)
        self.trace.append(("sub", lv))
        return self.o.sub(a2, b2)

    def mul_const(self, a: Ct, c: int) -> Ct:
        self.trace.append(("cmul", a.level))
        return self.o.mul_const(a, centred(c, self.p))

    def add_const(self, a: Ct, c: int) -> Ct:
        self.trace.append(("cadd", a.level))
        return self.o.add_const(a, centred(c, self.p))

    def neg(self, a: Ct) -> Ct:
        self.trace.append(("neg", a.level))
        return self.o.neg(a)

    def rotate(self, a: Ct, g: int) -> Ct:
        self.trace.append(("rot", a.level))
        return self.o.rotate(a, g, self.gk[g])

    def _slots(self) -> SlotStructure:
        if not hasattr(self, "_ss"):
            self._ss = SlotStructure(self.p, self.o.N)
        return self._ss

    def add_plain(self, a: Ct, slots) -> Ct:
        self.trace.append(("padd", a.level))
        return self.o.add_plain(a, self._slots().encode(slots), 1)

    def sub_plain(self, a: Ct, slots) -> Ct:
        self.trace.append(("psub", a.level))
        return self.o.add_plain(a, self._slots().encode(slots), -1)

    def mul_plain(self, a: Ct, slots) -> Ct:
        self.trace.append(("pmul", a.level))
        return self.o.mul_plain(a, self._slots().encode(slots))

    def mul_plain_coeffs(self, a: Ct, coeffs) -> Ct:
        """a times a plaintext given by its coefficients (any slot field)."""
        self.trace.append(("pmul", a.level))
        return self.o.mul_plain(a, coeffs)

    def mul_count(self) -> int:
        return sum(1 for t in self.trace if t[0] == "mul")

    # ---- per-digit circuit ---------------------------------------------------
    def digit(self, x: Ct, y: Ct, want_lt: bool, want_eq: bool):
        """(LT_k, EQ_k) for one digit pair (either may be None if unwanted)."""
        p = self.p
        z = self.sub(x, y)
        pw = {1: z}

        def power(n: int) -> Ct:
            if n in pw:
                return pw[n]
            if n & (n - 1) == 0:
                h = power(n // 2)
                r = self.mul(h, h)
            else:
                a = 1 << (n.bit_length() - 1)
                r = self.mul(power(a), power(n - a))
            pw[n] = r
            return r

        lt = None
        if want_lt:
            c = lt_coefficients(p)
            B = 1 << baby_log(p)
            nblocks = (p - 2) // B + 1  # odd exponents go up to p-2

            def leaf(k: int):
                terms = [(r, c[B * k + r]) for r in range(1, B, 2) if B * k + r <= p - 2 and c[B * k + r]]
                if not terms:
                    return None
                cts = [power(r) for r, _ in terms]
                lv = min(t.level for t in cts)
                acc = None
                for (r, cr), t in zip(terms, cts):
                    term = self.mul_const(self.lower(t, lv), cr)
                    acc = term if acc is None else self.add(acc, term)
                return acc

            def tree(k0: int, t: int):
                if k0 >= nblocks:
                    return None
                if t == 0:
                    return leaf(k0)
                half = 1 << (t - 1)
                lo = tree(k0, t - 1)
                hi = tree(k0 + half, t - 1)
                if hi is None:
                    return lo
                prod = self.mul(power(B * half), hi)
                return prod if lo is None else self.add(lo, prod)

            t = 0
            while (1 << t) < nblocks:
                t += 1
            odd = tree(0, t)
            zp = power(p - 1)
            lead = self.mul_const(zp, c[p - 1])
            lt = lead if odd is None else self.add(lead, odd)
        eq = None
        if want_eq:
            eq = self.add_const(self.neg(power(p - 1)), 1)
        return lt, eq

    def digit_bivariate(self, x: Ct, y: Ct, want_lt: bool, want_eq: bool):
        """(LT_k, EQ_k) of one pair of full digits in [0, p)."""
        p = self.p

        def power(pw: dict, n: int) -> Ct:
            if n in pw:
                return pw[n]
            if n & (n - 1) == 0:
                h = power(pw, n // 2)
                r = self.mul(h, h)
            else:
                a = 1 << (n.bit_length() - 1)
                r = self.mul(power(pw, a), power(pw, n - a))
            pw[n] = r
            return r

        lt = None
        if want_lt:
            c = lt_bivariate_coefficients(p)
            # no constant terms: L_y(0) = [y = 0] and no x lies below 0
            assert all(c[a][0] == 0 for a in range(p))
            px, py = {1: x}, {1: y}
            for a in range(p):
                ys = [(b, c[a][b]) for b in range(1, p) if c[a][b]]
                if not ys:
                    continue
                cts = [power(py, b) for b, _ in ys]
                lv = min(t.level for t in cts)
                h = None
                for (b, cb), t in zip(ys, cts):
                    term = self.mul_const(self.lower(t, lv), cb)
                    h = term if h is None else self.add(h, term)
                term = h if a == 0 else self.mul(power(px, a), h)
                lt = term if lt is None else self.add(lt, term)
        eq = None
        if want_eq:
            pz = {1: self.sub(x, y)}
            eq = self.add_const(self.neg(power(pz, p - 1)), 1)
        return lt, eq

    # ---- merge of digits -----------------------------------------------------
    def compare(self, xs, ys, want_lt=True, want_eq=False, bivariate=False):
        """LT(x, y) and/or EQ(x, y) for digit lists (least significant first);
        bivariate: full digits in [0, p) (else digits in [0, (p+1)/2))."""
        digit = self.digit_bivariate if bivariate else self.digit
        nodes = []
        for x, y in zip(xs, ys):
            nodes.append(digit(x, y, want_lt, True if len(xs) > 1 or want_eq else False))
        while len(nodes) > 1:
            root = len(nodes) == 2
            nxt = []
            for i in range(len(nodes) // 2):
                (llo, elo), (lhi, ehi) = nodes[2 * i], nodes[2 * i + 1]
                L = self.add(lhi, self.mul(ehi, llo)) if want_lt else None
                E = self.mul(ehi, elo) if (want_eq or not root) else None
                nxt.append((L, E))
            if len(nodes) % 2:
                nxt.append(nodes[-1])
            nodes = nxt
        L, E = nodes[0]
        return (L if want_lt else None), (E if want_eq else None)

    def compare_lt(self, xs, ys) -> Ct:
        return self.compare(xs, ys, True, False)[0]

    def compare_eq(self, xs, ys) -> Ct:
        return self.compare(xs, ys, False, True)[1]

    def max_min(self, xs, ys):
        """(max digits, min digits) of the two operands."""
        L = self.compare_lt(xs, ys)
        mx, mn = [], []
        for x, y in zip(xs, ys):
            t = self.mul(L, self.sub(y, x))
            mx.append(self.add(x, t))
            mn.append(self.sub(y, t))
        return mx, mn


def sort_galois(p: int, N: int) -> list:
    """Galois elements the sort needs: sigma_{5^s}, s = 1 .. cols-1."""
    ss = SlotStructure(p, N)
    cols = ss.ns // 2
    return [pow(5, s, 2 * N) for s in range(1, cols)]


def sort_rows(ev: "Evaluator", xs):
    """Digits (least significant first) of every row's values in increasing
    order; xs: the d digit ciphertexts (univariate digits)."""
    return sort_joint(ev, [xs])[0]


def sort_ranks(ev: "Evaluator", cts):
    """The rank step of sort_joint on sequences of any length n = K cols (the
    sort application, Sec. 6; for n > p the ranks wrap mod p, so they, and
    the comparisons they are summed from, are the result): returns the K rank
    ciphertexts and the comparison matrix, a dict (a, b, s) -> LT(sigma_{5^s}
    x^b, x^a) over (b, s) != (a, 0), whose slot (r, c) is [x_j < x_i] for the
    global indices i = a cols + c and j = b cols + (c + s) mod cols of row r.

    rank^a = sum over (b, s) != (a, 0), b and then s ascending, of
    LT(sigma_{5^s} x^b, x^a) + w * EQ(sigma_{5^s} x^b, x^a), with the
    tie-break mask w[c] = [b cols + (c + s) mod cols < a cols + c]: slot
    (r, c) of rank^a is the number of values of row r below x_i, plus those
    equal to it at a lower index, mod p."""
    ss = ev._slots()
    assert ss.kind == "linear" and ss.ns >= 4, "sorting needs p = 1 mod 4 and two columns or more"
    cols, twoN = ss.ns // 2, 2 * ev.o.N
    K = len(cts)
    ranks, matrix = [], {}
    for a in range(K):
        rank = None
        for b in range(K):
            for s in range(cols):
                if b == a and s == 0:
                    continue
                xr = [ev.rotate(x, pow(5, s, twoN)) for x in cts[b]] if s else list(cts[b])
                lt, eq = ev.compare(xr, cts[a], True, True)
                matrix[(a, b, s)] = lt
                w = [1 if b * cols + (c + s) % cols < a * cols + c else 0 for _ in range(2) for c in range(cols)]
                t = ev.add(lt, ev.mul_plain(eq, w))
                rank = t if rank is None else ev.add(rank, t)
        ranks.append(rank)
    return ranks, matrix


def sort_joint(ev: "Evaluator", cts):
    """Row r of the K ciphertexts cts[0..K) (each a list of d digit
    ciphertexts) is one sequence of K cols values, global index a cols + c
    for column c of ciphertext a.  Returns K digit lists whose row r holds
    that sequence in increasing order (ciphertext t: positions t cols ..
    t cols + cols - 1); needs K cols <= p.

    rank^a = sum over (b, s) != (a, 0), b and then s ascending, of
    LT(sigma_{5^s} x^b, x^a) + w * EQ(sigma_{5^s} x^b, x^a), with the
    tie-break mask w[c] = [b cols + (c + s) mod cols < a cols + c]; then for
    a and s ascending (sigma_{5^s} of rank^a and of x^a taken once) and t
    ascending: out^t += EQ(sigma_{5^s} rank^a - (t cols + c)) sigma_{5^s} x^a
    per digit."""
    ss = ev._slots()
    p, cols, twoN = ev.p, ss.ns // 2, 2 * ev.o.N
    K, d = len(cts), len(cts[0])
    assert K * cols <= p, "ranks must stay below p"
    ranks, _ = sort_ranks(ev, cts)
    outs = [[None] * d for _ in range(K)]
    for a in range(K):
        for s in range(cols):
            g = pow(5, s, twoN)
            rr = ev.rotate(ranks[a], g) if s else ranks[a]
            xr = [ev.rotate(x, g) for x in cts[a]] if s else list(cts[a])
            for t in range(K):
                u = ev.sub_plain(rr, [t * cols + c for _ in range(2) for c in range(cols)])
                e = ev.add_const(ev.neg(_powers(ev, u)(p - 1)), 1)
                for k in range(d):
                    term = ev.mul(e, xr[k])
                    outs[t][k] = term if outs[t][k] is None else ev.add(outs[t][k], term)
    return outs

def slot_plan(ns: int, useful):
    """The slot manager's placement of useful slots into as few outputs as
    possible (Sec. 5.3, slot compaction).  useful[j] lists input j's useful slot
    indices.  Returns (outputs, pieces, dest): each piece (j, o, src, s, b)
    moves input j's slots src to output o by shifting columns right by s and
    swapping rows when b; dest[j][u] = o n_s + slot, or -1 for a slot left
    behind."""
    cols, rows = (ns // 2, 2) if ns >= 2 else (1, 1)

    def image(u, s, b):
        r, c = divmod(u, cols)
        return (r ^ b) * cols + (c + s) % cols

    occ = []
    pieces = []
    dest = [[-1] * ns for _ in useful]
    for j, u_j in enumerate(useful):
        rest = sorted(set(u_j))
        while rest:
            best, where = 0, None
            for o in range(len(occ)):
                for b in range(rows):
                    for s in range(cols):
                        n = sum(1 for u in rest if image(u, s, b) not in occ[o])
                        if n > best:
                            best, where = n, (o, s, b)
            if where is None:
                occ.append(set())
                continue
            o, s, b = where
            src = [u for u in rest if image(u, s, b) not in occ[o]]
            for u in src:
                occ[o].add(image(u, s, b))
                dest[j][u] = o * ns + image(u, s, b)
            pieces.append((j, o, tuple(src), s, b))
            rest = [u for u in rest if u not in src]
    return len(occ), pieces, dest


def slot_galois(ns: int, N: int, pieces) -> list:
    """Rotation keys the pieces need: column shifts (ascending), then the row
    swap."""
    cols = ns // 2 if ns >= 2 else 1
    gs = sorted({pow(5, (cols - s) % cols, 2 * N) for _, _, _, s, _ in pieces if s})
    if any(b for *_, b in pieces):
        gs.append(2 * N - 1)
    return gs


def slot_pack(ev: "Evaluator", cts, useful):
    """Compacts the inputs' useful slots: per piece, in plan order, mask the
    input to the piece's slots, shift the columns (sigma_{5^(cols - s)}), swap
    the rows (sigma_{2N-1}) and add into the piece's output."""
    ss = ev._slots()
    N = ev.o.N
    cols = ss.ns // 2 if ss.ns >= 2 else 1
    n_out, pieces, _ = slot_plan(ss.ns, useful)
    outs = [None] * n_out
    for j, o, src, s, b in pieces:
        keep = set(src)
        t = ev.mul_plain(cts[j], [1 if i in keep else 0 for i in range(ss.ns)])
        if s:
            t = ev.rotate(t, pow(5, (cols - s) % cols, 2 * N))
        if b:
            t = ev.rotate(t, 2 * N - 1)
        outs[o] = t if outs[o] is None else ev.add(outs[o], t)
    return outs


def _powers(ev: "Evaluator", x: Ct):
    """z^n by the fixed power rule (n = 1: z; n a power of two: square of
    z^(n/2); else z^(2^a) z^(n - 2^a), 2^a the largest power of two below n),
    results cached."""
    pw = {1: x}

    def power(n: int) -> Ct:
        if n in pw:
            return pw[n]
        if n & (n - 1) == 0:
            h = power(n // 2)
            r = ev.mul(h, h)
        else:
            a = 1 << (n.bit_length() - 1)
            r = ev.mul(power(a), power(n - a))
        pw[n] = r
        return r

    return power


def eq_const(ev: "Evaluator", x: Ct, k: int) -> Ct:
    """EQ(x, k) for a public constant k: 1 - (x - k)^(p-1)."""
    z = ev.add_const(x, -k)
    return ev.add_const(ev.neg(_powers(ev, z)(ev.p - 1)), 1)


def private_query(ev: "Evaluator", q: Ct, data: Ct, op1: Ct, op2: int, codes) -> Ct:
    """The private query of Sec. 5.3 with its branches straight-lined: the
    query type q is compared with the three public codes (add, multiply,
    power); the three candidate results data + op1, data * op1 and
    data^op2 are computed; the answer is sum_i result_i * EQ(q, code_i).
    Issue order: the branch evaluation (the three EQs, in code order), then
    the three results, then the selection."""
    c = [eq_const(ev, q, k) for k in codes]
    r1 = ev.add(data, op1)
    r2 = ev.mul(data, op1)
    r3 = _powers(ev, data)(op2)
    out = ev.mul(r1, c[0])
    out = ev.add(out, ev.mul(r2, c[1]))
    return ev.add(out, ev.mul(r3, c[2]))


def extract_digits(ev: "Evaluator", ct: Ct, d: int, xs=None):
    """Mod extract: the d digits of every F_{p^d} slot of ct, digit k in a
    ciphertext of its own (F_p constants).  B_t = sigma_{p^t}(ct) for t =
    1 .. d-1; D_k = sum_t B_t * L[k][t], t ascending (extension.ExtSlots)."""
    from .extension import ExtSlots

    xs = xs or ExtSlots(ev.p, ev.o.N, d)
    L = xs.extraction_plaintexts()
    B = [ct] + [ev.rotate(ct, g) for g in xs.galois()]
    out = []
    for k in range(d):
        acc = None
        for t in range(d):
            term = ev.mul_plain_coeffs(B[t], L[k][t])
            acc = term if acc is None else ev.add(acc, term)
        out.append(acc)
    return out


def round_depth(p: int, d: int) -> int:
    """Levels one max/min round consumes: LT (PS depth + merge depth) + select."""
    lg = (p - 2).bit_length()
    return lg + (d - 1).bit_length() + 1


def galois_schedule(ns: int, N: int, linear: bool = True):
    """In-slot rounds: column rotations by cols/2, .., 1, then the row swap."""
    if not linear or ns <= 2:
        return [2 * N - 1] if ns == 2 else []
    cols = ns // 2
    out, step = [], cols // 2
    while step >= 1:
        out.append(pow(5, step, 2 * N))
        step //= 2
    out.append(2 * N - 1)
    return out


class Tournament:
    """max and/or min over every slot of n ciphertexts (per digit)."""

    def __init__(self, ev: "Evaluator", d: int, ns: int, N: int, refresh=None):
        self.ev, self.d, self.ns, self.N = ev, d, ns, N
        self.refresh = refresh  # callable(list of Ct) -> list of Ct, or None
        self.depth = round_depth(ev.p, d)
        self.refreshes = 0

    def _maybe_refresh(self, digits):
        lv = min(c.level for dig in digits for c in dig)
        if lv - self.depth >= 1:  # the round ends at level >= 1
            return digits
        assert self.refresh is not None, "round needs more levels than remain and no refresh is given"
        self.refreshes += 1
        return [self.refresh(dig) for dig in digits]

    def _select(self, xs, ys, want_max):
        mx, mn = self.ev.max_min(xs, ys)
        return mx if want_max else mn

    def run(self, digits, want_max=True, want_min=True):
        """digits[k] is the list of n ciphertexts of digit k."""
        n = len(digits[0])
        out = {}
        cur = {}
        first = True
        while n > 1:
            h = n // 2
            kinds = [k for k, w in (("max", want_max), ("min", want_min)) if w]
            if first:
                src = self._maybe_refresh(digits)
                A = [dig[:h] for dig in src]
                B = [dig[h:2 * h] for dig in src]
                R = [dig[2 * h:] for dig in src]
                res = {"max": [[] for _ in range(self.d)], "min": [[] for _ in range(self.d)]}
                for i in range(h):
                    mx, mn = self.ev.max_min([A[k][i] for k in range(self.d)], [B[k][i] for k in range(self.d)])
                    for k in range(self.d):
                        res["max"][k].append(mx[k])
                        res["min"][k].append(mn[k])
                for kind in kinds:
                    cur[kind] = [res[kind][k] + R[k] for k in range(self.d)]
                first = False
            else:
                for kind in kinds:
                    src = self._maybe_refresh(cur[kind])
                    A = [dig[:h] for dig in src]
                    B = [dig[h:2 * h] for dig in src]
                    R = [dig[2 * h:] for dig in src]
                    sel = [[] for _ in range(self.d)]
                    for i in range(h):
                        r = self._select([A[k][i] for k in range(self.d)], [B[k][i] for k in range(self.d)],
                                         kind == "max")
                        for k in range(self.d):
                            sel[k].append(r[k])
                    cur[kind] = [sel[k] + R[k] for k in range(self.d)]
            n = h + (n % 2)
        if first:  # a single ciphertext: no cross round
            for kind, w in (("max", want_max), ("min", want_min)):
                if w:
                    cur[kind] = [list(dig) for dig in digits]
        for g in galois_schedule(self.ns, self.N):
            for kind in [k for k, w in (("max", want_max), ("min", want_min)) if w]:
                src = self._maybe_refresh(cur[kind])
                x = [dig[0] for dig in src]
                r = [self.ev.rotate(c, g) for c in x]
                cur[kind] = [[c] for c in self._select(x, r, kind == "max")]
        for kind in cur:
            out[kind] = [dig[0] for dig in cur[kind]]
        return out
