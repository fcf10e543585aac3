"""Host check of the NTT engine's thread schedules and unit decompositions
(emulated thread by thread in Python, exact arithmetic mod a small prime):

- a unit of 128 threads x 16 residues holds NS = 2^(11-M) sub-transforms of
  2^M points (M = 5..8); the radix-16 round (threads t -> sub-transform t % NS, residues
  k G + t / NS) and the remaining-stages round (t -> sub-transform t / G, blocks of G contiguous
  residues) together compute, forward and inverse, the same as the plain
  radix-2 stages of every sub-transform;
- the column units of every ring degree 2^10..2^15 (NC columns of NJ jobs),
  also in the paired form (two jobs that read the same source limbs, half
  the columns each, where both jobs' twiddle tables fit the staging table),
  and the row units (grouped: one row of 16 jobs of a prime times R rows;
  single: NS adjacent rows of one job) touch every residue of every job
  exactly once, with ragged job counts."""
import random

import pytest

q = 1000003  # a prime; the schedule check needs no lazy reduction
T = 128


def W(s, j):  # any deterministic twiddle function
    return (1 + 7919 * s + 104729 * j) % q


def ct(x, y, w):
    t = y * w % q
    return (x + t) % q, (x - t) % q


def gs(x, y, w):
    return (x + y) % q, (x - y) * w % q


def fwd_round(x, R, s0, hi):
    for u in range(R):
        half = 1 << (R - 1 - u)
        for t in range(1 << u):
            w = W(s0 + u, (hi << u) + t)
            for k in range(half):
                e = t * 2 * half + k
                x[e], x[e + half] = ct(x[e], x[e + half], w)


def inv_round(x, R, s0, hi):
    for U in range(R - 1, -1, -1):
        half = 1 << (R - 1 - U)
        for t in range(1 << U):
            w = W(s0 + U, (hi << U) + t)
            for k in range(half):
                a, b = t * 2 * half + k, t * 2 * half + k + half
                x[a], x[b] = gs(x[a], x[b], w)


def unit_schedule(sm, M, FWD, S, his):
    """The engine's two rounds on NS sub-transforms (his[c]: block index of
    sub-transform c), every thread of the 128 emulated in turn."""
    SZ = 1 << M
    G = SZ // 16
    NS = T // G
    R2 = M - 4
    NB = 16 // G

    def round1():
        for tid in range(T):
            c, g = tid % NS, tid // NS
            x = [sm[c][k * G + g] for k in range(16)]
            (fwd_round if FWD else inv_round)(x, 4, S, his[c])
            for k in range(16):
                sm[c][k * G + g] = x[k]

    def round2():
        for tid in range(T):
            c, gp = tid // G, tid % G
            for i in range(NB):
                base = gp * 16 + i * G
                x = [sm[c][base + f] for f in range(1 << R2)]
                (fwd_round if FWD else inv_round)(x, R2, S + 4, his[c] * 16 + gp * NB + i)
                for f in range(1 << R2):
                    sm[c][base + f] = x[f]

    if FWD:
        round1()
        round2()
    else:
        round2()
        round1()


def plain_subtransform(x, M, FWD, S, hi):
    """The same stages on one sub-transform without any thread schedule."""
    (fwd_round if FWD else inv_round)(x, M, S, hi)


@pytest.mark.parametrize("M", [5, 6, 7, 8])
@pytest.mark.parametrize("FWD", [True, False])
def test_unit_rounds_equal_plain_stages(M, FWD):
    SZ = 1 << M
    NS = T // (SZ // 16)
    assert NS * SZ == 16 * T
    rnd = random.Random(M * 2 + FWD)
    S = 3
    his = [rnd.randrange(64) for _ in range(NS)]
    sm = [[rnd.randrange(q) for _ in range(SZ)] for _ in range(NS)]
    want = [list(r) for r in sm]
    for c in range(NS):
        plain_subtransform(want[c], M, FWD, S, his[c])
    unit_schedule(sm, M, FWD, S, his)
    assert sm == want


def split(logN):
    n1, n2 = (logN + 1) // 2, logN // 2
    return n1, n2, 2048 >> n1, 2048 >> n2


def twp_size(n):  # staged twiddle entries of a table of n (one pad per 8)
    return n + n // 8 + 1


TW_WORDS = max(twp_size(256), 2 * twp_size(128))


def col_geometry(logN, xj):
    n1, n2, ns1, _ = split(logN)
    nc = min(ns1, 1 << n2)
    paired = xj == 2 and nc == ns1 and 2 * twp_size(1 << n1) <= TW_WORDS
    if paired:
        nc //= 2
    return nc, ns1 // nc, (1 << n2) // nc, paired


@pytest.mark.parametrize("logN", [10, 11, 12, 13, 14, 15])
@pytest.mark.parametrize("njobs", [1, 3, 16, 37])
@pytest.mark.parametrize("xj", [1, 2])
def test_column_units_cover_every_residue_once(logN, njobs, xj):
    n1, n2, ns1, _ = split(logN)
    NC, NJ, BLK, paired = col_geometry(logN, xj)
    assert NJ <= 2 and NJ * twp_size(1 << n1) <= TW_WORDS
    SZ = 1 << n1
    units = ((njobs + NJ - 1) // NJ) * BLK
    seen = {}
    for lu in range(units):
        job0, lo0 = (lu // BLK) * NJ, (lu % BLK) * NC
        pos = {}
        for r in range(16 * T):  # word r of the unit: job slot, column, element
            j = 0 if NJ == 1 else r // (NC * SZ)
            col, e = r % NC, (r % (NC * SZ)) // NC
            assert 0 <= e < SZ
            pos[r] = (e << n2) + lo0 + col
            if job0 + j >= njobs:
                continue
            key = (job0 + j, pos[r])
            seen[key] = seen.get(key, 0) + 1
        if paired:
            # the paired load: thread t's words t + 128 k (k < 8) of slot 0
            # and t + 128 k + NC SZ of slot 1 read the same source position
            assert NJ == 2 and 2 * NC * SZ == 16 * T
            for t in range(T):
                for k in range(8):
                    r = t + k * T
                    assert r < NC * SZ and pos[r] == pos[r + NC * SZ]
    assert len(seen) == njobs << logN and set(seen.values()) == {1}


def test_paired_geometry_where_it_applies():
    """Pairing halves the columns of the rings whose column unit holds one
    job (2^11..2^14); 2^10 already holds two jobs and 2^15's two 256-entry
    twiddle tables would not fit the staging table."""
    assert [col_geometry(n, 2)[3] for n in range(10, 16)] == [False, True, True, True, True, False]
    assert all(col_geometry(n, 2)[1] == 2 for n in range(10, 15))


@pytest.mark.parametrize("logN", [10, 11, 12, 13, 14, 15])
@pytest.mark.parametrize("outer,nl", [(1, 3), (5, 2), (16, 3), (21, 2), (40, 1)])
def test_row_units_cover_every_residue_once(logN, outer, nl):
    n1, n2, _, ns2 = split(logN)
    SZ = 1 << n2
    grouped = outer >= 12 or (1 << n1) < ns2
    seen = {}
    if grouped:
        R = ns2 // 16
        CH = (1 << n1) // R
        OC = (outer + 15) // 16
        units = nl * OC * CH
        for lu in range(units):
            hc, t = lu % CH, lu // CH
            oc, l = t % OC, t // OC
            hi0 = hc * R
            nvalid = min(16, outer - oc * 16)
            for r in range(16 * T):
                c, f = r >> n2, r & (SZ - 1)
                slot, row = c // R, hi0 + c % R
                if slot >= nvalid:
                    continue
                job = (oc * 16 + slot) * nl + l
                key = (job, (row << n2) + f)
                seen[key] = seen.get(key, 0) + 1
    else:
        CHS = (1 << n1) // ns2
        units = outer * nl * CHS
        for lu in range(units):
            hi0, job = (lu % CHS) * ns2, lu // CHS
            for r in range(16 * T):
                c, f = r >> n2, r & (SZ - 1)
                key = (job, ((hi0 + c) << n2) + f)
                seen[key] = seen.get(key, 0) + 1
    assert len(seen) == (outer * nl) << logN and set(seen.values()) == {1}


def test_grouped_rows_share_a_prime():
    """A grouped row unit's 16 jobs differ only in the outer index, so they
    share the limb index l and hence the prime."""
    for logN in (13, 14, 15):
        n1, n2, _, ns2 = split(logN)
        R = ns2 // 16
        outer, nl = 33, 4
        OC = (outer + 15) // 16
        CH = (1 << n1) // R
        for lu in range(nl * OC * CH):
            t = lu // CH
            oc, l = t % OC, t // OC
            jobs = [(oc * 16 + s) * nl + l for s in range(min(16, outer - oc * 16))]
            assert {j % nl for j in jobs} == {l}
