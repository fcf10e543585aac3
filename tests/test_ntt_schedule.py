"""Host check of the NTT kernels' thread schedules: the 8-elements-per-thread
sub-transform schedule (autotuner variant 3: round A of 3 stages in
registers; round B of 3 stages in registers and the rest across the lanes of
a block, lanes h and h ^ delta) is emulated thread by thread with exact
arithmetic mod a small prime and compared with the 16-elements-per-thread
schedule it replaces, forward and inverse, for sub-transforms of 2^6 .. 2^8
points; the cross-lane partners always share a warp."""
import random

import pytest

q = 1000003  # a prime; the schedule check needs no lazy reduction


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


def sub16(sm, M, FWD, S, hi0, hstep):
    """16 sub-transforms of 2^M points, 16 elements per thread (the kernels'
    default schedule), every thread emulated in turn."""
    SZ = 1 << M; G = SZ // 16; R2 = M - 4; NB = 16 // G; T = 16 * G
    def round1():
        for tid in range(T):
            c, g = tid & 15, tid >> 4
            hi = hi0 + c * hstep
            x = [sm[c][k * G + g] for k in range(16)]
            (fwd_round if FWD else inv_round)(x, 4, S, hi)
            for k in range(16): sm[c][k * G + g] = x[k]
    def round2():
        for tid in range(T):
            c, gp = tid // G, tid % G
            hi = hi0 + c * hstep
            for i in range(NB):
                b = gp * NB + i
                x = [sm[c][b * G + f] for f in range(1 << R2)]  # blocks of G contiguous
                (fwd_round if FWD else inv_round)(x, R2, S + 4, hi * 16 + b)
                for f in range(1 << R2): sm[c][b * G + f] = x[f]
    if FWD: round1(); round2()
    else: round2(); round1()


def sub8(sm, M, FWD, S, hi0, hstep):
    """The same with 8 elements per thread; cross-lane stages exchange whole
    register arrays between lanes h and h ^ delta."""
    SZ = 1 << M; G8 = SZ // 8; T = 16 * G8; R2 = M - 3; P = G8 // 8
    def roundA():
        for tid in range(T):
            c, g = tid & 15, tid >> 4
            hi = hi0 + c * hstep
            x = [sm[c][k * G8 + g] for k in range(8)]
            (fwd_round if FWD else inv_round)(x, 3, S, hi)
            for k in range(8): sm[c][k * G8 + g] = x[k]
    def roundB():
        regs = {}
        for tid in range(T):
            c, gp = tid // G8, tid % G8
            b, h = gp // P, gp % P
            regs[tid] = [sm[c][b * G8 + h + j * P] for j in range(8)]
        def inreg(tid):
            c, gp = tid // G8, tid % G8
            b = gp // P
            hi = hi0 + c * hstep
            (fwd_round if FWD else inv_round)(regs[tid], 3, S + 3, hi * 8 + b)
        def cross(r):
            # block-local stage r >= 3 at distance delta = P >> (r - 2) lanes
            delta = P >> (r - 2)
            new = {}
            for tid in range(T):
                c, gp = tid // G8, tid % G8
                b, h = gp // P, gp % P
                hi = hi0 + c * hstep
                other = regs[tid ^ delta]  # lane partner
                lower = (h & delta) == 0
                out = []
                for j in range(8):
                    tg = j * (1 << (r - 3)) + (h * (1 << (r - 3))) // P
                    w = W(S + 3 + r, ((hi * 8 + b) << r) + tg)
                    mine, theirs = regs[tid][j], other[j]
                    if FWD:
                        x, y = (mine, theirs) if lower else (theirs, mine)
                        X, Y = ct(x, y, w)
                    else:
                        x, y = (mine, theirs) if lower else (theirs, mine)
                        X, Y = gs(x, y, w)
                    out.append(X if lower else Y)
                new[tid] = out
            regs.update(new)
        if FWD:
            for tid in range(T): inreg(tid)
            for r in range(3, R2): cross(r)
        else:
            for r in range(R2 - 1, 2, -1): cross(r)
            for tid in range(T): inreg(tid)
        for tid in range(T):
            c, gp = tid // G8, tid % G8
            b, h = gp // P, gp % P
            for j in range(8): sm[c][b * G8 + h + j * P] = regs[tid][j]
    if FWD: roundA(); roundB()
    else: roundB(); roundA()


@pytest.mark.parametrize("M", [6, 7, 8])


def test_sub8_schedule_equals_sub16(M):
    for FWD in (True, False):
        for trial in range(3):
            rnd = random.Random(M * 10 + trial + FWD)
            base = [[rnd.randrange(q) for _ in range(1 << M)] for _ in range(16)]
            S, hi0, hstep = rnd.choice([(0, 0, 0), (7, 5, 1), (6, 3, 0)])
            a = [row[:] for row in base]
            b = [row[:] for row in base]
            sub16(a, M, FWD, S, hi0, hstep)
            sub8(b, M, FWD, S, hi0, hstep)
            assert a == b, (M, FWD, trial)
    G8 = (1 << M) // 8
    P = G8 // 8
    for tid in range(16 * G8):
        for r in range(3, M - 3):
            d = P >> (r - 2)
            assert (tid ^ d) // 32 == tid // 32
