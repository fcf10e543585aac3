// modarith.cuh -- exact modular arithmetic on u64 residues (q < 2^58).
//
// Two published methods, both exact (the result is the canonical residue):
//  * Shoup's precomputed-quotient product for multiplication by a known
//    constant w:  w' = floor(w 2^64 / q);  a w - floor(a w' / 2^64) q lies in
//    [0, 2q) for every a < 2^64 (V. Shoup, NTL; D. Harvey, "Faster arithmetic
//    for number-theoretic transforms", J. Symb. Comp. 2014, which also gives
//    the lazy butterflies used by the NTT);
//  * Barrett reduction (P. Barrett 1986) of a 128-bit value x < 2^(2b+3),
//    b = bitlength(q): t = floor(x / 2^(b-2)), mu = floor(2^(2b+4) / q),
//    qhat = floor(t mu / 2^(b+6)) satisfies x/q - 2 < qhat <= x/q, so
//    x - qhat q lies in [0, 3q).  That bound admits sums of up to eight
//    products of canonical residues before one reduction.
// Every function is __host__ __device__ so the library's CPU self-test checks
// the very code the kernels run.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define FHE_HD __host__ __device__ __forceinline__
#else
#define FHE_HD inline
#endif

typedef uint64_t u64;
typedef unsigned __int128 u128;

FHE_HD u64 fhe_mulhi(u64 a, u64 b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (u64)(((u128)a * b) >> 64);
#endif
}

// Per-prime constants used by the kernels.
struct ModQ {
    u64 q;       // the prime
    u64 q2;      // 2q
    u64 mu;      // floor(2^(2b+4) / q) * 2^(58-b): Barrett constant, pre-shifted
    int bshift;  // b - 2, the shift that forms t
    int pad;
    u64 mu64;    // floor(2^64 / q)
};

// a * w mod q in [0, 2q), w < q, ws = floor(w 2^64 / q), any a < 2^64.
FHE_HD u64 shoup_lazy(u64 a, u64 w, u64 ws, u64 q) { return a * w - fhe_mulhi(a, ws) * q; }

// Shoup's product with a cheaper quotient (the NTT butterflies' form): with
// a = ah 2^32 + al and ws = wh 2^32 + wl, floor(a ws / 2^64) = ah wh +
// floor((ah wl + al wh) / 2^32 + al wl / 2^64), and the estimate
// ah wh + floor(ah wl / 2^32) + floor(al wh / 2^32) drops three fractions
// below 1 each, so it is 0, 1 or 2 below the exact quotient.  Shoup's bound
// a w - floor(a ws / 2^64) q in [0, 2q) then gives a w - qhat q in [0, 4q),
// for any a < 2^64; the difference fits in 64 bits, so the arithmetic mod
// 2^64 is exact.  One 32x32->64 and two 32x32->hi products instead of the
// four 32x32->64 products (and their carries) of the exact high half.
FHE_HD u64 shoup_lazy4(u64 a, u64 w, u64 ws, u64 q)
{
    const uint32_t al = (uint32_t)a, ah = (uint32_t)(a >> 32), wl = (uint32_t)ws, wh = (uint32_t)(ws >> 32);
#ifdef __CUDA_ARCH__
    const u64 qhat = (u64)ah * wh + ((u64)__umulhi(ah, wl) + __umulhi(al, wh));
#else
    const u64 qhat = (u64)ah * wh + ((((u64)ah * wl) >> 32) + (((u64)al * wh) >> 32));
#endif
    return a * w - qhat * q;
}

// shoup_lazy4 as one multiply-add chain: with nq = 2^64 - q, a w - qhat q =
// a w + qhat nq (mod 2^64), so on the device the low words of a w and of
// qhat nq are summed by a wide multiply-add and the high word by four 32-bit
// multiply-adds, with no separate 64-bit subtraction; the two high partial
// products of the quotient are summed by a wide multiply-add too (t1 * 1 +
// t2), so the whole product runs on the multiply-add pipe.  Same result as
// shoup_lazy4 for every input (the host form is that expression in C).
FHE_HD u64 shoup_lazy4_chain(u64 a, u64 w, u64 ws, u64 nq)
{
#ifdef __CUDA_ARCH__
    u64 r;
    asm("{\n\t"
        ".reg .u32 al, ah, wl, wh, sl, sh, ql, qh, t1, t2, hl, hh, rl, rh;\n\t"
        ".reg .u64 qhat, t12, lo, t2w;\n\t"
        "mov.b64 {al, ah}, %1;\n\t"
        "mov.b64 {wl, wh}, %2;\n\t"
        "mov.b64 {sl, sh}, %3;\n\t"
        "mov.b64 {ql, qh}, %4;\n\t"
        "mul.hi.u32 t1, ah, sl;\n\t"
        "mul.hi.u32 t2, al, sh;\n\t"
        "cvt.u64.u32 t2w, t2;\n\t"
        "mad.wide.u32 t12, t1, 1, t2w;\n\t"
        "mad.wide.u32 qhat, ah, sh, t12;\n\t"
        "mov.b64 {hl, hh}, qhat;\n\t"
        "mul.wide.u32 lo, al, wl;\n\t"
        "mad.wide.u32 lo, hl, ql, lo;\n\t"
        "mov.b64 {rl, rh}, lo;\n\t"
        "mad.lo.u32 rh, ah, wl, rh;\n\t"
        "mad.lo.u32 rh, al, wh, rh;\n\t"
        "mad.lo.u32 rh, hh, ql, rh;\n\t"
        "mad.lo.u32 rh, hl, qh, rh;\n\t"
        "mov.b64 %0, {rl, rh};\n\t"
        "}"
        : "=l"(r)
        : "l"(a), "l"(w), "l"(ws), "l"(nq));
    return r;
#else
    const uint32_t al = (uint32_t)a, ah = (uint32_t)(a >> 32), wl = (uint32_t)ws, wh = (uint32_t)(ws >> 32);
    const u64 qhat = (u64)ah * wh + ((((u64)ah * wl) >> 32) + (((u64)al * wh) >> 32));
    return a * w + qhat * nq;
#endif
}

FHE_HD u64 shoup(u64 a, u64 w, u64 ws, u64 q)
{
    u64 r = shoup_lazy(a, w, ws, q);
    return r >= q ? r - q : r;
}

// Canonical residue of x < 2^(2b+3).
FHE_HD u64 barrett128(u128 x, const ModQ &m)
{
    u64 lo = (u64)x, hi = (u64)(x >> 64);
    int s = m.bshift;                                   // 1 <= s <= 56
    u64 t = (hi << (64 - s)) | (lo >> s);               // floor(x / 2^(b-2)) < 2^(b+5)
    u64 qhat = fhe_mulhi(t, m.mu);                      // floor(t mu / 2^(b+6))
    u64 r = lo - qhat * m.q;                            // in [0, 3q)
    if (r >= m.q2) r -= m.q2;
    if (r >= m.q) r -= m.q;
    return r;
}

// The same reduction without its two corrections: a residue of x in [0, 3q).
FHE_HD u64 barrett128_lazy(u128 x, const ModQ &m)
{
    u64 lo = (u64)x, hi = (u64)(x >> 64);
    int s = m.bshift;
    u64 t = (hi << (64 - s)) | (lo >> s);
    return lo - fhe_mulhi(t, m.mu) * m.q;
}

FHE_HD u64 mulmod(u64 a, u64 b, const ModQ &m) { return barrett128((u128)a * b, m); }

FHE_HD u64 addmod(u64 a, u64 b, u64 q)
{
    u64 r = a + b;
    return r >= q ? r - q : r;
}

FHE_HD u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

FHE_HD u64 negmod(u64 a, u64 q) { return a ? q - a : 0; }

// Any v < 2^64 -> [0, q): v - floor(v mu64 / 2^64) q lies in [0, 2q).
FHE_HD u64 reduce64(u64 v, const ModQ &m)
{
    const u64 r = v - fhe_mulhi(v, m.mu64) * m.q;
    return r >= m.q ? r - m.q : r;
}

// [0, 2q) -> [0, q)
FHE_HD u64 reduce2q(u64 a, u64 q) { return a >= q ? a - q : a; }

// [0, 4q) -> [0, q)
FHE_HD u64 reduce4q(u64 a, u64 q2, u64 q)
{
    if (a >= q2) a -= q2;
    return a >= q ? a - q : a;
}

// Host-side constructors.
inline ModQ make_modq(u64 q)
{
    ModQ m;
    int b = 0;
    while (b < 64 && (q >> b)) b++;
    m.q = q;
    m.q2 = 2 * q;
    u128 mu = ((u128)1 << (2 * b + 4)) / q;             // < 2^(b+5)
    m.mu = (u64)(mu << (58 - b));
    m.bshift = b - 2;
    m.pad = 0;
    m.mu64 = (u64)((((u128)1) << 64) / q);
    return m;
}

inline u64 shoup_const(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }
