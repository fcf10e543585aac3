// ntt_engine.cuh -- the NTT engine: negacyclic NTT / inverse NTT over batches of RNS
// limbs, with the key-switching and modulus-switching steps fused into their
// loads and stores.
//
// Transform (BoostCom Sec. 2.2: radix-2 NTT, Cooley-Tukey forward and
// Gentleman-Sande inverse, for power-of-two N):
//   forward  A[k] = a(psi^(2 brv(k) + 1)), natural-order input, bit-reversed
//            output; stage s (s = 0..logN-1) pairs j, j + N/2^(s+1) with the
//            twiddle psi^brv(2^s + (j >> (logN - s)));
//   inverse  the stages undone in reverse order with psi^-brv(.), then N^-1.
//
// GB300 mapping.  N = 2^n is split as 2^n1 x 2^n2 (n1 = ceil(n/2)).  The
// forward transform is two passes: "columns" runs global stages 0..n1-1,
// which only combine residues j = e 2^n2 + lo of one column lo, and "rows"
// runs stages n1..n-1 inside contiguous rows of 2^n2 residues.  Each pass is
// made of sub-transforms of size 2^M (M = n1 or n2) whose twiddles are
// entries of the full table: at local stage u, element e of a sub-transform
// with block index hi uses psi^brv(2^(S+u) + hi 2^u + (e >> (M-u))), S its
// first global stage.  The inverse runs rows first, then columns.  The
// half-transformed limb between the passes lives in the job's output limb.
//
// Units.  Every CTA has 128 threads holding 16 residues each, so a unit of
// work is 2048 residues in shared memory: NS = 2^(11-M) sub-transforms of 2^M
// points.  A sub-transform runs as one radix-16 round (4 stages on strided
// residues) and one round of the remaining M-4 stages (contiguous blocks),
// with shared-memory exchanges in between.  A column unit is NC adjacent
// columns of each of NS/NC jobs (one job except at n = 10); a row unit is
// either one row of each of 16 jobs that share a prime times NS/16 adjacent
// rows (the batched case: the CTA stages those rows' twiddles once), or NS
// adjacent rows of one job (small batches; twiddles read through the cache).
// Global memory is read and written in coalesced runs of at least 64 bytes.
//
// Segments and persistence.  A launch carries a table of up to FHE_SEGS
// segments; a segment is one batch of limb jobs with its own context (ring
// degree, twiddle and constant tables), pointers and level.  One launch can
// therefore serve ciphertexts of different ring degree, level and origin:
// the units of all segments are numbered in order and every CTA walks them
// with a grid stride, dispatching each unit on its segment's ring degree.
// The grid is either one CTA per unit or a fixed number of resident CTAs per
// SM (the autotuner's choice per context).
//
// Load/store functors let one kernel body serve the plain transform and the
// fused variants: ModUp (basis conversion of a key-switching digit computed
// while loading, then NTT), ModDown and modulus switching (correction
// computed while loading, subtract-and-scale applied while storing).
// Butterflies are Harvey's lazy ones (values below (4s+1)q after s forward
// stages, in [0, 4q) inverse) with Shoup twiddles.
//
// The kernels and functors are templates instantiated by ntt.cu (limb maps,
// the plain and scaled transforms, the autotuner), ntt_ks.cu (key switching:
// ModUp, ModDown, relinearise + switch) and ntt_ms.cu (modulus switching),
// which compile in parallel.
#pragma once
#include <string.h>

#include <algorithm>

#include "fhe_internal.h"

namespace {

// The butterflies' twiddle product: shoup_lazy4 as one multiply-add chain.
// Measured on the GB300 (16-pair comparison at N = 2^14, identical results):
// the C form 2454 slot-comparisons/s, the chain with its quotient's two high
// products summed by an add-with-carry 2563, by a wide multiply-add 2606
// (register-resident forward butterflies: 1015 -> 1173 G/s for the first
// chain).  Also measured and not kept: X + t by multiply-adds as well (2606,
// no gain on its own: 2570), and the inverse's 4q reduction as an unsigned
// minimum (2554).
__device__ __forceinline__ u64 bfly_mul(u64 a, const ulonglong2 w, u64 q)
{
    return shoup_lazy4_chain(a, w.x, w.y, 0 - q);
}

// Forward butterfly without normalisation: t = [Y w] in [0, 4q) for any
// 64-bit Y (shoup_lazy4), so if X, Y < B then X + t and X - t + 4q lie in
// [0, B + 4q).  Inputs below 4q (canonical residues, or the lazy results of
// the fused conversions) stay below (4s + 4) q <= 64 q < 2^63 after s <= 15
// stages for primes below 2^57; one reduction at the end brings every value
// to [0, q).  q4 = 4q.
__device__ __forceinline__ void ct_bfly(u64 &X, u64 &Y, const ulonglong2 w, u64 q, u64 q4)
{
    const u64 t = bfly_mul(Y, w, q);
    const u64 x = X;
    X = x + t;
    Y = x - t + q4;
}

// Inverse butterfly on values in [0, 4q): X + Y reduced once by 4q, and
// [(X - Y + 4q) w] in [0, 4q).
__device__ __forceinline__ void gs_bfly(u64 &X, u64 &Y, const ulonglong2 w, u64 q, u64 q4)
{
    u64 s = X + Y;
    s = s >= q4 ? s - q4 : s;
    u64 d = X - Y + q4;
    Y = bfly_mul(d, w, q);
    X = s;
}

// Stages s0 .. s0+R-1 of the forward transform on one group x[0..2^R) whose
// block index is hi.
template <int R, class TW>
__device__ __forceinline__ void fwd_round(u64 (&x)[1 << R], int s0, int hi, const TW &W, u64 q, u64 q2)
{
#pragma unroll
    for (int u = 0; u < R; u++) {
        const int half = 1 << (R - 1 - u);
#pragma unroll
        for (int t = 0; t < (1 << u); t++) {
            const ulonglong2 w = W.get(s0 + u, (hi << u) + t);
#pragma unroll
            for (int k = 0; k < half; k++) {
                const int e = t * 2 * half + k;
                ct_bfly(x[e], x[e + half], w, q, q2);
            }
        }
    }
}

// One stage of the inverse on x[0..2^R): local stage U, butterflies of
// half-distance 2^(R-1-U).  A template per stage keeps every index a
// compile-time constant, so x stays in registers.
template <int R, int U, class TW>
__device__ __forceinline__ void inv_stage(u64 (&x)[1 << R], int s0, int hi, const TW &W, u64 q, u64 q2)
{
    constexpr int half = 1 << (R - 1 - U);
#pragma unroll
    for (int t = 0; t < (1 << U); t++) {
        const ulonglong2 w = W.get(s0 + U, (hi << U) + t);
#pragma unroll
        for (int k = 0; k < half; k++) gs_bfly(x[t * 2 * half + k], x[t * 2 * half + k + half], w, q, q2);
    }
    if constexpr (U > 0) inv_stage<R, U - 1>(x, s0, hi, W, q, q2);
}

template <int R, class TW>
__device__ __forceinline__ void inv_round(u64 (&x)[1 << R], int s0, int hi, const TW &W, u64 q, u64 q2)
{
    inv_stage<R, R - 1>(x, s0, hi, W, q, q2);
}

// Conversions computed by the loads of a forward transform (ModUp, ModDown,
// the switch corrections) hand it a residue in [0, 3q) (a Barrett reduction
// without its two corrections) or [0, 4q) (a lazy Shoup product) instead of
// [0, q): the forward butterflies accept any 64-bit input whose lazy bound
// stays below 2^64 ((4s + 4) q after s stages) and the transform's last step
// reduces every output to [0, q), so the outputs are the same.  Measured on
// the 16-pair comparison at N = 2^14: 2564 -> 2587 slot-comparisons/s.
// (The chained product with two corrections in place of Shoup's exact one
// for the constant products of the stores measured slower: 2577.)
__device__ __forceinline__ u64 conv_reduce(u128 x, const ModQ &m) { return barrett128_lazy(x, m); }

// ---------------------------------------------------------------------------
// unit geometry
// ---------------------------------------------------------------------------

constexpr int T = 128;  // threads per CTA, 16 residues each

// Register cap: FHE_NTT_MINB resident CTAs of 128 threads per SM (9: 56
// registers a thread).  Measured on the headline comparison (16 pairs,
// N = 2^14): with the C-form butterflies 8 CTAs 2291 slot-comparisons/s, 6
// CTAs (80 registers) 2285, 7 with staged multi-limb loads 2152; with the
// chained butterflies 7 CTAs 2574, 8 CTAs 2653, 9 CTAs 2672, and 2689 with the
// forward row kernels of two-operand stores kept at 8 (FHE_NTT_MINB_ST2: at 9
// they spill 116 bytes); 10 CTAs spill 170-1100 bytes.
#ifndef FHE_NTT_MINB
#define FHE_NTT_MINB 9
#endif
// The same for the column kernels of paired units (two targets per load).
#ifndef FHE_NTT_MINB_PAIRED
#define FHE_NTT_MINB_PAIRED FHE_NTT_MINB
#endif
// The same for the forward row kernels whose stores read two operands
// besides the transform (ModDown, relinearise + switch: accumulator, addend).
#ifndef FHE_NTT_MINB_ST2
#define FHE_NTT_MINB_ST2 8
#endif
// Paired column units whose two jobs read different sources (a digit or
// ciphertext boundary) load in a rolled loop (1) or the unrolled staged one (0).
#ifndef FHE_NTT_PAIRED_FALLBACK_ROLLED
#define FHE_NTT_PAIRED_FALLBACK_ROLLED 1
#endif
// Positions of a paired unit's load loop unrolled together (8 per thread).
#ifndef FHE_NTT_PAIRED_UNROLL
#define FHE_NTT_PAIRED_UNROLL 2
#endif
constexpr int PAIRED_UNROLL = FHE_NTT_PAIRED_UNROLL;
// Launches that mix ring degrees 2^13..2^15 take the kernel that dispatches
// every unit on its degree (1), or one launch per degree in turn (0).
#ifndef FHE_NTT_MIXED_KERNEL
#define FHE_NTT_MIXED_KERNEL 1
#endif
// Words staged per chunk by the loads that read several limbs each (ModUp,
// relinearise + switch, multi-prime switch); 0 = not staged (each word's
// loads, arithmetic and shared-memory store in turn, four words unrolled).
// Measured: staging 2 or 4 words costs 4-5% on the headline (2190 / 2225
// against 2291 slot-comparisons/s).
#ifndef FHE_NTT_MULTI_LDCH
#define FHE_NTT_MULTI_LDCH 0
#endif

// Shared-memory twiddle tables: entry k at k + k / 8 (one 16-byte pad per 8
// entries), so that the second round's strided twiddle reads (stride up to 8
// entries across threads) hit distinct banks.
__host__ __device__ constexpr int twp(int k) { return k + (k >> 3); }
__host__ __device__ constexpr int twp_size(int n) { return n + n / 8 + 1; }

// smem layout: sub-transform c at c*P(M), element e at e + (e >> 4); P is odd
// mod 16 in u64 units, so the strided, blocked and row-wise access patterns
// spread over the banks.
template <int M>
struct Sub {
    static constexpr int SZ = 1 << M;           // elements per sub-transform
    static constexpr int G = SZ / 16;           // threads per sub-transform
    static constexpr int NS = T / G;            // sub-transforms per unit
    static constexpr int R2 = M - 4;            // stages of the second round
    static constexpr int P = SZ + SZ / 16 + 1;  // padded stride
    static constexpr int WORDS = NS * P;        // shared memory words
    static_assert(M >= 5 && M <= 8, "sub-transform size");
    static_assert(NS * SZ == 16 * T, "16 residues a thread");
    __device__ static int at(int c, int e) { return c * P + e + (e >> 4); }
};

constexpr int SM_WORDS = Sub<5>::WORDS > Sub<8>::WORDS ? Sub<5>::WORDS : Sub<8>::WORDS;
// largest staged twiddle table (ulonglong2): one table of 256 entries, or two
// of 128 (paired column units)
constexpr int TW_WORDS = twp_size(256) > 2 * twp_size(128) ? twp_size(256) : 2 * twp_size(128);
constexpr int ROW_J = 16;                    // jobs per grouped row unit

// Twiddle accessors: get(s, j) = psi^brv(2^s + j), the twiddle of global
// stage s with in-stage index j < 2^s.
struct GTw {  // the full table in global memory, read-only path
    const ulonglong2 *__restrict__ p;
    __device__ ulonglong2 get(int s, int j) const { return __ldg(p + (1 << s) + j); }
};

struct PrefixTw {  // the first entries of the table, copied to shared memory
    const ulonglong2 *sm;
    __device__ ulonglong2 get(int s, int j) const { return sm[twp((1 << s) + j)]; }
};

// Row twiddles of one row hi (stages N1.., in-stage index hi 2^u + t) staged
// at offset 2^u - 1 + t.
struct RowTw {
    const ulonglong2 *sm;
    int N1, hi;
    __device__ ulonglong2 get(int s, int j) const
    {
        const int u = s - N1;
        return sm[twp((1 << u) - 1 + j - (hi << u))];
    }
};

// Radix-16 round: thread t = (g, c) with c = t % NS, g = t / NS holds elements
// e = k G + g (k < 16) of sub-transform c: local stages 0..3.
// Remaining-stages round: thread t = (c, g') with c = t / G, g' = t % G holds the 16/G
// blocks b = g' (16/G) + i of G contiguous elements: local stages 4..M-1.
// geo gives each sub-transform's twiddle accessor, block index and prime.
template <int M, bool FWD, class Geo>
__device__ __forceinline__ void subtx(u64 *sm, int tid, const Geo &geo)
{
    using C = Sub<M>;
    constexpr int G = C::G, R2 = C::R2, NB = 16 / G, NS = C::NS;
    // Addresses as a per-thread base plus compile-time offsets: for e = kG + g
    // (g < G <= 16, kG a multiple of G) e >> 4 = (kG) >> 4, and for
    // e = 16 g' + iG + f (iG + f < 16) e >> 4 = g'.
    auto round1 = [&]() {
        const int c = tid % NS, g = tid / NS;
        const auto W = geo.tw(c);
        const int hi = geo.hi(c);
        const u64 q = geo.q(c), q2 = 4 * q;  // lazy bound of the butterflies
        u64 *b1 = sm + c * C::P + g;
        u64 x[16];
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = b1[k * G + ((k * G) >> 4)];
        if (FWD)
            fwd_round<4>(x, geo.S, hi, W, q, q2);
        else
            inv_round<4>(x, geo.S, hi, W, q, q2);
#pragma unroll
        for (int k = 0; k < 16; k++) b1[k * G + ((k * G) >> 4)] = x[k];
    };
    auto round2 = [&]() {
        const int c = tid / G, gp = tid % G;
        const auto W = geo.tw(c);
        const int hi = geo.hi(c);
        const u64 q = geo.q(c), q2 = 4 * q;  // lazy bound of the butterflies
        u64 *b2 = sm + c * C::P + gp * 17;
#pragma unroll
        for (int i = 0; i < NB; i++) {
            u64 x[1 << R2];
#pragma unroll
            for (int f = 0; f < (1 << R2); f++) x[f] = b2[i * G + f];
            if (FWD)
                fwd_round<R2>(x, geo.S + 4, hi * 16 + gp * NB + i, W, q, q2);
            else
                inv_round<R2>(x, geo.S + 4, hi * 16 + gp * NB + i, W, q, q2);
#pragma unroll
            for (int f = 0; f < (1 << R2); f++) b2[i * G + f] = x[f];
        }
    };
    if (FWD) {
        round1();
        __syncthreads();
        round2();
    } else {
        round2();
        __syncthreads();
        round1();
    }
}

// Column pass of ring degree 2^(N1+N2): NC adjacent columns of NJ jobs.
// XJ = 2 asks for two jobs per unit where one would hold all NS columns
// (half as many columns each) and both jobs' twiddles fit the staging table:
// functors whose loads convert several source limbs pair jobs that read the
// same sources (fwd_cols_unit).
__host__ __device__ constexpr bool col_paired(int xj, int n1, int ns, int nc1)
{
    return xj == 2 && nc1 == ns && 2 * twp_size(1 << n1) <= TW_WORDS;
}

template <int N1, int N2, int XJ = 1>
struct ColGeo {
    using C = Sub<N1>;
    static constexpr int NS = C::NS, SZ = C::SZ, NN = 1 << (N1 + N2);
    static constexpr int NC1 = NS < (1 << N2) ? NS : (1 << N2);
    static constexpr bool PAIRED = col_paired(XJ, N1, NS, NC1);
    static constexpr int NC = PAIRED ? NC1 / 2 : NC1;                  // columns per job
    static constexpr int NJ = NS / NC;                                 // jobs per unit
    static constexpr int BLK = (1 << N2) / NC;                         // column blocks per job
    static constexpr int TWC = twp_size(1 << N1);                      // staged twiddles per job
    static_assert(NJ * TWC <= TW_WORDS, "twiddle staging");
    static_assert(NJ <= 2, "jobs per column unit");
    // word r of the unit: job slot, column in job, element
    __device__ static int jslot(int r) { return NJ == 1 ? 0 : r / (NC * SZ); }
    __device__ static int col(int r) { return r % NC; }
    __device__ static int elem(int r) { return (r % (NC * SZ)) / NC; }
};

template <int N1, int N2, int XJ = 1>
struct ColTw {
    using Gm = ColGeo<N1, N2, XJ>;
    const ulonglong2 *W;
    u64 q0, q1;
    static constexpr int S = 0;
    __device__ PrefixTw tw(int c) const { return PrefixTw{W + (c / Gm::NC) * Gm::TWC}; }
    __device__ int hi(int) const { return 0; }
    __device__ u64 q(int c) const { return c / Gm::NC == 0 ? q0 : q1; }
};

// Row pass: grouped (16 jobs of one prime x R adjacent rows) or single (NS
// adjacent rows of one job).
template <int N1, int N2>
struct RowGeo {
    using C = Sub<N2>;
    static constexpr int NS = C::NS, SZ = C::SZ, NN = 1 << (N1 + N2);
    static constexpr int R = NS / ROW_J;         // rows per grouped unit
    static constexpr int CH = (1 << N1) / R;     // row chunks per limb (grouped)
    // row chunks per limb (single; a limb with fewer than NS rows, n = 10,
    // always takes the grouped form)
    static constexpr int CHS = (1 << N1) >= NS ? (1 << N1) / NS : 1;
    static constexpr int TWR = twp_size(SZ - 1); // staged twiddles per row
    static_assert(NS >= ROW_J && NS % ROW_J == 0, "row units");
    static_assert(R * TWR <= TW_WORDS, "twiddle staging");
};

template <int N1, int N2>
struct RowGrpTw {
    const ulonglong2 *W;
    int hi0;
    u64 qq;
    int S;
    __device__ RowTw tw(int c) const
    {
        constexpr int R = RowGeo<N1, N2>::R;
        return RowTw{W + (c % R) * RowGeo<N1, N2>::TWR, N1, hi0 + c % R};
    }
    __device__ int hi(int c) const { return hi0 + c % RowGeo<N1, N2>::R; }
    __device__ u64 q(int) const { return qq; }
};

struct RowOneTw {
    GTw g;
    int hi0;
    u64 qq;
    int S;
    __device__ GTw tw(int) const { return g; }
    __device__ int hi(int c) const { return hi0 + c; }
    __device__ u64 q(int) const { return qq; }
};

// ---------------------------------------------------------------------------
// segment tables
// ---------------------------------------------------------------------------

// Per segment: jobs = outer * nl, job = o * nl + l, and the prime of a job
// depends on l only (so the jobs l, nl + l, 2 nl + l ... can share a CTA).
struct SegHdr {
    int logN, outer, nl, grouped;  // grouped: row units of 16 jobs
    int u_cols, u_rows, xj, pad1;  // xj: the functor's XJ (0 read as 1)
    const ModQ *mq;
    const ulonglong2 *tw;    // forward or inverse table of the segment's context
    const ulonglong2 *ninv;  // N^-1 per prime (Shoup pairs)
};

template <class S>
struct SegIO {
    int nseg, ucols, urows, pad;
    SegHdr h[FHE_SEGS];
    S s[FHE_SEGS];
    // jobs per column unit asked for (2: functors with load2 / same_src)
    static constexpr int XJ = 1;
};

template <class IO>
__device__ __forceinline__ int seg_of(const IO &io, int u, bool rows)
{
    int sg = 0;
    while (sg + 1 < io.nseg && (rows ? io.h[sg + 1].u_rows : io.h[sg + 1].u_cols) <= u) sg++;
    return sg;
}

// ---------------------------------------------------------------------------
// the unit bodies
// ---------------------------------------------------------------------------

// Moves words r = tid + k T (k < 16) through src(r) -> dst(r, v), staged in
// chunks of CH: the chunk's reads are all issued before its first write (the
// compiler does not reorder a global read past a shared-memory write on its
// own), so they overlap; CH = 0 keeps read/write pairs (better for loads
// that already hold several reads each, like ModUp's basis conversion).
template <int CH, class Src, class Dst>
__device__ __forceinline__ void tile_in(int tid, Src src, Dst dst)
{
    constexpr int IT = 16;
    if constexpr (CH > 0) {
        constexpr int K = CH < IT ? CH : IT;
#pragma unroll
        for (int k0 = 0; k0 < IT; k0 += K) {
            u64 v[K];
#pragma unroll
            for (int k = 0; k < K; k++) v[k] = src(tid + (k0 + k) * T);
#pragma unroll
            for (int k = 0; k < K; k++) dst(tid + (k0 + k) * T, v[k]);
        }
    } else {
#pragma unroll 4
        for (int k = 0; k < IT; k++) dst(tid + k * T, src(tid + k * T));
    }
}

// Stores of a forward row pass: word r goes to index idx(r) of state st(r)
// with value val(r) when ok(r).  Staged: the operands the store reads
// (IO::NPRE per word) are loaded for a chunk of words before any of the
// chunk's writes, so those loads overlap.
template <class IO, class StF, class Ok, class Idx, class Val>
__device__ __forceinline__ void tile_out(const IO &io, int tid, StF st, Ok ok, Idx idx, Val val)
{
    constexpr int IT = 16;
    if constexpr (IO::NPRE > 0) {
        constexpr int CH = IO::NPRE == 1 ? IT : IT / 2;
#pragma unroll
        for (int k0 = 0; k0 < IT; k0 += CH) {
            u64 a[CH][IO::NPRE];
#pragma unroll
            for (int k = 0; k < CH; k++) {
                const int r = tid + (k0 + k) * T;
#pragma unroll
                for (int w = 0; w < IO::NPRE; w++) a[k][w] = ok(r) ? io.pre(st(r), idx(r), w) : 0;
            }
#pragma unroll
            for (int k = 0; k < CH; k++) {
                const int r = tid + (k0 + k) * T;
                if (ok(r)) io.store_pre(st(r), idx(r), val(r), a[k]);
            }
        }
    } else {
#pragma unroll 4
        for (int k = 0; k < IT; k++) {
            const int r = tid + k * T;
            if (ok(r)) io.store(st(r), idx(r), val(r));
        }
    }
}

// The jobs of a column unit: slot j (j < NJ) holds job0 + j.
template <int N1, int N2, class IO>
__device__ __forceinline__ int col_jobs(const IO &io, int sg, int lu, typename IO::St *sts, int *lo0)
{
    using Gm = ColGeo<N1, N2, IO::XJ>;
    const SegHdr &H = io.h[sg];
    const int njobs = H.outer * H.nl;
    const int job0 = (lu / Gm::BLK) * Gm::NJ;
    *lo0 = (lu % Gm::BLK) * Gm::NC;
    if (threadIdx.x < Gm::NJ && job0 + (int)threadIdx.x < njobs) io.begin(sg, job0 + threadIdx.x, sts[threadIdx.x]);
    __syncthreads();
    return njobs - job0;  // valid job slots (>= 1)
}

// Stages the first 2^N1 twiddles of each job's prime (the column stages):
// loaded into registers first, stored after the tile loads (latency overlap).
template <int N1, int N2, int XJ = 1>
struct ColTwStage {
    using Gm = ColGeo<N1, N2, XJ>;
    static constexpr int NW = Gm::NJ << N1;
    static constexpr int PER = (NW + T - 1) / T;
    ulonglong2 v[PER];
    template <class St>
    __device__ void load(const SegHdr &H, const St *sts, int nvalid)
    {
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int i = threadIdx.x + k * T, j = i >> N1;
            v[k] = (i < NW && j < nvalid) ? __ldg(H.tw + (size_t)sts[j].prime * Gm::NN + (i & ((1 << N1) - 1)))
                                          : make_ulonglong2(0, 0);
        }
    }
    __device__ void load1(const SegHdr &H, int prime)  // one job per unit
    {
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int i = threadIdx.x + k * T;
            v[k] = i < NW ? __ldg(H.tw + (size_t)prime * Gm::NN + i) : make_ulonglong2(0, 0);
        }
    }
    __device__ void store(ulonglong2 *W) const
    {
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int i = threadIdx.x + k * T;
            if (i < NW) W[(i >> N1) * Gm::TWC + twp(i & ((1 << N1) - 1))] = v[k];
        }
    }
};

// Column units of one job (every ring degree but 2^10): the job's state is
// computed by every thread and stays in registers.
template <int N1, int N2, class IO>
__device__ __forceinline__ void fwd_cols_unit1(const IO &io, int sg, int lu, u64 *sm, ulonglong2 *W)
{
    using Gm = ColGeo<N1, N2, IO::XJ>;
    using C = typename Gm::C;
    const int tid = threadIdx.x;
    const SegHdr &H = io.h[sg];
    const int lo0 = (lu % Gm::BLK) * Gm::NC;
    typename IO::St st;
    io.begin(sg, lu / Gm::BLK, st);
    ColTwStage<N1, N2, IO::XJ> tws;
    tws.load1(H, st.prime);
    const u64 q = H.mq[st.prime].q;
    tile_in<IO::LDCH>(
        tid, [&](int r) { return io.load(st, (Gm::elem(r) << N2) + lo0 + Gm::col(r)); },
        [&](int r, u64 v) { sm[C::at(Gm::col(r), Gm::elem(r))] = v; });
    tws.store(W);
    __syncthreads();
    subtx<N1, true>(sm, tid, ColTw<N1, N2, IO::XJ>{W, q, q});
    __syncthreads();
    u64 *mid = io.inter(st);
#pragma unroll 4
    for (int k = 0; k < 16; k++) {
        const int r = tid + k * T;
        mid[(Gm::elem(r) << N2) + lo0 + Gm::col(r)] = sm[C::at(Gm::col(r), Gm::elem(r))];
    }
}

template <int N1, int N2, class IO>
__device__ __forceinline__ void inv_cols_unit1(const IO &io, int sg, int lu, u64 *sm, ulonglong2 *W)
{
    using Gm = ColGeo<N1, N2, IO::XJ>;
    using C = typename Gm::C;
    const int tid = threadIdx.x;
    const SegHdr &H = io.h[sg];
    const int lo0 = (lu % Gm::BLK) * Gm::NC;
    typename IO::St st;
    io.begin(sg, lu / Gm::BLK, st);
    ColTwStage<N1, N2, IO::XJ> tws;
    tws.load1(H, st.prime);
    const u64 q = H.mq[st.prime].q;
    const ulonglong2 ni = io.final_scale(st);
    const u64 *mid = io.inter(st);
    tile_in<16>(
        tid, [&](int r) { return mid[(Gm::elem(r) << N2) + lo0 + Gm::col(r)]; },
        [&](int r, u64 v) { sm[C::at(Gm::col(r), Gm::elem(r))] = v; });
    tws.store(W);
    __syncthreads();
    subtx<N1, false>(sm, tid, ColTw<N1, N2, IO::XJ>{W, q, q});
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < 16; k++) {
        const int r = tid + k * T;
        io.store(st, (Gm::elem(r) << N2) + lo0 + Gm::col(r),
                 shoup(sm[C::at(Gm::col(r), Gm::elem(r))], ni.x, ni.y, q));
    }
}

// Forward, columns: global stages 0..N1-1.
template <int N1, int N2, class IO>
__device__ __forceinline__ void fwd_cols_unit(const IO &io, int sg, int lu, u64 *sm, ulonglong2 *W,
                                              typename IO::St *sts)
{
    using Gm = ColGeo<N1, N2, IO::XJ>;
    using C = typename Gm::C;
    if constexpr (Gm::NJ == 1) {
        fwd_cols_unit1<N1, N2>(io, sg, lu, sm, W);
        return;
    }
    const int tid = threadIdx.x;
    int lo0;
    const int nvalid = col_jobs<N1, N2>(io, sg, lu, sts, &lo0);
    const SegHdr &H = io.h[sg];
    ColTwStage<N1, N2, IO::XJ> tws;
    tws.load(H, sts, nvalid);
    const u64 q0 = H.mq[sts[0].prime].q, q1 = nvalid > 1 ? H.mq[sts[Gm::NJ - 1].prime].q : q0;
    bool paired = false;
    if constexpr (Gm::PAIRED) {
        // both slots at once: word r (slot 0) and word r + NC SZ (slot 1)
        // share column and element, so each source word is loaded once
        static_assert(Gm::NJ == 2 && 2 * Gm::NC * Gm::SZ == 16 * T, "paired column unit");
        paired = nvalid >= 2 && io.same_src(sts[0], sts[1]);  // uniform in the CTA
        if (paired) {
#pragma unroll PAIRED_UNROLL
            for (int k = 0; k < 8; k++) {
                const int r = tid + k * T;
                u64 v0, v1;
                io.load2(sts[0], sts[1], (Gm::elem(r) << N2) + lo0 + Gm::col(r), v0, v1);
                sm[C::at(Gm::col(r), Gm::elem(r))] = v0;
                sm[C::at(Gm::NC + Gm::col(r), Gm::elem(r))] = v1;
            }
        }
    }
    if (!paired) {
        if constexpr (Gm::PAIRED && FHE_NTT_PAIRED_FALLBACK_ROLLED) {
            // the rare unit whose jobs read different sources: a rolled loop
            // (small code beside the paired path)
#pragma unroll 1
            for (int k = 0; k < 16; k++) {
                const int r = tid + k * T, j = Gm::jslot(r);
                sm[C::at(j * Gm::NC + Gm::col(r), Gm::elem(r))] =
                    j < nvalid ? io.load(sts[j], (Gm::elem(r) << N2) + lo0 + Gm::col(r)) : 0;
            }
        } else {
            tile_in<IO::LDCH>(
                tid,
                [&](int r) {
                    const int j = Gm::jslot(r);
                    return j < nvalid ? io.load(sts[j], (Gm::elem(r) << N2) + lo0 + Gm::col(r)) : 0;
                },
                [&](int r, u64 v) { sm[C::at(Gm::jslot(r) * Gm::NC + Gm::col(r), Gm::elem(r))] = v; });
        }
    }
    tws.store(W);
    __syncthreads();
    subtx<N1, true>(sm, tid, ColTw<N1, N2, IO::XJ>{W, q0, q1});
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < 16; k++) {
        const int r = tid + k * T, j = Gm::jslot(r);
        if (j < nvalid)
            io.inter(sts[j])[(Gm::elem(r) << N2) + lo0 + Gm::col(r)] =
                sm[C::at(j * Gm::NC + Gm::col(r), Gm::elem(r))];
    }
}

// Inverse, columns: undoes global stages N1-1..0, then scales (N^-1 times the
// job's constant) and stores.
template <int N1, int N2, class IO>
__device__ __forceinline__ void inv_cols_unit(const IO &io, int sg, int lu, u64 *sm, ulonglong2 *W,
                                              typename IO::St *sts)
{
    using Gm = ColGeo<N1, N2, IO::XJ>;
    using C = typename Gm::C;
    if constexpr (Gm::NJ == 1) {
        inv_cols_unit1<N1, N2>(io, sg, lu, sm, W);
        return;
    }
    const int tid = threadIdx.x;
    int lo0;
    const int nvalid = col_jobs<N1, N2>(io, sg, lu, sts, &lo0);
    const SegHdr &H = io.h[sg];
    ColTwStage<N1, N2, IO::XJ> tws;
    tws.load(H, sts, nvalid);
    const u64 q0 = H.mq[sts[0].prime].q, q1 = nvalid > 1 ? H.mq[sts[Gm::NJ - 1].prime].q : q0;
    tile_in<16>(
        tid,
        [&](int r) {
            const int j = Gm::jslot(r);
            return j < nvalid ? io.inter(sts[j])[(Gm::elem(r) << N2) + lo0 + Gm::col(r)] : 0;
        },
        [&](int r, u64 v) { sm[C::at(Gm::jslot(r) * Gm::NC + Gm::col(r), Gm::elem(r))] = v; });
    tws.store(W);
    __syncthreads();
    subtx<N1, false>(sm, tid, ColTw<N1, N2, IO::XJ>{W, q0, q1});
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < 16; k++) {
        const int r = tid + k * T, j = Gm::jslot(r);
        if (j < nvalid) {
            const ulonglong2 ni = io.final_scale(sts[j]);
            const u64 q = j == 0 ? q0 : q1;
            io.store(sts[j], (Gm::elem(r) << N2) + lo0 + Gm::col(r),
                     shoup(sm[C::at(j * Gm::NC + Gm::col(r), Gm::elem(r))], ni.x, ni.y, q));
        }
    }
}

// The jobs of a row unit.  Grouped: slots jj < 16 hold jobs (oc 16 + jj) nl
// + l, rows hi0 .. hi0+R-1; single: slot 0 holds the job, rows hi0 ..
// hi0+NS-1.  Returns the number of valid slots.
template <int N1, int N2, bool GRP, class IO>
__device__ __forceinline__ int row_jobs(const IO &io, int sg, int lu, typename IO::St *sts, int *hi0)
{
    using Gm = RowGeo<N1, N2>;
    const SegHdr &H = io.h[sg];
    int nvalid;
    if (GRP) {
        const int OC = (H.outer + ROW_J - 1) / ROW_J;
        const int hc = lu % Gm::CH, t = lu / Gm::CH;
        const int oc = t % OC, l = t / OC;
        *hi0 = hc * Gm::R;
        nvalid = min(ROW_J, H.outer - oc * ROW_J);
        if ((int)threadIdx.x < nvalid) io.begin(sg, (oc * ROW_J + threadIdx.x) * H.nl + l, sts[threadIdx.x]);
    } else {
        *hi0 = (lu % Gm::CHS) * Gm::NS;
        nvalid = 1;
        if (threadIdx.x == 0) io.begin(sg, lu / Gm::CHS, sts[0]);
    }
    __syncthreads();
    return nvalid;
}

// Grouped rows stage the R rows' twiddles: entry k of row r is the stage
// u = floor(log2(k+1)) twiddle with in-stage index (hi0 + r) 2^u + k+1-2^u.
template <int N1, int N2>
struct RowTwStage {
    using Gm = RowGeo<N1, N2>;
    static constexpr int NW = Gm::R * (Gm::SZ - 1);
    static constexpr int PER = (NW + T - 1) / T;
    ulonglong2 v[PER];
    __device__ void load(const ulonglong2 *tw, int hi0)
    {
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int i = threadIdx.x + k * T;
            v[k] = make_ulonglong2(0, 0);
            if (i < NW) {
                const int r = i / (Gm::SZ - 1), e = i % (Gm::SZ - 1);
                const int u = 31 - __clz(e + 1);
                v[k] = __ldg(tw + (1 << (N1 + u)) + ((hi0 + r) << u) + (e + 1 - (1 << u)));
            }
        }
    }
    __device__ void store(ulonglong2 *W) const
    {
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int i = threadIdx.x + k * T;
            if (i < NW) W[(i / (Gm::SZ - 1)) * Gm::TWR + twp(i % (Gm::SZ - 1))] = v[k];
        }
    }
};

// word r of a row unit -> (sub-transform c = r >> N2, element f); the job
// slot and row of c
template <int N1, int N2, bool GRP>
struct RowMap {
    using Gm = RowGeo<N1, N2>;
    int hi0;
    __device__ int c(int r) const { return r >> N2; }
    __device__ int f(int r) const { return r & (Gm::SZ - 1); }
    __device__ int slot(int r) const { return GRP ? c(r) / Gm::R : 0; }
    __device__ int row(int r) const { return hi0 + (GRP ? c(r) % Gm::R : c(r)); }
};

// Forward, rows: global stages N1..N1+N2-1, reduction to [0, q), store.
template <int N1, int N2, bool GRP, class IO>
__device__ __forceinline__ void fwd_rows_unit(const IO &io, int sg, int lu, u64 *sm, ulonglong2 *W,
                                          typename IO::St *sts)
{
    using Gm = RowGeo<N1, N2>;
    using C = typename Gm::C;
    const int tid = threadIdx.x;
    const SegHdr &H = io.h[sg];
    int hi0;
    const int nvalid = row_jobs<N1, N2, GRP>(io, sg, lu, sts, &hi0);
    const RowMap<N1, N2, GRP> mp{hi0};
    const int prime = sts[0].prime;
    const ModQ mqp = H.mq[prime];
    const ulonglong2 *tw = H.tw + (size_t)prime * Gm::NN;
    RowTwStage<N1, N2> tws;
    if (GRP) tws.load(tw, hi0);
    tile_in<16>(
        tid,
        [&](int r) {
            const int j = mp.slot(r);
            return j < nvalid ? io.inter(sts[j])[(mp.row(r) << N2) + mp.f(r)] : 0;
        },
        [&](int r, u64 v) { sm[C::at(mp.c(r), mp.f(r))] = v; });
    if (GRP) tws.store(W);
    __syncthreads();
    if (GRP)
        subtx<N2, true>(sm, tid, RowGrpTw<N1, N2>{W, hi0, mqp.q, N1});
    else
        subtx<N2, true>(sm, tid, RowOneTw{GTw{tw}, hi0, mqp.q, N1});
    __syncthreads();
    tile_out(
        io, tid, [&](int r) -> const typename IO::St & { return sts[mp.slot(r)]; },
        [&](int r) { return mp.slot(r) < nvalid; }, [&](int r) { return (mp.row(r) << N2) + mp.f(r); },
        [&](int r) { return reduce64(sm[C::at(mp.c(r), mp.f(r))], mqp); });
}

// Inverse, rows first: undoes global stages N1+N2-1..N1.
template <int N1, int N2, bool GRP, class IO>
__device__ __forceinline__ void inv_rows_unit(const IO &io, int sg, int lu, u64 *sm, ulonglong2 *W,
                                          typename IO::St *sts)
{
    using Gm = RowGeo<N1, N2>;
    using C = typename Gm::C;
    const int tid = threadIdx.x;
    const SegHdr &H = io.h[sg];
    int hi0;
    const int nvalid = row_jobs<N1, N2, GRP>(io, sg, lu, sts, &hi0);
    const RowMap<N1, N2, GRP> mp{hi0};
    const int prime = sts[0].prime;
    const u64 q = H.mq[prime].q;
    const ulonglong2 *tw = H.tw + (size_t)prime * Gm::NN;
    RowTwStage<N1, N2> tws;
    if (GRP) tws.load(tw, hi0);
    tile_in<IO::LDCH>(
        tid,
        [&](int r) {
            const int j = mp.slot(r);
            return j < nvalid ? io.load(sts[j], (mp.row(r) << N2) + mp.f(r)) : 0;
        },
        [&](int r, u64 v) { sm[C::at(mp.c(r), mp.f(r))] = v; });
    if (GRP) tws.store(W);
    __syncthreads();
    if (GRP)
        subtx<N2, false>(sm, tid, RowGrpTw<N1, N2>{W, hi0, q, N1});
    else
        subtx<N2, false>(sm, tid, RowOneTw{GTw{tw}, hi0, q, N1});
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < 16; k++) {
        const int r = tid + k * T, j = mp.slot(r);
        if (j < nvalid) io.inter(sts[j])[(mp.row(r) << N2) + mp.f(r)] = sm[C::at(mp.c(r), mp.f(r))];
    }
}

// ---------------------------------------------------------------------------
// kernels: one per (functor, direction, pass, range of ring degrees).  A
// launch whose segments share one ring degree takes the kernel of that
// degree alone (the smallest code, the best instruction-fetch behaviour);
// only a launch that mixes ring degrees takes the 2^13..2^15 kernel, which
// dispatches every unit on its segment's degree.
// ---------------------------------------------------------------------------

template <int L>
struct Deg {
    static constexpr int N1 = (L + 1) / 2, N2 = L / 2;
};

// f(Deg<logN>) for logN in [L, HI]; with L == HI no test (the host sends only
// that degree), otherwise the last degree is the fall-through.
template <int L, int HI, class F>
__device__ __forceinline__ void by_degree(int logN, F f)
{
    if constexpr (L == HI) {
        f(Deg<L>{});
    } else {
        if (logN == L)
            f(Deg<L>{});
        else
            by_degree<L + 1, HI>(logN, f);
    }
}

template <class IO, int LO, int HI>
__global__ void __launch_bounds__(T, IO::XJ == 2 ? FHE_NTT_MINB_PAIRED : FHE_NTT_MINB)
    k_fwd_cols(const __grid_constant__ IO io)
{
    pdl_begin();
    __shared__ u64 sm[SM_WORDS];
    __shared__ ulonglong2 W[TW_WORDS];
    __shared__ typename IO::St sts[ROW_J];
    for (int u = blockIdx.x; u < io.ucols; u += gridDim.x) {
        const int sg = seg_of(io, u, false), lu = u - io.h[sg].u_cols;
        by_degree<LO, HI>(io.h[sg].logN, [&](auto d) {
            fwd_cols_unit<decltype(d)::N1, decltype(d)::N2>(io, sg, lu, sm, W, sts);
        });
        __syncthreads();
    }
}

template <class IO, int LO, int HI>
__global__ void __launch_bounds__(T, IO::NPRE >= 2 ? FHE_NTT_MINB_ST2 : FHE_NTT_MINB)
    k_fwd_rows(const __grid_constant__ IO io)
{
    pdl_begin();
    __shared__ u64 sm[SM_WORDS];
    __shared__ ulonglong2 W[TW_WORDS];
    __shared__ typename IO::St sts[ROW_J];
    for (int u = blockIdx.x; u < io.urows; u += gridDim.x) {
        const int sg = seg_of(io, u, true), lu = u - io.h[sg].u_rows;
        if (io.h[sg].grouped)
            by_degree<LO, HI>(io.h[sg].logN, [&](auto d) {
                fwd_rows_unit<decltype(d)::N1, decltype(d)::N2, true>(io, sg, lu, sm, W, sts);
            });
        else
            by_degree<LO, HI>(io.h[sg].logN, [&](auto d) {
                fwd_rows_unit<decltype(d)::N1, decltype(d)::N2, false>(io, sg, lu, sm, W, sts);
            });
        __syncthreads();
    }
}

template <class IO, int LO, int HI>
__global__ void __launch_bounds__(T, FHE_NTT_MINB) k_inv_rows(const __grid_constant__ IO io)
{
    pdl_begin();
    __shared__ u64 sm[SM_WORDS];
    __shared__ ulonglong2 W[TW_WORDS];
    __shared__ typename IO::St sts[ROW_J];
    for (int u = blockIdx.x; u < io.urows; u += gridDim.x) {
        const int sg = seg_of(io, u, true), lu = u - io.h[sg].u_rows;
        if (io.h[sg].grouped)
            by_degree<LO, HI>(io.h[sg].logN, [&](auto d) {
                inv_rows_unit<decltype(d)::N1, decltype(d)::N2, true>(io, sg, lu, sm, W, sts);
            });
        else
            by_degree<LO, HI>(io.h[sg].logN, [&](auto d) {
                inv_rows_unit<decltype(d)::N1, decltype(d)::N2, false>(io, sg, lu, sm, W, sts);
            });
        __syncthreads();
    }
}

template <class IO, int LO, int HI>
__global__ void __launch_bounds__(T, FHE_NTT_MINB) k_inv_cols(const __grid_constant__ IO io)
{
    pdl_begin();
    __shared__ u64 sm[SM_WORDS];
    __shared__ ulonglong2 W[TW_WORDS];
    __shared__ typename IO::St sts[ROW_J];
    for (int u = blockIdx.x; u < io.ucols; u += gridDim.x) {
        const int sg = seg_of(io, u, false), lu = u - io.h[sg].u_cols;
        by_degree<LO, HI>(io.h[sg].logN, [&](auto d) {
            inv_cols_unit<decltype(d)::N1, decltype(d)::N2>(io, sg, lu, sm, W, sts);
        });
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// load/store functors (one payload per segment)
// ---------------------------------------------------------------------------

// A limb map: job (o, l) reads limb in_limb[l] of outer item o and writes
// limb out_limb[l]; prime[l]; the inverse's final scale is N^-1 times the
// map entry's constant (scale[l], device) or plain N^-1.
struct MapSeg {
    const u64 *in;
    u64 *out;
    long long in_outer, out_outer;  // u64 elements
    const ulonglong2 *scale;
    uint8_t in_limb[FHE_MAXP], out_limb[FHE_MAXP], prime[FHE_MAXP];
};

struct IOMap : SegIO<MapSeg> {
    struct St {
        const u64 *in;
        u64 *out;
        ulonglong2 fs;
        int prime;
    };
    __device__ void begin(int sg, int job, St &t) const
    {
        const SegHdr &H = h[sg];
        const MapSeg &S = s[sg];
        const int N = 1 << H.logN, o = job / H.nl, l = job % H.nl;
        t.in = S.in + o * S.in_outer + (long long)S.in_limb[l] * N;
        t.out = S.out + o * S.out_outer + (long long)S.out_limb[l] * N;
        t.prime = S.prime[l];
        t.fs = S.scale ? S.scale[l] : H.ninv[t.prime];
    }
    __device__ u64 load(const St &t, int i) const { return t.in[i]; }
    __device__ void store(const St &t, int i, u64 v) const { t.out[i] = v; }
    static constexpr int NPRE = 0;   // operands the store reads
    static constexpr int LDCH = 16;  // loads staged per chunk (0: not staged)
    __device__ u64 pre(const St &, int, int) const { return 0; }
    __device__ void store_pre(const St &t, int i, u64 v, const u64 *) const { t.out[i] = v; }
    __device__ u64 *inter(const St &t) const { return t.out; }
    __device__ ulonglong2 final_scale(const St &t) const { return t.fs; }
};

// A scaled inverse whose last map entry (limb l-1 of the relinearisation
// accumulators) loads y = acc + (P mod q) addend: the first step of the
// relinearisation fused with the modulus switch.  Job = (ct, poly) * nl + entry.
struct YSeg : MapSeg {
    const u64 *abase;
    long long a_outer, a_poly;
    int amask, alimb;
    u64 Pm, Pm_s, qm;
};

struct IOScaledY : SegIO<YSeg> {
    struct St {
        const u64 *in, *add;
        u64 *out;
        ulonglong2 fs;
        u64 Pm, Pm_s, qm;
        int prime;
    };
    __device__ void begin(int sg, int job, St &t) const
    {
        const SegHdr &H = h[sg];
        const YSeg &S = s[sg];
        const int N = 1 << H.logN, o = job / H.nl, e = job % H.nl, pi = o & 1;
        const long long c = o >> 1;
        t.in = S.in + o * S.in_outer + (long long)S.in_limb[e] * N;
        t.out = S.out + o * S.out_outer + (long long)S.out_limb[e] * N;
        t.prime = S.prime[e];
        t.fs = S.scale[e];
        t.add = (e == H.nl - 1 && ((S.amask >> pi) & 1)) ? S.abase + c * S.a_outer + pi * S.a_poly + (long long)S.alimb * N
                                                          : nullptr;
        t.Pm = S.Pm;
        t.Pm_s = S.Pm_s;
        t.qm = S.qm;
    }
    __device__ u64 load(const St &t, int i) const
    {
        return t.add ? addmod(t.in[i], shoup(t.add[i], t.Pm, t.Pm_s, t.qm), t.qm) : t.in[i];
    }
    __device__ void store(const St &t, int i, u64 v) const { t.out[i] = v; }
    static constexpr int NPRE = 0;
    static constexpr int LDCH = 16;
    __device__ u64 pre(const St &, int, int) const { return 0; }
    __device__ void store_pre(const St &t, int i, u64 v, const u64 *) const { t.out[i] = v; }
    __device__ u64 *inter(const St &t) const { return t.out; }
    __device__ ulonglong2 final_scale(const St &t) const { return t.fs; }
};

// ModUp: extended limb t of digit j of ct c:  y = sum_a t_a (Q_j/q_a) mod r,
// where the source limbs already hold t_a = [x_a (Q_j/q_a)^-1]_{q_a} (the
// inverse NTT that produced them applied that factor).  Job = c * njobs + e
// (entry e: digit, target limb, prime).
struct ModUpSeg {
    const u64 *d2c;  // [count][l][N] coefficient domain
    u64 *ext;        // [count][dnum][l+K][N]
    const ModUpParams *P;
    int l, K, dnum, pad;
};

struct IOModUp : SegIO<ModUpSeg> {
    struct St {
        const u64 *src;
        u64 *dst;
        int nsrc, prime, N, pad;
        ModQ mt;
        u64 hat[FHE_MAXK];
    };
    __device__ void begin(int sg, int job, St &t) const
    {
        const SegHdr &H = h[sg];
        const ModUpSeg &S = s[sg];
        const int N = 1 << H.logN, c = job / H.nl, e = job % H.nl;
        const ModUpParams *P = S.P;
        const int j = P->job_digit[e], tg = P->job_tgt[e];
        const int lo = P->digit_lo[j];
        t.nsrc = P->digit_n[j];
        t.N = N;
        t.src = S.d2c + ((long long)c * S.l + lo) * N;
        t.dst = S.ext + (((long long)c * S.dnum + j) * (S.l + S.K) + tg) * N;
        t.prime = P->job_prime[e];
        t.mt = H.mq[t.prime];
#pragma unroll
        for (int a = 0; a < FHE_MAXK; a++)
            if (a < t.nsrc) t.hat[a] = P->hat[j][a][tg];
    }
    __device__ u64 load(const St &t, int n) const
    {
        u128 acc = 0;
#pragma unroll
        for (int a = 0; a < FHE_MAXK; a++)
            if (a < t.nsrc) acc += (u128)t.src[(long long)a * t.N + n] * t.hat[a];
        return conv_reduce(acc, t.mt);
    }
    // two targets of one digit (same sources): each source word loaded once
    static constexpr int XJ = 2;
    __device__ bool same_src(const St &a, const St &b) const { return a.src == b.src && a.nsrc == b.nsrc; }
    __device__ void load2(const St &a, const St &b, int n, u64 &v0, u64 &v1) const
    {
        u128 s0 = 0, s1 = 0;
#pragma unroll
        for (int i = 0; i < FHE_MAXK; i++)
            if (i < a.nsrc) {
                const u64 x = a.src[(long long)i * a.N + n];
                s0 += (u128)x * a.hat[i];
                s1 += (u128)x * b.hat[i];
            }
        v0 = conv_reduce(s0, a.mt);
        v1 = conv_reduce(s1, b.mt);
    }
    __device__ void store(const St &t, int k, u64 v) const { t.dst[k] = v; }
    static constexpr int NPRE = 0;
    static constexpr int LDCH = FHE_NTT_MULTI_LDCH;  // each load reads several limbs
    __device__ u64 pre(const St &, int, int) const { return 0; }
    __device__ void store_pre(const St &t, int k, u64 v, const u64 *) const { t.dst[k] = v; }
    __device__ u64 *inter(const St &t) const { return t.dst; }
    __device__ ulonglong2 final_scale(const St &) const { return make_ulonglong2(0, 0); }
};

// ModDown of poly pi of ct c, data limb i:
//   delta_i = sum_k t_k * (p P/p_k mod q_i),  out_i = (acc_i - delta_i) P^-1 + addend_i,
// where the special limbs already hold t_k = [acc_{P,k} p^-1 (P/p_k)^-1]_{p_k}
// (applied by the inverse NTT that produced them).  Job = (c, pi) * l + i.
struct ModDownSeg {
    const u64 *accP;  // [count][2][K][N] coefficient domain
    const u64 *acc;   // [count][2][l+K][N] NTT domain
    const u64 *abase;
    long long a_outer, a_poly;
    u64 *out;         // [count][2][l][N]
    const ModDownParams *P;
    int l, K, amask, pad;
};

struct IOModDown : SegIO<ModDownSeg> {
    struct St {
        const u64 *w, *acc, *add;
        u64 *out;
        int prime, K, N, pad;
        ModQ mi;
        u64 pinv, pinv_s;
        u64 phat[FHE_MAXK];
    };
    __device__ void begin(int sg, int job, St &t) const
    {
        const SegHdr &H = h[sg];
        const ModDownSeg &S = s[sg];
        const int N = 1 << H.logN, l = S.l, K = S.K;
        const int c = job / (2 * l), pi = (job / l) % 2, i = job % l;
        t.w = S.accP + ((long long)c * 2 + pi) * K * N;
        t.acc = S.acc + (((long long)c * 2 + pi) * (l + K) + i) * N;
        t.add = ((S.amask >> pi) & 1) ? S.abase + c * S.a_outer + pi * S.a_poly + (long long)i * N : nullptr;
        t.out = S.out + (((long long)c * 2 + pi) * l + i) * N;
        t.prime = i;
        t.K = K;
        t.N = N;
        t.mi = H.mq[i];
        t.pinv = S.P->pinv[i];
        t.pinv_s = S.P->pinv_s[i];
#pragma unroll
        for (int k = 0; k < FHE_MAXK; k++)
            if (k < K) t.phat[k] = S.P->phat[k][i];
    }
    __device__ u64 load(const St &t, int n) const
    {
        u128 a = 0;
#pragma unroll
        for (int k = 0; k < FHE_MAXK; k++)
            if (k < t.K) a += (u128)t.w[(long long)k * t.N + n] * t.phat[k];
        return conv_reduce(a, t.mi);
    }
    // two data limbs of one (ct, poly): the special limbs loaded once
    static constexpr int XJ = 2;
    __device__ bool same_src(const St &a, const St &b) const { return a.w == b.w && a.K == b.K; }
    __device__ void load2(const St &a, const St &b, int n, u64 &v0, u64 &v1) const
    {
        u128 s0 = 0, s1 = 0;
#pragma unroll
        for (int k = 0; k < FHE_MAXK; k++)
            if (k < a.K) {
                const u64 x = a.w[(long long)k * a.N + n];
                s0 += (u128)x * a.phat[k];
                s1 += (u128)x * b.phat[k];
            }
        v0 = conv_reduce(s0, a.mi);
        v1 = conv_reduce(s1, b.mi);
    }
    __device__ void store(const St &t, int k, u64 v) const
    {
        const u64 q = t.mi.q;
        u64 r = shoup(submod(t.acc[k], v, q), t.pinv, t.pinv_s, q);
        if (t.add) r = addmod(r, t.add[k], q);
        t.out[k] = r;
    }
    static constexpr int NPRE = 2;  // accumulator, addend
    static constexpr int LDCH = 16;
    __device__ u64 pre(const St &t, int k, int w) const { return w == 0 ? t.acc[k] : (t.add ? t.add[k] : 0); }
    __device__ void store_pre(const St &t, int k, u64 v, const u64 *pv) const
    {
        const u64 q = t.mi.q;
        u64 r = shoup(submod(pv[0], v, q), t.pinv, t.pinv_s, q);
        if (t.add) r = addmod(r, pv[1], q);
        t.out[k] = r;
    }
    __device__ u64 *inter(const St &t) const { return t.out; }
    __device__ ulonglong2 final_scale(const St &) const { return make_ulonglong2(0, 0); }
};

// Modulus switch l -> l-1 of poly pi of ct c, limb i < l-1:
//   delta_i = p w mod q_i,  out_i = (x_i - delta_i) q_{l-1}^-1,
// where `last` already holds w = [x_{l-1} p^-1]_{q_{l-1}} in the coefficient
// domain (applied by the inverse NTT that produced it).
// Job = (c, pi) * (l-1) + i.
struct SwitchSeg {
    const u64 *last;  // [count][npoly][N] coefficient domain
    const u64 *in;    // [count][npoly][l][N]
    u64 *out;         // [count][npoly][l-1][N]
    const ModSwitchParams *P;
    int l, npoly;
};

struct IOModSwitch : SegIO<SwitchSeg> {
    struct St {
        const u64 *last, *in;
        u64 *out;
        int prime, pad;
        u64 q, pi, pis, qi, qis;
    };
    __device__ void begin(int sg, int job, St &t) const
    {
        const SegHdr &H = h[sg];
        const SwitchSeg &S = s[sg];
        const int N = 1 << H.logN, l = S.l, np = S.npoly;
        const int c = job / (np * (l - 1)), pi = (job / (l - 1)) % np, i = job % (l - 1);
        t.last = S.last + ((long long)c * np + pi) * N;
        t.in = S.in + (((long long)c * np + pi) * l + i) * N;
        t.out = S.out + (((long long)c * np + pi) * (l - 1) + i) * N;
        t.prime = i;
        t.q = H.mq[i].q;
        t.pi = S.P->p_i[i];
        t.pis = S.P->p_i_s[i];
        t.qi = S.P->qinv[i];
        t.qis = S.P->qinv_s[i];
    }
    // [0, 4q): feeds the forward transform
    __device__ u64 load(const St &t, int n) const { return shoup_lazy4_chain(t.last[n], t.pi, t.pis, 0 - t.q); }
    __device__ void store(const St &t, int k, u64 v) const { t.out[k] = shoup(submod(t.in[k], v, t.q), t.qi, t.qis, t.q); }
    static constexpr int NPRE = 1;  // the limb being switched
    static constexpr int LDCH = 16;
    __device__ u64 pre(const St &t, int k, int) const { return t.in[k]; }
    __device__ void store_pre(const St &t, int k, u64 v, const u64 *pv) const
    {
        t.out[k] = shoup(submod(pv[0], v, t.q), t.qi, t.qis, t.q);
    }
    __device__ u64 *inter(const St &t) const { return t.out; }
    __device__ ulonglong2 final_scale(const St &) const { return make_ulonglong2(0, 0); }
};

// Relinearisation fused with the modulus switch that follows it (l -> l-1)
// for poly pi of ct c, kept limb i < l-1:
//   correction_i = sum_{k<K} t_k h[k][i] + w h[K][i] (coefficient domain),
//   out_i = (acc_i P^-1 + add_i - NTT(correction)_i) q_{l-1}^-1,
// where src holds t_0..t_{K-1} (the special limbs, already scaled) and w.
// Job = (c, pi) * (l-1) + i.
struct RelinMSSeg {
    const u64 *src;  // [count][2][K+1][N] coefficient domain
    const u64 *acc;  // [count][2][l+K][N] NTT domain
    const u64 *abase;
    long long a_outer, a_poly;
    u64 *out;        // [count][2][l-1][N]
    const RelinMSParams *P;
    int l, K, amask, pad;
};

struct IORelinMS : SegIO<RelinMSSeg> {
    struct St {
        const u64 *w, *acc, *add;
        u64 *out;
        int prime, K, N, pad;
        ModQ mi;
        u64 pinv, pinv_s, qminv, qminv_s;
        u64 h[FHE_MAXK];
    };
    __device__ void begin(int sg, int job, St &t) const
    {
        const SegHdr &H = h[sg];
        const RelinMSSeg &S = s[sg];
        const int N = 1 << H.logN, l = S.l, K = S.K, m = l - 1;
        const int c = job / (2 * m), pi = (job / m) % 2, i = job % m;
        t.w = S.src + ((long long)c * 2 + pi) * (K + 1) * N;
        t.acc = S.acc + (((long long)c * 2 + pi) * (l + K) + i) * N;
        t.add = ((S.amask >> pi) & 1) ? S.abase + c * S.a_outer + pi * S.a_poly + (long long)i * N : nullptr;
        t.out = S.out + (((long long)c * 2 + pi) * m + i) * N;
        t.prime = i;
        t.K = K;
        t.N = N;
        t.mi = H.mq[i];
        t.pinv = S.P->pinv[i];
        t.pinv_s = S.P->pinv_s[i];
        t.qminv = S.P->qminv[i];
        t.qminv_s = S.P->qminv_s[i];
#pragma unroll
        for (int k = 0; k < FHE_MAXK; k++)
            if (k <= K) t.h[k] = S.P->h[k][i];
    }
    // K + 1 <= FHE_MAXK products of canonical residues: below 2^(2b+3)
    __device__ u64 load(const St &t, int n) const
    {
        u128 a = 0;
#pragma unroll
        for (int k = 0; k < FHE_MAXK; k++)
            if (k <= t.K) a += (u128)t.w[(long long)k * t.N + n] * t.h[k];
        return conv_reduce(a, t.mi);
    }
    // two data limbs of one (ct, poly): the K + 1 sources loaded once
    static constexpr int XJ = 2;
    __device__ bool same_src(const St &a, const St &b) const { return a.w == b.w && a.K == b.K; }
    __device__ void load2(const St &a, const St &b, int n, u64 &v0, u64 &v1) const
    {
        u128 s0 = 0, s1 = 0;
#pragma unroll
        for (int k = 0; k < FHE_MAXK; k++)
            if (k <= a.K) {
                const u64 x = a.w[(long long)k * a.N + n];
                s0 += (u128)x * a.h[k];
                s1 += (u128)x * b.h[k];
            }
        v0 = conv_reduce(s0, a.mi);
        v1 = conv_reduce(s1, b.mi);
    }
    __device__ u64 combine(const St &t, u64 accv, u64 addv, u64 v) const
    {
        const u64 q = t.mi.q;
        u64 r = shoup(accv, t.pinv, t.pinv_s, q);
        if (t.add) r = addmod(r, addv, q);
        return shoup(submod(r, v, q), t.qminv, t.qminv_s, q);
    }
    __device__ void store(const St &t, int k, u64 v) const { t.out[k] = combine(t, t.acc[k], t.add ? t.add[k] : 0, v); }
    static constexpr int NPRE = 2;  // accumulator, addend
    static constexpr int LDCH = FHE_NTT_MULTI_LDCH;  // each load reads several limbs
    __device__ u64 pre(const St &t, int k, int w) const { return w == 0 ? t.acc[k] : (t.add ? t.add[k] : 0); }
    __device__ void store_pre(const St &t, int k, u64 v, const u64 *pv) const { t.out[k] = combine(t, pv[0], pv[1], v); }
    __device__ u64 *inter(const St &t) const { return t.out; }
    __device__ ulonglong2 final_scale(const St &) const { return make_ulonglong2(0, 0); }
};

// k modulus switches at once (l -> l-k), poly pi of ct c, kept limb i < l-k:
//   correction_i = sum_{t<k} w_t G[t][i],  out_i = (x_i - NTT(correction)_i) D_k^-1.
// Job = (c, pi) * (l-k) + i.
struct MultiSeg {
    const u64 *src;  // [count][npoly][k][N] coefficient domain: w_0 .. w_{k-1}
    const u64 *in;   // [count][npoly][l][N]
    u64 *out;        // [count][npoly][l-k][N]
    const MultiSwitchParams *P;
    int l, k, npoly, pad;
};

struct IOMultiSwitch : SegIO<MultiSeg> {
    struct St {
        const u64 *w, *in;
        u64 *out;
        int prime, k, N, pad;
        ModQ mi;
        u64 dinv, dinv_s;
        u64 g[FHE_MAXK];
    };
    __device__ void begin(int sg, int job, St &t) const
    {
        const SegHdr &H = h[sg];
        const MultiSeg &S = s[sg];
        const int N = 1 << H.logN, kept = S.l - S.k, np = S.npoly;
        const int c = job / (np * kept), pi = (job / kept) % np, i = job % kept;
        t.w = S.src + ((long long)c * np + pi) * S.k * N;
        t.in = S.in + (((long long)c * np + pi) * S.l + i) * N;
        t.out = S.out + (((long long)c * np + pi) * kept + i) * N;
        t.prime = i;
        t.k = S.k;
        t.N = N;
        t.mi = H.mq[i];
        t.dinv = S.P->Dinv[i];
        t.dinv_s = S.P->Dinv_s[i];
#pragma unroll
        for (int j = 0; j < FHE_MAXK; j++)
            if (j < S.k) t.g[j] = S.P->G[j][i];
    }
    __device__ u64 load(const St &t, int n) const
    {
        u128 a = 0;
#pragma unroll
        for (int j = 0; j < FHE_MAXK; j++)
            if (j < t.k) a += (u128)t.w[(long long)j * t.N + n] * t.g[j];
        return conv_reduce(a, t.mi);
    }
    // two kept limbs of one (ct, poly): the k switch values loaded once
    static constexpr int XJ = 2;
    __device__ bool same_src(const St &a, const St &b) const { return a.w == b.w && a.k == b.k; }
    __device__ void load2(const St &a, const St &b, int n, u64 &v0, u64 &v1) const
    {
        u128 s0 = 0, s1 = 0;
#pragma unroll
        for (int j = 0; j < FHE_MAXK; j++)
            if (j < a.k) {
                const u64 x = a.w[(long long)j * a.N + n];
                s0 += (u128)x * a.g[j];
                s1 += (u128)x * b.g[j];
            }
        v0 = conv_reduce(s0, a.mi);
        v1 = conv_reduce(s1, b.mi);
    }
    __device__ void store(const St &t, int j, u64 v) const
    {
        t.out[j] = shoup(submod(t.in[j], v, t.mi.q), t.dinv, t.dinv_s, t.mi.q);
    }
    static constexpr int NPRE = 1;
    static constexpr int LDCH = FHE_NTT_MULTI_LDCH;  // each load reads several limbs
    __device__ u64 pre(const St &t, int j, int) const { return t.in[j]; }
    __device__ void store_pre(const St &t, int j, u64 v, const u64 *pv) const
    {
        t.out[j] = shoup(submod(pv[0], v, t.mi.q), t.dinv, t.dinv_s, t.mi.q);
    }
    __device__ u64 *inter(const St &t) const { return t.out; }
    __device__ ulonglong2 final_scale(const St &) const { return make_ulonglong2(0, 0); }
};

// ---------------------------------------------------------------------------
// host side: unit counts, grids, launches
// ---------------------------------------------------------------------------

struct Split {
    int n1, n2, ns1, ns2;
};

Split split_of(int logN)
{
    Split s;
    s.n1 = (logN + 1) / 2;
    s.n2 = logN / 2;
    s.ns1 = 2048 >> s.n1;
    s.ns2 = 2048 >> s.n2;
    return s;
}

// Row units are grouped (16 jobs of one prime) once a segment has at least
// this many outer items; below it a unit holds adjacent rows of one job.
constexpr int GROUP_MIN_OUTER = 12;

// Unit counts of a segment (column and row passes) from its geometry.
void unit_counts(SegHdr &H)
{
    const Split sp = split_of(H.logN);
    const int njobs = H.outer * H.nl;
    int nc = std::min(sp.ns1, 1 << sp.n2);
    if (col_paired(H.xj, sp.n1, sp.ns1, nc)) nc /= 2;  // ColGeo's paired units
    const int nj = sp.ns1 / nc, blk = (1 << sp.n2) / nc;
    H.u_cols = ((njobs + nj - 1) / nj) * blk;
    H.u_rows = H.grouped ? H.nl * ((H.outer + ROW_J - 1) / ROW_J) * ((1 << sp.n1) / (sp.ns2 / ROW_J))
                         : njobs * ((1 << sp.n1) / sp.ns2);
}

// Fills the header of a segment (jobs = outer * nl) with its unit counts
// (turned into first units by finish()).
void seg_header(SegHdr &H, const fhe_ctx *c, bool fwd, int outer, int nl)
{
    memset(&H, 0, sizeof(H));
    const Split sp = split_of(c->logN);
    H.logN = c->logN;
    H.outer = outer;
    H.nl = nl;
    H.mq = c->d_mq;
    H.tw = fwd ? c->d_fwd : c->d_inv;
    H.ninv = c->d_ninv;
    H.grouped = outer >= GROUP_MIN_OUTER || (1 << sp.n1) < sp.ns2;
    unit_counts(H);
}

// Grid of a pass: one CTA per unit (variant 0) or a fixed number of resident
// CTAs per SM that walk the units (variants 1..3: 6, 4 and 2 per SM).
int grid_of(const fhe_ctx *c, int units)
{
    static const int per_sm[FHE_NTT_VARIANTS] = {0, 6, 4, 2};
    const int v = c->ntt_variant;
    if (v <= 0 || v >= FHE_NTT_VARIANTS || c->sms <= 0) return units;
    return std::min(units, per_sm[v] * c->sms);
}

// Unit counts per segment (seg_header) -> first unit of each segment.
template <class IO>
void finish(IO &io)
{
    int uc = 0, ur = 0;
    for (int s = 0; s < io.nseg; s++) {
        const int nc = io.h[s].u_cols, nr = io.h[s].u_rows;
        io.h[s].u_cols = uc;
        io.h[s].u_rows = ur;
        uc += nc;
        ur += nr;
    }
    io.ucols = uc;
    io.urows = ur;
}

// The unit counts of a subset's segments, recomputed from their geometry
// (for a launch split by ring degree after finish()).
template <class IO>
void recount(IO &io)
{
    for (int s = 0; s < io.nseg; s++) unit_counts(io.h[s]);
}

template <class IO, int LO, int HI>
void launch_passes(fhe_ctx *c, const IO &io, bool fwd)
{
    if (fwd) {
        launch_pdl(k_fwd_cols<IO, LO, HI>, grid_of(c, io.ucols), T, c->stream, io);
        launch_pdl(k_fwd_rows<IO, LO, HI>, grid_of(c, io.urows), T, c->stream, io);
    } else {
        launch_pdl(k_inv_rows<IO, LO, HI>, grid_of(c, io.urows), T, c->stream, io);
        launch_pdl(k_inv_cols<IO, LO, HI>, grid_of(c, io.ucols), T, c->stream, io);
    }
    c->launches += 2;
}

// Segments of one degree take that degree's kernels; a mix within
// 2^13..2^15 takes the mixed kernels; any other mix is split by degree.
template <class IO>
void launch_segments(fhe_ctx *c, IO &io, bool fwd)
{
    int lo = 99, hi = 0;
    for (int s = 0; s < io.nseg; s++) lo = std::min(lo, io.h[s].logN), hi = std::max(hi, io.h[s].logN);
    finish(io);
    if (io.ucols == 0) return;
    if (lo == hi) {
        switch (lo) {
        case 10: launch_passes<IO, 10, 10>(c, io, fwd); break;
        case 11: launch_passes<IO, 11, 11>(c, io, fwd); break;
        case 12: launch_passes<IO, 12, 12>(c, io, fwd); break;
        case 13: launch_passes<IO, 13, 13>(c, io, fwd); break;
        case 14: launch_passes<IO, 14, 14>(c, io, fwd); break;
        case 15: launch_passes<IO, 15, 15>(c, io, fwd); break;
        default: break;
        }
    } else if (FHE_NTT_MIXED_KERNEL && lo >= 13 && hi <= 15) {
        launch_passes<IO, 13, 15>(c, io, fwd);
    } else {
        for (int n = lo; n <= hi; n++) {
            IO sub;
            memset(&sub, 0, sizeof(sub));
            for (int s = 0; s < io.nseg; s++)
                if (io.h[s].logN == n) {
                    sub.h[sub.nseg] = io.h[s];
                    sub.s[sub.nseg] = io.s[s];
                    sub.nseg++;
                }
            if (sub.nseg) {
                recount(sub);
                launch_segments(c, sub, fwd);
            }
        }
    }
}

// Launches both passes of the segments in io on the stream of `c` (the
// first segment's context).  bytes / bfly: algorithmic traffic and butterflies
// of the whole launch, for the per-class timing.
template <class IO>
void run(fhe_ctx *c, IO &io, bool fwd, int cls, double bytes, double bfly)
{
    if (io.nseg == 0) return;
    prof_begin(c, cls, bytes, bfly);
    launch_segments(c, io, fwd);
    prof_end(c);
}

double bfly_of(const fhe_ctx *c, double njobs) { return njobs * (c->N / 2) * c->logN; }

void map_seg(MapSeg &S, const u64 *in, u64 *out, const LimbMap &m, const ulonglong2 *scale)
{
    memset(&S, 0, sizeof(S));
    S.in = in;
    S.out = out;
    S.in_outer = m.in_outer;
    S.out_outer = m.out_outer;
    S.scale = scale;
    for (int i = 0; i < m.nl; i++) {
        S.in_limb[i] = (uint8_t)m.in_limb[i];
        S.out_limb[i] = (uint8_t)m.out_limb[i];
        S.prime[i] = (uint8_t)m.prime[i];
    }
}

// Runs `fill(io, item)` over items in launches of at most FHE_SEGS segments.
template <class IO, class Item, class Fill>
void run_many(const std::vector<Item> &items, bool fwd, int cls, Fill fill)
{
    size_t i = 0;
    while (i < items.size()) {
        IO io;
        memset(&io, 0, sizeof(io));
        fhe_ctx *c0 = items[i].c;
        double bytes = 0, bfly = 0;
        for (; i < items.size() && io.nseg < FHE_SEGS; i++) {
            double b = 0, f = 0;
            if (fill(io, io.nseg, items[i], &b, &f)) {
                if (IO::XJ != 1) {
                    io.h[io.nseg].xj = IO::XJ;
                    unit_counts(io.h[io.nseg]);
                }
                io.nseg++;
            }
            bytes += b;
            bfly += f;
        }
        run(c0, io, fwd, cls, bytes, bfly);
    }
}

}  // namespace
