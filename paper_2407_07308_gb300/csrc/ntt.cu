// ntt.cu -- negacyclic NTT / inverse NTT over batches of RNS limbs, and the
// key-switching / modulus-switching steps fused into them.
//
// Transform (BoostCom Sec. 2.2: radix-2 NTT, Cooley-Tukey forward and
// Gentleman-Sande inverse, for power-of-two N):
//   forward  A[k] = a(psi^(2 brv(k) + 1)), natural-order input, bit-reversed
//            output; stage s (s = 0..logN-1) pairs j, j + N/2^(s+1) with the
//            twiddle psi^brv(2^s + (j >> (logN - s)));
//   inverse  the stages undone in reverse order with psi^-brv(.), then N^-1.
//
// GB300 mapping: N = 2^n is split as 2^n1 x 2^n2 (n1 = ceil(n/2)).  The
// forward transform is two kernels: "columns" runs global stages 0..n1-1,
// which only combine residues j = e 2^n2 + lo of one column lo, and "rows"
// runs stages n1..n-1 inside contiguous rows of 2^n2 residues.  Each is a
// sub-transform of size 2^M (M = n1 or n2) whose twiddles are entries of the
// full table: at local stage u, element e of a sub-transform with block index
// hi uses psi^brv(2^(S+u) + hi 2^u + (e >> (M-u))), S its first global stage.
// A CTA holds 16 sub-transforms in shared memory ([16][2^M], padded), every
// thread 16 residues in registers; a sub-transform runs as one radix-16 round
// (4 stages, strided residues) and one round of the remaining M-4 stages
// (contiguous blocks), with shared-memory exchanges in between.  Global
// memory is always read and written in coalesced runs of 16 residues or more
// (128 B).  The inverse runs the same kernels in reverse order (rows first),
// undoing stages n-1..0.  ~17 KB of shared memory and 128 threads per CTA
// (n = 14) leave room for many CTAs per SM; N up to 2^16 needs no cluster.
// Butterflies are Harvey's lazy ones (values in [0,4q) forward, [0,2q)
// inverse) with Shoup twiddles.
//
// Load/store functors let one kernel body serve the plain transform and the
// fused variants: ModUp (basis conversion of a key-switching digit computed
// while loading, then NTT), ModDown and modulus switching (correction
// computed while loading, subtract-and-scale applied while storing).  The
// half-transformed limb between the two kernels lives in the job's output
// limb.
#include <cooperative_groups.h>

#include "fhe_internal.h"

namespace cg = cooperative_groups;

namespace {

// Forward butterfly without normalisation: t = [Y w] in [0, 2q) for any
// 64-bit Y, so if X, Y < B then X + t and X - t + 2q lie in [0, B + 2q).
// After s stages every value is below (2s + 1) q <= 31 q < 2^63 (primes
// below 2^58, s <= 15); one reduction at the end brings it to [0, q).
__device__ __forceinline__ void ct_bfly(u64 &X, u64 &Y, const ulonglong2 w, u64 q, u64 q2)
{
    const u64 t = shoup_lazy(Y, w.x, w.y, q);
    const u64 x = X;
    X = x + t;
    Y = x - t + q2;
}

__device__ __forceinline__ void gs_bfly(u64 &X, u64 &Y, const ulonglong2 w, u64 q, u64 q2)
{
    u64 s = X + Y;
    s = s >= q2 ? s - q2 : s;
    u64 d = X - Y + q2;
    Y = shoup_lazy(d, w.x, w.y, q);
    X = s;
}

// Stages s0 .. s0+R-1 of the forward transform on one group x[0..2^R) whose
// block index is hi.
template <int R, class TW>
__device__ __forceinline__ void fwd_round(u64 (&x)[1 << R], int s0, int hi, TW W, u64 q, u64 q2)
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
__device__ __forceinline__ void inv_stage(u64 (&x)[1 << R], int s0, int hi, TW W, u64 q, u64 q2)
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
__device__ __forceinline__ void inv_round(u64 (&x)[1 << R], int s0, int hi, TW W, u64 q, u64 q2)
{
    inv_stage<R, R - 1>(x, s0, hi, W, q, q2);
}

// ---------------------------------------------------------------------------
// 16 sub-transforms of size 2^M in shared memory
// ---------------------------------------------------------------------------

// Register cap of every NTT kernel: enough for 768 resident threads per SM
// (85 registers a thread), measured faster than both the uncapped kernels
// and a 64-register cap.
#ifndef FHE_NTT_THREADS_PER_SM
#define FHE_NTT_THREADS_PER_SM 768
#endif
#define FHE_MINB(T) (FHE_NTT_THREADS_PER_SM / (T) > 0 ? FHE_NTT_THREADS_PER_SM / (T) : 1)
// The 8-elements-per-thread kernels exist to put more warps on each SM, so
// they are capped for 1024 resident threads (64 registers a thread).
#ifndef FHE_NTT8_THREADS_PER_SM
#define FHE_NTT8_THREADS_PER_SM 1024
#endif
#define FHE_MINB_V(T, V) ((V) == 8 ? (FHE_NTT8_THREADS_PER_SM / (T) > 0 ? FHE_NTT8_THREADS_PER_SM / (T) : 1) : FHE_MINB(T))

// Shared-memory twiddle tables: entry k at k + k / 8 (one 16-byte pad per 8
// entries), so that the second round's strided twiddle reads (stride up to 8
// entries across threads) hit distinct banks.
__host__ __device__ constexpr int twp(int k) { return k + (k >> 3); }
__host__ __device__ constexpr int twp_size(int n) { return n + n / 8 + 1; }

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

// smem layout: sub-transform c at c*P(M), element e at e + (e >> 4); P is odd
// mod 16 in u64 units, so the strided, blocked and row-wise access patterns
// below all spread over the banks.
template <int M>
struct Sub {
    static constexpr int SZ = 1 << M;                 // elements per sub-transform
    static constexpr int G = SZ / 16;                 // threads per sub-transform
    static constexpr int T = 16 * G;                  // threads per CTA
    static constexpr int R2 = M - 4;                  // stages of the second round
    static constexpr int P = SZ + SZ / 16 + 1;        // padded stride
    static constexpr int WORDS = 16 * P;              // shared memory words
    static_assert(M >= 5 && M <= 8, "sub-transform size");
    __device__ static int at(int c, int e) { return c * P + e + (e >> 4); }
};

// Round 1: thread t = (g, c) with c = t % 16, g = t / 16 holds elements
// e = k G + g (k < 16) of sub-transform c: local stages 0..3.
// Round 2: thread t = (c, g') with c = t / G, g' = t % G holds the 16/G
// blocks b = g' (16/G) + i of G contiguous elements: local stages 4..M-1.
// hi of sub-transform c is hi0 + c * hstep.
template <int M, bool FWD, class TW>
__device__ __forceinline__ void sub16(u64 *sm, int tid, TW W, int S, int hi0, int hstep, u64 q, u64 q2)
{
    using C = Sub<M>;
    constexpr int G = C::G, R2 = C::R2, NB = 16 / G;
    // Addresses as a per-thread base plus compile-time offsets: for e = kG + g
    // (g < G <= 16, kG a multiple of G) e >> 4 = (kG) >> 4, and for
    // e = 16 g' + iG + f (iG + f < 16) e >> 4 = g'.
    auto round1 = [&]() {
        const int c = tid & 15, g = tid >> 4;
        const int hi = hi0 + c * hstep;
        u64 *b1 = sm + c * C::P + g;
        u64 x[16];
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = b1[k * G + ((k * G) >> 4)];
        if (FWD)
            fwd_round<4>(x, S, hi, W, q, q2);
        else
            inv_round<4>(x, S, hi, W, q, q2);
#pragma unroll
        for (int k = 0; k < 16; k++) b1[k * G + ((k * G) >> 4)] = x[k];
    };
    auto round2 = [&]() {
        const int c = tid / G, gp = tid % G;
        const int hi = hi0 + c * hstep;
        u64 *b2 = sm + c * C::P + gp * 17;
#pragma unroll
        for (int i = 0; i < NB; i++) {
            u64 x[1 << R2];
#pragma unroll
            for (int f = 0; f < (1 << R2); f++) x[f] = b2[i * G + f];
            if (FWD)
                fwd_round<R2>(x, S + 4, hi * 16 + gp * NB + i, W, q, q2);
            else
                inv_round<R2>(x, S + 4, hi * 16 + gp * NB + i, W, q, q2);
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

// The same 16 sub-transforms with 8 elements per thread (twice the threads,
// for launches too small to fill the SMs): round A holds e = k G + g (k < 8,
// G = 2^M / 8) for local stages 0..2; round B holds, of block b (G
// contiguous elements, 8 per sub-transform), the elements b G + h + j PT
// (j < 8, PT = G / 8 threads per block, h < PT) for local stages 3..5 in
// registers and the remaining M - 6 stages across the PT lanes of a block
// (lanes h and h ^ delta, one 64-bit shuffle per element).  Same butterflies,
// same order per element: the results are identical to sub16's.
template <int M>
struct Sub8 {
    static constexpr int SZ = 1 << M;       // elements per sub-transform
    static constexpr int G = SZ / 8;        // threads per sub-transform
    static constexpr int T = 16 * G;        // threads per CTA
    static constexpr int R2 = M - 3;        // stages of round B
    static constexpr int PT = G / 8;        // lanes per block in round B
    static constexpr int P = Sub<M>::P;     // padded stride (same layout as Sub)
    static constexpr int WORDS = Sub<M>::WORDS;
    static_assert(M >= 6 && M <= 8, "8-element sub-transforms need 64 <= 2^M <= 256");
    __device__ static int at(int c, int e) { return Sub<M>::at(c, e); }
};

template <int M, int V>
struct SubSel {
    using type = Sub<M>;
};
template <int M>
struct SubSel<M, 8> {
    using type = Sub8<M>;
};

// Block-local stage R >= 3 of round B across lanes h and h ^ delta.
template <int M, bool FWD, int R, class TW>
__device__ __forceinline__ void sub8_cross(u64 (&x)[8], int h, int hb, TW W, int S, u64 q, u64 q2)
{
    constexpr int PT = Sub8<M>::PT, DELTA = PT >> (R - 2);
    const bool lower = (h & DELTA) == 0;
    const int tg0 = (h << (R - 3)) / PT;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const ulonglong2 w = W.get(S + 3 + R, (hb << R) + j * (1 << (R - 3)) + tg0);
        const u64 other = __shfl_xor_sync(0xffffffffu, x[j], DELTA);
        const u64 a = lower ? x[j] : other, b = lower ? other : x[j];
        if (FWD) {
            const u64 t = shoup_lazy(b, w.x, w.y, q);
            x[j] = lower ? a + t : a - t + q2;
        } else {
            u64 s2 = a + b;
            s2 = s2 >= q2 ? s2 - q2 : s2;
            x[j] = lower ? s2 : shoup_lazy(a - b + q2, w.x, w.y, q);
        }
    }
}

template <int M, bool FWD, class TW>
__device__ __forceinline__ void sub8(u64 *sm, int tid, TW W, int S, int hi0, int hstep, u64 q, u64 q2)
{
    using C = Sub8<M>;
    constexpr int G = C::G, R2 = C::R2, PT = C::PT;
    auto roundA = [&]() {
        const int c = tid & 15, g = tid >> 4;
        const int hi = hi0 + c * hstep;
        u64 x[8];
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = sm[C::at(c, k * G + g)];
        if (FWD)
            fwd_round<3>(x, S, hi, W, q, q2);
        else
            inv_round<3>(x, S, hi, W, q, q2);
#pragma unroll
        for (int k = 0; k < 8; k++) sm[C::at(c, k * G + g)] = x[k];
    };
    auto roundB = [&]() {
        const int c = tid / G, gp = tid % G, b = gp / PT, h = gp % PT;
        const int hb = (hi0 + c * hstep) * 8 + b;
        u64 x[8];
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = sm[C::at(c, b * G + h + j * PT)];
        if (FWD) {
            fwd_round<3>(x, S + 3, hb, W, q, q2);
            if constexpr (R2 > 3) sub8_cross<M, true, 3>(x, h, hb, W, S, q, q2);
            if constexpr (R2 > 4) sub8_cross<M, true, 4>(x, h, hb, W, S, q, q2);
        } else {
            if constexpr (R2 > 4) sub8_cross<M, false, 4>(x, h, hb, W, S, q, q2);
            if constexpr (R2 > 3) sub8_cross<M, false, 3>(x, h, hb, W, S, q, q2);
            inv_round<3>(x, S + 3, hb, W, q, q2);
        }
#pragma unroll
        for (int j = 0; j < 8; j++) sm[C::at(c, b * G + h + j * PT)] = x[j];
    };
    if (FWD) {
        roundA();
        __syncthreads();
        roundB();
    } else {
        roundB();
        __syncthreads();
        roundA();
    }
}

template <int M, int V, bool FWD, class TW>
__device__ __forceinline__ void subtx(u64 *sm, int tid, TW W, int S, int hi0, int hstep, u64 q, u64 q2)
{
    if constexpr (V == 16)
        sub16<M, FWD>(sm, tid, W, S, hi0, hstep, q, q2);
    else
        sub8<M, FWD>(sm, tid, W, S, hi0, hstep, q, q2);
}

// Moves a CTA's 16 x 2^M words into shared memory: word r (r = tid + k T)
// is read by src(r) and written by dst(r, v).  Staged in chunks of CH: the
// chunk's reads are all issued before its first write (the compiler does not
// reorder a global read past a shared-memory write on its own), so they
// overlap; CH = 0 keeps read/write pairs (better for loads that already hold
// several reads each, like ModUp's basis conversion).
template <class C, int CH = 16, class Src, class Dst>
__device__ __forceinline__ void tile_in(int tid, Src src, Dst dst)
{
    constexpr int IT = 16 * C::SZ / C::T;
    if constexpr (CH > 0) {
        constexpr int K = CH < IT ? CH : IT;
#pragma unroll
        for (int k0 = 0; k0 < IT; k0 += K) {
            u64 v[K];
#pragma unroll
            for (int k = 0; k < K; k++) v[k] = src(tid + (k0 + k) * C::T);
#pragma unroll
            for (int k = 0; k < K; k++) dst(tid + (k0 + k) * C::T, v[k]);
        }
    } else {
        for (int r = tid; r < 16 * C::SZ; r += C::T) dst(r, src(r));
    }
}

// Stores a CTA's 16 x 2^M results of a forward row pass: word r goes to
// index idx(r) of state st(r) with value val(r).  Staged: the operands the
// store reads (IO::NPRE per word) are loaded for a chunk of words before
// any of the chunk's writes, so those loads overlap (otherwise every write
// to global memory would order the next word's reads behind it).
template <class C, class IO, class StF, class Idx, class Val>
__device__ __forceinline__ void tile_out(const IO &io, int tid, StF st, Idx idx, Val val)
{
    constexpr int IT = 16 * C::SZ / C::T;
    if constexpr (IO::NPRE > 0) {
        constexpr int CH = IO::NPRE == 1 ? IT : IT / 2;
#pragma unroll
        for (int k0 = 0; k0 < IT; k0 += CH) {
            u64 a[CH][IO::NPRE];
#pragma unroll
            for (int k = 0; k < CH; k++) {
                const int r = tid + (k0 + k) * C::T;
#pragma unroll
                for (int w = 0; w < IO::NPRE; w++) a[k][w] = io.pre(st(r), idx(r), w);
            }
#pragma unroll
            for (int k = 0; k < CH; k++) {
                const int r = tid + (k0 + k) * C::T;
                io.store_pre(st(r), idx(r), val(r), a[k]);
            }
        }
    } else {
        for (int r = tid; r < 16 * C::SZ; r += C::T) io.store(st(r), idx(r), val(r));
    }
}

// Grouped row kernels: all 16 sub-transforms of the CTA are row hi of 16
// limbs with one prime, so the CTA needs only the 2^N2 - 1 twiddles of that
// row: stage N1+u, in-stage index hi 2^u + t, at offset 2^u - 1 + t.
struct RowTw {
    const ulonglong2 *sm;
    int N1, hi;
    __device__ ulonglong2 get(int s, int j) const
    {
        const int u = s - N1;
        return sm[twp((1 << u) - 1 + j - (hi << u))];
    }
};

// ---------------------------------------------------------------------------
// kernels.  Grid: one CTA per (job, block of 16 columns / rows).
// ---------------------------------------------------------------------------

// Forward, columns: global stages 0..N1-1 on columns lo0..lo0+15.
template <int N1, int N2, class IO, int V = 16>
__global__ void __launch_bounds__(SubSel<N1, V>::type::T, FHE_MINB_V((SubSel<N1, V>::type::T), V))
    k_fwd_cols(const __grid_constant__ IO io, const ModQ *__restrict__ mq, const ulonglong2 *__restrict__ tw)
{
    using C = typename SubSel<N1, V>::type;
    constexpr int NN = 1 << (N1 + N2), BLK = (1 << N2) / 16;
    __shared__ u64 sm[C::WORDS];
    __shared__ ulonglong2 W[twp_size(1 << N1)];  // stages 0..N1-1 use only the table's prefix
    const int job = blockIdx.x / BLK, lo0 = (blockIdx.x % BLK) * 16, tid = threadIdx.x;
    const typename IO::St st = io.begin(job, NN);
    const u64 q = mq[st.prime].q, q2 = 2 * q;
    // at most one twiddle per thread (T >= 2^N1), loaded before the tile and
    // stored after it, so that its latency overlaps the tile's loads
    static_assert(C::T >= (1 << N1), "one twiddle per thread");
    const bool has_w = tid < (1 << N1);
    const ulonglong2 wv = has_w ? __ldg(tw + (size_t)st.prime * NN + tid) : make_ulonglong2(0, 0);
    tile_in<C, IO::LDCH>(
        tid, [&](int r) { return io.load(st, ((r >> 4) << N2) + lo0 + (r & 15)); },
        [&](int r, u64 v) { sm[C::at(r & 15, r >> 4)] = v; });
    if (has_w) W[twp(tid)] = wv;
    __syncthreads();
    subtx<N1, V, true>(sm, tid, PrefixTw{W}, 0, 0, 0, q, q2);
    __syncthreads();
    u64 *mid = io.inter(st);
    for (int r = tid; r < 16 * C::SZ; r += C::T) {
        const int c = r & 15, e = r >> 4;
        mid[(e << N2) + lo0 + c] = sm[C::at(c, e)];
    }
}

// Forward, rows: global stages N1..N1+N2-1 on rows hi0..hi0+15.
template <int N1, int N2, class IO, int V = 16>
__global__ void __launch_bounds__(SubSel<N2, V>::type::T, FHE_MINB_V((SubSel<N2, V>::type::T), V))
    k_fwd_rows(const __grid_constant__ IO io, const ModQ *__restrict__ mq, const ulonglong2 *__restrict__ tw)
{
    using C = typename SubSel<N2, V>::type;
    constexpr int NN = 1 << (N1 + N2), BLK = (1 << N1) / 16;
    __shared__ u64 sm[C::WORDS];
    const int job = blockIdx.x / BLK, hi0 = (blockIdx.x % BLK) * 16, tid = threadIdx.x;
    const typename IO::St st = io.begin(job, NN);
    const u64 q = mq[st.prime].q, q2 = 2 * q;
    const GTw W{tw + (size_t)st.prime * NN};
    const u64 *mid = io.inter(st) + ((size_t)hi0 << N2);
    tile_in<C>(tid, [&](int r) { return mid[r]; }, [&](int r, u64 v) { sm[C::at(r >> N2, r & (C::SZ - 1))] = v; });
    __syncthreads();
    subtx<N2, V, true>(sm, tid, W, N1, hi0, 1, q, q2);
    __syncthreads();
    const ModQ mqp = mq[st.prime];
    tile_out<C>(
        io, tid, [&](int) -> const typename IO::St & { return st; }, [&](int r) { return (hi0 << N2) + r; },
        [&](int r) { return reduce64(sm[C::at(r >> N2, r & (C::SZ - 1))], mqp); });
}

// Inverse, rows first: undoes global stages N1+N2-1..N1.
template <int N1, int N2, class IO, int V = 16>
__global__ void __launch_bounds__(SubSel<N2, V>::type::T, FHE_MINB_V((SubSel<N2, V>::type::T), V))
    k_inv_rows(const __grid_constant__ IO io, const ModQ *__restrict__ mq, const ulonglong2 *__restrict__ tw)
{
    using C = typename SubSel<N2, V>::type;
    constexpr int NN = 1 << (N1 + N2), BLK = (1 << N1) / 16;
    __shared__ u64 sm[C::WORDS];
    const int job = blockIdx.x / BLK, hi0 = (blockIdx.x % BLK) * 16, tid = threadIdx.x;
    const typename IO::St st = io.begin(job, NN);
    const u64 q = mq[st.prime].q, q2 = 2 * q;
    const GTw W{tw + (size_t)st.prime * NN};
    tile_in<C>(
        tid, [&](int r) { return io.load(st, (hi0 << N2) + r); },
        [&](int r, u64 v) { sm[C::at(r >> N2, r & (C::SZ - 1))] = v; });
    __syncthreads();
    subtx<N2, V, false>(sm, tid, W, N1, hi0, 1, q, q2);
    __syncthreads();
    u64 *mid = io.inter(st) + ((size_t)hi0 << N2);
    for (int r = tid; r < 16 * C::SZ; r += C::T) mid[r] = sm[C::at(r >> N2, r & (C::SZ - 1))];
}

// Grouped rows.  Jobs j and j + stride share a prime; the launch holds
// `groups` x 16 such jobs per residue class of j mod stride.  CTA
// (group g, row hi): sub-transform c is row hi of job base + (16 kb + c) stride
// with base = g % stride, kb = g / stride.
template <int N1, int N2, class IO, int V = 16>
__global__ void __launch_bounds__(SubSel<N2, V>::type::T, FHE_MINB_V((SubSel<N2, V>::type::T), V))
    k_fwd_rows_grp(const __grid_constant__ IO io, const ModQ *__restrict__ mq, const ulonglong2 *__restrict__ tw, int stride)
{
    using C = typename SubSel<N2, V>::type;
    constexpr int NN = 1 << (N1 + N2), ROWS = 1 << N1;
    __shared__ u64 sm[C::WORDS];
    __shared__ ulonglong2 tws[twp_size((1 << N2) - 1)];
    __shared__ typename IO::St sts[16];
    const int tid = threadIdx.x, hi = blockIdx.x % ROWS, g = blockIdx.x / ROWS;
    const int base = g % stride, kb = g / stride;
    if (tid < 16) sts[tid] = io.begin(base + (16 * kb + tid) * stride, NN);
    __syncthreads();
    const int prime = sts[0].prime;
    const ModQ mqp = mq[prime];
    const u64 q = mqp.q, q2 = 2 * q;
    const ulonglong2 *W = tw + (size_t)prime * NN;
    // at most one twiddle per thread (T = 2^N2), loaded before the tile and
    // stored after it, so that its latency overlaps the tile's loads
    static_assert(C::T >= (1 << N2) - 1, "one twiddle per thread");
    const bool has_w = tid < (1 << N2) - 1;
    ulonglong2 wv = make_ulonglong2(0, 0);
    if (has_w) {
        const int u = 31 - __clz(tid + 1);  // stage of entry tid
        wv = __ldg(W + (1 << (N1 + u)) + (hi << u) + (tid + 1 - (1 << u)));
    }
    tile_in<C>(
        tid, [&](int r) { return io.inter(sts[r >> N2])[(hi << N2) + (r & (C::SZ - 1))]; },
        [&](int r, u64 v) { sm[C::at(r >> N2, r & (C::SZ - 1))] = v; });
    if (has_w) tws[twp(tid)] = wv;
    __syncthreads();
    subtx<N2, V, true>(sm, tid, RowTw{tws, N1, hi}, N1, hi, 0, q, q2);
    __syncthreads();
    tile_out<C>(
        io, tid, [&](int r) -> const typename IO::St & { return sts[r >> N2]; },
        [&](int r) { return (hi << N2) + (r & (C::SZ - 1)); },
        [&](int r) { return reduce64(sm[C::at(r >> N2, r & (C::SZ - 1))], mqp); });
}

template <int N1, int N2, class IO, int V = 16>
__global__ void __launch_bounds__(SubSel<N2, V>::type::T, FHE_MINB_V((SubSel<N2, V>::type::T), V))
    k_inv_rows_grp(const __grid_constant__ IO io, const ModQ *__restrict__ mq, const ulonglong2 *__restrict__ tw, int stride)
{
    using C = typename SubSel<N2, V>::type;
    constexpr int NN = 1 << (N1 + N2), ROWS = 1 << N1;
    __shared__ u64 sm[C::WORDS];
    __shared__ ulonglong2 tws[twp_size((1 << N2) - 1)];
    __shared__ typename IO::St sts[16];
    const int tid = threadIdx.x, hi = blockIdx.x % ROWS, g = blockIdx.x / ROWS;
    const int base = g % stride, kb = g / stride;
    if (tid < 16) sts[tid] = io.begin(base + (16 * kb + tid) * stride, NN);
    __syncthreads();
    const int prime = sts[0].prime;
    const u64 q = mq[prime].q, q2 = 2 * q;
    const ulonglong2 *W = tw + (size_t)prime * NN;
    static_assert(C::T >= (1 << N2) - 1, "one twiddle per thread");
    const bool has_w = tid < (1 << N2) - 1;
    ulonglong2 wv = make_ulonglong2(0, 0);
    if (has_w) {  // stored after the tile (latency overlap)
        const int u = 31 - __clz(tid + 1);
        wv = __ldg(W + (1 << (N1 + u)) + (hi << u) + (tid + 1 - (1 << u)));
    }
    tile_in<C>(
        tid, [&](int r) { return io.load(sts[r >> N2], (hi << N2) + (r & (C::SZ - 1))); },
        [&](int r, u64 v) { sm[C::at(r >> N2, r & (C::SZ - 1))] = v; });
    if (has_w) tws[twp(tid)] = wv;
    __syncthreads();
    subtx<N2, V, false>(sm, tid, RowTw{tws, N1, hi}, N1, hi, 0, q, q2);
    __syncthreads();
    for (int r = tid; r < 16 * C::SZ; r += C::T) {
        const int c = r >> N2, f = r & (C::SZ - 1);
        io.inter(sts[c])[(hi << N2) + f] = sm[C::at(c, f)];
    }
}

// Inverse, columns: undoes global stages N1-1..0, then scales by N^-1.
template <int N1, int N2, class IO, int V = 16>
__global__ void __launch_bounds__(SubSel<N1, V>::type::T, FHE_MINB_V((SubSel<N1, V>::type::T), V))
    k_inv_cols(const __grid_constant__ IO io, const ModQ *__restrict__ mq, const ulonglong2 *__restrict__ tw,
               const ulonglong2 *__restrict__ ninv)
{
    using C = typename SubSel<N1, V>::type;
    constexpr int NN = 1 << (N1 + N2), BLK = (1 << N2) / 16;
    __shared__ u64 sm[C::WORDS];
    __shared__ ulonglong2 W[twp_size(1 << N1)];
    const int job = blockIdx.x / BLK, lo0 = (blockIdx.x % BLK) * 16, tid = threadIdx.x;
    const typename IO::St st = io.begin(job, NN);
    const u64 q = mq[st.prime].q, q2 = 2 * q;
    static_assert(C::T >= (1 << N1), "one twiddle per thread");
    const bool has_w = tid < (1 << N1);  // stored after the tile (latency overlap)
    const ulonglong2 wv = has_w ? __ldg(tw + (size_t)st.prime * NN + tid) : make_ulonglong2(0, 0);
    const ulonglong2 ni = io.final_scale(st, ninv);
    const u64 *mid = io.inter(st);
    tile_in<C>(
        tid, [&](int r) { return mid[((r >> 4) << N2) + lo0 + (r & 15)]; },
        [&](int r, u64 v) { sm[C::at(r & 15, r >> 4)] = v; });
    if (has_w) W[twp(tid)] = wv;
    __syncthreads();
    subtx<N1, V, false>(sm, tid, PrefixTw{W}, 0, 0, 0, q, q2);
    __syncthreads();
    for (int r = tid; r < 16 * C::SZ; r += C::T) {
        const int c = r & 15, e = r >> 4;
        io.store(st, (e << N2) + lo0 + c, reduce2q(shoup_lazy(sm[C::at(c, e)], ni.x, ni.y, q), q));
    }
}

// ---------------------------------------------------------------------------
// load/store functors
// ---------------------------------------------------------------------------

struct IOPlain {
    const u64 *in;
    u64 *out;
    LimbMap m;
    struct St {
        const u64 *in;
        u64 *out;
        int prime;
    };
    __device__ St begin(int job, int N) const
    {
        const int o = job / m.nl, l = job % m.nl;
        St s;
        s.in = in + o * m.in_outer + (long long)m.in_limb[l] * N;
        s.out = out + o * m.out_outer + (long long)m.out_limb[l] * N;
        s.prime = m.prime[l];
        return s;
    }
    __device__ u64 load(const St &s, int i) const { return s.in[i]; }
    __device__ void store(const St &s, int i, u64 v) const { s.out[i] = v; }
    static constexpr int NPRE = 0;  // operands the store reads
    static constexpr int LDCH = 16;  // loads staged per chunk (0: not staged)
    __device__ u64 pre(const St &, int, int) const { return 0; }
    __device__ void store_pre(const St &s, int i, u64 v, const u64 *) const { s.out[i] = v; }
    __device__ u64 *inter(const St &s) const { return s.out; }
    __device__ ulonglong2 final_scale(const St &s, const ulonglong2 *ninv) const { return ninv[s.prime]; }
    int prime_stride() const { return m.nl; }  // jobs j and j + nl use one prime
};

// Inverse transform whose output limb l is also multiplied by a constant:
// the final scaling uses N^-1 c_l (and its Shoup word) from scale[l].
struct IOScaled {
    const u64 *in;
    u64 *out;
    LimbMap m;
    ulonglong2 scale[FHE_MAXP];
    struct St {
        const u64 *in;
        u64 *out;
        int prime, limb;
    };
    __device__ St begin(int job, int N) const
    {
        const int o = job / m.nl, l = job % m.nl;
        St s;
        s.in = in + o * m.in_outer + (long long)m.in_limb[l] * N;
        s.out = out + o * m.out_outer + (long long)m.out_limb[l] * N;
        s.prime = m.prime[l];
        s.limb = l;
        return s;
    }
    __device__ u64 load(const St &s, int i) const { return s.in[i]; }
    __device__ void store(const St &s, int i, u64 v) const { s.out[i] = v; }
    __device__ u64 *inter(const St &s) const { return s.out; }
    __device__ ulonglong2 final_scale(const St &s, const ulonglong2 *) const { return scale[s.limb]; }
    int prime_stride() const { return m.nl; }
};

// IOScaled whose last map entry (limb l-1 of the relinearisation
// accumulators) loads y = acc + (P mod q) addend: the first step of the
// relinearisation fused with the modulus switch.  Job = (ct, poly) * nl + entry.
struct IOScaledY : IOScaled {
    const u64 *abase;
    long long a_outer, a_poly;
    int amask, alimb;
    u64 Pm, Pm_s, qm;
    struct St : IOScaled::St {
        const u64 *add;
    };
    __device__ St begin(int job, int N) const
    {
        St s;
        static_cast<IOScaled::St &>(s) = IOScaled::begin(job, N);
        const int o = job / m.nl, e = job % m.nl, pi = o & 1;
        const long long c = o >> 1;
        s.add = (e == m.nl - 1 && ((amask >> pi) & 1)) ? abase + c * a_outer + pi * a_poly + (long long)alimb * N
                                                      : nullptr;
        return s;
    }
    __device__ u64 load(const St &s, int i) const
    {
        return s.add ? addmod(s.in[i], shoup(s.add[i], Pm, Pm_s, qm), qm) : s.in[i];
    }
};

// ModUp: extended limb t of digit j of ct c:  y = sum_a t_a (Q_j/q_a) mod r,
// where the source limbs already hold t_a = [x_a (Q_j/q_a)^-1]_{q_a} (the
// inverse NTT that produced them applied that factor).
struct IOModUp {
    const u64 *d2c;  // [count][l][N] coefficient domain
    u64 *ext;        // [count][dnum][l+K][N]
    const ModUpParams *P;
    const ModQ *mq;
    int l, K, dnum, njobs;
    struct St {
        const u64 *src;
        u64 *dst;
        int nsrc, prime;
        ModQ mt;
        u64 hat[FHE_MAXK];
    };
    __device__ St begin(int job, int N) const
    {
        const int c = job / njobs, e = job % njobs;
        const int j = P->job_digit[e], t = P->job_tgt[e];
        St s;
        const int lo = P->digit_lo[j];
        s.nsrc = P->digit_n[j];
        s.src = d2c + ((long long)c * l + lo) * N;
        s.dst = ext + (((long long)c * dnum + j) * (l + K) + t) * N;
        s.prime = P->job_prime[e];
        s.mt = mq[s.prime];
#pragma unroll
        for (int a = 0; a < FHE_MAXK; a++)
            if (a < s.nsrc) s.hat[a] = P->hat[j][a][t];
        return s;
    }
    __device__ u64 load(const St &s, int n) const
    {
        u128 acc = 0;
#pragma unroll
        for (int a = 0; a < FHE_MAXK; a++)
            if (a < s.nsrc) acc += (u128)s.src[(long long)a * stride + n] * s.hat[a];
        return barrett128(acc, s.mt);
    }
    __device__ void store(const St &s, int k, u64 v) const { s.dst[k] = v; }
    static constexpr int NPRE = 0;
    static constexpr int LDCH = 0;  // each load already sums several limbs
    __device__ u64 pre(const St &, int, int) const { return 0; }
    __device__ void store_pre(const St &s, int k, u64 v, const u64 *) const { s.dst[k] = v; }
    __device__ u64 *inter(const St &s) const { return s.dst; }
    int prime_stride() const { return njobs; }  // one entry per (digit, target) and ct
    int stride;  // N
};

// ModDown of poly pi of ct c, data limb i:
//   delta_i = sum_k t_k * (p P/p_k mod q_i),  out_i = (acc_i - delta_i) P^-1 + addend_i,
// where the special limbs already hold t_k = [acc_{P,k} p^-1 (P/p_k)^-1]_{p_k}
// (applied by the inverse NTT that produced them).
struct IOModDown {
    const u64 *accP;  // [count][2][K][N] coefficient domain
    const u64 *acc;   // [count][2][l+K][N] NTT domain
    const u64 *abase;
    long long a_outer, a_poly;
    int amask;
    u64 *out;         // [count][2][l][N]
    const ModDownParams *P;
    const ModQ *mq;
    int l, K, stride;
    struct St {
        const u64 *w, *acc, *add;
        u64 *out;
        int prime;
        ModQ mi;
        u64 pinv, pinv_s;
        u64 phat[FHE_MAXK];
    };
    __device__ St begin(int job, int N) const
    {
        const int c = job / (2 * l), pi = (job / l) % 2, i = job % l;
        St s;
        s.w = accP + ((long long)c * 2 + pi) * K * N;
        s.acc = acc + (((long long)c * 2 + pi) * (l + K) + i) * N;
        s.add = ((amask >> pi) & 1) ? abase + c * a_outer + pi * a_poly + (long long)i * N : nullptr;
        s.out = out + (((long long)c * 2 + pi) * l + i) * N;
        s.prime = i;
        s.mi = mq[i];
        s.pinv = P->pinv[i];
        s.pinv_s = P->pinv_s[i];
#pragma unroll
        for (int k = 0; k < FHE_MAXK; k++)
            if (k < K) s.phat[k] = P->phat[k][i];
        return s;
    }
    __device__ u64 load(const St &s, int n) const
    {
        u128 a = 0;
#pragma unroll
        for (int k = 0; k < FHE_MAXK; k++)
            if (k < K) a += (u128)s.w[(long long)k * stride + n] * s.phat[k];
        return barrett128(a, s.mi);
    }
    __device__ void store(const St &s, int k, u64 v) const
    {
        const u64 q = s.mi.q;
        u64 r = shoup(submod(s.acc[k], v, q), s.pinv, s.pinv_s, q);
        if (s.add) r = addmod(r, s.add[k], q);
        s.out[k] = r;
    }
    static constexpr int NPRE = 2;  // accumulator, addend
    static constexpr int LDCH = 16;
    __device__ u64 pre(const St &s, int k, int w) const { return w == 0 ? s.acc[k] : (s.add ? s.add[k] : 0); }
    __device__ void store_pre(const St &s, int k, u64 v, const u64 *pv) const
    {
        const u64 q = s.mi.q;
        u64 r = shoup(submod(pv[0], v, q), s.pinv, s.pinv_s, q);
        if (s.add) r = addmod(r, pv[1], q);
        s.out[k] = r;
    }
    __device__ u64 *inter(const St &s) const { return s.out; }
    int prime_stride() const { return l; }  // job = (ct, poly) * l + limb
};

// Modulus switch l -> l-1 of poly pi of ct c, limb i < l-1:
//   delta_i = p w mod q_i,  out_i = (x_i - delta_i) q_{l-1}^-1,
// where `last` already holds w = [x_{l-1} p^-1]_{q_{l-1}} in the coefficient
// domain (applied by the inverse NTT that produced it).
struct IOModSwitch {
    const u64 *last;  // [count][npoly][N] coefficient domain
    const u64 *in;    // [count][npoly][l][N]
    u64 *out;         // [count][npoly][l-1][N]
    const ModSwitchParams *P;
    const ModQ *mq;
    int l, npoly;
    struct St {
        const u64 *last, *in;
        u64 *out;
        int prime;
        u64 q, ql, pl, pls, pi, pis, qi, qis;
    };
    __device__ St begin(int job, int N) const
    {
        const int c = job / (npoly * (l - 1)), pi = (job / (l - 1)) % npoly, i = job % (l - 1);
        St s;
        s.last = last + ((long long)c * npoly + pi) * N;
        s.in = in + (((long long)c * npoly + pi) * l + i) * N;
        s.out = out + (((long long)c * npoly + pi) * (l - 1) + i) * N;
        s.prime = i;
        s.q = mq[i].q;
        s.ql = mq[l - 1].q;
        s.pl = P->pinv_last;
        s.pls = P->pinv_last_s;
        s.pi = P->p_i[i];
        s.pis = P->p_i_s[i];
        s.qi = P->qinv[i];
        s.qis = P->qinv_s[i];
        return s;
    }
    __device__ u64 load(const St &s, int n) const { return shoup(s.last[n], s.pi, s.pis, s.q); }
    __device__ void store(const St &s, int k, u64 v) const
    {
        s.out[k] = shoup(submod(s.in[k], v, s.q), s.qi, s.qis, s.q);
    }
    static constexpr int NPRE = 1;  // the limb being switched
    static constexpr int LDCH = 16;
    __device__ u64 pre(const St &s, int k, int) const { return s.in[k]; }
    __device__ void store_pre(const St &s, int k, u64 v, const u64 *pv) const
    {
        s.out[k] = shoup(submod(pv[0], v, s.q), s.qi, s.qis, s.q);
    }
    __device__ u64 *inter(const St &s) const { return s.out; }
    int prime_stride() const { return l - 1; }  // job = (ct, poly) * (l-1) + limb
};

// Relinearisation fused with the modulus switch that follows it (l -> l-1)
// for poly pi of ct c, kept limb i < l-1:
//   correction_i = sum_{k<K} t_k h[k][i] + w h[K][i] (coefficient domain),
//   out_i = (acc_i P^-1 + add_i - NTT(correction)_i) q_{l-1}^-1,
// where src holds t_0..t_{K-1} (the special limbs, already scaled) and w.
struct IORelinMS {
    const u64 *src;  // [count][2][K+1][N] coefficient domain
    const u64 *acc;  // [count][2][l+K][N] NTT domain
    const u64 *abase;
    long long a_outer, a_poly;
    int amask;
    u64 *out;        // [count][2][l-1][N]
    const RelinMSParams *P;
    const ModQ *mq;
    int l, K, stride;
    struct St {
        const u64 *w, *acc, *add;
        u64 *out;
        int prime;
        ModQ mi;
        u64 pinv, pinv_s, qminv, qminv_s;
        u64 h[FHE_MAXK];
    };
    __device__ St begin(int job, int N) const
    {
        const int m = l - 1;
        const int c = job / (2 * m), pi = (job / m) % 2, i = job % m;
        St s;
        s.w = src + ((long long)c * 2 + pi) * (K + 1) * N;
        s.acc = acc + (((long long)c * 2 + pi) * (l + K) + i) * N;
        s.add = ((amask >> pi) & 1) ? abase + c * a_outer + pi * a_poly + (long long)i * N : nullptr;
        s.out = out + (((long long)c * 2 + pi) * m + i) * N;
        s.prime = i;
        s.mi = mq[i];
        s.pinv = P->pinv[i];
        s.pinv_s = P->pinv_s[i];
        s.qminv = P->qminv[i];
        s.qminv_s = P->qminv_s[i];
#pragma unroll
        for (int k = 0; k < FHE_MAXK; k++)
            if (k <= K) s.h[k] = P->h[k][i];
        return s;
    }
    // K + 1 <= FHE_MAXK products of canonical residues: below 2^(2b+3)
    __device__ u64 load(const St &s, int n) const
    {
        u128 a = 0;
#pragma unroll
        for (int k = 0; k < FHE_MAXK; k++)
            if (k <= K) a += (u128)s.w[(long long)k * stride + n] * s.h[k];
        return barrett128(a, s.mi);
    }
    __device__ u64 combine(const St &s, u64 accv, u64 addv, u64 v) const
    {
        const u64 q = s.mi.q;
        u64 t = shoup(accv, s.pinv, s.pinv_s, q);
        if (s.add) t = addmod(t, addv, q);
        return shoup(submod(t, v, q), s.qminv, s.qminv_s, q);
    }
    __device__ void store(const St &s, int k, u64 v) const
    {
        s.out[k] = combine(s, s.acc[k], s.add ? s.add[k] : 0, v);
    }
    static constexpr int NPRE = 2;  // accumulator, addend
    static constexpr int LDCH = 0;  // each load sums K + 1 limbs
    __device__ u64 pre(const St &s, int k, int w) const { return w == 0 ? s.acc[k] : (s.add ? s.add[k] : 0); }
    __device__ void store_pre(const St &s, int k, u64 v, const u64 *pv) const
    {
        s.out[k] = combine(s, pv[0], pv[1], v);
    }
    __device__ u64 *inter(const St &s) const { return s.out; }
    int prime_stride() const { return l - 1; }  // job = (ct, poly) * (l-1) + limb
};

// k modulus switches at once (l -> l-k), poly pi of ct c, kept limb i < l-k:
//   correction_i = sum_{t<k} w_t G[t][i],  out_i = (x_i - NTT(correction)_i) D_k^-1.
struct IOMultiSwitch {
    const u64 *src;  // [count][npoly][k][N] coefficient domain: w_0 .. w_{k-1}
    const u64 *in;   // [count][npoly][l][N]
    u64 *out;        // [count][npoly][l-k][N]
    const MultiSwitchParams *P;
    const ModQ *mq;
    int l, k, npoly, stride;
    struct St {
        const u64 *w, *in;
        u64 *out;
        int prime;
        ModQ mi;
        u64 dinv, dinv_s;
        u64 g[FHE_MAXK];
    };
    __device__ St begin(int job, int N) const
    {
        const int kept = l - k;
        const int c = job / (npoly * kept), pi = (job / kept) % npoly, i = job % kept;
        St s;
        s.w = src + ((long long)c * npoly + pi) * k * N;
        s.in = in + (((long long)c * npoly + pi) * l + i) * N;
        s.out = out + (((long long)c * npoly + pi) * kept + i) * N;
        s.prime = i;
        s.mi = mq[i];
        s.dinv = P->Dinv[i];
        s.dinv_s = P->Dinv_s[i];
#pragma unroll
        for (int t = 0; t < FHE_MAXK; t++)
            if (t < k) s.g[t] = P->G[t][i];
        return s;
    }
    __device__ u64 load(const St &s, int n) const
    {
        u128 a = 0;
#pragma unroll
        for (int t = 0; t < FHE_MAXK; t++)
            if (t < k) a += (u128)s.w[(long long)t * stride + n] * s.g[t];
        return barrett128(a, s.mi);
    }
    __device__ void store(const St &s, int j, u64 v) const
    {
        s.out[j] = shoup(submod(s.in[j], v, s.mi.q), s.dinv, s.dinv_s, s.mi.q);
    }
    static constexpr int NPRE = 1;
    static constexpr int LDCH = 0;
    __device__ u64 pre(const St &s, int j, int) const { return s.in[j]; }
    __device__ void store_pre(const St &s, int j, u64 v, const u64 *pv) const
    {
        s.out[j] = shoup(submod(pv[0], v, s.mi.q), s.dinv, s.dinv_s, s.mi.q);
    }
    __device__ u64 *inter(const St &s) const { return s.out; }
    int prime_stride() const { return l - k; }
};

// ---------------------------------------------------------------------------
// one-launch NTT for square splits N = 2^M x 2^M (M = 5, 6, 7)
// ---------------------------------------------------------------------------
//
// A cluster of CL = 2^M / 16 CTAs holds one limb.  Forward: CTA k transforms
// columns 16k .. 16k+15 (global stages 0..M-1), writes each element (row e,
// column 16k + c) into the shared memory of CTA e / 16 (distributed shared
// memory), and after one cluster barrier transforms rows 16k .. 16k+15
// (stages M..2M-1).  Inverse: rows first, then columns.  The half-transformed
// limb never leaves the cluster, and the transform is one launch.  Every CTA
// runs the same two barriers (no early exit), and no CTA touches another's
// shared memory after the second one.

__device__ __forceinline__ void cluster_arrive_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory"); }

template <int M, class IO>
__global__ void __cluster_dims__((1 << M) / 16, 1, 1) __launch_bounds__(Sub<M>::T, FHE_MINB(Sub<M>::T))
    k_fwd_fused(const __grid_constant__ IO io, const ModQ *__restrict__ mq, const ulonglong2 *__restrict__ tw)
{
    using C = Sub<M>;
    constexpr int CL = (1 << M) / 16, NN = 1 << (2 * M);
    __shared__ u64 sm[C::WORDS];   // columns 16k .. 16k+15, all rows
    __shared__ u64 sm2[C::WORDS];  // rows 16k .. 16k+15, all columns (written by the cluster)
    __shared__ ulonglong2 W[twp_size(1 << M)];
    cg::cluster_group cluster = cg::this_cluster();
    cluster_arrive_relaxed();  // matched by cluster_wait before the first remote write
    const int k = (int)cluster.block_rank();
    const int job = blockIdx.x / CL, lo0 = 16 * k, hi0 = 16 * k, tid = threadIdx.x;
    const typename IO::St st = io.begin(job, NN);
    const u64 q = mq[st.prime].q, q2 = 2 * q;
    for (int r = tid; r < (1 << M); r += C::T) W[twp(r)] = tw[(size_t)st.prime * NN + r];
    tile_in<C, IO::LDCH>(
        tid, [&](int r) { return io.load(st, ((r >> 4) << M) + lo0 + (r & 15)); },
        [&](int r, u64 v) { sm[C::at(r & 15, r >> 4)] = v; });
    __syncthreads();
    sub16<M, true>(sm, tid, PrefixTw{W}, 0, 0, 0, q, q2);
    __syncthreads();
    cluster_wait();
    for (int r = tid; r < 16 * C::SZ; r += C::T) {
        const int c = r & 15, e = r >> 4;
        u64 *dst = cluster.map_shared_rank(sm2, e >> 4);
        dst[C::at(e & 15, lo0 + c)] = sm[C::at(c, e)];
    }
    cluster.sync();
    sub16<M, true>(sm2, tid, GTw{tw + (size_t)st.prime * NN}, M, hi0, 1, q, q2);
    __syncthreads();
    const ModQ mqp = mq[st.prime];
    tile_out<C>(
        io, tid, [&](int) -> const typename IO::St & { return st; }, [&](int r) { return (hi0 << M) + r; },
        [&](int r) { return reduce64(sm2[C::at(r >> M, r & (C::SZ - 1))], mqp); });
}

template <int M, class IO>
__global__ void __cluster_dims__((1 << M) / 16, 1, 1) __launch_bounds__(Sub<M>::T, FHE_MINB(Sub<M>::T))
    k_inv_fused(const __grid_constant__ IO io, const ModQ *__restrict__ mq, const ulonglong2 *__restrict__ tw,
                const ulonglong2 *__restrict__ ninv)
{
    using C = Sub<M>;
    constexpr int CL = (1 << M) / 16, NN = 1 << (2 * M);
    __shared__ u64 sm[C::WORDS];   // rows 16k .. 16k+15
    __shared__ u64 sm2[C::WORDS];  // columns 16k .. 16k+15 (written by the cluster)
    __shared__ ulonglong2 W[twp_size(1 << M)];
    cg::cluster_group cluster = cg::this_cluster();
    cluster_arrive_relaxed();
    const int k = (int)cluster.block_rank();
    const int job = blockIdx.x / CL, lo0 = 16 * k, hi0 = 16 * k, tid = threadIdx.x;
    const typename IO::St st = io.begin(job, NN);
    const u64 q = mq[st.prime].q, q2 = 2 * q;
    for (int r = tid; r < (1 << M); r += C::T) W[twp(r)] = tw[(size_t)st.prime * NN + r];
    const ulonglong2 ni = io.final_scale(st, ninv);
    tile_in<C>(
        tid, [&](int r) { return io.load(st, (hi0 << M) + r); },
        [&](int r, u64 v) { sm[C::at(r >> M, r & (C::SZ - 1))] = v; });
    __syncthreads();
    sub16<M, false>(sm, tid, GTw{tw + (size_t)st.prime * NN}, M, hi0, 1, q, q2);
    __syncthreads();
    cluster_wait();
    // element (row hi0 + rl, column f) goes to CTA f / 16 as its column f % 16
    for (int r = tid; r < 16 * C::SZ; r += C::T) {
        const int rl = r & 15, f = r >> 4;
        u64 *dst = cluster.map_shared_rank(sm2, f >> 4);
        dst[C::at(f & 15, hi0 + rl)] = sm[C::at(rl, f)];
    }
    cluster.sync();
    sub16<M, false>(sm2, tid, PrefixTw{W}, 0, 0, 0, q, q2);
    __syncthreads();
    for (int r = tid; r < 16 * C::SZ; r += C::T) {
        const int c = r & 15, e = r >> 4;
        io.store(st, (e << M) + lo0 + c, reduce2q(shoup_lazy(sm2[C::at(c, e)], ni.x, ni.y, q), q));
    }
}

template <int M, class IO>
void fwd_fused(fhe_ctx *c, const IO &io, int njobs)
{
    k_fwd_fused<M, IO><<<njobs * ((1 << M) / 16), Sub<M>::T, 0, c->stream>>>(io, c->d_mq, c->d_fwd);
}

template <int M, class IO>
void inv_fused(fhe_ctx *c, const IO &io, int njobs)
{
    k_inv_fused<M, IO><<<njobs * ((1 << M) / 16), Sub<M>::T, 0, c->stream>>>(io, c->d_mq, c->d_inv, c->d_ninv);
}

// Row kernels take the grouped form when every prime of the launch has a
// multiple of 16 jobs (the batched case); otherwise 16 rows of one limb.
template <class IO>
bool groupable(const IO &io, int njobs)
{
    const int st = io.prime_stride();
    return st > 0 && njobs % st == 0 && (njobs / st) % 16 == 0;
}

template <int N1, int N2, class IO, int V = 16>
void fwd_pair(fhe_ctx *c, const IO &io, int njobs)
{
    constexpr int T1 = SubSel<N1, V>::type::T, T2 = SubSel<N2, V>::type::T;
    k_fwd_cols<N1, N2, IO, V><<<njobs * ((1 << N2) / 16), T1, 0, c->stream>>>(io, c->d_mq, c->d_fwd);
    if (groupable(io, njobs))
        k_fwd_rows_grp<N1, N2, IO, V><<<(njobs / 16) * (1 << N1), T2, 0, c->stream>>>(io, c->d_mq, c->d_fwd,
                                                                                      io.prime_stride());
    else
        k_fwd_rows<N1, N2, IO, V><<<njobs * ((1 << N1) / 16), T2, 0, c->stream>>>(io, c->d_mq, c->d_fwd);
}

template <int N1, int N2, class IO, int V = 16>
void inv_pair(fhe_ctx *c, const IO &io, int njobs)
{
    constexpr int T1 = SubSel<N1, V>::type::T, T2 = SubSel<N2, V>::type::T;
    if (groupable(io, njobs))
        k_inv_rows_grp<N1, N2, IO, V><<<(njobs / 16) * (1 << N1), T2, 0, c->stream>>>(io, c->d_mq, c->d_inv,
                                                                                      io.prime_stride());
    else
        k_inv_rows<N1, N2, IO, V><<<njobs * ((1 << N1) / 16), T2, 0, c->stream>>>(io, c->d_mq, c->d_inv);
    k_inv_cols<N1, N2, IO, V><<<njobs * ((1 << N2) / 16), T1, 0, c->stream>>>(io, c->d_mq, c->d_inv, c->d_ninv);
}

// Factorisations N = 2^n1 x 2^n2 per ring degree (the autotuner picks one
// per context; all compute the same transform): variant 0 and 1 are the two
// two-kernel splits, variant 2 the one-launch cluster form of a square split,
// variant 3 variant 0's split with 8 elements per thread (twice the warps).
// Returns the number of kernels launched.
template <class IO>
int fwd_dispatch(fhe_ctx *c, const IO &io, int njobs)
{
    const int v = c->ntt_variant;
    switch (c->logN) {
    case 10: if (v == 2) return fwd_fused<5>(c, io, njobs), 1;
        fwd_pair<5, 5>(c, io, njobs); return 2;
    case 11: v ? fwd_pair<5, 6>(c, io, njobs) : fwd_pair<6, 5>(c, io, njobs); return 2;
    case 12: if (v == 2) return fwd_fused<6>(c, io, njobs), 1;
        if (v == 3) return fwd_pair<6, 6, IO, 8>(c, io, njobs), 2;
        v ? fwd_pair<7, 5>(c, io, njobs) : fwd_pair<6, 6>(c, io, njobs); return 2;
    case 13: if (v == 3) return fwd_pair<7, 6, IO, 8>(c, io, njobs), 2;
        v ? fwd_pair<6, 7>(c, io, njobs) : fwd_pair<7, 6>(c, io, njobs); return 2;
    case 14: if (v == 2) return fwd_fused<7>(c, io, njobs), 1;
        if (v == 3) return fwd_pair<7, 7, IO, 8>(c, io, njobs), 2;
        v ? fwd_pair<8, 6>(c, io, njobs) : fwd_pair<7, 7>(c, io, njobs); return 2;
    case 15: if (v == 3) return fwd_pair<8, 7, IO, 8>(c, io, njobs), 2;
        v ? fwd_pair<7, 8>(c, io, njobs) : fwd_pair<8, 7>(c, io, njobs); return 2;
    default: return 0;
    }
}

template <class IO>
int inv_dispatch(fhe_ctx *c, const IO &io, int njobs)
{
    const int v = c->ntt_variant;
    switch (c->logN) {
    case 10: if (v == 2) return inv_fused<5>(c, io, njobs), 1;
        inv_pair<5, 5>(c, io, njobs); return 2;
    case 11: v ? inv_pair<5, 6>(c, io, njobs) : inv_pair<6, 5>(c, io, njobs); return 2;
    case 12: if (v == 2) return inv_fused<6>(c, io, njobs), 1;
        if (v == 3) return inv_pair<6, 6, IO, 8>(c, io, njobs), 2;
        v ? inv_pair<7, 5>(c, io, njobs) : inv_pair<6, 6>(c, io, njobs); return 2;
    case 13: if (v == 3) return inv_pair<7, 6, IO, 8>(c, io, njobs), 2;
        v ? inv_pair<6, 7>(c, io, njobs) : inv_pair<7, 6>(c, io, njobs); return 2;
    case 14: if (v == 2) return inv_fused<7>(c, io, njobs), 1;
        if (v == 3) return inv_pair<7, 7, IO, 8>(c, io, njobs), 2;
        v ? inv_pair<8, 6>(c, io, njobs) : inv_pair<7, 7>(c, io, njobs); return 2;
    case 15: if (v == 3) return inv_pair<8, 7, IO, 8>(c, io, njobs), 2;
        v ? inv_pair<7, 8>(c, io, njobs) : inv_pair<8, 7>(c, io, njobs); return 2;
    default: return 0;
    }
}

// words_per_job: u64 words of global traffic per limb job (algorithmic: the
// transform reads and writes each limb once; fused variants add their operands)
template <class IO>
void run_fwd(fhe_ctx *c, const IO &io, int njobs, int cls, double words_per_job = 2.0)
{
    if (njobs <= 0) return;
    prof_begin(c, cls, 8.0 * words_per_job * c->N * njobs, (double)njobs * (c->N / 2) * c->logN);
    c->launches += fwd_dispatch(c, io, njobs);
    prof_end(c);
}

template <class IO>
void run_inv(fhe_ctx *c, const IO &io, int njobs, int cls, double words_per_job = 2.0)
{
    if (njobs <= 0) return;
    prof_begin(c, cls, 8.0 * words_per_job * c->N * njobs, (double)njobs * (c->N / 2) * c->logN);
    c->launches += inv_dispatch(c, io, njobs);
    prof_end(c);
}

}  // namespace

bool ntt_supported_logn(int logN) { return logN >= 10 && logN <= 15; }

void launch_ntt_fwd_plain(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, int njobs)
{
    IOPlain io{in, out, m};
    run_fwd(c, io, njobs, FHE_K_NTT_FWD);
}

void launch_ntt_inv_plain(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, int njobs)
{
    IOPlain io{in, out, m};
    run_inv(c, io, njobs, FHE_K_NTT_INV);
}

void launch_ntt_inv_scaled(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, const ulonglong2 *scale,
                           int njobs)
{
    IOScaled io;
    io.in = in;
    io.out = out;
    io.m = m;
    for (int i = 0; i < m.nl; i++) io.scale[i] = scale[i];
    run_inv(c, io, njobs, FHE_K_NTT_INV);
}

void launch_ntt_inv_scaled_y(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, const ulonglong2 *scale,
                             int njobs, const u64 *abase, long long a_outer, long long a_poly, int amask, int level)
{
    IOScaledY io;
    io.in = in;
    io.out = out;
    io.m = m;
    for (int i = 0; i < m.nl; i++) io.scale[i] = scale[i];
    io.abase = abase;
    io.a_outer = a_outer;
    io.a_poly = a_poly;
    io.amask = amask;
    io.alimb = level - 1;
    io.qm = c->q[level - 1];
    io.Pm = c->rms[level].Pm;
    io.Pm_s = c->rms[level].Pm_s;
    // the y entry (one of nl) also reads the addend limb
    run_inv(c, io, njobs, FHE_K_NTT_INV, 2.0 + 1.0 / m.nl);
}

void launch_ntt_modup(fhe_ctx *c, const u64 *d2c, u64 *ext, int level, int count)
{
    const ModUpParams &P = c->modup[level];
    IOModUp io;
    io.d2c = d2c;
    io.ext = ext;
    io.P = c->d_modup + level;
    io.mq = c->d_mq;
    io.l = level;
    io.K = c->K;
    io.dnum = P.dnum;
    io.njobs = P.njobs;
    io.stride = c->N;
    double words = 0;
    for (int e = 0; e < P.njobs; e++) words += P.digit_n[P.job_digit[e]] + 1.0;
    run_fwd(c, io, P.njobs * count, FHE_K_NTT_MODUP, words / P.njobs);
}

void launch_ntt_moddown(fhe_ctx *c, const u64 *accP, const u64 *acc, const u64 *abase, long long a_outer,
                        long long a_poly, int amask, u64 *out, int level, int count)
{
    IOModDown io;
    io.accP = accP;
    io.acc = acc;
    io.abase = abase;
    io.a_outer = a_outer;
    io.a_poly = a_poly;
    io.amask = amask;
    io.out = out;
    io.P = c->d_moddown + level;
    io.mq = c->d_mq;
    io.l = level;
    io.K = c->K;
    io.stride = c->N;
    // reads K special limbs, acc_i and (for masked polys) the addend; writes out_i
    const double add_frac = ((amask & 1) + ((amask >> 1) & 1)) / 2.0;
    run_fwd(c, io, 2 * level * count, FHE_K_NTT_MODDOWN, c->K + 2.0 + add_frac);
}

void launch_ntt_relin_ms(fhe_ctx *c, const u64 *src, const u64 *acc, const u64 *abase, long long a_outer,
                         long long a_poly, int amask, u64 *out, int level, int count)
{
    IORelinMS io;
    io.src = src;
    io.acc = acc;
    io.abase = abase;
    io.a_outer = a_outer;
    io.a_poly = a_poly;
    io.amask = amask;
    io.out = out;
    io.P = c->d_rms + level;
    io.mq = c->d_mq;
    io.l = level;
    io.K = c->K;
    io.stride = c->N;
    // reads K + 1 correction sources, acc_i and (for masked polys) the addend; writes out_i
    const double add_frac = ((amask & 1) + ((amask >> 1) & 1)) / 2.0;
    run_fwd(c, io, 2 * (level - 1) * count, FHE_K_NTT_MODDOWN, c->K + 3.0 + add_frac);
}

void launch_ntt_multiswitch(fhe_ctx *c, const u64 *src, const u64 *in, u64 *out, int level, int k, int npoly,
                            int count)
{
    IOMultiSwitch io;
    io.src = src;
    io.in = in;
    io.out = out;
    io.P = c->d_mss + (size_t)level * (FHE_MAXK + 1) + k;
    io.mq = c->d_mq;
    io.l = level;
    io.k = k;
    io.npoly = npoly;
    io.stride = c->N;
    // reads the k switch values and x_i, writes out_i
    run_fwd(c, io, npoly * (level - k) * count, FHE_K_NTT_MODSWITCH, k + 2.0);
}

void launch_ntt_modswitch(fhe_ctx *c, const u64 *last, const u64 *in, u64 *out, int level, int npoly, int count)
{
    IOModSwitch io;
    io.last = last;
    io.in = in;
    io.out = out;
    io.P = c->d_modswitch + level;
    io.mq = c->d_mq;
    io.l = level;
    io.npoly = npoly;
    run_fwd(c, io, npoly * (level - 1) * count, FHE_K_NTT_MODSWITCH, 3.0);
}

// ---------------------------------------------------------------------------
// autotuner: times both factorisations on a representative batch
// ---------------------------------------------------------------------------

bool ntt_variant_ok(int logN, int v)
{
    if (v == 0) return true;
    if (v == 1) return logN >= 11 && logN <= 15;
    if (v == 2) return logN == 10 || logN == 12 || logN == 14;
    if (v == 3) return logN >= 12 && logN <= 15;
    return false;
}

// Times forward + inverse of `outer` x nl limbs (nl = min(primes, 10)),
// `outer` rounded to a multiple of 16 when >= 16 so that the row kernels take
// their grouped form as in batched use; keeps the faster variant.
int ntt_autotune(fhe_ctx *c, int njobs, float *ms_out)
{
    LimbMap m;
    memset(&m, 0, sizeof(m));
    m.nl = std::min(c->np, 10);
    int outer = std::max(1, njobs / m.nl);
    if (outer >= 16) outer -= outer % 16;
    const int jobs = outer * m.nl;
    m.in_outer = m.out_outer = (long long)m.nl * c->N;
    for (int i = 0; i < m.nl; i++) m.in_limb[i] = m.out_limb[i] = i, m.prime[i] = i;
    u64 *buf = nullptr;
    const size_t words = (size_t)jobs * c->N;
    if (cudaMalloc(&buf, words * sizeof(u64)) != cudaSuccess) return FHE_ENOMEM;
    cudaMemsetAsync(buf, 0, words * sizeof(u64), c->stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool prof = c->prof_on;
    const long long launches = c->launches;
    c->prof_on = false;
    float best = 1e30f;
    int best_v = 0;
    for (int v = 0; v < FHE_NTT_VARIANTS; v++) {
        if (ms_out) ms_out[v] = 0;
        if (!ntt_variant_ok(c->logN, v)) continue;
        c->ntt_variant = v;
        IOPlain io{buf, buf, m};
        for (int w = 0; w < 2; w++) {
            fwd_dispatch(c, io, jobs);
            inv_dispatch(c, io, jobs);
        }
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 5; r++) {
            fwd_dispatch(c, io, jobs);
            inv_dispatch(c, io, jobs);
        }
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 5;
        if (ms_out) ms_out[v] = ms;
        // the first factorisation stays unless another is clearly faster
        // (3%), so that near-ties do not flip from one context to the next
        if (v == 0 || ms < 0.97f * best) best = ms, best_v = v;
    }
    c->ntt_variant = best_v;
    c->prof_on = prof;
    c->launches = launches;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return fhe_cuda_check(c, cudaGetLastError(), "autotune");
}
