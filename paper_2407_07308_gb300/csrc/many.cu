// many.cu -- the streaming kernels of a product or a switch over several
// batches in one launch: element-wise ciphertext arithmetic, the tensor
// product, the key-switching inner product and the switch folds.
//
// A launch carries a table of up to FHE_SEGS segments (one batch each, of any
// context, level and size on one device); segment s owns a contiguous range
// of blocks, so a block never straddles two segments and every warp still
// reads 256 contiguous bytes.  The arithmetic per element is the one of the
// single-batch kernels in kernels.cu; only the addressing differs.
#include <string.h>

#include "fhe_internal.h"

namespace {

constexpr int TPB = 256;
constexpr int EW_ELEMS = TPB * 4;  // elements per block of the element-wise kernels

// |k| < q: k mod q in [0, q)
__device__ __forceinline__ u64 small_mod(int64_t k, u64 q) { return k >= 0 ? (u64)k : q - (u64)(-k); }

template <class S>
__device__ __forceinline__ int block_seg(const S *s, int n)
{
    int sg = 0;
    while (sg + 1 < n && s[sg + 1].b0 <= (int)blockIdx.x) sg++;
    return sg;
}

// ---- element-wise: x0 + x1, x0 - x1, -x0, sum_t k_t x_t, k0 x0, x0 + k0 on
// poly 0 of 2-poly ciphertexts (poly 1 copied) ------------------------------

struct EwSeg {
    const u64 *x[8];
    u64 *out;
    const ModQ *mq;
    long long total;  // elements: outer * level * N
    int logN, level, n, op, b0, vec;  // vec: every pointer 16-byte aligned
    int small, pad;   // small: q sum |k_j| < 2^64 for every prime (see ew_scaled)
    int64_t k[8];     // centred scalars, |k| < p
};

// Scalar products with small centred scalars without 128-bit arithmetic:
// a k = (q - a) |k| mod q for k < 0, and with a < q every term (q - a or a)
// |k| is at most q |k|, so the terms sum to at most q sum |k_j|, which fits
// 64 bits when small is set; reduce64 then gives [0, q).
__device__ __forceinline__ u64 ew_scaled(u64 a, int64_t k, u64 q) { return (k < 0 ? q - a : a) * (u64)(k < 0 ? -k : k); }

struct EwTable {
    int nseg, pad;
    EwSeg s[FHE_SEGS];
};

// V adjacent elements (one limb: N is even) as one load per operand
template <int V>
struct Vec {
    u64 v[V];
};

template <int V>
__device__ __forceinline__ Vec<V> ld_vec(const u64 *p)
{
    Vec<V> r;
    if constexpr (V == 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(p);
        r.v[0] = t.x;
        r.v[1] = t.y;
    } else {
        r.v[0] = *p;
    }
    return r;
}

template <int V>
__device__ __forceinline__ void st_vec(u64 *p, const Vec<V> &r)
{
    if constexpr (V == 2)
        *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(r.v[0], r.v[1]);
    else
        *p = r.v[0];
}

// A block's EW_ELEMS elements lie in one limb (EW_ELEMS divides N, N >= 2^10),
// so the limb's prime and the polynomial index are per-block constants
// (measured with the tensor's per-block addressing and 16-byte loads, and the
// 64-bit scalar products: tensor 0.83 -> 0.67 ms, element-wise 1.40 -> 1.35 ms
// per step on the 16-pair comparison at N = 2^14).
template <int V>
__device__ __forceinline__ void ew_block(const EwSeg &S)
{
    const long long base = (long long)(blockIdx.x - S.b0) * EW_ELEMS;
    const long long li = base >> S.logN;
    const int i = (int)(li % S.level);
    const u64 q = S.mq[i].q;
#pragma unroll
    for (int e = threadIdx.x * V; e < EW_ELEMS; e += TPB * V) {
        const long long idx = base + e;
        if (idx >= S.total) break;
        Vec<V> r;
        switch (S.op) {
        case FHE_EW_ADD: {
            const Vec<V> a = ld_vec<V>(S.x[0] + idx), b = ld_vec<V>(S.x[1] + idx);
#pragma unroll
            for (int u = 0; u < V; u++) r.v[u] = addmod(a.v[u], b.v[u], q);
            break;
        }
        case FHE_EW_SUB: {
            const Vec<V> a = ld_vec<V>(S.x[0] + idx), b = ld_vec<V>(S.x[1] + idx);
#pragma unroll
            for (int u = 0; u < V; u++) r.v[u] = submod(a.v[u], b.v[u], q);
            break;
        }
        case FHE_EW_NEG: {
            const Vec<V> a = ld_vec<V>(S.x[0] + idx);
#pragma unroll
            for (int u = 0; u < V; u++) r.v[u] = negmod(a.v[u], q);
            break;
        }
        case FHE_EW_CMUL: {
            const Vec<V> a = ld_vec<V>(S.x[0] + idx);
            if (S.small) {
#pragma unroll
                for (int u = 0; u < V; u++) r.v[u] = reduce64(ew_scaled(a.v[u], S.k[0], q), S.mq[i]);
                break;
            }
            const u64 k = small_mod(S.k[0], q);
#pragma unroll
            for (int u = 0; u < V; u++) r.v[u] = barrett128((u128)a.v[u] * k, S.mq[i]);
            break;
        }
        case FHE_EW_CADD: {
            const int poly = (int)((li / S.level) % 2);
            const Vec<V> a = ld_vec<V>(S.x[0] + idx);
            const u64 k = small_mod(S.k[0], q);
#pragma unroll
            for (int u = 0; u < V; u++) r.v[u] = poly == 0 ? addmod(a.v[u], k, q) : a.v[u];
            break;
        }
        default: {  // FHE_EW_LINCOMB: at most eight products below the Barrett bound
            if (S.small) {
                u64 acc[V];
#pragma unroll
                for (int u = 0; u < V; u++) acc[u] = 0;
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (j < S.n) {
                        const Vec<V> a = ld_vec<V>(S.x[j] + idx);
#pragma unroll
                        for (int u = 0; u < V; u++) acc[u] += ew_scaled(a.v[u], S.k[j], q);
                    }
#pragma unroll
                for (int u = 0; u < V; u++) r.v[u] = reduce64(acc[u], S.mq[i]);
                break;
            }
            u128 acc[V];
#pragma unroll
            for (int u = 0; u < V; u++) acc[u] = 0;
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (j < S.n) {
                    const Vec<V> a = ld_vec<V>(S.x[j] + idx);
                    const u64 k = small_mod(S.k[j], q);
#pragma unroll
                    for (int u = 0; u < V; u++) acc[u] += (u128)a.v[u] * k;
                }
#pragma unroll
            for (int u = 0; u < V; u++) r.v[u] = barrett128(acc[u], S.mq[i]);
        }
        }
        st_vec<V>(S.out + idx, r);
    }
}

__global__ void k_ew_many(const __grid_constant__ EwTable t)
{
    pdl_begin();
    const EwSeg &S = t.s[block_seg(t.s, t.nseg)];
    if (S.vec)
        ew_block<2>(S);
    else
        ew_block<1>(S);
}

// ---- tensor: (a0,a1) x (b0,b1) -> (a0 b0, a0 b1 + a1 b0, a1 b1) -----------

struct TensorSeg {
    const u64 *a, *b;
    u64 *out;
    const ModQ *mq;
    long long total;  // count * level * N
    int logN, level, b0, vec;  // vec: every pointer 16-byte aligned
};

struct TensorTable {
    int nseg, pad;
    TensorSeg s[FHE_SEGS];
};

template <int V>
__device__ __forceinline__ void tensor_block(const TensorSeg &S)
{
    // one limb of one ciphertext per block (EW_ELEMS divides N)
    const long long LN = (long long)S.level << S.logN;
    const long long base = (long long)(blockIdx.x - S.b0) * EW_ELEMS;
    if (base >= S.total) return;
    const long long c = base / LN, r0 = base % LN;
    const ModQ m = S.mq[(int)(r0 >> S.logN)];
    const u64 *a0 = S.a + 2 * c * LN + r0, *a1 = a0 + LN;
    const u64 *b0 = S.b + 2 * c * LN + r0, *b1 = b0 + LN;
    u64 *o0 = S.out + 3 * c * LN + r0, *o1 = o0 + LN, *o2 = o1 + LN;
#pragma unroll
    for (int e = threadIdx.x * V; e < EW_ELEMS; e += TPB * V) {
        const Vec<V> x0 = ld_vec<V>(a0 + e), x1 = ld_vec<V>(a1 + e), y0 = ld_vec<V>(b0 + e), y1 = ld_vec<V>(b1 + e);
        Vec<V> r0v, r1v, r2v;
#pragma unroll
        for (int u = 0; u < V; u++) {
            r0v.v[u] = barrett128((u128)x0.v[u] * y0.v[u], m);
            r1v.v[u] = barrett128((u128)x0.v[u] * y1.v[u] + (u128)x1.v[u] * y0.v[u], m);
            r2v.v[u] = barrett128((u128)x1.v[u] * y1.v[u], m);
        }
        st_vec<V>(o0 + e, r0v);
        st_vec<V>(o1 + e, r1v);
        st_vec<V>(o2 + e, r2v);
    }
}

__global__ void k_tensor_many(const __grid_constant__ TensorTable t)
{
    pdl_begin();
    const TensorSeg &S = t.s[block_seg(t.s, t.nseg)];
    if (S.vec)
        tensor_block<2>(S);
    else
        tensor_block<1>(S);
}

// ---- key-switching inner product ------------------------------------------
// acc[c][pi][r] = sum_j y_j[r] ksk_j[pi][prime(r)], y_j[r] = x_c[r] for r in
// digit j, else the ModUp limb.  A block covers TPB coefficients of one
// extended limb r for CB ciphertexts; each thread loads its 2 dnum key words
// once for its CB ciphertexts.

#ifndef FHE_KS_CB
#define FHE_KS_CB 4
#endif
#ifndef FHE_KS_MINB
#define FHE_KS_MINB 3
#endif
constexpr int KS_CB = FHE_KS_CB;  // ciphertexts per thread (key words reused across them)

struct KsSeg {
    const u64 *ext, *xbase, *ksk;
    u64 *acc;
    const ModQ *mq;
    long long x_outer;
    int count, l, K, L, dnum, logN, b0, nbx;  // nbx: blocks along n
};

struct KsTable {
    int nseg, pad;
    KsSeg s[FHE_SEGS];
};

__global__ void __launch_bounds__(TPB, FHE_KS_MINB) k_ks_inner_many(const __grid_constant__ KsTable t)
{
    pdl_begin();
    const KsSeg &S = t.s[block_seg(t.s, t.nseg)];
    const int lb = blockIdx.x - S.b0;
    const int lK = S.l + S.K, N = 1 << S.logN;
    const int bx = lb % S.nbx, r = (lb / S.nbx) % lK, cz = lb / (S.nbx * lK);
    const int n = bx * TPB + threadIdx.x;
    if (n >= N) return;
    const int prime = r < S.l ? r : S.L + (r - S.l);
    const ModQ m = S.mq[prime];
    const int LK = S.L + S.K;
    const int rdig = r < S.l ? r / S.K : -1;
    const int c0 = cz * KS_CB;
    const int ncb = min(KS_CB, S.count - c0);
    u128 a0[KS_CB], a1[KS_CB];
#pragma unroll
    for (int cc = 0; cc < KS_CB; cc++) a0[cc] = a1[cc] = 0;
    // digit j's two key words and CB inputs; the next digit's are loaded
    // before this digit's products (two digits' loads in flight)
    auto load = [&](int j, u64 &k0, u64 &k1, u64 (&y)[KS_CB]) {
        k0 = S.ksk[(((long long)j * 2 + 0) * LK + prime) * N + n];
        k1 = S.ksk[(((long long)j * 2 + 1) * LK + prime) * N + n];
#pragma unroll
        for (int cc = 0; cc < KS_CB; cc++) {
            const int c = c0 + cc;
            y[cc] = cc >= ncb ? 0
                    : (j == rdig) ? S.xbase[c * S.x_outer + (long long)r * N + n]
                                  : S.ext[(((long long)c * S.dnum + j) * lK + r) * N + n];
        }
    };
    u64 k0, k1, y[KS_CB];
    load(0, k0, k1, y);
    for (int j = 0; j < S.dnum; j++) {
        u64 nk0 = 0, nk1 = 0, ny[KS_CB];
#pragma unroll
        for (int cc = 0; cc < KS_CB; cc++) ny[cc] = 0;
        if (j + 1 < S.dnum) load(j + 1, nk0, nk1, ny);
#pragma unroll
        for (int cc = 0; cc < KS_CB; cc++) {
            a0[cc] += (u128)y[cc] * k0;
            a1[cc] += (u128)y[cc] * k1;
        }
        k0 = nk0;
        k1 = nk1;
#pragma unroll
        for (int cc = 0; cc < KS_CB; cc++) y[cc] = ny[cc];
    }
#pragma unroll
    for (int cc = 0; cc < KS_CB; cc++) {
        const int c = c0 + cc;
        if (cc < ncb) {
            S.acc[(((long long)c * 2 + 0) * lK + r) * N + n] = barrett128(a0[cc], m);
            S.acc[(((long long)c * 2 + 1) * lK + r) * N + n] = barrett128(a1[cc], m);
        }
    }
}

// ---- folds of the fused relinearise + switch and of the multi-prime switch

struct FoldSeg {
    u64 *src;
    const ModQ *mq;
    const void *P;    // RelinMSParams (k = 0) or MultiSwitchParams
    long long total;  // outer * N
    int logN, l, k, K, b0, vec;  // vec: src 16-byte aligned
};

struct FoldTable {
    int nseg, rms;
    FoldSeg s[FHE_SEGS];
};

// The relinearise + switch fold with its block's polynomial and constants
// found once (a block's EW_ELEMS words lie in one polynomial: EW_ELEMS
// divides N) and two adjacent words per 16-byte access (measured: the
// element-wise class 1.356 -> 1.308 ms per step on the 16-pair comparison at
// N = 2^14).
__device__ __forceinline__ void fold_rms_block(const FoldSeg &S)
{
    const int N = 1 << S.logN;
    const long long base = (long long)(blockIdx.x - S.b0) * EW_ELEMS;
    if (base >= S.total) return;
    const long long o = base >> S.logN;
    const int n0 = (int)(base & (N - 1));
    const RelinMSParams *P = (const RelinMSParams *)S.P;
    const ModQ mm = S.mq[S.l - 1];
    u64 pk[FHE_MAXK];
#pragma unroll
    for (int k = 0; k < FHE_MAXK; k++) pk[k] = k < S.K ? P->pkinv[k] : 0;
    u64 *b = S.src + o * (S.K + 1) * N + n0;
#pragma unroll
    for (int e = threadIdx.x * 2; e < EW_ELEMS; e += TPB * 2) {
        u128 a0 = 0, a1 = 0;
#pragma unroll
        for (int k = 0; k < FHE_MAXK; k++)
            if (k < S.K) {
                const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(b + (long long)k * N + e);
                a0 += (u128)v.x * pk[k];
                a1 += (u128)v.y * pk[k];
            }
        u64 *y = b + (long long)S.K * N + e;
        const ulonglong2 yv = *reinterpret_cast<const ulonglong2 *>(y);
        *reinterpret_cast<ulonglong2 *>(y) =
            make_ulonglong2(submod(yv.x, barrett128(a0, mm), mm.q), submod(yv.y, barrett128(a1, mm), mm.q));
    }
}

// rms: src[c][pi] = (t_0 .. t_{K-1}, Y') -> Y' - sum_k t_k p_k^-1 mod q_{l-1}.
// multi-switch: src[o] = (X'_0 .. X'_{k-1}) -> w_j = X'_j - sum_{t<j} w_t F[j][t].
__global__ void k_fold_many(const __grid_constant__ FoldTable t)
{
    pdl_begin();
    const FoldSeg &S = t.s[block_seg(t.s, t.nseg)];
    if (t.rms && S.vec) {
        fold_rms_block(S);
        return;
    }
    const int N = 1 << S.logN;
    const long long base = (long long)(blockIdx.x - S.b0) * EW_ELEMS;
    for (int e = threadIdx.x; e < EW_ELEMS; e += TPB) {
        const long long idx = base + e;
        if (idx >= S.total) break;
        const long long o = idx >> S.logN;
        const int n = (int)(idx & (N - 1));
        if (t.rms) {
            const RelinMSParams *P = (const RelinMSParams *)S.P;
            const ModQ mm = S.mq[S.l - 1];
            u64 *b = S.src + o * (S.K + 1) * N + n;
            u128 a = 0;
            for (int k = 0; k < S.K; k++) a += (u128)b[(long long)k * N] * P->pkinv[k];
            b[(long long)S.K * N] = submod(b[(long long)S.K * N], barrett128(a, mm), mm.q);
        } else {
            const MultiSwitchParams *P = (const MultiSwitchParams *)S.P;
            u64 *b = S.src + o * S.k * N + n;
            u64 w[FHE_MAXK];
#pragma unroll
            for (int j = 0; j < FHE_MAXK; j++) {
                if (j < S.k) {
                    const ModQ mj = S.mq[S.l - 1 - j];
                    u128 a = 0;
#pragma unroll
                    for (int q = 0; q < FHE_MAXK; q++)
                        if (q < j) a += (u128)w[q] * P->F[j][q];
                    w[j] = submod(b[(long long)j * N], barrett128(a, mj), mj.q);
                    b[(long long)j * N] = w[j];
                }
            }
        }
    }
}

int ew_blocks(long long total) { return (int)((total + EW_ELEMS - 1) / EW_ELEMS); }

// Launches kern over `items` in tables of at most FHE_SEGS segments; fill
// sets segment s from an item and returns its blocks (0 = nothing to do) and
// its algorithmic bytes.
template <class Table, class Item, class Fill, class Launch>
void launch_tables(const std::vector<Item> &items, int cls, Fill fill, Launch launch)
{
    size_t i = 0;
    while (i < items.size()) {
        Table t;
        memset(&t, 0, sizeof(t));
        fhe_ctx *c = items[i].c;
        int blocks = 0;
        double bytes = 0;
        for (; i < items.size() && t.nseg < FHE_SEGS; i++) {
            double b = 0;
            const int nb = fill(t.s[t.nseg], items[i], &b);
            if (nb <= 0) continue;
            t.s[t.nseg].b0 = blocks;
            blocks += nb;
            bytes += b;
            t.nseg++;
        }
        if (!t.nseg) continue;
        prof_begin(c, cls, bytes);
        launch(t, blocks, c->stream);
        prof_end(c);
        c->launches++;
    }
}

}  // namespace

void launch_ew_many(const std::vector<EwArgs> &items)
{
    launch_tables<EwTable>(
        items, FHE_K_ELEMWISE,
        [](EwSeg &S, const EwArgs &a, double *bytes) {
            S.total = (long long)a.outer * a.level * a.c->N;
            if (S.total <= 0) return 0;
            for (int j = 0; j < 8; j++) S.x[j] = a.x[j], S.k[j] = a.k[j];
            S.out = a.out;
            S.mq = a.c->d_mq;
            S.logN = a.c->logN;
            S.level = a.level;
            S.n = a.n;
            S.op = a.op;
            bool vec = ((uintptr_t)a.out & 15) == 0;
            for (int j = 0; j < 8; j++) vec = vec && ((uintptr_t)a.x[j] & 15) == 0;
            S.vec = vec;
            // the 64-bit form applies when q_max * sum |k_j| < 2^64
            {
                u64 qmax = 0;
                for (u64 q : a.c->q) qmax = q > qmax ? q : qmax;
                const int nk = a.op == FHE_EW_LINCOMB ? a.n : 1;
                unsigned __int128 ksum = 0;
                for (int j = 0; j < nk && j < 8; j++) ksum += (u64)(a.k[j] < 0 ? -a.k[j] : a.k[j]);
                S.small = (a.op == FHE_EW_LINCOMB || a.op == FHE_EW_CMUL) && ksum * qmax < ((unsigned __int128)1 << 64);
            }
            const int reads = a.op == FHE_EW_LINCOMB ? a.n : (a.op == FHE_EW_ADD || a.op == FHE_EW_SUB) ? 2 : 1;
            *bytes = 8.0 * (reads + 1) * S.total;
            return ew_blocks(S.total);
        },
        [](const EwTable &t, int blocks, cudaStream_t s) { launch_pdl(k_ew_many, blocks, TPB, s, t); });
}

void launch_tensor_many(const std::vector<TensorArgs> &items)
{
    launch_tables<TensorTable>(
        items, FHE_K_TENSOR,
        [](TensorSeg &S, const TensorArgs &a, double *bytes) {
            S.total = (long long)a.count * a.level * a.c->N;
            if (S.total <= 0) return 0;
            S.a = a.a;
            S.b = a.b;
            S.out = a.out;
            S.mq = a.c->d_mq;
            S.logN = a.c->logN;
            S.level = a.level;
            S.vec = (((uintptr_t)a.a | (uintptr_t)a.b | (uintptr_t)a.out) & 15) == 0;
            *bytes = 8.0 * 7 * S.total;
            return ew_blocks(S.total);
        },
        [](const TensorTable &t, int blocks, cudaStream_t s) { launch_pdl(k_tensor_many, blocks, TPB, s, t); });
}

void launch_ks_inner_many(const std::vector<KsInnerArgs> &items)
{
    launch_tables<KsTable>(
        items, FHE_K_KS_INNER,
        [](KsSeg &S, const KsInnerArgs &a, double *bytes) {
            fhe_ctx *c = a.c;
            if (a.count <= 0) return 0;
            S.ext = a.ext;
            S.xbase = a.xbase;
            S.ksk = a.ksk;
            S.acc = a.acc;
            S.mq = c->d_mq;
            S.x_outer = a.x_outer;
            S.count = a.count;
            S.l = a.level;
            S.K = c->K;
            S.L = c->L;
            S.dnum = c->modup[a.level].dnum;
            S.logN = c->logN;
            S.nbx = (c->N + TPB - 1) / TPB;
            // per (r, n): 2 dnum key words once per CB ciphertexts, dnum inputs and 2 outputs per ciphertext
            *bytes = 8.0 * (double)(a.level + c->K) * c->N * (2.0 * S.dnum + a.count * (S.dnum + 2.0));
            return S.nbx * (a.level + c->K) * ((a.count + KS_CB - 1) / KS_CB);
        },
        [](const KsTable &t, int blocks, cudaStream_t s) { launch_pdl(k_ks_inner_many, blocks, TPB, s, t); });
}

void launch_rms_fold_many(const std::vector<FoldArgs> &items)
{
    launch_tables<FoldTable>(
        items, FHE_K_ELEMWISE,
        [](FoldSeg &S, const FoldArgs &a, double *bytes) {
            fhe_ctx *c = a.c;
            S.total = (long long)a.outer * 2 * c->N;  // (ct, poly) pairs
            if (S.total <= 0) return 0;
            S.src = a.src;
            S.mq = c->d_mq;
            S.P = c->d_rms + a.level;
            S.logN = c->logN;
            S.l = a.level;
            S.K = c->K;
            S.vec = ((uintptr_t)a.src & 15) == 0;
            *bytes = 8.0 * (c->K + 2.0) * S.total;
            return ew_blocks(S.total);
        },
        [](FoldTable &t, int blocks, cudaStream_t s) {
            t.rms = 1;
            launch_pdl(k_fold_many, blocks, TPB, s, t);
        });
}

void launch_ms_fold_many(const std::vector<FoldArgs> &items)
{
    launch_tables<FoldTable>(
        items, FHE_K_ELEMWISE,
        [](FoldSeg &S, const FoldArgs &a, double *bytes) {
            fhe_ctx *c = a.c;
            S.total = (long long)a.outer * c->N;
            if (S.total <= 0 || a.k < 2) return 0;
            S.src = a.src;
            S.mq = c->d_mq;
            S.P = c->d_mss + (size_t)a.level * (FHE_MAXK + 1) + a.k;
            S.logN = c->logN;
            S.l = a.level;
            S.k = a.k;
            *bytes = 8.0 * 2.0 * a.k * S.total;
            return ew_blocks(S.total);
        },
        [](FoldTable &t, int blocks, cudaStream_t s) {
            t.rms = 0;
            launch_pdl(k_fold_many, blocks, TPB, s, t);
        });
}
