// kernels.cu -- streaming (HBM-bound) kernels on NTT-domain limbs: add, sub,
// neg, scalar and constant terms, the ciphertext tensor product, the
// key-switching inner product, Galois automorphisms as index permutations, and
// small helpers for key generation, encryption and decryption.
//
// Layout: a batch of ciphertexts is u64 [count][npoly][level][N]; an "outer"
// index runs over count*npoly polys, and the limb of element idx is
// (idx >> logN) % level, so one flat grid covers the batch and every warp
// reads 256 contiguous bytes.
#include <string.h>

#include "fhe_internal.h"

namespace {

constexpr int TPB = 256;

inline int grid_for(long long n, int per_thread = 1)
{
    long long b = (n + (long long)TPB * per_thread - 1) / ((long long)TPB * per_thread);
    if (b > (1 << 30)) b = 1 << 30;
    return (int)(b > 0 ? b : 1);
}

__global__ void k_add(const u64 *__restrict__ a, const u64 *__restrict__ b, u64 *__restrict__ out,
                      long long total, int logN, int level, const ModQ *__restrict__ mq, int sub)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const u64 q = mq[(int)((idx >> logN) % level)].q;
        out[idx] = sub ? submod(a[idx], b[idx], q) : addmod(a[idx], b[idx], q);
    }
}

__global__ void k_neg(const u64 *__restrict__ a, u64 *__restrict__ out, long long total, int logN, int level,
                      const ModQ *__restrict__ mq)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const u64 q = mq[(int)((idx >> logN) % level)].q;
        out[idx] = negmod(a[idx], q);
    }
}

struct LimbConsts {
    u64 w[FHE_MAXP], ws[FHE_MAXP];
};

__global__ void k_mul_const(const u64 *__restrict__ a, u64 *__restrict__ out, long long total, int logN, int level,
                            const ModQ *__restrict__ mq, const LimbConsts k)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)((idx >> logN) % level);
        out[idx] = shoup(a[idx], k.w[i], k.ws[i], mq[i].q);
    }
}

// Adds the constant k_i (mod q_i) at every NTT point of poly 0; copies poly 1.
__global__ void k_add_const(const u64 *__restrict__ a, u64 *__restrict__ out, long long total, int logN, int level,
                            const ModQ *__restrict__ mq, const LimbConsts k)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long li = idx >> logN;
        const int i = (int)(li % level);
        const int poly = (int)((li / level) % 2);
        out[idx] = poly == 0 ? addmod(a[idx], k.w[i], mq[i].q) : a[idx];
    }
}

// (a0,a1) x (b0,b1) -> (a0 b0, a0 b1 + a1 b0, a1 b1), all NTT domain.
__global__ void k_tensor(const u64 *__restrict__ a, const u64 *__restrict__ b, u64 *__restrict__ out,
                         long long total, int logN, int level, const ModQ *__restrict__ mq)
{
    const long long LN = (long long)level << logN;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long c = idx / LN, r = idx % LN;
        const ModQ m = mq[(int)(r >> logN)];
        const u64 a0 = a[2 * c * LN + r], a1 = a[(2 * c + 1) * LN + r];
        const u64 b0 = b[2 * c * LN + r], b1 = b[(2 * c + 1) * LN + r];
        out[3 * c * LN + r] = barrett128((u128)a0 * b0, m);
        out[(3 * c + 1) * LN + r] = barrett128((u128)a0 * b1 + (u128)a1 * b0, m);
        out[(3 * c + 2) * LN + r] = barrett128((u128)a1 * b1, m);
    }
}

// Key-switching inner product.  Extended limb r = blockIdx.y of Q_l P
// (r < l: data prime r; else special prime L + r - l); ciphertexts
// blockIdx.z * CB .. + CB - 1 of the batch.  Every thread loads its 2*dnum
// key words once and reuses them for its CB ciphertexts, whose input words
// are all loaded before the first product so that the loads overlap.
template <int CB>
__global__ void __launch_bounds__(256, 3)
    k_ks_inner(const u64 *__restrict__ ext, const u64 *__restrict__ xbase, long long x_outer,
               const u64 *__restrict__ ksk, u64 *__restrict__ acc, int count, int l, int K, int L, int dnum,
               int logN, const ModQ *__restrict__ mq)
{
    const int N = 1 << logN;
    const int r = blockIdx.y;
    const int prime = r < l ? r : L + (r - l);
    const ModQ m = mq[prime];
    const int LK = L + K, lK = l + K;
    const int rdig = r < l ? r / K : -1;
    const int c0 = blockIdx.z * CB;
    const int ncb = min(CB, count - c0);
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        u128 a0[CB], a1[CB];
#pragma unroll
        for (int cc = 0; cc < CB; cc++) a0[cc] = a1[cc] = 0;
        for (int j = 0; j < dnum; j++) {
            const u64 k0 = ksk[(((long long)j * 2 + 0) * LK + prime) * N + n];
            const u64 k1 = ksk[(((long long)j * 2 + 1) * LK + prime) * N + n];
            u64 y[CB];
#pragma unroll
            for (int cc = 0; cc < CB; cc++) {
                const int c = c0 + cc;
                if (cc < ncb)
                    y[cc] = (j == rdig) ? xbase[c * x_outer + (long long)r * N + n]
                                        : ext[(((long long)c * dnum + j) * lK + r) * N + n];
            }
#pragma unroll
            for (int cc = 0; cc < CB; cc++) {
                if (cc < ncb) {
                    a0[cc] += (u128)y[cc] * k0;
                    a1[cc] += (u128)y[cc] * k1;
                }
            }
        }
#pragma unroll
        for (int cc = 0; cc < CB; cc++) {
            const int c = c0 + cc;
            if (cc < ncb) {
                acc[(((long long)c * 2 + 0) * lK + r) * N + n] = barrett128(a0[cc], m);
                acc[(((long long)c * 2 + 1) * lK + r) * N + n] = barrett128(a1[cc], m);
            }
        }
    }
}

// Relinearisation fused with the modulus switch (the inverse NTT that
// precedes this step formed y = acc_m + (P mod q_m) add_m while loading):
// after the scaled inverse NTT of the special limbs and of y, in
// src[c][pi] = (t_0 .. t_{K-1}, Y'), Y' = INTT(y) (p P)^-1, replace Y' by
// w = Y' - sum_k t_k p_k^-1 mod q_m, i.e. [x_m p^-1]_{q_m} of the
// relinearised x.
__global__ void k_rms_fold(u64 *__restrict__ src, long long total, int logN, int l, int K,
                           const RelinMSParams *__restrict__ P, const ModQ *__restrict__ mq)
{
    const int N = 1 << logN;
    const ModQ mm = mq[l - 1];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long cp = idx >> logN;
        const int n = (int)(idx & (N - 1));
        u64 *base = src + cp * (K + 1) * N + n;
        u128 a = 0;
        for (int k = 0; k < K; k++) a += (u128)base[(long long)k * N] * P->pkinv[k];
        base[(long long)K * N] = submod(base[(long long)K * N], barrett128(a, mm), mm.q);
    }
}

// k modulus switches at once: src[o] = (X'_0 .. X'_{k-1}) becomes
// (w_0 .. w_{k-1}), w_j = X'_j - sum_{t<j} w_t F[j][t] mod q_{l-1-j}.
__global__ void k_ms_fold(u64 *__restrict__ src, long long total, int logN, int l, int k,
                          const MultiSwitchParams *__restrict__ P, const ModQ *__restrict__ mq)
{
    const int N = 1 << logN;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long o = idx >> logN;
        const int n = (int)(idx & (N - 1));
        u64 *base = src + o * k * N + n;
        u64 w[FHE_MAXK];
#pragma unroll
        for (int j = 0; j < FHE_MAXK; j++) {
            if (j < k) {
                const ModQ mj = mq[l - 1 - j];
                u128 a = 0;
#pragma unroll
                for (int t = 0; t < FHE_MAXK; t++)
                    if (t < j) a += (u128)w[t] * P->F[j][t];
                w[j] = submod(base[(long long)j * N], barrett128(a, mj), mj.q);
                base[(long long)j * N] = w[j];
            }
        }
    }
}

// c0 of every ciphertext of a batch plus / minus one plaintext m[level][N]
// (NTT domain); c1 and further polynomials are left as they are (the caller
// copied them).  out may equal a.
__global__ void k_add_plain(const u64 *__restrict__ a, const u64 *__restrict__ m, u64 *__restrict__ out,
                            long long total, int logN, int level, long long ct_stride, int sub,
                            const ModQ *__restrict__ mq)
{
    const long long LN = (long long)level << logN;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long c = idx / LN, r = idx % LN;
        const u64 q = mq[(int)(r >> logN)].q;
        const u64 x = a[c * ct_stride + r], y = m[r];
        out[c * ct_stride + r] = sub ? submod(x, y, q) : addmod(x, y, q);
    }
}

// out[o][i][k] = in[o][i][perm[k]]: sigma_g in the NTT domain.
__global__ void k_automorphism(const u64 *__restrict__ in, u64 *__restrict__ out, long long total, int logN,
                               const int *__restrict__ perm)
{
    const int mask = (1 << logN) - 1;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long base = idx & ~(long long)mask;
        out[idx] = in[base + perm[idx & mask]];
    }
}

// out[o][i] = a[o][i] * b[o'][i] pointwise, b's outer stride b_outer (0 = broadcast).
__global__ void k_mul_poly(const u64 *__restrict__ a, const u64 *__restrict__ b, u64 *__restrict__ out,
                           long long total, int logN, int level, long long b_outer, const ModQ *__restrict__ mq)
{
    const long long LN = (long long)level << logN;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long o = idx / LN, r = idx % LN;
        out[idx] = barrett128((u128)a[idx] * b[o * b_outer + r], mq[(int)(r >> logN)]);
    }
}

__global__ void k_copy_limbs(const u64 *__restrict__ in, u64 *__restrict__ out, long long total, int logN, int nl,
                             long long in_outer, long long out_outer)
{
    const long long LN = (long long)nl << logN;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long o = idx / LN, r = idx % LN;
        out[o * out_outer + r] = in[o * in_outer + r];
    }
}

// out[o][i][n] = (scale * x[o][n] + y[o][n]) mod q_{prime[i]}  (y may be NULL)
__global__ void k_rns_from_i64(const int64_t *__restrict__ x, const int64_t *__restrict__ y, int64_t scale,
                               u64 *__restrict__ out, long long total, int logN, int nl, const LimbConsts pm,
                               const ModQ *__restrict__ mq)
{
    const int N = 1 << logN;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long li = idx >> logN;
        const int i = (int)(li % nl);
        const long long o = li / nl;
        const int n = (int)(idx & (N - 1));
        const u64 q = mq[(int)pm.w[i]].q;
        const int64_t v = scale * x[o * N + n] + (y ? y[o * N + n] : 0);
        const int64_t r = v % (int64_t)q;
        out[idx] = (u64)(r < 0 ? r + (int64_t)q : r);
    }
}

// out = c + a * b (pointwise), b with outer stride b_outer; c may be NULL.
// With neg != 0: out = c - a * b.
__global__ void k_muladd(const u64 *__restrict__ a, const u64 *__restrict__ b, const u64 *__restrict__ cc,
                         u64 *__restrict__ out, long long total, int logN, int level, long long b_outer, int neg,
                         const ModQ *__restrict__ mq)
{
    const long long LN = (long long)level << logN;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long o = idx / LN, r = idx % LN;
        const ModQ m = mq[(int)(r >> logN)];
        const u64 t = barrett128((u128)a[idx] * b[o * b_outer + r], m);
        const u64 base = cc ? cc[idx] : 0;
        out[idx] = neg ? submod(base, t, m.q) : addmod(base, t, m.q);
    }
}

// One digit of a switching key over the L+K primes (NTT domain):
//   k0 = e - a s + [i in D_j] (P mod q_i) s',  k1 = a.
__global__ void k_ksk_digit(const u64 *__restrict__ a, const u64 *__restrict__ e, const u64 *__restrict__ s,
                            const u64 *__restrict__ sp, u64 *__restrict__ k0, u64 *__restrict__ k1, long long total,
                            int logN, int dlo, int dhi, const LimbConsts Pm, const ModQ *__restrict__ mq)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx >> logN);
        const ModQ m = mq[i];
        u64 v = submod(e[idx], barrett128((u128)a[idx] * s[idx], m), m.q);
        if (i >= dlo && i < dhi) v = addmod(v, shoup(sp[idx], Pm.w[i], Pm.ws[i], m.q), m.q);
        k0[idx] = v;
        k1[idx] = a[idx];
    }
}

// Decryption residues (limb 0, canonical mod q0) -> plaintext coefficients:
// the centred representative in (-q0/2, q0/2], reduced mod p into [0, p).
__global__ void k_centre_mod_p(const u64 *__restrict__ x, int64_t *__restrict__ out, long long n, u64 q0, int64_t p)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const u64 v = x[i];
        const int64_t cv = v > q0 / 2 ? -(int64_t)(q0 - v) : (int64_t)v;
        int64_t r = cv % p;
        out[i] = r < 0 ? r + p : r;
    }
}

// out = sum_t w_t x_t (mod q_i), up to 8 ciphertext batches of one shape;
// w[t][i] is the scalar of term t reduced mod q_i.  Eight products of
// canonical residues stay below the Barrett bound, so one reduction suffices.
struct LinComb {
    const u64 *x[8];
    u64 w[8][FHE_MAXP];
    int n;
};

__global__ void k_lincomb(const LinComb lc, u64 *__restrict__ out, long long total, int logN, int level,
                          const ModQ *__restrict__ mq)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)((idx >> logN) % level);
        u128 acc = 0;
#pragma unroll
        for (int t = 0; t < 8; t++)
            if (t < lc.n) acc += (u128)lc.x[t][idx] * lc.w[t][i];
        out[idx] = barrett128(acc, mq[i]);
    }
}

}  // namespace

// words: u64 words read + written per element (algorithmic traffic)
#define LAUNCH_CLS_W(cls, words, kern, total, ...)                                          \
    do {                                                                                    \
        long long _t = (total);                                                             \
        if (_t > 0) {                                                                       \
            prof_begin(c, cls, 8.0 * (words) * (double)_t);                                 \
            kern<<<grid_for(_t), TPB, 0, c->stream>>>(__VA_ARGS__);                         \
            prof_end(c);                                                                    \
            c->launches++;                                                                  \
        }                                                                                   \
    } while (0)
#define LAUNCH_CLS(cls, kern, total, ...) LAUNCH_CLS_W(cls, 2, kern, total, __VA_ARGS__)
#define LAUNCH(kern, total, ...) LAUNCH_CLS_W(FHE_K_ELEMWISE, 2, kern, total, __VA_ARGS__)

void launch_add(fhe_ctx *c, const u64 *a, const u64 *b, u64 *out, int outer, int level, int sub)
{
    LAUNCH_CLS_W(FHE_K_ELEMWISE, 3, k_add, (long long)outer * level * c->N, a, b, out, (long long)outer * level * c->N, c->logN, level,
           c->d_mq, sub);
}

void launch_neg(fhe_ctx *c, const u64 *a, u64 *out, int outer, int level)
{
    LAUNCH(k_neg, (long long)outer * level * c->N, a, out, (long long)outer * level * c->N, c->logN, level, c->d_mq);
}

void launch_mul_const(fhe_ctx *c, const u64 *a, u64 *out, int outer, int level, const u64 *w, const u64 *ws)
{
    LimbConsts k;
    for (int i = 0; i < level; i++) k.w[i] = w[i], k.ws[i] = ws[i];
    LAUNCH(k_mul_const, (long long)outer * level * c->N, a, out, (long long)outer * level * c->N, c->logN, level,
           c->d_mq, k);
}

void launch_add_const(fhe_ctx *c, const u64 *a, u64 *out, int count, int level, const u64 *kv)
{
    LimbConsts k;
    for (int i = 0; i < level; i++) k.w[i] = kv[i], k.ws[i] = 0;
    LAUNCH(k_add_const, (long long)count * 2 * level * c->N, a, out, (long long)count * 2 * level * c->N, c->logN,
           level, c->d_mq, k);
}

void launch_tensor(fhe_ctx *c, const u64 *a, const u64 *b, u64 *out, int count, int level)
{
    LAUNCH_CLS_W(FHE_K_TENSOR, 7, k_tensor, (long long)count * level * c->N, a, b, out, (long long)count * level * c->N, c->logN, level,
           c->d_mq);
}

void launch_ks_inner(fhe_ctx *c, const u64 *ext, const u64 *xbase, long long x_outer, const u64 *ksk, u64 *acc,
                     int count, int level)
{
    const int dnum = c->modup[level].dnum;
    constexpr int CB = 4;  // ciphertexts per thread
    dim3 grid((c->N + TPB - 1) / TPB, level + c->K, (count + CB - 1) / CB);
    // per (r, n): 2 dnum key words once, dnum inputs and 2 outputs per ciphertext
    prof_begin(c, FHE_K_KS_INNER, 8.0 * (double)(level + c->K) * c->N * (2.0 * dnum + count * (dnum + 2.0)));
    k_ks_inner<CB><<<grid, TPB, 0, c->stream>>>(ext, xbase, x_outer, ksk, acc, count, level, c->K, c->L, dnum, c->logN,
                                            c->d_mq);
    prof_end(c);
    c->launches++;
}

void launch_automorphism(fhe_ctx *c, const u64 *in, u64 *out, int outer, int level, const int *perm)
{
    LAUNCH_CLS(FHE_K_AUTOMORPHISM, k_automorphism, (long long)outer * level * c->N, in, out, (long long)outer * level * c->N, c->logN, perm);
}

void launch_ms_fold(fhe_ctx *c, u64 *src, int outer, int level, int k)
{
    const long long total = (long long)outer * c->N;
    LAUNCH_CLS_W(FHE_K_ELEMWISE, 2.0 * k, k_ms_fold, total, src, total, c->logN, level, k,
                 c->d_mss + (size_t)level * (FHE_MAXK + 1) + k, c->d_mq);
}

void launch_rms_fold(fhe_ctx *c, u64 *src, int count, int level)
{
    const long long total = (long long)count * 2 * c->N;
    LAUNCH_CLS_W(FHE_K_ELEMWISE, c->K + 2.0, k_rms_fold, total, src, total, c->logN, level, c->K, c->d_rms + level,
                 c->d_mq);
}

void launch_add_plain(fhe_ctx *c, const u64 *a, const u64 *m, u64 *out, int count, int npoly, int level, int sub)
{
    const long long total = (long long)count * level * c->N;
    LAUNCH_CLS_W(FHE_K_ELEMWISE, 3, k_add_plain, total, a, m, out, total, c->logN, level,
                 (long long)npoly * level * c->N, sub, c->d_mq);
}

void launch_mul_poly(fhe_ctx *c, const u64 *a, const u64 *b, u64 *out, int outer, int level, long long b_outer)
{
    LAUNCH(k_mul_poly, (long long)outer * level * c->N, a, b, out, (long long)outer * level * c->N, c->logN, level,
           b_outer, c->d_mq);
}

void launch_copy_limbs(fhe_ctx *c, const u64 *in, u64 *out, int outer, int nl, long long in_outer,
                       long long out_outer)
{
    LAUNCH(k_copy_limbs, (long long)outer * nl * c->N, in, out, (long long)outer * nl * c->N, c->logN, nl, in_outer,
           out_outer);
}

void launch_rns_from_i64(fhe_ctx *c, const int64_t *x, const int64_t *y, int64_t scale, u64 *out, int outer, int nl,
                         const int *primes)
{
    LimbConsts pm;
    for (int i = 0; i < nl; i++) pm.w[i] = (u64)primes[i], pm.ws[i] = 0;
    LAUNCH(k_rns_from_i64, (long long)outer * nl * c->N, x, y, scale, out, (long long)outer * nl * c->N, c->logN, nl,
           pm, c->d_mq);
}

void launch_muladd(fhe_ctx *c, const u64 *a, const u64 *b, const u64 *cc, u64 *out, int outer, int level,
                   long long b_outer, int neg)
{
    LAUNCH(k_muladd, (long long)outer * level * c->N, a, b, cc, out, (long long)outer * level * c->N, c->logN, level,
           b_outer, neg, c->d_mq);
}

void launch_ksk_digit(fhe_ctx *c, const u64 *a, const u64 *e, const u64 *s, const u64 *sp, u64 *k0, u64 *k1, int dlo,
                      int dhi, const u64 *Pw, const u64 *Pws)
{
    LimbConsts Pm;
    for (int i = 0; i < c->np; i++) Pm.w[i] = Pw[i], Pm.ws[i] = Pws[i];
    LAUNCH(k_ksk_digit, (long long)c->np * c->N, a, e, s, sp, k0, k1, (long long)c->np * c->N, c->logN, dlo, dhi, Pm,
           c->d_mq);
}

// ---------------------------------------------------------------------------
// per-class event timing
// ---------------------------------------------------------------------------

static cudaEvent_t prof_event(fhe_ctx *c)
{
    if (!c->prof_events.empty()) {
        cudaEvent_t e = c->prof_events.back();
        c->prof_events.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// Inside a stream capture a plain event record is only a dependency marker;
// recorded as external it becomes an event-record node of the graph.
static void prof_record(fhe_ctx *c, cudaEvent_t e)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->stream, &st);
    if (st == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal);
    else
        cudaEventRecord(e, c->stream);
}

void prof_begin(fhe_ctx *c, int cls, double bytes, double bfly)
{
    if (!c->prof_on) return;
    cudaEvent_t a = prof_event(c), b = prof_event(c);
    prof_record(c, a);
    c->prof_rec.push_back({a, b});
    c->prof_rec_cls.push_back(cls);
    c->prof_rec_bytes.push_back(bytes);
    c->prof_rec_bfly.push_back(bfly);
}

void prof_end(fhe_ctx *c)
{
    if (!c->prof_on || c->prof_rec.empty()) return;
    prof_record(c, c->prof_rec.back().second);
}

extern "C" int fhe_ctx_profile(fhe_ctx *c, int on)
{
    if (!c) return FHE_EINVAL;
    c->prof_on = on != 0;
    return 0;
}

extern "C" int fhe_ctx_profile_read(fhe_ctx *c, double *ms, int64_t *count, double *bytes, double *bfly, int ncls)
{
    if (!c || ncls < 0) return FHE_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return FHE_ECUDA;
    for (int i = 0; i < ncls; i++) {
        if (ms) ms[i] = 0;
        if (count) count[i] = 0;
        if (bytes) bytes[i] = 0;
        if (bfly) bfly[i] = 0;
    }
    for (size_t r = 0; r < c->prof_rec.size(); r++) {
        float t = 0;
        cudaEventElapsedTime(&t, c->prof_rec[r].first, c->prof_rec[r].second);
        const int k = c->prof_rec_cls[r];
        if (k >= 0 && k < ncls) {
            if (ms) ms[k] += t;
            if (count) count[k] += 1;
            if (bytes) bytes[k] += c->prof_rec_bytes[r];
            if (bfly) bfly[k] += c->prof_rec_bfly[r];
        }
        c->prof_events.push_back(c->prof_rec[r].first);
        c->prof_events.push_back(c->prof_rec[r].second);
    }
    c->prof_rec.clear();
    c->prof_rec_cls.clear();
    c->prof_rec_bytes.clear();
    c->prof_rec_bfly.clear();
    return FHE_K_COUNT;
}

void launch_lincomb(fhe_ctx *c, const u64 *const *x, const u64 (*w)[FHE_MAXP], int n, u64 *out, int outer,
                    int level)
{
    LinComb lc;
    memset(&lc, 0, sizeof(lc));
    lc.n = n;
    for (int t = 0; t < n; t++) {
        lc.x[t] = x[t];
        for (int i = 0; i < level; i++) lc.w[t][i] = w[t][i];
    }
    LAUNCH_CLS_W(FHE_K_ELEMWISE, n + 1, k_lincomb, (long long)outer * level * c->N, lc, out,
                 (long long)outer * level * c->N, c->logN, level, c->d_mq);
}

void launch_centre_mod_p(fhe_ctx *c, const u64 *x, int64_t *out, long long n)
{
    LAUNCH(k_centre_mod_p, n, x, out, n, c->q[0], (int64_t)c->p);
}
