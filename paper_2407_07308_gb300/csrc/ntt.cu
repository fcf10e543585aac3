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
// GB300 mapping: one CTA per limb, N/32 threads, every thread keeps 32
// residues in registers.  The logN stages are split into 2-3 rounds of up to
// five stages; within a round each thread runs all butterflies of its groups
// of 2^R elements in registers, and the rounds exchange data through shared
// memory (padded by one word per 32 so every round's access pattern is
// bank-conflict free).  The first forward round reads global memory directly
// in coalesced strided order, and the last inverse round writes it the same
// way; the other end goes through shared memory so global accesses are always
// coalesced.  Butterflies are Harvey's lazy ones (values in [0,4q) forward,
// [0,2q) inverse) with Shoup twiddles.
//
// Load/store functors let one kernel body serve the plain transform and the
// fused variants: ModUp (basis conversion of a key-switching digit computed
// while loading, then NTT), ModDown and modulus switching (correction
// computed while loading, subtract-and-scale applied while storing).
#include "fhe_internal.h"

namespace {

__device__ __forceinline__ int padi(int j) { return j + (j >> 5); }

__device__ __forceinline__ void ct_bfly(u64 &X, u64 &Y, const ulonglong2 w, u64 q, u64 q2)
{
    u64 x = X >= q2 ? X - q2 : X;
    u64 t = shoup_lazy(Y, w.x, w.y, q);
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
template <int R>
__device__ __forceinline__ void fwd_round(u64 (&x)[1 << R], int s0, int hi, const ulonglong2 *__restrict__ W,
                                          u64 q, u64 q2)
{
#pragma unroll
    for (int u = 0; u < R; u++) {
        const int half = 1 << (R - 1 - u);
#pragma unroll
        for (int t = 0; t < (1 << u); t++) {
            const ulonglong2 w = __ldg(W + (1 << (s0 + u)) + (hi << u) + t);
#pragma unroll
            for (int k = 0; k < half; k++) {
                const int e = t * 2 * half + k;
                ct_bfly(x[e], x[e + half], w, q, q2);
            }
        }
    }
}

template <int R>
__device__ __forceinline__ void inv_round(u64 (&x)[1 << R], int s0, int hi, const ulonglong2 *__restrict__ W,
                                          u64 q, u64 q2)
{
#pragma unroll
    for (int u = R - 1; u >= 0; u--) {
        const int half = 1 << (R - 1 - u);
#pragma unroll
        for (int t = 0; t < (1 << u); t++) {
            const ulonglong2 w = __ldg(W + (1 << (s0 + u)) + (hi << u) + t);
#pragma unroll
            for (int k = 0; k < half; k++) {
                const int e = t * 2 * half + k;
                gs_bfly(x[e], x[e + half], w, q, q2);
            }
        }
    }
}

// One round held in shared memory: groups j = hi 2^(LOGN-S0) + e 2^LOB + lo.
template <int LOGN, int S0, int R, bool FWD>
__device__ __forceinline__ void smem_round(u64 *sm, int tid, const ulonglong2 *__restrict__ W, u64 q, u64 q2)
{
    constexpr int N = 1 << LOGN, T = N / 32, E = 1 << R, G = N / E, PER = G / T;
    constexpr int LOB = LOGN - S0 - R;
#pragma unroll
    for (int gi = 0; gi < PER; gi++) {
        const int g = tid + gi * T;
        const int hi = g >> LOB, lo = g & ((1 << LOB) - 1);
        const int base = (hi << (LOGN - S0)) + lo;
        u64 x[E];
#pragma unroll
        for (int e = 0; e < E; e++) x[e] = sm[padi(base + (e << LOB))];
        if (FWD)
            fwd_round<R>(x, S0, hi, W, q, q2);
        else
            inv_round<R>(x, S0, hi, W, q, q2);
#pragma unroll
        for (int e = 0; e < E; e++) sm[padi(base + (e << LOB))] = x[e];
    }
}

// ---------------------------------------------------------------------------
// forward kernel: rounds R0, R1, R2 (R2 may be 0)
// ---------------------------------------------------------------------------
template <int LOGN, int R0, int R1, int R2, class IO>
__global__ void __launch_bounds__((1 << LOGN) / 32)
    k_ntt_fwd(const IO io, const ModQ *__restrict__ mq, const ulonglong2 *__restrict__ tw)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    static_assert(R0 + R1 + R2 == LOGN, "rounds must cover every stage");
    extern __shared__ u64 sm[];
    const int tid = threadIdx.x;
    const typename IO::St st = io.begin(blockIdx.x, N);
    const u64 q = mq[st.prime].q, q2 = 2 * q;
    const ulonglong2 *W = tw + (size_t)st.prime * N;
    {
        constexpr int E = 1 << R0, G = N / E, PER = G / T;
#pragma unroll
        for (int gi = 0; gi < PER; gi++) {
            const int lo = tid + gi * T;
            u64 x[E];
#pragma unroll
            for (int e = 0; e < E; e++) x[e] = io.load(st, e * G + lo);
            fwd_round<R0>(x, 0, 0, W, q, q2);
#pragma unroll
            for (int e = 0; e < E; e++) sm[padi(e * G + lo)] = x[e];
        }
    }
    __syncthreads();
    smem_round<LOGN, R0, R1, true>(sm, tid, W, q, q2);
    if constexpr (R2 > 0) {
        __syncthreads();
        smem_round<LOGN, R0 + R1, R2, true>(sm, tid, W, q, q2);
    }
    __syncthreads();
    for (int k = tid; k < N; k += T) io.store(st, k, reduce4q(sm[padi(k)], q2, q));
}

template <int LOGN, int R0, int R1, int R2, class IO>
__global__ void __launch_bounds__((1 << LOGN) / 32)
    k_ntt_inv(const IO io, const ModQ *__restrict__ mq, const ulonglong2 *__restrict__ tw,
              const ulonglong2 *__restrict__ ninv)
{
    constexpr int N = 1 << LOGN, T = N / 32;
    static_assert(R0 + R1 + R2 == LOGN, "rounds must cover every stage");
    extern __shared__ u64 sm[];
    const int tid = threadIdx.x;
    const typename IO::St st = io.begin(blockIdx.x, N);
    const u64 q = mq[st.prime].q, q2 = 2 * q;
    const ulonglong2 *W = tw + (size_t)st.prime * N;
    const ulonglong2 ni = ninv[st.prime];
    for (int k = tid; k < N; k += T) sm[padi(k)] = io.load(st, k);
    __syncthreads();
    if constexpr (R2 > 0) {
        smem_round<LOGN, R0 + R1, R2, false>(sm, tid, W, q, q2);
        __syncthreads();
    }
    smem_round<LOGN, R0, R1, false>(sm, tid, W, q, q2);
    __syncthreads();
    {
        constexpr int E = 1 << R0, G = N / E, PER = G / T;
#pragma unroll
        for (int gi = 0; gi < PER; gi++) {
            const int lo = tid + gi * T;
            u64 x[E];
#pragma unroll
            for (int e = 0; e < E; e++) x[e] = sm[padi(e * G + lo)];
            inv_round<R0>(x, 0, 0, W, q, q2);
#pragma unroll
            for (int e = 0; e < E; e++) io.store(st, e * G + lo, reduce2q(shoup_lazy(x[e], ni.x, ni.y, q), q));
        }
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
};

// ModUp: extended limb t of digit j of ct c, from the coefficient-domain
// limbs of the digit:  y = sum_a [x_a (Q_j/q_a)^-1]_{q_a} (Q_j/q_a) mod r.
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
        u64 inv[FHE_MAXK], invs[FHE_MAXK], hat[FHE_MAXK], qs[FHE_MAXK];
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
        for (int a = 0; a < FHE_MAXK; a++) {
            if (a < s.nsrc) {
                s.inv[a] = P->inv_hat[j][a];
                s.invs[a] = P->inv_hat_s[j][a];
                s.hat[a] = P->hat[j][a][t];
                s.qs[a] = mq[lo + a].q;
            }
        }
        return s;
    }
    __device__ u64 load(const St &s, int n) const
    {
        u128 acc = 0;
#pragma unroll
        for (int a = 0; a < FHE_MAXK; a++) {
            if (a < s.nsrc) {
                const u64 x = s.src[(long long)a * stride + n];
                const u64 t = shoup(x, s.inv[a], s.invs[a], s.qs[a]);
                acc += (u128)t * s.hat[a];
            }
        }
        return barrett128(acc, s.mt);
    }
    __device__ void store(const St &s, int k, u64 v) const { s.dst[k] = v; }
    int stride;  // N
};

// ModDown of poly pi of ct c, data limb i:
//   delta_i = sum_k [w_k c_k]_{p_k} * (p P/p_k mod q_i)   (w = INTT'd special limbs)
//   out_i   = (acc_i - delta_i) P^-1 + addend_i
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
        u64 cinv[FHE_MAXK], cinv_s[FHE_MAXK], phat[FHE_MAXK], qk[FHE_MAXK];
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
        for (int k = 0; k < FHE_MAXK; k++) {
            if (k < K) {
                s.cinv[k] = P->cinv[k];
                s.cinv_s[k] = P->cinv_s[k];
                s.phat[k] = P->phat[k][i];
                s.qk[k] = mq[P->sprime[k]].q;
            }
        }
        return s;
    }
    __device__ u64 load(const St &s, int n) const
    {
        u128 a = 0;
#pragma unroll
        for (int k = 0; k < FHE_MAXK; k++) {
            if (k < K) {
                const u64 t = shoup(s.w[(long long)k * stride + n], s.cinv[k], s.cinv_s[k], s.qk[k]);
                a += (u128)t * s.phat[k];
            }
        }
        return barrett128(a, s.mi);
    }
    __device__ void store(const St &s, int k, u64 v) const
    {
        const u64 q = s.mi.q;
        u64 r = shoup(submod(s.acc[k], v, q), s.pinv, s.pinv_s, q);
        if (s.add) r = addmod(r, s.add[k], q);
        s.out[k] = r;
    }
};

// Modulus switch l -> l-1 of poly pi of ct c, limb i < l-1:
//   w = [x_{l-1} p^-1]_{q_{l-1}} (coefficient domain), delta_i = p w mod q_i,
//   out_i = (x_i - delta_i) q_{l-1}^-1.
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
    __device__ u64 load(const St &s, int n) const
    {
        const u64 w = shoup(s.last[n], s.pl, s.pls, s.ql);
        return shoup(w, s.pi, s.pis, s.q);
    }
    __device__ void store(const St &s, int k, u64 v) const
    {
        s.out[k] = shoup(submod(s.in[k], v, s.q), s.qi, s.qis, s.q);
    }
};

template <class IO>
void run_fwd(fhe_ctx *c, const IO &io, int njobs)
{
    if (njobs <= 0) return;
    const int N = c->N;
    const size_t smem = sizeof(u64) * (N + N / 32);
    switch (c->logN) {
#define FWD_CASE(LG, A, B, C)                                                                       \
    case LG: {                                                                                      \
        auto k = k_ntt_fwd<LG, A, B, C, IO>;                                                        \
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);            \
        k<<<njobs, (1 << LG) / 32, smem, c->stream>>>(io, c->d_mq, c->d_fwd);                       \
        break;                                                                                      \
    }
        FWD_CASE(10, 5, 5, 0)
        FWD_CASE(11, 4, 4, 3)
        FWD_CASE(12, 4, 4, 4)
        FWD_CASE(13, 5, 4, 4)
        FWD_CASE(14, 5, 5, 4)
#undef FWD_CASE
    default:
        break;
    }
    c->launches++;
}

template <class IO>
void run_inv(fhe_ctx *c, const IO &io, int njobs)
{
    if (njobs <= 0) return;
    const int N = c->N;
    const size_t smem = sizeof(u64) * (N + N / 32);
    switch (c->logN) {
#define INV_CASE(LG, A, B, C)                                                                       \
    case LG: {                                                                                      \
        auto k = k_ntt_inv<LG, A, B, C, IO>;                                                        \
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);            \
        k<<<njobs, (1 << LG) / 32, smem, c->stream>>>(io, c->d_mq, c->d_inv, c->d_ninv);            \
        break;                                                                                      \
    }
        INV_CASE(10, 5, 5, 0)
        INV_CASE(11, 4, 4, 3)
        INV_CASE(12, 4, 4, 4)
        INV_CASE(13, 5, 4, 4)
        INV_CASE(14, 5, 5, 4)
#undef INV_CASE
    default:
        break;
    }
    c->launches++;
}

}  // namespace

bool ntt_supported_logn(int logN) { return logN >= 10 && logN <= 14; }

void launch_ntt_fwd_plain(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, int njobs)
{
    IOPlain io{in, out, m};
    run_fwd(c, io, njobs);
}

void launch_ntt_inv_plain(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, int njobs)
{
    IOPlain io{in, out, m};
    run_inv(c, io, njobs);
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
    run_fwd(c, io, P.njobs * count);
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
    run_fwd(c, io, 2 * level * count);
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
    run_fwd(c, io, npoly * (level - 1) * count);
}
