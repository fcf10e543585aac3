// ntt.cu -- NTT launches through limb maps (plain, scaled, and the scaled inverse whose
// last entry forms the relinearisation's y), the raw transforms' launchers,
// and the autotuner.
// The engine's kernels and functors are in ntt_engine.cuh.
#include "ntt_engine.cuh"

bool ntt_supported_logn(int logN) { return logN >= 10 && logN <= 15; }

// ---------------------------------------------------------------------------
// multi-segment launchers
// ---------------------------------------------------------------------------

void launch_ntt_map_many(const std::vector<NttMapArgs> &a, bool fwd, int cls)
{
    run_many<IOMap>(a, fwd, cls, [fwd](IOMap &io, int sg, const NttMapArgs &x, double *b, double *f) {
        if (x.njobs <= 0) return false;
        seg_header(io.h[sg], x.c, fwd, x.njobs / x.m.nl, x.m.nl);
        map_seg(io.s[sg], x.in, x.out, x.m, x.scale);
        *b = 16.0 * x.c->N * x.njobs;
        *f = bfly_of(x.c, x.njobs);
        return true;
    });
}

void launch_ntt_inv_scaled_y_many(const std::vector<NttYArgs> &a)
{
    run_many<IOScaledY>(a, false, FHE_K_NTT_INV, [](IOScaledY &io, int sg, const NttYArgs &x, double *b, double *f) {
        if (x.njobs <= 0) return false;
        seg_header(io.h[sg], x.c, false, x.njobs / x.m.nl, x.m.nl);
        YSeg &S = io.s[sg];
        map_seg(S, x.in, x.out, x.m, x.scale);
        S.abase = x.abase;
        S.a_outer = x.a_outer;
        S.a_poly = x.a_poly;
        S.amask = x.amask;
        S.alimb = x.level - 1;
        S.qm = x.c->q[x.level - 1];
        S.Pm = x.c->rms[x.level].Pm;
        S.Pm_s = x.c->rms[x.level].Pm_s;
        // the y entry (one of nl) also reads the addend limb
        *b = 8.0 * x.c->N * x.njobs * (2.0 + 1.0 / x.m.nl);
        *f = bfly_of(x.c, x.njobs);
        return true;
    });
}

// ---------------------------------------------------------------------------
// single-segment launchers
// ---------------------------------------------------------------------------

void launch_ntt_fwd_plain(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, int njobs)
{
    launch_ntt_map_many({NttMapArgs{c, in, out, m, nullptr, njobs}}, true, FHE_K_NTT_FWD);
}

void launch_ntt_inv_plain(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, int njobs)
{
    launch_ntt_map_many({NttMapArgs{c, in, out, m, nullptr, njobs}}, false, FHE_K_NTT_INV);
}

void launch_ntt_inv_scaled(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, const ulonglong2 *scale,
                           int njobs)
{
    launch_ntt_map_many({NttMapArgs{c, in, out, m, scale, njobs}}, false, FHE_K_NTT_INV);
}

void launch_ntt_inv_scaled_y(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, const ulonglong2 *scale,
                             int njobs, const u64 *abase, long long a_outer, long long a_poly, int amask, int level)
{
    NttYArgs y;
    static_cast<NttMapArgs &>(y) = NttMapArgs{c, in, out, m, scale, njobs};
    y.abase = abase;
    y.a_outer = a_outer;
    y.a_poly = a_poly;
    y.amask = amask;
    y.level = level;
    launch_ntt_inv_scaled_y_many({y});
}

// ---------------------------------------------------------------------------
// autotuner: the grid policy (one CTA per unit, or 6 / 4 / 2 resident CTAs
// per SM walking the units), timed on a representative batch
// ---------------------------------------------------------------------------

bool ntt_variant_ok(int logN, int v) { return ntt_supported_logn(logN) && v >= 0 && v < FHE_NTT_VARIANTS; }

// Times forward + inverse of `outer` x nl limbs (nl = min(primes, 10)),
// `outer` rounded to a multiple of 16 when >= 16 so that the row units take
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
        for (int w = 0; w < 2; w++) {
            launch_ntt_fwd_plain(c, buf, buf, m, jobs);
            launch_ntt_inv_plain(c, buf, buf, m, jobs);
        }
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 5; r++) {
            launch_ntt_fwd_plain(c, buf, buf, m, jobs);
            launch_ntt_inv_plain(c, buf, buf, m, jobs);
        }
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 5;
        if (ms_out) ms_out[v] = ms;
        // the first policy stays unless another is clearly faster (3%), so
        // that near-ties do not flip from one context to the next
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
