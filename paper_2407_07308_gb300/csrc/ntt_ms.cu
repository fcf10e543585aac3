// ntt_ms.cu -- the modulus-switching transforms: one prime (IOModSwitch) and several
// primes at once (IOMultiSwitch), corrections fused with the forward NTT.
// The engine's kernels and functors are in ntt_engine.cuh.
#include "ntt_engine.cuh"

void launch_ntt_modswitch_many(const std::vector<NttSwitchArgs> &a)
{
    run_many<IOModSwitch>(a, true, FHE_K_NTT_MODSWITCH, [](IOModSwitch &io, int sg, const NttSwitchArgs &x, double *b,
                                                           double *f) {
        if (x.count <= 0 || x.level < 2) return false;
        seg_header(io.h[sg], x.c, true, x.npoly * x.count, x.level - 1);
        SwitchSeg &S = io.s[sg];
        S.last = x.src;
        S.in = x.in;
        S.out = x.out;
        S.P = x.c->d_modswitch + x.level;
        S.l = x.level;
        S.npoly = x.npoly;
        // each (ct, poly)'s switch value read once; x_i read, out_i written
        const double njobs = (double)x.npoly * (x.level - 1) * x.count;
        *b = 8.0 * x.c->N * ((double)x.npoly * x.count + 2.0 * njobs);
        *f = bfly_of(x.c, njobs);
        return true;
    });
}

void launch_ntt_multiswitch_many(const std::vector<NttSwitchArgs> &a)
{
    run_many<IOMultiSwitch>(a, true, FHE_K_NTT_MODSWITCH, [](IOMultiSwitch &io, int sg, const NttSwitchArgs &x,
                                                             double *b, double *f) {
        if (x.count <= 0 || x.k < 2 || x.k >= x.level) return false;
        seg_header(io.h[sg], x.c, true, x.npoly * x.count, x.level - x.k);
        MultiSeg &S = io.s[sg];
        S.src = x.src;
        S.in = x.in;
        S.out = x.out;
        S.P = x.c->d_mss + (size_t)x.level * (FHE_MAXK + 1) + x.k;
        S.l = x.level;
        S.k = x.k;
        S.npoly = x.npoly;
        // each (ct, poly)'s k switch values read once; x_i read, out_i written
        const double njobs = (double)x.npoly * (x.level - x.k) * x.count;
        *b = 8.0 * x.c->N * ((double)x.npoly * x.count * x.k + 2.0 * njobs);
        *f = bfly_of(x.c, njobs);
        return true;
    });
}

void launch_ntt_multiswitch(fhe_ctx *c, const u64 *src, const u64 *in, u64 *out, int level, int k, int npoly,
                            int count)
{
    launch_ntt_multiswitch_many({NttSwitchArgs{c, src, in, out, level, k, npoly, count}});
}

void launch_ntt_modswitch(fhe_ctx *c, const u64 *last, const u64 *in, u64 *out, int level, int npoly, int count)
{
    launch_ntt_modswitch_many({NttSwitchArgs{c, last, in, out, level, 1, npoly, count}});
}

