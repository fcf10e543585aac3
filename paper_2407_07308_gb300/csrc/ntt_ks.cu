// ntt_ks.cu -- the key-switching transforms: ModUp (basis conversion fused with the
// forward NTT), ModDown and the relinearisation + modulus switch (corrections
// fused with the forward NTT).
// The engine's kernels and functors are in ntt_engine.cuh.
#include "ntt_engine.cuh"

void launch_ntt_modup_many(const std::vector<NttModUpArgs> &a)
{
    run_many<IOModUp>(a, true, FHE_K_NTT_MODUP, [](IOModUp &io, int sg, const NttModUpArgs &x, double *b, double *f) {
        const ModUpParams &P = x.c->modup[x.level];
        if (x.count <= 0 || P.njobs <= 0) return false;
        seg_header(io.h[sg], x.c, true, x.count, P.njobs);
        ModUpSeg &S = io.s[sg];
        S.d2c = x.d2c;
        S.ext = x.ext;
        S.P = x.c->d_modup + x.level;
        S.l = x.level;
        S.K = x.c->K;
        S.dnum = P.dnum;
        // the level's l coefficient limbs read once per ciphertext (every
        // digit's targets convert from them), one limb written per job
        *b = 8.0 * x.c->N * ((double)x.level + P.njobs) * x.count;
        *f = bfly_of(x.c, (double)P.njobs * x.count);
        return true;
    });
}

void launch_ntt_moddown_many(const std::vector<NttDownArgs> &a)
{
    run_many<IOModDown>(a, true, FHE_K_NTT_MODDOWN, [](IOModDown &io, int sg, const NttDownArgs &x, double *b, double *f) {
        if (x.count <= 0) return false;
        seg_header(io.h[sg], x.c, true, 2 * x.count, x.level);
        ModDownSeg &S = io.s[sg];
        S.accP = x.src;
        S.acc = x.acc;
        S.abase = x.abase;
        S.a_outer = x.a_outer;
        S.a_poly = x.a_poly;
        S.amask = x.amask;
        S.out = x.out;
        S.P = x.c->d_moddown + x.level;
        S.l = x.level;
        S.K = x.c->K;
        // the K special limbs of each (ct, poly) read once; acc_i and (for
        // masked polys) the addend read, out_i written
        const double add_frac = ((x.amask & 1) + ((x.amask >> 1) & 1)) / 2.0;
        const double njobs = 2.0 * x.level * x.count;
        *b = 8.0 * x.c->N * (2.0 * x.count * x.c->K + njobs * (2.0 + add_frac));
        *f = bfly_of(x.c, njobs);
        return true;
    });
}

void launch_ntt_relin_ms_many(const std::vector<NttDownArgs> &a)
{
    run_many<IORelinMS>(a, true, FHE_K_NTT_MODDOWN, [](IORelinMS &io, int sg, const NttDownArgs &x, double *b, double *f) {
        if (x.count <= 0 || x.level < 2) return false;
        seg_header(io.h[sg], x.c, true, 2 * x.count, x.level - 1);
        RelinMSSeg &S = io.s[sg];
        S.src = x.src;
        S.acc = x.acc;
        S.abase = x.abase;
        S.a_outer = x.a_outer;
        S.a_poly = x.a_poly;
        S.amask = x.amask;
        S.out = x.out;
        S.P = x.c->d_rms + x.level;
        S.l = x.level;
        S.K = x.c->K;
        // the K + 1 correction sources of each (ct, poly) read once; acc_i
        // and (for masked polys) the addend read, out_i written
        const double add_frac = ((x.amask & 1) + ((x.amask >> 1) & 1)) / 2.0;
        const double njobs = 2.0 * (x.level - 1) * x.count;
        *b = 8.0 * x.c->N * (2.0 * x.count * (x.c->K + 1.0) + njobs * (2.0 + add_frac));
        *f = bfly_of(x.c, njobs);
        return true;
    });
}

void launch_ntt_modup(fhe_ctx *c, const u64 *d2c, u64 *ext, int level, int count)
{
    launch_ntt_modup_many({NttModUpArgs{c, d2c, ext, level, count}});
}

void launch_ntt_moddown(fhe_ctx *c, const u64 *accP, const u64 *acc, const u64 *abase, long long a_outer,
                        long long a_poly, int amask, u64 *out, int level, int count)
{
    launch_ntt_moddown_many({NttDownArgs{c, accP, acc, abase, a_outer, a_poly, amask, out, level, count}});
}

void launch_ntt_relin_ms(fhe_ctx *c, const u64 *src, const u64 *acc, const u64 *abase, long long a_outer,
                         long long a_poly, int amask, u64 *out, int level, int count)
{
    launch_ntt_relin_ms_many({NttDownArgs{c, src, acc, abase, a_outer, a_poly, amask, out, level, count}});
}

