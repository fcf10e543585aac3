// eval.cu -- BGV operations on ciphertext batches and the comparison circuits.
//
// Each operation acts on a whole batch (count ciphertexts of one level) with a
// handful of launches: one kernel per step for the batch, never one per
// ciphertext or per limb.
//
// Key switching (hybrid, BGV flavour) of the poly X at level l, K special
// primes, dnum = ceil(l/K) digits D_j = data limbs [jK, min((j+1)K, l)):
//   1. INTT(X)                                            (l limbs per ct)
//   2. ModUp: for every digit j and every limb t of Q_l P outside D_j, fast
//      basis conversion of X_{D_j} to t, fused with the forward NTT of t
//   3. inner product  acc_pi[t] = sum_j X_j[t] ksk_j[pi][t]   (pi = 0, 1)
//   4. INTT of the K special limbs of acc_0 and acc_1
//   5. ModDown fused with NTT: delta = p FBC_{P->Q}([acc_P p^-1]_P),
//      out_pi = addend_pi + (acc_pi - delta) P^-1
// Modulus switching l -> l-1: INTT of the last limb, then one fused kernel
// that forms delta = p [x_last p^-1]_{q_last}, transforms it and applies
// (x - delta) q_last^-1.
#include <algorithm>
#include <functional>
#include <map>
#include <set>

#include "fhe_internal.h"

namespace {

struct Tmp {
    fhe_ctx *c;
    u64 *p = nullptr;
    Tmp(fhe_ctx *ctx, size_t words, int *err) : c(ctx)
    {
        if (*err) return;
        p = (u64 *)c->pool.get(words * sizeof(u64), err);
    }
    ~Tmp()
    {
        if (p) c->pool.put(p);
    }
};

LimbMap identity_map(int nl, long long in_outer, long long out_outer, int in_off, int out_off, int prime_off)
{
    LimbMap m;
    memset(&m, 0, sizeof(m));
    m.nl = nl;
    m.in_outer = in_outer;
    m.out_outer = out_outer;
    for (int i = 0; i < nl; i++) {
        m.in_limb[i] = in_off + i;
        m.out_limb[i] = out_off + i;
        m.prime[i] = prime_off + i;
    }
    return m;
}

void trace(fhe_ctx *c, int op, int level)
{
    if (c->tracing) {
        c->trace_op.push_back(op);
        c->trace_level.push_back(level);
    }
}

}  // namespace

int64_t centred_const(const fhe_ctx *c, int64_t k)
{
    const int64_t p = (int64_t)c->p;
    int64_t r = k % p;
    if (r < 0) r += p;
    return r > p / 2 ? r - p : r;
}

int op_modswitch1(fhe_ctx *c, const fhe_ct *a, fhe_ct **out)
{
    const int l = a->level, N = c->N;
    if (l < 2) return fhe_fail(c, FHE_ELEVEL, "modulus switch below level 1");
    int err = 0;
    fhe_ct *r = ct_new(c, a->count, a->npoly, l - 1, &err);
    if (!r) return err;
    Tmp last(c, (size_t)a->count * a->npoly * N, &err);
    if (err) {
        fhe_ct_destroy(r);
        return err;
    }
    const int outer = a->count * a->npoly;
    // last = [x_{l-1} p^-1]_{q_{l-1}} in the coefficient domain
    LimbMap m = identity_map(1, (long long)l * N, N, l - 1, 0, l - 1);
    launch_ntt_inv_scaled(c, a->d, last.p, m, c->d_ms_lastscale + l, outer);
    launch_ntt_modswitch(c, last.p, a->d, r->d, l, a->npoly, a->count);
    *out = r;
    return 0;
}

// k single switches at once (2 <= k <= FHE_MAXK, k < level); the same residues.
int op_modswitch_k(fhe_ctx *c, const fhe_ct *a, int k, fhe_ct **out)
{
    const int l = a->level, N = c->N;
    if (k == 1) return op_modswitch1(c, a, out);
    if (k < 1 || k > FHE_MAXK || k >= l) return fhe_fail(c, FHE_ELEVEL, "modulus switch below level 1");
    int err = 0;
    fhe_ct *r = ct_new(c, a->count, a->npoly, l - k, &err);
    if (!r) return err;
    const int outer = a->count * a->npoly;
    Tmp src(c, (size_t)outer * k * N, &err);
    if (err) {
        fhe_ct_destroy(r);
        return err;
    }
    // X'_j = INTT(x_{l-1-j}) p^-1 D_j^-1 into src[o][j]
    LimbMap m;
    memset(&m, 0, sizeof(m));
    m.nl = k;
    m.in_outer = (long long)l * N;
    m.out_outer = (long long)k * N;
    for (int j = 0; j < k; j++) m.in_limb[j] = l - 1 - j, m.out_limb[j] = j, m.prime[j] = l - 1 - j;
    launch_ntt_inv_scaled(c, a->d, src.p, m, c->d_mss_scale + ((size_t)l * (FHE_MAXK + 1) + k) * FHE_MAXK,
                          outer * k);
    launch_ms_fold(c, src.p, outer, l, k);
    launch_ntt_multiswitch(c, src.p, a->d, r->d, l, k, a->npoly, a->count);
    *out = r;
    return 0;
}

int op_lower(fhe_ctx *c, const fhe_ct *a, int level, fhe_ct **out)
{
    if (level < 1 || level > a->level) return fhe_fail(c, FHE_ELEVEL, "bad target level");
    if (level == a->level) {
        int err = 0;
        fhe_ct *r = ct_new(c, a->count, a->npoly, a->level, &err);
        if (!r) return err;
        cudaMemcpyAsync(r->d, a->d, a->bytes, cudaMemcpyDeviceToDevice, c->stream);
        *out = r;
        return 0;
    }
    const fhe_ct *cur = a;
    fhe_ct *owned = nullptr;
    while (cur->level > level) {
        fhe_ct *nx = nullptr;
        int e = op_modswitch_k(c, cur, std::min(cur->level - level, FHE_MAXK), &nx);
        if (owned) fhe_ct_destroy(owned);
        if (e) return e;
        owned = nx;
        cur = nx;
    }
    *out = owned;
    return 0;
}

int op_addsub(fhe_ctx *c, const fhe_ct *a, const fhe_ct *b, int sub, fhe_ct **out)
{
    if (a->level != b->level || a->count != b->count || a->npoly != b->npoly)
        return fhe_fail(c, FHE_EMISMATCH, "add/sub: shapes differ");
    int err = 0;
    fhe_ct *r = ct_new(c, a->count, a->npoly, a->level, &err);
    if (!r) return err;
    launch_add(c, a->d, b->d, r->d, a->count * a->npoly, a->level, sub);
    *out = r;
    return 0;
}

int op_neg(fhe_ctx *c, const fhe_ct *a, fhe_ct **out)
{
    int err = 0;
    fhe_ct *r = ct_new(c, a->count, a->npoly, a->level, &err);
    if (!r) return err;
    launch_neg(c, a->d, r->d, a->count * a->npoly, a->level);
    *out = r;
    return 0;
}

int op_mul_const(fhe_ctx *c, const fhe_ct *a, int64_t k, fhe_ct **out)
{
    int err = 0;
    fhe_ct *r = ct_new(c, a->count, a->npoly, a->level, &err);
    if (!r) return err;
    const int64_t kc = centred_const(c, k);
    u64 w[FHE_MAXP], ws[FHE_MAXP];
    for (int i = 0; i < a->level; i++) {
        const u64 q = c->q[i];
        w[i] = kc >= 0 ? (u64)kc % q : (q - ((u64)(-kc) % q)) % q;
        ws[i] = shoup_const(w[i], q);
    }
    launch_mul_const(c, a->d, r->d, a->count * a->npoly, a->level, w, ws);
    *out = r;
    return 0;
}

int op_add_const(fhe_ctx *c, const fhe_ct *a, int64_t k, fhe_ct **out)
{
    if (a->npoly != 2) return fhe_fail(c, FHE_EINVAL, "add_const needs a 2-poly ciphertext");
    int err = 0;
    fhe_ct *r = ct_new(c, a->count, 2, a->level, &err);
    if (!r) return err;
    const int64_t kc = centred_const(c, k);
    u64 w[FHE_MAXP];
    for (int i = 0; i < a->level; i++) {
        const u64 q = c->q[i];
        w[i] = kc >= 0 ? (u64)kc % q : (q - ((u64)(-kc) % q)) % q;
    }
    launch_add_const(c, a->d, r->d, a->count, a->level, w);
    *out = r;
    return 0;
}

// sum_t k_t x_t for n <= 8 batches of one shape, constants lifted to (-p/2, p/2]
int op_lincomb(fhe_ctx *c, const fhe_ct *const *x, const int64_t *k, int n, fhe_ct **out)
{
    if (n < 1 || n > 8) return fhe_fail(c, FHE_EINVAL, "lincomb: 1..8 terms");
    for (int t = 1; t < n; t++)
        if (x[t]->level != x[0]->level || x[t]->count != x[0]->count || x[t]->npoly != x[0]->npoly)
            return fhe_fail(c, FHE_EMISMATCH, "lincomb: shapes differ");
    int err = 0;
    fhe_ct *r = ct_new(c, x[0]->count, x[0]->npoly, x[0]->level, &err);
    if (!r) return err;
    const u64 *ptr[8];
    u64 w[8][FHE_MAXP];
    for (int t = 0; t < n; t++) {
        ptr[t] = x[t]->d;
        const int64_t kc = centred_const(c, k[t]);
        for (int i = 0; i < x[0]->level; i++) {
            const u64 q = c->q[i];
            w[t][i] = kc >= 0 ? (u64)kc % q : (q - ((u64)(-kc) % q)) % q;
        }
    }
    launch_lincomb(c, ptr, w, n, r->d, x[0]->count * x[0]->npoly, x[0]->level);
    *out = r;
    return 0;
}

int op_tensor(fhe_ctx *c, const fhe_ct *a, const fhe_ct *b, fhe_ct **out)
{
    if (a->level != b->level || a->count != b->count || a->npoly != 2 || b->npoly != 2)
        return fhe_fail(c, FHE_EMISMATCH, "tensor: shapes differ");
    int err = 0;
    fhe_ct *r = ct_new(c, a->count, 3, a->level, &err);
    if (!r) return err;
    launch_tensor(c, a->d, b->d, r->d, a->count, a->level);
    *out = r;
    return 0;
}

// Key-switch the poly X_c = xbase + c*x_outer (NTT domain, l limbs) of each
// ct of the batch; out_c[pi] = addend + ModDown(sum_j ModUp_j(X_c) ksk_j[pi]).
static int keyswitch(fhe_ctx *c, const u64 *xbase, long long x_outer, const u64 *abase, long long a_outer,
                     long long a_poly, int amask, const KeySwitchKey &k, int count, int l, u64 *out)
{
    const int N = c->N, K = c->K, dnum = c->modup[l].dnum;
    int err = 0;
    Tmp xc(c, (size_t)count * l * N, &err);
    Tmp ext(c, (size_t)count * dnum * (l + K) * N, &err);
    Tmp acc(c, (size_t)count * 2 * (l + K) * N, &err);
    Tmp accP(c, (size_t)count * 2 * K * N, &err);
    if (err) return fhe_fail(c, err, "key switching: out of device memory");
    // 1. INTT of X, each limb i of digit j times (Q_j/q_i)^-1 (the first step of
    //    the basis conversion)
    LimbMap m1 = identity_map(l, x_outer, (long long)l * N, 0, 0, 0);
    launch_ntt_inv_scaled(c, xbase, xc.p, m1, c->d_ks_xscale + (size_t)l * FHE_MAXP, count * l);
    // 2. ModUp (basis conversion fused with NTT)
    launch_ntt_modup(c, xc.p, ext.p, l, count);
    // 3. inner product with the key
    launch_ks_inner(c, ext.p, xbase, x_outer, k.d, acc.p, count, l);
    // 4. INTT of the special limbs of both accumulators, times p^-1 (P/p_k)^-1
    LimbMap m4 = identity_map(K, (long long)(l + K) * N, (long long)K * N, l, 0, c->L);
    launch_ntt_inv_scaled(c, acc.p, accP.p, m4, c->d_ks_pscale, count * 2 * K);
    // 5. ModDown fused with NTT, plus the addend
    launch_ntt_moddown(c, accP.p, acc.p, abase, a_outer, a_poly, amask, out, l, count);
    return 0;
}

// Key switching whose ModDown also drops the last prime (l -> l-1): the same
// residues as keyswitch() followed by op_modswitch1, with one forward NTT
// per kept limb instead of two and no inverse NTT of the switched output
// (see RelinMSParams).  Needs K + 1 <= FHE_MAXK.
static int keyswitch_ms(fhe_ctx *c, const u64 *xbase, long long x_outer, const u64 *abase, long long a_outer,
                        long long a_poly, int amask, const KeySwitchKey &k, int count, int l, u64 *out)
{
    const int N = c->N, K = c->K, dnum = c->modup[l].dnum;
    int err = 0;
    Tmp xc(c, (size_t)count * l * N, &err);
    Tmp ext(c, (size_t)count * dnum * (l + K) * N, &err);
    Tmp acc(c, (size_t)count * 2 * (l + K) * N, &err);
    Tmp src(c, (size_t)count * 2 * (K + 1) * N, &err);
    if (err) return fhe_fail(c, err, "key switching: out of device memory");
    LimbMap m1 = identity_map(l, x_outer, (long long)l * N, 0, 0, 0);
    launch_ntt_inv_scaled(c, xbase, xc.p, m1, c->d_ks_xscale + (size_t)l * FHE_MAXP, count * l);
    launch_ntt_modup(c, xc.p, ext.p, l, count);
    launch_ks_inner(c, ext.p, xbase, x_outer, k.d, acc.p, count, l);
    // t_k = INTT(acc_P,k) p^-1 (P/p_k)^-1 and Y' = INTT(y) (p P)^-1 with
    // y = acc_{l-1} + P add_{l-1} formed while loading
    LimbMap m4;
    memset(&m4, 0, sizeof(m4));
    m4.nl = K + 1;
    m4.in_outer = (long long)(l + K) * N;
    m4.out_outer = (long long)(K + 1) * N;
    for (int j = 0; j < K; j++) {
        m4.in_limb[j] = l + j;
        m4.out_limb[j] = j;
        m4.prime[j] = c->L + j;
    }
    m4.in_limb[K] = l - 1;
    m4.out_limb[K] = K;
    m4.prime[K] = l - 1;
    // scales (ks_pscale[0..K-1], rms_yscale[l])
    launch_ntt_inv_scaled_y(c, acc.p, src.p, m4, c->d_ms4scale + (size_t)l * (FHE_MAXK + 1), count * 2 * (K + 1),
                            abase, a_outer, a_poly, amask, l);
    launch_rms_fold(c, src.p, count, l);
    launch_ntt_relin_ms(c, src.p, acc.p, abase, a_outer, a_poly, amask, out, l, count);
    return 0;
}

int op_relin(fhe_ctx *c, const KeySwitchKey &k, const fhe_ct *d, fhe_ct **out)
{
    if (d->npoly != 3) return fhe_fail(c, FHE_EINVAL, "relinearize needs a 3-poly ciphertext");
    const int l = d->level, N = c->N;
    int err = 0;
    fhe_ct *r = ct_new(c, d->count, 2, l, &err);
    if (!r) return err;
    const long long LN = (long long)l * N;
    err = keyswitch(c, d->d + 2 * LN, 3 * LN, d->d, 3 * LN, LN, 3, k, d->count, l, r->d);
    if (err) {
        fhe_ct_destroy(r);
        return err;
    }
    *out = r;
    return 0;
}

int galois_perm(fhe_ctx *c, int64_t g, const int **perm)
{
    auto it = c->d_perm.find(g);
    if (it != c->d_perm.end()) {
        *perm = it->second;
        return 0;
    }
    const int N = c->N, logN = c->logN;
    const int64_t twoN = 2 * (int64_t)N;
    if (g <= 0 || g >= twoN || (g & 1) == 0) return fhe_fail(c, FHE_EINVAL, "Galois element must be odd in (0, 2N)");
    auto brv = [logN](int x) {
        int r = 0;
        for (int i = 0; i < logN; i++) r |= ((x >> i) & 1) << (logN - 1 - i);
        return r;
    };
    // NTT slot k holds a(psi^(2 brv(k)+1)); sigma_g(a) there is a(psi^(g(2 brv(k)+1))).
    std::vector<int> h(N);
    for (int k = 0; k < N; k++) {
        const int64_t e = (g * (2 * (int64_t)brv(k) + 1)) % twoN;
        h[k] = brv((int)((e - 1) / 2));
    }
    int *d = nullptr;
    if (cudaMalloc(&d, sizeof(int) * N) != cudaSuccess) return fhe_fail(c, FHE_ENOMEM, "Galois map");
    cudaMemcpy(d, h.data(), sizeof(int) * N, cudaMemcpyHostToDevice);
    c->d_perm[g] = d;
    *perm = d;
    return 0;
}

int op_rotate(fhe_ctx *c, const KeySwitchKey &k, const fhe_ct *a, fhe_ct **out)
{
    if (a->npoly != 2) return fhe_fail(c, FHE_EINVAL, "rotate needs a 2-poly ciphertext");
    const int l = a->level, N = c->N;
    const int *perm = nullptr;
    int err = galois_perm(c, k.galois, &perm);
    if (err) return err;
    fhe_ct *sg = ct_new(c, a->count, 2, l, &err);
    if (!sg) return err;
    launch_automorphism(c, a->d, sg->d, a->count * 2, l, perm);
    fhe_ct *r = ct_new(c, a->count, 2, l, &err);
    if (!r) {
        fhe_ct_destroy(sg);
        return err;
    }
    const long long LN = (long long)l * N;
    err = keyswitch(c, sg->d + LN, 2 * LN, sg->d, 2 * LN, LN, 1, k, a->count, l, r->d);
    fhe_ct_destroy(sg);
    if (err) {
        fhe_ct_destroy(r);
        return err;
    }
    *out = r;
    return 0;
}

int op_mul_relin(fhe_ctx *c, const KeySwitchKey &rlk, const fhe_ct *a, const fhe_ct *b, fhe_ct **out)
{
    fhe_ct *d = nullptr, *r = nullptr;
    int err = op_tensor(c, a, b, &d);
    if (err) return err;
    if (d->level > 1 && c->K + 1 <= FHE_MAXK && !c->separate_ms) {
        // relinearise and switch down one prime in one ModDown
        const int l = d->level;
        const long long LN = (long long)l * c->N;
        r = ct_new(c, d->count, 2, l - 1, &err);
        if (r) err = keyswitch_ms(c, d->d + 2 * LN, 3 * LN, d->d, 3 * LN, LN, 3, rlk, d->count, l, r->d);
        fhe_ct_destroy(d);
        if (err) {
            fhe_ct_destroy(r);
            return err;
        }
        *out = r;
        return 0;
    }
    err = op_relin(c, rlk, d, &r);
    fhe_ct_destroy(d);
    if (err) return err;
    if (r->level > 1) {
        fhe_ct *s = nullptr;
        err = op_modswitch1(c, r, &s);
        fhe_ct_destroy(r);
        if (err) return err;
        r = s;
    }
    *out = r;
    return 0;
}

// ---------------------------------------------------------------------------
// the same operations over several batches at once: every step is one launch
// for all of them (segment tables, see ntt.cu and many.cu), so the launches
// of independent products are as large as their sum.  Items may belong to
// different contexts of one device; the launches run on the stream of the
// first item's context.
// ---------------------------------------------------------------------------

int op_mul_relin_many(std::vector<MulItem> &it)
{
    std::vector<size_t> fused;
    for (size_t i = 0; i < it.size(); i++) {
        MulItem &m = it[i];
        fhe_ctx *c = m.c;
        if (m.a->level != m.b->level || m.a->count != m.b->count || m.a->npoly != 2 || m.b->npoly != 2)
            return fhe_fail(c, FHE_EMISMATCH, "tensor: shapes differ");
        if (m.a->level > 1 && c->K + 1 <= FHE_MAXK && !c->separate_ms)
            fused.push_back(i);
        else if (int e = op_mul_relin(c, *m.rlk, m.a, m.b, &m.out))
            return e;
    }
    if (fused.empty()) return 0;
    struct Tm {
        fhe_ct *d = nullptr, *r = nullptr;
        u64 *xc = nullptr, *ext = nullptr, *acc = nullptr, *src = nullptr;
    };
    std::vector<Tm> tm(fused.size());
    int err = 0;
    auto release = [&]() {
        for (size_t j = 0; j < fused.size(); j++) {
            fhe_ctx *c = it[fused[j]].c;
            Tm &t = tm[j];
            if (t.d) fhe_ct_destroy(t.d);
            for (u64 *q : {t.xc, t.ext, t.acc, t.src})
                if (q) c->pool.put(q);
            t = Tm();
        }
    };
    for (size_t j = 0; j < fused.size() && !err; j++) {
        const MulItem &m = it[fused[j]];
        fhe_ctx *c = m.c;
        const int l = m.a->level, count = m.a->count, N = c->N, K = c->K, dnum = c->modup[l].dnum;
        Tm &t = tm[j];
        t.d = ct_new(c, count, 3, l, &err);
        if (!err) t.r = ct_new(c, count, 2, l - 1, &err);
        if (!err) t.xc = (u64 *)c->pool.get(sizeof(u64) * (size_t)count * l * N, &err);
        if (!err) t.ext = (u64 *)c->pool.get(sizeof(u64) * (size_t)count * dnum * (l + K) * N, &err);
        if (!err) t.acc = (u64 *)c->pool.get(sizeof(u64) * (size_t)count * 2 * (l + K) * N, &err);
        if (!err) t.src = (u64 *)c->pool.get(sizeof(u64) * (size_t)count * 2 * (K + 1) * N, &err);
    }
    if (err) {
        for (Tm &t : tm)
            if (t.r) fhe_ct_destroy(t.r);
        release();
        return fhe_fail(it[0].c, err, "product: out of device memory");
    }
    std::vector<TensorArgs> ta;
    std::vector<NttMapArgs> m1;
    std::vector<NttModUpArgs> mu;
    std::vector<KsInnerArgs> ks;
    std::vector<NttYArgs> ys;
    std::vector<FoldArgs> fo;
    std::vector<NttDownArgs> dn;
    for (size_t j = 0; j < fused.size(); j++) {
        const MulItem &m = it[fused[j]];
        fhe_ctx *c = m.c;
        const Tm &t = tm[j];
        const int l = m.a->level, count = m.a->count, K = c->K;
        const long long LN = (long long)l * c->N;
        const u64 *x2 = t.d->d + 2 * LN;  // the key-switched poly c2
        ta.push_back(TensorArgs{c, m.a->d, m.b->d, t.d->d, count, l});
        // INTT of c2, each limb i of digit j times (Q_j/q_i)^-1
        m1.push_back(NttMapArgs{c, x2, t.xc, identity_map(l, 3 * LN, LN, 0, 0, 0),
                                c->d_ks_xscale + (size_t)l * FHE_MAXP, count * l});
        mu.push_back(NttModUpArgs{c, t.xc, t.ext, l, count});
        ks.push_back(KsInnerArgs{c, t.ext, x2, 3 * LN, m.rlk->d, t.acc, count, l});
        // t_k = INTT(acc_P,k) p^-1 (P/p_k)^-1 and Y' = INTT(y) (p P)^-1 with
        // y = acc_{l-1} + P add_{l-1} formed while loading
        NttYArgs y;
        LimbMap m4;
        memset(&m4, 0, sizeof(m4));
        m4.nl = K + 1;
        m4.in_outer = (long long)(l + K) * c->N;
        m4.out_outer = (long long)(K + 1) * c->N;
        for (int q = 0; q < K; q++) m4.in_limb[q] = l + q, m4.out_limb[q] = q, m4.prime[q] = c->L + q;
        m4.in_limb[K] = l - 1;
        m4.out_limb[K] = K;
        m4.prime[K] = l - 1;
        static_cast<NttMapArgs &>(y) =
            NttMapArgs{c, t.acc, t.src, m4, c->d_ms4scale + (size_t)l * (FHE_MAXK + 1), count * 2 * (K + 1)};
        y.abase = t.d->d;
        y.a_outer = 3 * LN;
        y.a_poly = LN;
        y.amask = 3;
        y.level = l;
        ys.push_back(y);
        fo.push_back(FoldArgs{c, t.src, count, l, 0});
        dn.push_back(NttDownArgs{c, t.src, t.acc, t.d->d, 3 * LN, LN, 3, t.r->d, l, count});
    }
    launch_tensor_many(ta);
    launch_ntt_map_many(m1, false, FHE_K_NTT_INV);
    launch_ntt_modup_many(mu);
    launch_ks_inner_many(ks);
    launch_ntt_inv_scaled_y_many(ys);
    launch_rms_fold_many(fo);
    launch_ntt_relin_ms_many(dn);
    for (size_t j = 0; j < fused.size(); j++) it[fused[j]].out = tm[j].r;
    release();
    return 0;
}

int op_modswitch_many(std::vector<SwitchItem> &it)
{
    std::vector<NttMapArgs> inv;
    std::vector<FoldArgs> fold;
    std::vector<NttSwitchArgs> one, multi;
    std::vector<std::pair<fhe_ctx *, u64 *>> tmp;
    int err = 0;
    for (SwitchItem &s : it) {
        fhe_ctx *c = s.c;
        const fhe_ct *a = s.a;
        const int l = a->level, k = s.k, N = c->N, outer = a->count * a->npoly;
        if (k < 1 || k > FHE_MAXK || k >= l) {
            err = fhe_fail(c, FHE_ELEVEL, "modulus switch below level 1");
            break;
        }
        s.out = ct_new(c, a->count, a->npoly, l - k, &err);
        if (err) break;
        u64 *src = (u64 *)c->pool.get(sizeof(u64) * (size_t)outer * k * N, &err);
        if (err) break;
        tmp.push_back({c, src});
        LimbMap m;
        memset(&m, 0, sizeof(m));
        m.nl = k;
        m.in_outer = (long long)l * N;
        m.out_outer = (long long)k * N;
        for (int j = 0; j < k; j++) m.in_limb[j] = l - 1 - j, m.out_limb[j] = j, m.prime[j] = l - 1 - j;
        if (k == 1) {
            // w = [x_{l-1} p^-1]_{q_{l-1}} in the coefficient domain
            inv.push_back(NttMapArgs{c, a->d, src, m, c->d_ms_lastscale + l, outer});
            one.push_back(NttSwitchArgs{c, src, a->d, s.out->d, l, 1, a->npoly, a->count});
        } else {
            // X'_j = INTT(x_{l-1-j}) p^-1 D_j^-1
            inv.push_back(NttMapArgs{c, a->d, src, m, c->d_mss_scale + ((size_t)l * (FHE_MAXK + 1) + k) * FHE_MAXK,
                                     outer * k});
            fold.push_back(FoldArgs{c, src, outer, l, k});
            multi.push_back(NttSwitchArgs{c, src, a->d, s.out->d, l, k, a->npoly, a->count});
        }
    }
    if (!err) {
        launch_ntt_map_many(inv, false, FHE_K_NTT_INV);
        launch_ms_fold_many(fold);
        launch_ntt_modswitch_many(one);
        launch_ntt_multiswitch_many(multi);
    }
    for (auto &t : tmp) t.first->pool.put(t.second);
    if (err)
        for (SwitchItem &s : it)
            if (s.out) fhe_ct_destroy(s.out), s.out = nullptr;
    return err;
}

int op_ew_many(std::vector<EwItem> &it)
{
    std::vector<EwArgs> args;
    int err = 0;
    for (EwItem &e : it) {
        fhe_ctx *c = e.c;
        const fhe_ct *x0 = e.x[0];
        for (int j = 1; j < e.n; j++)
            if (e.x[j]->level != x0->level || e.x[j]->count != x0->count || e.x[j]->npoly != x0->npoly)
                err = fhe_fail(c, FHE_EMISMATCH, "element-wise operation: shapes differ");
        if (e.op == FHE_EW_CADD && x0->npoly != 2) err = fhe_fail(c, FHE_EINVAL, "add_const needs a 2-poly ciphertext");
        if (err) break;
        e.out = ct_new(c, x0->count, x0->npoly, x0->level, &err);
        if (err) break;
        EwArgs a;
        memset(&a, 0, sizeof(a));
        a.c = c;
        a.op = e.op;
        a.n = e.n;
        for (int j = 0; j < e.n; j++) a.x[j] = e.x[j]->d, a.k[j] = centred_const(c, e.k[j]);
        a.out = e.out->d;
        a.outer = x0->count * x0->npoly;
        a.level = x0->level;
        args.push_back(a);
    }
    if (err) {
        for (EwItem &e : it)
            if (e.out) fhe_ct_destroy(e.out), e.out = nullptr;
        return err;
    }
    launch_ew_many(args);
    return 0;
}

// Plaintext operand: coefficients m[N] (any residues mod p) lifted to
// (-p/2, p/2], reduced mod q_0 .. q_{level-1} and transformed: [level][N] in
// the NTT domain, in the ciphertext `out` (count 1, one poly).
static int plain_ntt(fhe_ctx *c, const int64_t *m_in, int level, fhe_ct **out)
{
    const int N = c->N;
    std::vector<int64_t> m(m_in, m_in + N);
    const int64_t p = (int64_t)c->p;
    for (int64_t &x : m) {
        x %= p;
        if (x < 0) x += p;
        if (x > p / 2) x -= p;
    }
    int err = 0;
    fhe_ct *r = ct_new(c, 1, 1, level, &err);
    if (!r) return err;
    Tmp t(c, (size_t)N, &err);
    if (err) {
        fhe_ct_destroy(r);
        return err;
    }
    // pageable source: the copy is staged before the call returns
    cudaMemcpyAsync(t.p, m.data(), sizeof(int64_t) * N, cudaMemcpyHostToDevice, c->stream);
    std::vector<int> primes(level);
    for (int i = 0; i < level; i++) primes[i] = i;
    launch_rns_from_i64(c, (const int64_t *)t.p, nullptr, 1, r->d, 1, level, primes.data());
    LimbMap lm = identity_map(level, (long long)level * N, (long long)level * N, 0, 0, 0);
    launch_ntt_fwd_plain(c, r->d, r->d, lm, level);
    *out = r;
    return 0;
}

// ct (+ | - | *) plaintext given by its coefficients (kind 0 / 1 / 2); no
// level is consumed.
int op_plain_coeffs(fhe_ctx *c, const fhe_ct *a, const int64_t *coeffs, int kind, fhe_ct **out)
{
    if (kind < 0 || kind > 2 || (kind < 2 && a->npoly != 2)) return fhe_fail(c, FHE_EINVAL, "plaintext operation");
    fhe_ct *m = nullptr;
    int err = plain_ntt(c, coeffs, a->level, &m);
    if (err) return err;
    fhe_ct *r = ct_new(c, a->count, a->npoly, a->level, &err);
    if (r) {
        if (kind == 2) {
            launch_mul_poly(c, a->d, m->d, r->d, a->count * a->npoly, a->level, 0);
        } else {
            cudaMemcpyAsync(r->d, a->d, a->bytes, cudaMemcpyDeviceToDevice, c->stream);
            launch_add_plain(c, a->d, m->d, r->d, a->count, a->npoly, a->level, kind);
        }
    }
    fhe_ct_destroy(m);
    if (!r) return err;
    *out = r;
    return 0;
}

// ct (+ | - | *) plaintext slot vector (n_s values in F_p; kind 0 / 1 / 2)
int op_plain(fhe_ctx *c, const fhe_ct *a, const uint64_t *slots, int kind, fhe_ct **out)
{
    std::vector<int64_t> m(c->N);
    encode_slot_vector(c, slots, m.data());
    return op_plain_coeffs(c, a, m.data(), kind, out);
}

// ---------------------------------------------------------------------------
// comparison circuits
// ---------------------------------------------------------------------------
//
// The schedule below is the exact one of the CPU oracle (bit-exact agreement
// depends on it): products align levels by switching the higher operand down
// one prime at a time (lowered copies cached), then tensor -> relinearise ->
// modulus-switch when the level is above 1; additions align the same way.
// Powers: z^n = (z^(n/2))^2 for n a power of two, else z^(2^a) z^(n-2^a).
// Paterson-Stockmeyer on the odd part with baby powers z^1..z^(B-1),
// B = 2^ceil(log2(p-1)/2), and blocks combined pairwise; LT = c_{p-1} z^(p-1)
// + odd part; EQ = 1 - z^(p-1).  Digits are merged pairwise (2i+1 high, 2i
// low) into L = L_hi + E_hi L_lo and E = E_hi E_lo.
namespace {

// Dependency-driven streams while a plan is captured (or a batch runs with
// c->multistream).  Every circuit op is issued on one of S streams (round
// robin) after waiting for the events of its inputs, and records an event for
// its output; a capture therefore holds the circuit's true dependency graph,
// and independent products (digits, the baby powers of one wave, the leaves,
// the tree nodes of one level, other requests of a batch) run concurrently.
// Every stream first waits for an event recorded on the original stream, so
// blocks freed there earlier are idle.  Scratch freed on a stream goes to
// that stream's private free list, so no block crosses streams before the
// final join, where the original stream waits for every stream used and the
// blocks go back to the plan (capture) or to the pool (direct).
struct Dag {
    static constexpr int S = 8;
    using FreeMap = std::unordered_map<size_t, std::vector<void *>>;
    fhe_ctx *c;  // the leader: its streams and events serve every member
    bool on = false;
    cudaStream_t main = nullptr;
    // members (contexts whose batches the circuit touches; [0] = the leader),
    // each with its own free lists: scratch freed on branch k goes to
    // frees[m][k] and back to member m's pool or capture list at the join
    std::vector<fhe_ctx *> mem;
    std::vector<FreeMap *> main_free;
    std::vector<std::vector<FreeMap>> frees;
    bool used[S] = {false};
    int rr = 0, ev_next = 0, err = 0;
    std::vector<fhe_ct *> marked;
    cudaEvent_t origin = nullptr;

    explicit Dag(fhe_ctx *ctx) : c(ctx)
    {
        if (!c->capturing && !c->multistream) return;
        on = true;
        main = c->stream;
        while ((int)c->branch_streams.size() < S) {
            cudaStream_t s;
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            c->branch_streams.push_back(s);
        }
        add(c);
        origin = event();
        err = fhe_cuda_check(c, cudaEventRecord(origin, main), "dag fork");
    }
    // another context whose stream is the leader's for the circuit's span
    void add(fhe_ctx *m)
    {
        if (!on) return;
        for (fhe_ctx *x : mem)
            if (x == m) return;
        mem.push_back(m);
        main_free.push_back(m->pool.cap_free);
        frees.emplace_back(S);
    }
    cudaEvent_t event()
    {
        if (ev_next == (int)c->branch_events.size()) {
            cudaEvent_t ev;
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            c->branch_events.push_back(ev);
        }
        return c->branch_events[ev_next++];
    }
    void use(int k)
    {
        cudaStream_t s = c->branch_streams[k];
        for (size_t m = 0; m < mem.size(); m++) {
            mem[m]->stream = s;
            mem[m]->pool.stream = s;
            mem[m]->pool.cap_free = &frees[m][k];
        }
    }
    // issue the next op after its inputs
    void begin(std::initializer_list<const fhe_ct *> ins)
    {
        if (!on || err) return;
        const int k = rr;
        rr = (rr + 1) % S;
        cudaStream_t s = c->branch_streams[k];
        if (!used[k]) {
            used[k] = true;
            err = fhe_cuda_check(c, cudaStreamWaitEvent(s, origin, 0), "dag fork");
        }
        for (const fhe_ct *x : ins)
            if (x && x->ready && x->on != s) err = err ? err : fhe_cuda_check(c, cudaStreamWaitEvent(s, x->ready, 0), "dag wait");
        use(k);
    }
    void begin(const std::vector<const fhe_ct *> &ins)
    {
        if (!on || err) return;
        begin({});
        for (const fhe_ct *x : ins)
            if (x && x->ready && x->on != c->stream)
                err = err ? err : fhe_cuda_check(c, cudaStreamWaitEvent(c->stream, x->ready, 0), "dag wait");
    }
    // one event for all outputs of a merged operation
    void end_all(const std::vector<fhe_ct *> &outs)
    {
        if (!on || err || outs.empty() || !outs[0]) return;
        end(outs[0]);
        for (size_t i = 1; i < outs.size(); i++)
            if (outs[i]) {
                outs[i]->ready = outs[0]->ready;
                outs[i]->on = outs[0]->on;
                marked.push_back(outs[i]);
            }
    }
    void end(fhe_ct *out)
    {
        if (!on || err || !out) return;
        cudaEvent_t ev = event();
        err = fhe_cuda_check(c, cudaEventRecord(ev, c->stream), "dag record");
        out->ready = ev;
        out->on = c->stream;
        marked.push_back(out);
    }
    int join()
    {
        if (!on) return 0;
        for (int k = 0; k < S; k++) {
            if (!used[k]) continue;
            cudaEvent_t ev = event();
            if (!err) err = fhe_cuda_check(c, cudaEventRecord(ev, c->branch_streams[k]), "dag join");
            if (!err) err = fhe_cuda_check(c, cudaStreamWaitEvent(main, ev, 0), "dag join");
        }
        for (size_t m = 0; m < mem.size(); m++) {
            fhe_ctx *x = mem[m];
            x->stream = main;
            x->pool.stream = main;
            x->pool.cap_free = main_free[m];
            for (auto &f : frees[m])
                for (auto &kv : f) {
                    if (main_free[m]) {  // capture: the plan keeps them
                        auto &dst = (*main_free[m])[kv.first];
                        dst.insert(dst.end(), kv.second.begin(), kv.second.end());
                    } else {  // direct: back to the pool, usable on the original stream
                        auto &dst = x->pool.free_lists[kv.first];
                        dst.insert(dst.end(), kv.second.begin(), kv.second.end());
                        x->pool.in_use -= kv.first * kv.second.size();
                    }
                }
        }
        for (fhe_ct *x : marked) x->ready = nullptr, x->on = nullptr;
        on = false;
        return err;
    }
    ~Dag() { join(); }
};

struct Circuit {
    fhe_ctx *c;
    const fhe_evk *evk;
    const KeySwitchKey *rlk;
    int err = 0;
    std::vector<fhe_ct *> owned;
    std::map<std::pair<const fhe_ct *, int>, fhe_ct *> lowered;
    Dag dag;

    std::map<const fhe_ctx *, const fhe_evk *> evks;  // keys of every member context

    Circuit(fhe_ctx *ctx, const fhe_evk *e) : c(ctx), evk(e), rlk(&e->keys[0]), dag(ctx) { evks[ctx] = e; }
    // batches of another context (same device and plaintext prime; its
    // stream is the leader's while the circuit runs) take part with keys e
    void add_member(const fhe_evk *e)
    {
        evks[e->ctx] = e;
        dag.add(e->ctx);
    }
    const KeySwitchKey *rlk_of(const fhe_ctx *cx) const { return &evks.at(cx)->keys[0]; }
    ~Circuit()
    {
        finish();
        for (fhe_ct *x : owned)
            if (x) fhe_ct_destroy(x);
        for (auto &kv : lowered) fhe_ct_destroy(kv.second);
    }
    // joins the captured streams (before anything is freed or returned)
    void finish()
    {
        const int e2 = dag.join();
        if (!err) err = e2;
    }
    fhe_ct *keep(fhe_ct *x)
    {
        owned.push_back(x);
        return x;
    }
    // remove x from the owned set so the caller receives it
    fhe_ct *release(fhe_ct *x)
    {
        for (auto &o : owned)
            if (o == x) o = nullptr;
        return x;
    }
    // x at `level`: from the nearest cached copy above it, all remaining
    // primes dropped in one step (op_modswitch_k: the residues of dropping
    // them one at a time)
    const fhe_ct *lower(const fhe_ct *x, int level)
    {
        if (err || !x) return nullptr;
        if (x->level == level) return x;
        auto key = std::make_pair(x, level);
        auto it = lowered.find(key);
        if (it != lowered.end()) return it->second;
        const fhe_ct *from = x;
        for (int lv = level + 1; lv < x->level; lv++) {
            auto f = lowered.find(std::make_pair(x, lv));
            if (f != lowered.end()) {
                from = f->second;
                break;
            }
        }
        if (from->level - level > FHE_MAXK) from = lower(x, level + FHE_MAXK);
        if (!from) return nullptr;
        fhe_ct *r = nullptr;
        dag.begin({from});
        if ((err = op_modswitch_k(c, from, from->level - level, &r))) return nullptr;
        dag.end(r);
        lowered[key] = r;
        return r;
    }
    fhe_ct *mul(const fhe_ct *a, const fhe_ct *b)
    {
        FHE_RANGE("circuit mul");
        if (err || !a || !b) return nullptr;
        const int lv = std::min(a->level, b->level);
        const fhe_ct *a2 = lower(a, lv), *b2 = lower(b, lv);
        if (!a2 || !b2) return nullptr;
        fhe_ct *r = nullptr;
        dag.begin({a2, b2});
        if ((err = op_mul_relin(c, *rlk, a2, b2, &r))) return nullptr;
        dag.end(r);
        trace(c, FHE_OP_MUL, lv);
        return keep(r);
    }
    fhe_ct *addsub(const fhe_ct *a, const fhe_ct *b, int sub)
    {
        if (err || !a || !b) return nullptr;
        const int lv = std::min(a->level, b->level);
        const fhe_ct *a2 = lower(a, lv), *b2 = lower(b, lv);
        if (!a2 || !b2) return nullptr;
        fhe_ct *r = nullptr;
        dag.begin({a2, b2});
        if ((err = op_addsub(c, a2, b2, sub, &r))) return nullptr;
        dag.end(r);
        trace(c, sub ? FHE_OP_SUB : FHE_OP_ADD, lv);
        return keep(r);
    }
    fhe_ct *add(const fhe_ct *a, const fhe_ct *b) { return addsub(a, b, 0); }
    fhe_ct *sub(const fhe_ct *a, const fhe_ct *b) { return addsub(a, b, 1); }
    fhe_ct *cmul(const fhe_ct *a, int64_t k)
    {
        if (err || !a) return nullptr;
        fhe_ct *r = nullptr;
        dag.begin({a});
        if ((err = op_mul_const(c, a, k, &r))) return nullptr;
        dag.end(r);
        trace(c, FHE_OP_CMUL, a->level);
        return keep(r);
    }
    fhe_ct *cadd(const fhe_ct *a, int64_t k)
    {
        if (err || !a) return nullptr;
        fhe_ct *r = nullptr;
        dag.begin({a});
        if ((err = op_add_const(c, a, k, &r))) return nullptr;
        dag.end(r);
        trace(c, FHE_OP_CADD, a->level);
        return keep(r);
    }
    fhe_ct *neg(const fhe_ct *a)
    {
        if (err || !a) return nullptr;
        fhe_ct *r = nullptr;
        dag.begin({a});
        if ((err = op_neg(c, a, &r))) return nullptr;
        dag.end(r);
        trace(c, FHE_OP_NEG, a->level);
        return keep(r);
    }

    fhe_ct *rot(const fhe_ct *a, int64_t g)
    {
        FHE_RANGE("circuit rot");
        if (err || !a) return nullptr;
        const KeySwitchKey *key = evk->find(g);
        if (!key) {
            err = fhe_fail(c, FHE_ENOKEY, "no rotation key for this Galois element");
            return nullptr;
        }
        fhe_ct *r = nullptr;
        dag.begin({a});
        if ((err = op_rotate(c, *key, a, &r))) return nullptr;
        dag.end(r);
        trace(c, FHE_OP_ROT, a->level);
        return keep(r);
    }
    fhe_ct *plain_coeffs(const fhe_ct *a, const std::vector<int64_t> &m)
    {
        if (err || !a) return nullptr;
        fhe_ct *r = nullptr;
        dag.begin({a});
        if ((err = op_plain_coeffs(c, a, m.data(), 2, &r))) return nullptr;
        dag.end(r);
        trace(c, FHE_OP_PMUL, a->level);
        return keep(r);
    }
    fhe_ct *plain(const fhe_ct *a, const std::vector<uint64_t> &slots, int kind)
    {
        if (err || !a) return nullptr;
        fhe_ct *r = nullptr;
        dag.begin({a});
        if ((err = op_plain(c, a, slots.data(), kind, &r))) return nullptr;
        dag.end(r);
        trace(c, kind == 0 ? FHE_OP_PADD : kind == 1 ? FHE_OP_PSUB : FHE_OP_PMUL, a->level);
        return keep(r);
    }

    // sum_i c_i lower(x_i, lv): one fused kernel for the scalar products and
    // additions; the trace records them as the individual operations
    // (cmul, cmul, add, cmul, add, ...).
    // sum_i c_i x_i at level lv (the scalar products and additions of the
    // schedule, traced as such): chunks of up to 8 terms with one reduction
    // each, the chunks added in order
    fhe_ct *lincomb(const std::vector<fhe_ct *> &xs, const std::vector<std::pair<int, int>> &terms, int lv)
    {
        if (err) return nullptr;
        const int n = (int)xs.size();
        std::vector<const fhe_ct *> low(n);
        std::vector<int64_t> k(n);
        for (int i = 0; i < n; i++) {
            low[i] = lower(xs[i], lv);
            if (!low[i]) return nullptr;
            k[i] = terms[i].second;
        }
        fhe_ct *r = nullptr;
        dag.begin({});
        for (int i = 0; i < n && !dag.err; i++)  // inputs of any arity
            if (low[i]->ready && low[i]->on != c->stream)
                dag.err = fhe_cuda_check(c, cudaStreamWaitEvent(c->stream, low[i]->ready, 0), "dag wait");
        for (int i0 = 0; i0 < n && !err; i0 += 8) {
            fhe_ct *part = nullptr;
            if ((err = op_lincomb(c, low.data() + i0, k.data() + i0, std::min(8, n - i0), &part))) return nullptr;
            if (!r) {
                r = part;
                continue;
            }
            fhe_ct *sum = nullptr;
            err = op_addsub(c, r, part, 0, &sum);
            fhe_ct_destroy(r);
            fhe_ct_destroy(part);
            if (err) return nullptr;
            r = sum;
        }
        dag.end(r);
        for (int i = 0; i < n; i++) {
            trace(c, FHE_OP_CMUL, lv);
            if (i) trace(c, FHE_OP_ADD, lv);
        }
        return keep(r);
    }

    // ---- merged operations: every item of one call runs in the same
    // launches (one per step), traced item by item as the single forms are

    // x lowered to each requested level.  Per source, the targets run in
    // descending order, each from the nearest copy above it (cached, made
    // earlier in the chain, or the source; at most FHE_MAXK primes a step);
    // step r of every chain is one merged switch.  Multi-prime switches give
    // the residues of single ones, so every path yields the same bits.
    std::vector<const fhe_ct *> lower_many(const std::vector<std::pair<const fhe_ct *, int>> &req)
    {
        std::vector<const fhe_ct *> res(req.size(), nullptr);
        if (err) return res;
        std::map<const fhe_ct *, std::set<int, std::greater<int>>> want;
        for (auto &r : req) {
            if (!r.first) return res;
            if (r.second < 1 || r.second > r.first->level) {
                err = fhe_fail(c, FHE_ELEVEL, "bad target level");
                return res;
            }
            if (r.second < r.first->level && !lowered.count(r)) want[r.first].insert(r.second);
        }
        struct Step {
            const fhe_ct *x;
            int from, to;
        };
        std::vector<std::vector<Step>> chains;
        for (auto &kv : want) {
            const fhe_ct *x = kv.first;
            std::set<int> have;
            std::vector<Step> ch;
            for (int t : kv.second) {
                int from = x->level;
                for (int lv = t + 1; lv < x->level; lv++)
                    if (have.count(lv) || lowered.count({x, lv})) {
                        from = lv;
                        break;
                    }
                while (from - t > FHE_MAXK) {
                    ch.push_back({x, from, from - FHE_MAXK});
                    from -= FHE_MAXK;
                    have.insert(from);
                }
                ch.push_back({x, from, t});
                have.insert(t);
            }
            chains.push_back(ch);
        }
        for (size_t r = 0; !err; r++) {
            std::vector<SwitchItem> items;
            std::vector<std::pair<const fhe_ct *, int>> keys;
            std::vector<const fhe_ct *> ins;
            for (auto &ch : chains)
                if (r < ch.size()) {
                    const Step &st = ch[r];
                    const fhe_ct *src = st.from == st.x->level ? st.x : lowered.at({st.x, st.from});
                    items.push_back(SwitchItem{src->ctx, src, st.from - st.to, nullptr});
                    keys.push_back({st.x, st.to});
                    ins.push_back(src);
                }
            if (items.empty()) break;
            dag.begin(ins);
            if ((err = op_modswitch_many(items))) return res;
            std::vector<fhe_ct *> outs;
            for (size_t i = 0; i < items.size(); i++) {
                lowered[keys[i]] = items[i].out;
                outs.push_back(items[i].out);
            }
            dag.end_all(outs);
        }
        for (size_t i = 0; i < req.size(); i++)
            res[i] = req[i].second == req[i].first->level ? req[i].first : lowered.at(req[i]);
        return res;
    }

    std::vector<fhe_ct *> mul_many(const std::vector<std::pair<const fhe_ct *, const fhe_ct *>> &pr)
    {
        FHE_RANGE("circuit mul");
        std::vector<fhe_ct *> out(pr.size(), nullptr);
        if (err || pr.empty()) return out;
        std::vector<std::pair<const fhe_ct *, int>> req;
        for (auto &q : pr) {
            if (!q.first || !q.second) return out;
            const int lv = std::min(q.first->level, q.second->level);
            req.push_back({q.first, lv});
            req.push_back({q.second, lv});
        }
        std::vector<const fhe_ct *> low = lower_many(req);
        if (err) return out;
        // the wave in `parts` merged operations (items dealt round robin),
        // each on a stream of its own under the scheduler, so that one
        // part's streaming steps overlap another's transforms
        const int parts = dag.on ? std::max(1, std::min((int)pr.size(), c->wave_split)) : 1;
        for (int part = 0; part < parts && !err; part++) {
            std::vector<MulItem> items;
            std::vector<size_t> at;
            std::vector<const fhe_ct *> ins;
            for (size_t i = part; i < pr.size(); i += parts) {
                fhe_ctx *cx = low[2 * i]->ctx;
                items.push_back(MulItem{cx, rlk_of(cx), low[2 * i], low[2 * i + 1], nullptr});
                at.push_back(i);
                ins.push_back(low[2 * i]);
                ins.push_back(low[2 * i + 1]);
            }
            dag.begin(ins);
            if ((err = op_mul_relin_many(items))) return out;
            std::vector<fhe_ct *> po;
            for (size_t j = 0; j < at.size(); j++) po.push_back(out[at[j]] = items[j].out);
            dag.end_all(po);
        }
        for (size_t i = 0; i < pr.size() && !err; i++) {
            trace(low[2 * i]->ctx, FHE_OP_MUL, low[2 * i]->level);
            keep(out[i]);
        }
        return out;
    }

    // element-wise items; add / sub / lincomb operands aligned to their
    // lowest level (lincomb: to lv when lv > 0)
    std::vector<fhe_ct *> ew_many(std::vector<EwItem> items, const std::vector<int> &lv = {})
    {
        std::vector<fhe_ct *> out(items.size(), nullptr);
        if (err || items.empty()) return out;
        std::vector<std::pair<const fhe_ct *, int>> req;
        for (size_t i = 0; i < items.size(); i++) {
            const EwItem &e = items[i];
            int l = 1 << 30;
            for (int j = 0; j < e.n; j++) {
                if (!e.x[j]) return out;
                l = std::min(l, e.x[j]->level);
            }
            if (!lv.empty() && lv[i] > 0) l = lv[i];
            for (int j = 0; j < e.n; j++) req.push_back({e.x[j], l});
        }
        std::vector<const fhe_ct *> low = lower_many(req);
        if (err) return out;
        size_t q = 0;
        for (EwItem &e : items)
            for (int j = 0; j < e.n; j++) e.x[j] = low[q++];
        dag.begin(low);
        if ((err = op_ew_many(items))) return out;
        for (size_t i = 0; i < items.size(); i++) out[i] = items[i].out;
        dag.end_all(out);
        for (size_t i = 0; i < items.size(); i++) {
            const EwItem &e = items[i];
            const int l = e.x[0]->level;
            switch (e.op) {
            case FHE_EW_ADD: trace(e.c, FHE_OP_ADD, l); break;
            case FHE_EW_SUB: trace(e.c, FHE_OP_SUB, l); break;
            case FHE_EW_NEG: trace(e.c, FHE_OP_NEG, l); break;
            case FHE_EW_CMUL: trace(e.c, FHE_OP_CMUL, l); break;
            case FHE_EW_CADD: trace(e.c, FHE_OP_CADD, l); break;
            default:
                for (int j = 0; j < e.n; j++) {
                    trace(e.c, FHE_OP_CMUL, l);
                    if (j) trace(e.c, FHE_OP_ADD, l);
                }
            }
            keep(out[i]);
        }
        return out;
    }

    static EwItem ew(int op, std::initializer_list<const fhe_ct *> xs, std::initializer_list<int64_t> ks = {})
    {
        EwItem e;
        memset(&e, 0, sizeof(e));
        e.op = op;
        for (const fhe_ct *x : xs) e.x[e.n++] = x;
        int j = 0;
        for (int64_t k : ks) e.k[j++] = k;
        e.c = e.x[0] ? e.x[0]->ctx : nullptr;
        return e;
    }

    // (LT_k, EQ_k) of every digit pair k < d at once.  The schedule (the
    // oracle's): z = x - y; powers z^n = (z^(n/2))^2 for n a power of two,
    // else z^(2^a) z^(n-2^a); Paterson-Stockmeyer on the odd part with baby
    // powers z^1..z^(B-1), B = 2^ceil(log2(p-1)/2): leaves L_k = sum_r
    // c_(Bk+r) z^r at the level of their lowest power, blocks combined
    // pairwise as lo + z^(B 2^(t-1)) hi; LT = c_(p-1) z^(p-1) + odd part;
    // EQ = 1 - z^(p-1).  It runs wave by wave across digits (powers by depth,
    // the leaves, each level of the block tree, the leading term), every
    // wave one merged operation over all its products and digits; the
    // operations and their levels are those of evaluating it digit by digit.
    void digits(const fhe_ct *const *xs, const fhe_ct *const *ys, int d, bool want_lt, bool want_eq,
                std::vector<fhe_ct *> &lt, std::vector<fhe_ct *> &eq)
    {
        const int p = (int)c->p;
        lt.assign(d, nullptr);
        eq.assign(d, nullptr);
        std::vector<EwItem> zs;
        for (int k = 0; k < d; k++) zs.push_back(ew(FHE_EW_SUB, {xs[k], ys[k]}));
        std::vector<fhe_ct *> z = ew_many(zs);
        if (err) return;
        const std::vector<int> &cf = c->lt;
        int lg = 0;
        while ((1 << lg) < p - 1) lg++;  // ceil(log2(p-1))
        const int B = 1 << ((lg + 1) / 2);
        const int nblocks = (p - 2) / B + 1;
        int T = 0;
        while ((1 << T) < nblocks) T++;
        // leaf terms and which tree nodes are empty
        std::vector<std::vector<std::pair<int, int>>> terms(nblocks);
        for (int k = 0; k < nblocks; k++)
            for (int r = 1; r < B; r += 2)
                if (B * k + r <= p - 2 && cf[B * k + r]) terms[k].push_back({r, cf[B * k + r]});
        auto nonempty = [&](int k0, int t) {  // tree(k0, t) of digit() is not null
            for (int k = k0; k < std::min(nblocks, k0 + (1 << t)); k++)
                if (!terms[k].empty()) return true;
            return false;
        };
        // exponents the schedule needs, with the power rule's operands
        std::set<int> need;
        std::function<void(int)> add_exp = [&](int n) {
            if (need.count(n)) return;
            need.insert(n);
            if (n == 1) return;
            if ((n & (n - 1)) == 0) {
                add_exp(n / 2);
            } else {
                int a = 1;
                while (a * 2 < n) a *= 2;
                add_exp(a);
                add_exp(n - a);
            }
        };
        if (want_lt) {
            for (auto &tk : terms)
                for (auto &tm : tk) add_exp(tm.first);
            for (int t = 1; t <= T; t++)
                for (int k0 = 0; k0 < nblocks; k0 += 1 << t)
                    if (k0 + (1 << (t - 1)) < nblocks && nonempty(k0 + (1 << (t - 1)), t - 1))
                        add_exp(B * (1 << (t - 1)));
        }
        add_exp(p - 1);
        std::map<int, std::vector<fhe_ct *>> pw;
        pw[1] = z;
        auto depth = [](int n) {
            int r = 0;
            while ((1 << r) < n) r++;
            return r;
        };
        int maxd = 0;
        for (int n : need) maxd = std::max(maxd, depth(n));
        for (int dd = 1; dd <= maxd && !err; dd++) {
            std::vector<int> ex;
            std::vector<std::pair<const fhe_ct *, const fhe_ct *>> pr;
            for (int n : need) {
                if (n == 1 || depth(n) != dd) continue;
                int a, b;
                if ((n & (n - 1)) == 0) {
                    a = b = n / 2;
                } else {
                    a = 1;
                    while (a * 2 < n) a *= 2;
                    b = n - a;
                }
                ex.push_back(n);
                for (int k = 0; k < d; k++) pr.push_back({pw.at(a)[k], pw.at(b)[k]});
            }
            std::vector<fhe_ct *> r = mul_many(pr);
            for (size_t i = 0; i < ex.size(); i++) pw[ex[i]] = std::vector<fhe_ct *>(r.begin() + i * d, r.begin() + (i + 1) * d);
        }
        if (err) return;
        if (want_lt) {
            // leaves L_k = sum_r c_{Bk+r} z^r at the level of their lowest power
            // (chunks of at most 8 terms, one reduction each, the chunks
            // then added in order: the traced operations are the terms'
            // scalar products and additions either way)
            std::map<std::pair<int, int>, std::vector<fhe_ct *>> node;  // (k0, t) -> per digit
            std::vector<EwItem> li;
            std::vector<int> llv;
            std::vector<std::pair<int, int>> lkd;  // (block, digit) of each chunk
            for (int k = 0; k < nblocks; k++) {
                if (terms[k].empty()) continue;
                for (int dg = 0; dg < d; dg++) {
                    int lv = 1 << 30;
                    for (auto &tm : terms[k]) lv = std::min(lv, pw.at(tm.first)[dg]->level);
                    for (size_t t0 = 0; t0 < terms[k].size(); t0 += 8) {
                        EwItem e = ew(FHE_EW_LINCOMB, {});
                        for (size_t t = t0; t < std::min(terms[k].size(), t0 + 8); t++) {
                            e.x[e.n] = pw.at(terms[k][t].first)[dg];
                            e.k[e.n++] = terms[k][t].second;
                        }
                        e.c = e.x[0]->ctx;
                        li.push_back(e);
                        llv.push_back(lv);
                        lkd.push_back({k, dg});
                    }
                }
            }
            std::vector<fhe_ct *> lr = ew_many(li, llv);
            if (err) return;
            std::map<std::pair<int, int>, std::vector<fhe_ct *>> parts;
            for (size_t i = 0; i < lkd.size(); i++) parts[lkd[i]].push_back(lr[i]);
            for (;;) {  // chunk sums, first two at a time, for every leaf at once
                std::vector<EwItem> ad;
                std::vector<std::pair<int, int>> who;
                for (auto &kv : parts)
                    if (kv.second.size() > 1) {
                        ad.push_back(ew(FHE_EW_ADD, {kv.second[0], kv.second[1]}));
                        who.push_back(kv.first);
                    }
                if (ad.empty()) break;
                std::vector<fhe_ct *> sm = ew_many(ad);
                if (err) return;
                for (size_t i = 0; i < who.size(); i++) {
                    auto &v = parts[who[i]];
                    v.erase(v.begin(), v.begin() + 2);
                    v.insert(v.begin(), sm[i]);
                }
            }
            for (auto &kv : parts) {
                auto &v = node[{kv.first.first, 0}];
                v.resize(d, nullptr);
                v[kv.first.second] = kv.second[0];
            }
            // the block tree, one level at a time: node(k0, t) = lo + z^(B half) hi
            for (int t = 1; t <= T && !err; t++) {
                const int half = 1 << (t - 1);
                std::vector<std::pair<const fhe_ct *, const fhe_ct *>> pr;
                std::vector<int> pk;
                for (int k0 = 0; k0 < nblocks; k0 += 1 << t) {
                    auto hi = node.find({k0 + half, t - 1});
                    if (hi == node.end()) {
                        auto lo = node.find({k0, t - 1});
                        if (lo != node.end()) node[{k0, t}] = lo->second;
                        continue;
                    }
                    for (int dg = 0; dg < d; dg++) pr.push_back({pw.at(B * half)[dg], hi->second[dg]});
                    pk.push_back(k0);
                }
                std::vector<fhe_ct *> prod = mul_many(pr);
                if (err) return;
                std::vector<EwItem> ad;
                std::vector<int> ak;
                for (size_t i = 0; i < pk.size(); i++) {
                    const int k0 = pk[i];
                    std::vector<fhe_ct *> pv(prod.begin() + i * d, prod.begin() + (i + 1) * d);
                    auto lo = node.find({k0, t - 1});
                    if (lo == node.end()) {
                        node[{k0, t}] = pv;
                        continue;
                    }
                    for (int dg = 0; dg < d; dg++) ad.push_back(ew(FHE_EW_ADD, {lo->second[dg], pv[dg]}));
                    ak.push_back(k0);
                }
                std::vector<fhe_ct *> sums = ew_many(ad);
                if (err) return;
                for (size_t i = 0; i < ak.size(); i++)
                    node[{ak[i], t}] = std::vector<fhe_ct *>(sums.begin() + i * d, sums.begin() + (i + 1) * d);
            }
            // LT_k = c_{p-1} z^(p-1) + odd part
            std::vector<EwItem> ld;
            for (int dg = 0; dg < d; dg++) ld.push_back(ew(FHE_EW_CMUL, {pw.at(p - 1)[dg]}, {cf[p - 1]}));
            std::vector<fhe_ct *> lead = ew_many(ld);
            if (err) return;
            auto odd = node.find({0, T});
            if (odd == node.end()) {
                lt = lead;
            } else {
                std::vector<EwItem> ad;
                for (int dg = 0; dg < d; dg++) ad.push_back(ew(FHE_EW_ADD, {lead[dg], odd->second[dg]}));
                lt = ew_many(ad);
            }
        }
        if (want_eq && !err) {
            // EQ_k = 1 - z^(p-1)
            std::vector<EwItem> ng, ca;
            for (int dg = 0; dg < d; dg++) ng.push_back(ew(FHE_EW_NEG, {pw.at(p - 1)[dg]}));
            std::vector<fhe_ct *> n = ew_many(ng);
            if (err) return;
            for (int dg = 0; dg < d; dg++) ca.push_back(ew(FHE_EW_CADD, {n[dg]}, {1}));
            eq = ew_many(ca);
        }
    }

    // (LT_k, EQ_k) of one pair of full digits in [0, p): the bivariate LT
    // polynomial sum_a x^a h_a(y), h_a = sum_{b>=1} c[a][b] y^b (no constant
    // terms), rows in order of a, powers computed when first needed; EQ_k =
    // 1 - (x - y)^(p-1).  The schedule of the oracle's bivariate circuit.
    void digit_bv(const fhe_ct *x, const fhe_ct *y, bool want_lt, bool want_eq, fhe_ct **lt_out, fhe_ct **eq_out)
    {
        const int p = (int)c->p;
        *lt_out = *eq_out = nullptr;
        using Powers = std::map<int, const fhe_ct *>;
        std::function<const fhe_ct *(Powers &, int)> power = [&](Powers &pw, int n) -> const fhe_ct * {
            auto it = pw.find(n);
            if (it != pw.end()) return it->second;
            const fhe_ct *r;
            if ((n & (n - 1)) == 0) {
                const fhe_ct *h = power(pw, n / 2);
                r = mul(h, h);
            } else {
                int a = 1;
                while (a * 2 < n) a *= 2;
                const fhe_ct *A = power(pw, a);
                const fhe_ct *Bp = power(pw, n - a);
                r = mul(A, Bp);
            }
            pw[n] = r;
            return r;
        };
        if (want_lt) {
            if (c->ltbv.empty()) lt_bivariate_coefficients(p, c->ltbv);
            const std::vector<int> &cf = c->ltbv;
            Powers px, py;
            px[1] = x;
            py[1] = y;
            fhe_ct *acc = nullptr;
            for (int a = 0; a < p && !err; a++) {
                std::vector<std::pair<int, int>> terms;
                for (int b = 1; b < p; b++)
                    if (cf[(size_t)a * p + b]) terms.push_back({b, cf[(size_t)a * p + b]});
                if (terms.empty()) continue;
                std::vector<fhe_ct *> cts;
                for (auto &t : terms) cts.push_back(const_cast<fhe_ct *>(power(py, t.first)));
                if (err) return;
                int lv = 1 << 30;
                for (auto *t : cts) lv = std::min(lv, t->level);
                fhe_ct *h = lincomb(cts, terms, lv);
                fhe_ct *term = h;
                if (a > 0) {
                    const fhe_ct *xa = power(px, a);
                    term = mul(xa, h);
                }
                acc = acc ? add(acc, term) : term;
            }
            *lt_out = acc;
        }
        if (want_eq) {
            Powers pz;
            pz[1] = sub(x, y);
            if (!pz[1]) return;
            *eq_out = cadd(neg(power(pz, p - 1)), 1);
        }
    }

    // Several comparisons (and max/min selections) at once: the digit
    // polynomials of all of them in one digits() call per kind, the merge
    // trees level by level and the selections as merged operations.  Each
    // result equals the comparison run alone.
    struct Req {
        const fhe_ct *const *x;
        const fhe_ct *const *y;
        int d;
        bool want_lt, want_eq, maxmin;
        fhe_ct **lt, **eq;  // comparison outputs (either may be null)
        fhe_ct **mx, **mn;  // max / min digits (maxmin; either may be null)
    };
    void compare_many(std::vector<Req> &rq)
    {
        if (err || rq.empty()) return;
        // digit results (L_k, E_k) of every request; requests of one kind
        // (what the digit circuit must produce) share one digits() call
        std::vector<std::vector<std::pair<fhe_ct *, fhe_ct *>>> nodes(rq.size());
        for (int kind = 0; kind < 4 && !err; kind++) {
            const bool wl = kind & 1, we = kind & 2;
            std::vector<const fhe_ct *> X, Y;
            std::vector<size_t> who;
            for (size_t i = 0; i < rq.size(); i++) {
                const Req &r = rq[i];
                const bool rl = r.want_lt || r.maxmin, re = r.d > 1 || (r.want_eq && !r.maxmin);
                if (rl != wl || re != we) continue;
                for (int k = 0; k < r.d; k++) X.push_back(r.x[k]), Y.push_back(r.y[k]);
                who.push_back(i);
            }
            if (who.empty()) continue;
            std::vector<fhe_ct *> L, E;
            digits(X.data(), Y.data(), (int)X.size(), wl, we, L, E);
            size_t q = 0;
            for (size_t i : who)
                for (int k = 0; k < rq[i].d; k++, q++) nodes[i].push_back({L[q], E[q]});
        }
        if (err) return;
        // merge trees, one level of every request at a time: pairs (2i+1
        // high, 2i low) -> (L_hi + E_hi L_lo, E_hi E_lo); the root skips the
        // E product unless EQ is wanted; an odd last node passes up
        for (;;) {
            std::vector<std::pair<const fhe_ct *, const fhe_ct *>> pr;
            struct Slot {
                size_t req, pair;
                int mi, ei;  // indices into pr (-1: none)
            };
            std::vector<Slot> slots;
            for (size_t i = 0; i < rq.size(); i++) {
                auto &nd = nodes[i];
                if (nd.size() < 2) continue;
                const bool root = nd.size() == 2, wl = rq[i].want_lt || rq[i].maxmin;
                const bool we = rq[i].want_eq && !rq[i].maxmin;
                for (size_t j = 0; j < nd.size() / 2; j++) {
                    auto lo = nd[2 * j], hi = nd[2 * j + 1];
                    Slot sl{i, j, -1, -1};
                    if (wl) sl.mi = (int)pr.size(), pr.push_back({hi.second, lo.first});
                    if (we || !root) sl.ei = (int)pr.size(), pr.push_back({hi.second, lo.second});
                    slots.push_back(sl);
                }
            }
            if (slots.empty()) break;
            std::vector<fhe_ct *> prod = mul_many(pr);
            if (err) return;
            std::vector<EwItem> ad;
            std::vector<size_t> ai;
            for (size_t s = 0; s < slots.size(); s++)
                if (slots[s].mi >= 0) {
                    auto hi = nodes[slots[s].req][2 * slots[s].pair + 1];
                    ad.push_back(ew(FHE_EW_ADD, {hi.first, prod[slots[s].mi]}));
                    ai.push_back(s);
                }
            std::vector<fhe_ct *> sums = ew_many(ad);
            if (err) return;
            std::vector<fhe_ct *> Ls(slots.size(), nullptr);
            for (size_t a = 0; a < ai.size(); a++) Ls[ai[a]] = sums[a];
            std::vector<std::vector<std::pair<fhe_ct *, fhe_ct *>>> nxt(rq.size());
            for (size_t s = 0; s < slots.size(); s++)
                nxt[slots[s].req].push_back({Ls[s], slots[s].ei >= 0 ? prod[slots[s].ei] : nullptr});
            for (size_t i = 0; i < rq.size(); i++) {
                if (nodes[i].size() < 2) continue;
                if (nodes[i].size() % 2) nxt[i].push_back(nodes[i].back());
                nodes[i] = nxt[i];
            }
        }
        // comparison outputs
        for (size_t i = 0; i < rq.size(); i++) {
            const Req &r = rq[i];
            if (r.maxmin) continue;
            if (r.lt) *r.lt = r.want_lt ? release(nodes[i][0].first) : nullptr;
            if (r.eq) *r.eq = r.want_eq ? release(nodes[i][0].second) : nullptr;
        }
        // selections: t_k = L (y_k - x_k), max_k = x_k + t_k, min_k = y_k - t_k
        std::vector<EwItem> df;
        std::vector<std::pair<size_t, int>> at;
        for (size_t i = 0; i < rq.size(); i++)
            if (rq[i].maxmin)
                for (int k = 0; k < rq[i].d; k++) {
                    df.push_back(ew(FHE_EW_SUB, {rq[i].y[k], rq[i].x[k]}));
                    at.push_back({i, k});
                }
        if (df.empty()) return;
        std::vector<fhe_ct *> diff = ew_many(df);
        if (err) return;
        std::vector<std::pair<const fhe_ct *, const fhe_ct *>> pr;
        for (size_t a = 0; a < at.size(); a++) pr.push_back({nodes[at[a].first][0].first, diff[a]});
        std::vector<fhe_ct *> t = mul_many(pr);
        if (err) return;
        std::vector<EwItem> sel;
        for (size_t a = 0; a < at.size(); a++) {
            const Req &r = rq[at[a].first];
            const int k = at[a].second;
            sel.push_back(ew(FHE_EW_ADD, {r.x[k], t[a]}));
            sel.push_back(ew(FHE_EW_SUB, {r.y[k], t[a]}));
        }
        std::vector<fhe_ct *> mm = ew_many(sel);
        if (err) return;
        for (size_t a = 0; a < at.size(); a++) {
            const Req &r = rq[at[a].first];
            const int k = at[a].second;
            if (r.mx) r.mx[k] = release(mm[2 * a]);
            if (r.mn) r.mn[k] = release(mm[2 * a + 1]);
        }
    }

    void compare(const fhe_ct *const *xs, const fhe_ct *const *ys, int d, bool want_lt, bool want_eq,
                 fhe_ct **lt, fhe_ct **eq, bool bivariate = false)
    {
        if (!bivariate) {
            std::vector<Req> rq{Req{xs, ys, d, want_lt, want_eq, false, lt, eq, nullptr, nullptr}};
            compare_many(rq);
            return;
        }
        std::vector<std::pair<fhe_ct *, fhe_ct *>> nodes(d, {nullptr, nullptr});
        for (int k = 0; k < d && !err; k++)
            digit_bv(xs[k], ys[k], want_lt, d > 1 || want_eq, &nodes[k].first, &nodes[k].second);
        while (nodes.size() > 1 && !err) {
            const bool root = nodes.size() == 2;
            std::vector<std::pair<fhe_ct *, fhe_ct *>> nxt;
            for (size_t i = 0; i < nodes.size() / 2; i++) {
                auto lo = nodes[2 * i], hi = nodes[2 * i + 1];
                fhe_ct *L = nullptr, *E = nullptr;
                if (want_lt) {
                    fhe_ct *m = mul(hi.second, lo.first);
                    L = add(hi.first, m);
                }
                if (want_eq || !root) E = mul(hi.second, lo.second);
                nxt.push_back({L, E});
            }
            if (nodes.size() % 2) nxt.push_back(nodes.back());
            nodes = nxt;
        }
        if (err) return;
        if (lt) *lt = want_lt ? release(nodes[0].first) : nullptr;
        if (eq) *eq = want_eq ? release(nodes[0].second) : nullptr;
    }
};

}  // namespace

// max / min digits of one pair of operands inside an open circuit
static int circuit_max_min_in(Circuit &C, const fhe_ct *const *x, const fhe_ct *const *y, int d, fhe_ct **mx,
                              fhe_ct **mn)
{
    std::vector<Circuit::Req> rq{Circuit::Req{x, y, d, true, false, true, nullptr, nullptr, mx, mn}};
    C.compare_many(rq);
    return C.err;
}

// Several independent comparisons and selections in one circuit: their
// digit polynomials, merge trees and selections run as merged operations.
int circuit_multi(fhe_ctx *c, const fhe_evk *evk, const std::vector<MultiItem> &items)
{
    Circuit C(c, evk);
    std::vector<Circuit::Req> rq;
    for (const MultiItem &it : items) {
        if (it.maxmin)
            rq.push_back(Circuit::Req{it.x, it.y, it.d, true, false, true, nullptr, nullptr, it.out0, it.out1});
        else
            rq.push_back(Circuit::Req{it.x, it.y, it.d, it.out0 != nullptr, it.out1 != nullptr, false, it.out0,
                                      it.out1, nullptr, nullptr});
    }
    C.compare_many(rq);
    C.finish();
    return C.err;
}

// The same over several contexts of one device and plaintext prime (one
// circuit: every merged step is one launch across their ring degrees and
// levels).  Item i uses keys evks[i]; evks[0]'s context leads.  The caller
// holds every context's lock and has pointed every context's stream (and
// pool stream) at the leader's for the call.
int circuit_multi_ctx(const std::vector<const fhe_evk *> &evks, const std::vector<MultiItem> &items)
{
    if (evks.empty() || evks.size() != items.size()) return FHE_EINVAL;
    fhe_ctx *lead = evks[0]->ctx;
    for (const fhe_evk *e : evks)
        if (e->ctx->p != lead->p || e->ctx->device != lead->device)
            return fhe_fail(lead, FHE_EMISMATCH, "fused contexts differ in plaintext prime or device");
    Circuit C(lead, evks[0]);
    for (const fhe_evk *e : evks) C.add_member(e);
    std::vector<Circuit::Req> rq;
    for (const MultiItem &it : items) {
        if (it.maxmin)
            rq.push_back(Circuit::Req{it.x, it.y, it.d, true, false, true, nullptr, nullptr, it.out0, it.out1});
        else
            rq.push_back(Circuit::Req{it.x, it.y, it.d, it.out0 != nullptr, it.out1 != nullptr, false, it.out0,
                                      it.out1, nullptr, nullptr});
    }
    C.compare_many(rq);
    C.finish();
    return C.err;
}

int circuit_compare_bv(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                       fhe_ct **lt, fhe_ct **eq)
{
    Circuit C(c, evk);
    C.compare(x, y, d, lt != nullptr, eq != nullptr, lt, eq, true);
    C.finish();
    return C.err;
}

int circuit_compare(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                    fhe_ct **lt, fhe_ct **eq)
{
    Circuit C(c, evk);
    C.compare(x, y, d, lt != nullptr, eq != nullptr, lt, eq);
    C.finish();
    return C.err;
}

int circuit_max_min(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                    fhe_ct **mx, fhe_ct **mn)
{
    Circuit C(c, evk);
    circuit_max_min_in(C, x, y, d, mx, mn);
    C.finish();
    return C.err;
}

// ---------------------------------------------------------------------------
// tournament max / min
// ---------------------------------------------------------------------------
//
// Same schedule as the CPU oracle: cross rounds pair ciphertexts [0, h) with
// [h, 2h) of the batch (h = n / 2, an odd last one passes on after the
// winners), then in-slot rounds x <- sel(x, rotate(x, g)) with
// g = 5^(2^i) mod 2N for 2^i = cols/2 .. 1 and finally g = 2N - 1.  The first
// cross round computes max and min from one LT; afterwards the two
// tournaments run separately.  A round that would end below level 1 is
// preceded by a refresh of the batch (a stand-in for bootstrapping).

int op_slice(fhe_ctx *c, const fhe_ct *a, int start, int n, fhe_ct **out)
{
    if (start < 0 || n < 1 || start + n > a->count) return fhe_fail(c, FHE_EINVAL, "slice out of range");
    int err = 0;
    fhe_ct *r = ct_new(c, n, a->npoly, a->level, &err);
    if (!r) return err;
    const size_t per = (size_t)a->npoly * a->level * c->N;
    cudaMemcpyAsync(r->d, a->d + per * start, sizeof(u64) * per * n, cudaMemcpyDeviceToDevice, c->stream);
    *out = r;
    return 0;
}

int op_concat(fhe_ctx *c, const fhe_ct *a, const fhe_ct *b, fhe_ct **out)
{
    if (a->level != b->level || a->npoly != b->npoly) return fhe_fail(c, FHE_EMISMATCH, "concat: shapes differ");
    int err = 0;
    fhe_ct *r = ct_new(c, a->count + b->count, a->npoly, a->level, &err);
    if (!r) return err;
    cudaMemcpyAsync(r->d, a->d, a->bytes, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(r->d + a->bytes / sizeof(u64), b->d, b->bytes, cudaMemcpyDeviceToDevice, c->stream);
    *out = r;
    return 0;
}

namespace {

struct Tourney {
    fhe_ctx *c;
    const fhe_evk *evk;
    const fhe_sk *sk;
    const fhe_pk *pk;
    int d, depth;
    uint64_t seed;
    int refreshes = 0, err = 0;
    std::vector<fhe_ct *> owned;

    fhe_ct *own(fhe_ct *x)
    {
        owned.push_back(x);
        return x;
    }
    ~Tourney()
    {
        for (fhe_ct *x : owned)
            if (x) fhe_ct_destroy(x);
    }
    fhe_ct *release(fhe_ct *x)
    {
        for (auto &o : owned)
            if (o == x) o = nullptr;
        return x;
    }
    // refresh every digit batch when the next round would end below level 1
    bool ready(std::vector<fhe_ct *> &digs)
    {
        if (err) return false;
        if (digs[0]->level - depth >= 1) return true;
        if (!sk || !pk) {
            err = fhe_fail(c, FHE_ELEVEL, "tournament round needs a refresh: pass the secret and public keys");
            return false;
        }
        for (int k = 0; k < d && !err; k++) {
            fhe_ct *r = nullptr;
            if ((err = refresh_seeded(c, sk, pk, digs[k], seed + 1000003ull * (uint64_t)refreshes + k, &r)))
                return false;
            digs[k] = own(r);
        }
        refreshes++;
        return !err;
    }
    // one cross round on the batch: winners of [0,h) vs [h,2h), leftover after
    void cross(std::vector<fhe_ct *> &src, bool both, std::vector<fhe_ct *> *mx, std::vector<fhe_ct *> *mn)
    {
        const int n = src[0]->count, h = n / 2;
        std::vector<fhe_ct *> A(d), B(d), R(d, nullptr), smx(d, nullptr), smn(d, nullptr);
        for (int k = 0; k < d && !err; k++) {
            fhe_ct *t = nullptr;
            if ((err = op_slice(c, src[k], 0, h, &t))) return;
            A[k] = own(t);
            if ((err = op_slice(c, src[k], h, h, &t))) return;
            B[k] = own(t);
            if (n % 2) {
                if ((err = op_slice(c, src[k], 2 * h, 1, &t))) return;
                R[k] = own(t);
            }
        }
        if ((err = circuit_max_min(c, evk, A.data(), B.data(), d, mx ? smx.data() : nullptr,
                                   mn ? smn.data() : nullptr)))
            return;
        (void)both;
        for (int s = 0; s < 2; s++) {
            std::vector<fhe_ct *> *dst = s == 0 ? mx : mn;
            std::vector<fhe_ct *> &sel = s == 0 ? smx : smn;
            if (!dst) continue;
            for (int k = 0; k < d && !err; k++) {
                own(sel[k]);
                if (!R[k]) {
                    (*dst)[k] = sel[k];
                    continue;
                }
                fhe_ct *low = nullptr, *cat = nullptr;
                if ((err = op_lower(c, R[k], sel[k]->level, &low))) return;
                own(low);
                if ((err = op_concat(c, sel[k], low, &cat))) return;
                (*dst)[k] = own(cat);
            }
        }
    }
    // in-slot round: x <- sel(x, sigma_g(x))
    void inslot(std::vector<fhe_ct *> &cur, int64_t g, bool want_max)
    {
        const KeySwitchKey *key = evk->find(g);
        if (!key) {
            err = fhe_fail(c, FHE_ENOKEY, "tournament: missing rotation key");
            return;
        }
        std::vector<fhe_ct *> r(d), sel(d, nullptr);
        for (int k = 0; k < d && !err; k++) {
            fhe_ct *t = nullptr;
            if ((err = op_rotate(c, *key, cur[k], &t))) return;
            r[k] = own(t);
        }
        if ((err = circuit_max_min(c, evk, cur.data(), r.data(), d, want_max ? sel.data() : nullptr,
                                   want_max ? nullptr : sel.data())))
            return;
        for (int k = 0; k < d; k++) cur[k] = own(sel[k]);
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// sorting (rows of cols = n_s / 2 columns, each row on its own)
// ---------------------------------------------------------------------------
//
// The oracle's schedule: for shifts s = 1 .. cols-1, x_s = sigma_{5^s}(x)
// (column i holds x_{i+s}), (LT, EQ) = compare(x_s, x), rank += LT + w_s EQ
// with the plaintext tie-break mask w_s[i] = [i + s >= cols]; then for shifts
// s = 0 .. cols-1, e = 1 - (sigma_{5^s}(rank) - idx)^(p-1) (idx[i] = i) and
// out_k += e sigma_{5^s}(x_k) for every digit k.

std::vector<int64_t> sort_galois(const fhe_ctx *c)
{
    std::vector<int64_t> g;
    if (!c->slots_linear || c->ns < 4) return g;
    const int64_t twoN = 2 * (int64_t)c->N;
    for (int s = 1; s < c->ns / 2; s++) g.push_back((int64_t)host_powmod(5, (u64)s, (u64)twoN));
    return g;
}

// Each shift runs in a circuit of its own, so that its temporaries are
// freed before the next one; only the running rank and outputs are carried.
// Joint sort: row r of the K inputs x[a * d + k] (ciphertext a, digit k) is
// one sequence of K cols values, global index a cols + c.  rank^a sums, over
// (b, s) != (a, 0) with b and then s ascending, LT(sigma_{5^s} x^b, x^a) +
// w EQ(sigma_{5^s} x^b, x^a), w[c] = [b cols + (c + s) mod cols < a cols + c];
// then for a and s ascending (the rotations of rank^a and x^a taken once) and
// each target t: out^t += EQ(sigma_{5^s} rank^a - (t cols + c)) sigma_{5^s} x^a.
// Each comparison, and each (a, s) of the selection, is a sub-circuit of its
// own, so only the running sums outlive it.  K = 1 is the row sort.
// The rank step: for every ciphertext a and every other (b, s), (LT, EQ) =
// compare(sigma_{5^s} x^b, x^a) and rank^a += LT + w EQ (the tie-break mask
// of the schedule above); up to SORT_MERGE shifts of one (a, b) run in one
// circuit (merged operations), so only the running ranks outlive it and the
// scratch stays that many comparisons' worth.  matrix, when
// given, receives LT at [(a K + b) cols + s] (null at (a, a, 0)).  No bound on
// K cols: the ranks are counts mod p.
int circuit_sort_ranks(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, int K, int d, fhe_ct **rank_out,
                       fhe_ct **matrix)
{
    constexpr int SORT_MERGE = FHE_SORT_MERGE;
    if (!c->slots_linear || c->ns < 4)
        return fhe_fail(c, FHE_EUNSUPPORTED, "sorting needs p = 1 mod 4 (two columns or more)");
    if (K < 1 || d < 1) return fhe_fail(c, FHE_EINVAL, "sort ranks: K and d must be positive");
    const int cols = c->ns / 2;
    const std::vector<int64_t> gs = sort_galois(c);
    auto X = [&](int a) { return std::vector<const fhe_ct *>(x + (size_t)a * d, x + (size_t)(a + 1) * d); };
    std::vector<fhe_ct *> rank(K, nullptr);
    std::vector<fhe_ct *> mat(matrix ? (size_t)K * K * cols : 0, nullptr);
    int err = 0;
    for (int a = 0; a < K && !err; a++) {
        const std::vector<const fhe_ct *> xa = X(a);
        for (int bs = 0; bs < K * ((cols + SORT_MERGE - 1) / SORT_MERGE) && !err; bs++) {
            const int b = bs / ((cols + SORT_MERGE - 1) / SORT_MERGE);
            const int s0 = (bs % ((cols + SORT_MERGE - 1) / SORT_MERGE)) * SORT_MERGE;
            const std::vector<const fhe_ct *> xb = X(b);
            Circuit S(c, evk);
            std::vector<int> sh;
            std::vector<std::vector<const fhe_ct *>> xr;
            for (int s = s0; s < std::min(cols, s0 + SORT_MERGE) && !S.err; s++) {
                if (b == a && s == 0) continue;
                std::vector<const fhe_ct *> r(d);
                for (int k = 0; k < d; k++) r[k] = s ? S.rot(xb[k], gs[s - 1]) : xb[k];
                sh.push_back(s);
                xr.push_back(r);
            }
            if (sh.empty()) continue;
            std::vector<fhe_ct *> lt(sh.size(), nullptr), eq(sh.size(), nullptr);
            std::vector<Circuit::Req> rq;
            for (size_t i = 0; i < sh.size(); i++)
                rq.push_back(Circuit::Req{xr[i].data(), xa.data(), d, true, true, false, &lt[i], &eq[i], nullptr,
                                          nullptr});
            if (!S.err) S.compare_many(rq);
            fhe_ct *nr = nullptr;
            for (size_t i = 0; i < sh.size() && !S.err; i++) {
                const int s = sh[i];
                S.keep(lt[i]);
                S.keep(eq[i]);
                std::vector<uint64_t> w(c->ns);
                for (int r = 0; r < 2; r++)
                    for (int j = 0; j < cols; j++)
                        w[(size_t)r * cols + j] = (b * cols + (j + s) % cols < a * cols + j) ? 1 : 0;
                fhe_ct *t = S.add(lt[i], S.plain(eq[i], w, 2));
                nr = nr ? S.add(nr, t) : (rank[a] ? S.add(rank[a], t) : t);
            }
            S.finish();
            if (!S.err) {
                if (rank[a]) fhe_ct_destroy(rank[a]);
                rank[a] = S.release(nr);
                if (matrix)
                    for (size_t i = 0; i < sh.size(); i++) mat[((size_t)a * K + b) * cols + sh[i]] = S.release(lt[i]);
            }
            err = S.err;
        }
    }
    if (err) {
        for (fhe_ct *r : rank)
            if (r) fhe_ct_destroy(r);
        for (fhe_ct *m : mat)
            if (m) fhe_ct_destroy(m);
        return err;
    }
    for (int a = 0; a < K; a++) rank_out[a] = rank[a];
    for (size_t i = 0; i < mat.size(); i++) matrix[i] = mat[i];
    return 0;
}

int circuit_sort_joint(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, int K, int d, fhe_ct **out)
{
    if (!c->slots_linear || c->ns < 4)
        return fhe_fail(c, FHE_EUNSUPPORTED, "sorting needs p = 1 mod 4 (two columns or more)");
    const int cols = c->ns / 2, p = (int)c->p;
    if (K < 1 || (long long)K * cols > p) return fhe_fail(c, FHE_EINVAL, "joint sort: K cols must not exceed p");
    const std::vector<int64_t> gs = sort_galois(c);
    auto X = [&](int a) { return std::vector<const fhe_ct *>(x + (size_t)a * d, x + (size_t)(a + 1) * d); };
    std::vector<fhe_ct *> rank(K, nullptr), outs((size_t)K * d, nullptr);
    auto carry = [](fhe_ct *&held, fhe_ct *next) {
        if (held) fhe_ct_destroy(held);
        held = next;
    };
    int err = circuit_sort_ranks(c, evk, x, K, d, rank.data(), nullptr);
    for (int a = 0; a < K && !err; a++) {
        const std::vector<const fhe_ct *> xa = X(a);
        for (int s = 0; s < cols && !err; s++) {
            Circuit S(c, evk);
            const fhe_ct *rr = s ? S.rot(rank[a], gs[s - 1]) : rank[a];
            std::vector<const fhe_ct *> xr(d);
            for (int k = 0; k < d; k++) xr[k] = s ? S.rot(xa[k], gs[s - 1]) : xa[k];
            std::vector<fhe_ct *> nxt((size_t)K * d, nullptr);
            for (int t = 0; t < K && !S.err; t++) {
                std::vector<uint64_t> idx(c->ns);
                for (int r = 0; r < 2; r++)
                    for (int i = 0; i < cols; i++) idx[(size_t)r * cols + i] = (uint64_t)(t * cols + i);
                std::map<int, const fhe_ct *> pw;
                pw[1] = S.plain(rr, idx, 1);
                std::function<const fhe_ct *(int)> power = [&](int n) -> const fhe_ct * {
                    auto it = pw.find(n);
                    if (it != pw.end()) return it->second;
                    const fhe_ct *r;
                    if ((n & (n - 1)) == 0) {
                        const fhe_ct *h = power(n / 2);
                        r = S.mul(h, h);
                    } else {
                        int m = 1;
                        while (m * 2 < n) m *= 2;
                        const fhe_ct *A = power(m);
                        const fhe_ct *Bp = power(n - m);
                        r = S.mul(A, Bp);
                    }
                    pw[n] = r;
                    return r;
                };
                fhe_ct *e = S.cadd(S.neg(power(p - 1)), 1);
                for (int k = 0; k < d && !S.err; k++) {
                    fhe_ct *term = S.mul(e, xr[k]);
                    fhe_ct *&o = outs[(size_t)t * d + k];
                    nxt[(size_t)t * d + k] = o ? S.add(o, term) : term;
                }
            }
            S.finish();
            if (!S.err)
                for (size_t i = 0; i < nxt.size(); i++) carry(outs[i], S.release(nxt[i]));
            err = S.err;
        }
    }
    for (fhe_ct *r : rank)
        if (r) fhe_ct_destroy(r);
    if (err) {
        for (fhe_ct *o : outs)
            if (o) fhe_ct_destroy(o);
        return err;
    }
    for (size_t i = 0; i < outs.size(); i++) out[i] = outs[i];
    return 0;
}

int circuit_sort(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, int d, fhe_ct **out)
{
    return circuit_sort_joint(c, evk, x, 1, d, out);
}

// ---------------------------------------------------------------------------
// slot compaction and the slot manager (Sec. 5.3)
// ---------------------------------------------------------------------------
//
// Inputs are placed in order.  The useful slots of an input still to place go,
// under one slot rotation (columns shifted right by s, rows swapped when b),
// into the output that takes the most of them; the first (output, b, s) wins a
// tie, and an output opens only when every open one is full.  A piece is a
// plaintext mask, sigma_{5^(cols - s)} when s > 0, sigma_{2N-1} when b, and a
// sum into its output, in plan order.

int slot_plan(int ns, int n, const uint8_t *useful, std::vector<SlotPiece> &pieces, std::vector<int32_t> *dest)
{
    const int cols = ns >= 2 ? ns / 2 : 1, rows = ns >= 2 ? 2 : 1;
    auto image = [&](int u, int s, int b) { return ((u / cols) ^ b) * cols + (u % cols + s) % cols; };
    std::vector<std::vector<char>> occ;
    pieces.clear();
    if (dest) dest->assign((size_t)n * ns, -1);
    for (int j = 0; j < n; j++) {
        std::vector<int> rest;
        for (int u = 0; u < ns; u++)
            if (useful[(size_t)j * ns + u]) rest.push_back(u);
        while (!rest.empty()) {
            int best = 0, bo = -1, bs = 0, bb = 0;
            for (int o = 0; o < (int)occ.size(); o++)
                for (int b = 0; b < rows; b++)
                    for (int s2 = 0; s2 < cols; s2++) {
                        int cnt = 0;
                        for (int u : rest) cnt += !occ[o][image(u, s2, b)];
                        if (cnt > best) { best = cnt; bo = o; bs = s2; bb = b; }
                    }
            if (bo < 0) { occ.emplace_back(ns, 0); continue; }
            SlotPiece pc{j, bo, bs, bb, {}};
            std::vector<int> left;
            for (int u : rest) {
                const int t = image(u, bs, bb);
                if (occ[bo][t]) { left.push_back(u); continue; }
                occ[bo][t] = 1;
                pc.src.push_back(u);
                if (dest) (*dest)[(size_t)j * ns + u] = bo * ns + t;
            }
            pieces.push_back(std::move(pc));
            rest.swap(left);
        }
    }
    return (int)occ.size();
}

std::vector<int64_t> slot_galois(int ns, int64_t N, const std::vector<SlotPiece> &pieces)
{
    const int cols = ns >= 2 ? ns / 2 : 1;
    const u64 twoN = 2 * (u64)N;
    std::vector<int64_t> g;
    bool swap = false;
    for (const SlotPiece &pc : pieces) {
        if (pc.s) {
            const int64_t e = (int64_t)host_powmod(5, (u64)((cols - pc.s) % cols), twoN);
            if (std::find(g.begin(), g.end(), e) == g.end()) g.push_back(e);
        }
        swap = swap || pc.b;
    }
    std::sort(g.begin(), g.end());
    if (swap) g.push_back((int64_t)twoN - 1);
    return g;
}

int circuit_slot_pack(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *in, int n, const uint8_t *useful,
                      fhe_ct **out, int n_out)
{
    std::vector<SlotPiece> pieces;
    if (slot_plan(c->ns, n, useful, pieces, nullptr) != n_out) return FHE_EINVAL;
    const int ns = c->ns, cols = ns >= 2 ? ns / 2 : 1;
    const int64_t swap = 2 * (int64_t)c->N - 1;
    Circuit C(c, evk);
    std::vector<fhe_ct *> acc(n_out, nullptr);
    for (const SlotPiece &pc : pieces) {
        if (C.err) break;
        std::vector<uint64_t> mask(ns, 0);
        for (int u : pc.src) mask[u] = 1;
        fhe_ct *t = C.plain(in[pc.j], mask, 2);
        if (pc.s) t = C.rot(t, (int64_t)host_powmod(5, (u64)((cols - pc.s) % cols), 2 * (u64)c->N));
        if (pc.b) t = C.rot(t, swap);
        acc[pc.o] = acc[pc.o] ? C.add(acc[pc.o], t) : t;
    }
    if (!C.err)
        for (int o = 0; o < n_out; o++) out[o] = C.release(acc[o]);
    C.finish();
    return C.err;
}

// ---------------------------------------------------------------------------
// digit extraction from F_{p^d} slots (mod extract, Sec. 2.1)
// ---------------------------------------------------------------------------
//
// B_t = sigma_{p^t}(a), t = 1 .. d-1, in order of t; digit k = sum_t B_t *
// L[k][t], t ascending (extract.cu builds L).

int circuit_extract(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *a, const ExtTables *T, fhe_ct **out)
{
    const int d = T->d;
    Circuit C(c, evk);
    std::vector<const fhe_ct *> B{a};
    for (int t = 1; t < d && !C.err; t++) B.push_back(C.rot(a, T->galois[t - 1]));
    std::vector<fhe_ct *> D(d, nullptr);
    for (int k = 0; k < d && !C.err; k++)
        for (int t = 0; t < d && !C.err; t++) {
            fhe_ct *term = C.plain_coeffs(B[t], T->L[(size_t)k * d + t]);
            D[k] = D[k] ? C.add(D[k], term) : term;
        }
    if (!C.err)
        for (int k = 0; k < d; k++) out[k] = C.release(D[k]);
    C.finish();
    return C.err;
}

// ---------------------------------------------------------------------------
// private query with straight-lined branches (Sec. 5.3, non-blocking comparison)
// ---------------------------------------------------------------------------
//
// EQ(q, code_i) = 1 - (q - code_i)^(p-1) for the three public codes, then the
// candidates data + op1, data * op1, data^op2, then
// ((r1 EQ_1 + r2 EQ_2) + r3 EQ_3).  With overlap the circuit runs under the
// dependency scheduler: every operation is issued on one of its streams after
// its inputs, so the comparison branch and the arithmetic run concurrently on
// the device and join only at the selection.  The results are the same
// residues either way.

int circuit_private_query(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *q, const fhe_ct *data, const fhe_ct *op1,
                          int op2, const int64_t *codes, bool overlap, fhe_ct **out)
{
    const bool was = c->multistream;
    c->multistream = overlap;
    int e = 0;
    {
        Circuit C(c, evk);
        auto power_of = [&C](const fhe_ct *x, int n) -> fhe_ct * {
            std::map<int, const fhe_ct *> pw;
            pw[1] = x;
            std::function<const fhe_ct *(int)> power = [&](int m) -> const fhe_ct * {
                auto it = pw.find(m);
                if (it != pw.end()) return it->second;
                const fhe_ct *r;
                if ((m & (m - 1)) == 0) {
                    const fhe_ct *h = power(m / 2);
                    r = C.mul(h, h);
                } else {
                    int a = 1;
                    while (a * 2 < m) a *= 2;
                    const fhe_ct *A = power(a);
                    const fhe_ct *Bp = power(m - a);
                    r = C.mul(A, Bp);
                }
                pw[m] = r;
                return r;
            };
            return const_cast<fhe_ct *>(power(n));
        };
        const int p = (int)c->p;
        fhe_ct *eq[3];
        for (int i = 0; i < 3; i++) {
            fhe_ct *z = C.cadd(q, -codes[i]);
            eq[i] = C.cadd(C.neg(power_of(z, p - 1)), 1);
        }
        fhe_ct *r1 = C.add(data, op1);
        fhe_ct *r2 = C.mul(data, op1);
        fhe_ct *r3 = power_of(data, op2);
        fhe_ct *o = C.mul(r1, eq[0]);
        o = C.add(o, C.mul(r2, eq[1]));
        o = C.add(o, C.mul(r3, eq[2]));
        if (!C.err) *out = C.release(o);
        C.finish();
        e = C.err;
    }
    c->multistream = was;
    return e;
}

std::vector<int64_t> tournament_galois(const fhe_ctx *c)
{
    std::vector<int64_t> g;
    const int64_t twoN = 2 * (int64_t)c->N;
    if (!c->slots_linear || c->ns <= 2) {
        if (c->ns == 2) g.push_back(twoN - 1);
        return g;
    }
    for (int step = c->ns / 4; step >= 1; step /= 2) g.push_back((int64_t)host_powmod(5, step, twoN));
    g.push_back(twoN - 1);
    return g;
}

int circuit_tournament(fhe_ctx *c, const fhe_evk *evk, const fhe_sk *sk, const fhe_pk *pk, const fhe_ct *const *x,
                       int d, bool want_max, bool want_min, uint64_t seed, fhe_ct **out_max, fhe_ct **out_min)
{
    Tourney T{c, evk, sk, pk, d, 0, seed};
    int lg = 0;
    while ((1 << lg) < (int)c->p - 1) lg++;
    int ld = 0;
    while ((1 << ld) < d) ld++;
    T.depth = lg + ld + 1;
    std::vector<fhe_ct *> mx(d), mn(d);
    int n = x[0]->count;
    bool first = true;
    while (n > 1 && !T.err) {
        if (first) {
            std::vector<fhe_ct *> src(d);  // read only: slices and refreshes make new batches
            for (int k = 0; k < d; k++) src[k] = const_cast<fhe_ct *>(x[k]);
            if (!T.ready(src)) break;
            T.cross(src, want_max && want_min, want_max ? &mx : nullptr, want_min ? &mn : nullptr);
            first = false;
        } else {
            if (want_max && T.ready(mx)) {
                std::vector<fhe_ct *> src = mx;
                T.cross(src, false, &mx, nullptr);
            }
            if (want_min && T.ready(mn)) {
                std::vector<fhe_ct *> src = mn;
                T.cross(src, false, nullptr, &mn);
            }
        }
        n = n / 2 + n % 2;
    }
    if (first && !T.err)
        for (int k = 0; k < d; k++) {
            fhe_ct *cp = nullptr;
            if ((T.err = op_lower(c, x[k], x[k]->level, &cp))) break;  // a copy
            mx[k] = T.own(cp);
            if ((T.err = op_lower(c, x[k], x[k]->level, &cp))) break;
            mn[k] = T.own(cp);
        }
    for (int64_t g : tournament_galois(c)) {
        if (T.err) break;
        if (want_max && T.ready(mx)) T.inslot(mx, g, true);
        if (want_min && T.ready(mn)) T.inslot(mn, g, false);
    }
    if (T.err) return T.err;
    for (int k = 0; k < d; k++) {
        if (want_max) out_max[k] = T.release(mx[k]);
        if (want_min) out_min[k] = T.release(mn[k]);
    }
    return 0;
}
