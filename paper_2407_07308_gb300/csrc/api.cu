// api.cu -- the extern "C" boundary: contexts, keys, ciphertexts, encryption,
// decryption and the arithmetic / comparison entry points declared in fhe.h.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include <functional>

#include "fhe_internal.h"

// ---------------------------------------------------------------------------
// errors, pool
// ---------------------------------------------------------------------------

int fhe_fail(fhe_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int fhe_cuda_check(fhe_ctx *ctx, cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return 0;
    return fhe_fail(ctx, FHE_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Blocks come in size classes of a quarter power of two (at most 25% above
// the request), so that a freed block serves later requests of nearby sizes:
// batches of many levels and counts otherwise leave a cached block of every
// exact size behind and fill the device with them.
size_t pool_class(size_t bytes)
{
    if (bytes <= 1024) return 1024;
    int e = 63 - __builtin_clzll((unsigned long long)bytes);
    const size_t step = (size_t)1 << (e - 2);
    return (bytes + step - 1) / step * step;
}

void *Pool::get(size_t bytes, int *err)
{
    bytes = pool_class(bytes);
    if (cap_free) {
        auto &cf = (*cap_free)[bytes];
        if (!cf.empty()) {
            void *p = cf.back();
            cf.pop_back();
            return p;  // still counted in in_use
        }
    }
    auto &fl = free_lists[bytes];
    if (!fl.empty()) {
        void *p = fl.back();
        fl.pop_back();
        in_use += bytes;
        if (in_use > peak) peak = in_use;
        return p;
    }
    if (budget && reserved + bytes > budget) {
        trim();  // give cached blocks of other sizes back before refusing
        if (reserved + bytes > budget) {
            *err = FHE_EBUDGET;
            return nullptr;
        }
    }
    if (fail_after == 0) {
        *err = FHE_ENOMEM;
        return nullptr;
    }
    if (fail_after > 0) fail_after--;
    void *p = nullptr;
    if (in_capture) {
        // a miss while a graph is captured: plain cudaMalloc (permitted in a
        // relaxed capture), never the caller's allocator on a capturing stream
        if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
        if (p) raw[p] = true;
    } else if (alloc.alloc) {
        p = alloc.alloc(bytes, (void *)stream, alloc.user);
    } else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
        p = nullptr;
    }
    if (!p && !in_capture) {
        // out of device memory: wait for all queued work, hand every cached
        // free block (this pool's, and those of contexts not busy on another
        // thread, whose captured batch graphs are dropped too) back to the
        // allocator, and try once more
        cudaDeviceSynchronize();
        if (owner) batch_plans_release(owner, owner->bplan_active);
        trim();
        trim_other_pools(this);
        if (alloc.alloc) {
            p = alloc.alloc(bytes, (void *)stream, alloc.user);
        } else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
            p = nullptr;
        }
    }
    if (!p) {
        *err = FHE_ENOMEM;
        return nullptr;
    }
    live[p] = bytes;
    reserved += bytes;
    in_use += bytes;
    if (in_use > peak) peak = in_use;
    return p;
}

void Pool::put(void *p)
{
    auto it = live.find(p);
    if (it == live.end()) return;
    if (cap_free) {  // a graph being captured keeps using this block on every replay
        (*cap_free)[it->second].push_back(p);
        return;
    }
    free_lists[it->second].push_back(p);
    in_use -= it->second;
}

// Frees the cached (not handed out) blocks.
void Pool::trim()
{
    for (auto &kv : free_lists) {
        for (void *q : kv.second) {
            if (raw.count(q)) {
                cudaFree(q);
                raw.erase(q);
            } else if (alloc.free) {
                alloc.free(q, kv.first, (void *)stream, alloc.user);
            } else {
                cudaFreeAsync(q, stream);
            }
            live.erase(q);
            reserved -= kv.first;
        }
        kv.second.clear();
    }
}

// every live context, so that a pool out of memory can trim the others
static std::mutex g_ctx_mu;
static std::vector<fhe_ctx *> g_ctxs;

static void register_ctx(fhe_ctx *c, bool add)
{
    std::lock_guard<std::mutex> g(g_ctx_mu);
    if (add)
        g_ctxs.push_back(c);
    else
        g_ctxs.erase(std::remove(g_ctxs.begin(), g_ctxs.end(), c), g_ctxs.end());
}

void trim_other_pools(Pool *self)
{
    std::lock_guard<std::mutex> g(g_ctx_mu);
    for (fhe_ctx *o : g_ctxs) {
        if (&o->pool == self || !o->mu.try_lock()) continue;  // busy contexts keep theirs
        cudaStreamSynchronize(o->stream);
        batch_plans_release(o);  // captured batches are caches: rebuilt when needed
        o->pool.trim();
        o->mu.unlock();
    }
}

void Pool::release_all()
{
    for (auto &kv : live) {
        if (raw.count(kv.first))
            cudaFree(kv.first);
        else if (alloc.free)
            alloc.free(kv.first, kv.second, (void *)stream, alloc.user);
        else
            cudaFreeAsync(kv.first, stream);
    }
    raw.clear();
    live.clear();
    free_lists.clear();
    reserved = in_use = 0;
}

fhe_ct *ct_new(fhe_ctx *ctx, int count, int npoly, int level, int *err)
{
    const size_t bytes = sizeof(u64) * (size_t)count * npoly * level * ctx->N;
    void *p = ctx->pool.get(bytes, err);
    if (!p) {
        fhe_fail(ctx, *err, "out of device memory for a ciphertext");
        return nullptr;
    }
    fhe_ct *ct = new fhe_ct;
    ct->ctx = ctx;
    ct->count = count;
    ct->npoly = npoly;
    ct->level = level;
    ct->d = (u64 *)p;
    ct->bytes = bytes;
    return ct;
}

const KeySwitchKey *fhe_evk::find(int64_t g) const
{
    for (const auto &k : keys)
        if (k.galois == g) return &k;
    return nullptr;
}

namespace {

struct DevBuf {
    fhe_ctx *c;
    void *p = nullptr;
    DevBuf(fhe_ctx *ctx, size_t bytes, int *err) : c(ctx)
    {
        if (*err) return;
        p = c->pool.get(bytes, err);
    }
    ~DevBuf()
    {
        if (p) c->pool.put(p);
    }
    u64 *u() { return (u64 *)p; }
    int64_t *i() { return (int64_t *)p; }
};

LimbMap plain_map(int nl, int prime_off)
{
    LimbMap m;
    memset(&m, 0, sizeof(m));
    m.nl = nl;
    for (int i = 0; i < nl; i++) m.in_limb[i] = m.out_limb[i] = i, m.prime[i] = prime_off + i;
    return m;
}

// NTT (forward) of `outer` contiguous blocks of nl limbs, primes prime_off..
void ntt_blocks(fhe_ctx *c, const u64 *in, u64 *out, int outer, int nl, int prime_off, bool inverse)
{
    LimbMap m = plain_map(nl, prime_off);
    m.in_outer = m.out_outer = (long long)nl * c->N;
    if (inverse)
        launch_ntt_inv_plain(c, in, out, m, outer * nl);
    else
        launch_ntt_fwd_plain(c, in, out, m, outer * nl);
}

void primes_range(int *pr, int n, int off)
{
    for (int i = 0; i < n; i++) pr[i] = off + i;
}

// slot values (n_s) -> plaintext coefficients (N), values in [0, p)
void encode_slots(const fhe_ctx *c, const uint64_t *v, int64_t *m)
{
    const u64 p = c->p;
    const int M = c->M, stride = c->N / M;
    memset(m, 0, sizeof(int64_t) * c->N);
    if (c->slots_linear) {
        // m_j = M^-1 sum_s v_s zeta^(-e_s j)
        const u64 Minv = host_invmod(M % p, p);
        for (int j = 0; j < M; j++) {
            u64 acc = 0;
            for (int s = 0; s < c->ns; s++) {
                const u64 e = (u64)((2 * M - (int64_t)c->slot_exp[s] * j % (2 * M)) % (2 * M));
                acc = (acc + (v[s] % p) * host_powmod(c->zeta, e, p)) % p;
            }
            m[(size_t)j * stride] = (int64_t)host_mulmod(acc, Minv, p);
        }
    } else {
        // two slots: m = (v0+v1)/2 + (v0-v1)/2 h(Y), h = -(Y + Y^3)/gamma
        const u64 inv2 = host_invmod(2, p), ig = host_invmod(c->gamma, p);
        const u64 a = (v[0] % p + v[1] % p) % p * inv2 % p;
        const u64 b = (v[0] % p + p - v[1] % p) % p * inv2 % p;
        const u64 h = (p - ig) % p;
        m[0] = (int64_t)a;
        m[(size_t)1 * stride] = (int64_t)(b * h % p);
        m[(size_t)3 * stride] = (int64_t)(b * h % p);
    }
}

// plaintext coefficients in [0, p) -> slots; false if not a slot encoding
bool decode_slots(const fhe_ctx *c, const int64_t *m, uint64_t *v)
{
    const u64 p = c->p;
    const int M = c->M, stride = c->N / M;
    for (int n = 0; n < c->N; n++)
        if (n % stride && m[n]) return false;
    if (c->slots_linear) {
        for (int s = 0; s < c->ns; s++) {
            const u64 z = host_powmod(c->zeta, (u64)c->slot_exp[s], p);
            u64 acc = 0, zz = 1;
            for (int j = 0; j < M; j++) {
                acc = (acc + (u64)m[(size_t)j * stride] * zz) % p;
                zz = zz * z % p;
            }
            v[s] = acc;
        }
        return true;
    }
    for (int s = 0; s < 2; s++) {
        const u64 g = s == 0 ? c->gamma : p - c->gamma;  // factor Y^2 + g Y - 1
        u64 a0 = 0, a1 = 0, w0 = 1, w1 = 0;             // residue and Y^j mod factor
        for (int j = 0; j < M; j++) {
            const u64 mj = (u64)m[(size_t)j * stride];
            a0 = (a0 + mj * w0) % p;
            a1 = (a1 + mj * w1) % p;
            const u64 n0 = w1, n1 = (w0 + p - g * w1 % p) % p;  // Y (w0 + w1 Y), Y^2 = 1 - gY
            w0 = n0;
            w1 = n1;
        }
        if (a1) return false;
        v[s] = a0;
    }
    return true;
}

#define CHECK_CTX(c)                                  \
    do {                                              \
        if (!(c)) return FHE_EINVAL;                  \
    } while (0)
#define LOCK(c) std::lock_guard<std::mutex> _g((c)->mu)

int sync_check(fhe_ctx *c, const char *where)
{
    return fhe_cuda_check(c, cudaStreamSynchronize(c->stream), where);
}

}  // namespace

void encode_slot_vector(const fhe_ctx *c, const uint64_t *v, int64_t *m) { encode_slots(c, v, m); }

// Stream tags of the seeded samplers (see sample.cu).
enum { TAG_S = 1, TAG_E_PK = 2, TAG_A_PK = 3, TAG_U = 16, TAG_E0 = 17, TAG_E1 = 18, TAG_KSK = 1024 };

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

extern "C" int fhe_ctx_create(const fhe_params *P, const fhe_allocator *alloc, void *stream, fhe_ctx **out)
{
    if (!P || !out) return FHE_EINVAL;
    *out = nullptr;
    if (!ntt_supported_logn(P->log_n)) return FHE_EUNSUPPORTED;
    if (P->L < 1 || P->K < 1 || P->K > FHE_MAXK || P->L + P->K > FHE_MAXP || (P->L + P->K - 1) / P->K > FHE_MAXD)
        return FHE_EUNSUPPORTED;
    if (P->p < 3 || !host_is_prime(P->p) || P->p > (1u << 20)) return FHE_EINVAL;
    const u64 N = 1ull << P->log_n;
    if (P->prime_mod % (2 * N) || P->prime_mod % P->p) return FHE_EINVAL;
    fhe_ctx *c = new fhe_ctx;
    c->logN = P->log_n;
    c->N = (int)N;
    c->L = P->L;
    c->K = P->K;
    c->np = P->L + P->K;
    c->p = P->p;
    c->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) c->device = -1;
    if (const char *ws = getenv("FHE_WAVE_SPLIT")) c->wave_split = std::max(1, std::min(8, atoi(ws)));
    if (c->device < 0 || cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        c->sms = 0;
    c->q.resize(c->np);
    if (host_find_primes(P->prime_mod, P->prime_lo, P->prime_hi, c->np, c->q.data()) != c->np) {
        delete c;
        return FHE_EINVAL;
    }
    int bits0 = 64 - __builtin_clzll(c->q[0]);
    for (u64 q : c->q)
        if (64 - __builtin_clzll(q) != bits0 || bits0 > 57) {
            delete c;
            return FHE_EUNSUPPORTED;
        }
    if (alloc) c->pool.alloc = *alloc;
    else memset(&c->pool.alloc, 0, sizeof(fhe_allocator));
    c->pool.stream = c->stream;
    c->pool.owner = c;
    int e = build_tables(c);
    if (!e) e = fhe_cuda_check(c, cudaDeviceSynchronize(), "ctx_create");
    // choose the NTT factorisation for this ring degree on 32 polynomials
    // (16 ciphertexts) of up to 10 limbs, the scale of batched use
    // FHE_NTT_VARIANT pins the variant (e.g. to profile the one a timed run
    // chose: timings under a profiler are not representative)
    const char *pin = getenv("FHE_NTT_VARIANT");
    if (!e && pin && *pin >= '0' && *pin <= '9' && ntt_variant_ok(c->logN, atoi(pin)))
        c->ntt_variant = atoi(pin);
    else if (!e)
        e = ntt_autotune(c, 32 * 10, c->ntt_ms);
    if (e) {
        fhe_ctx_destroy(c);
        return e;
    }
    register_ctx(c, true);
    *out = c;
    return 0;
}

extern "C" void fhe_ctx_destroy(fhe_ctx *c)
{
    if (!c) return;
    register_ctx(c, false);
    cudaStreamSynchronize(c->stream);
    batch_plans_release(c);
    batch_family_release(c);
    c->pool.release_all();
    cudaFree(c->d_mq);
    cudaFree(c->d_fwd);
    cudaFree(c->d_inv);
    cudaFree(c->d_ninv);
    cudaFree(c->d_modup);
    cudaFree(c->d_moddown);
    cudaFree(c->d_modswitch);
    cudaFree(c->d_rms);
    cudaFree(c->d_mss);
    cudaFree(c->d_ks_xscale);
    cudaFree(c->d_ms4scale);
    cudaFree(c->d_ks_pscale);
    cudaFree(c->d_ms_lastscale);
    cudaFree(c->d_mss_scale);
    for (auto &kv : c->d_perm) cudaFree(kv.second);
    for (cudaStream_t s : c->branch_streams) cudaStreamDestroy(s);
    for (cudaEvent_t ev : c->branch_events) cudaEventDestroy(ev);
    cudaStreamSynchronize(c->stream);
    delete c;
}

extern "C" const char *fhe_last_error(const fhe_ctx *c) { return c ? c->err.c_str() : "no context"; }

extern "C" int fhe_ctx_info(const fhe_ctx *c, fhe_info *out)
{
    if (!c || !out) return FHE_EINVAL;
    out->N = c->N;
    out->L = c->L;
    out->K = c->K;
    out->slots = c->ns;
    out->subring = c->M;
    out->dnum_max = (c->L + c->K - 1) / c->K;
    out->p = c->p;
    return 0;
}

extern "C" int fhe_ctx_primes(const fhe_ctx *c, uint64_t *out)
{
    if (!c || !out) return FHE_EINVAL;
    memcpy(out, c->q.data(), sizeof(u64) * c->np);
    return 0;
}

extern "C" int fhe_ctx_set_stream(fhe_ctx *c, void *stream)
{
    CHECK_CTX(c);
    LOCK(c);
    c->stream = (cudaStream_t)stream;
    c->pool.stream = c->stream;
    return 0;
}

extern "C" int fhe_ctx_sync(fhe_ctx *c)
{
    CHECK_CTX(c);
    return sync_check(c, "sync");
}

extern "C" int fhe_ctx_memory(const fhe_ctx *c, uint64_t *reserved, uint64_t *in_use)
{
    if (!c) return FHE_EINVAL;
    if (reserved) *reserved = c->pool.reserved;
    if (in_use) *in_use = c->pool.in_use;
    return 0;
}

extern "C" int fhe_ctx_memory_peak(fhe_ctx *c, uint64_t *peak, int reset)
{
    CHECK_CTX(c);
    LOCK(c);
    if (peak) *peak = c->pool.peak;
    if (reset) c->pool.peak = c->pool.in_use;
    return 0;
}

extern "C" int fhe_ctx_fused_modswitch(fhe_ctx *c, int on)
{
    CHECK_CTX(c);
    LOCK(c);
    c->separate_ms = !on;
    return 0;
}

extern "C" int fhe_ctx_trim(fhe_ctx *c)
{
    CHECK_CTX(c);
    LOCK(c);
    int e = sync_check(c, "trim");
    if (!e) c->pool.trim();
    return e;
}

extern "C" int fhe_ctx_inject_alloc_failure(fhe_ctx *c, int64_t n)
{
    CHECK_CTX(c);
    LOCK(c);
    c->pool.fail_after = n < 0 ? -1 : n;
    return 0;
}

extern "C" int fhe_ctx_set_budget(fhe_ctx *c, uint64_t bytes)
{
    CHECK_CTX(c);
    LOCK(c);
    c->pool.budget = bytes;
    return 0;
}

extern "C" int64_t fhe_ctx_launches(const fhe_ctx *c) { return c ? c->launches : -1; }

// ---------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------

// Key generation from device-resident s, e (int64[N]) and a (u64[L][N],
// coefficient domain): pk = (-a s + p e, a).
static int keygen_dev(fhe_ctx *c, const int64_t *ds, const u64 *da, const int64_t *de, fhe_sk **sk, fhe_pk **pk)
{
    const int N = c->N, L = c->L, np = c->np;
    int err = 0;
    DevBuf ta(c, sizeof(u64) * L * N, &err), te(c, sizeof(u64) * L * N, &err);
    if (err) return fhe_fail(c, err, "keygen: out of memory");
    fhe_sk *S = new fhe_sk;
    S->ctx = c;
    S->s.assign(N, 0);
    S->d_s = (u64 *)c->pool.get(sizeof(u64) * np * N, &err);
    fhe_pk *Pk = new fhe_pk;
    Pk->ctx = c;
    Pk->d = err ? nullptr : (u64 *)c->pool.get(sizeof(u64) * 2 * L * N, &err);
    if (err) {
        fhe_sk_destroy(S);
        fhe_pk_destroy(Pk);
        return fhe_fail(c, err, "keygen: out of memory");
    }
    cudaMemcpyAsync(ta.p, da, sizeof(u64) * L * N, cudaMemcpyDeviceToDevice, c->stream);
    int pr[FHE_MAXP];
    primes_range(pr, np, 0);
    launch_rns_from_i64(c, ds, nullptr, 1, S->d_s, 1, np, pr);
    ntt_blocks(c, S->d_s, S->d_s, 1, np, 0, false);
    launch_rns_from_i64(c, de, nullptr, (int64_t)c->p, te.u(), 1, L, pr);
    ntt_blocks(c, te.u(), te.u(), 1, L, 0, false);
    u64 *pk1 = Pk->d + (size_t)L * N;
    ntt_blocks(c, ta.u(), pk1, 1, L, 0, false);
    launch_muladd(c, pk1, S->d_s, te.u(), Pk->d, 1, L, 0, 1);  // pk0 = e' - a s
    cudaMemcpyAsync(S->s.data(), ds, sizeof(int64_t) * N, cudaMemcpyDeviceToHost, c->stream);
    int r = sync_check(c, "keygen");
    if (r) {
        fhe_sk_destroy(S);
        fhe_pk_destroy(Pk);
        return r;
    }
    *sk = S;
    *pk = Pk;
    return 0;
}

extern "C" int fhe_keygen_explicit(fhe_ctx *c, const int64_t *s, const uint64_t *a, const int64_t *e, fhe_sk **sk,
                                   fhe_pk **pk)
{
    CHECK_CTX(c);
    if (!s || !a || !e || !sk || !pk) return FHE_EINVAL;
    LOCK(c);
    const int N = c->N, L = c->L;
    int err = 0;
    DevBuf ds(c, sizeof(int64_t) * N, &err), de(c, sizeof(int64_t) * N, &err), da(c, sizeof(u64) * L * N, &err);
    if (err) return fhe_fail(c, err, "keygen: out of memory");
    cudaMemcpyAsync(ds.p, s, sizeof(int64_t) * N, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(de.p, e, sizeof(int64_t) * N, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(da.p, a, sizeof(u64) * L * N, cudaMemcpyHostToDevice, c->stream);
    return keygen_dev(c, ds.i(), da.u(), de.i(), sk, pk);
}

extern "C" int fhe_keygen(fhe_ctx *c, uint64_t seed, fhe_sk **sk, fhe_pk **pk)
{
    CHECK_CTX(c);
    if (!sk || !pk) return FHE_EINVAL;
    LOCK(c);
    const int N = c->N, L = c->L;
    int err = 0;
    DevBuf ds(c, sizeof(int64_t) * N, &err), de(c, sizeof(int64_t) * N, &err), da(c, sizeof(u64) * L * N, &err);
    if (err) return fhe_fail(c, err, "keygen: out of memory");
    sample_ternary(c, ds.i(), N, seed, TAG_S);
    sample_gaussian(c, de.i(), N, seed, TAG_E_PK);
    sample_uniform(c, da.u(), 1, L, seed, TAG_A_PK);
    return keygen_dev(c, ds.i(), da.u(), de.i(), sk, pk);
}

extern "C" void fhe_sk_destroy(fhe_sk *sk)
{
    if (!sk) return;
    if (sk->d_s) sk->ctx->pool.put(sk->d_s);
    delete sk;
}

extern "C" void fhe_pk_destroy(fhe_pk *pk)
{
    if (!pk) return;
    if (pk->d) pk->ctx->pool.put(pk->d);
    delete pk;
}

// Switching keys; the masks a_j and errors e_j of key `key`, digit j come
// from the host arrays (explicit) or from the seeded samplers.
static int evk_create(fhe_ctx *c, const fhe_sk *sk, const int64_t *galois, int n_galois, const uint64_t *a,
                      const int64_t *e, bool seeded, uint64_t seed, fhe_evk **out)
{
    const int N = c->N, L = c->L, K = c->K, np = c->np, dnum = (L + K - 1) / K;
    int err = 0;
    DevBuf ta(c, sizeof(u64) * np * N, &err), te(c, sizeof(u64) * np * N, &err);
    DevBuf de(c, sizeof(int64_t) * N, &err), sp(c, sizeof(u64) * np * N, &err);
    if (err) return fhe_fail(c, err, "evk: out of memory");
    u64 Pw[FHE_MAXP], Pws[FHE_MAXP];
    for (int i = 0; i < np; i++) {
        u64 P = 1;
        for (int k = 0; k < K; k++) P = host_mulmod(P, c->q[L + k] % c->q[i], c->q[i]);
        Pw[i] = P;
        Pws[i] = shoup_const(P, c->q[i]);
    }
    int pr[FHE_MAXP];
    primes_range(pr, np, 0);
    fhe_evk *E = new fhe_evk;
    E->ctx = c;
    for (int key = 0; key <= n_galois && !err; key++) {
        KeySwitchKey k;
        k.galois = key == 0 ? 0 : galois[key - 1];
        // s' in the NTT domain: s*s, or sigma_g(s) as an index permutation
        if (key == 0) {
            launch_mul_poly(c, sk->d_s, sk->d_s, sp.u(), 1, np, 0);
        } else {
            const int *perm = nullptr;
            if ((err = galois_perm(c, k.galois, &perm))) break;
            launch_automorphism(c, sk->d_s, sp.u(), 1, np, perm);
        }
        k.d = (u64 *)c->pool.get(sizeof(u64) * dnum * 2 * np * N, &err);
        if (err) break;
        E->keys.push_back(k);
        for (int j = 0; j < dnum; j++) {
            const size_t off = ((size_t)key * dnum + j);
            if (seeded) {
                sample_uniform(c, ta.u(), 1, np, seed, TAG_KSK + 2 * (uint32_t)off);
                sample_gaussian(c, de.i(), N, seed, TAG_KSK + 2 * (uint32_t)off + 1);
            } else {
                cudaMemcpyAsync(ta.p, a + off * np * N, sizeof(u64) * np * N, cudaMemcpyHostToDevice, c->stream);
                cudaMemcpyAsync(de.p, e + off * N, sizeof(int64_t) * N, cudaMemcpyHostToDevice, c->stream);
            }
            ntt_blocks(c, ta.u(), ta.u(), 1, np, 0, false);
            launch_rns_from_i64(c, de.i(), nullptr, (int64_t)c->p, te.u(), 1, np, pr);
            ntt_blocks(c, te.u(), te.u(), 1, np, 0, false);
            u64 *k0 = k.d + (size_t)(j * 2 + 0) * np * N, *k1 = k.d + (size_t)(j * 2 + 1) * np * N;
            launch_ksk_digit(c, ta.u(), te.u(), sk->d_s, sp.u(), k0, k1, j * K, std::min((j + 1) * K, L), Pw, Pws);
            // the staging buffers are reused by the next digit
            if ((err = sync_check(c, "evk digit"))) break;
        }
    }
    if (err) {
        fhe_evk_destroy(E);
        return err;
    }
    *out = E;
    return 0;
}

extern "C" int fhe_evk_create_explicit(fhe_ctx *c, const fhe_sk *sk, const int64_t *galois, int n_galois,
                                       const uint64_t *a, const int64_t *e, fhe_evk **out)
{
    CHECK_CTX(c);
    if (!sk || !a || !e || !out || n_galois < 0 || (n_galois && !galois)) return FHE_EINVAL;
    LOCK(c);
    return evk_create(c, sk, galois, n_galois, a, e, false, 0, out);
}

extern "C" int fhe_evk_create(fhe_ctx *c, const fhe_sk *sk, const int64_t *galois, int n_galois, uint64_t seed,
                              fhe_evk **out)
{
    CHECK_CTX(c);
    if (!sk || !out || n_galois < 0 || (n_galois && !galois)) return FHE_EINVAL;
    LOCK(c);
    return evk_create(c, sk, galois, n_galois, nullptr, nullptr, true, seed, out);
}

extern "C" void fhe_evk_destroy(fhe_evk *evk)
{
    if (!evk) return;
    for (auto &k : evk->keys)
        if (k.d) evk->ctx->pool.put(k.d);
    delete evk;
}

// ---------------------------------------------------------------------------
// encryption, decryption, import/export
// ---------------------------------------------------------------------------

// Encryption from device-resident inputs: m, u, e0, e1 are int64[count][N].
// Enc(m) = (pk0 u + p e0 + m, pk1 u + p e1) at level L.
static int encrypt_dev(fhe_ctx *c, const fhe_pk *pk, const int64_t *dm, const int64_t *du, const int64_t *d0,
                       const int64_t *d1, int count, fhe_ct **out)
{
    const int N = c->N, L = c->L;
    int err = 0;
    DevBuf U(c, sizeof(u64) * count * L * N, &err), T0(c, sizeof(u64) * count * L * N, &err),
        T1(c, sizeof(u64) * count * L * N, &err);
    DevBuf C0(c, sizeof(u64) * count * L * N, &err), C1(c, sizeof(u64) * count * L * N, &err);
    if (err) return fhe_fail(c, err, "encrypt: out of memory");
    fhe_ct *ct = ct_new(c, count, 2, L, &err);
    if (!ct) return err;
    int pr[FHE_MAXP];
    primes_range(pr, L, 0);
    launch_rns_from_i64(c, du, nullptr, 1, U.u(), count, L, pr);
    launch_rns_from_i64(c, d0, dm, (int64_t)c->p, T0.u(), count, L, pr);
    launch_rns_from_i64(c, d1, nullptr, (int64_t)c->p, T1.u(), count, L, pr);
    ntt_blocks(c, U.u(), U.u(), count, L, 0, false);
    ntt_blocks(c, T0.u(), T0.u(), count, L, 0, false);
    ntt_blocks(c, T1.u(), T1.u(), count, L, 0, false);
    launch_muladd(c, U.u(), pk->d, T0.u(), C0.u(), count, L, 0, 0);
    launch_muladd(c, U.u(), pk->d + (size_t)L * N, T1.u(), C1.u(), count, L, 0, 0);
    launch_copy_limbs(c, C0.u(), ct->d, count, L, (long long)L * N, 2LL * L * N);
    launch_copy_limbs(c, C1.u(), ct->d + (size_t)L * N, count, L, (long long)L * N, 2LL * L * N);
    *out = ct;
    return 0;
}

static int encode_batch(fhe_ctx *c, const uint64_t *slots, int count, std::vector<int64_t> &m)
{
    for (long long i = 0; i < (long long)count * c->ns; i++)
        if (slots[i] >= c->p) return fhe_fail(c, FHE_EINVAL, "slot value out of [0, p)");
    m.assign((size_t)count * c->N, 0);
    for (int i = 0; i < count; i++) encode_slots(c, slots + (size_t)i * c->ns, m.data() + (size_t)i * c->N);
    return 0;
}

// F_{p^d} slot elements of a batch: digits [count][n_s][d] -> coefficients
static int encode_batch_ext(fhe_ctx *c, const uint64_t *digits, int count, int d, std::vector<int64_t> &m)
{
    int err = 0;
    const ExtTables *T = ext_tables(c, d, &err);
    if (!T) return err;
    const long long per = (long long)c->ns * d;
    for (long long i = 0; i < count * per; i++)
        if (digits[i] >= c->p) return fhe_fail(c, FHE_EINVAL, "digit out of [0, p)");
    m.assign((size_t)count * c->N, 0);
    for (int i = 0; i < count; i++) ext_encode(c, T, digits + i * per, m.data() + (size_t)i * c->N);
    return 0;
}

extern "C" int fhe_encrypt_explicit(fhe_ctx *c, const fhe_pk *pk, const uint64_t *slots, int count,
                                    const int64_t *u, const int64_t *e0, const int64_t *e1, fhe_ct **out)
{
    FHE_RANGE("fhe_encrypt_explicit");
    CHECK_CTX(c);
    if (!pk || !slots || !u || !e0 || !e1 || !out || count < 1) return FHE_EINVAL;
    LOCK(c);
    std::vector<int64_t> m;
    int err = encode_batch(c, slots, count, m);
    if (err) return err;
    const size_t vb = sizeof(int64_t) * count * c->N;
    DevBuf du(c, vb, &err), d0(c, vb, &err), d1(c, vb, &err), dm(c, vb, &err);
    if (err) return fhe_fail(c, err, "encrypt: out of memory");
    cudaMemcpyAsync(du.p, u, vb, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d0.p, e0, vb, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d1.p, e1, vb, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(dm.p, m.data(), vb, cudaMemcpyHostToDevice, c->stream);
    fhe_ct *ct = nullptr;
    if ((err = encrypt_dev(c, pk, dm.i(), du.i(), d0.i(), d1.i(), count, &ct))) return err;
    int r = sync_check(c, "encrypt");
    if (r) {
        fhe_ct_destroy(ct);
        return r;
    }
    *out = ct;
    return 0;
}

extern "C" int fhe_encrypt(fhe_ctx *c, const fhe_pk *pk, const uint64_t *slots, int count, uint64_t seed, fhe_ct **out)
{
    FHE_RANGE("fhe_encrypt");
    CHECK_CTX(c);
    if (!pk || !slots || !out || count < 1) return FHE_EINVAL;
    LOCK(c);
    std::vector<int64_t> m;
    int err = encode_batch(c, slots, count, m);
    if (err) return err;
    const long long n = (long long)count * c->N;
    DevBuf du(c, sizeof(int64_t) * n, &err), d0(c, sizeof(int64_t) * n, &err), d1(c, sizeof(int64_t) * n, &err),
        dm(c, sizeof(int64_t) * n, &err);
    if (err) return fhe_fail(c, err, "encrypt: out of memory");
    cudaMemcpyAsync(dm.p, m.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->stream);
    sample_ternary(c, du.i(), n, seed, TAG_U);
    sample_gaussian(c, d0.i(), n, seed, TAG_E0);
    sample_gaussian(c, d1.i(), n, seed, TAG_E1);
    fhe_ct *ct = nullptr;
    if ((err = encrypt_dev(c, pk, dm.i(), du.i(), d0.i(), d1.i(), count, &ct))) return err;
    int r = sync_check(c, "encrypt");
    if (r) {
        fhe_ct_destroy(ct);
        return r;
    }
    *out = ct;
    return 0;
}

// Plaintext coefficients of a batch, on the device: modulus switch a copy to
// one prime, t = c0 + c1 s (limb 0), INTT, centred mod q0, then mod p.
static int decrypt_coeffs_dev(fhe_ctx *c, const fhe_sk *sk, const fhe_ct *ct, int64_t *dm)
{
    const int N = c->N, count = ct->count;
    fhe_ct *one = nullptr;
    int err = op_lower(c, ct, 1, &one);
    if (err) return err;
    DevBuf t(c, sizeof(u64) * count * N, &err), c0(c, sizeof(u64) * count * N, &err),
        c1(c, sizeof(u64) * count * N, &err);
    if (err) {
        fhe_ct_destroy(one);
        return fhe_fail(c, err, "decrypt: out of memory");
    }
    launch_copy_limbs(c, one->d, c0.u(), count, 1, 2LL * N, N);
    launch_copy_limbs(c, one->d + N, c1.u(), count, 1, 2LL * N, N);
    launch_muladd(c, c1.u(), sk->d_s, c0.u(), t.u(), count, 1, 0, 0);
    ntt_blocks(c, t.u(), t.u(), count, 1, 0, true);
    launch_centre_mod_p(c, t.u(), dm, (long long)count * N);
    fhe_ct_destroy(one);
    return 0;
}

extern "C" int fhe_decrypt(fhe_ctx *c, const fhe_sk *sk, const fhe_ct *ct, uint64_t *slots)
{
    FHE_RANGE("fhe_decrypt");
    CHECK_CTX(c);
    if (!sk || !ct || !slots || ct->npoly != 2) return FHE_EINVAL;
    LOCK(c);
    const int N = c->N, count = ct->count;
    int err = 0;
    DevBuf dm(c, sizeof(int64_t) * count * N, &err);
    if (err) return fhe_fail(c, err, "decrypt: out of memory");
    if ((err = decrypt_coeffs_dev(c, sk, ct, dm.i()))) return err;
    std::vector<int64_t> m((size_t)count * N);
    cudaMemcpyAsync(m.data(), dm.p, sizeof(int64_t) * m.size(), cudaMemcpyDeviceToHost, c->stream);
    if ((err = sync_check(c, "decrypt"))) return err;
    for (int i = 0; i < count; i++)
        if (!decode_slots(c, m.data() + (size_t)i * N, slots + (size_t)i * c->ns))
            return fhe_fail(c, FHE_EINVAL, "decrypt: plaintext is not a slot encoding");
    return 0;
}

extern "C" int fhe_ext_galois(fhe_ctx *c, int d, int64_t *galois, int cap)
{
    CHECK_CTX(c);
    if (d < 1 || cap < 0 || (cap && !galois)) return FHE_EINVAL;
    LOCK(c);
    int err = 0;
    const ExtTables *T = ext_tables(c, d, &err);
    if (!T) return err;
    for (int i = 0; i < (int)T->galois.size() && i < cap; i++) galois[i] = T->galois[i];
    return (int)T->galois.size();
}

extern "C" int fhe_encrypt_ext(fhe_ctx *c, const fhe_pk *pk, const uint64_t *digits, int count, int d, uint64_t seed,
                               fhe_ct **out)
{
    FHE_RANGE("fhe_encrypt_ext");
    CHECK_CTX(c);
    if (!pk || !digits || !out || count < 1 || d < 1) return FHE_EINVAL;
    LOCK(c);
    std::vector<int64_t> m;
    int err = encode_batch_ext(c, digits, count, d, m);
    if (err) return err;
    const long long n = (long long)count * c->N;
    DevBuf du(c, sizeof(int64_t) * n, &err), d0(c, sizeof(int64_t) * n, &err), d1(c, sizeof(int64_t) * n, &err),
        dm(c, sizeof(int64_t) * n, &err);
    if (err) return fhe_fail(c, err, "encrypt: out of memory");
    cudaMemcpyAsync(dm.p, m.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->stream);
    sample_ternary(c, du.i(), n, seed, TAG_U);
    sample_gaussian(c, d0.i(), n, seed, TAG_E0);
    sample_gaussian(c, d1.i(), n, seed, TAG_E1);
    fhe_ct *ct = nullptr;
    if ((err = encrypt_dev(c, pk, dm.i(), du.i(), d0.i(), d1.i(), count, &ct))) return err;
    if ((err = sync_check(c, "encrypt"))) {
        fhe_ct_destroy(ct);
        return err;
    }
    *out = ct;
    return 0;
}

extern "C" int fhe_encrypt_ext_explicit(fhe_ctx *c, const fhe_pk *pk, const uint64_t *digits, int count, int d,
                                        const int64_t *u, const int64_t *e0, const int64_t *e1, fhe_ct **out)
{
    CHECK_CTX(c);
    if (!pk || !digits || !u || !e0 || !e1 || !out || count < 1 || d < 1) return FHE_EINVAL;
    LOCK(c);
    std::vector<int64_t> m;
    int err = encode_batch_ext(c, digits, count, d, m);
    if (err) return err;
    const size_t vb = sizeof(int64_t) * count * c->N;
    DevBuf du(c, vb, &err), d0(c, vb, &err), d1(c, vb, &err), dm(c, vb, &err);
    if (err) return fhe_fail(c, err, "encrypt: out of memory");
    cudaMemcpyAsync(du.p, u, vb, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d0.p, e0, vb, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d1.p, e1, vb, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(dm.p, m.data(), vb, cudaMemcpyHostToDevice, c->stream);
    fhe_ct *ct = nullptr;
    if ((err = encrypt_dev(c, pk, dm.i(), du.i(), d0.i(), d1.i(), count, &ct))) return err;
    if ((err = sync_check(c, "encrypt"))) {
        fhe_ct_destroy(ct);
        return err;
    }
    *out = ct;
    return 0;
}

extern "C" int fhe_decrypt_ext(fhe_ctx *c, const fhe_sk *sk, const fhe_ct *ct, int d, uint64_t *digits)
{
    FHE_RANGE("fhe_decrypt_ext");
    CHECK_CTX(c);
    if (!sk || !ct || !digits || ct->npoly != 2 || d < 1) return FHE_EINVAL;
    LOCK(c);
    int err = 0;
    const ExtTables *T = ext_tables(c, d, &err);
    if (!T) return err;
    const int N = c->N, count = ct->count;
    DevBuf dm(c, sizeof(int64_t) * count * N, &err);
    if (err) return fhe_fail(c, err, "decrypt: out of memory");
    if ((err = decrypt_coeffs_dev(c, sk, ct, dm.i()))) return err;
    std::vector<int64_t> m((size_t)count * N);
    cudaMemcpyAsync(m.data(), dm.p, sizeof(int64_t) * m.size(), cudaMemcpyDeviceToHost, c->stream);
    if ((err = sync_check(c, "decrypt"))) return err;
    for (int i = 0; i < count; i++)
        if (!ext_decode(c, T, m.data() + (size_t)i * N, digits + (size_t)i * c->ns * d))
            return fhe_fail(c, FHE_EINVAL, "decrypt: plaintext is not an F_(p^d) slot encoding");
    return 0;
}

// Refresh (a stand-in for bootstrapping, which the paper does not cover): the
// plaintext of every ciphertext is recovered with the secret key on the
// device and encrypted again at the top level with fresh randomness.
static int refresh_dev(fhe_ctx *c, const fhe_sk *sk, const fhe_pk *pk, const fhe_ct *ct, const int64_t *du,
                       const int64_t *d0, const int64_t *d1, fhe_ct **out)
{
    int err = 0;
    DevBuf dm(c, sizeof(int64_t) * ct->count * c->N, &err);
    if (err) return fhe_fail(c, err, "refresh: out of memory");
    if ((err = decrypt_coeffs_dev(c, sk, ct, dm.i()))) return err;
    return encrypt_dev(c, pk, dm.i(), du, d0, d1, ct->count, out);
}

extern "C" int fhe_refresh_explicit(fhe_ctx *c, const fhe_sk *sk, const fhe_pk *pk, const fhe_ct *ct,
                                    const int64_t *u, const int64_t *e0, const int64_t *e1, fhe_ct **out)
{
    CHECK_CTX(c);
    if (!sk || !pk || !ct || ct->npoly != 2 || !u || !e0 || !e1 || !out) return FHE_EINVAL;
    LOCK(c);
    const size_t vb = sizeof(int64_t) * ct->count * c->N;
    int err = 0;
    DevBuf du(c, vb, &err), d0(c, vb, &err), d1(c, vb, &err);
    if (err) return fhe_fail(c, err, "refresh: out of memory");
    cudaMemcpyAsync(du.p, u, vb, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d0.p, e0, vb, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d1.p, e1, vb, cudaMemcpyHostToDevice, c->stream);
    if ((err = refresh_dev(c, sk, pk, ct, du.i(), d0.i(), d1.i(), out))) return err;
    return sync_check(c, "refresh");
}

int refresh_seeded(fhe_ctx *c, const fhe_sk *sk, const fhe_pk *pk, const fhe_ct *ct, uint64_t seed, fhe_ct **out)
{
    const long long n = (long long)ct->count * c->N;
    int err = 0;
    DevBuf du(c, sizeof(int64_t) * n, &err), d0(c, sizeof(int64_t) * n, &err), d1(c, sizeof(int64_t) * n, &err);
    if (err) return fhe_fail(c, err, "refresh: out of memory");
    sample_ternary(c, du.i(), n, seed, TAG_U);
    sample_gaussian(c, d0.i(), n, seed, TAG_E0);
    sample_gaussian(c, d1.i(), n, seed, TAG_E1);
    return refresh_dev(c, sk, pk, ct, du.i(), d0.i(), d1.i(), out);
}

extern "C" int fhe_refresh(fhe_ctx *c, const fhe_sk *sk, const fhe_pk *pk, const fhe_ct *ct, uint64_t seed,
                           fhe_ct **out)
{
    FHE_RANGE("fhe_refresh");
    CHECK_CTX(c);
    if (!sk || !pk || !ct || ct->npoly != 2 || !out) return FHE_EINVAL;
    LOCK(c);
    int err = refresh_seeded(c, sk, pk, ct, seed, out);
    return err ? err : fhe_cuda_check(c, cudaGetLastError(), "refresh");
}

extern "C" int fhe_ct_load_coeff(fhe_ctx *c, fhe_ct *ct, const uint64_t *host)
{
    CHECK_CTX(c);
    if (!ct || ct->ctx != c || !host) return FHE_EINVAL;
    LOCK(c);
    cudaMemcpyAsync(ct->d, host, ct->bytes, cudaMemcpyHostToDevice, c->stream);
    ntt_blocks(c, ct->d, ct->d, ct->count * ct->npoly, ct->level, 0, false);
    return fhe_cuda_check(c, cudaGetLastError(), "load_coeff");
}

extern "C" void fhe_ct_destroy(fhe_ct *ct)
{
    if (!ct) return;
    if (ct->d) ct->ctx->pool.put(ct->d);
    delete ct;
}

extern "C" int fhe_ct_shape(const fhe_ct *ct, int *count, int *npoly, int *level)
{
    if (!ct) return FHE_EINVAL;
    if (count) *count = ct->count;
    if (npoly) *npoly = ct->npoly;
    if (level) *level = ct->level;
    return 0;
}

extern "C" int fhe_ct_export_coeff(fhe_ctx *c, const fhe_ct *ct, uint64_t *host)
{
    CHECK_CTX(c);
    if (!ct || !host) return FHE_EINVAL;
    LOCK(c);
    int err = 0;
    DevBuf t(c, ct->bytes, &err);
    if (err) return fhe_fail(c, err, "export: out of memory");
    ntt_blocks(c, ct->d, t.u(), ct->count * ct->npoly, ct->level, 0, true);
    cudaMemcpyAsync(host, t.p, ct->bytes, cudaMemcpyDeviceToHost, c->stream);
    return sync_check(c, "export");
}

extern "C" int fhe_ct_import_coeff(fhe_ctx *c, const uint64_t *host, int count, int npoly, int level, fhe_ct **out)
{
    CHECK_CTX(c);
    if (!host || !out || count < 1 || npoly < 2 || npoly > 3 || level < 1 || level > c->L) return FHE_EINVAL;
    LOCK(c);
    int err = 0;
    fhe_ct *ct = ct_new(c, count, npoly, level, &err);
    if (!ct) return err;
    cudaMemcpyAsync(ct->d, host, ct->bytes, cudaMemcpyHostToDevice, c->stream);
    ntt_blocks(c, ct->d, ct->d, count * npoly, level, 0, false);
    int r = sync_check(c, "import");
    if (r) {
        fhe_ct_destroy(ct);
        return r;
    }
    *out = ct;
    return 0;
}

// Checkpoint image of a ciphertext batch: a fixed header, the level's primes,
// then the coefficient-domain limbs [count][npoly][level][N] (u64 residues).
namespace {
struct CtImage {
    char magic[4];  // "FHEC"
    uint32_t version, log_n, npoly, count, level;
    uint64_t p;
};
static_assert(sizeof(CtImage) == 32, "image header layout");
}  // namespace

extern "C" int fhe_ct_serialize(fhe_ctx *c, const fhe_ct *ct, void *buf, uint64_t cap, uint64_t *size)
{
    CHECK_CTX(c);
    if (!ct || ct->ctx != c || !size) return FHE_EINVAL;
    const uint64_t need = sizeof(CtImage) + 8ull * ct->level + (uint64_t)ct->bytes;
    *size = need;
    if (!buf) return 0;
    if (cap < need) return fhe_fail(c, FHE_EINVAL, "serialize: buffer smaller than the image");
    CtImage h;
    memcpy(h.magic, "FHEC", 4);
    h.version = 1;
    h.log_n = (uint32_t)c->logN;
    h.npoly = (uint32_t)ct->npoly;
    h.count = (uint32_t)ct->count;
    h.level = (uint32_t)ct->level;
    h.p = c->p;
    char *o = (char *)buf;
    memcpy(o, &h, sizeof h);
    for (int i = 0; i < ct->level; i++) memcpy(o + sizeof h + 8 * i, &c->q[i], 8);
    return fhe_ct_export_coeff(c, ct, (uint64_t *)(o + sizeof h + 8ull * ct->level));
}

extern "C" int fhe_ct_deserialize(fhe_ctx *c, const void *buf, uint64_t size, fhe_ct **out)
{
    CHECK_CTX(c);
    if (!buf || !out || size < sizeof(CtImage)) return FHE_EINVAL;
    CtImage h;
    memcpy(&h, buf, sizeof h);
    if (memcmp(h.magic, "FHEC", 4) || h.version != 1) return fhe_fail(c, FHE_EINVAL, "deserialize: not an image");
    if ((int)h.log_n != c->logN || h.p != c->p || h.npoly < 2 || h.npoly > 3 || h.count < 1 || h.level < 1 ||
        (int)h.level > c->L)
        return fhe_fail(c, FHE_EMISMATCH, "deserialize: image of another ring, plaintext modulus or level");
    const uint64_t words = (uint64_t)h.count * h.npoly * h.level * (uint64_t)c->N;
    if (size != sizeof h + 8ull * h.level + 8 * words) return fhe_fail(c, FHE_EINVAL, "deserialize: size mismatch");
    const char *in = (const char *)buf;
    for (uint32_t i = 0; i < h.level; i++) {
        uint64_t q;
        memcpy(&q, in + sizeof h + 8 * i, 8);
        if (q != c->q[i]) return fhe_fail(c, FHE_EMISMATCH, "deserialize: image of another prime chain");
    }
    std::vector<uint64_t> limbs(words);
    memcpy(limbs.data(), in + sizeof h + 8ull * h.level, 8 * words);
    const uint64_t N = (uint64_t)c->N;
    for (uint64_t w = 0; w < words; w++)
        if (limbs[w] >= c->q[(w / N) % h.level]) return fhe_fail(c, FHE_EINVAL, "deserialize: residue out of range");
    return fhe_ct_import_coeff(c, limbs.data(), (int)h.count, (int)h.npoly, (int)h.level, out);
}

// ---------------------------------------------------------------------------
// arithmetic
// ---------------------------------------------------------------------------

namespace {

int same_ctx(fhe_ctx *c, const fhe_ct *a) { return a && a->ctx == c; }

// Align two batches to the lower level (temporaries owned by the caller).
int align2(fhe_ctx *c, const fhe_ct *a, const fhe_ct *b, const fhe_ct **a2, const fhe_ct **b2, fhe_ct **ta,
           fhe_ct **tb)
{
    *ta = *tb = nullptr;
    *a2 = a;
    *b2 = b;
    if (a->level > b->level) {
        int e = op_lower(c, a, b->level, ta);
        if (e) return e;
        *a2 = *ta;
    } else if (b->level > a->level) {
        int e = op_lower(c, b, a->level, tb);
        if (e) return e;
        *b2 = *tb;
    }
    return 0;
}

int launch_status(fhe_ctx *c, const char *where) { return fhe_cuda_check(c, cudaGetLastError(), where); }

}  // namespace

extern "C" int fhe_add(fhe_ctx *c, const fhe_ct *a, const fhe_ct *b, fhe_ct **out)
{
    CHECK_CTX(c);
    if (!same_ctx(c, a) || !same_ctx(c, b) || !out) return FHE_EINVAL;
    LOCK(c);
    const fhe_ct *a2, *b2;
    fhe_ct *ta, *tb;
    int e = align2(c, a, b, &a2, &b2, &ta, &tb);
    if (!e) e = op_addsub(c, a2, b2, 0, out);
    fhe_ct_destroy(ta);
    fhe_ct_destroy(tb);
    return e ? e : launch_status(c, "add");
}

extern "C" int fhe_sub(fhe_ctx *c, const fhe_ct *a, const fhe_ct *b, fhe_ct **out)
{
    CHECK_CTX(c);
    if (!same_ctx(c, a) || !same_ctx(c, b) || !out) return FHE_EINVAL;
    LOCK(c);
    const fhe_ct *a2, *b2;
    fhe_ct *ta, *tb;
    int e = align2(c, a, b, &a2, &b2, &ta, &tb);
    if (!e) e = op_addsub(c, a2, b2, 1, out);
    fhe_ct_destroy(ta);
    fhe_ct_destroy(tb);
    return e ? e : launch_status(c, "sub");
}

extern "C" int fhe_neg(fhe_ctx *c, const fhe_ct *a, fhe_ct **out)
{
    CHECK_CTX(c);
    if (!same_ctx(c, a) || !out) return FHE_EINVAL;
    LOCK(c);
    int e = op_neg(c, a, out);
    return e ? e : launch_status(c, "neg");
}

extern "C" int fhe_mul_const(fhe_ctx *c, const fhe_ct *a, int64_t k, fhe_ct **out)
{
    CHECK_CTX(c);
    if (!same_ctx(c, a) || !out) return FHE_EINVAL;
    LOCK(c);
    int e = op_mul_const(c, a, k, out);
    return e ? e : launch_status(c, "mul_const");
}

extern "C" int fhe_add_const(fhe_ctx *c, const fhe_ct *a, int64_t k, fhe_ct **out)
{
    CHECK_CTX(c);
    if (!same_ctx(c, a) || !out) return FHE_EINVAL;
    LOCK(c);
    int e = op_add_const(c, a, k, out);
    return e ? e : launch_status(c, "add_const");
}

extern "C" int fhe_mul(fhe_ctx *c, const fhe_ct *a, const fhe_ct *b, fhe_ct **out)
{
    FHE_RANGE("fhe_mul");
    CHECK_CTX(c);
    if (!same_ctx(c, a) || !same_ctx(c, b) || !out) return FHE_EINVAL;
    LOCK(c);
    const fhe_ct *a2, *b2;
    fhe_ct *ta, *tb;
    int e = align2(c, a, b, &a2, &b2, &ta, &tb);
    if (!e) e = op_tensor(c, a2, b2, out);
    fhe_ct_destroy(ta);
    fhe_ct_destroy(tb);
    return e ? e : launch_status(c, "mul");
}

extern "C" int fhe_relinearize(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *a, fhe_ct **out)
{
    FHE_RANGE("fhe_relinearize");
    CHECK_CTX(c);
    if (!evk || evk->ctx != c || !same_ctx(c, a) || !out) return FHE_EINVAL;
    LOCK(c);
    int e = op_relin(c, evk->keys[0], a, out);
    return e ? e : launch_status(c, "relinearize");
}

extern "C" int fhe_mod_switch(fhe_ctx *c, const fhe_ct *a, int target_level, fhe_ct **out)
{
    FHE_RANGE("fhe_mod_switch");
    CHECK_CTX(c);
    if (!same_ctx(c, a) || !out) return FHE_EINVAL;
    LOCK(c);
    int e = op_lower(c, a, target_level, out);
    return e ? e : launch_status(c, "mod_switch");
}

extern "C" int fhe_rotate(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *a, int64_t galois, fhe_ct **out)
{
    FHE_RANGE("fhe_rotate");
    CHECK_CTX(c);
    if (!evk || evk->ctx != c || !same_ctx(c, a) || !out) return FHE_EINVAL;
    LOCK(c);
    const KeySwitchKey *k = evk->find(galois);
    if (!k || galois == 0) return fhe_fail(c, FHE_ENOKEY, "no rotation key for this Galois element");
    int e = op_rotate(c, *k, a, out);
    if (!e && c->tracing) {
        c->trace_op.push_back(FHE_OP_ROT);
        c->trace_level.push_back(a->level);
    }
    return e ? e : launch_status(c, "rotate");
}

extern "C" int fhe_mul_relin(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *a, const fhe_ct *b, fhe_ct **out)
{
    FHE_RANGE("fhe_mul_relin");
    CHECK_CTX(c);
    if (!evk || evk->ctx != c || !same_ctx(c, a) || !same_ctx(c, b) || !out) return FHE_EINVAL;
    LOCK(c);
    const fhe_ct *a2, *b2;
    fhe_ct *ta, *tb;
    int e = align2(c, a, b, &a2, &b2, &ta, &tb);
    if (!e) e = op_mul_relin(c, evk->keys[0], a2, b2, out);
    fhe_ct_destroy(ta);
    fhe_ct_destroy(tb);
    return e ? e : launch_status(c, "mul_relin");
}

// ---------------------------------------------------------------------------
// comparison
// ---------------------------------------------------------------------------

namespace {

int check_digits(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d)
{
    if (!evk || evk->ctx != c || !x || !y || d < 1) return FHE_EINVAL;
    const int count = x[0] ? x[0]->count : 0;
    for (int k = 0; k < d; k++) {
        if (!same_ctx(c, x[k]) || !same_ctx(c, y[k])) return FHE_EINVAL;
        if (x[k]->count != count || y[k]->count != count || x[k]->npoly != 2 || y[k]->npoly != 2)
            return fhe_fail(c, FHE_EMISMATCH, "comparison operands differ in shape");
    }
    return 0;
}

}  // namespace

extern "C" int fhe_compare(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                           fhe_ct **lt, fhe_ct **eq)
{
    FHE_RANGE("fhe_compare");
    CHECK_CTX(c);
    int e = check_digits(c, evk, x, y, d);
    if (e) return e;
    if (!lt && !eq) return FHE_EINVAL;
    LOCK(c);
    e = circuit_compare(c, evk, x, y, d, lt, eq);
    return e ? e : launch_status(c, "compare");
}

extern "C" int fhe_compare_bivariate(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x,
                                     const fhe_ct *const *y, int d, fhe_ct **lt, fhe_ct **eq)
{
    FHE_RANGE("fhe_compare_bivariate");
    CHECK_CTX(c);
    int e = check_digits(c, evk, x, y, d);
    if (e) return e;
    if (!lt && !eq) return FHE_EINVAL;
    LOCK(c);
    e = circuit_compare_bv(c, evk, x, y, d, lt, eq);
    return e ? e : launch_status(c, "compare_bivariate");
}

static int plain_api(fhe_ctx *c, const fhe_ct *a, const uint64_t *slots, int kind, fhe_ct **out)
{
    CHECK_CTX(c);
    if (!same_ctx(c, a) || !slots || !out) return FHE_EINVAL;
    for (int i = 0; i < c->ns; i++)
        if (slots[i] >= c->p) return fhe_fail(c, FHE_EINVAL, "plaintext slot value not below p");
    LOCK(c);
    const int e = op_plain(c, a, slots, kind, out);
    return e ? e : launch_status(c, "plaintext operation");
}

extern "C" int fhe_add_plain(fhe_ctx *c, const fhe_ct *a, const uint64_t *slots, fhe_ct **out)
{
    FHE_RANGE("fhe_add_plain");
    return plain_api(c, a, slots, 0, out);
}

extern "C" int fhe_sub_plain(fhe_ctx *c, const fhe_ct *a, const uint64_t *slots, fhe_ct **out)
{
    FHE_RANGE("fhe_sub_plain");
    return plain_api(c, a, slots, 1, out);
}

extern "C" int fhe_mul_plain(fhe_ctx *c, const fhe_ct *a, const uint64_t *slots, fhe_ct **out)
{
    FHE_RANGE("fhe_mul_plain");
    return plain_api(c, a, slots, 2, out);
}

extern "C" int fhe_extract_digits(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *a, int d, fhe_ct **out)
{
    FHE_RANGE("fhe_extract_digits");
    CHECK_CTX(c);
    if (!evk || evk->ctx != c || !same_ctx(c, a) || a->npoly != 2 || !out || d < 1) return FHE_EINVAL;
    LOCK(c);
    int err = 0;
    const ExtTables *T = ext_tables(c, d, &err);
    if (!T) return err;
    for (int64_t g : T->galois)
        if (!evk->find(g)) return fhe_fail(c, FHE_ENOKEY, "extract: missing Frobenius key");
    if ((err = circuit_extract(c, evk, a, T, out))) return err;
    return launch_status(c, "extract");
}

extern "C" int fhe_private_query(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *q, const fhe_ct *data,
                                 const fhe_ct *op1, int op2, const int64_t *codes, int flags, fhe_ct **out)
{
    FHE_RANGE("fhe_private_query");
    CHECK_CTX(c);
    if (!evk || evk->ctx != c || !same_ctx(c, q) || !same_ctx(c, data) || !same_ctx(c, op1) || !codes || !out ||
        op2 < 1 || op2 >= (1 << 20) || (flags & ~FHE_QUERY_OVERLAP))
        return FHE_EINVAL;
    if (q->npoly != 2 || data->npoly != 2 || op1->npoly != 2 || q->count != data->count || op1->count != data->count)
        return fhe_fail(c, FHE_EMISMATCH, "private query: operands differ in shape");
    LOCK(c);
    const int e = circuit_private_query(c, evk, q, data, op1, op2, codes, (flags & FHE_QUERY_OVERLAP) != 0, out);
    return e ? e : launch_status(c, "private_query");
}

extern "C" int fhe_slot_plan(int slots, int64_t ring_n, int n, const uint8_t *useful, int32_t *dest,
                             int64_t *galois, int galois_cap, int *n_galois)
{
    if (slots < 1 || (slots > 1 && slots % 2) || ring_n < slots || ring_n > (1 << 20) || (ring_n & (ring_n - 1)))
        return FHE_EINVAL;
    if (n < 0 || (n && !useful) || galois_cap < 0 || (galois_cap && !galois)) return FHE_EINVAL;
    std::vector<SlotPiece> pieces;
    std::vector<int32_t> d;
    const int n_out = slot_plan(slots, n, useful, pieces, dest ? &d : nullptr);
    if (dest) std::copy(d.begin(), d.end(), dest);
    const std::vector<int64_t> g = slot_galois(slots, ring_n, pieces);
    for (int i = 0; i < (int)g.size() && i < galois_cap; i++) galois[i] = g[i];
    if (n_galois) *n_galois = (int)g.size();
    return n_out;
}

extern "C" int fhe_slot_pack(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *in, int n, const uint8_t *useful,
                             fhe_ct **out, int out_cap)
{
    FHE_RANGE("fhe_slot_pack");
    CHECK_CTX(c);
    if (!evk || evk->ctx != c || !in || n < 1 || !useful || !out || out_cap < 0) return FHE_EINVAL;
    for (int j = 0; j < n; j++) {
        if (!same_ctx(c, in[j])) return FHE_EINVAL;
        if (in[j]->npoly != 2 || in[j]->count != in[0]->count)
            return fhe_fail(c, FHE_EMISMATCH, "slot_pack: inputs differ in shape");
    }
    std::vector<SlotPiece> pieces;
    const int n_out = slot_plan(c->ns, n, useful, pieces, nullptr);
    if (n_out > out_cap) return fhe_fail(c, FHE_EINVAL, "slot_pack: more outputs than out_cap");
    if (n_out == 0) return 0;
    for (int64_t g : slot_galois(c->ns, c->N, pieces))
        if (!evk->find(g)) return fhe_fail(c, FHE_ENOKEY, "slot_pack: missing rotation key");
    LOCK(c);
    const int e = circuit_slot_pack(c, evk, in, n, useful, out, n_out);
    if (e) return e;
    const int st = launch_status(c, "slot_pack");
    return st ? st : n_out;
}

extern "C" int fhe_sort_galois(const fhe_ctx *c, int64_t *galois, int cap)
{
    if (!c || cap < 0) return FHE_EINVAL;
    const std::vector<int64_t> g = sort_galois(c);
    for (int i = 0; i < (int)g.size() && i < cap; i++) galois[i] = g[i];
    return (int)g.size();
}

extern "C" int fhe_sort(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, int d, fhe_ct **out)
{
    FHE_RANGE("fhe_sort");
    CHECK_CTX(c);
    if (!out) return FHE_EINVAL;
    int e = check_digits(c, evk, x, x, d);
    if (e) return e;
    LOCK(c);
    e = circuit_sort(c, evk, x, d, out);
    return e ? e : launch_status(c, "sort");
}

extern "C" int fhe_sort_joint(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, int K, int d, fhe_ct **out)
{
    FHE_RANGE("fhe_sort_joint");
    CHECK_CTX(c);
    if (!out || !x || K < 1 || d < 1) return FHE_EINVAL;
    int e = check_digits(c, evk, x, x, d);
    if (e) return e;
    for (int i = 0; i < K * d; i++) {
        if (!same_ctx(c, x[i])) return FHE_EINVAL;
        if (x[i]->npoly != 2 || x[i]->count != x[0]->count || x[i]->level != x[0]->level)
            return fhe_fail(c, FHE_EMISMATCH, "joint sort: inputs differ in shape or level");
    }
    LOCK(c);
    e = circuit_sort_joint(c, evk, x, K, d, out);
    return e ? e : launch_status(c, "sort");
}

extern "C" int fhe_sort_ranks(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, int K, int d, fhe_ct **ranks,
                              fhe_ct **matrix)
{
    FHE_RANGE("fhe_sort_ranks");
    CHECK_CTX(c);
    if (!ranks || !x || K < 1 || d < 1) return FHE_EINVAL;
    int e = check_digits(c, evk, x, x, d);
    if (e) return e;
    for (int i = 0; i < K * d; i++) {
        if (!same_ctx(c, x[i])) return FHE_EINVAL;
        if (x[i]->npoly != 2 || x[i]->count != x[0]->count || x[i]->level != x[0]->level)
            return fhe_fail(c, FHE_EMISMATCH, "sort ranks: inputs differ in shape or level");
    }
    LOCK(c);
    e = circuit_sort_ranks(c, evk, x, K, d, ranks, matrix);
    return e ? e : launch_status(c, "sort ranks");
}

extern "C" int fhe_compare_lt(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                              fhe_ct **out)
{
    if (!out) return FHE_EINVAL;
    return fhe_compare(c, evk, x, y, d, out, nullptr);
}

extern "C" int fhe_compare_eq(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                              fhe_ct **out)
{
    if (!out) return FHE_EINVAL;
    return fhe_compare(c, evk, x, y, d, nullptr, out);
}

extern "C" int fhe_max_min(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                           fhe_ct **out_max, fhe_ct **out_min)
{
    FHE_RANGE("fhe_max_min");
    CHECK_CTX(c);
    int e = check_digits(c, evk, x, y, d);
    if (e) return e;
    if (!out_max && !out_min) return FHE_EINVAL;
    LOCK(c);
    e = circuit_max_min(c, evk, x, y, d, out_max, out_min);
    return e ? e : launch_status(c, "max_min");
}

extern "C" int fhe_max(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                       fhe_ct **out)
{
    if (!out) return FHE_EINVAL;
    return fhe_max_min(c, evk, x, y, d, out, nullptr);
}

extern "C" int fhe_min(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                       fhe_ct **out)
{
    if (!out) return FHE_EINVAL;
    return fhe_max_min(c, evk, x, y, d, nullptr, out);
}

// ---------------------------------------------------------------------------
// trace, raw transforms, self test
// ---------------------------------------------------------------------------

extern "C" int fhe_trace_enable(fhe_ctx *c, int on)
{
    CHECK_CTX(c);
    LOCK(c);
    c->tracing = on != 0;
    c->trace_op.clear();
    c->trace_level.clear();
    return 0;
}

extern "C" int fhe_trace_get(const fhe_ctx *c, int32_t *ops, int32_t *levels, int cap)
{
    if (!c || cap < 0) return FHE_EINVAL;
    const int n = (int)c->trace_op.size();
    for (int i = 0; i < n && i < cap; i++) {
        if (ops) ops[i] = c->trace_op[i];
        if (levels) levels[i] = c->trace_level[i];
    }
    return n;
}

static int raw_ntt(fhe_ctx *c, uint64_t *data, const int32_t *prime_idx, int nlimbs, bool inverse)
{
    CHECK_CTX(c);
    if (!data || !prime_idx || nlimbs < 0) return FHE_EINVAL;
    LOCK(c);
    for (int i = 0; i < nlimbs; i++)
        if (prime_idx[i] < 0 || prime_idx[i] >= c->np) return FHE_EINVAL;
    for (int base = 0; base < nlimbs; base += FHE_MAXP) {
        const int n = std::min(FHE_MAXP, nlimbs - base);
        LimbMap m;
        memset(&m, 0, sizeof(m));
        m.nl = n;
        for (int i = 0; i < n; i++) m.in_limb[i] = m.out_limb[i] = i, m.prime[i] = prime_idx[base + i];
        u64 *p = data + (size_t)base * c->N;
        if (inverse)
            launch_ntt_inv_plain(c, p, p, m, n);
        else
            launch_ntt_fwd_plain(c, p, p, m, n);
    }
    return launch_status(c, "ntt");
}

static int raw_ntt_batch(fhe_ctx *c, uint64_t *data, int count, int nprimes, bool inverse)
{
    CHECK_CTX(c);
    if (!data || count < 1 || nprimes < 1 || nprimes > c->np) return FHE_EINVAL;
    LOCK(c);
    LimbMap m;
    memset(&m, 0, sizeof(m));
    m.nl = nprimes;
    m.in_outer = m.out_outer = (long long)nprimes * c->N;
    for (int i = 0; i < nprimes; i++) m.in_limb[i] = m.out_limb[i] = m.prime[i] = i;
    if (inverse)
        launch_ntt_inv_plain(c, data, data, m, count * nprimes);
    else
        launch_ntt_fwd_plain(c, data, data, m, count * nprimes);
    return launch_status(c, "ntt batch");
}

extern "C" int fhe_ntt_forward_batch(fhe_ctx *c, uint64_t *data, int count, int nprimes)
{
    FHE_RANGE("fhe_ntt_forward_batch");
    return raw_ntt_batch(c, data, count, nprimes, false);
}

extern "C" int fhe_ntt_inverse_batch(fhe_ctx *c, uint64_t *data, int count, int nprimes)
{
    FHE_RANGE("fhe_ntt_inverse_batch");
    return raw_ntt_batch(c, data, count, nprimes, true);
}

extern "C" int fhe_ntt_forward(fhe_ctx *c, uint64_t *data, const int32_t *prime_idx, int nlimbs)
{
    return raw_ntt(c, data, prime_idx, nlimbs, false);
}

extern "C" int fhe_ntt_inverse(fhe_ctx *c, uint64_t *data, const int32_t *prime_idx, int nlimbs)
{
    return raw_ntt(c, data, prime_idx, nlimbs, true);
}

extern "C" int fhe_selftest_modarith(uint64_t prime_mod, uint64_t prime_lo, uint64_t prime_hi, int nprimes, int iters)
{
    if (nprimes < 1 || nprimes > 64 || iters < 0) return -1;
    std::vector<u64> qs(nprimes);
    if (host_find_primes(prime_mod, prime_lo, prime_hi, nprimes, qs.data()) != nprimes) return -1;
    int bad = 0;
    u64 st = 0x9E3779B97F4A7C15ull;
    auto rnd = [&st]() {  // splitmix64
        u64 z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (u64 q : qs) {
        const ModQ m = make_modq(q);
        for (int it = 0; it < iters; it++) {
            const bool edge = it < 64;
            u64 a[8], b[8];
            for (int k = 0; k < 8; k++) {
                a[k] = edge ? q - 1 - (u64)((it >> k) & 1) : rnd() % q;
                b[k] = edge ? q - 1 - (u64)((it >> (k + 1)) & 1) : rnd() % q;
            }
            // single and summed products
            u128 acc = 0;
            for (int k = 0; k < 8; k++) {
                acc += (u128)a[k] * b[k];
                if (barrett128(acc, m) != (u64)(acc % q)) bad++;
                const u64 bl = barrett128_lazy(acc, m);
                if (bl >= 3 * q || bl % q != (u64)(acc % q)) bad++;
                if (mulmod(a[k], b[k], m) != (u64)(((u128)a[k] * b[k]) % q)) bad++;
            }
            // Shoup with any 64-bit multiplicand
            const u64 w = b[0], ws = shoup_const(w, q), x = edge ? ~0ull - (u64)it : rnd();
            const u64 lz = shoup_lazy(x, w, ws, q);
            if (lz >= 2 * q || lz % q != (u64)(((u128)x * w) % q)) bad++;
            const u64 l4 = shoup_lazy4(x, w, ws, q);
            if (l4 >= 4 * q || l4 % q != (u64)(((u128)x * w) % q)) bad++;
            if (shoup_lazy4_chain(x, w, ws, 0 - q) != l4) bad++;
            if (shoup(x, w, ws, q) != (u64)(((u128)x * w) % q)) bad++;
            if (reduce4q(4 * q - 1 - (x % (4 * q)), 2 * q, q) != (4 * q - 1 - (x % (4 * q))) % q) bad++;
            const u64 v = edge ? (it < 32 ? ~0ull - (u64)it : 31 * q - 1 - (u64)it) : rnd();
            if (reduce64(v, m) != v % q) bad++;
        }
    }
    return bad;
}

// ---------------------------------------------------------------------------
// captured comparison plans (CUDA graphs)
// ---------------------------------------------------------------------------

// Records a circuit into a CUDA graph.  run(o0, o1) enqueues the circuit and
// writes its result handles; it is called once uncaptured (the warm run fills
// the pool with every block size the circuit needs and builds any lazily
// created table, so the captured run allocates nothing) and once under
// capture, whose results become the plan's outputs.
static int capture_plan(fhe_ctx *c, int flags, const std::function<int(fhe_ct **, fhe_ct **)> &run, fhe_plan **out)
{
    const bool prof = c->prof_on, tr = c->tracing;
    c->prof_on = false;
    c->tracing = false;
    int e;
    {
        fhe_ct *o0 = nullptr, *o1 = nullptr;
        e = run(&o0, &o1);
        fhe_ct_destroy(o0);
        fhe_ct_destroy(o1);
        if (!e) e = sync_check(c, "plan warm-up");
        if (e) {
            c->prof_on = prof;
            c->tracing = tr;
            return e;
        }
    }
    fhe_plan *P = new fhe_plan;
    P->ctx = c;
    // with profiling on, the per-kernel event pairs become event-record nodes
    // of the graph and hold the times of the latest replay
    c->prof_on = prof;
    c->pool.cap_free = &P->held;
    c->pool.in_capture = true;
    // record on a private stream (the legacy NULL stream cannot be captured);
    // the graph is launched on the context's stream, whatever it is
    cudaStream_t user = c->stream, cap = nullptr;
    e = fhe_cuda_check(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
    if (!e) {
        c->stream = cap;
        c->pool.stream = cap;
        e = fhe_cuda_check(c, cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed), "begin capture");
        if (!e) {
            c->capturing = !(flags & FHE_PLAN_SERIAL);
            e = run(&P->out[0], &P->out[1]);
            c->capturing = false;
            cudaGraph_t g = nullptr;
            const int e2 = fhe_cuda_check(c, cudaStreamEndCapture(cap, &g), "end capture");
            if (!e) e = e2;
            P->graph = g;
        }
        c->stream = user;
        c->pool.stream = user;
        cudaStreamDestroy(cap);
    }
    c->pool.cap_free = nullptr;
    c->pool.in_capture = false;
    c->prof_on = prof;
    c->tracing = tr;
    if (!e) e = fhe_cuda_check(c, cudaGraphInstantiate(&P->exec, P->graph, 0), "graph instantiate");
    if (!e) {
        size_t n = 0;
        cudaGraphGetNodes(P->graph, nullptr, &n);
        P->nodes = (int)n;
    }
    if (e) {
        fhe_plan_destroy(P);
        return e;
    }
    *out = P;
    return 0;
}

extern "C" int fhe_compare_plan(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y,
                                int d, int want_lt, int want_eq, int flags, fhe_plan **out)
{
    FHE_RANGE("fhe_compare_plan");
    CHECK_CTX(c);
    if (!out || (!want_lt && !want_eq) || (flags & ~(FHE_PLAN_SERIAL | FHE_PLAN_BIVARIATE))) return FHE_EINVAL;
    int e = check_digits(c, evk, x, y, d);
    if (e) return e;
    LOCK(c);
    return capture_plan(
        c, flags,
        [&](fhe_ct **lt, fhe_ct **eq) {
            return (flags & FHE_PLAN_BIVARIATE)
                       ? circuit_compare_bv(c, evk, x, y, d, want_lt ? lt : nullptr, want_eq ? eq : nullptr)
                       : circuit_compare(c, evk, x, y, d, want_lt ? lt : nullptr, want_eq ? eq : nullptr);
        },
        out);
}

extern "C" int fhe_private_query_plan(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *q, const fhe_ct *data,
                                      const fhe_ct *op1, int op2, const int64_t *codes, int flags, fhe_plan **out)
{
    FHE_RANGE("fhe_private_query_plan");
    CHECK_CTX(c);
    if (!evk || evk->ctx != c || !same_ctx(c, q) || !same_ctx(c, data) || !same_ctx(c, op1) || !codes || !out ||
        op2 < 1 || op2 >= (1 << 20) || (flags & ~FHE_PLAN_SERIAL))
        return FHE_EINVAL;
    if (q->npoly != 2 || data->npoly != 2 || op1->npoly != 2 || q->count != data->count || op1->count != data->count)
        return fhe_fail(c, FHE_EMISMATCH, "private query: operands differ in shape");
    const int64_t k[3] = {codes[0], codes[1], codes[2]};
    LOCK(c);
    return capture_plan(
        c, flags,
        [&](fhe_ct **answer, fhe_ct **) {
            return circuit_private_query(c, evk, q, data, op1, op2, k, !(flags & FHE_PLAN_SERIAL), answer);
        },
        out);
}

extern "C" int fhe_plan_run(fhe_plan *P)
{
    FHE_RANGE("fhe_plan_run");
    if (!P || !P->exec) return FHE_EINVAL;
    fhe_ctx *c = P->ctx;
    LOCK(c);
    c->launches += P->nodes;
    return fhe_cuda_check(c, cudaGraphLaunch(P->exec, c->stream), "graph launch");
}

extern "C" int fhe_plan_result(const fhe_plan *P, int which, const fhe_ct **out)
{
    if (!P || !out || which < 0 || which > 1 || !P->out[which]) return FHE_EINVAL;
    *out = P->out[which];
    return 0;
}

extern "C" int fhe_plan_nodes(const fhe_plan *P) { return P ? P->nodes : FHE_EINVAL; }

extern "C" void fhe_plan_destroy(fhe_plan *P)
{
    if (!P) return;
    fhe_ctx *c = P->ctx;
    cudaStreamSynchronize(c->stream);
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    for (int i = 0; i < 2; i++) fhe_ct_destroy(P->out[i]);
    for (auto &kv : P->held)
        for (void *p : kv.second) c->pool.put(p);
    delete P;
}

// ---------------------------------------------------------------------------
// tournament
// ---------------------------------------------------------------------------

extern "C" int fhe_tournament_galois(const fhe_ctx *c, int64_t *galois, int cap)
{
    if (!c || cap < 0) return FHE_EINVAL;
    const std::vector<int64_t> g = tournament_galois(c);
    for (int i = 0; i < (int)g.size() && i < cap; i++) galois[i] = g[i];
    return (int)g.size();
}

extern "C" int fhe_tournament(fhe_ctx *c, const fhe_evk *evk, const fhe_sk *sk, const fhe_pk *pk,
                              const fhe_ct *const *x, int d, uint64_t seed, fhe_ct **out_max, fhe_ct **out_min)
{
    FHE_RANGE("fhe_tournament");
    CHECK_CTX(c);
    if (!evk || evk->ctx != c || !x || d < 1 || (!out_max && !out_min)) return FHE_EINVAL;
    for (int k = 0; k < d; k++)
        if (!same_ctx(c, x[k]) || x[k]->npoly != 2 || x[k]->count != x[0]->count || x[k]->level != x[0]->level)
            return fhe_fail(c, FHE_EMISMATCH, "tournament operands differ in shape");
    LOCK(c);
    int e = circuit_tournament(c, evk, sk, pk, x, d, out_max != nullptr, out_min != nullptr, seed, out_max, out_min);
    return e ? e : fhe_cuda_check(c, cudaGetLastError(), "tournament");
}

extern "C" int fhe_ctx_ntt_variant(fhe_ctx *c, int set, float *ms)
{
    CHECK_CTX(c);
    LOCK(c);
    if (set >= 0) {
        if (!ntt_variant_ok(c->logN, set)) return FHE_EINVAL;
        c->ntt_variant = set;
    }
    if (ms)
        for (int v = 0; v < FHE_NTT_VARIANTS; v++) ms[v] = c->ntt_ms[v];
    return c->ntt_variant;
}

extern "C" int fhe_ctx_autotune(fhe_ctx *c, int njobs)
{
    CHECK_CTX(c);
    if (njobs < 1) return FHE_EINVAL;
    LOCK(c);
    int e = ntt_autotune(c, njobs, c->ntt_ms);
    return e ? e : c->ntt_variant;
}
