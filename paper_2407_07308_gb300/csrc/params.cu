// params.cu -- host precomputation: prime chain, NTT twiddles, per-level
// basis-conversion / ModDown / modulus-switching constants, the less-than
// polynomial and the slot structure.  Everything is uploaded once at context
// creation and stays resident on the device.
#include <string.h>

#include <algorithm>

#include "fhe_internal.h"

u64 host_mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }

u64 host_powmod(u64 a, u64 e, u64 q)
{
    u64 r = 1 % q, b = a % q;
    for (; e; e >>= 1, b = host_mulmod(b, b, q))
        if (e & 1) r = host_mulmod(r, b, q);
    return r;
}

u64 host_invmod(u64 a, u64 q) { return host_powmod(a, q - 2, q); }  // q prime

// Deterministic Miller-Rabin for 64-bit n with the seven bases found by
// J. Sinclair (2011), which decide primality for every n < 2^64.
bool host_is_prime(u64 n)
{
    if (n < 2) return false;
    static const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 s : small)
        if (n % s == 0) return n == s;
    static const u64 bases[] = {2, 325, 9375, 28178, 450775, 9780504, 1795265022};
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) d >>= 1, r++;
    for (u64 a : bases) {
        a %= n;
        if (a == 0) continue;
        u64 x = host_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int i = 1; i < r && witness; i++) {
            x = host_mulmod(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

int host_find_primes(u64 U, u64 lo, u64 hi, int count, u64 *out)
{
    int found = 0;
    u64 q = (lo <= 1) ? U + 1 : ((lo - 2) / U + 1) * U + 1;  // smallest kU+1 >= lo
    while (found < count && q < hi) {
        if (host_is_prime(q)) out[found++] = q;
        q += U;
    }
    return found;
}

static u64 smallest_primitive_root(u64 q)
{
    std::vector<u64> f;
    u64 m = q - 1;
    for (u64 d = 2; d * d <= m; d++) {
        if (m % d) continue;
        f.push_back(d);
        while (m % d == 0) m /= d;
    }
    if (m > 1) f.push_back(m);
    for (u64 g = 2;; g++) {
        bool ok = true;
        for (u64 r : f)
            if (host_powmod(g, (q - 1) / r, q) == 1) { ok = false; break; }
        if (ok) return g;
    }
}

static unsigned bit_reverse(unsigned x, int bits)
{
    unsigned r = 0;
    for (int i = 0; i < bits; i++, x >>= 1) r = (r << 1) | (x & 1);
    return r;
}

// LT polynomial by power sums: for f: Z_p -> Z_p with f(0) = 0,
// c_j = -sum_{z=1}^{p-1} f(z) z^{p-1-j} (mod p), 1 <= j <= p-1, because
// sum_{z != 0} z^k is -1 when (p-1) | k and 0 otherwise.  Here f(z) = 1 for
// z in [(p+1)/2, p-1] (the digit difference is "negative"), else 0.
void lt_poly_coefficients(int p, std::vector<int> &out)
{
    out.assign(p, 0);
    for (int j = 1; j < p; j++) {
        u64 s = 0;
        for (int z = (p + 1) / 2; z < p; z++) s += host_powmod(z, p - 1 - j, p);
        out[j] = (int)((p - (s % p)) % p);
    }
}

// Bivariate LT on full digits: c[a p + b] with sum c x^a y^b = [x < y] on
// Z_p x Z_p.  The indicator of the point i is 1 - (Z - i)^(p-1) (Fermat),
// expanded by the binomial theorem; LT = sum_{i<j} 1_i(X) 1_j(Y), summed as
// sum_i 1_i(X) S_{i+1}(Y) with S_k the suffix sums of the indicators.
void lt_bivariate_coefficients(int p, std::vector<int> &out)
{
    const u64 P = (u64)p;
    std::vector<u64> binom(p);  // C(p-1, a) mod p
    binom[0] = 1;
    for (int a = 1; a < p; a++)
        binom[a] = host_mulmod(host_mulmod(binom[a - 1], (P - 1 - (a - 1)) % P, P), host_invmod((u64)a, P), P);
    std::vector<std::vector<u64>> ind(p, std::vector<u64>(p, 0));
    for (int i = 0; i < p; i++) {
        const u64 mi = (P - (u64)i) % P;  // -i
        for (int a = 0; a < p; a++) {
            const u64 t = host_mulmod(binom[a], host_powmod(mi, (u64)(p - 1 - a), P), P);
            ind[i][a] = (P - t) % P;
        }
        ind[i][0] = (ind[i][0] + 1) % P;
    }
    out.assign((size_t)p * p, 0);
    std::vector<u64> suffix(p, 0);
    for (int i = p - 1; i >= 0; i--) {
        for (int a = 0; a < p; a++) {
            if (!ind[i][a]) continue;
            for (int b = 0; b < p; b++)
                if (suffix[b]) out[(size_t)a * p + b] = (int)((out[(size_t)a * p + b] + ind[i][a] * suffix[b]) % P);
        }
        for (int b = 0; b < p; b++) suffix[b] = (suffix[b] + ind[i][b]) % P;
    }
}

static int two_adic(u64 x)
{
    int v = 0;
    while ((x & 1) == 0) x >>= 1, v++;
    return v;
}

static int slot_structure(fhe_ctx *c)
{
    u64 p = c->p;
    if (p % 4 == 1) {
        c->slots_linear = true;
        int M = 1 << (two_adic(p - 1) - 1);
        if (M > c->N) M = c->N;
        c->M = M;
        c->ns = M;
        c->zeta = host_powmod(smallest_primitive_root(p), (p - 1) / (2 * (u64)M), p);
        c->slot_exp.clear();
        int cols = M > 1 ? M / 2 : 1, rows = M > 1 ? 2 : 1;
        for (int r = 0; r < rows; r++)
            for (int col = 0; col < cols; col++) {
                int e = (int)host_powmod(5, col, 2 * M);
                c->slot_exp.push_back(r == 0 ? e : (2 * M - e) % (2 * M));
            }
        return 0;
    }
    if (p % 8 == 3) {
        c->slots_linear = false;
        c->M = 4;
        c->ns = 2;
        for (u64 g = 1; g < p; g++)
            if (host_mulmod(g, g, p) == p - 2) { c->gamma = g; break; }
        return 0;
    }
    return -1;
}

static int upload(fhe_ctx *c, void **dst, const void *src, size_t bytes)
{
    if (cudaMalloc(dst, bytes) != cudaSuccess) return FHE_ENOMEM;
    if (cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return FHE_ECUDA;
    return 0;
}

int build_tables(fhe_ctx *c)
{
    const int N = c->N, np = c->np, L = c->L, K = c->K;
    c->mq.resize(np);
    c->psi.resize(np);
    std::vector<ulonglong2> fwd((size_t)np * N), inv((size_t)np * N), ninv(np);
    for (int i = 0; i < np; i++) {
        u64 q = c->q[i];
        c->mq[i] = make_modq(q);
        u64 g = smallest_primitive_root(q);
        u64 psi = host_powmod(g, (q - 1) / (2 * (u64)N), q), ipsi = host_invmod(psi, q);
        c->psi[i] = psi;
        // psi^k for k < N, then scatter to bit-reversed positions
        std::vector<u64> pw(N), ipw(N);
        pw[0] = ipw[0] = 1;
        for (int k = 1; k < N; k++) {
            pw[k] = host_mulmod(pw[k - 1], psi, q);
            ipw[k] = host_mulmod(ipw[k - 1], ipsi, q);
        }
        for (int k = 0; k < N; k++) {
            u64 w = pw[bit_reverse(k, c->logN)], iw = ipw[bit_reverse(k, c->logN)];
            fwd[(size_t)i * N + k] = make_ulonglong2(w, shoup_const(w, q));
            inv[(size_t)i * N + k] = make_ulonglong2(iw, shoup_const(iw, q));
        }
        u64 ni = host_invmod((u64)N % q, q);
        ninv[i] = make_ulonglong2(ni, shoup_const(ni, q));
    }
    int e;
    if ((e = upload(c, (void **)&c->d_mq, c->mq.data(), sizeof(ModQ) * np))) return e;
    if ((e = upload(c, (void **)&c->d_fwd, fwd.data(), sizeof(ulonglong2) * fwd.size()))) return e;
    if ((e = upload(c, (void **)&c->d_inv, inv.data(), sizeof(ulonglong2) * inv.size()))) return e;
    if ((e = upload(c, (void **)&c->d_ninv, ninv.data(), sizeof(ulonglong2) * np))) return e;

    // P = product of the special primes; per-level constants.
    c->modup.assign(L + 1, ModUpParams());
    c->moddown.assign(L + 1, ModDownParams());
    c->modswitch.assign(L + 1, ModSwitchParams());
    for (int l = 1; l <= L; l++) {
        ModUpParams &U = c->modup[l];
        memset(&U, 0, sizeof(U));
        U.l = l;
        U.K = K;
        U.dnum = (l + K - 1) / K;
        auto eprime = [&](int r) { return r < l ? r : L + (r - l); };  // extended limb -> prime
        for (int j = 0; j < U.dnum; j++) {
            int lo = j * K, n = std::min(K, l - j * K);
            U.digit_lo[j] = lo;
            U.digit_n[j] = n;
            for (int a = 0; a < n; a++) {
                u64 qa = c->q[lo + a], hat_a = 1;
                for (int b = 0; b < n; b++)
                    if (b != a) hat_a = host_mulmod(hat_a, c->q[lo + b] % qa, qa);
                U.inv_hat[j][a] = host_invmod(hat_a, qa);
                U.inv_hat_s[j][a] = shoup_const(U.inv_hat[j][a], qa);
                for (int r = 0; r < l + K; r++) {
                    u64 tq = c->q[eprime(r)], h = 1;
                    for (int b = 0; b < n; b++)
                        if (b != a) h = host_mulmod(h, c->q[lo + b] % tq, tq);
                    U.hat[j][a][r] = h;
                }
            }
            for (int r = 0; r < l + K; r++) {
                if (r >= lo && r < lo + n) continue;
                U.job_digit[U.njobs] = j;
                U.job_tgt[U.njobs] = r;
                U.job_prime[U.njobs] = eprime(r);
                U.njobs++;
            }
        }

        ModDownParams &D = c->moddown[l];
        memset(&D, 0, sizeof(D));
        D.l = l;
        D.K = K;
        for (int k = 0; k < K; k++) {
            u64 pk = c->q[L + k], phk = 1;
            for (int m = 0; m < K; m++)
                if (m != k) phk = host_mulmod(phk, c->q[L + m] % pk, pk);
            D.sprime[k] = L + k;
            D.cinv[k] = host_mulmod(host_invmod(c->p % pk, pk), host_invmod(phk, pk), pk);
            D.cinv_s[k] = shoup_const(D.cinv[k], pk);
            for (int i = 0; i < l; i++) {
                u64 qi = c->q[i], h = c->p % qi;
                for (int m = 0; m < K; m++)
                    if (m != k) h = host_mulmod(h, c->q[L + m] % qi, qi);
                D.phat[k][i] = h;
            }
        }
        for (int i = 0; i < l; i++) {
            u64 qi = c->q[i], P = 1;
            for (int k = 0; k < K; k++) P = host_mulmod(P, c->q[L + k] % qi, qi);
            D.pinv[i] = host_invmod(P, qi);
            D.pinv_s[i] = shoup_const(D.pinv[i], qi);
        }

        ModSwitchParams &S = c->modswitch[l];
        memset(&S, 0, sizeof(S));
        S.l = l;
        if (l >= 2) {
            u64 ql = c->q[l - 1];
            S.pinv_last = host_invmod(c->p % ql, ql);
            S.pinv_last_s = shoup_const(S.pinv_last, ql);
            for (int i = 0; i < l - 1; i++) {
                u64 qi = c->q[i];
                S.p_i[i] = c->p % qi;
                S.p_i_s[i] = shoup_const(S.p_i[i], qi);
                S.qinv[i] = host_invmod(ql % qi, qi);
                S.qinv_s[i] = shoup_const(S.qinv[i], qi);
            }
        }
    }
    // relinearisation + modulus switch (level l -> l-1)
    c->rms.assign(L + 1, RelinMSParams());
    for (int l = 2; l <= L; l++) {
        RelinMSParams &R = c->rms[l];
        memset(&R, 0, sizeof(R));
        R.l = l;
        R.K = K;
        const u64 qm = c->q[l - 1];
        u64 Pm = 1;
        for (int k = 0; k < K; k++) {
            const u64 pk = c->q[L + k];
            Pm = host_mulmod(Pm, pk % qm, qm);
            R.pkinv[k] = host_invmod(pk % qm, qm);
        }
        R.Pm = Pm;
        R.Pm_s = shoup_const(Pm, qm);
        for (int i = 0; i < l - 1; i++) {
            const u64 qi = c->q[i], pi = c->p % qi;
            for (int k = 0; k < K; k++) R.h[k][i] = host_mulmod(pi, host_invmod(c->q[L + k] % qi, qi), qi);
            R.h[K][i] = pi;
            R.pinv[i] = c->moddown[l].pinv[i];
            R.pinv_s[i] = c->moddown[l].pinv_s[i];
            R.qminv[i] = c->modswitch[l].qinv[i];
            R.qminv_s[i] = c->modswitch[l].qinv_s[i];
        }
    }
    if ((e = upload(c, (void **)&c->d_rms, c->rms.data(), sizeof(RelinMSParams) * (L + 1)))) return e;

    // k switches at once
    c->mss.assign((size_t)(L + 1) * (FHE_MAXK + 1), MultiSwitchParams());
    c->mss_scale.assign((size_t)(L + 1) * (FHE_MAXK + 1) * FHE_MAXK, make_ulonglong2(0, 0));
    for (int l = 3; l <= L; l++)
        for (int k = 2; k <= FHE_MAXK && k < l; k++) {
            MultiSwitchParams &S = c->mss[(size_t)l * (FHE_MAXK + 1) + k];
            memset(&S, 0, sizeof(S));
            S.l = l;
            S.k = k;
            for (int i = 0; i < l - k; i++) {
                const u64 qi = c->q[i];
                u64 D = 1;
                for (int t = 0; t < k; t++) {
                    S.G[t][i] = host_mulmod(c->p % qi, D, qi);
                    D = host_mulmod(D, c->q[l - 1 - t] % qi, qi);
                }
                S.Dinv[i] = host_invmod(D, qi);
                S.Dinv_s[i] = shoup_const(S.Dinv[i], qi);
            }
            for (int j = 0; j < k; j++) {
                const u64 qj = c->q[l - 1 - j];
                std::vector<u64> D(j + 1, 1);  // D_t mod q_j, t <= j
                for (int t = 1; t <= j; t++) D[t] = host_mulmod(D[t - 1], c->q[l - t] % qj, qj);
                const u64 Djinv = host_invmod(D[j], qj);
                for (int t = 0; t < j; t++) S.F[j][t] = host_mulmod(D[t], Djinv, qj);
                const u64 ni = host_invmod((u64)N % qj, qj);
                const u64 v = host_mulmod(host_mulmod(ni, host_invmod(c->p % qj, qj), qj), Djinv, qj);
                c->mss_scale[((size_t)l * (FHE_MAXK + 1) + k) * FHE_MAXK + j] = make_ulonglong2(v, shoup_const(v, qj));
            }
        }
    if ((e = upload(c, (void **)&c->d_mss, c->mss.data(), sizeof(MultiSwitchParams) * c->mss.size()))) return e;
    if ((e = upload(c, (void **)&c->d_modup, c->modup.data(), sizeof(ModUpParams) * (L + 1)))) return e;
    if ((e = upload(c, (void **)&c->d_moddown, c->moddown.data(), sizeof(ModDownParams) * (L + 1)))) return e;
    if ((e = upload(c, (void **)&c->d_modswitch, c->modswitch.data(), sizeof(ModSwitchParams) * (L + 1))))
        return e;

    // constants folded into inverse NTTs
    auto sc = [](u64 v, u64 q) { return make_ulonglong2(v, shoup_const(v, q)); };
    c->ks_xscale.assign(L + 1, std::vector<ulonglong2>());
    c->ms_lastscale.assign(L + 1, make_ulonglong2(0, 0));
    c->rms_yscale.assign(L + 1, make_ulonglong2(0, 0));
    for (int l = 1; l <= L; l++) {
        const ModUpParams &U = c->modup[l];
        c->ks_xscale[l].resize(l);
        for (int j = 0; j < U.dnum; j++)
            for (int a = 0; a < U.digit_n[j]; a++) {
                const int i = U.digit_lo[j] + a;
                const u64 qi = c->q[i];
                c->ks_xscale[l][i] = sc(host_mulmod(ninv[i].x, U.inv_hat[j][a], qi), qi);
            }
        if (l >= 2) {
            const u64 ql = c->q[l - 1];
            c->ms_lastscale[l] = sc(host_mulmod(ninv[l - 1].x, c->modswitch[l].pinv_last, ql), ql);
            // (p P)^-1 = p^-1 P^-1 mod q_{l-1}
            const u64 pP_inv = host_mulmod(c->modswitch[l].pinv_last, host_invmod(c->rms[l].Pm, ql), ql);
            c->rms_yscale[l] = sc(host_mulmod(ninv[l - 1].x, pP_inv, ql), ql);
        }
    }
    c->ks_pscale.resize(K);
    for (int k = 0; k < K; k++) {
        const u64 pk = c->q[L + k];
        c->ks_pscale[k] = sc(host_mulmod(ninv[L + k].x, c->moddown[L].cinv[k], pk), pk);
    }

    // the same constants on the device, so that a launch serving several
    // contexts or levels reads each segment's own (ntt.cu takes pointers)
    {
        std::vector<ulonglong2> xs((size_t)(L + 1) * FHE_MAXP, make_ulonglong2(0, 0));
        std::vector<ulonglong2> m4((size_t)(L + 1) * (FHE_MAXK + 1), make_ulonglong2(0, 0));
        for (int l = 1; l <= L; l++) {
            for (int i = 0; i < l; i++) xs[(size_t)l * FHE_MAXP + i] = c->ks_xscale[l][i];
            for (int k = 0; k < K; k++) m4[(size_t)l * (FHE_MAXK + 1) + k] = c->ks_pscale[k];
            m4[(size_t)l * (FHE_MAXK + 1) + K] = c->rms_yscale[l];
        }
        if ((e = upload(c, (void **)&c->d_ks_xscale, xs.data(), sizeof(ulonglong2) * xs.size()))) return e;
        if ((e = upload(c, (void **)&c->d_ms4scale, m4.data(), sizeof(ulonglong2) * m4.size()))) return e;
        if ((e = upload(c, (void **)&c->d_ks_pscale, c->ks_pscale.data(), sizeof(ulonglong2) * K))) return e;
        if ((e = upload(c, (void **)&c->d_ms_lastscale, c->ms_lastscale.data(), sizeof(ulonglong2) * (L + 1))))
            return e;
        if ((e = upload(c, (void **)&c->d_mss_scale, c->mss_scale.data(), sizeof(ulonglong2) * c->mss_scale.size())))
            return e;
    }

    lt_poly_coefficients((int)c->p, c->lt);
    if (slot_structure(c)) return FHE_EUNSUPPORTED;
    if (c->N % c->M) return FHE_EUNSUPPORTED;
    return 0;
}
