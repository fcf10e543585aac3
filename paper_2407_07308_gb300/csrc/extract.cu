// F_{p^d}-valued slots and the tables of digit extraction (mod extract).
//
// BoostCom Sec. 2.1 ("Non-arithmetic Comparison of uFHE-based BGV"): an
// operand is held as an element of F_{p^d} per slot, and the mod-extract step
// splits every slot element into its d digits in F_p, one ciphertext per
// digit, before LT and EQ run per digit.
//
// Slot fields.  The F_p slots of the library are the factors g_s of Y^M + 1
// (Y = X^(N/M)): Y - zeta^e_s when p = 1 mod 4, Y^2 +- gamma Y - 1 when
// p = 3 mod 8.  For d = e deg(g_s), e a power of two, the subring generated by
// Y' = X^(N/(M e)) has the factors f_s(Y') = g_s(Y'^e) of Y'^(M e) + 1, one per
// slot, in the same slot order, each irreducible of degree d: slot s is the
// field F_p[Y']/(f_s) = F_{p^d}.  Digit k of a slot element is its coefficient
// of Y'^k.
//
// Extraction.  X -> X^p acts on every slot field as the Frobenius x -> x^p, so
// with lambda_k the trace-dual basis of 1, Y', .., Y'^(d-1),
//   digit_k(x) = Tr(lambda_k x) = sum_{t<d} lambda_k^(p^t) sigma_{p^t}(x),
// a sum of plaintext products with the Frobenius images of the ciphertext.
// This file builds the plaintexts L[k][t] (slot s = lambda_{k,s}^(p^t)) on the
// host, once per (context, d); the evaluation is in eval.cu.
#include <cstring>

#include "fhe_internal.h"

namespace {

using Poly = std::vector<u64>;  // coefficients mod p, lowest degree first

void trim(Poly &a)
{
    while (!a.empty() && a.back() == 0) a.pop_back();
}

Poly pmul(const Poly &a, const Poly &b, u64 p)
{
    if (a.empty() || b.empty()) return {};
    Poly r(a.size() + b.size() - 1, 0);
    for (size_t i = 0; i < a.size(); i++)
        if (a[i])
            for (size_t j = 0; j < b.size(); j++) r[i + j] = (r[i + j] + a[i] * b[j]) % p;
    trim(r);
    return r;
}

// quotient and remainder of a by f (f's leading coefficient non-zero)
void pdivmod(Poly a, const Poly &f, u64 p, Poly *q, Poly *r)
{
    const size_t nf = f.size();
    const u64 il = host_invmod(f.back(), p);
    Poly qq(a.size() >= nf ? a.size() - nf + 1 : 1, 0);
    for (long long i = (long long)a.size() - (long long)nf; i >= 0; i--) {
        const u64 c = a[i + nf - 1] * il % p;
        qq[i] = c;
        if (c)
            for (size_t j = 0; j < nf; j++) a[i + j] = (a[i + j] + p - c * f[j] % p) % p;
    }
    a.resize(std::min(a.size(), nf - 1));
    trim(a);
    trim(qq);
    if (q) *q = qq;
    if (r) *r = a;
}

Poly pmod(const Poly &a, const Poly &f, u64 p)
{
    Poly r;
    pdivmod(a, f, p, nullptr, &r);
    return r;
}

Poly psub(const Poly &a, const Poly &b, u64 p)
{
    Poly r(std::max(a.size(), b.size()), 0);
    for (size_t i = 0; i < r.size(); i++)
        r[i] = ((i < a.size() ? a[i] : 0) + p - (i < b.size() ? b[i] : 0)) % p;
    trim(r);
    return r;
}

// a^-1 mod f (gcd 1), extended Euclid; empty on failure
Poly pinv(const Poly &a, const Poly &f, u64 p)
{
    Poly r0 = f, r1 = pmod(a, f, p), s0, s1{1};
    while (!r1.empty()) {
        Poly q, r;
        pdivmod(r0, r1, p, &q, &r);
        r0 = r1;
        r1 = r;
        Poly s2 = psub(s0, pmul(q, s1, p), p);
        s0 = s1;
        s1 = s2;
    }
    if (r0.size() != 1) return {};
    const u64 c = host_invmod(r0[0], p);
    for (u64 &v : s0) v = v * c % p;
    return pmod(s0, f, p);
}

Poly fpow(const Poly &a, u64 n, const Poly &f, u64 p)
{
    Poly r{1}, b = pmod(a, f, p);
    for (; n; n >>= 1) {
        if (n & 1) r = pmod(pmul(r, b, p), f, p);
        b = pmod(pmul(b, b, p), f, p);
    }
    return r;
}

// Tr(a) in F_p[Y]/(f), degree d; UINT64_MAX if the sum is not a constant
u64 ftrace(const Poly &a, const Poly &f, int d, u64 p)
{
    Poly acc;
    Poly x = pmod(a, f, p);
    for (int t = 0; t < d; t++) {
        Poly s(std::max(acc.size(), x.size()), 0);
        for (size_t i = 0; i < s.size(); i++) s[i] = ((i < acc.size() ? acc[i] : 0) + (i < x.size() ? x[i] : 0)) % p;
        trim(s);
        acc = s;
        x = fpow(x, p, f, p);  // x^(p^(t+1))
    }
    if (acc.size() > 1) return UINT64_MAX;
    return acc.empty() ? 0 : acc[0];
}

// trace-dual basis of 1, Y, .., Y^(d-1): rows of the inverse of T[i][j] = Tr(Y^(i+j))
bool dual_basis(const Poly &f, int d, u64 p, std::vector<Poly> &lam)
{
    std::vector<std::vector<u64>> A(d, std::vector<u64>(2 * d, 0));
    for (int i = 0; i < d; i++) {
        for (int j = 0; j < d; j++) {
            Poly y(i + j + 1, 0);
            y[i + j] = 1;
            const u64 t = ftrace(y, f, d, p);
            if (t == UINT64_MAX) return false;
            A[i][j] = t;
        }
        A[i][d + i] = 1;
    }
    for (int c = 0; c < d; c++) {
        int piv = c;
        while (piv < d && !A[piv][c]) piv++;
        if (piv == d) return false;
        std::swap(A[c], A[piv]);
        const u64 iv = host_invmod(A[c][c], p);
        for (u64 &v : A[c]) v = v * iv % p;
        for (int r = 0; r < d; r++)
            if (r != c && A[r][c]) {
                const u64 m = A[r][c];
                for (int k = 0; k < 2 * d; k++) A[r][k] = (A[r][k] + p - m * A[c][k] % p) % p;
            }
    }
    lam.assign(d, {});
    for (int k = 0; k < d; k++) {
        lam[k].assign(A[k].begin() + d, A[k].end());
        trim(lam[k]);
    }
    return true;
}

}  // namespace

// Tables of the F_{p^d} slots for digit count d (nullptr + error code when the
// ring has no such slots).  Built once per (context, d) and kept.
const ExtTables *ext_tables(fhe_ctx *c, int d, int *err)
{
    auto it = c->ext.find(d);
    if (it != c->ext.end()) return it->second.get();
    const u64 p = c->p;
    const int d0 = c->slots_linear ? 1 : 2;
    const int e = d / d0;
    if (d < d0 || d % d0 || (e & (e - 1)) || (long long)c->M * e > c->N || d > 64) {
        *err = fhe_fail(c, FHE_EUNSUPPORTED, "no F_(p^d) slots for this digit count on this ring");
        return nullptr;
    }
    auto T = std::make_shared<ExtTables>();
    T->d = d;
    T->Me = c->M * e;
    T->stride = c->N / T->Me;
    for (int s = 0; s < c->ns; s++) {
        Poly f;
        if (c->slots_linear) {
            f.assign(e + 1, 0);
            f[0] = (p - host_powmod(c->zeta, (u64)c->slot_exp[s], p)) % p;
            f[e] = 1;
        } else {  // Y^(2e) + g Y^e - 1, g = gamma for slot 0, -gamma for slot 1
            f.assign(2 * e + 1, 0);
            f[0] = p - 1;
            f[e] = s == 0 ? c->gamma : p - c->gamma;
            f[2 * e] = 1;
        }
        T->factors.push_back(f);
    }
    Poly F(T->Me + 1, 0);
    F[0] = F[T->Me] = 1;
    for (const Poly &f : T->factors) {
        Poly cof, r;
        pdivmod(F, f, p, &cof, &r);
        Poly inv = pinv(cof, f, p);
        if (!r.empty() || inv.empty()) {
            *err = fhe_fail(c, FHE_EUNSUPPORTED, "slot factors do not split Y^(Me)+1");
            return nullptr;
        }
        T->idem.push_back(pmod(pmul(cof, inv, p), F, p));
    }
    // L[k][t]: slot s holds lambda_{k,s}^(p^t)
    std::vector<std::vector<Poly>> lam(c->ns);
    for (int s = 0; s < c->ns; s++)
        if (!dual_basis(T->factors[s], d, p, lam[s])) {
            *err = fhe_fail(c, FHE_EUNSUPPORTED, "trace form is degenerate");
            return nullptr;
        }
    T->L.assign((size_t)d * d, std::vector<int64_t>(c->N, 0));
    std::vector<uint64_t> el((size_t)c->ns * d);
    for (int k = 0; k < d; k++) {
        std::vector<Poly> cur(c->ns);
        for (int s = 0; s < c->ns; s++) cur[s] = lam[s][k];
        for (int t = 0; t < d; t++) {
            std::fill(el.begin(), el.end(), 0);
            for (int s = 0; s < c->ns; s++)
                for (size_t i = 0; i < cur[s].size(); i++) el[(size_t)s * d + i] = cur[s][i];
            ext_encode(c, T.get(), el.data(), T->L[(size_t)k * d + t].data());
            for (int s = 0; s < c->ns; s++) cur[s] = fpow(cur[s], p, T->factors[s], p);
        }
    }
    for (int t = 1; t < d; t++) T->galois.push_back((int64_t)host_powmod(p % (2 * (u64)c->N), (u64)t, 2 * (u64)c->N));
    const ExtTables *out = T.get();
    c->ext[d] = std::move(T);
    return out;
}

// digits[s * d + k] (values in [0, p)) -> plaintext coefficients m[N] in [0, p)
void ext_encode(const fhe_ctx *c, const ExtTables *T, const uint64_t *digits, int64_t *m)
{
    const u64 p = c->p;
    const int d = T->d, Me = T->Me;
    std::vector<u64> acc(Me, 0);
    for (int s = 0; s < c->ns; s++) {
        const Poly &E = T->idem[s];
        // (a_s * E_s) mod Y^Me + 1, negacyclic
        for (int k = 0; k < d; k++) {
            const u64 a = digits[(size_t)s * d + k] % p;
            if (!a) continue;
            for (size_t j = 0; j < E.size(); j++) {
                if (!E[j]) continue;
                const size_t n = j + k;
                const u64 v = a * E[j] % p;
                if (n < (size_t)Me) acc[n] = (acc[n] + v) % p;
                else acc[n - Me] = (acc[n - Me] + p - v) % p;
            }
        }
    }
    memset(m, 0, sizeof(int64_t) * c->N);
    for (int j = 0; j < Me; j++) m[(size_t)j * T->stride] = (int64_t)acc[j];
}

// plaintext coefficients in [0, p) -> digits[s * d + k]; false if m is not in
// the slot subring
bool ext_decode(const fhe_ctx *c, const ExtTables *T, const int64_t *m, uint64_t *digits)
{
    const u64 p = c->p;
    for (int n = 0; n < c->N; n++)
        if (n % T->stride && m[n]) return false;
    Poly y(T->Me);
    for (int j = 0; j < T->Me; j++) y[j] = (u64)m[(size_t)j * T->stride] % p;
    trim(y);
    for (int s = 0; s < c->ns; s++) {
        Poly r = pmod(y, T->factors[s], p);
        for (int k = 0; k < T->d; k++) digits[(size_t)s * T->d + k] = k < (int)r.size() ? r[k] : 0;
    }
    return true;
}
