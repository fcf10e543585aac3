/*
 * bgv_oracle.c -- plain, slow CPU oracle for BGV encrypted comparison.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  The CUDA product path
 * never links it, and it shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * Every routine is the plain definition (or the textbook algorithm) of the
 * operation it names, with exact integer arithmetic: products are formed in
 * unsigned __int128 and reduced with the C '%' operator.  Nothing is blocked,
 * fused or reordered.
 *
 * What the paper fixes (BoostCom, Sec. 2.1 "Basics and arithmetic ops",
 * Sec. 2.2 "Efficient Polynomial and NTT"):
 *   - ciphertexts live in C = R_Q x R_Q with R_Q = Z_Q[X]/Phi_m(X); here
 *     Phi_{2N}(X) = X^N + 1 with N a power of two;
 *   - Q = q_0 ... q_L is held in RNS: one residue polynomial per prime;
 *   - polynomial products go through a radix-2 NTT, Cooley-Tukey forward and
 *     Gentleman-Sande inverse.
 * The key-switching, modulus-switching and encryption details are not in the
 * paper (it defers to HElib); the readings used here are the standard
 * hybrid-key-switching BGV formulas, restated in each function's comment.
 *
 * Layouts: a "poly" at level l is u64[l][N] (limb i reduced mod q[i]); a
 * ciphertext is u64[npoly][l][N]; special-prime limbs of key material sit at
 * prime indices L .. L+K-1.  Everything is in the coefficient domain.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

#define ORC_MAXP 64

/* ------------------------------------------------------------------------ */
/* scalar modular arithmetic: the definitions                               */
/* ------------------------------------------------------------------------ */

static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static u64 submod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + q - (b % q)) % q); }

static u64 powmod(u64 a, u64 e, u64 q)
{
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* inverse modulo a prime (Fermat) */
static u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }

/* the residue in [0,q) of a signed integer */
static u64 mod_i64(i64 v, u64 q)
{
    i64 r = v % (i64)q;
    return (u64)(r < 0 ? r + (i64)q : r);
}

u64 orc_mulmod(u64 a, u64 b, u64 q) { return mulmod(a, b, q); }
u64 orc_powmod(u64 a, u64 e, u64 q) { return powmod(a, e, q); }

/* Deterministic Miller-Rabin: the first twelve prime bases decide every
 * n < 3.3e24 (Sorenson and Webster 2015), which covers u64. */
int orc_is_prime(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++)
        if (n % bases[i] == 0) return n == bases[i];
    u64 d = n - 1;
    int r = 0;
    while (!(d & 1)) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        u64 x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int k = 1; k < r; k++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* The `count` smallest primes q with q = 1 (mod U) and lo <= q < hi, in
 * increasing order.  Returns how many were found. */
int orc_find_primes(u64 U, u64 lo, u64 hi, int count, u64 *out)
{
    int n = 0;
    u64 k = (lo - 1) / U;               /* first q = kU+1 >= lo */
    if (k * U + 1 < lo) k++;
    for (; n < count; k++) {
        u64 q = k * U + 1;
        if (q >= hi) break;
        if (orc_is_prime(q)) out[n++] = q;
    }
    return n;
}

/* Smallest generator of the multiplicative group mod the prime q. */
u64 orc_smallest_generator(u64 q)
{
    u64 fac[64];
    int nf = 0;
    u64 m = q - 1;
    for (u64 f = 2; f * f <= m; f++)
        if (m % f == 0) {
            fac[nf++] = f;
            while (m % f == 0) m /= f;
        }
    if (m > 1) fac[nf++] = m;
    for (u64 g = 2;; g++) {
        int ok = 1;
        for (int i = 0; i < nf; i++)
            if (powmod(g, (q - 1) / fac[i], q) == 1) { ok = 0; break; }
        if (ok) return g;
    }
}

/* ------------------------------------------------------------------------ */
/* context                                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int logN, N, L, K;  /* ring degree N = 2^logN; L data primes; K special */
    u64 p;              /* plaintext modulus */
    u64 q[ORC_MAXP];    /* q[0..L-1] data primes, q[L..L+K-1] special primes */
    u64 psi[ORC_MAXP];  /* psi = g^((q-1)/2N): a primitive 2N-th root mod q */
    u64 *pw[ORC_MAXP];  /* pw[i][k]  = psi^brv(k)  (brv over logN bits) */
    u64 *ipw[ORC_MAXP]; /* ipw[i][k] = psi^-brv(k) */
} orc_ctx;

static unsigned brv(unsigned x, int bits)
{
    unsigned r = 0;
    for (int b = 0; b < bits; b++) r |= ((x >> b) & 1u) << (bits - 1 - b);
    return r;
}

void orc_ctx_free(orc_ctx *c)
{
    if (!c) return;
    for (int i = 0; i < c->L + c->K; i++) { free(c->pw[i]); free(c->ipw[i]); }
    free(c);
}

/* Prime chain: the L+K smallest primes q = 1 (mod U) in [lo,hi); the first
 * L are data primes, the next K special.  U must be a multiple of 2N (so the
 * negacyclic NTT exists) and of p (so that q^-1 = P^-1 = 1 mod p and
 * modulus switching leaves the plaintext unscaled). */
orc_ctx *orc_ctx_new(int logN, u64 p, int L, int K, u64 U, u64 lo, u64 hi)
{
    if (L + K > ORC_MAXP || logN < 1 || logN > 17) return NULL;
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    c->logN = logN; c->N = 1 << logN; c->L = L; c->K = K; c->p = p;
    if (orc_find_primes(U, lo, hi, L + K, c->q) != L + K) { free(c); return NULL; }
    for (int i = 0; i < L + K; i++) {
        u64 q = c->q[i];
        u64 g = orc_smallest_generator(q);
        c->psi[i] = powmod(g, (q - 1) / (2 * (u64)c->N), q);
        c->pw[i] = (u64 *)malloc(sizeof(u64) * c->N);
        c->ipw[i] = (u64 *)malloc(sizeof(u64) * c->N);
        u64 ipsi = invmod(c->psi[i], q);
        for (int k = 0; k < c->N; k++) {
            c->pw[i][k] = powmod(c->psi[i], brv(k, logN), q);
            c->ipw[i][k] = powmod(ipsi, brv(k, logN), q);
        }
    }
    return c;
}

void orc_ctx_primes(const orc_ctx *c, u64 *out) { memcpy(out, c->q, sizeof(u64) * (c->L + c->K)); }
u64 orc_ctx_psi(const orc_ctx *c, int i) { return c->psi[i]; }

/* ------------------------------------------------------------------------ */
/* NTT (Sec. 2.2): radix-2 Cooley-Tukey forward, Gentleman-Sande inverse      */
/* ------------------------------------------------------------------------ */

/* Definition: A[k] = sum_n a[n] * psi^((2 brv(k) + 1) n) mod q, i.e. the
 * evaluation of a(X) at the odd power psi^(2 brv(k)+1), stored in
 * bit-reversed order.  O(N^2); used to pin orc_ntt. */
void orc_ntt_direct(const orc_ctx *c, int i, const u64 *a, u64 *A)
{
    u64 q = c->q[i];
    for (int k = 0; k < c->N; k++) {
        u64 w = powmod(c->psi[i], 2 * (u64)brv(k, c->logN) + 1, q), x = 1, s = 0;
        for (int n = 0; n < c->N; n++) {
            s = addmod(s, mulmod(a[n], x, q), q);
            x = mulmod(x, w, q);
        }
        A[k] = s;
    }
}

/* In place, natural-order input, bit-reversed output, same result as
 * orc_ntt_direct.  Stage m (m = 1,2,4,..,N/2) pairs a[j] with a[j+t],
 * t = N/2m, for j in the g-th block of 2t, using psi^brv(m+g). */
void orc_ntt(const orc_ctx *c, int i, u64 *a)
{
    u64 q = c->q[i];
    int N = c->N;
    for (int m = 1, t = N / 2; m < N; m *= 2, t /= 2)
        for (int g = 0; g < m; g++) {
            u64 w = c->pw[i][m + g];
            for (int j = 2 * g * t; j < 2 * g * t + t; j++) {
                u64 u = a[j], v = mulmod(a[j + t], w, q);
                a[j] = addmod(u, v, q);
                a[j + t] = submod(u, v, q);
            }
        }
}

/* Exact inverse of orc_ntt: the stages of orc_ntt undone in reverse order
 * (Gentleman-Sande butterflies with psi^-brv(m+g)), then scaling by N^-1. */
void orc_intt(const orc_ctx *c, int i, u64 *a)
{
    u64 q = c->q[i];
    int N = c->N;
    for (int m = N / 2, t = 1; m >= 1; m /= 2, t *= 2)
        for (int g = 0; g < m; g++) {
            u64 w = c->ipw[i][m + g];
            for (int j = 2 * g * t; j < 2 * g * t + t; j++) {
                u64 u = a[j], v = a[j + t];
                a[j] = addmod(u, v, q);
                a[j + t] = mulmod(submod(u, v, q), w, q);
            }
        }
    u64 ninv = invmod((u64)N % q, q);
    for (int j = 0; j < N; j++) a[j] = mulmod(a[j], ninv, q);
}

/* Negacyclic product out = a*b mod (X^N+1, q[i]) through the NTT. */
void orc_polymul(const orc_ctx *c, int i, const u64 *a, const u64 *b, u64 *out)
{
    int N = c->N;
    u64 *A = (u64 *)malloc(sizeof(u64) * N), *B = (u64 *)malloc(sizeof(u64) * N);
    memcpy(A, a, sizeof(u64) * N);
    memcpy(B, b, sizeof(u64) * N);
    orc_ntt(c, i, A);
    orc_ntt(c, i, B);
    for (int k = 0; k < N; k++) out[k] = mulmod(A[k], B[k], c->q[i]);
    orc_intt(c, i, out);
    free(A);
    free(B);
}

/* Negacyclic product of two integer polynomials over Z (schoolbook).  Used
 * for s^2; inputs must be small enough that no i64 sum overflows. */
void orc_polymul_int(const orc_ctx *c, const i64 *a, const i64 *b, i64 *out)
{
    int N = c->N;
    memset(out, 0, sizeof(i64) * N);
    for (int x = 0; x < N; x++) {
        if (!a[x]) continue;
        for (int y = 0; y < N; y++) {
            i64 v = a[x] * b[y];
            if (x + y < N) out[x + y] += v;
            else out[x + y - N] -= v;
        }
    }
}

/* Automorphism sigma_g: a(X) -> a(X^g), g odd; X^n goes to X^(ng mod 2N),
 * and X^(N+r) = -X^r.  On integer polynomials. */
void orc_automorphism_int(const orc_ctx *c, const i64 *a, u64 g, i64 *out)
{
    int N = c->N;
    u64 twoN = 2 * (u64)N;
    for (int n = 0; n < N; n++) {
        u64 e = ((u64)n * g) % twoN;
        if (e < (u64)N) out[e] = a[n];
        else out[e - N] = -a[n];
    }
}

/* The same automorphism on residues: limb by limb, polys [npoly][l][N]. */
void orc_automorphism(const orc_ctx *c, const u64 *x, int l, int npoly, u64 g, u64 *out)
{
    int N = c->N;
    u64 twoN = 2 * (u64)N;
    for (int k = 0; k < npoly; k++)
        for (int i = 0; i < l; i++) {
            const u64 *a = x + ((size_t)k * l + i) * N;
            u64 *o = out + ((size_t)k * l + i) * N;
            u64 q = c->q[i];
            for (int n = 0; n < N; n++) {
                u64 e = ((u64)n * g) % twoN;
                if (e < (u64)N) o[e] = a[n];
                else o[e - N] = submod(0, a[n], q);
            }
        }
}

/* ------------------------------------------------------------------------ */
/* limb-wise ciphertext arithmetic (Sec. 2.1: add / mult on R_Q residues)    */
/* ------------------------------------------------------------------------ */

void orc_add(const orc_ctx *c, const u64 *a, const u64 *b, int l, int npoly, u64 *out)
{
    for (int k = 0; k < npoly; k++)
        for (int i = 0; i < l; i++)
            for (int n = 0; n < c->N; n++) {
                size_t o = ((size_t)k * l + i) * c->N + n;
                out[o] = addmod(a[o], b[o], c->q[i]);
            }
}

void orc_sub(const orc_ctx *c, const u64 *a, const u64 *b, int l, int npoly, u64 *out)
{
    for (int k = 0; k < npoly; k++)
        for (int i = 0; i < l; i++)
            for (int n = 0; n < c->N; n++) {
                size_t o = ((size_t)k * l + i) * c->N + n;
                out[o] = submod(a[o], b[o], c->q[i]);
            }
}

void orc_neg(const orc_ctx *c, const u64 *a, int l, int npoly, u64 *out)
{
    for (int k = 0; k < npoly; k++)
        for (int i = 0; i < l; i++)
            for (int n = 0; n < c->N; n++) {
                size_t o = ((size_t)k * l + i) * c->N + n;
                out[o] = submod(0, a[o], c->q[i]);
            }
}

/* Multiply every poly by the integer constant k (already lifted to Z). */
void orc_mul_const(const orc_ctx *c, const u64 *a, i64 k, int l, int npoly, u64 *out)
{
    for (int kk = 0; kk < npoly; kk++)
        for (int i = 0; i < l; i++) {
            u64 kq = mod_i64(k, c->q[i]);
            for (int n = 0; n < c->N; n++) {
                size_t o = ((size_t)kk * l + i) * c->N + n;
                out[o] = mulmod(a[o], kq, c->q[i]);
            }
        }
}

/* Add the constant plaintext polynomial k (integer) to a ciphertext: only
 * the constant coefficient of c0 changes. */
void orc_add_const(const orc_ctx *c, const u64 *a, i64 k, int l, u64 *out)
{
    memcpy(out, a, sizeof(u64) * 2 * (size_t)l * c->N);
    for (int i = 0; i < l; i++) {
        size_t o = (size_t)i * c->N;
        out[o] = addmod(out[o], mod_i64(k, c->q[i]), c->q[i]);
    }
}

/* Tensor product (x0,x1) (x) (y0,y1) = (x0 y0, x0 y1 + x1 y0, x1 y1). */
void orc_tensor(const orc_ctx *c, const u64 *x, const u64 *y, int l, u64 *out)
{
    int N = c->N;
    u64 *t = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < l; i++) {
        const u64 *x0 = x + (size_t)i * N, *x1 = x + ((size_t)l + i) * N;
        const u64 *y0 = y + (size_t)i * N, *y1 = y + ((size_t)l + i) * N;
        u64 *d0 = out + (size_t)i * N, *d1 = out + ((size_t)l + i) * N, *d2 = out + ((size_t)2 * l + i) * N;
        orc_polymul(c, i, x0, y0, d0);
        orc_polymul(c, i, x0, y1, d1);
        orc_polymul(c, i, x1, y0, t);
        for (int n = 0; n < N; n++) d1[n] = addmod(d1[n], t[n], c->q[i]);
        orc_polymul(c, i, x1, y1, d2);
    }
    free(t);
}

/* ------------------------------------------------------------------------ */
/* keys and encryption                                                      */
/* ------------------------------------------------------------------------ */

/* pk = (-a s + p e, a) over the L data primes. */
void orc_keygen(const orc_ctx *c, const i64 *s, const u64 *a, const i64 *e, u64 *pk)
{
    int N = c->N, L = c->L;
    u64 *sq = (u64 *)malloc(sizeof(u64) * N), *as = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < L; i++) {
        u64 q = c->q[i];
        for (int n = 0; n < N; n++) sq[n] = mod_i64(s[n], q);
        orc_polymul(c, i, a + (size_t)i * N, sq, as);
        for (int n = 0; n < N; n++) {
            u64 pe = mulmod(c->p % q, mod_i64(e[n], q), q);
            pk[(size_t)i * N + n] = addmod(submod(0, as[n], q), pe, q);
            pk[((size_t)L + i) * N + n] = a[(size_t)i * N + n];
        }
    }
    free(sq);
    free(as);
}

/* Enc(m) = (pk0 u + p e0 + m, pk1 u + p e1) over the L data primes. */
void orc_encrypt(const orc_ctx *c, const u64 *pk, const i64 *m, const i64 *u, const i64 *e0,
                 const i64 *e1, u64 *ct)
{
    int N = c->N, L = c->L;
    u64 *uq = (u64 *)malloc(sizeof(u64) * N), *t = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < L; i++) {
        u64 q = c->q[i], pq = c->p % q;
        for (int n = 0; n < N; n++) uq[n] = mod_i64(u[n], q);
        orc_polymul(c, i, pk + (size_t)i * N, uq, t);
        for (int n = 0; n < N; n++)
            ct[(size_t)i * N + n] =
                addmod(addmod(t[n], mulmod(pq, mod_i64(e0[n], q), q), q), mod_i64(m[n], q), q);
        orc_polymul(c, i, pk + ((size_t)L + i) * N, uq, t);
        for (int n = 0; n < N; n++)
            ct[((size_t)L + i) * N + n] = addmod(t[n], mulmod(pq, mod_i64(e1[n], q), q), q);
    }
    free(uq);
    free(t);
}

/* out_i = c0_i + c1_i s (mod q_i), i < l: the decryption residues. */
void orc_dot_sk(const orc_ctx *c, const u64 *ct, int l, const i64 *s, u64 *out)
{
    int N = c->N;
    u64 *sq = (u64 *)malloc(sizeof(u64) * N), *t = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < l; i++) {
        u64 q = c->q[i];
        for (int n = 0; n < N; n++) sq[n] = mod_i64(s[n], q);
        orc_polymul(c, i, ct + ((size_t)l + i) * N, sq, t);
        for (int n = 0; n < N; n++) out[(size_t)i * N + n] = addmod(ct[(size_t)i * N + n], t[n], q);
    }
    free(sq);
    free(t);
}

/* Number of key-switching digits at level l: ceil(l / K). */
int orc_dnum(const orc_ctx *c, int l) { return (l + c->K - 1) / c->K; }

/* P = product of the special primes, reduced mod q. */
static u64 P_mod(const orc_ctx *c, u64 q)
{
    u64 r = 1 % q;
    for (int k = 0; k < c->K; k++) r = mulmod(r, c->q[c->L + k] % q, q);
    return r;
}

/* Switching key from s' to s, one per digit j = 0..ceil(L/K)-1, over all
 * L+K primes:  ksk_j = (-a_j s + p e_j + P [i in D_j] s', a_j), with
 * D_j = data primes jK .. (j+1)K-1.  Layout [dnum][2][L+K][N].  At a lower
 * level l the same key is used with its limbs >= l (data) dropped. */
void orc_ksk_gen(const orc_ctx *c, const i64 *s, const i64 *sp, const u64 *a, const i64 *e, u64 *ksk)
{
    int N = c->N, L = c->L, K = c->K, LK = L + K, dnum = orc_dnum(c, L);
    u64 *sq = (u64 *)malloc(sizeof(u64) * N), *as = (u64 *)malloc(sizeof(u64) * N);
    for (int j = 0; j < dnum; j++)
        for (int i = 0; i < LK; i++) {
            u64 q = c->q[i], pq = c->p % q, Pq = P_mod(c, q);
            const u64 *aj = a + ((size_t)j * LK + i) * N;
            const i64 *ej = e + (size_t)j * N;
            u64 *k0 = ksk + (((size_t)j * 2 + 0) * LK + i) * N;
            u64 *k1 = ksk + (((size_t)j * 2 + 1) * LK + i) * N;
            for (int n = 0; n < N; n++) sq[n] = mod_i64(s[n], q);
            orc_polymul(c, i, aj, sq, as);
            int in_digit = (i < L) && (i >= j * K) && (i < (j + 1) * K);
            for (int n = 0; n < N; n++) {
                u64 v = addmod(submod(0, as[n], q), mulmod(pq, mod_i64(ej[n], q), q), q);
                if (in_digit) v = addmod(v, mulmod(Pq, mod_i64(sp[n], q), q), q);
                k0[n] = v;
                k1[n] = aj[n];
            }
        }
    free(sq);
    free(as);
}

/* ------------------------------------------------------------------------ */
/* basis conversion, key switching, modulus switching                       */
/* ------------------------------------------------------------------------ */

/* Fast basis conversion from the primes src[0..ns-1] (product Q_S) to the
 * primes dst[0..nd-1]:
 *   y_r = sum_{i in S} [x_i (Q_S/q_i)^-1]_{q_i} * (Q_S/q_i)   mod r,
 * with each bracket the non-centred residue in [0, q_i).  The result is
 * x + u Q_S with 0 <= u < ns, reduced mod r. */
void orc_fbc(const orc_ctx *c, const u64 *x, const int *src, int ns, const int *dst, int nd, u64 *y)
{
    int N = c->N;
    u64 inv_hat[ORC_MAXP];           /* (Q_S/q_a)^-1 mod q_a */
    for (int a = 0; a < ns; a++) {
        u64 qa = c->q[src[a]], hat = 1 % qa;
        for (int b = 0; b < ns; b++)
            if (b != a) hat = mulmod(hat, c->q[src[b]] % qa, qa);
        inv_hat[a] = invmod(hat, qa);
    }
    for (int d = 0; d < nd; d++) {
        u64 r = c->q[dst[d]];
        u64 hat_r[ORC_MAXP];         /* (Q_S/q_a) mod r */
        for (int a = 0; a < ns; a++) {
            hat_r[a] = 1 % r;
            for (int b = 0; b < ns; b++)
                if (b != a) hat_r[a] = mulmod(hat_r[a], c->q[src[b]] % r, r);
        }
        for (int n = 0; n < N; n++) {
            u64 acc = 0;
            for (int a = 0; a < ns; a++) {
                u64 qa = c->q[src[a]];
                u64 t = mulmod(x[(size_t)a * N + n], inv_hat[a], qa);
                acc = addmod(acc, mulmod(t % r, hat_r[a], r), r);
            }
            y[(size_t)d * N + n] = acc;
        }
    }
}

/* BGV ModDown of one poly over (q_0..q_{l-1}, P): x is [l+K][N] with the
 * special limbs last.  w = [x_P p^-1]_P limb by limb (non-centred),
 * delta = p * FBC_{P->Q}(w), out_i = (x_i - delta_i) P^-1 mod q_i.
 * delta = x (mod P) and delta = 0 (mod p), so x - delta is divisible by P
 * and the plaintext mod p is kept. */
static void moddown(const orc_ctx *c, const u64 *x, int l, u64 *out)
{
    int N = c->N, K = c->K;
    u64 *w = (u64 *)malloc(sizeof(u64) * (size_t)K * N);
    u64 *dl = (u64 *)malloc(sizeof(u64) * (size_t)l * N);
    int src[ORC_MAXP] = {0}, dst[ORC_MAXP] = {0};
    for (int k = 0; k < K; k++) {
        u64 pk = c->q[c->L + k], pinv = invmod(c->p % pk, pk);
        src[k] = c->L + k;
        for (int n = 0; n < N; n++) w[(size_t)k * N + n] = mulmod(x[((size_t)l + k) * N + n], pinv, pk);
    }
    for (int i = 0; i < l; i++) dst[i] = i;
    orc_fbc(c, w, src, K, dst, l, dl);
    for (int i = 0; i < l; i++) {
        u64 q = c->q[i], Pinv = invmod(P_mod(c, q), q), pq = c->p % q;
        for (int n = 0; n < N; n++) {
            u64 delta = mulmod(pq, dl[(size_t)i * N + n], q);
            out[(size_t)i * N + n] = mulmod(submod(x[(size_t)i * N + n], delta, q), Pinv, q);
        }
    }
    free(w);
    free(dl);
}

/* Hybrid key switching of one poly x (level l, [l][N]) with a key made by
 * orc_ksk_gen.  For each digit j (data primes D_j = jK .. min((j+1)K,l)-1):
 * ModUp x_{D_j} to every other prime of Q_l and P by orc_fbc (the D_j limbs
 * are x itself), multiply by ksk_j and sum over j; then ModDown both sums.
 * out is [2][l][N]:  out0 + out1 s = x s' + p (small)  (mod Q_l). */
void orc_keyswitch(const orc_ctx *c, const u64 *x, int l, const u64 *ksk, u64 *out)
{
    int N = c->N, L = c->L, K = c->K, LK = L + K, lk = l + K, dnum = orc_dnum(c, l);
    u64 *acc0 = (u64 *)calloc((size_t)lk * N, sizeof(u64));
    u64 *acc1 = (u64 *)calloc((size_t)lk * N, sizeof(u64));
    u64 *ext = (u64 *)malloc(sizeof(u64) * (size_t)lk * N);
    u64 *t = (u64 *)malloc(sizeof(u64) * N);
    int pidx[ORC_MAXP]; /* prime index of extended limb r: data 0..l-1, then special */
    for (int r = 0; r < lk; r++) pidx[r] = r < l ? r : L + (r - l);
    for (int j = 0; j < dnum; j++) {
        int lo = j * K, hi = (j + 1) * K < l ? (j + 1) * K : l;
        int src[ORC_MAXP], dst[ORC_MAXP], nd = 0, dpos[ORC_MAXP];
        for (int i = lo; i < hi; i++) src[i - lo] = i;
        for (int r = 0; r < lk; r++) {
            if (r >= lo && r < hi) memcpy(ext + (size_t)r * N, x + (size_t)r * N, sizeof(u64) * N);
            else { dst[nd] = pidx[r]; dpos[nd] = r; nd++; }
        }
        u64 *y = (u64 *)malloc(sizeof(u64) * (size_t)(nd ? nd : 1) * N);
        orc_fbc(c, x + (size_t)lo * N, src, hi - lo, dst, nd, y);
        for (int d = 0; d < nd; d++) memcpy(ext + (size_t)dpos[d] * N, y + (size_t)d * N, sizeof(u64) * N);
        free(y);
        for (int r = 0; r < lk; r++) {
            int pi = pidx[r];
            u64 q = c->q[pi];
            const u64 *k0 = ksk + (((size_t)j * 2 + 0) * LK + pi) * N;
            const u64 *k1 = ksk + (((size_t)j * 2 + 1) * LK + pi) * N;
            orc_polymul(c, pi, ext + (size_t)r * N, k0, t);
            for (int n = 0; n < N; n++) acc0[(size_t)r * N + n] = addmod(acc0[(size_t)r * N + n], t[n], q);
            orc_polymul(c, pi, ext + (size_t)r * N, k1, t);
            for (int n = 0; n < N; n++) acc1[(size_t)r * N + n] = addmod(acc1[(size_t)r * N + n], t[n], q);
        }
    }
    moddown(c, acc0, l, out);
    moddown(c, acc1, l, out + (size_t)l * N);
    free(acc0);
    free(acc1);
    free(ext);
    free(t);
}

/* Relinearise a 3-poly ciphertext (d0,d1,d2) with the key for s' = s^2:
 * (d0,d1) + KS(d2). */
void orc_relin(const orc_ctx *c, const u64 *d, int l, const u64 *ksk, u64 *out)
{
    size_t LN = (size_t)l * c->N;
    u64 *ks = (u64 *)malloc(sizeof(u64) * 2 * LN);
    orc_keyswitch(c, d + 2 * LN, l, ksk, ks);
    orc_add(c, d, ks, l, 2, out);
    free(ks);
}

/* Rotation by the Galois element g: (sigma_g c0, sigma_g c1) decrypts under
 * sigma_g(s); switch sigma_g c1 back to s with the key for s' = sigma_g(s):
 * (sigma c0 + KS0, KS1). */
void orc_rotate(const orc_ctx *c, const u64 *ct, int l, u64 g, const u64 *ksk, u64 *out)
{
    size_t LN = (size_t)l * c->N;
    u64 *sg = (u64 *)malloc(sizeof(u64) * 2 * LN), *ks = (u64 *)malloc(sizeof(u64) * 2 * LN);
    orc_automorphism(c, ct, l, 2, g, sg);
    orc_keyswitch(c, sg + LN, l, ksk, ks);
    orc_add(c, sg, ks, l, 1, out);
    memcpy(out + LN, ks + LN, sizeof(u64) * LN);
    free(sg);
    free(ks);
}

/* BGV modulus switching from level l to l-1 (drops q_{l-1}), per poly:
 * w = [x_{l-1} p^-1]_{q_{l-1}} in [0,q_{l-1}), delta = p w (an integer),
 * out_i = (x_i - delta) q_{l-1}^-1 mod q_i.  delta = x mod q_{l-1} and
 * delta = 0 mod p, so the plaintext mod p is unchanged (q = 1 mod p). */
void orc_modswitch(const orc_ctx *c, const u64 *ct, int l, int npoly, u64 *out)
{
    int N = c->N;
    u64 ql = c->q[l - 1], pinv = invmod(c->p % ql, ql);
    for (int k = 0; k < npoly; k++) {
        const u64 *x = ct + (size_t)k * l * N;
        u64 *o = out + (size_t)k * (l - 1) * N;
        for (int i = 0; i < l - 1; i++) {
            u64 q = c->q[i], qlinv = invmod(ql % q, q);
            for (int n = 0; n < N; n++) {
                u64 w = mulmod(x[(size_t)(l - 1) * N + n], pinv, ql);
                u64 delta = (u64)(((u128)c->p * w) % q);
                o[(size_t)i * N + n] = mulmod(submod(x[(size_t)i * N + n], delta, q), qlinv, q);
            }
        }
    }
}
