/*
 * fhe.h -- C ABI of the GB300 BGV encrypted-comparison library.
 *
 * What it computes follows BoostCom (Yudha et al., PACT'24): BGV ciphertexts
 * over R_Q = Z_Q[X]/(X^N+1) held in RNS (Sec. 2.1 "Basics and arithmetic
 * ops", Sec. 2.2 "Efficient Polynomial and NTT"), and the word-wise
 * comparison of Sec. 2.1 "Non-arithmetic Comparison": per-digit less-than and
 * equality through the univariate circuit, combined in lexicographic order.
 *
 * Conventions shared by every call
 *   - Handles are opaque.  Whatever a *_create / keygen / encrypt / arithmetic
 *     call returns through an out-pointer is owned by the caller and must be
 *     released with the matching *_destroy; a context must outlive every
 *     handle made from it.  Destroying NULL is a no-op.
 *   - Device memory comes from the allocator given to fhe_ctx_create (or
 *     cudaMallocAsync when none is given) through a pool owned by the context.
 *     Host buffers passed in are read during the call only; host buffers
 *     passed out are written before the call returns.
 *   - Every call returns 0 (FHE_OK) or a negative FHE_E* code and never
 *     aborts; fhe_last_error() describes the last failure on a context.
 *   - Work is enqueued on the context's stream (asynchronous with respect to
 *     the host) except where a call says it synchronises.
 *   - A ciphertext handle holds a batch of `count` ciphertexts of one level;
 *     binary operations act element-wise over two batches of equal count.
 *     On the device a batch is u64 [count][npoly][level][N] in the NTT
 *     (evaluation) domain; npoly is 2, or 3 after fhe_mul.
 *   - Slot values are integers in [0, p); a ciphertext holds n_s slots
 *     (fhe_info.slots).  Comparison digits must lie in [0, (p-1)/2].
 */
#ifndef FHE_GB300_H
#define FHE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fhe_ctx fhe_ctx;
typedef struct fhe_sk fhe_sk;
typedef struct fhe_pk fhe_pk;
typedef struct fhe_evk fhe_evk;
typedef struct fhe_ct fhe_ct;

enum {
    FHE_OK = 0,
    FHE_EINVAL = -1,      /* bad argument (NULL, size out of range, ...) */
    FHE_EMISMATCH = -2,   /* operands of different contexts, counts or shapes */
    FHE_ELEVEL = -3,      /* level too low for the operation */
    FHE_ENOMEM = -4,      /* device allocation failed */
    FHE_EBUDGET = -5,     /* the context's device-memory budget would be exceeded */
    FHE_ETIMEOUT = -6,    /* a bounded wait ran out */
    FHE_ECUDA = -7,       /* a CUDA runtime call failed */
    FHE_ENOKEY = -8,      /* no switching key for the requested Galois element */
    FHE_EUNSUPPORTED = -9, /* parameter combination not provided */
    FHE_ECANCELED = -10,   /* a served request was canceled before it ran */
    FHE_EBUSY = -11        /* the request already runs or is done */
};

/* BGV parameters.  The prime chain is the L+K smallest primes q with
 * q = 1 (mod prime_mod) in [prime_lo, prime_hi): the first L carry data, the
 * last K (alpha) are the special primes of hybrid key switching.  prime_mod
 * must be a multiple of 2N and of p; all primes must have one bit length
 * below 58.  log_n in [10, 14]; p an odd prime, p = 1 (mod 4) or p = 3 (mod 8). */
typedef struct {
    int log_n;
    uint64_t p;
    int L;
    int K;
    uint64_t prime_mod;
    uint64_t prime_lo;
    uint64_t prime_hi;
} fhe_params;

/* Device allocator.  alloc returns device memory of `bytes` usable in stream
 * order on `stream` (NULL on failure); free returns it. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} fhe_allocator;

typedef struct {
    int N;          /* ring degree */
    int L, K;       /* data and special primes */
    int slots;      /* n_s = N / ord_2N(p) values per ciphertext */
    int subring;    /* M: plaintexts live in Z_p[Y]/(Y^M+1), Y = X^(N/M) */
    int dnum_max;   /* key-switching digits at the top level, ceil(L/K) */
    uint64_t p;
} fhe_info;

/* ---- context ------------------------------------------------------------ */

/* Builds the prime chain, NTT tables and key-switching constants on the
 * current CUDA device.  stream: a cudaStream_t (NULL = legacy default).
 * alloc may be NULL.  Synchronises. */
int fhe_ctx_create(const fhe_params *params, const fhe_allocator *alloc, void *stream, fhe_ctx **out);
void fhe_ctx_destroy(fhe_ctx *ctx);
const char *fhe_last_error(const fhe_ctx *ctx);
int fhe_ctx_info(const fhe_ctx *ctx, fhe_info *out);
/* The L+K primes, data first.  out: host array of L+K entries. */
int fhe_ctx_primes(const fhe_ctx *ctx, uint64_t *out);
int fhe_ctx_set_stream(fhe_ctx *ctx, void *stream);
/* Waits for all work on the context's stream. */
int fhe_ctx_sync(fhe_ctx *ctx);
/* Device bytes held by the pool (reserved) and handed out (in_use).  The
 * pool hands out blocks in size classes of a quarter power of two (a block is
 * less than 25% larger than asked for), so a freed block serves later
 * requests of nearby sizes; both figures count whole blocks. */
int fhe_ctx_memory(const fhe_ctx *ctx, uint64_t *reserved, uint64_t *in_use);
/* Largest in_use since the last reset; reset != 0 restarts it from the
 * current in_use. */
int fhe_ctx_memory_peak(fhe_ctx *ctx, uint64_t *peak, int reset);
/* Every ciphertext product is tensor -> relinearise -> switch down one prime
 * (when above level 1).  With on != 0 (the default) the relinearisation's
 * ModDown and the modulus switch are carried out as one: the two
 * corrections are combined in the coefficient domain and go through one
 * forward NTT per kept limb, and the switched limb is never transformed
 * back.  The results are the same residues as with on = 0, which runs the
 * two steps separately.  Needs K + 1 <= 8 (else the steps stay separate). */
int fhe_ctx_fused_modswitch(fhe_ctx *ctx, int on);
/* Waits for the context's stream and returns the pool's cached free blocks
 * to the allocator (blocks held by handles and plans stay). */
int fhe_ctx_trim(fhe_ctx *ctx);
/* Host-side fault injection for tests of the error paths: the n-th device
 * block the pool has to obtain from now on (0 = the next one) fails as if
 * the device were out of memory (FHE_ENOMEM); n < 0 switches it off.  No
 * device fault is involved; the context stays usable. */
int fhe_ctx_inject_alloc_failure(fhe_ctx *ctx, int64_t n);
/* Cap on reserved bytes (0 = none); allocations past it fail with FHE_EBUDGET. */
int fhe_ctx_set_budget(fhe_ctx *ctx, uint64_t bytes);
/* Number of kernels this context has launched so far. */
int64_t fhe_ctx_launches(const fhe_ctx *ctx);

/* ---- keys ---------------------------------------------------------------- */

/* Key generation with caller randomness (the path the tests use).
 * s: int64[N] ternary secret; a: uint64[L][N] public-key mask, row i uniform
 * in [0, q_i), coefficient domain; e: int64[N] error.
 * pk = (-a s + p e, a) over the data primes (Sec. 2.1, RLWE public key). */
int fhe_keygen_explicit(fhe_ctx *ctx, const int64_t *s, const uint64_t *a, const int64_t *e, fhe_sk **sk,
                        fhe_pk **pk);
/* Key generation drawing s, a, e on the device from a Philox4x32-10 stream
 * keyed by seed (Salmon et al., SC'11). */
int fhe_keygen(fhe_ctx *ctx, uint64_t seed, fhe_sk **sk, fhe_pk **pk);
void fhe_sk_destroy(fhe_sk *sk);
void fhe_pk_destroy(fhe_pk *pk);

/* Evaluation keys: the relinearisation key (s^2 -> s) and one rotation key
 * (sigma_g(s) -> s) per Galois element galois[i] (odd, in (1, 2N)).
 * Hybrid key-switching keys, one per digit j of ceil(L/K) digits:
 *   ksk_j = (-a_j s + p e_j + P [i in D_j] s', a_j)  over all L+K primes,
 * D_j the data primes jK .. (j+1)K-1, P the product of the special primes.
 * Explicit randomness: a: uint64[1+n_galois][dnum][L+K][N] (coefficient
 * domain, uniform mod the prime of each row), e: int64[1+n_galois][dnum][N];
 * key 0 is the relinearisation key. */
int fhe_evk_create_explicit(fhe_ctx *ctx, const fhe_sk *sk, const int64_t *galois, int n_galois, const uint64_t *a,
                            const int64_t *e, fhe_evk **out);
int fhe_evk_create(fhe_ctx *ctx, const fhe_sk *sk, const int64_t *galois, int n_galois, uint64_t seed,
                   fhe_evk **out);
void fhe_evk_destroy(fhe_evk *evk);

/* ---- encryption ------------------------------------------------------------ */

/* Encrypts `count` slot vectors: slots uint64[count][n_s], each in [0, p).
 * Enc(m) = (pk0 u + p e0 + m, pk1 u + p e1) at level L, with m the slot
 * encoding.  u, e0, e1: int64[count][N].  Synchronises. */
int fhe_encrypt_explicit(fhe_ctx *ctx, const fhe_pk *pk, const uint64_t *slots, int count, const int64_t *u,
                         const int64_t *e0, const int64_t *e1, fhe_ct **out);
int fhe_encrypt(fhe_ctx *ctx, const fhe_pk *pk, const uint64_t *slots, int count, uint64_t seed, fhe_ct **out);
/* Decrypts every ciphertext of the batch: a copy is modulus-switched to one
 * prime, m = [c0 + c1 s]_{q0} (centred) mod p, then decoded.
 * slots: uint64[count][n_s].  Fails with FHE_EINVAL if a plaintext is not a
 * slot-constant encoding.  Synchronises. */
int fhe_decrypt(fhe_ctx *ctx, const fhe_sk *sk, const fhe_ct *ct, uint64_t *slots);
/* Refresh: a stand-in for bootstrapping, which the paper does not cover (it
 * needs the secret key).  Every ciphertext's plaintext is recovered on the
 * device (as in fhe_decrypt) and encrypted again at level L with fresh
 * randomness: explicit u, e0, e1 (int64[count][N]) or the seeded samplers.
 * Used by long max/min tournaments whose depth exceeds the modulus chain. */
int fhe_refresh_explicit(fhe_ctx *ctx, const fhe_sk *sk, const fhe_pk *pk, const fhe_ct *ct, const int64_t *u,
                         const int64_t *e0, const int64_t *e1, fhe_ct **out);
int fhe_refresh(fhe_ctx *ctx, const fhe_sk *sk, const fhe_pk *pk, const fhe_ct *ct, uint64_t seed, fhe_ct **out);
/* n blocks of Philox4x32-10 (4 words each) of stream `tag` under `seed`,
 * computed on the current device: the generator behind the seeded calls.
 * out: host uint32[4n].  Synchronises. */
int fhe_philox_blocks(uint64_t seed, uint32_t tag, int n, uint32_t *out);
void fhe_ct_destroy(fhe_ct *ct);
int fhe_ct_shape(const fhe_ct *ct, int *count, int *npoly, int *level);
/* Coefficient-domain residues, host uint64[count][npoly][level][N].  Synchronises. */
int fhe_ct_export_coeff(fhe_ctx *ctx, const fhe_ct *ct, uint64_t *host);
int fhe_ct_import_coeff(fhe_ctx *ctx, const uint64_t *host, int count, int npoly, int level, fhe_ct **out);
/* Overwrites an existing ciphertext batch in place from host coefficient-domain
 * residues of its own shape (uint64[count][npoly][level][N]); asynchronous on
 * the context's stream (host must stay valid until the stream reaches it).
 * This is how new inputs reach a captured plan (fhe_compare_plan). */
int fhe_ct_load_coeff(fhe_ctx *ctx, fhe_ct *ct, const uint64_t *host);

/* Checkpoint / resume of a ciphertext batch.  The image is a 32-byte header
 * ("FHEC", version 1, log2 N, polynomials, count, level as u32; p as u64),
 * the level's primes q_0 .. q_{level-1} (u64), then the coefficient-domain
 * limbs [count][npoly][level][N] (u64, as fhe_ct_export_coeff writes them);
 * host byte order.  fhe_ct_serialize stores the image size in *size and, when
 * buf is non-NULL, writes the image (FHE_EINVAL if cap is smaller); it
 * synchronises.  fhe_ct_deserialize creates a new handle in ctx from an image,
 * refusing one of another ring degree, plaintext modulus or prime chain
 * (FHE_EMISMATCH), a truncated or oversized buffer or a residue not below its
 * prime (FHE_EINVAL).  Keys are not imaged: the seeded key generators
 * recreate them. */
int fhe_ct_serialize(fhe_ctx *ctx, const fhe_ct *ct, void *buf, uint64_t cap, uint64_t *size);
int fhe_ct_deserialize(fhe_ctx *ctx, const void *buf, uint64_t size, fhe_ct **out);

/* ---- arithmetic (Sec. 2.1: add, mult, rotate; Sec. 2.2: RNS, NTT) -------- */

/* Operands at different levels are first modulus-switched (one prime at a
 * time) to the lower level. */
int fhe_add(fhe_ctx *ctx, const fhe_ct *a, const fhe_ct *b, fhe_ct **out);
int fhe_sub(fhe_ctx *ctx, const fhe_ct *a, const fhe_ct *b, fhe_ct **out);
int fhe_neg(fhe_ctx *ctx, const fhe_ct *a, fhe_ct **out);
/* Multiply by / add the constant c of Z_p (lifted to (-p/2, p/2]). */
int fhe_mul_const(fhe_ctx *ctx, const fhe_ct *a, int64_t c, fhe_ct **out);
int fhe_add_const(fhe_ctx *ctx, const fhe_ct *a, int64_t c, fhe_ct **out);
/* Tensor product: 3-poly result (c0 d0, c0 d1 + c1 d0, c1 d1). */
int fhe_mul(fhe_ctx *ctx, const fhe_ct *a, const fhe_ct *b, fhe_ct **out);
/* Hybrid key switching of the third poly with the relinearisation key:
 * INTT, ModUp per digit (fast basis conversion + NTT), inner product with the
 * key, ModDown (BGV: the correction is a multiple of p). */
int fhe_relinearize(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *a, fhe_ct **out);
/* BGV modulus switching down to target_level (>= 1), one prime at a time:
 * x' = (x - p [x_last p^-1]_{q_last}) q_last^-1.  q = 1 (mod p), so the
 * plaintext is unchanged. */
int fhe_mod_switch(fhe_ctx *ctx, const fhe_ct *a, int target_level, fhe_ct **out);
/* Galois automorphism X -> X^g followed by key switching back to s. */
int fhe_rotate(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *a, int64_t galois, fhe_ct **out);
/* The circuit product: align levels, tensor, relinearise, then
 * modulus-switch by one prime when the level is above 1. */
int fhe_mul_relin(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *a, const fhe_ct *b, fhe_ct **out);

/* ---- comparison (Sec. 2.1 "Non-arithmetic Comparison") ------------------- */

/* x, y: arrays of d ciphertext handles, digit k of both operands (least
 * significant first, digits in [0, (p-1)/2]); all handles of one call have
 * the same count.  Per digit z = x_k - y_k, LT_k = f(z) with f the
 * interpolating polynomial of [z >= (p+1)/2] evaluated by Paterson-Stockmeyer,
 * EQ_k = 1 - z^(p-1); digits merged pairwise, L = L_hi + E_hi L_lo,
 * E = E_hi E_lo.  Results decrypt to 1 / 0 in every slot. */
int fhe_compare_lt(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                   fhe_ct **out);
int fhe_compare_eq(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                   fhe_ct **out);
/* Both at once (they share z^(p-1)). */
int fhe_compare(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                fhe_ct **lt, fhe_ct **eq);
/* The bivariate circuit (Sec. 2.1) on full digits in [0, p), so values of d
 * digits span [0, p^d): per digit LT_k = sum_a x^a h_a(y), the unique
 * polynomial of degree <= p-1 in each variable equal to [x < y] on Z_p x Z_p
 * (h_a = sum_{b>=1} c[a][b] y^b; powers of x and y by squaring and products;
 * 2(p-2) power products plus one product per row a >= 1), EQ_k =
 * 1 - (x - y)^(p-1), the same digit merge.  Depth ceil(log2(p-1)) + 1 per
 * digit.  lt and/or eq as for fhe_compare. */
int fhe_compare_bivariate(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                          fhe_ct **lt, fhe_ct **eq);
/* max / min digit-wise: L = LT(x, y); t_k = L (y_k - x_k);
 * max_k = x_k + t_k, min_k = y_k - t_k.  out_max / out_min: d handles each
 * (either may be NULL). */
int fhe_max_min(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                fhe_ct **out_max, fhe_ct **out_min);
int fhe_max(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
            fhe_ct **out);
int fhe_min(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
            fhe_ct **out);

/* ---- captured batches (CUDA graphs) -------------------------------------------- */

typedef struct fhe_plan fhe_plan;

/* Plan flags. */
enum { FHE_PLAN_SERIAL = 1,    /* record every kernel on one stream (no parallel branches) */
       FHE_PLAN_BIVARIATE = 2 /* the bivariate circuit on full digits (fhe_compare_bivariate) */ };

/* Records fhe_compare(x, y) (the LT and/or EQ outputs selected by want_lt /
 * want_eq) as one CUDA graph: one warm run, then a capture.  Independent
 * digit circuits become parallel branches of the graph unless flags has
 * FHE_PLAN_SERIAL.  The plan owns its outputs and every temporary the graph
 * reuses; x and y stay bound to the plan (the caller keeps them alive and may
 * overwrite their contents between runs).  Synchronises. */
int fhe_compare_plan(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                     int want_lt, int want_eq, int flags, fhe_plan **out);
/* Enqueues one replay of the recorded comparison on the context's stream. */
int fhe_plan_run(fhe_plan *plan);
/* Borrowed handle of output `which` (0 = LT, 1 = EQ), valid until the plan is
 * destroyed; each run overwrites it. */
int fhe_plan_result(const fhe_plan *plan, int which, const fhe_ct **out);
/* Kernel nodes in the recorded graph. */
int fhe_plan_nodes(const fhe_plan *plan);
void fhe_plan_destroy(fhe_plan *plan);

/* ---- tournament max / min -------------------------------------------------------- */

/* Galois elements the tournament rotates by (write up to cap; returns how
 * many): 5^(2^i) mod 2N for 2^i = n_s/4 .. 1, then 2N-1.  The evaluation keys
 * passed to fhe_tournament must include all of them. */
int fhe_tournament_galois(const fhe_ctx *ctx, int64_t *galois, int cap);
/* Max and/or min over every slot of every ciphertext of the batches x[0..d-1]
 * (digit k of all values, least significant first; count n ciphertexts of
 * n_s slots each).  The maximum over max_min of Sec. 2.1 "Non-arithmetic
 * Comparison" (min/max of the BGV comparison work): cross rounds pair
 * ciphertexts [0, h) with [h, 2h) (h = n/2, an odd last one passes on), then
 * in-slot rounds combine each ciphertext with its rotation by the elements of
 * fhe_tournament_galois.  out_max / out_min: d single-ciphertext handles whose
 * every slot holds the result (either may be NULL).  A round that would end
 * below level 1 is preceded by fhe_refresh with seeds derived from `seed`
 * (needs sk and pk; without them such a round fails with FHE_ELEVEL). */
int fhe_tournament(fhe_ctx *ctx, const fhe_evk *evk, const fhe_sk *sk, const fhe_pk *pk, const fhe_ct *const *x,
                   int d, uint64_t seed, fhe_ct **out_max, fhe_ct **out_min);

/* ---- plaintext operands and sorting --------------------------------------------- */

/* ct + pt, ct - pt, ct * pt for one plaintext slot vector `slots` (n_s
 * values, host array, reduced mod p) applied to every ciphertext of the
 * batch.  The encoding's coefficients are lifted to (-p/2, p/2] before
 * reduction mod q_i; + and - change c0 only; no level is consumed. */
int fhe_add_plain(fhe_ctx *ctx, const fhe_ct *a, const uint64_t *slots, fhe_ct **out);
int fhe_sub_plain(fhe_ctx *ctx, const fhe_ct *a, const uint64_t *slots, fhe_ct **out);
int fhe_mul_plain(fhe_ctx *ctx, const fhe_ct *a, const uint64_t *slots, fhe_ct **out);

/* Sorting (the paper's sort application, Sec. 6): every row of cols = n_s / 2
 * slots of every ciphertext is sorted on its own, in increasing order, its
 * values given as d univariate digit handles x[0..d-1] (least significant
 * first).  rank_i counts the row's values below x_i, and equal values
 * earlier in the row: the sum over column shifts s of LT(x_{i+s}, x_i) plus
 * the plaintext tie-break mask [i + s >= cols] times EQ(x_{i+s}, x_i); the
 * sorted row is the sum over shifts of EQ(rank_{i+s} - i) x_{i+s}, EQ(u) =
 * 1 - u^(p-1) (exact because ranks are below cols <= p).  Needs p = 1 mod 4,
 * cols >= 2 and the column rotations of fhe_sort_galois in evk; consumes
 * the comparison's depth + ceil(log2(p-1)) + 1 levels.  out: d new handles. */
int fhe_sort_galois(const fhe_ctx *ctx, int64_t *galois, int cap);

/* Private query with straight-lined branches and non-blocking comparison
 * (Sec. 5.3): q holds the encrypted query type, compared for equality with
 * the three public codes codes[0..2] (add, multiply, power); the answer is
 *   (data + op1) EQ(q, codes[0]) + (data * op1) EQ(q, codes[1])
 *     + data^op2 EQ(q, codes[2]),
 * with EQ(q, k) = 1 - (q - k)^(p-1) (so 0 where q matches no code).  q, data
 * and op1: equal count, any levels (products align levels by switching
 * down).  Consumes ceil(log2(p-1)) + 1 levels beyond the lowest input, or
 * more when op2 needs a longer power chain.  flags FHE_QUERY_OVERLAP: the
 * comparison branch and the arithmetic are issued to the dependency
 * scheduler's streams and run concurrently on the device (the paper's helper
 * thread), joining at the selection; 0 issues everything on the context's
 * stream in order.  Same residues either way. */
enum { FHE_QUERY_OVERLAP = 1 };
int fhe_private_query(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *q, const fhe_ct *data, const fhe_ct *op1,
                      int op2, const int64_t *codes, int flags, fhe_ct **out);
/* The private query recorded as a CUDA graph (see fhe_compare_plan: the
 * plan binds the three input handles, whose contents the caller may
 * overwrite between runs; fhe_plan_run replays it; fhe_plan_result(plan, 0)
 * is the answer).  flags: 0 records the branches on parallel streams (the
 * overlap of FHE_QUERY_OVERLAP), FHE_PLAN_SERIAL records one stream. */
int fhe_private_query_plan(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *q, const fhe_ct *data,
                           const fhe_ct *op1, int op2, const int64_t *codes, int flags, fhe_plan **out);

/* F_{p^d} slots and digit extraction ("mod extract", Sec. 2.1): a d-digit
 * operand is held in ONE ciphertext whose every slot is an element of F_{p^d};
 * the server splits it into d ciphertexts of F_p digits, the form the
 * comparison calls take.
 *
 * Slot fields: slot s of the F_p-slot structure has the factor g_s of Y^M + 1
 * (Y - zeta^e_s for p = 1 mod 4, Y^2 +- gamma Y - 1 for p = 3 mod 8).  For
 * d = e deg(g_s), e a power of two with M e <= N, the subring generated by
 * Y' = X^(N/(M e)) has one factor f_s(Y') = g_s(Y'^e) per slot: slot s is the
 * field F_p[Y']/(f_s), and digit k of a slot element is its coefficient of
 * Y'^k (d = 1, 2, 4 .. for p = 17 and 257; 2, 4, .. for p = 131).
 * FHE_EUNSUPPORTED for a d the ring has no slots of.
 *
 * digits: count x n_s x d u64 in [0, p) (ciphertext, slot, digit; least
 * significant first).  fhe_encrypt_ext / _explicit encode and encrypt like
 * fhe_encrypt / _explicit.  fhe_decrypt_ext decrypts to that layout
 * (FHE_EINVAL if the plaintext is not such an encoding).
 *
 * fhe_extract_digits: out[0 .. d) receive new handles, digit k of every slot
 * as an F_p constant in out[k], at the input's level (none consumed):
 * digit k = Tr(lambda_k x) = sum_{t<d} lambda_k^(p^t) sigma_{p^t}(x), lambda
 * the trace-dual basis of 1, Y', .., Y'^(d-1).  Costs d - 1 rotations (keys:
 * fhe_ext_galois, p^t mod 2N for t = 1 .. d-1) and d^2 plaintext products.
 * fhe_ext_galois returns the count and writes up to cap elements. */
int fhe_ext_galois(fhe_ctx *ctx, int d, int64_t *galois, int cap);
int fhe_encrypt_ext(fhe_ctx *ctx, const fhe_pk *pk, const uint64_t *digits, int count, int d, uint64_t seed,
                    fhe_ct **out);
int fhe_encrypt_ext_explicit(fhe_ctx *ctx, const fhe_pk *pk, const uint64_t *digits, int count, int d,
                             const int64_t *u, const int64_t *e0, const int64_t *e1, fhe_ct **out);
int fhe_decrypt_ext(fhe_ctx *ctx, const fhe_sk *sk, const fhe_ct *ct, int d, uint64_t *digits);
int fhe_extract_digits(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *ct, int d, fhe_ct **out);

/* Slot manager and slot compaction (Sec. 5.3, "Slot Compaction"): inputs whose
 * useful values fill only some slots are compacted into as few ciphertexts as
 * the slot rotations allow, before comparison.
 *
 * useful: n x n_s bytes, row j for input j, nonzero where slot u (index
 * r cols + c, cols = n_s / 2, or 1 for n_s = 2) holds a useful value; the
 * other slots may hold anything and are masked off.  Placement, in order of
 * input: the slots of input j still to place go, under one slot rotation
 * (columns shifted right by s, rows swapped when b), into the open output
 * that takes the most of them (first output, then b, then s, wins a tie); an
 * output opens only when every open one is full.  Each such piece costs a
 * plaintext mask, sigma_{5^(cols - s)} when s > 0, sigma_{2N-1} when b, and
 * an addition.
 *
 * fhe_slot_plan (host only: slots = n_s and ring_n = N of the context, as
 * fhe_ctx_info reports them) returns the number of outputs and, when non-NULL,
 * fills dest (n x n_s int32: output * n_s + slot, or -1 for slots that are
 * not useful) and galois (up to galois_cap rotation elements the plan needs:
 * column shifts ascending, then 2N - 1) with their count in *n_galois.
 * fhe_slot_pack evaluates the plan on inputs of equal count (any levels; sums
 * are taken at the lower level) and returns the number of outputs written to
 * out[0 .. out_cap); FHE_EINVAL when out_cap is smaller, FHE_ENOKEY when evk
 * lacks a rotation the plan needs.  No level is consumed. */
int fhe_slot_plan(int slots, int64_t ring_n, int n, const uint8_t *useful, int32_t *dest, int64_t *galois,
                  int galois_cap, int *n_galois);
int fhe_slot_pack(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *const *in, int n, const uint8_t *useful,
                  fhe_ct **out, int out_cap);
int fhe_sort(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *const *x, int d, fhe_ct **out);
/* Joint sort of sequences longer than a row: row r of the K batches
 * x[a * d + k] (batch a, digit k; equal count and level) is one sequence of
 * K cols values, value (a, c) at global index a cols + c.  rank^a sums, over
 * every (b, s) != (a, 0), LT(sigma_{5^s} x^b, x^a) plus the tie-break mask
 * [b cols + (c + s) mod cols < a cols + c] times EQ; the output batch t holds
 * positions t cols .. t cols + cols - 1 of the sorted sequence: the sum over
 * (a, s) of EQ(sigma_{5^s} rank^a - (t cols + c)) sigma_{5^s} x^a.  Needs
 * K cols <= p (FHE_EINVAL otherwise) and the keys of fhe_sort_galois; K = 1
 * is fhe_sort.  Costs K^2 cols - K comparisons and K^2 cols selection
 * powers.  out: K * d new handles, out[t * d + k]. */
int fhe_sort_joint(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *const *x, int K, int d, fhe_ct **out);
/* The sort application (Sec. 6) on sequences of any length, K cols values a
 * row, including K cols > p, where the selection step of fhe_sort_joint would
 * no longer be exact: the rank step alone.  ranks[a] (K new handles) holds in
 * slot (r, c) the rank of value (a, c) of row r -- the number of values of
 * the row below it plus those equal to it at a lower global index -- mod p.
 * matrix, when not NULL, receives K * K * cols handles: matrix[(a K + b) cols
 * + s] = LT(sigma_{5^s} x^b, x^a), whose slot (r, c) is [x_j < x_i] for
 * i = a cols + c and j = b cols + (c + s) mod cols (NULL at s = 0, b = a).
 * Inputs as for fhe_sort_joint (keys of fhe_sort_galois); costs K^2 cols - K
 * comparisons. */
int fhe_sort_ranks(fhe_ctx *ctx, const fhe_evk *evk, const fhe_ct *const *x, int K, int d, fhe_ct **ranks,
                   fhe_ct **matrix);

/* ---- batches of uneven requests ------------------------------------------------- */

enum { FHE_JOB_COMPARE = 1, /* out0 -> &LT handle, out1 -> &EQ handle (either NULL) */
       FHE_JOB_MAXMIN = 2,  /* out0 -> d max digit handles, out1 -> d min digit handles */
       FHE_JOB_SORT = 3     /* rows of x sorted as fhe_sort does: y ignored (may be NULL),
                               out0 -> d sorted digit handles, out1 NULL; evk must hold
                               fhe_sort_galois; p = 1 mod 4 rings only */ };

/* One request: the d digit handles x[], y[] (equal count and level) of one
 * context.  Output handles are written at submission and hold the results
 * once fhe_batch_wait returns 0; the caller destroys them. */
typedef struct {
    fhe_ctx *ctx;
    const fhe_evk *evk;
    int kind;
    int d;
    const fhe_ct *const *x;
    const fhe_ct *const *y;
    fhe_ct **out0;
    fhe_ct **out1;
} fhe_job;

typedef struct fhe_batch fhe_batch;

/* Submits n jobs of any mix of contexts (ring degree, plaintext prime),
 * digit counts and levels.  Jobs of one (context, keys, kind, digits, level)
 * are concatenated into one batch; every group of a context runs in one
 * dependency-scheduled circuit on 8 streams, so groups overlap on the device;
 * contexts run on their own streams.  Each result equals what the job gives
 * alone.  Enqueues and returns; `*out` tracks completion. */
int fhe_batch_submit(const fhe_job *jobs, int n, fhe_batch **out);
/* fhe_batch_submit with options.  FHE_BATCH_ALIGN_LEVELS: within each
 * (context, keys, kind, digits, wanted outputs), jobs above the lowest level
 * among them are first switched down to it (copies; the caller's handles are
 * untouched), so that they share one group and its launches.  Each result
 * then equals the job run alone from that lower level.  The lowest level must
 * leave the circuit its depth, as it does when every job of the group could
 * run alone at its own level.
 * FHE_BATCH_FUSE_RINGS: the compare and max/min jobs of all contexts that
 * share a device and a plaintext prime (hence the digit polynomial) run in
 * one circuit, whose every step is one kernel launch over all their groups:
 * ring degrees, digit counts and levels mixed in one launch (the first such
 * context's stream carries the work; the others' streams wait for it).
 * A submission shape such a family has served before is captured (once)
 * into one CUDA graph for the family and replayed (up to 4 graphs per family;
 * they hold memory in every member's pool and are dropped when a member
 * context is destroyed -- do not destroy a context while another thread
 * submits a fused batch that involves it).  Results are those of each job
 * alone. */
enum { FHE_BATCH_ALIGN_LEVELS = 1, FHE_BATCH_FUSE_RINGS = 2 };
int fhe_batch_submit_ex(const fhe_job *jobs, int n, int flags, fhe_batch **out);
/* Graph capture of recurring submissions: the second time a context receives
 * the same group shapes (keys, kind, digits, level, ciphertexts per group),
 * its circuit is captured into a CUDA graph with operand and result buffers
 * of its own; later submissions of that shape copy the operands in, replay
 * the graph and slice the results out (identical bits).  At most max_plans
 * graphs are kept per context, least recently used evicted (default 4; 0
 * turns capture off and frees the kept graphs). */
int fhe_ctx_set_batch_graphs(fhe_ctx *ctx, int max_plans);
/* 0 once every job of the batch is complete; FHE_ETIMEOUT if that takes
 * longer than timeout_ms (the batch keeps running; wait again later). */
int fhe_batch_wait(fhe_batch *batch, int timeout_ms);
/* Per-job completion, without waiting: 1 once job i (its index in the
 * submission) has its results, 0 if not yet, FHE_EINVAL for a bad index.  A
 * submission runs its compare and max/min jobs before its sort jobs, with
 * one completion event per phase and context, so a job need not wait for
 * the sorts of its batch (or for other contexts' work). */
int fhe_batch_job_done(fhe_batch *batch, int i);
/* Waits for the batch and releases its tracking state (not the outputs). */
void fhe_batch_destroy(fhe_batch *batch);

/* ---- serving loop ---------------------------------------------------------------- */

/* A worker thread that serves requests (fhe_job) submitted from any thread.
 * It admits queued requests in arrival order while the sum of their
 * footprint estimates (fhe_job_footprint) stays within hbm_budget bytes (a
 * request that arrives at an empty server is always admitted; one whose
 * estimate alone exceeds the budget is refused with FHE_EBUDGET at
 * submission), and submits all requests admitted at one time as one
 * fhe_batch_submit; it enqueues the next batch while earlier ones still run
 * (continuous batching).  Contexts and keys stay resident and belong to the
 * caller, as do the input handles (valid until the request is done) and the
 * outputs: the handles are written to the job's out0/out1 arrays, which must
 * stay valid until fhe_server_poll reports the request done. */
enum { FHE_REQ_QUEUED = 0, FHE_REQ_RUNNING = 1, FHE_REQ_DONE = 2 };

typedef struct {
    uint64_t hbm_budget; /* bytes; 0 = no limit */
    int max_batch;       /* most requests per submission; 0 = no limit */
    int batch_flags;     /* passed to fhe_batch_submit_ex (e.g. FHE_BATCH_ALIGN_LEVELS) */
} fhe_server_config;

typedef struct {
    int state;           /* FHE_REQ_* */
    int error;           /* 0, or the FHE_E* code the request ended with */
    double t_submit_ms;  /* server clock (ms since fhe_server_start) */
    double t_start_ms;   /* admitted and submitted */
    double t_done_ms;    /* completion seen by the worker (polled every 50 us) */
    uint64_t est_bytes;  /* fhe_job_footprint */
} fhe_request_info;

typedef struct {
    long long queued, running, completed, failed, batches;
    uint64_t admitted_bytes, admitted_peak_bytes;
} fhe_server_status;

typedef struct fhe_server fhe_server;

/* Estimated device bytes a request allocates while it runs: the circuit's
 * working set per digit, the key-switching scratch of up to 8 concurrent
 * digits and the outputs, in whole pool blocks (0 for an invalid job). */
uint64_t fhe_job_footprint(const fhe_job *job);
/* cfg may be NULL (no budget, no batch limit). */
int fhe_server_start(const fhe_server_config *cfg, fhe_server **out);
/* Validates and queues a copy of *job (and of its x/y arrays); *ticket
 * identifies it.  FHE_EINVAL after fhe_server_stop has begun. */
int fhe_server_submit(fhe_server *server, const fhe_job *job, uint64_t *ticket);
/* Waits up to timeout_ms (0: does not wait) for the request; returns 1 when
 * it is done (the ticket is then retired), 0 when not yet, FHE_EINVAL for an
 * unknown ticket.  info may be NULL. */
int fhe_server_poll(fhe_server *server, uint64_t ticket, int timeout_ms, fhe_request_info *info);
/* Cancels a request that is still queued: it reports done with error
 * FHE_ECANCELED and writes no outputs.  FHE_EBUSY if it was already admitted
 * (its batch runs to completion), FHE_EINVAL for an unknown ticket (including
 * one retired by fhe_server_poll reporting it done). */
int fhe_server_cancel(fhe_server *server, uint64_t ticket);
int fhe_server_stats(fhe_server *server, fhe_server_status *status);
/* Serves every request already submitted, joins the worker and frees the
 * server; tickets not yet polled are retired with it. */
int fhe_server_stop(fhe_server *server);

/* ---- operation trace --------------------------------------------------------- */

/* Op codes recorded while tracing is on. */
enum { FHE_OP_MUL = 1, FHE_OP_ADD = 2, FHE_OP_SUB = 3, FHE_OP_CMUL = 4, FHE_OP_CADD = 5, FHE_OP_NEG = 6,
       FHE_OP_ROT = 7, FHE_OP_PADD = 8, FHE_OP_PSUB = 9, FHE_OP_PMUL = 10 };
/* on != 0 clears and starts recording circuit-level operations. */
int fhe_trace_enable(fhe_ctx *ctx, int on);
/* Copies up to cap entries (op code, level of the operands); returns the
 * number recorded (>= 0) or an error code. */
int fhe_trace_get(const fhe_ctx *ctx, int32_t *ops, int32_t *levels, int cap);

/* ---- transforms on caller buffers (device pointers) ------------------------- */

/* In-place forward / inverse negacyclic NTT of nlimbs limbs of N residues at
 * device address data (limb i reduced mod prime prime_idx[i], host array).
 * Forward output is in bit-reversed order: A[k] = a(psi^(2 brv(k)+1)). */
int fhe_ntt_forward(fhe_ctx *ctx, uint64_t *data, const int32_t *prime_idx, int nlimbs);
int fhe_ntt_inverse(fhe_ctx *ctx, uint64_t *data, const int32_t *prime_idx, int nlimbs);
/* The same transforms over count RNS polynomials in one launch:
 * data = uint64[count][nprimes][N] (device), limb i of every polynomial
 * reduced mod prime i (nprimes <= L + K). */
int fhe_ntt_forward_batch(fhe_ctx *ctx, uint64_t *data, int count, int nprimes);
int fhe_ntt_inverse_batch(fhe_ctx *ctx, uint64_t *data, int count, int nprimes);

/* ---- integer-pipe peaks --------------------------------------------------------- */

/* Measures this GPU's throughput of 32-bit multiply-adds and of 64-bit high
 * products (__umul64hi), in operations per second over all SMs, with fixed
 * trip count kernels on the current device.  The NTT's Shoup butterfly does
 * one 64-bit high product, so butterflies/s over mulhi64 is its integer-pipe
 * fraction.  Synchronises the device. */
int fhe_probe_int_peak(double *imad32, double *mulhi64);
/* Measured butterflies per second over all SMs: the NTT's lazy forward
 * butterfly with a Shoup twiddle, in the form the NTT kernels run (the
 * quotient from one 32x32->64 and two 32x32->high products, the product
 * a w - qhat q as one multiply-add chain; result in [0, 4q); then the two
 * lazy additions) on register-resident values, three dependent layers per
 * iteration, no memory traffic: the arithmetic roof the NTT kernels are
 * reported against.  Synchronises the device. */
int fhe_probe_bfly_peak(double *bfly_per_s);

/* ---- modulus switching without allocation -------------------------------------- */

/* No counterpart in the paper.  For callers that cannot allocate device
 * memory -- a host framework that owns all of it and lends fixed buffers, or
 * a loop that must not pay for a cudaMalloc -- one modulus switch
 * level -> level-1 of caller-owned device buffers:
 *   in  = uint64[count][npoly][level][N]    (NTT domain, read only)
 *   out = uint64[count][npoly][level-1][N]  (NTT domain, must not overlap in)
 * with npoly 2 or 3 and 2 <= level <= L.  Its only temporary is a fixed
 * device array of 2^20 words (8 MiB) inside the library, held on every device
 * that loads the library until the process exits; count*npoly*N above 2^20
 * fails with FHE_EINVAL.  It calls no allocator.  The device current at the
 * call must be the one the context was created on (else FHE_EINVAL, before
 * any GPU work).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and must come before any stream capture: a
 * first call while the context's stream is capturing fails with FHE_EINVAL.
 * All calls share the array, so calls whose GPU work overlaps (other streams
 * or contexts on the same device) race and must be serialised by the caller.
 * The result equals fhe_mod_switch(.., level-1). */
int fhe_mod_switch_noalloc(fhe_ctx *ctx, const uint64_t *in, uint64_t *out, int count, int npoly, int level);

/* ---- NTT autotuning ------------------------------------------------------------ */

/* The NTT splits N = 2^n1 x 2^n2 (n1 = ceil(n/2)) into a column pass and a
 * row pass, each one kernel whose CTAs (128 threads) work on units of 2048
 * residues; one launch serves batches of any ring degree 2^10..2^15 and
 * level.  The variant is the grid policy: variant 0 launches one CTA per
 * unit; variants 1, 2 and 3 launch 6, 4 and 2 resident CTAs per SM that walk
 * all units (persistent CTAs).  fhe_ctx_create times the variants on a
 * representative batch and keeps variant 0 unless another is at least 3%
 * faster; fhe_ctx_autotune(ctx, njobs) re-times them on njobs limbs.  Both
 * return the chosen variant.
 * fhe_ctx_ntt_variant(ctx, set, ms): set >= 0 forces a variant (FHE_EINVAL if
 * it does not exist; set < 0 only reads); ms[4] (may be NULL) receives the
 * last timings in milliseconds.  All variants give identical results.
 * The environment variable FHE_NTT_VARIANT (a digit) pins the variant for
 * contexts created afterwards, skipping the timing (for profiling runs,
 * whose timings would mislead the choice).
 * njobs counts limb transforms: polynomials of min(L+K, 10) limbs, rounded
 * to a multiple of 16 polynomials once there are 16 or more. */
int fhe_ctx_autotune(fhe_ctx *ctx, int njobs);
int fhe_ctx_ntt_variant(fhe_ctx *ctx, int set, float *ms);

/* ---- kernel timing ------------------------------------------------------------- */

/* Kernel classes timed by fhe_ctx_profile_read. */
enum { FHE_K_NTT_FWD = 0, FHE_K_NTT_INV = 1, FHE_K_NTT_MODUP = 2, FHE_K_NTT_MODDOWN = 3, FHE_K_NTT_MODSWITCH = 4,
       FHE_K_KS_INNER = 5, FHE_K_TENSOR = 6, FHE_K_ELEMWISE = 7, FHE_K_AUTOMORPHISM = 8, FHE_K_COUNT = 9 };
/* on != 0: record a CUDA event pair on the context's stream around every
 * kernel launch (for per-class device time); off by default. */
int fhe_ctx_profile(fhe_ctx *ctx, int on);
/* Synchronises, then writes per class (arrays of ncls entries, any may be
 * NULL) the summed device milliseconds, the number of launches, the
 * algorithmic bytes moved (global words each kernel must read and write, x8)
 * and the NTT butterflies executed, for the launches recorded since the last
 * read; then forgets the records.  Returns FHE_K_COUNT. */
int fhe_ctx_profile_read(fhe_ctx *ctx, double *ms, int64_t *count, double *bytes, double *bfly, int ncls);

/* ---- self test ---------------------------------------------------------------- */

/* Runs the library's modular-arithmetic routines (the same source the kernels
 * use, compiled for the host) against 128-bit reference arithmetic on `iters`
 * pseudo-random and edge-case inputs per prime of the given chain.  Needs no
 * GPU.  Returns 0 if all agree, else the number of mismatches. */
int fhe_selftest_modarith(uint64_t prime_mod, uint64_t prime_lo, uint64_t prime_hi, int nprimes, int iters);

#ifdef __cplusplus
}
#endif
#endif /* FHE_GB300_H */
