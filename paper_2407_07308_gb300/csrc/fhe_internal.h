// fhe_internal.h -- library-private types shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <map>
#include <memory>
#include <unordered_map>
#include <vector>

#include "../../include/fhe.h"
#include "modarith.cuh"
#include "pdl.cuh"

#include <nvtx3/nvToolsExt.h>

// NVTX range over a scope: every public evaluation call and every circuit
// product and rotation shows up by name on a profiler's timeline (the calls
// cost nothing measurable when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define FHE_RANGE(name) NvtxRange fhe_nvtx_range_(name)

#define FHE_MAXP 32  // max data + special primes
#define FHE_MAXK 8   // max special primes (alpha)
#define FHE_MAXD 8   // max key-switching digits

// ---------------------------------------------------------------------------
// kernel parameter blocks (passed by value)
// ---------------------------------------------------------------------------

// Which limbs a batched transform touches.  Job j of a launch handles limb
// (j % nl) of "outer" item (j / nl):
//   input  = in  + (j / nl) * in_outer  + in_limb[j % nl]  * N
//   output = out + (j / nl) * out_outer + out_limb[j % nl] * N
//   prime  = prime[j % nl]
struct LimbMap {
    int nl;
    int pad;
    long long in_outer, out_outer;  // in u64 elements
    int in_limb[FHE_MAXP];
    int out_limb[FHE_MAXP];
    int prime[FHE_MAXP];
};

// ModUp of all digits at one level (fast basis conversion, coefficient
// domain, fused with the forward NTT of each new limb).  Job j handles
// (ct c = j / njobs_per_ct, then entry e = j % njobs_per_ct): digit[e],
// target extended limb tgt[e] (0..l+K-1), its prime tprime[e].
struct ModUpParams {
    int l, K, dnum, njobs;          // njobs per ciphertext
    int digit_lo[FHE_MAXD];         // first data limb of digit j
    int digit_n[FHE_MAXD];          // limbs in digit j
    int job_digit[FHE_MAXD * FHE_MAXP];
    int job_tgt[FHE_MAXD * FHE_MAXP];
    int job_prime[FHE_MAXD * FHE_MAXP];
    u64 inv_hat[FHE_MAXD][FHE_MAXK];    // (Q_j/q_i)^-1 mod q_i
    u64 inv_hat_s[FHE_MAXD][FHE_MAXK];  // its Shoup constant
    // hat[j][i][t] = (Q_j/q_i) mod (prime of extended limb t)
    u64 hat[FHE_MAXD][FHE_MAXK][FHE_MAXP];
};

// ModDown of (acc0, acc1) from Q_l P to Q_l, fused with the forward NTT of
// the correction.  Job j: ct c = j / (2 l), poly = (j / l) % 2, limb i = j % l.
struct ModDownParams {
    int l, K;
    u64 cinv[FHE_MAXK], cinv_s[FHE_MAXK];  // p^-1 (P/p_k)^-1 mod p_k
    u64 phat[FHE_MAXK][FHE_MAXP];          // p (P/p_k) mod q_i
    u64 pinv[FHE_MAXP], pinv_s[FHE_MAXP];  // P^-1 mod q_i
    int sprime[FHE_MAXK];                  // prime index of special limb k
};

// Modulus switch l -> l-1, fused with the forward NTT of the correction.
// Job j: ct c = j / (npoly (l-1)), poly = (j / (l-1)) % npoly, limb i = j % (l-1).
struct ModSwitchParams {
    int l, npoly;
    u64 pinv_last, pinv_last_s;               // p^-1 mod q_{l-1}
    u64 p_i[FHE_MAXP], p_i_s[FHE_MAXP];       // p mod q_i
    u64 qinv[FHE_MAXP], qinv_s[FHE_MAXP];     // q_{l-1}^-1 mod q_i
};

// Relinearisation and the modulus switch that follows it, as one ModDown
// (level l -> l-1; m = l-1 the dropped prime).  The special limbs t_k =
// [acc_k p^-1 (P/p_k)^-1]_{p_k} and w = [x_m p^-1]_{q_m} of the relinearised
// x (computed from y = acc_m + P add_m without forming x) give every kept
// limb's combined correction sum_k t_k h[k][i] + w h[K][i] in the
// coefficient domain; out_i = (acc_i P^-1 + add_i - NTT(correction)_i) q_m^-1.
struct RelinMSParams {
    int l, K;
    u64 h[FHE_MAXK + 1][FHE_MAXP];          // h[k][i] = p p_k^-1 mod q_i, h[K][i] = p mod q_i
    u64 pinv[FHE_MAXP], pinv_s[FHE_MAXP];    // P^-1 mod q_i
    u64 qminv[FHE_MAXP], qminv_s[FHE_MAXP];  // q_m^-1 mod q_i
    u64 pkinv[FHE_MAXK];                     // p_k^-1 mod q_m
    u64 Pm, Pm_s;                            // P mod q_m
};

// k modulus switches l -> l-k at once (2 <= k <= FHE_MAXK).  With D_t the
// product of the t last primes q_{l-1} .. q_{l-t} (D_0 = 1), the switches'
// values w_j = [x^(j)_{l-1-j} p^-1] follow from X'_j = INTT(x_{l-1-j}) p^-1
// D_j^-1 by w_j = X'_j - sum_{t<j} w_t F[j][t] (mod q_{l-1-j}), and
// out_i = (x_i - NTT(sum_t w_t G[t][i])_i) D_k^-1: the residues of k single
// switches.
struct MultiSwitchParams {
    int l, k;
    u64 G[FHE_MAXK][FHE_MAXP];           // p D_t mod q_i
    u64 Dinv[FHE_MAXP], Dinv_s[FHE_MAXP];  // D_k^-1 mod q_i
    u64 F[FHE_MAXK][FHE_MAXK];           // D_t D_j^-1 mod q_{l-1-j}
};

// ---------------------------------------------------------------------------
// device memory pool
// ---------------------------------------------------------------------------

struct Pool {
    fhe_allocator alloc;  // alloc.alloc == NULL -> cudaMallocAsync
    cudaStream_t stream = 0;
    std::unordered_map<size_t, std::vector<void *>> free_lists;
    std::unordered_map<void *, size_t> live;  // every block ever obtained -> size
    std::unordered_map<void *, bool> raw;     // blocks from cudaMalloc (misses during a capture)
    size_t reserved = 0, in_use = 0, budget = 0;  // budget 0 = unlimited
    size_t peak = 0;                              // largest in_use since the last reset
    long long fail_after = -1;                    // fault injection: fail the n-th new block
    // While a graph is captured, freed blocks go to this capture-private free
    // list (reused within the capture, in stream order) instead of the pool's;
    // the plan keeps them afterwards because every replay reuses them.
    std::unordered_map<size_t, std::vector<void *>> *cap_free = nullptr;
    bool in_capture = false;                      // misses use cudaMalloc (never the caller's allocator)
    fhe_ctx *owner = nullptr;                     // the context (to drop its cached batch graphs)
    void *get(size_t bytes, int *err);
    void put(void *p);
    void trim();
    void release_all();
};

void trim_other_pools(Pool *self);

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------

struct BatchPlan;

// F_{p^d} slots of one digit count (extract.cu)
struct ExtTables {
    int d = 0, Me = 0, stride = 0;                // slot degree, subring size, N / Me
    std::vector<std::vector<u64>> factors, idem;  // f_s and CRT idempotents, lowest degree first
    std::vector<std::vector<int64_t>> L;          // [k * d + t]: plaintext, slot s = lambda_{k,s}^(p^t)
    std::vector<int64_t> galois;                  // p^t mod 2N, t = 1 .. d-1
};

struct fhe_ctx {
    // parameters
    int logN = 0, N = 0, L = 0, K = 0, np = 0;
    u64 p = 0;
    std::vector<u64> q;   // L + K primes
    std::vector<ModQ> mq;
    std::vector<u64> psi;

    // device tables
    ModQ *d_mq = nullptr;          // [np]
    ulonglong2 *d_fwd = nullptr;   // [np][N]: (psi^brv(k), Shoup)
    ulonglong2 *d_inv = nullptr;   // [np][N]: (psi^-brv(k), Shoup)
    ulonglong2 *d_ninv = nullptr;  // [np]:    (N^-1, Shoup)

    // per-level constants (index = level l, 1..L), host and device copies
    std::vector<ModUpParams> modup;
    std::vector<ModDownParams> moddown;
    std::vector<ModSwitchParams> modswitch;
    std::vector<RelinMSParams> rms;
    RelinMSParams *d_rms = nullptr;
    std::vector<ulonglong2> rms_yscale;  // per level: N^-1 (p P)^-1 mod q_{l-1}
    bool separate_ms = false;            // products: relinearise, then switch (two ModDowns)
    std::vector<MultiSwitchParams> mss;  // [l * (FHE_MAXK + 1) + k]
    MultiSwitchParams *d_mss = nullptr;
    std::vector<ulonglong2> mss_scale;   // [(l * (FHE_MAXK + 1) + k) * FHE_MAXK + j]: N^-1 p^-1 D_j^-1
    ModUpParams *d_modup = nullptr;
    ModDownParams *d_moddown = nullptr;
    ModSwitchParams *d_modswitch = nullptr;
    std::unordered_map<int64_t, int *> d_perm;  // NTT-domain automorphism maps
    // constants folded into the final N^-1 scaling of inverse NTTs (value, Shoup)
    std::vector<std::vector<ulonglong2>> ks_xscale;  // [level][i]: N^-1 (Q_j/q_i)^-1 mod q_i, i in digit j
    std::vector<ulonglong2> ks_pscale;               // [k]: N^-1 p^-1 (P/p_k)^-1 mod p_k
    std::vector<ulonglong2> ms_lastscale;            // [level]: N^-1 p^-1 mod q_{level-1}
    // device copies: ks_xscale as [level][FHE_MAXP]; ms4scale [level][FHE_MAXK + 1]
    // = (ks_pscale[0..K-1], rms_yscale[level]); ks_pscale [K]; ms_lastscale
    // [level]; mss_scale in its host layout
    ulonglong2 *d_ks_xscale = nullptr, *d_ms4scale = nullptr, *d_ks_pscale = nullptr;
    ulonglong2 *d_ms_lastscale = nullptr, *d_mss_scale = nullptr;

    // plaintext side
    int ns = 0, M = 0;             // slots and subring size
    bool slots_linear = true;
    u64 zeta = 0, gamma = 0;       // primitive 2M-th root / sqrt(-2) mod p
    std::vector<int> slot_exp;     // slot s <-> zeta^slot_exp[s] (linear case)
    std::vector<int> lt;           // LT polynomial coefficients c_0..c_{p-1}
    std::vector<int> ltbv;         // bivariate LT coefficients c[a p + b] (built on first use)
    std::map<int, std::shared_ptr<ExtTables>> ext;  // F_{p^d} slot tables by d (built on first use)

    int sms = 0;                // SMs of the device (persistent NTT grids)
    int ntt_variant = 0;        // NTT grid policy chosen by the autotuner
    float ntt_ms[4] = {0, 0, 0, 0};  // timings of each variant (forward + inverse, per batch; 0 = n/a)

    cudaStream_t stream = 0;
    int device = -1;  // the device current when the context was created
    Pool pool;
    std::string err;
    std::mutex mu;

    // per-kernel-class CUDA-event timing (off unless requested)
    bool prof_on = false;
    int prof_cls = 0;
    std::vector<cudaEvent_t> prof_events;      // recycled
    std::vector<int> prof_rec_cls;             // class of each recorded launch
    std::vector<double> prof_rec_bytes;        // algorithmic bytes of each launch
    std::vector<double> prof_rec_bfly;         // NTT butterflies of each launch
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_rec;

    bool tracing = false;
    std::vector<int32_t> trace_op, trace_level;

    // Parallel branches while a plan is captured: independent parts of a
    // circuit (the digits of a comparison) are issued on their own streams,
    // forked from and joined back into the capture stream, so the graph runs
    // them concurrently.  Each branch has its own capture-private free list.
    bool capturing = false;
    bool multistream = false;  // the same scheduling without capture (batch execution)
    int wave_split = 2;        // a circuit's product wave runs as this many merged operations (streams)
    std::vector<cudaStream_t> branch_streams;
    std::vector<cudaEvent_t> branch_events;  // reused by every capture

    // captured batches: a batch whose group shapes were seen before is
    // captured once and replayed (least recently used first out)
    std::vector<BatchPlan *> bplans;
    std::map<std::vector<u64>, int> bseen;
    int bplan_cap = 4;
    u64 bplan_clock = 0;
    BatchPlan *bplan_active = nullptr;  // the graph being replayed (kept when memory runs out)
    long long launches = 0;       // kernels launched since creation
};

struct fhe_batch;
int batch_job_done(fhe_batch *B, int job);  // 1 once job `job` of the batch has its results

struct fhe_sk {
    fhe_ctx *ctx;
    std::vector<int64_t> s;       // host copy (ternary)
    u64 *d_s = nullptr;           // [L+K][N] NTT domain
};

struct fhe_pk {
    fhe_ctx *ctx;
    u64 *d = nullptr;             // [2][L][N] NTT domain
};

struct KeySwitchKey {
    int64_t galois = 0;           // 0 = relinearisation key
    u64 *d = nullptr;             // [dnum][2][L+K][N] NTT domain
};

struct fhe_evk {
    fhe_ctx *ctx;
    std::vector<KeySwitchKey> keys;  // keys[0] = relinearisation
    const KeySwitchKey *find(int64_t g) const;
};

// A captured batch (see batch.cu): the graph of one context's circuit for a
// recurring set of job groups, with its own operand and result buffers.
struct BatchPlan {
    std::vector<u64> sig;                               // the group shapes it serves
    std::vector<std::vector<fhe_ct *>> X, Y, O0, O1;    // [group][digit]
    std::unordered_map<size_t, std::vector<void *>> held;  // temporaries reused on every replay
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int nodes = 0;
    u64 last = 0;
    // a fused-ring plan (several contexts of one plaintext prime in one
    // graph): its member contexts and the temporaries it holds in each pool
    std::vector<fhe_ctx *> members;
    std::map<fhe_ctx *, std::unordered_map<size_t, std::vector<void *>>> mheld;
};
void batch_plans_release(fhe_ctx *c, const BatchPlan *keep = nullptr);
void batch_family_release(fhe_ctx *c);  // fused-ring graphs holding memory of c (context destruction)

struct fhe_plan {
    fhe_ctx *ctx;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    fhe_ct *out[2] = {nullptr, nullptr};  // LT, EQ (either may be NULL)
    std::unordered_map<size_t, std::vector<void *>> held;  // temporaries the graph reuses on every replay
    int nodes = 0;
};

struct fhe_ct {
    fhe_ctx *ctx;
    int count = 0, npoly = 0, level = 0;
    u64 *d = nullptr;             // [count][npoly][level][N] NTT domain
    size_t bytes = 0;
    // set only while a plan is captured: the event after the kernel that
    // produced this ciphertext, and the stream it was issued on
    cudaEvent_t ready = nullptr;
    cudaStream_t on = nullptr;
};

// kernel classes for fhe_ctx_profile_read (index = FHE_K_* in fhe.h)
void prof_begin(fhe_ctx *c, int cls, double bytes = 0, double bfly = 0);
void prof_end(fhe_ctx *c);

// ---------------------------------------------------------------------------
// internal helpers
// ---------------------------------------------------------------------------

int fhe_fail(fhe_ctx *ctx, int code, const std::string &msg);
int fhe_cuda_check(fhe_ctx *ctx, cudaError_t e, const char *where);
fhe_ct *ct_new(fhe_ctx *ctx, int count, int npoly, int level, int *err);

// host precomputation (params.cu)
bool host_is_prime(u64 n);
int host_find_primes(u64 U, u64 lo, u64 hi, int count, u64 *out);
u64 host_powmod(u64 a, u64 e, u64 q);
u64 host_invmod(u64 a, u64 q);
u64 host_mulmod(u64 a, u64 b, u64 q);
int build_tables(fhe_ctx *ctx);
void lt_poly_coefficients(int p, std::vector<int> &out);
void lt_bivariate_coefficients(int p, std::vector<int> &out);

// NTT engine (ntt.cu).  A multi-segment launch takes one argument record per
// segment (up to FHE_SEGS per kernel launch; more are split over launches);
// segments may belong to different contexts on one device (the launch runs
// on the first segment's context's stream) and differ in level and size.
#define FHE_SEGS 24
struct NttMapArgs {  // transform through a limb map; scale: device (N^-1 c_l, Shoup) per entry, or null
    fhe_ctx *c;
    const u64 *in;
    u64 *out;
    LimbMap m;
    const ulonglong2 *scale;
    int njobs;
};
struct NttYArgs : NttMapArgs {  // scaled inverse whose last entry loads y = acc + P add
    const u64 *abase;
    long long a_outer, a_poly;
    int amask, level;
};
struct NttModUpArgs {
    fhe_ctx *c;
    const u64 *d2c;
    u64 *ext;
    int level, count;
};
struct NttDownArgs {  // ModDown (src = special limbs) or relinearise + switch (src = t_k and w)
    fhe_ctx *c;
    const u64 *src, *acc, *abase;
    long long a_outer, a_poly;
    int amask;
    u64 *out;
    int level, count;
};
struct NttSwitchArgs {  // k = 1: src = the switched limb's w; k > 1: the k values w_t
    fhe_ctx *c;
    const u64 *src, *in;
    u64 *out;
    int level, k, npoly, count;
};
void launch_ntt_map_many(const std::vector<NttMapArgs> &a, bool fwd, int cls);
void launch_ntt_inv_scaled_y_many(const std::vector<NttYArgs> &a);
void launch_ntt_modup_many(const std::vector<NttModUpArgs> &a);
void launch_ntt_moddown_many(const std::vector<NttDownArgs> &a);
void launch_ntt_relin_ms_many(const std::vector<NttDownArgs> &a);
void launch_ntt_modswitch_many(const std::vector<NttSwitchArgs> &a);
void launch_ntt_multiswitch_many(const std::vector<NttSwitchArgs> &a);

// Streaming kernels over several batches per launch (many.cu).
enum { FHE_EW_ADD = 0, FHE_EW_SUB = 1, FHE_EW_NEG = 2, FHE_EW_LINCOMB = 3, FHE_EW_CMUL = 4, FHE_EW_CADD = 5 };
struct EwArgs {  // out = op(x[0..n)) over outer polys of `level` limbs; k: centred scalars
    fhe_ctx *c;
    int op, n;
    const u64 *x[8];
    int64_t k[8];
    u64 *out;
    int outer, level;
};
struct TensorArgs {
    fhe_ctx *c;
    const u64 *a, *b;
    u64 *out;
    int count, level;
};
struct KsInnerArgs {
    fhe_ctx *c;
    const u64 *ext, *xbase;
    long long x_outer;
    const u64 *ksk;
    u64 *acc;
    int count, level;
};
struct FoldArgs {  // rms: outer = ciphertexts; multi-switch: outer = polys, k switches
    fhe_ctx *c;
    u64 *src;
    int outer, level, k;
};
void launch_ew_many(const std::vector<EwArgs> &items);
void launch_tensor_many(const std::vector<TensorArgs> &items);
void launch_ks_inner_many(const std::vector<KsInnerArgs> &items);
void launch_rms_fold_many(const std::vector<FoldArgs> &items);
void launch_ms_fold_many(const std::vector<FoldArgs> &items);

// kernel launchers (ntt.cu, kernels.cu); scale arrays are device pointers
void launch_ntt_fwd_plain(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, int njobs);
void launch_add_plain(fhe_ctx *c, const u64 *a, const u64 *m, u64 *out, int count, int npoly, int level, int sub);
void encode_slot_vector(const fhe_ctx *c, const uint64_t *v, int64_t *m);  // n_s slots -> N coefficients in [0, p)
int op_plain(fhe_ctx *c, const fhe_ct *a, const uint64_t *slots, int kind, fhe_ct **out);
int circuit_sort(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, int d, fhe_ct **out);
int circuit_sort_joint(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, int K, int d, fhe_ct **out);
int circuit_sort_ranks(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, int K, int d, fhe_ct **rank,
                       fhe_ct **matrix);
#define FHE_SORT_MERGE 4  // comparisons of a sort's rank step merged into one circuit
std::vector<int64_t> sort_galois(const fhe_ctx *c);
struct SlotPiece {
    int j, o, s, b;        // input, output, column shift right, row swap
    std::vector<int> src;  // input slots the piece moves
};
int slot_plan(int ns, int n, const uint8_t *useful, std::vector<SlotPiece> &pieces, std::vector<int32_t> *dest);
std::vector<int64_t> slot_galois(int ns, int64_t N, const std::vector<SlotPiece> &pieces);
const ExtTables *ext_tables(fhe_ctx *c, int d, int *err);
void ext_encode(const fhe_ctx *c, const ExtTables *T, const uint64_t *digits, int64_t *m);
bool ext_decode(const fhe_ctx *c, const ExtTables *T, const int64_t *m, uint64_t *digits);
int op_plain_coeffs(fhe_ctx *c, const fhe_ct *a, const int64_t *m, int kind, fhe_ct **out);
int circuit_private_query(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *q, const fhe_ct *data, const fhe_ct *op1,
                          int op2, const int64_t *codes, bool overlap, fhe_ct **out);
int circuit_extract(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *a, const ExtTables *T, fhe_ct **out);
int circuit_slot_pack(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *in, int n, const uint8_t *useful,
                      fhe_ct **out, int n_out);
void launch_ntt_inv_plain(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, int njobs);
// inverse NTT whose output limb l (of the map) is also multiplied by scale[l]/N^-1:
// scale[l] = (N^-1 c_l mod q, Shoup word)
void launch_ntt_inv_scaled(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, const ulonglong2 *scale,
                           int njobs);
void launch_ntt_modup(fhe_ctx *c, const u64 *d2c, u64 *ext, int level, int count);
// addend for ModDown output poly pi of ct c: abase + c*a_outer + pi*a_poly when (amask>>pi)&1
void launch_ntt_moddown(fhe_ctx *c, const u64 *accP, const u64 *acc, const u64 *abase, long long a_outer,
                        long long a_poly, int amask, u64 *out, int level, int count);
void launch_ntt_relin_ms(fhe_ctx *c, const u64 *src, const u64 *acc, const u64 *abase, long long a_outer,
                         long long a_poly, int amask, u64 *out, int level, int count);
void launch_ntt_inv_scaled_y(fhe_ctx *c, const u64 *in, u64 *out, const LimbMap &m, const ulonglong2 *scale,
                             int njobs, const u64 *abase, long long a_outer, long long a_poly, int amask, int level);
void launch_rms_fold(fhe_ctx *c, u64 *src, int count, int level);
void launch_ntt_multiswitch(fhe_ctx *c, const u64 *src, const u64 *in, u64 *out, int level, int k, int npoly,
                            int count);
void launch_ms_fold(fhe_ctx *c, u64 *src, int outer, int level, int k);
int op_modswitch_k(fhe_ctx *c, const fhe_ct *a, int k, fhe_ct **out);
void launch_ntt_modswitch(fhe_ctx *c, const u64 *last, const u64 *in, u64 *out, int level, int npoly, int count);

void launch_add(fhe_ctx *c, const u64 *a, const u64 *b, u64 *out, int outer, int level, int sub);
void launch_neg(fhe_ctx *c, const u64 *a, u64 *out, int outer, int level);
void launch_mul_const(fhe_ctx *c, const u64 *a, u64 *out, int outer, int level, const u64 *w, const u64 *ws);
void launch_add_const(fhe_ctx *c, const u64 *a, u64 *out, int count, int level, const u64 *k);
void launch_tensor(fhe_ctx *c, const u64 *a, const u64 *b, u64 *out, int count, int level);
// acc[c][pi][r] = sum_j y_j[r] ksk_j[pi][prime(r)], y_j[r] = x_c[r] for r in digit j, else ext
void launch_ks_inner(fhe_ctx *c, const u64 *ext, const u64 *xbase, long long x_outer, const u64 *ksk, u64 *acc,
                     int count, int level);
void launch_automorphism(fhe_ctx *c, const u64 *in, u64 *out, int outer, int level, const int *perm);
void launch_mul_poly(fhe_ctx *c, const u64 *a, const u64 *b, u64 *out, int outer, int level, long long b_outer);
void launch_rns_from_i64(fhe_ctx *c, const int64_t *x, const int64_t *y, int64_t scale, u64 *out, int outer, int nl,
                         const int *primes);
void launch_muladd(fhe_ctx *c, const u64 *a, const u64 *b, const u64 *cc, u64 *out, int outer, int level,
                   long long b_outer, int neg);
void launch_ksk_digit(fhe_ctx *c, const u64 *a, const u64 *e, const u64 *s, const u64 *sp, u64 *k0, u64 *k1, int dlo,
                      int dhi, const u64 *Pw, const u64 *Pws);
bool ntt_supported_logn(int logN);
#define FHE_NTT_VARIANTS 4
bool ntt_variant_ok(int logN, int v);
int ntt_autotune(fhe_ctx *c, int njobs, float *ms_out);
// out = sum_{t<n} w[t] x[t], n <= 8, every x[t] an [outer][level][N] batch
void launch_lincomb(fhe_ctx *c, const u64 *const *x, const u64 (*w)[FHE_MAXP], int n, u64 *out, int outer,
                    int level);
int op_lincomb(fhe_ctx *c, const fhe_ct *const *x, const int64_t *k, int n, fhe_ct **out);

// seeded samplers (sample.cu)
void sample_ternary(fhe_ctx *c, int64_t *out, long long n, uint64_t seed, uint32_t tag);
void sample_gaussian(fhe_ctx *c, int64_t *out, long long n, uint64_t seed, uint32_t tag);
void sample_uniform(fhe_ctx *c, u64 *out, int outer, int nl, uint64_t seed, uint32_t tag);
// out[i] = centred(x[i] mod q0) mod p, as int64 in [0, p)
void launch_centre_mod_p(fhe_ctx *c, const u64 *x, int64_t *out, long long n);
int refresh_seeded(fhe_ctx *c, const fhe_sk *sk, const fhe_pk *pk, const fhe_ct *ct, uint64_t seed, fhe_ct **out);

// evaluation (eval.cu)
int op_lower(fhe_ctx *c, const fhe_ct *a, int level, fhe_ct **out);
int op_modswitch1(fhe_ctx *c, const fhe_ct *a, fhe_ct **out);
int op_addsub(fhe_ctx *c, const fhe_ct *a, const fhe_ct *b, int sub, fhe_ct **out);
int op_neg(fhe_ctx *c, const fhe_ct *a, fhe_ct **out);
int op_mul_const(fhe_ctx *c, const fhe_ct *a, int64_t k, fhe_ct **out);
int op_add_const(fhe_ctx *c, const fhe_ct *a, int64_t k, fhe_ct **out);
int op_tensor(fhe_ctx *c, const fhe_ct *a, const fhe_ct *b, fhe_ct **out);
int op_relin(fhe_ctx *c, const KeySwitchKey &k, const fhe_ct *d, fhe_ct **out);
int op_rotate(fhe_ctx *c, const KeySwitchKey &k, const fhe_ct *a, fhe_ct **out);
int op_mul_relin(fhe_ctx *c, const KeySwitchKey &rlk, const fhe_ct *a, const fhe_ct *b, fhe_ct **out);
int galois_perm(fhe_ctx *c, int64_t g, const int **perm);
// several batches at once (one launch per step for all; eval.cu)
struct MulItem {  // out = relinearised (and, above level 1, switched) a * b
    fhe_ctx *c;
    const KeySwitchKey *rlk;
    const fhe_ct *a, *b;
    fhe_ct *out;
};
struct SwitchItem {  // out = a with its k last primes dropped
    fhe_ctx *c;
    const fhe_ct *a;
    int k;
    fhe_ct *out;
};
struct EwItem {  // out = op(x[0..n)) with centred scalars k (FHE_EW_*)
    fhe_ctx *c;
    int op, n;
    const fhe_ct *x[8];
    int64_t k[8];
    fhe_ct *out;
};
int op_mul_relin_many(std::vector<MulItem> &items);
int op_modswitch_many(std::vector<SwitchItem> &items);
int op_ew_many(std::vector<EwItem> &items);
int circuit_compare_bv(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                       fhe_ct **lt, fhe_ct **eq);
int circuit_compare(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                    fhe_ct **lt, fhe_ct **eq);
int circuit_max_min(fhe_ctx *c, const fhe_evk *evk, const fhe_ct *const *x, const fhe_ct *const *y, int d,
                    fhe_ct **mx, fhe_ct **mn);
int64_t centred_const(const fhe_ctx *c, int64_t k);
// one comparison (LT -> out0, EQ -> out1; either NULL) or max/min (digits to
// out0 / out1) of an independent batch
struct MultiItem {
    const fhe_ct *const *x;
    const fhe_ct *const *y;
    int d;
    bool maxmin;
    fhe_ct **out0;
    fhe_ct **out1;
};
int circuit_multi(fhe_ctx *c, const fhe_evk *evk, const std::vector<MultiItem> &items);
int circuit_multi_ctx(const std::vector<const fhe_evk *> &evks, const std::vector<MultiItem> &items);
int op_slice(fhe_ctx *c, const fhe_ct *a, int start, int n, fhe_ct **out);
int op_concat(fhe_ctx *c, const fhe_ct *a, const fhe_ct *b, fhe_ct **out);
std::vector<int64_t> tournament_galois(const fhe_ctx *c);
int batch_check_job(const fhe_job &j);
int circuit_tournament(fhe_ctx *c, const fhe_evk *evk, const fhe_sk *sk, const fhe_pk *pk, const fhe_ct *const *x,
                       int d, bool want_max, bool want_min, uint64_t seed, fhe_ct **out_max, fhe_ct **out_min);

void launch_copy_limbs(fhe_ctx *c, const u64 *in, u64 *out, int outer, int nl, long long in_outer,
                       long long out_outer);
