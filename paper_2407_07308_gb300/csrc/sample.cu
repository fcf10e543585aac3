// sample.cu -- device-side randomness for seeded key generation, encryption
// and refresh: the Philox4x32-10 counter-based generator (J. Salmon,
// M. Moraes, R. Dror, D. Shaw, "Parallel random numbers: as easy as 1, 2,
// 3", SC'11) and the samplers the scheme draws from.
//
// Stream layout: sample n of stream `tag` under key `seed` is the Philox
// block of counter (n, n >> 32, tag, 0) and key (seed, seed >> 32).
//   ternary   : {-1, 0, 1} from floor(w0 * 3 / 2^32) - 1
//   gaussian  : Box-Muller on (w0, w1), sigma 3.2, rounded, cut at +-20
//   uniform q : ((w1 << 32) | w0) mod q
#include "fhe_internal.h"

namespace {

struct Philox {
    uint32_t v[4];
};

__host__ __device__ inline Philox philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; r++) {
        const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    Philox o;
    o.v[0] = c0;
    o.v[1] = c1;
    o.v[2] = c2;
    o.v[3] = c3;
    return o;
}

__device__ inline Philox draw(uint64_t seed, uint32_t tag, uint64_t n)
{
    return philox4x32_10((uint32_t)n, (uint32_t)(n >> 32), tag, 0, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// kind: 0 ternary, 1 gaussian  -> int64 out[n]
__global__ void k_sample_small(int64_t *__restrict__ out, long long n, uint64_t seed, uint32_t tag, int kind)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const Philox r = draw(seed, tag, (uint64_t)i);
        if (kind == 0) {
            out[i] = (int64_t)(((uint64_t)r.v[0] * 3u) >> 32) - 1;
        } else {
            const float u1 = ((float)r.v[0] + 1.0f) * 2.3283064e-10f;  // (0, 1]
            const float u2 = (float)r.v[1] * 2.3283064e-10f;           // [0, 1)
            const float g = 3.2f * sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
            long long v = llrintf(g);
            out[i] = v > 20 ? 20 : (v < -20 ? -20 : v);
        }
    }
}

// uniform residues: out[o][i][n] in [0, q_i), o < outer, i < nl (primes 0..nl-1)
__global__ void k_sample_uniform(u64 *__restrict__ out, long long total, int logN, int nl, uint64_t seed, uint32_t tag,
                                 const ModQ *__restrict__ mq)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)((idx >> logN) % nl);
        const Philox r = draw(seed, tag, (uint64_t)idx);
        const u64 x = ((u64)r.v[1] << 32) | r.v[0];
        out[idx] = x % mq[i].q;
    }
}

// raw Philox blocks (for known-answer and parity checks)
__global__ void k_philox_raw(uint32_t *__restrict__ out, int n, uint64_t seed, uint32_t tag)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Philox r = draw(seed, tag, (uint64_t)i);
        for (int k = 0; k < 4; k++) out[4 * (size_t)i + k] = r.v[k];
    }
}

int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 1 << 20); }

}  // namespace

void sample_ternary(fhe_ctx *c, int64_t *out, long long n, uint64_t seed, uint32_t tag)
{
    k_sample_small<<<blocks_for(n), 256, 0, c->stream>>>(out, n, seed, tag, 0);
    c->launches++;
}

void sample_gaussian(fhe_ctx *c, int64_t *out, long long n, uint64_t seed, uint32_t tag)
{
    k_sample_small<<<blocks_for(n), 256, 0, c->stream>>>(out, n, seed, tag, 1);
    c->launches++;
}

void sample_uniform(fhe_ctx *c, u64 *out, int outer, int nl, uint64_t seed, uint32_t tag)
{
    const long long total = (long long)outer * nl * c->N;
    k_sample_uniform<<<blocks_for(total), 256, 0, c->stream>>>(out, total, c->logN, nl, seed, tag, c->d_mq);
    c->launches++;
}

// Writes n Philox4x32-10 blocks (4 words each) of stream `tag` under `seed`,
// computed on the device, to the host array out[4n].  Synchronises.
extern "C" int fhe_philox_blocks(uint64_t seed, uint32_t tag, int n, uint32_t *out)
{
    if (n < 0 || !out) return FHE_EINVAL;
    uint32_t *d = nullptr;
    if (cudaMalloc(&d, sizeof(uint32_t) * 4 * (size_t)(n ? n : 1)) != cudaSuccess) return FHE_ENOMEM;
    k_philox_raw<<<blocks_for(n ? n : 1), 256>>>(d, n, seed, tag);
    cudaError_t e = cudaMemcpy(out, d, sizeof(uint32_t) * 4 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : FHE_ECUDA;
}
