// probe.cu -- measured integer-pipe peaks of this GPU, the denominators of
// the integer roofline the NTT kernels are reported against: 32-bit
// multiply-adds and 64-bit high products (the Shoup butterfly's one
// __umul64hi) per second over all SMs.  Fixed trip counts; each thread
// carries 8 independent chains so that latency is hidden; the results are
// stored so that nothing is optimised away.
#include "fhe_internal.h"

namespace {

constexpr int PROBE_ITERS = 4096;

__global__ void k_probe_imad32(uint32_t *out, uint32_t seed)
{
    uint32_t a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = seed + threadIdx.x * 8 + k;
    for (int i = 0; i < PROBE_ITERS; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = a[k] * a[k] + (uint32_t)k;  // one multiply-add each (no closed form)
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) r ^= a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void k_probe_mulhi64(u64 *out, u64 seed)
{
    u64 a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = seed + threadIdx.x * 8 + k;
    const u64 m = 0x9E3779B97F4A7C15ull;
    for (int i = 0; i < PROBE_ITERS; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = __umul64hi(a[k], m) ^ (u64)k;  // one 64-bit high product each
    }
    u64 r = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) r ^= a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// The NTT's butterfly (Harvey's lazy forward butterfly with a Shoup twiddle
// whose quotient is estimated from three 32-bit partial products, in the
// multiply-add chain the NTT kernels use: t = Y w - qhat q in [0, 4q),
// X <- X + t, Y <- X - t + 4q) on 8
// register-resident values per thread, three butterfly layers per iteration
// (strides 4, 2, 1) so that every value depends on every other: the roof of
// the NTT's arithmetic with no memory traffic at all.
constexpr int BFLY_ITERS = 512;

__global__ void k_probe_bfly(u64 *out, u64 seed, u64 q, u64 w, u64 ws)
{
    u64 x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = seed + threadIdx.x * 8 + k;
    const u64 q4 = 4 * q, nq = 0 - q;
    for (int i = 0; i < BFLY_ITERS; i++) {
#pragma unroll
        for (int h = 4; h >= 1; h >>= 1) {
#pragma unroll
            for (int k = 0; k < 8; k++) {
                if (k & h) continue;
                const u64 t = shoup_lazy4_chain(x[k + h], w, ws, nq);
                const u64 a = x[k];
                x[k] = a + t;
                x[k + h] = a - t + q4;
            }
        }
    }
    u64 r = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) r ^= x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace

// Butterflies per second over all SMs (k_probe_bfly with a 50-bit prime and
// twiddle).  Synchronises; allocates a small buffer.
extern "C" int fhe_probe_bfly_peak(double *bfly)
{
    if (!bfly) return FHE_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FHE_ECUDA;
    const int threads = 256, blocks = sms * 8;
    void *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(u64) * threads * blocks) != cudaSuccess) return FHE_ENOMEM;
    const u64 q = 564395044569089ull, w = 123456789012345ull % q;
    const u64 ws = (u64)(((unsigned __int128)w << 64) / q);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int r = 0; r < 2; r++) k_probe_bfly<<<blocks, threads>>>((u64 *)buf, 1ull, q, w, ws);
    cudaEventRecord(e0);
    for (int r = 0; r < 10; r++) k_probe_bfly<<<blocks, threads>>>((u64 *)buf, (u64)r, q, w, ws);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    *bfly = 10.0 * threads * blocks * BFLY_ITERS * 12 / (ms / 1e3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t e = cudaGetLastError();
    cudaFree(buf);
    return e == cudaSuccess ? 0 : FHE_ECUDA;
}

// Writes the measured rates (operations per second, all SMs) to
// imad32[0] and mulhi64[0].  Synchronises; allocates a small buffer.
extern "C" int fhe_probe_int_peak(double *imad32, double *mulhi64)
{
    if (!imad32 || !mulhi64) return FHE_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FHE_ECUDA;
    const int threads = 256, blocks = sms * 8;
    void *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(u64) * threads * blocks) != cudaSuccess) return FHE_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const double ops = (double)threads * blocks * PROBE_ITERS * 8;
    float ms = 0;
    for (int w = 0; w < 2; w++) k_probe_imad32<<<blocks, threads>>>((uint32_t *)buf, 1u);
    cudaEventRecord(e0);
    for (int r = 0; r < 10; r++) k_probe_imad32<<<blocks, threads>>>((uint32_t *)buf, (uint32_t)r);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *imad32 = 10 * ops / (ms / 1e3);
    for (int w = 0; w < 2; w++) k_probe_mulhi64<<<blocks, threads>>>((u64 *)buf, 1ull);
    cudaEventRecord(e0);
    for (int r = 0; r < 10; r++) k_probe_mulhi64<<<blocks, threads>>>((u64 *)buf, (u64)r);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *mulhi64 = 10 * ops / (ms / 1e3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t e = cudaGetLastError();
    cudaFree(buf);
    return e == cudaSuccess ? 0 : FHE_ECUDA;
}
