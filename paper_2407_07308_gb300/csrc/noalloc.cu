// noalloc.cu -- modulus switching for callers that cannot allocate device
// memory.
//
// Some callers own every byte of device memory themselves: a host framework
// that reserves the GPU's memory up front and hands plugins only fixed
// buffers, or a latency-critical loop where a cudaMalloc (which can
// synchronise the device) is not acceptable.  They cannot use the pool-based
// entry points, which obtain their temporaries on demand.  This file gives
// them one entry point, fhe_mod_switch_noalloc, whose only temporary -- the
// coefficient-domain copy of the dropped limb -- lives in a fixed device array
// compiled into the library.  The caller passes the input and output buffers.
#include <string.h>

#include <mutex>

#include "fhe_internal.h"

// 2^20 words (8 MiB): count * npoly * N must not exceed this, e.g. 32
// two-poly ciphertexts at N = 2^14.  Every device that loads the library
// holds this array until the process exits.
#define FHE_NOALLOC_SCRATCH_WORDS (1u << 20)

static __device__ __align__(256) uint64_t g_noalloc_scratch[FHE_NOALLOC_SCRATCH_WORDS];

// Device address of the scratch array, looked up once per device with that
// device current (the host-side symbol is only a stand-in for it).  The
// lookup may load the library's module on that device, which a stream under
// capture does not allow: a first call while `capturing` is refused.
static int scratch_address(int dev, bool capturing, u64 **out)
{
    static std::mutex mu;
    static u64 *addr[64] = {nullptr};
    if (dev < 0 || dev >= 64) return FHE_EINVAL;
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev]) {
        if (capturing) return FHE_EINVAL;
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FHE_ECUDA;
        addr[dev] = (u64 *)p;
    }
    *out = addr[dev];
    return 0;
}

extern "C" int fhe_mod_switch_noalloc(fhe_ctx *c, const uint64_t *in, uint64_t *out, int count, int npoly, int level)
{
    if (!c || !in || !out || count < 1 || npoly < 2 || npoly > 3) return FHE_EINVAL;
    if (level < 2 || level > c->L) return fhe_fail(c, FHE_ELEVEL, "mod_switch_noalloc: level must be in [2, L]");
    const unsigned long long words = (unsigned long long)count * npoly * c->N;
    if (words > FHE_NOALLOC_SCRATCH_WORDS)
        return fhe_fail(c, FHE_EINVAL,
                        "mod_switch_noalloc: count * npoly * N exceeds the fixed scratch of 2^20 words");
    std::lock_guard<std::mutex> lock(c->mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fhe_fail(c, FHE_ECUDA, "mod_switch_noalloc: no current device");
    // the kernels run on the context's stream, i.e. on the context's device:
    // the scratch address must be that device's
    if (dev != c->device)
        return fhe_fail(c, FHE_EINVAL, "mod_switch_noalloc: the current device is not the context's device");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cap) != cudaSuccess)
        return fhe_fail(c, FHE_ECUDA, "mod_switch_noalloc: stream query failed");
    u64 *scratch = nullptr;
    int e = scratch_address(dev, cap != cudaStreamCaptureStatusNone, &scratch);
    if (e == FHE_EINVAL)
        return fhe_fail(c, e, "mod_switch_noalloc: the first call on a device must not be made during stream capture");
    if (e) return fhe_fail(c, e, "mod_switch_noalloc: cudaGetSymbolAddress failed");
    // per-launch event timing would create events; this path creates nothing
    const bool prof = c->prof_on;
    c->prof_on = false;
    const int N = c->N;
    LimbMap m;
    memset(&m, 0, sizeof(m));
    m.nl = 1;
    m.in_outer = (long long)level * N;
    m.out_outer = N;
    m.in_limb[0] = level - 1;
    m.out_limb[0] = 0;
    m.prime[0] = level - 1;
    // every scratch word read below is written by this inverse NTT first,
    // so nothing needs clearing between calls
    launch_ntt_inv_scaled(c, in, scratch, m, c->d_ms_lastscale + level, count * npoly);
    launch_ntt_modswitch(c, scratch, in, out, level, npoly, count);
    c->prof_on = prof;
    return fhe_cuda_check(c, cudaGetLastError(), "mod_switch_noalloc");
}
