// noalloc.cu -- ns_fft_c2r_noalloc: the FP32 inverse 3D transform for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// owned by a caching pool allocator (a raw cudaMalloc there can fail, or
// fragment memory the pool has already reserved), and real-time loops that
// forbid any allocation after start-up.  ns_fft_c2r needs a context, and the
// context allocates its tables and a one-field scratch buffer; this entry
// point needs neither.  Its scratch (one complex half-layout field) and its
// twiddle table live in file-scope __device__ arrays of fixed size, which
// every GPU that loads libns holds until the process exits.
#include <math.h>

#include <mutex>

#include "../../include/ns.h"
#include "ns_internal.h"

namespace {

// Largest supported grid: one FP32 complex half-layout field of 128^3
// (128 * 128 * 65 * 8 bytes = 8,519,680 bytes) plus a 128-entry table.
constexpr int kNoAllocMaxN = 128;
constexpr long kNoAllocScratch = (long)kNoAllocMaxN * kNoAllocMaxN * (kNoAllocMaxN / 2 + 1);

static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocScratch];
static __device__ __align__(256) float2 g_noalloc_twiddles[kNoAllocMaxN];

constexpr int kMaxDevices = 64;

struct DeviceSlot {
    bool ready = false;
    float2 *scratch = nullptr;   // device address of g_noalloc_scratch
    float2 *twiddles = nullptr;  // device address of g_noalloc_twiddles
};

std::mutex g_mu;
DeviceSlot g_slots[kMaxDevices];

// In host code the arrays' names stand for host-side shadows, not device
// addresses; the addresses come from cudaGetSymbolAddress, taken once per
// device with that device current.
ns_status setup_current_device(DeviceSlot *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return NS_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_mu);
    DeviceSlot &s = g_slots[dev];
    if (!s.ready) {
        void *p = nullptr, *q = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return NS_ERR_CUDA;
        if (cudaGetSymbolAddress(&q, g_noalloc_twiddles) != cudaSuccess) return NS_ERR_CUDA;
        s.scratch = (float2 *)p;
        s.twiddles = (float2 *)q;
        s.ready = true;
    }
    *out = s;
    return NS_OK;
}

}  // namespace

extern "C" ns_status ns_fft_c2r_noalloc(int n, int ncomp, const void *in, void *out,
                                        void *cuda_stream) {
    using namespace nsk;
    if (!in || !out || ncomp < 1) return NS_ERR_ARG;
    if (!supported_n(n) || n > kNoAllocMaxN) return NS_ERR_UNSUPPORTED_N;
    Plan plN, plH;
    if (!make_plan(n, &plN) || !make_plan(n / 2, &plH)) return NS_ERR_UNSUPPORTED_N;
    DeviceSlot dev;
    ns_status st = setup_current_device(&dev);
    if (st != NS_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    (void)cudaGetLastError();

    // exp(-2 pi i t / n) in FP64 on the host, rounded once to float; the copy
    // is staged out of this stack buffer before cudaMemcpyToSymbolAsync returns.
    float2 tw[kNoAllocMaxN];
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < n; t++) {
        const double a = two_pi * (double)t / (double)n;
        tw[t] = make_float2((float)cos(a), (float)(-sin(a)));
    }
    if (cudaMemcpyToSymbolAsync(g_noalloc_twiddles, tw, sizeof(float2) * n, 0,
                                cudaMemcpyHostToDevice, s) != cudaSuccess)
        return NS_ERR_CUDA;

    const long nh = n / 2 + 1, plane = (long)n * nh, M = (long)n * plane, V = (long)n * n * n;
    const int ct = default_ct(sizeof(float2), n);
    const float2 *src = (const float2 *)in;
    float *dst = (float *)out;
    for (int c = 0; c < ncomp; c++) {
        if (fft_strided<float>(src + c * M, dev.scratch, plane, plane, M, M, 1, +1, plN,
                               dev.twiddles, n, ct, s) != cudaSuccess)
            return NS_ERR_CUDA;
        if (fft_strided<float>(dev.scratch, dev.scratch, nh, nh, plane, plane, n, +1, plN,
                               dev.twiddles, n, ct, s) != cudaSuccess)
            return NS_ERR_CUDA;
        if (fft_z_c2r<float>(dev.scratch, dst + c * V, n, (long)n * n, plH, dev.twiddles, s) !=
            cudaSuccess)
            return NS_ERR_CUDA;
    }
    return NS_OK;
}
