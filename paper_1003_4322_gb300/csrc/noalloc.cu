// noalloc.cu -- ns_fft_c2r_noalloc: the FP32 inverse 3D transform for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// owned by a caching pool allocator (a raw cudaMalloc there can fail, or
// fragment memory the pool has already reserved), and real-time loops that
// forbid any allocation after start-up.  ns_fft_c2r needs a context, and the
// context allocates its tables and a one-field scratch buffer; this entry
// point needs neither.  Its scratch (one complex half-layout field) and its
// twiddle tables live in file-scope __device__ arrays of fixed size, which
// every GPU that loads libns holds until the process exits.
#include <math.h>

#include <mutex>
#include <vector>

#include "../../include/ns.h"
#include "ns_internal.h"

namespace {

// Largest supported grid: one FP32 complex half-layout field of 128^3
// (128 * 128 * 65 * 8 bytes = 8,519,680 bytes).
constexpr int kNoAllocMaxN = 128;
constexpr long kNoAllocScratch = (long)kNoAllocMaxN * kNoAllocMaxN * (kNoAllocMaxN / 2 + 1);
// The twiddle tables exp(-2 pi i t / n), t < n, of every supported n up to
// 128 (8, 12, 16, 18, 24, 32, 36, 48, 54, 64, 72, 96, 108, 128: 716
// entries), one after another in increasing n.
constexpr int kNoAllocTwiddles = 1024;

static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocScratch];
static __device__ __align__(256) float2 g_noalloc_twiddles[kNoAllocTwiddles];

constexpr int kMaxDevices = 64;

struct DeviceSlot {
    bool ready = false;
    float2 *scratch = nullptr;   // device address of g_noalloc_scratch
    float2 *twiddles = nullptr;  // device address of g_noalloc_twiddles
};

std::mutex g_mu;
DeviceSlot g_slots[kMaxDevices];

// Offset of the table of length n inside g_noalloc_twiddles (-1 if n is not
// a supported size up to the maximum).
int table_offset(int n) {
    int off = 0;
    for (int m = 8; m <= kNoAllocMaxN; m += 2) {
        if (!nsk::supported_n(m)) continue;
        if (m == n) return off;
        off += m;
    }
    return -1;
}

// Once per device, with that device current: look up the arrays' device
// addresses (in host code their names stand for host-side shadows, not device
// addresses) and fill every twiddle table, computed in FP64 on the host and
// rounded once to float.  The copy is ordered on the caller's stream and
// waited for, so that the tables are in place before any later call on any
// stream; later calls copy nothing.
ns_status setup_current_device(cudaStream_t s, DeviceSlot *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return NS_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_mu);
    DeviceSlot &slot = g_slots[dev];
    if (!slot.ready) {
        void *p = nullptr, *q = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return NS_ERR_CUDA;
        if (cudaGetSymbolAddress(&q, g_noalloc_twiddles) != cudaSuccess) return NS_ERR_CUDA;
        std::vector<float2> tw;
        tw.reserve(kNoAllocTwiddles);
        const double two_pi = 6.283185307179586476925286766559;
        for (int n = 8; n <= kNoAllocMaxN; n += 2) {
            if (!nsk::supported_n(n)) continue;
            for (int t = 0; t < n; t++) {
                const double a = two_pi * (double)t / (double)n;
                tw.push_back(make_float2((float)cos(a), (float)(-sin(a))));
            }
        }
        if (tw.size() > (size_t)kNoAllocTwiddles) return NS_ERR_UNSUPPORTED_N;
        if (cudaMemcpyAsync(q, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice,
                            s) != cudaSuccess)
            return NS_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return NS_ERR_CUDA;
        slot.scratch = (float2 *)p;
        slot.twiddles = (float2 *)q;
        slot.ready = true;
    }
    *out = slot;
    return NS_OK;
}

}  // namespace

extern "C" ns_status ns_fft_c2r_noalloc(int n, int ncomp, const void *in, void *out,
                                        void *cuda_stream) {
    using namespace nsk;
    if (!in || !out || ncomp < 1) return NS_ERR_ARG;
    if (!supported_n(n) || n > kNoAllocMaxN) return NS_ERR_UNSUPPORTED_N;
    const int off = table_offset(n);
    Plan plN, plH;
    if (off < 0 || !make_plan(n, &plN) || !make_plan(n / 2, &plH)) return NS_ERR_UNSUPPORTED_N;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    DeviceSlot dev;
    ns_status st = setup_current_device(s, &dev);
    if (st != NS_OK) return st;
    const float2 *tw = dev.twiddles + off;

    const long nh = n / 2 + 1, plane = (long)n * nh, M = (long)n * plane, V = (long)n * n * n;
    const int ct = default_ct(sizeof(float2), n);
    const float2 *src = (const float2 *)in;
    float *dst = (float *)out;
    for (int c = 0; c < ncomp; c++) {
        if (fft_strided<float>(src + c * M, dev.scratch, plane, plane, M, M, 1, +1, plN, tw, n,
                               ct, s) != cudaSuccess)
            return NS_ERR_CUDA;
        if (fft_strided<float>(dev.scratch, dev.scratch, nh, nh, plane, plane, n, +1, plN, tw, n,
                               ct, s) != cudaSuccess)
            return NS_ERR_CUDA;
        if (fft_z_c2r<float>(dev.scratch, dst + c * V, n, (long)n * n, plH, tw, s) != cudaSuccess)
            return NS_ERR_CUDA;
    }
    return NS_OK;
}
