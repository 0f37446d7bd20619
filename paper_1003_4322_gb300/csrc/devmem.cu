// devmem.cu -- the library's device allocations, with optional guard bands.
//
// With NS_GUARD=1 in the environment (read at the first allocation), every
// buffer the library allocates gets kGuard bytes of a fixed pattern on each
// side; ns_guard_check scans every live guard band on the GPU and reports how
// many bytes no longer hold the pattern, so that a kernel writing outside its
// buffers shows up as a nonzero count in the tests (a debug stand-in for a
// device memory-error detector).  Without NS_GUARD the allocator is plain
// cudaMalloc.
#include <stdlib.h>

#include <map>
#include <mutex>

#include "../../include/ns.h"
#include "ns_internal.h"

namespace nsk {

namespace {
const size_t kGuard = 4096;
const unsigned char kPattern = 0xA5;
struct Alloc {
    unsigned char *base;
    size_t bytes;
};
std::mutex mu;
std::map<void *, Alloc> live;
int mode = -1;

bool guards() {
    std::lock_guard<std::mutex> g(mu);
    if (mode < 0) {
        const char *v = getenv("NS_GUARD");
        mode = (v && atoi(v) > 0) ? 1 : 0;
    }
    return mode == 1;
}

__global__ void k_guard_scan(const unsigned char *__restrict__ g, size_t n, unsigned char pattern,
                             unsigned long long *bad) {
    unsigned long long cnt = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        cnt += g[i] != pattern;
    if (cnt) atomicAdd(bad, cnt);
}
}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    if (!guards()) return cudaMalloc(p, bytes);
    unsigned char *base = nullptr;
    cudaError_t e = cudaMalloc((void **)&base, bytes + 2 * kGuard);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemset(base, kPattern, kGuard)) != cudaSuccess ||
        (e = cudaMemset(base + kGuard + bytes, kPattern, kGuard)) != cudaSuccess) {
        cudaFree(base);
        return e;
    }
    *p = base + kGuard;
    std::lock_guard<std::mutex> g(mu);
    live[*p] = Alloc{base, bytes};
    return cudaSuccess;
}

void dev_free(void *p) {
    if (!p) return;
    if (!guards()) {
        cudaFree(p);
        return;
    }
    std::lock_guard<std::mutex> g(mu);
    auto it = live.find(p);
    if (it == live.end()) {
        cudaFree(p);
        return;
    }
    cudaFree(it->second.base);
    live.erase(it);
}

// Bytes of every live guard band that no longer hold the pattern.
static cudaError_t scan_all(long long *bad) {
    unsigned long long *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    if ((e = cudaMemset(d, 0, sizeof(unsigned long long))) == cudaSuccess) {
        std::lock_guard<std::mutex> g(mu);
        for (const auto &kv : live) {
            const Alloc &a = kv.second;
            k_guard_scan<<<8, 256>>>(a.base, kGuard, kPattern, d);
            k_guard_scan<<<8, 256>>>(a.base + kGuard + a.bytes, kGuard, kPattern, d);
        }
        e = cudaGetLastError();
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    *bad = (long long)h;
    return e;
}

}  // namespace nsk

using namespace nsk;

extern "C" ns_status ns_guard_check(long long *bad_bytes) {
    if (!bad_bytes) return NS_ERR_ARG;
    if (!guards()) {
        *bad_bytes = -1;
        return NS_OK;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = scan_all(bad_bytes);
    return e == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}

extern "C" ns_status ns_guard_selftest(long long *detected) {
    if (!detected) return NS_ERR_ARG;
    *detected = -1;
    if (!guards()) return NS_OK;
    long long before = 0, after = 0;
    if (ns_guard_check(&before) != NS_OK) return NS_ERR_CUDA;
    void *p = nullptr;
    cudaError_t e = dev_malloc(&p, 1024);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NS_ERR_OOM : NS_ERR_CUDA;
    // one byte just past the buffer: inside the allocation, in its back guard
    e = cudaMemset((unsigned char *)p + 1024, 0, 1);
    if (e == cudaSuccess && ns_guard_check(&after) == NS_OK) *detected = after - before;
    dev_free(p);
    return e == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}
