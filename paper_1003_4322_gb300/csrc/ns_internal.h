// ns_internal.h -- host-side declarations shared by the translation units of
// libns (not part of the public ABI, which is include/ns.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fft_core.cuh"

namespace nsk {

// Optional per-launch timing: when a Tracer is active, every kernel launch of
// a step is bracketed by a pair of CUDA events on the launching stream.
struct Tracer {
    struct Rec {
        const char *name;
        cudaEvent_t a, b;
    };
    cudaStream_t s = nullptr;
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    cudaError_t err = cudaSuccess;
    cudaEvent_t take() {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) {
                err = r;
                return nullptr;
            }
            pool.push_back(e);
        }
        return pool[used++];
    }
    void begin(const char *name) {
        Rec r{name, take(), nullptr};
        if (r.a) cudaEventRecord(r.a, s);
        recs.push_back(r);
    }
    void end() {
        cudaEvent_t b = take();
        if (b) cudaEventRecord(b, s);
        recs.back().b = b;
    }
    ~Tracer() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

// Run one launch expression, timed when tr is non-null; yields its error.
#define NSK_TIMED(tr, name, expr)                         \
    ([&]() -> cudaError_t {                               \
        if (tr) (tr)->begin(name);                        \
        cudaError_t _te = (expr);                         \
        if (tr) (tr)->end();                              \
        return _te;                                       \
    }())

// Standalone FP32 transforms of an nx x ny x nz grid on the compile-time
// kernels (axis lengths 64 ... 1024 of the compiled set), with the twiddle
// table exp(-2 pi i t / n_i) of every axis: r2c of ncomp real fields into the
// half layout, c2r of one half field through tmp (one half field).  False
// when a length has no compiled kernel (nothing launched); else *err holds
// the launch status.
struct StdGrid {
    int nx, ny, nz;
    const float2 *twx, *twy, *twz;
};
bool std_r2c_fp32_grid(const float *in, float2 *out, const StdGrid &g, int ncomp, cudaStream_t s,
                       cudaError_t *err);
bool std_c2r_fp32_grid(const float2 *in, float2 *tmp, float *out, const StdGrid &g, cudaStream_t s,
                       cudaError_t *err);

// Radix plan for a line of length n = 2^a 3^b (false if n has another factor).
bool make_plan(int n, Plan *pl);

// Radix plan with E elements per thread (the first, largest radix is E and
// every radix divides E); false if E does not suit n.
bool make_plan_e(int n, int E, Plan *pl);

// Is N a supported grid size (2^a 3^b, even, >= 8)?
bool supported_n(int n);

// Twiddle table exp(-2 pi i t / n), t < n, computed on the host in FP64 and
// uploaded (rounded once to float for the FP32 path).
template <typename T> typename Cx<T>::type *make_twiddles(int n, cudaError_t *err);

// A subset of the columns and rows of a strided pass: the lines that the
// dealiasing rule leaves zero (inverse) or whose result it discards
// (forward).  A plane's ncols columns are nouter rows of `inner` columns
// (inner x nouter = ncols); the pass transforms the first `keep` columns of
// rows [0, o1) and [o2, nouter), and treats the elements e of the transform
// axis in [gap_lo, gap_hi) as zero on input (dir +1) or leaves them
// unwritten (dir -1).  The other columns are neither read nor written.
struct StridedSel {
    long inner = 0;
    int keep = 0, nouter = 1, o1 = 1, o2 = 1;
    int gap_lo = 0, gap_hi = 0;
};

// Batched FFT along a strided axis.  Element e (< pl.n) of column c (< ncols)
// of plane b (< planes) sits at base + b * plane_stride + e * es + c (in
// complex units); columns are contiguous.  dir = -1 forward, +1 inverse.
// in == out is allowed (in place).  ct = columns per CTA.  sel (optional):
// only the selected columns and rows.
template <typename T>
cudaError_t fft_strided(const typename Cx<T>::type *in, typename Cx<T>::type *out, long ncols,
                        long es, long ps_in, long ps_out, int planes, int dir, const Plan &pl,
                        const typename Cx<T>::type *tw, int ntab, int ct, cudaStream_t s,
                        const StridedSel *sel = nullptr);

// Real-to-complex transform along z (contiguous) of nlines lines of N reals
// into nlines lines of N/2+1 complex values; pl is the plan of length N/2 (one
// line per transform) or N (two), tw the table of length N.  kzk in
// [0, N/2+1]: only the entries kz < kzk are written (-1: all).
template <typename T>
cudaError_t fft_z_r2c(const T *in, typename Cx<T>::type *out, int N, long nlines, const Plan &pl,
                      const typename Cx<T>::type *tw, cudaStream_t s, int kzk = -1);

// Complex-to-real transform along z: nlines lines of N/2+1 complex values into
// nlines lines of N reals (real parts of the kz = 0 and N/2 entries only).
// kzk: the entries kz >= kzk are taken as zero and not read (-1: all read).
template <typename T>
cudaError_t fft_z_c2r(const typename Cx<T>::type *in, T *out, int N, long nlines,
                      const Plan &pl, const typename Cx<T>::type *tw, cudaStream_t s, int kzk = -1);

// Columns per CTA of the strided pass for a given precision and length.
int default_ct(int elem_bytes, int n);

// Opt a kernel into more than 48 KB of dynamic shared memory (once per
// device); fails if bytes exceeds the device's opt-in maximum.
cudaError_t allow_smem(const void *kernel, size_t bytes);
// The library's device allocations (devmem.cu): plain cudaMalloc, or with
// guard bands when NS_GUARD=1.
cudaError_t dev_malloc(void **p, size_t bytes);
void dev_free(void *p);

// Opt every transform kernel in up front (called by ns_init, so that nothing
// of the kind happens while a step is being captured into a graph).
cudaError_t prepare_fft_kernels();

}  // namespace nsk
