// fft_passes.cu -- the axis passes of the unpruned 3D r2c / c2r transforms
// (Sec. 2, Fig. 1: 1D FFTs along each direction of the N^3 box with the
// (N/2+1) x N x N half storage).  On one GPU the slab transposes of the
// paper become the data layout of these passes: the strided passes read and
// write rows of contiguous columns (coalesced 128-byte rows), so no separate
// transpose ever touches HBM.
#include <math.h>

#include <mutex>
#include <set>
#include <vector>

#include "ns_internal.h"

namespace nsk {

// ---------------------------------------------------------------- plans

static void factor23(int n, int &a, int &b, int &rest) {
    a = b = 0;
    while (n > 1 && n % 2 == 0) { n /= 2; a++; }
    while (n > 1 && n % 3 == 0) { n /= 3; b++; }
    rest = n;
}

bool make_plan(int n, Plan *pl) {
    int a, b, rest;
    if (n < 4) return false;
    factor23(n, a, b, rest);
    if (rest != 1) return false;
    int E;
    if (b == 0) E = n < 16 ? n : 16;
    else if (a >= 2) E = 12;
    else if (a == 1) E = 6;
    else E = b >= 2 ? 9 : 3;
    return make_plan_e(n, E, pl);
}

bool make_plan_e(int n, int E, Plan *pl) {
    int a, b, rest;
    if (n < 4) return false;
    factor23(n, a, b, rest);
    if (rest != 1 || n % E != 0) return false;
    if (E != 4 && E != 6 && E != 8 && E != 9 && E != 12 && E != 16) return false;
    static const int cand[] = {16, 12, 9, 8, 6, 4, 3, 2};
    pl->n = n;
    pl->E = E;
    pl->nst = 0;
    pl->radix = 0;
    int m = n;
    while (m > 1) {
        int R = 0;
        for (int r : cand)
            if (E % r == 0 && m % r == 0) { R = r; break; }
        if (R == 0 || pl->nst >= 12) return false;
        pl->radix |= (unsigned long long)R << (5 * pl->nst);
        pl->nst++;
        m /= R;
    }
    return true;
}

bool supported_n(int n) {
    if (n < 8 || n % 2) return false;
    Plan p;
    return make_plan(n, &p) && make_plan(n / 2, &p);
}

int default_ct(int elem_bytes, int n) {
    // 128-byte rows, within the thread bound of the strided kernel
    // (512 threads for float, 384 for double: no register spills).
    int ct = 128 / elem_bytes;
    const int bound = elem_bytes == 8 ? 512 : 384;
    Plan p;
    if (make_plan(n, &p)) {
        const int T = n / p.E;
        while (ct > 1 && ct * T > bound) ct /= 2;
    }
    return ct;
}

// Raise a kernel's dynamic shared-memory opt-in to the device maximum, once
// per (device, kernel).  Occupancy depends on what a launch asks for, not on
// this limit, so one setting serves every launch size.
cudaError_t allow_smem(const void *kernel, size_t bytes) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(dev, kernel);
    if (done.count(key)) return cudaSuccess;
    int maxopt = 0;
    e = cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    // the opt-in maximum covers static and dynamic shared memory together
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    if (fa.sharedSizeBytes >= (size_t)maxopt) return cudaErrorInvalidValue;
    const int maxdyn = maxopt - (int)fa.sharedSizeBytes;
    if (bytes > (size_t)maxdyn) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, maxdyn);
    if (e == cudaSuccess) done.insert(key);
    return e;
}

template <typename T> typename Cx<T>::type *make_twiddles(int n, cudaError_t *err) {
    typedef typename Cx<T>::type C;
    std::vector<C> h(n);
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < n; t++) {
        const double a = two_pi * (double)t / (double)n;
        h[t].x = (T)cos(a);
        h[t].y = (T)(-sin(a));
    }
    C *d = nullptr;
    *err = dev_malloc((void **)&d, sizeof(C) * n);
    if (*err != cudaSuccess) return nullptr;
    *err = cudaMemcpy(d, h.data(), sizeof(C) * n, cudaMemcpyHostToDevice);
    if (*err != cudaSuccess) {
        dev_free(d);
        return nullptr;
    }
    return d;
}
template float2 *make_twiddles<float>(int, cudaError_t *);
template double2 *make_twiddles<double>(int, cudaError_t *);

// ---------------------------------------------------------------- strided pass

template <typename T> struct Bounds;
template <> struct Bounds<float> { enum { threads = 512 }; };
template <> struct Bounds<double> { enum { threads = 384 }; };

// The columns of a plane a strided launch transforms, as the kernel sees
// them: the plane is nouter rows of `inner` columns, of which rows [0, o1)
// and [o2, nouter) and the first `keep` columns of each are done, tpr tiles
// of ct columns per row; rows e of the transform axis in [gap_lo, gap_hi)
// read as zero (inverse) or are not written (forward).
struct SelK {
    long inner;
    int keep, tpr, o1, o2, gap_lo, gap_hi;
};

// One CTA: ct contiguous columns of one plane, T = n/E threads per column,
// lanes along columns (coalesced rows).  Shared tile: element (e, c) at
// e * ct + c.
template <typename T, int E, int DIR>
__global__ void __launch_bounds__(Bounds<T>::threads)
k_fft_strided(const typename Cx<T>::type *__restrict__ in, typename Cx<T>::type *out, SelK sel,
              long es, long ps_in, long ps_out, Plan pl, const typename Cx<T>::type *__restrict__ tw,
              int ntab) {
    typedef typename Cx<T>::type C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    const int ct = blockDim.x / (pl.n / E);
    const int c = threadIdx.x % ct;
    const int slot = threadIdx.x / ct;
    const int ro = blockIdx.x / sel.tpr;
    const long inner = (long)(blockIdx.x - ro * sel.tpr) * ct + c;
    const long col = (long)(ro < sel.o1 ? ro : ro - sel.o1 + sel.o2) * sel.inner + inner;
    const bool valid = inner < sel.keep;
    const C *src = in + (long)blockIdx.y * ps_in + col;
    C *dst = out + (long)blockIdx.y * ps_out + col;
    auto in_gap = [&](int e) { return e >= sel.gap_lo && e < sel.gap_hi; };
    auto gl = [&](int e) -> C { return valid && (DIR < 0 || !in_gap(e)) ? src[e * es] : czero<C>(); };
    auto gs = [&](int e, C v) {
        if (valid && (DIR > 0 || !in_gap(e))) dst[e * es] = v;
    };
    auto sl = [&](int e) -> C { return sm[e * ct + c]; };
    auto ss = [&](int e, C v) { sm[e * ct + c] = v; };
    fft_line<E, DIR, false, false, true>(pl, slot, tw, ntab, gl, sl, ss, gs);
}

template <typename T, int DIR>
static const void *strided_kernel(int E) {
    switch (E) {
    case 4: return (const void *)k_fft_strided<T, 4, DIR>;
    case 6: return (const void *)k_fft_strided<T, 6, DIR>;
    case 8: return (const void *)k_fft_strided<T, 8, DIR>;
    case 9: return (const void *)k_fft_strided<T, 9, DIR>;
    case 12: return (const void *)k_fft_strided<T, 12, DIR>;
    case 16: return (const void *)k_fft_strided<T, 16, DIR>;
    }
    return nullptr;
}

template <typename T>
cudaError_t fft_strided(const typename Cx<T>::type *in, typename Cx<T>::type *out, long ncols,
                        long es, long ps_in, long ps_out, int planes, int dir, const Plan &pl,
                        const typename Cx<T>::type *tw, int ntab, int ct, cudaStream_t s,
                        const StridedSel *sel) {
    typedef typename Cx<T>::type C;
    const void *k = dir < 0 ? strided_kernel<T, -1>(pl.E) : strided_kernel<T, +1>(pl.E);
    if (!k || planes < 1 || planes > 65535) return cudaErrorInvalidValue;
    const int T_ = pl.n / pl.E;
    if (ct < 1 || ct * T_ > (int)Bounds<T>::threads) return cudaErrorInvalidValue;
    if (ncols < 1 || ncols > 0x7fff0000L) return cudaErrorInvalidValue;
    SelK sk{ncols, (int)ncols, 0, 1, 1, 0, 0};
    int nrows = 1;
    if (sel) {
        if (sel->nouter < 1 || sel->inner < 1 || sel->keep < 0 || sel->keep > sel->inner ||
            sel->inner * sel->nouter != ncols || sel->o1 < 0 || sel->o1 > sel->o2 || sel->o2 > sel->nouter ||
            sel->gap_lo < 0 || sel->gap_lo > sel->gap_hi || sel->gap_hi > pl.n)
            return cudaErrorInvalidValue;
        sk = SelK{sel->inner, sel->keep, 0, sel->o1, sel->o2, sel->gap_lo, sel->gap_hi};
        nrows = sel->o1 + sel->nouter - sel->o2;
    }
    if (sk.keep > 0x7fffffffL - ct) return cudaErrorInvalidValue;
    sk.tpr = (sk.keep + ct - 1) / ct;
    if (nrows < 1 || sk.tpr < 1) return cudaSuccess;   // nothing selected
    if ((long)nrows * sk.tpr > 0x7fffffffL) return cudaErrorInvalidValue;
    const size_t smem = (size_t)pl.n * ct * sizeof(C);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(nrows * sk.tpr), (unsigned)planes);
    Plan p = pl;
    void *args[] = {(void *)&in, (void *)&out, (void *)&sk, (void *)&es, (void *)&ps_in,
                    (void *)&ps_out, (void *)&p, (void *)&tw, (void *)&ntab};
    return cudaLaunchKernel(k, grid, dim3(ct * T_), args, smem, s);
}
template cudaError_t fft_strided<float>(const float2 *, float2 *, long, long, long, long, int, int,
                                        const Plan &, const float2 *, int, int, cudaStream_t,
                                        const StridedSel *);
template cudaError_t fft_strided<double>(const double2 *, double2 *, long, long, long, long, int,
                                         int, const Plan &, const double2 *, int, int,
                                         cudaStream_t, const StridedSel *);

// ---------------------------------------------------------------- z passes

// Shared-memory line with a skew of one element every 128 bytes, so that the
// stride-R writes of the early Stockham stages spread over the banks.
template <typename C> struct Skew;
template <> struct Skew<float2> { enum { shift = 4 }; };
template <> struct Skew<double2> { enum { shift = 3 }; };
template <typename C> __host__ __device__ inline int skew_len(int n) {
    return n + (n >> Skew<C>::shift) + 2;
}

// r2c along z.  The N reals of a line, read as n = N/2 complex values
// z[m] = x[2m] + i x[2m+1], go through one length-n FFT; then
// X[k] = (Z[k] + conj Z[n-k])/2 - i W^k (Z[k] - conj Z[n-k])/2, W = e^{-2 pi i/N},
// for k = 0..n (Z[n] = Z[0]), of which those below kzk are written.  One CTA
// holds lb lines, T = n/E threads each.
template <typename T, int E>
__global__ void __launch_bounds__(256)
k_fft_z_r2c(const T *__restrict__ in, typename Cx<T>::type *__restrict__ out, int N, long nlines,
            Plan pl, const typename Cx<T>::type *__restrict__ tw, int kzk) {
    typedef typename Cx<T>::type C;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = N / 2, Tn = n / E;
    const int slot = threadIdx.x % Tn, li = threadIdx.x / Tn;
    const int lb = blockDim.x / Tn;
    const long line = (long)blockIdx.x * lb + li;
    const bool valid = line < nlines;
    C *ls = reinterpret_cast<C *>(smraw) + li * skew_len<C>(n);
    const int sh = Skew<C>::shift;
    const C *src = reinterpret_cast<const C *>(in + line * N);
    auto gl = [&](int e) -> C { return valid ? src[e] : czero<C>(); };
    auto sl = [&](int e) -> C { return ls[e + (e >> sh)]; };
    auto ss = [&](int e, C v) { ls[e + (e >> sh)] = v; };
    fft_line<E, -1, false, true, false>(pl, slot, tw, N, gl, sl, ss, ss);
    if (!valid) return;
    C *dst = out + line * (n + 1);
    for (int k = slot; k <= n && k < kzk; k += Tn) {
        dst[k] = r2c_unpack(sl(k == n ? 0 : k), sl(k == 0 ? 0 : n - k), ldg_c(tw + k));
    }
}

// c2r along z: Z[k] = (X[k] + conj X[n-k]) + i W^{-k} (X[k] - conj X[n-k]),
// k < n, with the real parts of X[0] and X[n]; one inverse length-n FFT gives
// z[m] = x[2m] + i x[2m+1].  Entries X[k], k >= kzk, read as zero.
template <typename T, int E>
__global__ void __launch_bounds__(256)
k_fft_z_c2r(const typename Cx<T>::type *__restrict__ in, T *__restrict__ out, int N, long nlines,
            Plan pl, const typename Cx<T>::type *__restrict__ tw, int kzk) {
    typedef typename Cx<T>::type C;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = N / 2, Tn = n / E;
    const int slot = threadIdx.x % Tn, li = threadIdx.x / Tn;
    const int lb = blockDim.x / Tn;
    const long line = (long)blockIdx.x * lb + li;
    const bool valid = line < nlines;
    C *ls = reinterpret_cast<C *>(smraw) + li * skew_len<C>(n);
    const int sh = Skew<C>::shift;
    auto sl = [&](int e) -> C { return ls[e + (e >> sh)]; };
    auto ss = [&](int e, C v) { ls[e + (e >> sh)] = v; };
    const C *src = in + line * (n + 1);
    for (int k = slot; k < n; k += Tn) {
        C xk = czero<C>(), xm = czero<C>();
        if (valid) {
            if (k < kzk) xk = src[k];
            if (n - k < kzk) xm = src[n - k];
            if (k == 0) {
                xk.y = 0;
                xm.y = 0;
            }
        }
        ss(k, c2r_pack(xk, xm, ldg_c(tw + k)));
    }
    __syncthreads();
    C *dst = reinterpret_cast<C *>(out + line * N);
    auto gs = [&](int e, C v) {
        if (valid) dst[e] = v;
    };
    fft_line<E, +1, true, false, false>(pl, slot, tw, N, sl, sl, ss, gs);
}

// Two real lines through one complex transform of length N (the plan of
// length N selects this form; one of length N/2 the packed form above).  Per
// line pair the length-N transform costs 5N flops more than two of length
// N/2 but needs no even/odd packing, which saves about 14 % of the
// arithmetic instructions of c2r and 8 % of r2c.
//  c2r: the spectra X1, X2 of lines 2p and 2p + 1 (the imaginary parts of
//       X[0] and X[N/2] dropped) form Z[k] = X1[k] + i X2[k] for k <= N/2 and
//       Z[k] = conj X1[N-k] + i conj X2[N-k] above, a Hermitian pair; the
//       inverse transform of Z is x1 + i x2.
//  r2c: the forward transform Z of x1 + i x2 gives
//       X1[k] = (Z[k] + conj Z[N-k]) / 2 and X2[k] = (Z[k] - conj Z[N-k]) / 2i.
// A missing second line (odd line count) reads as zero and is not written.
// Only the entries below kzk are read (c2r; the others are zero) or written
// (r2c).
template <typename T, int E>
__global__ void __launch_bounds__(256)
k_fft_z_r2c2(const T *__restrict__ in, typename Cx<T>::type *__restrict__ out, int N, long nlines,
             Plan pl, const typename Cx<T>::type *__restrict__ tw, int kzk) {
    typedef typename Cx<T>::type C;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nh = N / 2, Tn = N / E;
    const int slot = threadIdx.x % Tn, li = threadIdx.x / Tn;
    const int lb = blockDim.x / Tn;
    const long l1 = 2 * ((long)blockIdx.x * lb + li), l2 = l1 + 1;
    const bool v1 = l1 < nlines, v2 = l2 < nlines;
    C *ls = reinterpret_cast<C *>(smraw) + li * skew_len<C>(N);
    const int sh = Skew<C>::shift;
    const T *s1 = in + l1 * N, *s2 = in + l2 * N;
    auto gl = [&](int e) -> C { return mkc(v1 ? s1[e] : (T)0, v2 ? s2[e] : (T)0); };
    auto sl = [&](int e) -> C { return ls[e + (e >> sh)]; };
    auto ss = [&](int e, C v) { ls[e + (e >> sh)] = v; };
    fft_line<E, -1, false, true, false>(pl, slot, tw, N, gl, sl, ss, ss);
    C *d1 = out + l1 * (nh + 1), *d2 = out + l2 * (nh + 1);
    const T half = (T)0.5;
    for (int k = slot; k <= nh && k < kzk; k += Tn) {
        const C a = sl(k), b = sl(k == 0 ? 0 : N - k);
        if (v1) d1[k] = mkc((a.x + b.x) * half, (a.y - b.y) * half);
        if (v2) d2[k] = mkc((a.y + b.y) * half, (b.x - a.x) * half);
    }
}

template <typename T, int E>
__global__ void __launch_bounds__(256)
k_fft_z_c2r2(const typename Cx<T>::type *__restrict__ in, T *__restrict__ out, int N, long nlines,
             Plan pl, const typename Cx<T>::type *__restrict__ tw, int kzk) {
    typedef typename Cx<T>::type C;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nh = N / 2, Tn = N / E;
    const int slot = threadIdx.x % Tn, li = threadIdx.x / Tn;
    const int lb = blockDim.x / Tn;
    const long l1 = 2 * ((long)blockIdx.x * lb + li), l2 = l1 + 1;
    const bool v1 = l1 < nlines, v2 = l2 < nlines;
    C *ls = reinterpret_cast<C *>(smraw) + li * skew_len<C>(N);
    const int sh = Skew<C>::shift;
    auto sl = [&](int e) -> C { return ls[e + (e >> sh)]; };
    auto ss = [&](int e, C v) { ls[e + (e >> sh)] = v; };
    const C *s1 = in + l1 * (nh + 1), *s2 = in + l2 * (nh + 1);
    for (int k = slot; k < N; k += Tn) {
        const int m = k <= nh ? k : N - k;
        C a = v1 && m < kzk ? s1[m] : czero<C>(), b = v2 && m < kzk ? s2[m] : czero<C>();
        if (m == 0 || m == nh) {
            a.y = 0;
            b.y = 0;
        }
        ss(k, k <= nh ? mkc(a.x - b.y, a.y + b.x) : mkc(a.x + b.y, b.x - a.y));
    }
    __syncthreads();
    T *d1 = out + l1 * N, *d2 = out + l2 * N;
    auto gs = [&](int e, C v) {
        if (v1) d1[e] = v.x;
        if (v2) d2[e] = v.y;
    };
    fft_line<E, +1, true, false, false>(pl, slot, tw, N, sl, sl, ss, gs);
}

template <typename T, bool R2C>
static const void *z_kernel2(int E) {
#define NSK_ZK2(EE) \
    return R2C ? (const void *)k_fft_z_r2c2<T, EE> : (const void *)k_fft_z_c2r2<T, EE>
    switch (E) {
    case 4: NSK_ZK2(4);
    case 6: NSK_ZK2(6);
    case 8: NSK_ZK2(8);
    case 9: NSK_ZK2(9);
    case 12: NSK_ZK2(12);
    case 16: NSK_ZK2(16);
    }
#undef NSK_ZK2
    return nullptr;
}

template <typename T, bool R2C>
static const void *z_kernel(int E) {
#define NSK_ZK(EE) \
    return R2C ? (const void *)k_fft_z_r2c<T, EE> : (const void *)k_fft_z_c2r<T, EE>
    switch (E) {
    case 4: NSK_ZK(4);
    case 6: NSK_ZK(6);
    case 8: NSK_ZK(8);
    case 9: NSK_ZK(9);
    case 12: NSK_ZK(12);
    case 16: NSK_ZK(16);
    }
#undef NSK_ZK
    return nullptr;
}

// pl.n == N / 2: one line per complex transform (even/odd packing);
// pl.n == N: two lines per complex transform.
template <typename T, bool R2C>
static cudaError_t launch_z(const void *in, void *out, int N, long nlines, const Plan &pl,
                            const typename Cx<T>::type *tw, cudaStream_t s, int kzk) {
    typedef typename Cx<T>::type C;
    const bool paired = pl.n == N;
    const void *k = paired ? z_kernel2<T, R2C>(pl.E) : z_kernel<T, R2C>(pl.E);
    if (!k || (!paired && pl.n * 2 != N) || nlines < 1) return cudaErrorInvalidValue;
    if (kzk < 0 || kzk > N / 2 + 1) kzk = N / 2 + 1;   // every entry
    const int Tn = pl.n / pl.E;
    int lb = 256 / Tn;
    if (lb < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)lb * skew_len<C>(pl.n) * sizeof(C);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    const long units = paired ? (nlines + 1) / 2 : nlines;   // transforms
    const long blocks = (units + lb - 1) / lb;
    if (blocks > 0x7fffffffL) return cudaErrorInvalidValue;
    Plan p = pl;
    void *args[] = {(void *)&in, (void *)&out, (void *)&N, (void *)&nlines, (void *)&p,
                    (void *)&tw, (void *)&kzk};
    return cudaLaunchKernel(k, dim3((unsigned)blocks), dim3(lb * Tn), args, smem, s);
}

template <typename T>
cudaError_t fft_z_r2c(const T *in, typename Cx<T>::type *out, int N, long nlines, const Plan &pl,
                      const typename Cx<T>::type *tw, cudaStream_t s, int kzk) {
    return launch_z<T, true>(in, out, N, nlines, pl, tw, s, kzk);
}
template <typename T>
cudaError_t fft_z_c2r(const typename Cx<T>::type *in, T *out, int N, long nlines,
                      const Plan &pl, const typename Cx<T>::type *tw, cudaStream_t s, int kzk) {
    return launch_z<T, false>(in, out, N, nlines, pl, tw, s, kzk);
}
cudaError_t prepare_fft_kernels() {
    const size_t big = 48 * 1024 + 1;
    const int Es[] = {4, 6, 8, 9, 12, 16};
    for (int E : Es) {
        const void *ks[] = {strided_kernel<float, -1>(E), strided_kernel<float, 1>(E),
                            strided_kernel<double, -1>(E), strided_kernel<double, 1>(E),
                            z_kernel<float, true>(E), z_kernel<float, false>(E),
                            z_kernel<double, true>(E), z_kernel<double, false>(E),
                            z_kernel2<float, true>(E), z_kernel2<float, false>(E),
                            z_kernel2<double, true>(E), z_kernel2<double, false>(E)};
        for (const void *k : ks) {
            cudaError_t e = allow_smem(k, big);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

template cudaError_t fft_z_r2c<float>(const float *, float2 *, int, long, const Plan &,
                                      const float2 *, cudaStream_t, int);
template cudaError_t fft_z_r2c<double>(const double *, double2 *, int, long, const Plan &,
                                       const double2 *, cudaStream_t, int);
template cudaError_t fft_z_c2r<float>(const float2 *, float *, int, long, const Plan &,
                                      const float2 *, cudaStream_t, int);
template cudaError_t fft_z_c2r<double>(const double2 *, double *, int, long, const Plan &,
                                       const double2 *, cudaStream_t, int);

}  // namespace nsk
