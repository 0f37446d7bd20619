// reduce.cuh -- deterministic FP64 reductions shared by the plain and fused
// forms: a fixed-order block tree and the shell-spectrum kernel (the
// reductions for global quantities and spectra of Sec. 3, done without
// floating-point atomics so that repeated runs agree bit for bit).
#pragma once
#include <cuda_runtime.h>

namespace nsk {

// Block tree sum of two doubles in a fixed order (deterministic).
__device__ __forceinline__ void block_sum2(double &s0, double &s1, double *sh) {
    const int t = threadIdx.x;
    sh[2 * t] = s0;
    sh[2 * t + 1] = s1;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w) {
            sh[2 * t] += sh[2 * (t + w)];
            sh[2 * t + 1] += sh[2 * (t + w) + 1];
        }
        __syncthreads();
    }
    s0 = sh[0];
    s1 = sh[1];
}

// Blocks per shell of the spectrum kernels (grid y).  Their partial sums sit
// after the nbins results in spec and ens, which hold nbins (1 + kShellParts)
// doubles each; k_shell_finish adds them in a fixed order.
constexpr int kShellParts = 8;

// Shell spectrum: blocks (K, p) sum the modes with round-half-up(|k|) = K,
// i.e. K^2 - K + 1 <= |k|^2 <= K^2 + K (|k|^2 = 0 for K = 0), enumerating
// the (kx, ky) pairs p, p + kShellParts, ... (in units of the block size) and
// the kz interval each allows.  Per-thread sums in a fixed order and a fixed
// tree make the result deterministic.  Acc maps signed (kx, ky, kz) with
// kz >= 0 to the squared magnitude of the 3-vector coefficient, or 0.
template <class Acc>
__global__ void __launch_bounds__(256)
k_shell_spectrum(Acc acc, int n, int nbins, double *spec, double *ens) {
    __shared__ double sh[512];
    const int K = blockIdx.x, part = blockIdx.y;
    if (K >= nbins) return;
    const long lo = K == 0 ? 0 : (long)K * K - K + 1, hi = (long)K * K + K;
    const int kmin = -n / 2, kmax = n / 2 - 1;
    const int lim = K;   // |k_i| <= K inside the shell
    const int a0 = max(kmin, -lim), a1 = min(kmax, lim);
    const long side = a1 - a0 + 1;
    double e = 0.0, om = 0.0;
    for (long pidx = (long)part * blockDim.x + threadIdx.x; pidx < side * side;
         pidx += (long)blockDim.x * gridDim.y) {
        const int kx = a0 + (int)(pidx / side), ky = a0 + (int)(pidx % side);
        const long r2 = (long)kx * kx + (long)ky * ky;
        if (r2 > hi) continue;
        long zlo2 = lo - r2;
        int z0 = 0;
        if (zlo2 > 0) {
            z0 = (int)ceil(sqrt((double)zlo2));
            while ((long)z0 * z0 < zlo2) z0++;
            while (z0 > 0 && (long)(z0 - 1) * (z0 - 1) >= zlo2) z0--;
        }
        int z1 = (int)floor(sqrt((double)(hi - r2)));
        while ((long)(z1 + 1) * (z1 + 1) <= hi - r2) z1++;
        while (z1 >= 0 && (long)z1 * z1 > hi - r2) z1--;
        z1 = min(z1, n / 2);
        for (int kz = z0; kz <= z1; kz++) {
            const double w = (kz == 0 || 2 * kz == n) ? 0.5 : 1.0;
            const double de = w * acc(kx, ky, kz);
            e += de;
            om += de * (double)(r2 + (long)kz * kz);
        }
    }
    block_sum2(e, om, sh);
    if (threadIdx.x == 0) {
        spec[nbins + K * kShellParts + part] = e;
        ens[nbins + K * kShellParts + part] = om;
    }
}

// spec[K] = the sum of the shell's kShellParts partials, in order (and ens).
static __global__ void k_shell_finish(double *spec, double *ens, int nbins) {
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    if (K >= nbins) return;
    double e = 0.0, om = 0.0;
    for (int p = 0; p < kShellParts; p++) {
        e += spec[nbins + K * kShellParts + p];
        om += ens[nbins + K * kShellParts + p];
    }
    spec[K] = e;
    ens[K] = om;
}

// Launch a shell-spectrum kernel over nbins x kShellParts blocks, then the
// ordered sum of the partials.
template <class Kernel, class... Args>
static cudaError_t shell_launch(Kernel k, int nbins, double *spec, double *ens, cudaStream_t s, Args... args) {
    k<<<dim3(nbins, kShellParts), 256, 0, s>>>(args..., spec, ens);
    k_shell_finish<<<(nbins + 255) / 256, 256, 0, s>>>(spec, ens, nbins);
    return cudaGetLastError();
}

// Re(a . conj(w)) with w = i k x a, for the helicity 1/2 <u . w>.
__device__ __forceinline__ double helicity_density(double kx, double ky, double kz, double axr,
                                                   double axi, double ayr, double ayi, double azr,
                                                   double azi) {
    // k x a
    const double cxr = ky * azr - kz * ayr, cxi = ky * azi - kz * ayi;
    const double cyr = kz * axr - kx * azr, cyi = kz * axi - kx * azi;
    const double czr = kx * ayr - ky * axr, czi = kx * ayi - ky * axi;
    // w = i (k x a) = (-ci, cr); Re(a conj w) = ar * wr + ai * wi = -ar ci + ai cr
    return -axr * cxi + axi * cxr - ayr * cyi + ayi * cyr - azr * czi + azi * czr;
}

}  // namespace nsk
