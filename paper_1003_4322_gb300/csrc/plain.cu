// plain.cu -- the unfused, unpruned ("plain") form of the solver's pointwise
// steps on full half-layout arrays [3][N][N][N/2+1] (Sec. 2, Eqs. 1-2): the
// vorticity i k x a, the cross product u x w on the grid, and the projected,
// dealiased, forced integrating-factor RK2 update; plus the deterministic
// FP64 reductions for energy, enstrophy and the shell spectrum (the global
// quantities and spectra of Sec. 3).
#include "ns_internal.h"
#include "plain.h"
#include "reduce.cuh"

namespace nsk {

__device__ __forceinline__ int wavenum(int i, int n) { return 2 * i < n ? i : i - n; }

// ---------------------------------------------------------------- curl

template <typename T>
__global__ void k_curl(const typename Cx<T>::type *__restrict__ a, typename Cx<T>::type *__restrict__ w,
                       int n, long M) {
    typedef typename Cx<T>::type C;
    const int nh = n / 2 + 1;
    for (long m = blockIdx.x * (long)blockDim.x + threadIdx.x; m < M; m += (long)gridDim.x * blockDim.x) {
        const int kz = (int)(m % nh);
        const int iy = (int)((m / nh) % n);
        const int ix = (int)(m / ((long)nh * n));
        const T kx = (T)wavenum(ix, n), ky = (T)wavenum(iy, n), kzz = (T)kz;
        const C ax = a[m], ay = a[M + m], az = a[2 * M + m];
        // w = i k x a
        w[m] = cmul_i<1>(csub(cscale(az, ky), cscale(ay, kzz)));
        w[M + m] = cmul_i<1>(csub(cscale(ax, kzz), cscale(az, kx)));
        w[2 * M + m] = cmul_i<1>(csub(cscale(ay, kx), cscale(ax, ky)));
    }
}

// ---------------------------------------------------------------- cross product

// c = u x w at every grid point; c may alias u.
template <typename T>
__global__ void k_cross(T *u, const T *__restrict__ w, long V) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V; i += (long)gridDim.x * blockDim.x) {
        const T ux = u[i], uy = u[V + i], uz = u[2 * V + i];
        const T wx = w[i], wy = w[V + i], wz = w[2 * V + i];
        u[i] = uy * wz - uz * wy;
        u[V + i] = uz * wx - ux * wz;
        u[2 * V + i] = ux * wy - uy * wx;
    }
}

// MHD products on the grid: g = [u, w, b, j] (3 components each, V points
// per component); on return g[0..3V) = u x w + j x b and g[3V..6V) = u x b.
template <typename T>
__global__ void k_cross_mhd(T *g, long V) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < V; i += (long)gridDim.x * blockDim.x) {
        const T ux = g[i], uy = g[V + i], uz = g[2 * V + i];
        const T wx = g[3 * V + i], wy = g[4 * V + i], wz = g[5 * V + i];
        const T bx = g[6 * V + i], by = g[7 * V + i], bz = g[8 * V + i];
        const T jx = g[9 * V + i], jy = g[10 * V + i], jz = g[11 * V + i];
        g[i] = uy * wz - uz * wy + (jy * bz - jz * by);
        g[V + i] = uz * wx - ux * wz + (jz * bx - jx * bz);
        g[2 * V + i] = ux * wy - uy * wx + (jx * by - jy * bx);
        g[3 * V + i] = uy * bz - uz * by;
        g[4 * V + i] = uz * bx - ux * bz;
        g[5 * V + i] = ux * by - uy * bx;
    }
}

// ---------------------------------------------------------------- update

// ABC forcing coefficients at signed k (closed form of
// f = F (sin kf z + cos kf y, sin kf x + cos kf z, sin kf y + cos kf x)).
template <typename C, typename T>
__device__ __forceinline__ void abc_forcing(int kx, int ky, int kz, int kf, T F, C &fx, C &fy, C &fz) {
    const T h = F * (T)0.5;
    if (kf <= 0) return;
    if (kx == 0 && ky == 0 && kz == kf) {          // e^{i kf z}: sin -> -i/2, cos -> 1/2
        fx = cadd(fx, mkc((T)0, -h));
        fy = cadd(fy, mkc(h, (T)0));
    }
    if (kx == 0 && kz == 0 && (ky == kf || ky == -kf)) {
        fx = cadd(fx, mkc(h, (T)0));
        fz = cadd(fz, mkc((T)0, ky > 0 ? -h : h));
    }
    if (ky == 0 && kz == 0 && (kx == kf || kx == -kf)) {
        fy = cadd(fy, mkc((T)0, kx > 0 ? -h : h));
        fz = cadd(fz, mkc(h, (T)0));
    }
}

__device__ __forceinline__ bool kept(int kx, int ky, int kz, int n, int dealias) {
    int m = abs(kx);
    m = max(m, abs(ky));
    m = max(m, abs(kz));
    if (dealias == 2) return 2 * m < n && 9L * (kx * kx + ky * ky + kz * kz) < 2L * n * n;
    if (3 * m >= n) return false;
    if (dealias == 1 && 9L * (kx * kx + ky * ky + kz * kz) >= (long)n * n) return false;
    return true;
}

// Stage 1: a1 = E (a + dt N);  stage 2: a = E a / 2 + (a1 + dt N) / 2, with
// N = P Pi (nl / N^3) + f_hat; every mode outside Pi (and k = 0) set to 0.
template <typename T>
__global__ void k_update(typename Cx<T>::type *__restrict__ a, typename Cx<T>::type *__restrict__ a1,
                         const typename Cx<T>::type *__restrict__ nl, const T *__restrict__ etab,
                         int n, long M, UpdateArgs ua) {
    typedef typename Cx<T>::type C;
    const int nh = n / 2 + 1;
    const T inv = (T)(1.0 / ((double)n * n * n));
    const T dt = (T)ua.dt, F = (T)ua.force_amp;
    for (long m = blockIdx.x * (long)blockDim.x + threadIdx.x; m < M; m += (long)gridDim.x * blockDim.x) {
        const int kz = (int)(m % nh);
        const int iy = (int)((m / nh) % n);
        const int ix = (int)(m / ((long)nh * n));
        const int kx = wavenum(ix, n), ky = wavenum(iy, n);
        const int k2 = kx * kx + ky * ky + kz * kz;
        C o0 = czero<C>(), o1 = czero<C>(), o2 = czero<C>();
        if (kept(kx, ky, kz, n, ua.dealias) && k2 > 0) {
            C vx = cscale(nl[m], inv), vy = cscale(nl[M + m], inv), vz = cscale(nl[2 * M + m], inv);
            if (ua.rot != 0.0) {   // Coriolis -2 rot z x u of the stage's state, before P
                const C *cur = ua.stage == 1 ? a : a1;
                const T r2 = (T)(2.0 * ua.rot);
                vx = cadd(vx, cscale(cur[M + m], r2));
                vy = csub(vy, cscale(cur[m], r2));
            }
            const T fkx = (T)kx, fky = (T)ky, fkz = (T)kz, ik2 = (T)1 / (T)k2;
            const C kv = cadd(cadd(cscale(vx, fkx), cscale(vy, fky)), cscale(vz, fkz));
            vx = csub(vx, cscale(kv, fkx * ik2));
            vy = csub(vy, cscale(kv, fky * ik2));
            vz = csub(vz, cscale(kv, fkz * ik2));
            abc_forcing(kx, ky, kz, ua.force_k, F, vx, vy, vz);
            const T e = etab[k2];
            if (ua.stage == 1) {
                o0 = cscale(cadd(a[m], cscale(vx, dt)), e);
                o1 = cscale(cadd(a[M + m], cscale(vy, dt)), e);
                o2 = cscale(cadd(a[2 * M + m], cscale(vz, dt)), e);
            } else {
                const T he = (T)0.5 * e, h = (T)0.5;
                o0 = cadd(cscale(a[m], he), cscale(cadd(a1[m], cscale(vx, dt)), h));
                o1 = cadd(cscale(a[M + m], he), cscale(cadd(a1[M + m], cscale(vy, dt)), h));
                o2 = cadd(cscale(a[2 * M + m], he), cscale(cadd(a1[2 * M + m], cscale(vz, dt)), h));
            }
        }
        C *dst = ua.stage == 1 ? a1 : a;
        dst[m] = o0;
        dst[M + m] = o1;
        dst[2 * M + m] = o2;
    }
}

// Induction update of the magnetic field: N_b = Pi (i k x nb / N^3) with nb
// the transform of u x b, then the IF-RK2 stage with the factor of eta.  The
// mean field b(k = 0) has N_b = 0 and factor 1, so it is carried unchanged.
template <typename T>
__global__ void k_update_b(typename Cx<T>::type *__restrict__ b, typename Cx<T>::type *__restrict__ b1,
                           const typename Cx<T>::type *__restrict__ nb, const T *__restrict__ etab,
                           int n, long M, int stage, double dt_, int dealias) {
    typedef typename Cx<T>::type C;
    const int nh = n / 2 + 1;
    const T inv = (T)(1.0 / ((double)n * n * n));
    const T dt = (T)dt_;
    for (long m = blockIdx.x * (long)blockDim.x + threadIdx.x; m < M; m += (long)gridDim.x * blockDim.x) {
        const int kz = (int)(m % nh);
        const int iy = (int)((m / nh) % n);
        const int ix = (int)(m / ((long)nh * n));
        const int kx = wavenum(ix, n), ky = wavenum(iy, n);
        const int k2 = kx * kx + ky * ky + kz * kz;
        C o0 = czero<C>(), o1 = czero<C>(), o2 = czero<C>();
        if (kept(kx, ky, kz, n, dealias)) {
            const C vx = cscale(nb[m], inv), vy = cscale(nb[M + m], inv), vz = cscale(nb[2 * M + m], inv);
            const T fkx = (T)kx, fky = (T)ky, fkz = (T)kz;
            // i k x v
            const C nx = cmul_i<1>(csub(cscale(vz, fky), cscale(vy, fkz)));
            const C ny = cmul_i<1>(csub(cscale(vx, fkz), cscale(vz, fkx)));
            const C nz = cmul_i<1>(csub(cscale(vy, fkx), cscale(vx, fky)));
            const T e = etab[k2];
            if (stage == 1) {
                o0 = cscale(cadd(b[m], cscale(nx, dt)), e);
                o1 = cscale(cadd(b[M + m], cscale(ny, dt)), e);
                o2 = cscale(cadd(b[2 * M + m], cscale(nz, dt)), e);
            } else {
                const T he = (T)0.5 * e, h = (T)0.5;
                o0 = cadd(cscale(b[m], he), cscale(cadd(b1[m], cscale(nx, dt)), h));
                o1 = cadd(cscale(b[M + m], he), cscale(cadd(b1[M + m], cscale(ny, dt)), h));
                o2 = cadd(cscale(b[2 * M + m], he), cscale(cadd(b1[2 * M + m], cscale(nz, dt)), h));
            }
        }
        C *dst = stage == 1 ? b1 : b;
        dst[m] = o0;
        dst[M + m] = o1;
        dst[2 * M + m] = o2;
    }
}

// Phase-shift dealiasing: dst = src exp(i k.D), D = (pi/N)(1,1,1), the
// coefficients of the field on the shifted grid (three components).
template <typename T>
__global__ void k_phase(const typename Cx<T>::type *__restrict__ src, typename Cx<T>::type *__restrict__ dst,
                        int n, long M) {
    typedef typename Cx<T>::type C;
    const int nh = n / 2 + 1;
    for (long m = blockIdx.x * (long)blockDim.x + threadIdx.x; m < M; m += (long)gridDim.x * blockDim.x) {
        const int kz = (int)(m % nh), iy = (int)((m / nh) % n), ix = (int)(m / ((long)nh * n));
        double s, c;
        sincospi((double)(wavenum(ix, n) + wavenum(iy, n) + kz) / n, &s, &c);
        const C ph = mkc((T)c, (T)s);
#pragma unroll
        for (int d = 0; d < 3; d++) dst[d * M + m] = cmul(src[d * M + m], ph);
    }
}

// acc = (acc + sh exp(-i k.D)) / 2: the product on the grid and, shifted
// back, on the shifted grid, averaged (three components).
template <typename T>
__global__ void k_phase_avg(typename Cx<T>::type *__restrict__ acc, const typename Cx<T>::type *__restrict__ sh,
                            int n, long M) {
    typedef typename Cx<T>::type C;
    const int nh = n / 2 + 1;
    for (long m = blockIdx.x * (long)blockDim.x + threadIdx.x; m < M; m += (long)gridDim.x * blockDim.x) {
        const int kz = (int)(m % nh), iy = (int)((m / nh) % n), ix = (int)(m / ((long)nh * n));
        double s, c;
        sincospi((double)(wavenum(ix, n) + wavenum(iy, n) + kz) / n, &s, &c);
        const C ph = mkc((T)c, (T)-s);
#pragma unroll
        for (int d = 0; d < 3; d++)
            acc[d * M + m] = cscale(cadd(acc[d * M + m], cmul(sh[d * M + m], ph)), (T)0.5);
    }
}

// ---------------------------------------------------------------- reductions

// Per-block partial energy and enstrophy of a half-layout state.  Block b
// owns the contiguous chunk [b*chunk, (b+1)*chunk) of modes.
template <typename T>
__global__ void __launch_bounds__(256)
k_energy_partials(const typename Cx<T>::type *__restrict__ a, int n, long M, long chunk, double *part) {
    __shared__ double sh[512];
    const int nh = n / 2 + 1;
    double e = 0.0, om = 0.0;
    const long beg = blockIdx.x * chunk, end = min(M, beg + chunk);
    for (long m = beg + threadIdx.x; m < end; m += blockDim.x) {
        const int kz = (int)(m % nh);
        const int iy = (int)((m / nh) % n);
        const int ix = (int)(m / ((long)nh * n));
        const double kx = wavenum(ix, n), ky = wavenum(iy, n);
        const double w = (kz == 0 || 2 * kz == n) ? 0.5 : 1.0;   // 1/2 * multiplicity
        double a2 = 0.0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const double re = (double)a[c * M + m].x, im = (double)a[c * M + m].y;
            a2 += re * re + im * im;
        }
        e += w * a2;
        om += w * a2 * (kx * kx + ky * ky + (double)kz * kz);
    }
    block_sum2(e, om, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = e;
        part[2 * blockIdx.x + 1] = om;
    }
}

// Sum nparts partials in a fixed order, append (E, Omega) to the run's ring
// buffer series[cap][2] at slot counter % cap, bump the counter, and raise
// bit 0 of *flags if E is not finite.
__global__ void __launch_bounds__(256)
k_energy_final(const double *__restrict__ part, int nparts, double *series, int cap,
               unsigned long long *counter, int *flags) {
    __shared__ double sh[512];
    double e = 0.0, om = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        e += part[2 * i];
        om += part[2 * i + 1];
    }
    block_sum2(e, om, sh);
    if (threadIdx.x == 0) {
        const unsigned long long c = *counter;
        series[2 * (c % cap)] = e;
        series[2 * (c % cap) + 1] = om;
        *counter = c + 1;
        if (!isfinite(e)) atomicOr(flags, 1);
    }
}

template <typename T> struct HalfAcc {
    const typename Cx<T>::type *a;
    int n;
    long M;
    __device__ double operator()(int kx, int ky, int kz) const {
        const long m = ((long)((kx + n) % n) * n + (ky + n) % n) * (n / 2 + 1) + kz;
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const double re = (double)a[c * M + m].x, im = (double)a[c * M + m].y;
            s += re * re + im * im;
        }
        return s;
    }
};

template <typename T> struct HalfHelAcc {
    const typename Cx<T>::type *a;
    int n;
    long M;
    __device__ double operator()(int kx, int ky, int kz) const {
        const long m = ((long)((kx + n) % n) * n + (ky + n) % n) * (n / 2 + 1) + kz;
        return helicity_density(kx, ky, kz, a[m].x, a[m].y, a[M + m].x, a[M + m].y, a[2 * M + m].x,
                                a[2 * M + m].y);
    }
};

// ---------------------------------------------------------------- launchers

static unsigned grid_for(long work, int threads) {
    long b = (work + threads - 1) / threads;
    if (b > 152L * 32) b = 152L * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

template <typename T>
cudaError_t plain_curl(const typename Cx<T>::type *a, typename Cx<T>::type *w, int n, cudaStream_t s) {
    const long M = (long)n * n * (n / 2 + 1);
    k_curl<T><<<grid_for(M, 256), 256, 0, s>>>(a, w, n, M);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_cross(T *u, const T *w, int n, cudaStream_t s) {
    const long V = (long)n * n * n;
    k_cross<T><<<grid_for(V, 256), 256, 0, s>>>(u, w, V);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_cross_mhd(T *g, int n, cudaStream_t s) {
    const long V = (long)n * n * n;
    k_cross_mhd<T><<<grid_for(V, 256), 256, 0, s>>>(g, V);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_update_b(typename Cx<T>::type *b, typename Cx<T>::type *b1,
                           const typename Cx<T>::type *nb, const T *etab, int n, int stage, double dt,
                           int dealias, cudaStream_t s) {
    const long M = (long)n * n * (n / 2 + 1);
    k_update_b<T><<<grid_for(M, 256), 256, 0, s>>>(b, b1, nb, etab, n, M, stage, dt, dealias);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_phase(const typename Cx<T>::type *src, typename Cx<T>::type *dst, int n, cudaStream_t s) {
    const long M = (long)n * n * (n / 2 + 1);
    k_phase<T><<<grid_for(M, 256), 256, 0, s>>>(src, dst, n, M);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_phase_avg(typename Cx<T>::type *acc, const typename Cx<T>::type *sh, int n, cudaStream_t s) {
    const long M = (long)n * n * (n / 2 + 1);
    k_phase_avg<T><<<grid_for(M, 256), 256, 0, s>>>(acc, sh, n, M);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_update(typename Cx<T>::type *a, typename Cx<T>::type *a1,
                         const typename Cx<T>::type *nl, const T *etab, int n, const UpdateArgs &ua,
                         cudaStream_t s) {
    const long M = (long)n * n * (n / 2 + 1);
    k_update<T><<<grid_for(M, 256), 256, 0, s>>>(a, a1, nl, etab, n, M, ua);
    return cudaGetLastError();
}

int energy_nparts(int n) {
    const long M = (long)n * n * (n / 2 + 1);
    long np = (M + 4095) / 4096;
    if (np > 1024) np = 1024;
    return (int)(np < 1 ? 1 : np);
}

template <typename T>
cudaError_t plain_energy_partials(const typename Cx<T>::type *a, int n, double *part, cudaStream_t s) {
    const long M = (long)n * n * (n / 2 + 1);
    const int np = energy_nparts(n);
    const long chunk = (M + np - 1) / np;
    k_energy_partials<T><<<np, 256, 0, s>>>(a, n, M, chunk, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_spectrum(const typename Cx<T>::type *a, int n, int nbins, double *spec, double *ens,
                           cudaStream_t s) {
    HalfAcc<T> acc{a, n, (long)n * n * (n / 2 + 1)};
    k_shell_spectrum<<<nbins, 256, 0, s>>>(acc, n, nbins, spec, ens);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_helicity(const typename Cx<T>::type *a, int n, int nbins, double *spec, double *aux,
                           cudaStream_t s) {
    HalfHelAcc<T> acc{a, n, (long)n * n * (n / 2 + 1)};
    k_shell_spectrum<<<nbins, 256, 0, s>>>(acc, n, nbins, spec, aux);
    return cudaGetLastError();
}

cudaError_t energy_final(const double *part, int nparts, double *series, int cap,
                         unsigned long long *counter, int *flags, cudaStream_t s) {
    k_energy_final<<<1, 256, 0, s>>>(part, nparts, series, cap, counter, flags);
    return cudaGetLastError();
}

#define NSK_INST(T)                                                                                \
    template cudaError_t plain_curl<T>(const Cx<T>::type *, Cx<T>::type *, int, cudaStream_t);    \
    template cudaError_t plain_cross<T>(T *, const T *, int, cudaStream_t);                       \
    template cudaError_t plain_cross_mhd<T>(T *, int, cudaStream_t);                              \
    template cudaError_t plain_phase<T>(const Cx<T>::type *, Cx<T>::type *, int, cudaStream_t);   \
    template cudaError_t plain_phase_avg<T>(Cx<T>::type *, const Cx<T>::type *, int, cudaStream_t); \
    template cudaError_t plain_update_b<T>(Cx<T>::type *, Cx<T>::type *, const Cx<T>::type *,     \
                                           const T *, int, int, double, int, cudaStream_t);       \
    template cudaError_t plain_update<T>(Cx<T>::type *, Cx<T>::type *, const Cx<T>::type *,       \
                                         const T *, int, const UpdateArgs &, cudaStream_t);       \
    template cudaError_t plain_energy_partials<T>(const Cx<T>::type *, int, double *, cudaStream_t); \
    template cudaError_t plain_spectrum<T>(const Cx<T>::type *, int, int, double *, double *,     \
                                           cudaStream_t);                                         \
    template cudaError_t plain_helicity<T>(const Cx<T>::type *, int, int, double *, double *,     \
                                           cudaStream_t);
NSK_INST(float)
NSK_INST(double)
#undef NSK_INST

}  // namespace nsk
