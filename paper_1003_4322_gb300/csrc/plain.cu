// plain.cu -- the unfused, unpruned ("plain") form of the solver's pointwise
// steps on full half-layout arrays [3][N_x][N_y][N_z/2+1] (Sec. 2, Eqs. 1-2):
// the vorticity i k x a, the cross product u x w on the grid, and the
// projected, dealiased, forced integrating-factor RK2 update; plus the
// deterministic FP64 reductions for energy, enstrophy and the shell spectrum
// (the global quantities and spectra of Sec. 3).  Grids of N_x x N_y x N_z
// points on boxes of sides 2 pi l_i (the domains of aspect ratio other than
// one of Sec. 5) go through the same kernels: index m along axis i is the
// wavenumber m / l_i, and the 2/3 rule holds per axis in grid indices.
#include <math.h>

#include "ns_internal.h"
#include "plain.h"
#include "reduce.cuh"

namespace nsk {

static long gcd_l(long a, long b) { return b ? gcd_l(b, a % b) : a; }

Grid make_grid(int nx, int ny, int nz, double lx, double ly, double lz) {
    Grid g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.lx = lx;
    g.ly = ly;
    g.lz = lz;
    g.ilx = 1.0 / lx;
    g.ily = 1.0 / ly;
    g.ilz = 1.0 / lz;
    long D = nx;
    D = D / gcd_l(D, ny) * ny;
    D = D / gcd_l(D, nz) * nz;
    g.D = D;
    g.qx = D / nx;
    g.qy = D / ny;
    g.qz = D / nz;
    g.unit = lx == 1.0 && ly == 1.0 && lz == 1.0;
    g.m32 = g.M() < (1L << 31);
    g.cube = g.unit && nx == ny && ny == nz;
    const double lm = fmax(lx, fmax(ly, lz));
    g.lmax = 1.0 / (1.0 / lm);   // as the shell width 1 / k_min, k_min = 1 / max l
    return g;
}

int grid_nbins(const Grid &g) {
    if (g.cube) return (int)ceil(sqrt(3.0) * g.nx / 2.0) + 1;
    const double cx = g.nx / 2 / g.lx, cy = g.ny / 2 / g.ly, cz = g.nz / 2 / g.lz;
    const double kmin = 1.0 / fmax(g.lx, fmax(g.ly, g.lz));
    return (int)ceil(sqrt(cx * cx + cy * cy + cz * cz) / kmin) + 1;
}

long grid_max_k2(const Grid &g) {
    const long hx = g.nx / 2, hy = g.ny / 2, hz = g.nz / 2;
    return hx * hx + hy * hy + hz * hz;
}

// Wavevector of a mode in precision T and |k|^2.  On the unit box (UNIT) the
// wavenumbers are the integer indices and |k|^2 an integer (the index of the
// factor table); elsewhere k = m / l is formed from the reciprocals in FP64.
template <typename T, bool UNIT> struct Wave {
    T kx, ky, kz;
    double k2;     // |k|^2
    long i2;       // |k|^2 as an integer (UNIT only)
    int px, py, pz;   // array positions of the mode along x, y, z
    __device__ __forceinline__ Wave(const Idx &q, const Grid &g) {
        px = q.x < 0 ? q.x + g.nx : q.x;
        py = q.y < 0 ? q.y + g.ny : q.y;
        pz = q.z;
        if constexpr (UNIT) {
            i2 = (long)q.x * q.x + (long)q.y * q.y + (long)q.z * q.z;
            kx = (T)q.x;
            ky = (T)q.y;
            kz = (T)q.z;
            k2 = (double)i2;
        } else {
            const double dx = kmul(q.x, g.ilx), dy = kmul(q.y, g.ily), dz = kmul(q.z, g.ilz);
            i2 = 0;
            kx = (T)dx;
            ky = (T)dy;
            kz = (T)dz;
            k2 = dx * dx + dy * dy + dz * dz;
        }
    }
    // exp(-c |k|^2) from the run's table: by integer |k|^2 on the unit box;
    // elsewhere the product of the per-axis factors exp(-c k_x^2) exp(-c k_y^2)
    // exp(-c k_z^2), tabulated by array position ([N_x | N_y | N_z/2+1]).
    __device__ __forceinline__ T factor(const T *etab, const Grid &g) const {
        if constexpr (UNIT) return etab[i2];
        else return etab[px] * etab[g.nx + py] * etab[g.nx + g.ny + pz];
    }
};

// ---------------------------------------------------------------- curl

// Bits of the six parts of a complex vector OR-ed together: zero exactly when
// every part is +0 (an integer test, which keeps the FP64 pipe free).
__device__ __forceinline__ unsigned long long cbits(double2 a, double2 b, double2 c) {
    return (unsigned long long)(__double_as_longlong(a.x) | __double_as_longlong(a.y) |
                                __double_as_longlong(b.x) | __double_as_longlong(b.y) |
                                __double_as_longlong(c.x) | __double_as_longlong(c.y));
}
__device__ __forceinline__ unsigned long long cbits(float2 a, float2 b, float2 c) {
    return (unsigned long long)(__float_as_uint(a.x) | __float_as_uint(a.y) | __float_as_uint(b.x) |
                                __float_as_uint(b.y) | __float_as_uint(c.x) | __float_as_uint(c.y));
}

// The state is zero outside the kept set (every dealiasing rule); there the
// curl is written as zeros without arithmetic, which on GB300's slow FP64
// pipe is most of this kernel's time (about 70 % of the half-layout modes lie
// outside the 2/3 cube).  With the rectangle on, only its modes are read and
// written (the transforms that follow read no others).
template <typename T, bool UNIT>
__global__ void k_curl(const typename Cx<T>::type *__restrict__ a, typename Cx<T>::type *__restrict__ w,
                       Grid g, long M, Rect rc) {
    typedef typename Cx<T>::type C;
    const long cnt = rect_size(rc, g);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < cnt; i += (long)gridDim.x * blockDim.x) {
        const long m = rect_at(i, rc, g);
        const C ax = a[m], ay = a[M + m], az = a[2 * M + m];
        if (cbits(ax, ay, az) == 0) {
            w[m] = w[M + m] = w[2 * M + m] = czero<C>();
            continue;
        }
        const Wave<T, UNIT> k(mode_at(m, g), g);
        const T kx = k.kx, ky = k.ky, kzz = k.kz;
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

// ABC forcing coefficients at signed grid index k (closed form of
// f = F (sin kf z + cos kf y, sin kf x + cos kf z, sin kf y + cos kf x));
// kf sits at grid index kf l_i along axis i (mfx, mfy, mfz).
template <typename C, typename T>
__device__ __forceinline__ void abc_forcing(const Idx &k, const UpdateArgs &ua, T F, C &fx, C &fy, C &fz) {
    const T h = F * (T)0.5;
    if (ua.force_k <= 0) return;
    if (k.x == 0 && k.y == 0 && k.z == ua.mfz) {   // e^{i kf z}: sin -> -i/2, cos -> 1/2
        fx = cadd(fx, mkc((T)0, -h));
        fy = cadd(fy, mkc(h, (T)0));
    }
    if (k.x == 0 && k.z == 0 && (k.y == ua.mfy || k.y == -ua.mfy)) {
        fx = cadd(fx, mkc(h, (T)0));
        fz = cadd(fz, mkc((T)0, k.y > 0 ? -h : h));
    }
    if (k.y == 0 && k.z == 0 && (k.x == ua.mfx || k.x == -ua.mfx)) {
        fy = cadd(fy, mkc((T)0, k.x > 0 ? -h : h));
        fz = cadd(fz, mkc(h, (T)0));
    }
}


// Stage 1: a1 = E (a + dt N);  stage 2: a = E a / 2 + (a1 + dt N) / 2, with
// N = P Pi (nl / N^3) + f_hat; every mode outside Pi (and k = 0) set to 0.
// The projection is applied to nl itself (it is linear) and dt / N^3 joins the
// stage's weights, so that a kept mode costs about 40 FP64 instructions
// instead of 60; the forcing enters as dt f_hat at the forced modes only.
template <typename T, bool UNIT>
__global__ void k_update(typename Cx<T>::type *__restrict__ a, typename Cx<T>::type *__restrict__ a1,
                         const typename Cx<T>::type *__restrict__ nl, const T *__restrict__ etab,
                         Grid g, long M, UpdateArgs ua, Rect rc) {
    typedef typename Cx<T>::type C;
    const double vol = (double)g.nx * g.ny * g.nz;
    const T gdt = (T)(ua.dt / vol), dt = (T)ua.dt, F = (T)ua.force_amp;
    const T rn = (T)(2.0 * ua.rot * vol);   // the Coriolis factor in the units of nl
    const long cnt = rect_size(rc, g);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < cnt; i += (long)gridDim.x * blockDim.x) {
        const long m = rect_at(i, rc, g);
        const Idx q = mode_at(m, g);
        const Wave<T, UNIT> k(q, g);
        C o0 = czero<C>(), o1 = czero<C>(), o2 = czero<C>();
        if (kept(q, g, ua.dealias) && k.k2 > 0) {
            // v = N^3 (nl / N^3 + Coriolis), in the units of nl
            C vx = nl[m], vy = nl[M + m], vz = nl[2 * M + m];
            if (ua.rot != 0.0) {   // Coriolis -2 rot z x u of the stage's state, before P
                const C *cur = ua.stage == 1 ? a : a1;
                vx = cadd(vx, cscale(cur[M + m], rn));
                vy = csub(vy, cscale(cur[m], rn));
            }
            const T fkx = k.kx, fky = k.ky, fkz = k.kz, ik2 = (T)1 / (T)k.k2;
            const C s = cscale(cadd(cadd(cscale(vx, fkx), cscale(vy, fky)), cscale(vz, fkz)), ik2);
            vx = mkc(vx.x - fkx * s.x, vx.y - fkx * s.y);   // P(k) v = v - k (k.v) / k^2
            vy = mkc(vy.x - fky * s.x, vy.y - fky * s.y);
            vz = mkc(vz.x - fkz * s.x, vz.y - fkz * s.y);
            const T e = k.factor(etab, g);
            const C f0 = a[m], f1 = a[M + m], f2 = a[2 * M + m];
            if (ua.stage == 1) {   // E (a + (dt/N^3) v + dt f)
                C t0 = mkc(f0.x + gdt * vx.x, f0.y + gdt * vx.y);
                C t1 = mkc(f1.x + gdt * vy.x, f1.y + gdt * vy.y);
                C t2 = mkc(f2.x + gdt * vz.x, f2.y + gdt * vz.y);
                abc_forcing(q, ua, F * dt, t0, t1, t2);
                o0 = cscale(t0, e);
                o1 = cscale(t1, e);
                o2 = cscale(t2, e);
            } else {               // (E/2) a + a1 / 2 + (dt/N^3 / 2) v + (dt / 2) f
                const T he = (T)0.5 * e, h = (T)0.5, hg = (T)0.5 * gdt;
                const C g0 = a1[m], g1 = a1[M + m], g2 = a1[2 * M + m];
                o0 = mkc(he * f0.x + (h * g0.x + hg * vx.x), he * f0.y + (h * g0.y + hg * vx.y));
                o1 = mkc(he * f1.x + (h * g1.x + hg * vy.x), he * f1.y + (h * g1.y + hg * vy.y));
                o2 = mkc(he * f2.x + (h * g2.x + hg * vz.x), he * f2.y + (h * g2.y + hg * vz.y));
                abc_forcing(q, ua, F * dt * h, o0, o1, o2);
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
template <typename T, bool UNIT>
__global__ void k_update_b(typename Cx<T>::type *__restrict__ b, typename Cx<T>::type *__restrict__ b1,
                           const typename Cx<T>::type *__restrict__ nb, const T *__restrict__ etab,
                           Grid g, long M, int stage, double dt_, int dealias, Rect rc) {
    typedef typename Cx<T>::type C;
    const T inv = (T)(1.0 / ((double)g.nx * g.ny * g.nz));
    const T dt = (T)dt_;
    const long cnt = rect_size(rc, g);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < cnt; i += (long)gridDim.x * blockDim.x) {
        const long m = rect_at(i, rc, g);
        const Idx q = mode_at(m, g);
        const Wave<T, UNIT> k(q, g);
        C o0 = czero<C>(), o1 = czero<C>(), o2 = czero<C>();
        if (kept(q, g, dealias)) {
            const C vx = cscale(nb[m], inv), vy = cscale(nb[M + m], inv), vz = cscale(nb[2 * M + m], inv);
            const T fkx = k.kx, fky = k.ky, fkz = k.kz;
            // i k x v
            const C nx = cmul_i<1>(csub(cscale(vz, fky), cscale(vy, fkz)));
            const C ny = cmul_i<1>(csub(cscale(vx, fkz), cscale(vz, fkx)));
            const C nz = cmul_i<1>(csub(cscale(vy, fkx), cscale(vx, fky)));
            const T e = k.factor(etab, g);
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

// Phase-shift dealiasing: dst = src exp(i k.D), D half a grid spacing along
// every axis (k.D = pi sum_i m_i / N_i), the coefficients of the field on the
// shifted grid (three components).  The factor is the product of the per-axis
// factors exp(i pi m_i / N_i), tabulated in FP64 by array position
// ([N_x | N_y | N_z/2+1], rounded once to T).
template <typename T>
__device__ __forceinline__ typename Cx<T>::type shift_factor(long m, const Grid &g,
                                                             const typename Cx<T>::type *__restrict__ ph) {
    const Idx q = mode_at(m, g);
    const int px = q.x < 0 ? q.x + g.nx : q.x, py = q.y < 0 ? q.y + g.ny : q.y;
    return cmul(cmul(ph[px], ph[g.nx + py]), ph[g.nx + g.ny + q.z]);
}

template <typename T>
__global__ void k_phase(const typename Cx<T>::type *__restrict__ src, typename Cx<T>::type *__restrict__ dst,
                        const typename Cx<T>::type *__restrict__ ph, Grid g, long M) {
    typedef typename Cx<T>::type C;
    for (long m = blockIdx.x * (long)blockDim.x + threadIdx.x; m < M; m += (long)gridDim.x * blockDim.x) {
        const C f = shift_factor<T>(m, g, ph);
#pragma unroll
        for (int d = 0; d < 3; d++) dst[d * M + m] = cmul(src[d * M + m], f);
    }
}

// acc = (acc + sh exp(-i k.D)) / 2: the product on the grid and, shifted
// back, on the shifted grid, averaged (three components).
template <typename T>
__global__ void k_phase_avg(typename Cx<T>::type *__restrict__ acc, const typename Cx<T>::type *__restrict__ sh,
                            const typename Cx<T>::type *__restrict__ ph, Grid g, long M) {
    typedef typename Cx<T>::type C;
    for (long m = blockIdx.x * (long)blockDim.x + threadIdx.x; m < M; m += (long)gridDim.x * blockDim.x) {
        const C f = cconj(shift_factor<T>(m, g, ph));
#pragma unroll
        for (int d = 0; d < 3; d++)
            acc[d * M + m] = cscale(cadd(acc[d * M + m], cmul(sh[d * M + m], f)), (T)0.5);
    }
}

// ---------------------------------------------------------------- reductions

// Per-block partial energy and enstrophy of a half-layout state.  Block b
// owns the contiguous chunk [b*chunk, (b+1)*chunk) of modes.
template <typename T, bool UNIT>
__global__ void __launch_bounds__(256)
k_energy_partials(const typename Cx<T>::type *__restrict__ a, Grid g, long M, long chunk, double *part,
                  Rect rc) {
    __shared__ double sh[512];
    double e = 0.0, om = 0.0;
    const long beg = blockIdx.x * chunk, end = min(M, beg + chunk);
    for (long m = beg + threadIdx.x; m < end; m += blockDim.x) {
        const Idx q = mode_at(m, g);
        if (!in_rect(q, rc)) continue;   // zero there: the sums, in the same order, are unchanged
        const Wave<double, UNIT> k(q, g);
        const double w = (q.z == 0 || 2 * q.z == g.nz) ? 0.5 : 1.0;   // 1/2 * multiplicity
        double a2 = 0.0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const double re = (double)a[c * M + m].x, im = (double)a[c * M + m].y;
            a2 += re * re + im * im;
        }
        e += w * a2;
        om += w * a2 * k.k2;
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

// Per-mode sums for grids other than the cube: signed indices and their
// wavenumbers -> |a|^2 summed over components, or the helicity density.
template <typename T> struct GridAcc {
    const typename Cx<T>::type *a;
    Grid g;
    __device__ double operator()(int mx, int my, int mz, double, double, double) const {
        const long m = ((long)((mx + g.nx) % g.nx) * g.ny + (my + g.ny) % g.ny) * g.nzh() + mz;
        const long M = g.M();
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const double re = (double)a[c * M + m].x, im = (double)a[c * M + m].y;
            s += re * re + im * im;
        }
        return s;
    }
};

template <typename T> struct GridHelAcc {
    const typename Cx<T>::type *a;
    Grid g;
    __device__ double operator()(int mx, int my, int mz, double kx, double ky, double kz) const {
        const long m = ((long)((mx + g.nx) % g.nx) * g.ny + (my + g.ny) % g.ny) * g.nzh() + mz;
        const long M = g.M();
        return helicity_density(kx, ky, kz, a[m].x, a[m].y, a[M + m].x, a[M + m].y, a[2 * M + m].x,
                                a[2 * M + m].y);
    }
};

// Shell spectrum on any grid and box: block K sums the modes whose shell
// round-half-up(|k| lmax) is K.  Threads take the (m_x, m_y) pairs that can
// reach the shell; for each, every m_z of a slightly widened interval is
// tested with the shell formula itself, in FP64 with each operation rounded
// as written (no contraction), so that the binning is the definition's.
// Fixed per-thread order and a fixed tree: deterministic.
template <class Acc>
__global__ void __launch_bounds__(256)
k_grid_spectrum(Acc acc, Grid g, int nbins, double *spec, double *aux) {
    __shared__ double sh[512];
    const int K = blockIdx.x, part = blockIdx.y;   // pairs part, part + kShellParts, ... (blocks)
    if (K >= nbins) return;
    const double hi = (K + 0.5) / g.lmax, lo = (K - 0.5) / g.lmax;
    const int bx = (int)(hi * g.lx) + 1, by = (int)(hi * g.ly) + 1;
    const int x0 = max(-bx, -g.nx / 2), x1 = min(bx, g.nx / 2 - 1);
    const int y0 = max(-by, -g.ny / 2), y1 = min(by, g.ny / 2 - 1);
    const long sy = y1 - y0 + 1, pairs = (long)(x1 - x0 + 1) * sy;
    const double hi2 = hi * hi * (1.0 + 1e-9) + 1e-12;
    double e = 0.0, om = 0.0;
    for (long p = (long)part * blockDim.x + threadIdx.x; p < pairs; p += (long)blockDim.x * gridDim.y) {
        const int mx = x0 + (int)(p / sy), my = y0 + (int)(p % sy);
        const double kx = kof(mx, g.lx), ky = kof(my, g.ly);
        const double r2 = __dadd_rn(__dmul_rn(kx, kx), __dmul_rn(ky, ky));
        if (r2 > hi2) continue;
        const double zlo = lo > 0.0 && lo * lo > r2 ? sqrt(lo * lo - r2) : 0.0;
        const double zhi = sqrt(fmax(0.0, hi2 - r2));
        const int z0 = max(0, (int)floor(zlo * g.lz) - 1);
        const int z1 = min(g.nz / 2, (int)ceil(zhi * g.lz) + 1);
        for (int mz = z0; mz <= z1; mz++) {
            const double kz = kof(mz, g.lz);
            const double k2 = __dadd_rn(r2, __dmul_rn(kz, kz));
            if ((long)floor(__dadd_rn(__dmul_rn(__dsqrt_rn(k2), g.lmax), 0.5)) != K) continue;
            const double w = (mz == 0 || 2 * mz == g.nz) ? 0.5 : 1.0;
            const double de = w * acc(mx, my, mz, kx, ky, kz);
            e += de;
            om += de * k2;
        }
    }
    block_sum2(e, om, sh);
    if (threadIdx.x == 0) {
        spec[nbins + K * kShellParts + part] = e;
        aux[nbins + K * kShellParts + part] = om;
    }
}

// ---------------------------------------------------------------- launchers

static unsigned grid_for(long work, int threads) {
    long b = (work + threads - 1) / threads;
    if (b > 152L * 32) b = 152L * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

template <typename T>
cudaError_t plain_curl(const typename Cx<T>::type *a, typename Cx<T>::type *w, const Grid &g, const Rect &rc,
                       cudaStream_t s) {
    const long M = g.M(), cnt = rect_size(rc, g);
    if (cnt > 0x7fffffffL) return cudaErrorInvalidValue;
    if (g.unit) k_curl<T, true><<<grid_for(cnt, 256), 256, 0, s>>>(a, w, g, M, rc);
    else k_curl<T, false><<<grid_for(cnt, 256), 256, 0, s>>>(a, w, g, M, rc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_cross(T *u, const T *w, const Grid &g, cudaStream_t s) {
    const long V = g.V();
    k_cross<T><<<grid_for(V, 256), 256, 0, s>>>(u, w, V);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_cross_mhd(T *f, const Grid &g, cudaStream_t s) {
    const long V = g.V();
    k_cross_mhd<T><<<grid_for(V, 256), 256, 0, s>>>(f, V);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_update_b(typename Cx<T>::type *b, typename Cx<T>::type *b1,
                           const typename Cx<T>::type *nb, const T *etab, const Grid &g, int stage,
                           double dt, int dealias, const Rect &rc, cudaStream_t s) {
    const long M = g.M(), cnt = rect_size(rc, g);
    if (cnt > 0x7fffffffL) return cudaErrorInvalidValue;
    if (g.unit)
        k_update_b<T, true><<<grid_for(cnt, 256), 256, 0, s>>>(b, b1, nb, etab, g, M, stage, dt, dealias, rc);
    else
        k_update_b<T, false><<<grid_for(cnt, 256), 256, 0, s>>>(b, b1, nb, etab, g, M, stage, dt, dealias, rc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_phase(const typename Cx<T>::type *src, typename Cx<T>::type *dst,
                        const typename Cx<T>::type *ph, const Grid &g, cudaStream_t s) {
    const long M = g.M();
    k_phase<T><<<grid_for(M, 256), 256, 0, s>>>(src, dst, ph, g, M);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_phase_avg(typename Cx<T>::type *acc, const typename Cx<T>::type *sh,
                            const typename Cx<T>::type *ph, const Grid &g, cudaStream_t s) {
    const long M = g.M();
    k_phase_avg<T><<<grid_for(M, 256), 256, 0, s>>>(acc, sh, ph, g, M);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_update(typename Cx<T>::type *a, typename Cx<T>::type *a1,
                         const typename Cx<T>::type *nl, const T *etab, const Grid &g,
                         const UpdateArgs &ua, const Rect &rc, cudaStream_t s) {
    const long M = g.M(), cnt = rect_size(rc, g);
    if (cnt > 0x7fffffffL) return cudaErrorInvalidValue;
    if (g.unit) k_update<T, true><<<grid_for(cnt, 256), 256, 0, s>>>(a, a1, nl, etab, g, M, ua, rc);
    else k_update<T, false><<<grid_for(cnt, 256), 256, 0, s>>>(a, a1, nl, etab, g, M, ua, rc);
    return cudaGetLastError();
}

int energy_nparts(long M) {
    long np = (M + 4095) / 4096;
    if (np > 1024) np = 1024;
    return (int)(np < 1 ? 1 : np);
}

template <typename T>
cudaError_t plain_energy_partials(const typename Cx<T>::type *a, const Grid &g, double *part, const Rect &rc,
                                  cudaStream_t s) {
    const long M = g.M();
    const int np = energy_nparts(M);
    const long chunk = (M + np - 1) / np;
    if (g.unit) k_energy_partials<T, true><<<np, 256, 0, s>>>(a, g, M, chunk, part, rc);
    else k_energy_partials<T, false><<<np, 256, 0, s>>>(a, g, M, chunk, part, rc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t plain_spectrum(const typename Cx<T>::type *a, const Grid &g, int nbins, double *spec,
                           double *ens, cudaStream_t s) {
    if (g.cube)
        return shell_launch(k_shell_spectrum<HalfAcc<T>>, nbins, spec, ens, s, HalfAcc<T>{a, g.nx, g.M()}, g.nx,
                            nbins);
    return shell_launch(k_grid_spectrum<GridAcc<T>>, nbins, spec, ens, s, GridAcc<T>{a, g}, g, nbins);
}

template <typename T>
cudaError_t plain_helicity(const typename Cx<T>::type *a, const Grid &g, int nbins, double *spec,
                           double *aux, cudaStream_t s) {
    if (g.cube)
        return shell_launch(k_shell_spectrum<HalfHelAcc<T>>, nbins, spec, aux, s, HalfHelAcc<T>{a, g.nx, g.M()},
                            g.nx, nbins);
    return shell_launch(k_grid_spectrum<GridHelAcc<T>>, nbins, spec, aux, s, GridHelAcc<T>{a, g}, g, nbins);
}

cudaError_t energy_final(const double *part, int nparts, double *series, int cap,
                         unsigned long long *counter, int *flags, cudaStream_t s) {
    k_energy_final<<<1, 256, 0, s>>>(part, nparts, series, cap, counter, flags);
    return cudaGetLastError();
}

#define NSK_INST(T)                                                                                \
    template cudaError_t plain_curl<T>(const Cx<T>::type *, Cx<T>::type *, const Grid &, const Rect &,   \
                                       cudaStream_t);                                             \
    template cudaError_t plain_cross<T>(T *, const T *, const Grid &, cudaStream_t);              \
    template cudaError_t plain_cross_mhd<T>(T *, const Grid &, cudaStream_t);                     \
    template cudaError_t plain_phase<T>(const Cx<T>::type *, Cx<T>::type *, const Cx<T>::type *,  \
                                        const Grid &, cudaStream_t);                              \
    template cudaError_t plain_phase_avg<T>(Cx<T>::type *, const Cx<T>::type *, const Cx<T>::type *, \
                                            const Grid &, cudaStream_t);                          \
    template cudaError_t plain_update_b<T>(Cx<T>::type *, Cx<T>::type *, const Cx<T>::type *,     \
                                           const T *, const Grid &, int, double, int, const Rect &,  \
                                           cudaStream_t);                                         \
    template cudaError_t plain_update<T>(Cx<T>::type *, Cx<T>::type *, const Cx<T>::type *,       \
                                         const T *, const Grid &, const UpdateArgs &, const Rect &, \
                                         cudaStream_t);                                           \
    template cudaError_t plain_energy_partials<T>(const Cx<T>::type *, const Grid &, double *,    \
                                                  const Rect &, cudaStream_t);                    \
    template cudaError_t plain_spectrum<T>(const Cx<T>::type *, const Grid &, int, double *, double *, \
                                           cudaStream_t);                                         \
    template cudaError_t plain_helicity<T>(const Cx<T>::type *, const Grid &, int, double *, double *, \
                                           cudaStream_t);
NSK_INST(float)
NSK_INST(double)
#undef NSK_INST

}  // namespace nsk
