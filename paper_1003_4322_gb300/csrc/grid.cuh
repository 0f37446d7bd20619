// grid.cuh -- the grid and box of a plain-form run and the per-mode index
// helpers shared by its kernels: N_x x N_y x N_z points on the box of sides
// 2 pi l_i (the (2 pi)^3 cube of Sec. 2, or a domain of aspect ratio other
// than one, Sec. 5), half layout [c][N_x][N_y][N_z/2+1], index m along axis i
// standing for the wavenumber m / l_i, the 2/3 rule per axis in grid indices.
#pragma once
#include <cuda_runtime.h>
#include <stdlib.h>

namespace nsk {

struct Grid {
    int nx = 0, ny = 0, nz = 0;
    double lx = 1.0, ly = 1.0, lz = 1.0;
    double ilx = 1.0, ily = 1.0, ilz = 1.0;   // 1 / l_i (1 on the unit box)
    long D = 0;                  // lcm(N_x, N_y, N_z): the ellipsoid masks in integers
    long qx = 0, qy = 0, qz = 0; // D / N_i
    int unit = 1;                // every l_i = 1: integer wavenumbers, factor table by |k|^2
    int m32 = 1;                 // half-layout positions fit 32 bits (index decoding in 32 bits)
    int cube = 1;                // unit and N_x = N_y = N_z
    double lmax = 1.0;           // 1 / k_min with k_min = 1 / max l_i: shell K = [|k| lmax]
    __host__ __device__ long nzh() const { return nz / 2 + 1; }
    __host__ __device__ long M() const { return (long)nx * ny * (nz / 2 + 1); }
    __host__ __device__ long V() const { return (long)nx * ny * nz; }
};

__device__ __forceinline__ int wavenum(int i, int n) { return 2 * i < n ? i : i - n; }

// Signed grid indices (mx, my, mz) of half-layout position m.
struct Idx {
    int x, y, z;
};
__device__ __forceinline__ Idx mode_at(long m, const Grid &g) {
    Idx r;
    if (g.m32) {   // 32-bit divisions (the 64-bit ones are emulated)
        const unsigned um = (unsigned)m, nh = (unsigned)(g.nz / 2 + 1), ny = (unsigned)g.ny;
        const unsigned q = um / nh;
        r.z = (int)(um - q * nh);
        const unsigned x = q / ny;
        r.y = wavenum((int)(q - x * ny), g.ny);
        r.x = wavenum((int)x, g.nx);
        return r;
    }
    const long nh = g.nzh();
    r.z = (int)(m % nh);
    r.y = wavenum((int)((m / nh) % g.ny), g.ny);
    r.x = wavenum((int)(m / (nh * g.ny)), g.nx);
    return r;
}

// Wavenumber of index m along an axis of side 2 pi l, as the definition
// m / l (the shell decisions of the spectra use this form).
__device__ __forceinline__ double kof(int m, double l) { return (double)m / l; }

// The same from the reciprocal il = 1 / l: one multiplication instead of an
// FP64 division on the step's hot kernels; exact on the unit box, within one
// rounding of m / l otherwise.
__device__ __forceinline__ double kmul(int m, double il) { return (double)m * il; }

// Dealiasing mask Pi in grid indices: 3 |m_i| < N_i on every axis, and the
// ellipsoid sum_i (3 m_i / N_i)^2 < 1 (dealias 1); dealias 2: 2 |m_i| < N_i
// and the ellipsoid < 2.  The ellipsoid is tested exactly over D = lcm(N_i).
// On the cube these are 3 max|k_i| < N, 9 |k|^2 < N^2 and 9 |k|^2 < 2 N^2.
__host__ __device__ __forceinline__ bool kept(const Idx &k, const Grid &g, int dealias) {
    const long ax = abs(k.x), ay = abs(k.y), az = abs(k.z);
    const long sx = ax * g.qx, sy = ay * g.qy, sz = az * g.qz;
    const long s = sx * sx + sy * sy + sz * sz;
    if (dealias == 2) return 2 * ax < g.nx && 2 * ay < g.ny && 2 * az < g.nz && 9 * s < 2 * g.D * g.D;
    if (3 * ax >= g.nx || 3 * ay >= g.ny || 3 * az >= g.nz) return false;
    if (dealias == 1 && 9 * s >= g.D * g.D) return false;
    return true;
}

// The rectangle |m_x| <= kx, |m_y| <= ky, m_z <= kz of the half layout that
// holds every mode a run's rule keeps (on = 0: the whole layout).  Its size
// stays below 2^31 for every supported grid.
struct Rect {
    int on, kx, ky, kz;
};
__host__ __device__ __forceinline__ long rect_size(const Rect &r, const Grid &g) {
    return r.on ? (long)(2 * r.kx + 1) * (2 * r.ky + 1) * (r.kz + 1) : g.M();
}
// Half-layout position of entry i of the rectangle (i itself when off).
__device__ __forceinline__ long rect_at(long i, const Rect &r, const Grid &g) {
    if (!r.on) return i;
    const unsigned mz = r.kz + 1, my = 2 * r.ky + 1, ui = (unsigned)i;
    const unsigned z = ui % mz, t = ui / mz, iy = t % my, ix = t / my;
    const long x = ix <= (unsigned)r.kx ? (long)ix : (long)ix - (2 * r.kx + 1) + g.nx;
    const long y = iy <= (unsigned)r.ky ? (long)iy : (long)iy - my + g.ny;
    return (x * g.ny + y) * g.nzh() + z;
}
__device__ __forceinline__ bool in_rect(const Idx &q, const Rect &r) {
    return !r.on || (abs(q.x) <= r.kx && abs(q.y) <= r.ky && q.z <= r.kz);
}

}  // namespace nsk
