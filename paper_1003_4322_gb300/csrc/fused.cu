// fused.cu -- the fused, pruned FP32 form of the RK2 step (Sec. 2, Eqs. 1-2).
//
// Only the modes the 2/3 rule keeps (|kx|, |ky|, kz <= K, K = ceil(N/3) - 1)
// are ever stored or read, and the physical fields u and w never reach HBM.
// One RK2 stage is five transform passes and an update:
//
//   A  x inverse + curl:  S[c][ikx][iky][kz] (3 comps)  -> A[f][iky][x][kz] (6: u, w)
//   B  y inverse:         A[f][iky][x][kz]              -> B[f][y][x][kz]
//   C  z c2r, u x w, z r2c (shared memory only):  B (6 fields) -> B (3 fields, in place)
//   D  y forward:         B[f][y][x][kz]                -> D[f][x][iky][kz] (kept ky only)
//   E  x forward:         D[f][x][iky][kz]              -> N[c][ikx][iky][kz] (kept kx only)
//   update: 1/N^3, mask, projection P(k), ABC forcing, integrating-factor RK2
//           stage, and (stage 2) the FP64 energy / enstrophy partial sums.
//
// Every strided pass sees its columns flattened and contiguous, so a CTA tile
// is always ct consecutive complex values of one row (128 bytes for ct = 16).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <string>
#include <mutex>
#include <vector>

#include "fused.h"
#include "fused_k.cuh"
#include "fused_update.cuh"
#include "plain.h"
#include "fused_access.cuh"
#include "reduce.cuh"

namespace nsk {

bool fused_enabled() { return true; }

// One CTA: field f, ct consecutive columns; lanes run along the columns.
// IN_C: the input rows are compact (only kept wavenumbers stored), the
// others are read as zero.  OUT_C: only the kept output rows are stored.
// CURL: pass A, whose fields 3..5 are the vorticity i k x a of the input.
template <int E, int DIR, bool IN_C, bool OUT_C, bool CURL>
__global__ void __launch_bounds__(512)
k_fused_strided(FzPass ps, Plan pl, const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int n = pl.n;
    const int ct = blockDim.x / (n / E);
    const int c = threadIdx.x % ct, slot = threadIdx.x / ct;
    const FzColumn<IN_C, OUT_C, CURL> col(ps, n, ct, c);
    auto gl = [&](int e) -> float2 { return col.load(ps, e); };
    auto gs = [&](int e, float2 v) { col.store(ps, e, v); };
    // tile rows padded by one element: with 8 or 16 columns, the rows a warp
    // touches in any Stockham stage cover the banks with no extra wavefront
    const int rs = ct + 1;
    auto sl = [&](int e) -> float2 { return sm[e * rs + c]; };
    auto ss = [&](int e, float2 v) { sm[e * rs + c] = v; };
    fft_line<E, DIR, false, false, false>(pl, slot, tw, n, gl, sl, ss, gs);
}

// Line stride (complex elements) of a shared-memory line in pass C: room for
// n values plus the skew of one element per 16, rounded to 8 (mod 16) so that
// the lines a warp touches fall in alternate halves of the banks.
__host__ __device__ inline int fz_line_stride(int n) {
    int ls = n + (n >> 4) + 1;
    while (ls % 16 != 8) ls++;
    return ls;
}

// Pass C.  One CTA holds L (y, x) lines, each with the six fields u, w.  Per
// field: c2r along z through one complex FFT of length n = N/2 (even/odd
// packing), which leaves the N real samples in shared memory; then u x w at
// every point; then r2c of the three products and the kept kz < Mz written
// back over fields 0..2 of the same lines.
template <int E>
__global__ void __launch_bounds__(256)
k_fused_z(float2 *buf, long fs, int N, int Mz, long nlines, int L, long brun, Plan pl,
          const float2 *__restrict__ tw) {
    buf += blockIdx.y * brun;   // run of the group
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int n = N / 2, Tn = n / E;
    const int g = threadIdx.x / Tn, slot = threadIdx.x % Tn;
    const int l = g / 6, f = g % 6;
    const long line = (long)blockIdx.x * L + l;
    const bool valid = line < nlines;
    const int LS = fz_line_stride(n);
    float2 *ls = sm + (long)g * LS;
    auto sl = [&](int e) -> float2 { return ls[e + (e >> 4)]; };
    auto ss = [&](int e, float2 v) { ls[e + (e >> 4)] = v; };

    // c2r packing: Z[k] = (X[k] + conj X[n-k]) + i W^{-k} (X[k] - conj X[n-k]),
    // with X[k] = 0 for k >= Mz and the real parts of X[0], X[n].
    // The n/Tn = E iterations are unrolled so that all 2E loads of a thread
    // are in flight together.
    const float2 *src = buf + f * fs + line * Mz;
    float2 xk[E], xm[E];
#pragma unroll
    for (int j = 0; j < E; j++) {
        const int k = slot + j * Tn;
        xk[j] = (valid && k < Mz) ? src[k] : make_float2(0.f, 0.f);
        xm[j] = (valid && n - k < Mz) ? src[n - k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < E; j++) {
        const int k = slot + j * Tn;
        float2 a0 = xk[j], am = xm[j];
        if (k == 0) {
            a0.y = 0.f;
            am.y = 0.f;
        }
        const float2 xc = cconj(am);
        const float2 a = cadd(a0, xc);
        const float2 wb = cmulc(csub(a0, xc), ldg_c(tw + k));
        ss(k, cadd(a, cmul_i<1>(wb)));
    }
    __syncthreads();
    fft_line<E, +1, true, true, false>(pl, slot, tw, N, sl, sl, ss, ss);

    // u x w at the 2n points of each line (complex element m holds points 2m, 2m+1)
    for (int idx = threadIdx.x; idx < L * n; idx += blockDim.x) {
        const int l2 = idx / n, m = idx % n;
        const int o = m + (m >> 4);
        float2 *base = sm + (long)(6 * l2) * LS + o;
        const float2 ux = base[0], uy = base[LS], uz = base[2 * LS];
        const float2 wx = base[3 * LS], wy = base[4 * LS], wz = base[5 * LS];
        base[0] = make_float2(uy.x * wz.x - uz.x * wy.x, uy.y * wz.y - uz.y * wy.y);
        base[LS] = make_float2(uz.x * wx.x - ux.x * wz.x, uz.y * wx.y - ux.y * wz.y);
        base[2 * LS] = make_float2(ux.x * wy.x - uy.x * wx.x, ux.y * wy.y - uy.y * wx.y);
    }
    __syncthreads();
    fft_line_masked<E, -1, true, true>(f < 3, pl, slot, tw, N, sl, sl, ss, ss);

    // r2c unpacking of the kept kz:
    // X[k] = (Z[k] + conj Z[n-k])/2 - i W^k (Z[k] - conj Z[n-k])/2
    if (f < 3 && valid) {
        float2 *dst = buf + f * fs + line * Mz;
        for (int k = slot; k < Mz; k += Tn) {
            const float2 zk = sl(k);
            const float2 zc = cconj(sl(k == 0 ? 0 : n - k));
            const float2 ev = cscale(cadd(zk, zc), 0.5f);
            const float2 od = cmul_i<-1>(cscale(csub(zk, zc), 0.5f));
            dst[k] = cadd(ev, cmul(od, ldg_c(tw + k)));
        }
    }
}

// Two modes per thread and iteration, every operand load issued before any
// arithmetic, so that enough bytes are in flight to stream HBM.  GRID: the
// state of a grid or box (fz_update_mode_grid).
template <bool GRID>
__global__ void __launch_bounds__(256)
k_fused_update(float2 *__restrict__ a, float2 *__restrict__ a1, const float2 *__restrict__ nl,
               const float *__restrict__ etab, const FzRunParams *__restrict__ rp, FzUpdate u,
               double *part) {
    __shared__ double sh[512];
    const long M = u.M;
    const int run = blockIdx.y;
    a += run * 3 * M;
    a1 += run * 3 * M;
    nl += run * 3 * M;
    etab += (long)run * u.nk2;
    const FzRunParams q = rp[run];
    const float inv = (float)(1.0 / ((double)u.n * u.n * u.n));
    const bool two = u.stage == 2;
    float2 *dst = two ? a : a1;
    DfAcc e_acc, o_acc;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long m0 = blockIdx.x * (long)blockDim.x + threadIdx.x; m0 < M; m0 += 2 * stride) {
        const long m1 = m0 + stride;
        const bool has1 = m1 < M;
        const float2 z = make_float2(0.f, 0.f);
        float2 v[2][3], b[2][3], c[2][3];
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const long m = i ? m1 : m0;
            const bool ok = i == 0 || has1;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                v[i][d] = ok ? nl[d * M + m] : z;
                b[i][d] = ok ? a[d * M + m] : z;
                c[i][d] = (ok && two) ? a1[d * M + m] : z;
            }
        }
#pragma unroll
        for (int i = 0; i < 2; i++) {
            if (i == 1 && !has1) break;
            const long m = i ? m1 : m0;
            FzMode r;
            if constexpr (GRID)
                r = fz_update_mode_grid(m, u, q, etab, v[i][0], v[i][1], v[i][2], b[i][0], b[i][1], b[i][2],
                                        c[i][0], c[i][1], c[i][2]);
            else
                r = fz_update_mode(m, u, q, etab, inv, v[i][0], v[i][1], v[i][2], b[i][0], b[i][1], b[i][2],
                                   c[i][0], c[i][1], c[i][2]);
            dst[m] = r.o0;
            dst[M + m] = r.o1;
            dst[2 * M + m] = r.o2;
            if (two) {
                if constexpr (GRID) fz_accumulate_grid(r, e_acc, o_acc);
                else fz_accumulate(r, e_acc, o_acc);
            }
        }
    }
    if (two) {
        double e = e_acc.value(), o = o_acc.value();
        block_sum2(e, o, sh);
        if (threadIdx.x == 0) {
            double *pp = part + 2 * ((long)run * u.nparts + blockIdx.x);
            pp[0] = e;
            pp[1] = o;
        }
    }
}

// One block per run: sum that run's partials in a fixed order, append
// (E, Omega) to its ring buffer at slot counter % cap, bump the counter, and
// raise bit 0 of *flags if E is not finite.
__global__ void __launch_bounds__(256)
k_fz_energy_final(const double *__restrict__ part, int nparts, double *series, int cap,
                  unsigned long long *counter, int *flags) {
    __shared__ double sh[512];
    const int run = blockIdx.x;
    const double *pp = part + 2L * run * nparts;
    double e = 0.0, om = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        e += pp[2 * i];
        om += pp[2 * i + 1];
    }
    block_sum2(e, om, sh);
    if (threadIdx.x == 0) {
        const unsigned long long c = counter[run];
        double *sr = series + 2L * run * cap;
        sr[2 * (c % cap)] = e;
        sr[2 * (c % cap) + 1] = om;
        counter[run] = c + 1;
        if (!isfinite(e)) atomicOr(flags, 1);
    }
}

// ---------------------------------------------------------------- state transfer

// The half layout [N_x][N_y][N_z/2+1] and the compact one of a group: the
// axis lengths, the kept |m| and compact rows along x and y, the kept kz,
// and the sphere of the spherical rule in integers (D = lcm N_i, q_i = D / N_i).
struct FzHalfGeom {
    int nx, ny, nz, K, Ky, Mx, My, Mz;
    long D, qx, qy, qz;
};
static FzHalfGeom half_geom(const FusedRun &f) {
    return FzHalfGeom{f.n, f.ny, f.nz, f.K, f.Ky, f.Mx, f.My, f.Mz, f.D, f.qx, f.qy, f.qz};
}

// cnt full kx planes starting at kx0 (FP64 half layout, plane = N_y (N_z/2+1)
// modes) -> compact rows; modes outside the sphere (dealias = 1) dropped.
__global__ void k_fz_load(const double2 *__restrict__ src, float2 *__restrict__ dst, int kx0, int cnt,
                          FzHalfGeom g, int dealias) {
    const int nh = g.nz / 2 + 1;
    const long total = (long)cnt * g.My * g.Mz;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int kz = (int)(i % g.Mz);
        const int iky = (int)((i / g.Mz) % g.My);
        const int p = (int)(i / ((long)g.Mz * g.My));
        const int fx = kx0 + p;
        const int ikx = fz_compact(fx, g.nx, g.K, g.Mx);
        if (ikx < 0) continue;
        const int ky = fz_compact_signed(iky, g.My, g.Ky);
        const int fy = ky >= 0 ? ky : ky + g.ny;
        const int kx = fz_full_signed(fx, g.nx);
        double2 v = src[(long)p * g.ny * nh + (long)fy * nh + kz];
        const long ax = kx * g.qx, ay = ky * g.qy, az = kz * g.qz;
        if (dealias == 1 && 9 * (ax * ax + ay * ay + az * az) >= g.D * g.D) v = make_double2(0.0, 0.0);
        dst[((long)ikx * g.My + iky) * g.Mz + kz] = make_float2((float)v.x, (float)v.y);
    }
}

NSK_DEV void fz_put(double2 *d, float2 v) { *d = make_double2((double)v.x, (double)v.y); }
NSK_DEV void fz_put(float2 *d, float2 v) { *d = v; }

// compact -> cnt full kx planes starting at kx0 (zeros outside the kept set),
// FP64 (state transfer) or FP32 (the input of the grid spectra)
template <typename D2>
__global__ void k_fz_store(const float2 *__restrict__ src, D2 *__restrict__ dst, int kx0, int cnt, FzHalfGeom g) {
    const int nh = g.nz / 2 + 1;
    const long total = (long)cnt * g.ny * nh;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int kz = (int)(i % nh);
        const int fy = (int)((i / nh) % g.ny);
        const int p = (int)(i / ((long)nh * g.ny));
        const int ikx = fz_compact(kx0 + p, g.nx, g.K, g.Mx);
        const int iky = fz_compact(fy, g.ny, g.Ky, g.My);
        float2 v = make_float2(0.f, 0.f);
        if (ikx >= 0 && iky >= 0 && kz < g.Mz) v = src[((long)ikx * g.My + iky) * g.Mz + kz];
        fz_put(dst + i, v);
    }
}

struct CompactAcc {
    const float2 *a;
    int K, Mx, Mz;
    long M;
    __device__ double operator()(int kx, int ky, int kz) const {
        if (kx > K || kx < -K || ky > K || ky < -K || kz >= Mz) return 0.0;
        const int ikx = kx >= 0 ? kx : kx + Mx, iky = ky >= 0 ? ky : ky + Mx;
        const long m = ((long)ikx * Mx + iky) * Mz + kz;
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const double re = (double)a[c * M + m].x, im = (double)a[c * M + m].y;
            s += re * re + im * im;
        }
        return s;
    }
};

struct CompactHelAcc {
    const float2 *a;
    int K, Mx, Mz;
    long M;
    __device__ double operator()(int kx, int ky, int kz) const {
        if (kx > K || kx < -K || ky > K || ky < -K || kz >= Mz) return 0.0;
        const int ikx = kx >= 0 ? kx : kx + Mx, iky = ky >= 0 ? ky : ky + Mx;
        const long m = ((long)ikx * Mx + iky) * Mz + kz;
        return helicity_density(kx, ky, kz, a[m].x, a[m].y, a[M + m].x, a[M + m].y, a[2 * M + m].x,
                                a[2 * M + m].y);
    }
};

// ---------------------------------------------------------------- host side

static unsigned grid_of(long work, int threads, long cap) {
    long b = (work + threads - 1) / threads;
    b = std::min(b, cap);
    return (unsigned)std::max(b, 1L);
}

template <int E, int DIR, bool IN_C, bool OUT_C, bool CURL>
static const void *strided_k() {
    return (const void *)k_fused_strided<E, DIR, IN_C, OUT_C, CURL>;
}

template <int DIR, bool IN_C, bool OUT_C, bool CURL>
static const void *strided_for(int E) {
    switch (E) {
    case 4: return strided_k<4, DIR, IN_C, OUT_C, CURL>();
    case 6: return strided_k<6, DIR, IN_C, OUT_C, CURL>();
    case 8: return strided_k<8, DIR, IN_C, OUT_C, CURL>();
    case 9: return strided_k<9, DIR, IN_C, OUT_C, CURL>();
    case 12: return strided_k<12, DIR, IN_C, OUT_C, CURL>();
    case 16: return strided_k<16, DIR, IN_C, OUT_C, CURL>();
    }
    return nullptr;
}

static const void *z_for(int E) {
    switch (E) {
    case 4: return (const void *)k_fused_z<4>;
    case 6: return (const void *)k_fused_z<6>;
    case 8: return (const void *)k_fused_z<8>;
    case 9: return (const void *)k_fused_z<9>;
    case 12: return (const void *)k_fused_z<12>;
    case 16: return (const void *)k_fused_z<16>;
    }
    return nullptr;
}

// Compile-time-length strided kernel of a pass mode (0: A, 1: B, 2: D/E).
static bool fzs_lookup(int which, int N, int E, int CT, FzsKernel *o) {
    return which == 0 ? fzs_lookup_A(N, E, CT, o)
         : which == 1 ? fzs_lookup_B(N, E, CT, o)
                      : fzs_lookup_DE(N, E, CT, o);
}

// Constant-geometry kernel of pass 0..3 (A, B, D, E) on the grid nx x ny x nz.
static bool fzk_lookup(int pass, int nx, int ny, int nz, int E, int CT, FzsKernel *o) {
    switch (pass) {
    case 0: return fzk_lookup_A(nx, ny, nz, E, CT, o);
    case 1: return fzk_lookup_B(nx, ny, nz, E, CT, o);
    case 2: return fzk_lookup_D(nx, ny, nz, E, CT, o);
    case 3: return fzk_lookup_E(nx, ny, nz, E, CT, o);
    }
    return false;
}

// The same for a run: the kernels of a cube keep the unit box, so a cube on
// another box has none.
static bool fzk_for(const FusedRun &f, int pass, int E, int CT, FzsKernel *o) {
    if (!f.cube && f.n == f.ny && f.n == f.nz) return false;
    return fzk_lookup(pass, f.n, f.ny, f.nz, E, CT, o);
}

cudaError_t prepare_fused_kernels() {
    const int Ns[] = {32, 64, 96, 128, 192, 256, 384, 512, 768, 1024};
    const int zEs[] = {16, 12, 8, 6};
    for (int N : Ns)
        for (int zE : zEs)
            for (int wpb = 1; wpb <= 4; wpb *= 2) {
                ZctKernel z;
                if (zct_lookup(N, zE, wpb, &z)) {
                    cudaError_t e = allow_smem(z.k, 48 * 1024 + 1);
                    if (e != cudaSuccess) return e;
                }
            }
    const int zrEs[] = {16, 12, 8, 6, 4};
    int zrTiles[3 * 6];
    for (int d = 0, k = 0; d < 3; d++)
        for (int t : {1, 2, ZR_PARK + 1, ZR_PARK + 2, 2 * ZR_PARK + 1, 2 * ZR_PARK + 2})
            zrTiles[k++] = d * ZR_ASYNC + t;   // loads: registers, per-lane copies, bulk copies
    for (int N : Ns)
        for (int zE : zrEs)
            for (int tile : zrTiles) {
                ZctKernel z;
                if (zr_lookup(N, zE, tile, &z)) {
                    cudaError_t e = allow_smem(z.k, 48 * 1024 + 1);
                    if (e != cudaSuccess) return e;
                }
            }
    const int Ects[] = {8, 12, 16, 32};
    for (int N : Ns)
        for (int E : Ects)
            for (int ct = 8; ct <= 16; ct *= 2) {
                for (int which = 0; which < 3; which++) {
                    FzsKernel z;
                    if (fzs_lookup(which, N, E, ct, &z)) {
                        cudaError_t e = allow_smem(z.k, 48 * 1024 + 1);
                        if (e != cudaSuccess) return e;
                    }
                }
                for (int pass = 0; pass < 5; pass++) {
                    FzsKernel z;
                    if (pass < 4 ? fzk_lookup(pass, N, N, N, E, ct, &z) : fzeu_lookup(N, E, ct, &z)) {
                        cudaError_t e = allow_smem(z.k, 48 * 1024 + 1);
                        if (e != cudaSuccess) return e;
                    }
                }
            }
#define NSK_CASE(nx_, ny_, nz_, e_, ct_) {nx_, ny_, nz_, e_, ct_},
    static const int grids[][5] = {NSK_FZK_GRIDS(NSK_CASE)};
#undef NSK_CASE
    for (const auto &g : grids)
        for (int pass = 0; pass < 4; pass++) {
            FzsKernel z;
            if (fzk_lookup(pass, g[0], g[1], g[2], g[3], g[4], &z)) {
                cudaError_t e = allow_smem(z.k, 48 * 1024 + 1);
                if (e != cudaSuccess) return e;
            }
        }
    const int Es[] = {4, 6, 8, 9, 12, 16};
    for (int E : Es) {
        const void *ks[] = {strided_for<+1, true, false, true>(E), strided_for<+1, true, false, false>(E),
                            strided_for<-1, false, true, false>(E), z_for(E)};
        for (const void *k : ks) {
            cudaError_t e = allow_smem(k, 48 * 1024 + 1);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

static cudaError_t launch_strided(const void *k, const FzPass &ps, const Plan &pl, const float2 *tw,
                                  int ct, int nr, cudaStream_t s) {
    if (!k || ct < 1 || ct * (pl.n / pl.E) > 512) return cudaErrorInvalidValue;
    const int T = pl.n / pl.E;
    const size_t smem = (size_t)pl.n * (ct + 1) * sizeof(float2);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    const long tiles = (ps.ncols + ct - 1) / ct;
    const long blocks = tiles * ps.nfields;
    if (blocks > 0x7fffffffL) return cudaErrorInvalidValue;
    FzPass p = ps;
    Plan q = pl;
    void *args[] = {(void *)&p, (void *)&q, (void *)&tw};
    return cudaLaunchKernel(k, dim3((unsigned)blocks, (unsigned)nr), dim3(ct * T), args, smem, s);
}

// CTAs of a kernel that the device holds at once (its occupancy per SM times
// the SM count), cached per device and kernel; 0 if the query fails.
static long resident_blocks(const void *k, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, long> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(dev, k);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const long r = (long)(per > 0 ? per : 1) * sms;
    cache[key] = r;
    return r;
}

// NS_TEST_ZR_SKIP_COPY=1 (tests only): every warp of the bulk-copy pass C
// leaves its first copy unissued, so that the wait for it runs out (after
// about a millisecond) and the kernel reports the timeout in the error word.
static ZrCtl zr_ctl(const FusedRun &f) {
    const char *v = getenv("NS_TEST_ZR_SKIP_COPY");
    const bool skip = v && v[0] == '1';
    return ZrCtl{f.flags, skip ? (1LL << 21) : (1LL << 31), skip ? 1 : 0};   // about 1 ms / 1 s
}

static cudaError_t launch_zr(FusedRun &f, const PassCfg &cfg, cudaStream_t s) {
    ZctKernel z;
    if (!zr_lookup(f.nz, cfg.pl.E, cfg.ct, &z) || f.Mz != (f.nz - 1) / 3 + 1) return cudaErrorInvalidValue;
    long nlines = (long)f.n * f.ny;
    long fs = (long)f.n * f.ny * f.Mz;
    long brun = f.sB;
    if (z.bulk_bytes) {
        // bulk copies: every copy starts on a 16-byte boundary and moves a
        // whole number of 16-byte units (the kernel copies the LPW lines of a
        // group, groups never straddle the end)
        const int lpw = z.lines_per_block / (z.threads / 32);
        if (((uintptr_t)f.bbuf & 15) || (fs * 8) % 16 || (brun * 8) % 16 || z.bulk_bytes % 16 ||
            (long)z.bulk_bytes != (long)lpw * f.Mz * 8 || nlines % lpw)
            return cudaErrorInvalidValue;
    }
    cudaError_t e = allow_smem(z.k, z.smem);
    if (e != cudaSuccess) return e;
    // the kernel walks its line groups (k_fused_zr): one resident wave of
    // CTAs, shared among the runs of the group
    long blocks = (nlines + z.lines_per_block - 1) / z.lines_per_block;
    const long per_run = resident_blocks(z.k, z.threads, z.smem) / f.nr;
    if (per_run >= 1 && blocks > per_run) blocks = per_run;
    float2 *buf = f.bbuf;
    const float2 *tw = f.twz;
    ZrCtl ctl = zr_ctl(f);
    void *args[] = {(void *)&buf, (void *)&fs, (void *)&nlines, (void *)&brun, (void *)&tw, (void *)&ctl};
    return cudaLaunchKernel(z.k, dim3((unsigned)blocks, (unsigned)f.nr), dim3(z.threads), args, z.smem,
                            s);
}

static cudaError_t launch_z_ct(FusedRun &f, const PassCfg &cfg, cudaStream_t s) {
    ZctKernel z;
    if (!zct_lookup(f.nz, cfg.pl.E, cfg.ct, &z)) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem(z.k, z.smem);
    if (e != cudaSuccess) return e;
    long nlines = (long)f.n * f.ny;
    const long blocks = (nlines + z.lines_per_block - 1) / z.lines_per_block;
    float2 *buf = f.bbuf;
    long fs = (long)f.n * f.ny * f.Mz;
    int Mz = f.Mz;
    long brun = f.sB;
    const float2 *tw = f.twz;
    void *args[] = {(void *)&buf, (void *)&fs, (void *)&Mz, (void *)&nlines, (void *)&brun, (void *)&tw};
    return cudaLaunchKernel(z.k, dim3((unsigned)blocks, (unsigned)f.nr), dim3(z.threads), args, z.smem,
                            s);
}

static cudaError_t launch_z(FusedRun &f, const PassCfg &cfg, cudaStream_t s) {
    if (cfg.kind == 1) return launch_z_ct(f, cfg, s);
    if (cfg.kind == 2) return launch_zr(f, cfg, s);
    const void *k = z_for(cfg.pl.E);
    if (!k) return cudaErrorInvalidValue;
    const int n = f.nz / 2, Tn = n / cfg.pl.E;
    const int L = cfg.ct;
    if (L < 1 || 6 * L * Tn > 256 || cfg.pl.n != n) return cudaErrorInvalidValue;
    const size_t smem = (size_t)6 * L * fz_line_stride(n) * sizeof(float2);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    const long nlines = (long)f.n * f.ny;
    const long blocks = (nlines + L - 1) / L;
    float2 *buf = f.bbuf;
    long fs = (long)f.n * f.ny * f.Mz;
    int N = f.nz, Mz = f.Mz;
    Plan q = cfg.pl;
    const float2 *tw = f.twz;
    int LL = L;
    long brun = f.sB;
    void *args[] = {(void *)&buf, (void *)&fs, (void *)&N, (void *)&Mz, (void *)&nlines, (void *)&LL,
                    (void *)&brun, (void *)&q, (void *)&tw};
    return cudaLaunchKernel(k, dim3((unsigned)blocks, (unsigned)f.nr), dim3(6 * L * Tn), args, smem, s);
}

// Pass descriptors of one RK2 stage reading the state src.
// Layouts: A out [6][iky][x][kz], B out [6][y][x][kz] (pass C in place), D
// out [3][x][iky][kz], E out compact [3][ikx][iky][kz]; on the cube
// N_y = N_x = n and My = Mx.
static void pass_descs(const FusedRun &f, const float2 *src, FzPass &A, FzPass &B, FzPass &D, FzPass &Ep) {
    const int Nx = f.n, Ny = f.ny, K = f.K, Mx = f.Mx, My = f.My, Mz = f.Mz;
    const long MyMz = (long)My * Mz, NxMz = (long)Nx * Mz;
    const long S3 = 3 * f.M;
    A = FzPass{src, f.abuf, MyMz, f.M, MyMz, (long)My * NxMz, Mz, NxMz, 6, Mz, K, Mx, S3, f.sA, Mz};
    B = FzPass{f.abuf, f.bbuf, NxMz, (long)My * NxMz, NxMz, (long)Ny * NxMz, NxMz, Mz, 6, Mz, f.Ky, My, f.sA,
               f.sB, Mz};
    D = FzPass{f.bbuf, f.abuf, NxMz, (long)Ny * NxMz, NxMz, (long)Nx * MyMz, Mz, MyMz, 3, Mz, f.Ky, My, f.sB,
               f.sA, Mz};
    Ep = FzPass{f.abuf, f.nl, MyMz, (long)Nx * MyMz, MyMz, f.M, MyMz, Mz, 3, Mz, K, Mx, f.sA, S3, Mz};
    if (!f.cube) {   // the curl of pass A: y compaction and the box
        A.Ko = f.Ky;
        A.Mo = My;
        A.sx = f.sx;
        A.sy = f.sy;
        A.sz = f.sz;
    }
}

// Transform length, twiddle table and default plan of pass 0..3 (A, B, D, E).
static int pass_len(const FusedRun &f, int pass) { return pass == 1 || pass == 2 ? f.ny : f.n; }
static const float2 *pass_tw(const FusedRun &f, int pass) { return pass == 1 || pass == 2 ? f.twy : f.tw; }
static const Plan &pass_plan(const FusedRun &f, int pass) { return pass == 1 || pass == 2 ? f.plY : f.plN; }

static cudaError_t run_pass_ct(FusedRun &f, int pass, const PassCfg &cfg, const FzPass &ps,
                               cudaStream_t s) {
    FzsKernel z;
    const int which = pass < 2 ? pass : 2;
    if (!fzs_lookup(which, pass_len(f, pass), cfg.pl.E, cfg.ct, &z)) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem(z.k, z.smem);
    if (e != cudaSuccess) return e;
    const long tiles = (ps.ncols + cfg.ct - 1) / cfg.ct;
    const long blocks = tiles * ps.nfields;
    if (blocks > 0x7fffffffL) return cudaErrorInvalidValue;
    FzPass p = ps;
    const float2 *tw = pass_tw(f, pass);
    void *args[] = {(void *)&p, (void *)&tw};
    return cudaLaunchKernel(z.k, dim3((unsigned)blocks, (unsigned)f.nr), dim3(z.threads), args, z.smem, s);
}

static cudaError_t run_pass_k(FusedRun &f, int pass, const PassCfg &cfg, const FzPass &ps, cudaStream_t s) {
    FzsKernel z;
    if (!fzk_for(f, pass, cfg.pl.E, cfg.ct, &z)) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem(z.k, z.smem);
    if (e != cudaSuccess) return e;
    const long tiles = (ps.ncols + cfg.ct - 1) / cfg.ct;
    const long blocks = tiles * ps.nfields;
    if (blocks > 0x7fffffffL) return cudaErrorInvalidValue;
    const float2 *in = ps.in, *tw = pass_tw(f, pass);
    float2 *out = ps.out;
    float3 sc = make_float3(f.sx, f.sy, f.sz);
    void *args[] = {(void *)&in, (void *)&out, (void *)&tw, (void *)&sc};
    return cudaLaunchKernel(z.k, dim3((unsigned)blocks, (unsigned)f.nr), dim3(z.threads), args, z.smem, s);
}

// Pass 0..3 (A, B, D, E) with configuration cfg on the buffers of ps.
static cudaError_t run_pass(FusedRun &f, int pass, const PassCfg &cfg, const FzPass &ps, cudaStream_t s) {
    if (cfg.kind == 2) return run_pass_k(f, pass, cfg, ps, s);
    const int which = pass < 2 ? pass : 2;
    if (cfg.kind == 1) return run_pass_ct(f, pass, cfg, ps, s);
    const int E = cfg.pl.E;
    const void *k = which == 0 ? strided_for<+1, true, false, true>(E)
                  : which == 1 ? strided_for<+1, true, false, false>(E)
                               : strided_for<-1, false, true, false>(E);
    if (cfg.pl.n != pass_len(f, pass)) return cudaErrorInvalidValue;
    return launch_strided(k, ps, cfg.pl, pass_tw(f, pass), cfg.ct, f.nr, s);
}

// Induction update of the MHD form's magnetic block: N_b = i k x nb / N^3
// (nb the transform of u x b; the cubic rule is the compact layout, the
// spherical one a mask), then the IF-RK2 stage with exp(-eta k^2 dt); the
// mean field b(k = 0) has N_b = 0 and factor 1.
__global__ void __launch_bounds__(256)
k_fused_update_b(float2 *__restrict__ b, float2 *__restrict__ b1, const float2 *__restrict__ nb,
                 const float *__restrict__ etab, const FzRunParams *__restrict__ rp, FzUpdate u) {
    const long M = u.M;
    const int run = blockIdx.y;
    b += run * 3 * M;
    b1 += run * 3 * M;
    nb += run * 3 * M;
    etab += (long)run * u.nk2;
    const FzRunParams q = rp[run];
    const float inv = (float)(1.0 / ((double)u.n * u.n * u.n));
    const bool two = u.stage == 2;
    float2 *dst = two ? b : b1;
    const unsigned Mz = (unsigned)u.Mz, Mx = (unsigned)u.Mx;
    for (long m = blockIdx.x * (long)blockDim.x + threadIdx.x; m < M; m += (long)gridDim.x * blockDim.x) {
        const float2 v0 = nb[m], v1 = nb[M + m], v2 = nb[2 * M + m];
        const float2 c0 = b[m], c1 = b[M + m], c2 = b[2 * M + m];
        const float2 z = make_float2(0.f, 0.f);
        const float2 d0 = two ? b1[m] : z, d1 = two ? b1[M + m] : z, d2 = two ? b1[2 * M + m] : z;
        const unsigned row = (unsigned)m / Mz;
        const int kz = (int)((unsigned)m - row * Mz);
        const int ky = fz_compact_signed((int)(row % Mx), u.Mx, u.K);
        const int kx = fz_compact_signed((int)(row / Mx), u.Mx, u.K);
        const int k2 = kx * kx + ky * ky + kz * kz;
        float2 o0 = z, o1 = z, o2 = z;
        if (!(q.dealias == 1 && 9L * k2 >= (long)u.n * u.n)) {
            const float fkx = (float)kx, fky = (float)ky, fkz = (float)kz;
            const float2 vx = cscale(v0, inv), vy = cscale(v1, inv), vz = cscale(v2, inv);
            const float2 nx = cmul_i<1>(csub(cscale(vz, fky), cscale(vy, fkz)));   // i k x v
            const float2 ny = cmul_i<1>(csub(cscale(vx, fkz), cscale(vz, fkx)));
            const float2 nz = cmul_i<1>(csub(cscale(vy, fkx), cscale(vx, fky)));
            const float e = etab[k2];
            if (!two) {
                o0 = cscale(cadd(c0, cscale(nx, q.dt)), e);
                o1 = cscale(cadd(c1, cscale(ny, q.dt)), e);
                o2 = cscale(cadd(c2, cscale(nz, q.dt)), e);
            } else {
                const float he = 0.5f * e;
                o0 = cadd(cscale(c0, he), cscale(cadd(d0, cscale(nx, q.dt)), 0.5f));
                o1 = cadd(cscale(c1, he), cscale(cadd(d1, cscale(ny, q.dt)), 0.5f));
                o2 = cadd(cscale(c2, he), cscale(cadd(d2, cscale(nz, q.dt)), 0.5f));
            }
        }
        dst[m] = o0;
        dst[M + m] = o1;
        dst[2 * M + m] = o2;
    }
}

// MHD pass C: E elements per thread, wpb warps per CTA.
static cudaError_t launch_zm(FusedRun &f, int E, int wpb, cudaStream_t s) {
    ZctKernel z;
    if (!zrm_lookup(f.n, E, wpb, &z) || f.Mz != (f.n - 1) / 3 + 1) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem(z.k, z.smem);
    if (e != cudaSuccess) return e;
    long nlines = (long)f.n * f.n;
    const long blocks = (nlines + z.lines_per_block - 1) / z.lines_per_block;
    float2 *bu = f.bbuf, *bb = f.bbuf + f.blk_B;
    long fs = (long)f.n * f.n * f.Mz;
    long brun = f.sB;
    const float2 *tw = f.tw;
    void *args[] = {(void *)&bu, (void *)&bb, (void *)&fs, (void *)&nlines, (void *)&brun, (void *)&tw};
    return cudaLaunchKernel(z.k, dim3((unsigned)blocks, (unsigned)f.nr), dim3(z.threads), args, z.smem, s);
}

// The separate update kernel, u.nparts blocks (partials) per run.
static cudaError_t launch_update_n(FusedRun &f, const FzUpdate &u, cudaStream_t s) {
    if (f.cube) k_fused_update<false><<<dim3(u.nparts, f.nr), 256, 0, s>>>(f.a, f.a1, f.nl, f.etab, f.rp, u, f.part);
    else k_fused_update<true><<<dim3(u.nparts, f.nr), 256, 0, s>>>(f.a, f.a1, f.nl, f.etab, f.rp, u, f.part);
    return cudaGetLastError();
}

// Update arguments of stage `stage` with nparts partial sums per run.
static FzUpdate make_update(const FusedRun &f, int stage, int nparts) {
    FzUpdate u{f.n, f.K, f.Mx, f.Mz, stage, f.M, f.nk2, nparts};
    if (!f.cube) {
        u.My = f.My;
        u.Ky = f.Ky;
        u.inv = (float)(1.0 / ((double)f.n * f.ny * f.nz));
        u.sx = f.sx;
        u.sy = f.sy;
        u.sz = f.sz;
        u.D = f.D;
        u.qx = f.qx;
        u.qy = f.qy;
        u.qz = f.qz;
        u.k2tab = f.k2tab;
    }
    return u;
}

// Column tiles (and energy partials per run) of pass E fused with the update.
static long eu_tiles(const FusedRun &f, int ct) { return ((long)f.Mx * f.Mz + ct - 1) / ct; }

// Pass E fused with the update at RK2 stage `stage`: reads pass D's output,
// updates the state in place (a1 at stage 1, a at stage 2).
static cudaError_t launch_eu(FusedRun &f, int E, int ct, int stage, cudaStream_t s) {
    FzsKernel z;
    if (!fzeu_lookup(f.n, E, ct, &z)) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem(z.k, z.smem);
    if (e != cudaSuccess) return e;
    const long tiles = eu_tiles(f, ct);
    FzUpdate u = make_update(f, stage, (int)tiles);
    const float2 *din = f.abuf, *tw = f.tw;
    float2 *a = f.a, *a1 = f.a1;
    const float *etab = f.etab;
    const FzRunParams *rp = f.rp;
    double *part = f.part;
    void *args[] = {(void *)&din, (void *)&a, (void *)&a1, (void *)&etab, (void *)&rp,
                    (void *)&u, (void *)&tw, (void *)&part};
    return cudaLaunchKernel(z.k, dim3((unsigned)tiles, (unsigned)f.nr), dim3(z.threads), args, z.smem, s);
}

template <class F> static float time_launch(F launch, cudaStream_t s, int reps);

// Fastest compiled MHD pass-C kernel for the group, timed on its own buffers.
static cudaError_t tune_zm(FusedRun &f, cudaStream_t s) {
    float best = -1.f;
    const int Es[] = {16, 12, 8, 6};
    for (int E : Es)
        for (int wpb = 1; wpb <= 2; wpb++) {
            ZctKernel z;
            if (!zrm_lookup(f.n, E, wpb, &z)) continue;
            const float ms = time_launch([&]() { return launch_zm(f, E, wpb, s); }, s, 3);
            if (ms > 0.f && (best < 0.f || ms < best)) {
                best = ms;
                f.zm_E = E;
                f.zm_wpb = wpb;
            }
        }
    return best < 0.f ? cudaErrorInvalidValue : cudaSuccess;
}

// ---------------------------------------------------------------- autotuner

// Candidate radix splits (elements per thread) for a line of length n.
static std::vector<Plan> plan_candidates(int n) {
    std::vector<Plan> out;
    const int Es[] = {16, 12, 9, 8, 6, 4};
    for (int E : Es) {
        Plan p;
        if (make_plan_e(n, E, &p) && p.nst <= 4) out.push_back(p);
    }
    return out;
}

struct TunedCfgs {
    PassCfg s[4];   // A, B, D, E
    PassCfg c;      // pass C (ct = lines per CTA)
    int eu_E = 0, eu_ct = 0;   // pass E fused with the update, 0: separate
};

// Time `launch` (after one warm-up) over `reps` launches; returns ms per launch
// or a negative number if it failed.
template <class F> static float time_launch(F launch, cudaStream_t s, int reps) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.f;
    }
    float ms = -1.f;
    if (launch() == cudaSuccess && cudaEventRecord(a, s) == cudaSuccess) {
        bool ok = true;
        for (int i = 0; i < reps && ok; i++) ok = launch() == cudaSuccess;
        if (ok && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
            ms /= reps;
        else
            ms = -1.f;
    }
    cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

// Plan cache file (environment variable NS_PLAN_CACHE): one JSON object
// mapping N to five [kind, E, tile] triples (passes A, B, D, E, C).  Entries
// found there are used as they are; newly tuned sizes are written back.
static bool cfg_from_triple(int n, int kind, int E, int tile, bool zpass, PassCfg &out) {
    Plan pl;
    const int len = zpass ? n / 2 : n;
    if (kind == 1 || kind == 2) {
        if (!make_plan(len, &pl)) return false;
        pl.E = E;   // compile-time kernels carry their own plan; E names the shape
    } else if (!make_plan_e(len, E, &pl)) {
        return false;
    }
    out = PassCfg{pl, tile, kind};
    return true;
}

static void plan_cache_read(std::map<int, TunedCfgs> &cache) {
    const char *path = getenv("NS_PLAN_CACHE");
    if (!path) return;
    FILE *fp = fopen(path, "r");
    if (!fp) return;
    std::string txt;
    char buf[4096];
    size_t r;
    while ((r = fread(buf, 1, sizeof(buf), fp)) > 0) txt.append(buf, r);
    fclose(fp);
    size_t pos = 0;
    while ((pos = txt.find('"', pos)) != std::string::npos) {
        int n = 0, v[18] = {0}, used = 0;
        const char *at = txt.c_str() + pos;
        bool six = sscanf(at, "\"%d\": [[%d, %d, %d], [%d, %d, %d], [%d, %d, %d], [%d, %d, %d], [%d, %d, %d], [%d, %d, %d]]%n",
                          &n, &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6], &v[7], &v[8], &v[9], &v[10],
                          &v[11], &v[12], &v[13], &v[14], &v[15], &v[16], &v[17], &used) == 19 && used > 0;
        if (!six) {
            used = 0;
            v[15] = v[16] = v[17] = 0;
        }
        if (six || (sscanf(at, "\"%d\": [[%d, %d, %d], [%d, %d, %d], [%d, %d, %d], [%d, %d, %d], [%d, %d, %d]]%n",
                           &n, &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6], &v[7], &v[8], &v[9], &v[10],
                           &v[11], &v[12], &v[13], &v[14], &used) == 16 && used > 0)) {
            TunedCfgs t;
            bool ok = true;
            for (int i = 0; i < 4 && ok; i++) ok = cfg_from_triple(n, v[3 * i], v[3 * i + 1], v[3 * i + 2], false, t.s[i]);
            ok = ok && cfg_from_triple(n, v[12], v[13], v[14], true, t.c);
            FzsKernel z;
            if (v[15] == 3 && fzeu_lookup(n, v[16], v[17], &z)) {
                t.eu_E = v[16];
                t.eu_ct = v[17];
            }
            if (ok) cache[n] = t;
            pos += used;
        } else {
            pos++;
        }
    }
}

static void plan_cache_write(const std::map<int, TunedCfgs> &cache) {
    const char *path = getenv("NS_PLAN_CACHE");
    if (!path) return;
    FILE *fp = fopen(path, "w");
    if (!fp) return;
    fprintf(fp, "{");
    bool first = true;
    for (const auto &kv : cache) {
        const TunedCfgs &t = kv.second;
        fprintf(fp, "%s\n  \"%d\": [", first ? "" : ",", kv.first);
        for (int i = 0; i < 4; i++)
            fprintf(fp, "[%d, %d, %d], ", t.s[i].kind, t.s[i].pl.E, t.s[i].ct);
        fprintf(fp, "[%d, %d, %d], [%d, %d, %d]]", t.c.kind, t.c.pl.E, t.c.ct, t.eu_E ? 3 : 0, t.eu_E,
                t.eu_ct);
        first = false;
    }
    fprintf(fp, "\n}\n");
    fclose(fp);
}

// Choose, per pass, the kernel (runtime or compile-time length), the radix
// split E and the tile (columns per CTA for the strided passes, lines or warps
// per CTA for pass C) that run fastest on this run's own buffers; results
// are kept per N for the life of the process (and in the plan cache file).
// The final choice of a sweep.  The sweep times every candidate over a few
// launches; candidates within a few percent of each other are then ordered
// by noise as much as by speed.  So the three fastest are timed again over
// more launches, in turn and twice, and each keeps its best time; the
// fastest of those is kept.  time_of(cfg, reps) returns ms per launch.
template <class Cfg, class TimeOf>
static bool pick_best(std::vector<std::pair<float, Cfg>> &cands, TimeOf time_of, Cfg *out) {
    if (cands.empty()) return false;
    std::stable_sort(cands.begin(), cands.end(),
                     [](const std::pair<float, Cfg> &a, const std::pair<float, Cfg> &b) {
                         return a.first < b.first;
                     });
    const size_t top = std::min<size_t>(3, cands.size());
    std::vector<float> best(top, -1.f);
    for (int round = 0; round < 2; round++)
        for (size_t i = 0; i < top; i++) {
            const float ms = time_of(cands[i].second, 8);
            if (ms > 0.f && (best[i] < 0.f || ms < best[i])) best[i] = ms;
        }
    size_t k = 0;
    for (size_t i = 1; i < top; i++)
        if (best[i] > 0.f && (best[k] < 0.f || best[i] < best[k])) k = i;
    *out = cands[k].second;
    return true;
}

static cudaError_t fused_autotune(FusedRun &f, cudaStream_t s) {
    static std::mutex mu;
    static std::map<int, TunedCfgs> cache;   // cubes, by N (also in the plan-cache file)
    static std::map<std::tuple<int, int, int>, TunedCfgs> gcache;   // grids, for the process
    static bool loaded = false;
    const auto gkey = std::make_tuple(f.n, f.ny, f.nz);
    {
        std::lock_guard<std::mutex> g(mu);
        if (!loaded) {
            plan_cache_read(cache);
            loaded = true;
        }
        const TunedCfgs *hit = nullptr;
        if (f.cube) {
            auto it = cache.find(f.n);
            if (it != cache.end()) hit = &it->second;
        } else {
            auto it = gcache.find(gkey);
            if (it != gcache.end()) hit = &it->second;
        }
        if (hit) {
            for (int i = 0; i < 4; i++) f.sp[i] = hit->s[i];
            f.zc = hit->c;
            f.eu_E = hit->eu_E;
            f.eu_ct = hit->eu_ct;
            return cudaSuccess;
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const int reps = 3;
    FzPass P[4];
    pass_descs(f, f.a, P[0], P[1], P[2], P[3]);
    const int which[4] = {0, 1, 2, 2};
    for (int i = 0; i < 4; i++) {
        std::vector<std::pair<float, PassCfg>> cands;
        auto time_of = [&](const PassCfg &cfg, int r) {
            return time_launch([&]() { return run_pass(f, i, cfg, P[i], s); }, s, r);
        };
        const int Es[] = {8, 12, 16, 32};
        const int len = pass_len(f, i);
        for (int kind = 2; kind >= 1; kind--)
            for (int E : Es)
                for (int ct = 8; ct <= 16; ct *= 2) {
                    FzsKernel z;
                    if (kind == 1 ? !fzs_lookup(which[i], len, E, ct, &z) : !fzk_for(f, i, E, ct, &z))
                        continue;
                    PassCfg cfg{pass_plan(f, i), ct, kind};
                    cfg.pl.E = E;
                    const float ms = time_of(cfg, reps);
                    if (ms > 0.f) cands.push_back({ms, cfg});
                }
        for (const Plan &pl : plan_candidates(len)) {
            const int T = pl.n / pl.E;
            for (int ct = 8; ct <= 16; ct *= 2) {
                if (ct * T > 512 || (ct * T < 32 && ct < 16)) continue;
                PassCfg cfg{pl, ct, 0};
                const float ms = time_of(cfg, reps);
                if (ms > 0.f) cands.push_back({ms, cfg});
            }
        }
        if (!pick_best(cands, time_of, &f.sp[i])) return cudaErrorInvalidValue;
    }
    {
        std::vector<std::pair<float, PassCfg>> cands;
        auto time_of = [&](const PassCfg &cfg, int r) {
            return time_launch([&]() { return launch_z(f, cfg, s); }, s, r);
        };
        const int zEs[] = {16, 12, 8, 6};
        for (int zE : zEs)
        for (int wpb = 1; wpb <= 4; wpb *= 2) {
            ZctKernel z;
            if (!zct_lookup(f.nz, zE, wpb, &z)) continue;
            PassCfg cfg{f.plH, wpb, 1};
            cfg.pl.E = zE;
            const float ms = time_of(cfg, reps);
            if (ms > 0.f) cands.push_back({ms, cfg});
        }
        const int zrEs[] = {16, 12, 8, 6, 4};
        int zrTiles[3 * 6];
        for (int d = 0, k = 0; d < 3; d++)
            for (int t : {1, 2, ZR_PARK + 1, ZR_PARK + 2, 2 * ZR_PARK + 1, 2 * ZR_PARK + 2})
                zrTiles[k++] = d * ZR_ASYNC + t;   // loads: registers, per-lane copies, bulk copies
        for (int zE : zrEs)
            for (int tile : zrTiles) {
                ZctKernel z;
                if (!zr_lookup(f.nz, zE, tile, &z)) continue;
                PassCfg cfg{f.plH, tile, 2};
                cfg.pl.E = zE;
                const float ms = time_of(cfg, reps);
                if (ms > 0.f) cands.push_back({ms, cfg});
            }
        for (const Plan &pl : plan_candidates(f.nz / 2)) {
            const int Tn = pl.n / pl.E;
            for (int L = 1; 6 * L * Tn <= 256; L *= 2) {
                PassCfg cfg{pl, L, 0};
                const float ms = time_of(cfg, reps);
                if (ms > 0.f) cands.push_back({ms, cfg});
            }
        }
        if (!pick_best(cands, time_of, &f.zc)) return cudaErrorInvalidValue;
    }
    // pass E then the update, against pass E fused with the update (stage 2;
    // its kernels are compiled for the cube)
    if (f.cube) {
        FzUpdate u = make_update(f, 2, f.nparts_upd);
        const float sep = time_launch([&]() { return run_pass(f, 3, f.sp[3], P[3], s); }, s, reps) +
                          time_launch([&]() { return launch_update_n(f, u, s); }, s, reps);
        float best = sep > 0.f ? sep : -1.f;
        f.eu_E = f.eu_ct = 0;
        const int Es[] = {8, 12, 16, 32};
        for (int E : Es)
            for (int ct = 8; ct <= 16; ct *= 2) {
                FzsKernel z;
                if (!fzeu_lookup(f.n, E, ct, &z)) continue;
                const float ms = time_launch([&]() { return launch_eu(f, E, ct, 2, s); }, s, reps);
                if (ms > 0.f && (best < 0.f || ms < best)) {
                    best = ms;
                    f.eu_E = E;
                    f.eu_ct = ct;
                }
            }
    }
    std::lock_guard<std::mutex> g(mu);
    TunedCfgs t;
    for (int i = 0; i < 4; i++) t.s[i] = f.sp[i];
    t.c = f.zc;
    t.eu_E = f.eu_E;
    t.eu_ct = f.eu_ct;
    if (!f.cube) {
        gcache[gkey] = t;
        return cudaSuccess;
    }
    cache[f.n] = t;
    plan_cache_write(cache);
    return cudaSuccess;
}

static long gcd_l(long a, long b) { return b ? gcd_l(b, a % b) : a; }

// Grid and box of a run: (N_x, N_y, N_z) and l_i (0 in the parameters: N, 1).
static void run_dims(const ns_run_params &p, int d[3], double l[3]) {
    d[0] = p.n;
    d[1] = p.ny > 0 ? p.ny : p.n;
    d[2] = p.nz > 0 ? p.nz : p.n;
    l[0] = p.lx > 0 ? p.lx : 1.0;
    l[1] = p.ly > 0 ? p.ly : 1.0;
    l[2] = p.lz > 0 ? p.lz : 1.0;
}

bool fused_grid_supported(const ns_run_params &p) {
    int d[3];
    double l[3];
    run_dims(p, d, l);
    const bool cube = d[0] == d[1] && d[0] == d[2] && l[0] == 1.0 && l[1] == 1.0 && l[2] == 1.0;
    return cube || (!p.mhd && (p.dealias == 0 || p.dealias == 1));
}

cudaError_t fused_alloc(FusedRun &f, const std::vector<ns_run_params> &runs, const float2 *tw,
                        const float2 *twy, const float2 *twz, int series_cap, cudaStream_t s) {
    if (runs.empty()) return cudaErrorInvalidValue;
    f.p = runs;
    f.nr = (int)runs.size();
    int d[3];
    double l[3];
    run_dims(runs[0], d, l);
    for (const ns_run_params &q : runs) {
        int dq[3];
        double lq[3];
        run_dims(q, dq, lq);
        for (int i = 0; i < 3; i++)
            if (dq[i] != d[i] || lq[i] != l[i]) return cudaErrorInvalidValue;
    }
    f.n = d[0];
    f.ny = d[1];
    f.nz = d[2];
    f.unit = l[0] == 1.0 && l[1] == 1.0 && l[2] == 1.0;
    f.cube = f.unit && f.n == f.ny && f.n == f.nz;
    f.K = (f.n - 1) / 3;     // largest m with 3m < N_i, per axis
    f.Ky = (f.ny - 1) / 3;
    f.Kz = (f.nz - 1) / 3;
    f.Mx = 2 * f.K + 1;
    f.My = 2 * f.Ky + 1;
    f.Mz = f.Kz + 1;
    f.sx = (float)(1.0 / l[0]);
    f.sy = (float)(1.0 / l[1]);
    f.sz = (float)(1.0 / l[2]);
    f.D = (long)f.n / gcd_l(f.n, f.ny) * f.ny;
    f.D = f.D / gcd_l(f.D, f.nz) * f.nz;
    f.qx = f.D / f.n;
    f.qy = f.D / f.ny;
    f.qz = f.D / f.nz;
    f.tw = tw;
    f.twy = f.cube ? tw : twy;
    f.twz = f.cube ? tw : twz;
    f.cap = series_cap;
    if (!make_plan(f.n, &f.plN) || !make_plan(f.ny, &f.plY) || !make_plan(f.nz / 2, &f.plH))
        return cudaErrorInvalidValue;
    f.M = (long)f.Mx * f.My * f.Mz;
    f.sA = 6L * f.My * f.n * f.Mz;          // also holds D (3 fields)
    f.sB = 6L * f.ny * f.n * f.Mz;          // also holds C (3 fields)
    const long S3 = 3 * f.M, nr = f.nr;
    f.mhd = runs[0].mhd != 0;
    for (const ns_run_params &q : runs)
        if ((q.mhd != 0) != f.mhd || !fused_grid_supported(q)) return cudaErrorInvalidValue;
    const int nb = f.mhd ? 2 : 1;            // blocks: velocity (and magnetic)
    f.blk_s = nr * S3;
    f.blk_A = nr * f.sA;
    f.blk_B = nr * f.sB;
    cudaError_t e;
    if ((e = dev_malloc((void **)&f.a, nb * nr * S3 * sizeof(float2))) != cudaSuccess) return e;
    if ((e = dev_malloc((void **)&f.a1, nb * nr * S3 * sizeof(float2))) != cudaSuccess) return e;
    if ((e = dev_malloc((void **)&f.nl, nb * nr * S3 * sizeof(float2))) != cudaSuccess) return e;
    if ((e = dev_malloc((void **)&f.abuf, nb * nr * f.sA * sizeof(float2))) != cudaSuccess) return e;
    if ((e = dev_malloc((void **)&f.bbuf, nb * nr * f.sB * sizeof(float2))) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(f.a, 0, nb * nr * S3 * sizeof(float2), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(f.a1, 0, nb * nr * S3 * sizeof(float2), s)) != cudaSuccess) return e;
    // factor tables exp(-nu k^2 dt) in FP64, rounded once (the cube: by integer
    // k^2; a grid or box: per axis by compact index, exp(-nu (m_i / l_i)^2 dt)),
    // and per-run parameters
    f.nk2 = f.cube ? 3 * f.K * f.K + 1 : f.Mx + f.My + f.Mz;
    std::vector<float> h((size_t)nr * f.nk2);
    std::vector<FzRunParams> hp(nr);
    for (long r = 0; r < nr; r++) {
        const ns_run_params &q = runs[r];
        if (f.cube) {
            for (int k2 = 0; k2 < f.nk2; k2++) h[r * f.nk2 + k2] = (float)exp(-q.nu * (double)k2 * q.dt);
        } else {
            const int Ms[3] = {f.Mx, f.My, f.Mz}, Ks[3] = {f.K, f.Ky, f.Kz};
            for (int a = 0, o = 0; a < 3; o += Ms[a], a++)
                for (int i = 0; i < Ms[a]; i++) {
                    const int m = a < 2 && i > Ks[a] ? i - Ms[a] : i;
                    const double k = (double)m / l[a];
                    h[r * f.nk2 + o + i] = (float)exp(-q.nu * k * k * q.dt);
                }
        }
        hp[r] = FzRunParams{(float)q.dt, (float)q.force_amp, q.force_k, q.dealias, (float)q.rot,
                            (int)lround(q.force_k * l[0]), (int)lround(q.force_k * l[1]),
                            (int)lround(q.force_k * l[2])};
    }
    if ((e = dev_malloc((void **)&f.etab, h.size() * sizeof(float))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(f.etab, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    if (!f.cube) {   // (m_i / l_i)^2 per axis in FP64, split into FP32 hi + lo
        std::vector<float2> k2h;
        const int Ms[3] = {f.Mx, f.My, f.Mz}, Ks[3] = {f.K, f.Ky, f.Kz};
        for (int a = 0; a < 3; a++)
            for (int i = 0; i < Ms[a]; i++) {
                const int m = a < 2 && i > Ks[a] ? i - Ms[a] : i;
                const double k = (double)m / l[a], v = k * k;
                const float hi = (float)v;
                k2h.push_back(make_float2(hi, (float)(v - (double)hi)));
            }
        if ((e = dev_malloc((void **)&f.k2tab, k2h.size() * sizeof(float2))) != cudaSuccess) return e;
        if ((e = cudaMemcpy(f.k2tab, k2h.data(), k2h.size() * sizeof(float2), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return e;
    }
    if (f.mhd) {   // exp(-eta k^2 dt) per run
        for (long r = 0; r < nr; r++)
            for (int k2 = 0; k2 < f.nk2; k2++)
                h[r * f.nk2 + k2] = (float)exp(-runs[r].eta * (double)k2 * runs[r].dt);
        if ((e = dev_malloc((void **)&f.etab_b, h.size() * sizeof(float))) != cudaSuccess) return e;
        if ((e = cudaMemcpy(f.etab_b, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return e;
    }
    if ((e = dev_malloc((void **)&f.rp, nr * sizeof(FzRunParams))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(f.rp, hp.data(), nr * sizeof(FzRunParams), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    // partials per run: the separate update's blocks, or one per column tile of
    // pass E fused with the update (at most eu_tiles(f, 8))
    f.nparts_upd = (int)std::min<long>(1024, std::max<long>(1, (f.M + 4095) / 4096));
    f.nparts = f.nparts_upd;
    const long parts_max = std::max<long>(f.nparts_upd, eu_tiles(f, 8));
    if ((e = dev_malloc((void **)&f.part, nr * parts_max * 2 * sizeof(double))) != cudaSuccess) return e;
    if ((e = dev_malloc((void **)&f.series, nr * (long)f.cap * 2 * sizeof(double))) != cudaSuccess) return e;
    if ((e = dev_malloc((void **)&f.counter, nr * sizeof(unsigned long long))) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(f.counter, 0, nr * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if ((e = prepare_fused_kernels()) != cudaSuccess) return e;
    const int ct = default_ct(sizeof(float2), f.n);
    for (int i = 0; i < 4; i++) f.sp[i] = PassCfg{pass_plan(f, i), ct};
    f.zc = PassCfg{f.plH, std::max(1, 192 / (6 * (f.nz / 2 / f.plH.E)))};
    cudaError_t e2 = fused_autotune(f, s);
    if (e2 != cudaSuccess) return e2;
    // Diagnostic override of pass E + update: NS_FORCE_EU="off" (separate
    // kernels) or "E,ct" (that fused kernel, if compiled for N).
    if (const char *fe = getenv("NS_FORCE_EU")) {
        int E = 0, ct = 0;
        FzsKernel z;
        if (strcmp(fe, "off") == 0) f.eu_E = f.eu_ct = 0;
        else if (f.cube && sscanf(fe, "%d,%d", &E, &ct) == 2 && fzeu_lookup(f.n, E, ct, &z)) {
            f.eu_E = E;
            f.eu_ct = ct;
        }
    }
    if (f.mhd) {
        f.eu_E = f.eu_ct = 0;   // the magnetic block has its own update
        cudaError_t e3 = tune_zm(f, s);
        if (e3 != cudaSuccess) return e3;
    }
    f.nparts = f.eu_E ? (int)eu_tiles(f, f.eu_ct) : f.nparts_upd;
    // Diagnostic override of the pass-C kernel, NS_FORCE_PASS_C="kind,E,tile"
    // (the plan-cache triple); ignored when no such kernel is compiled for N.
    if (const char *fz = getenv("NS_FORCE_PASS_C")) {
        int kind = -1, E = 0, tile = 0;
        PassCfg c;
        ZctKernel z;
        if (sscanf(fz, "%d,%d,%d", &kind, &E, &tile) == 3 && cfg_from_triple(f.nz, kind, E, tile, true, c)) {
            const bool ok = kind == 2   ? zr_lookup(f.nz, E, tile, &z)
                            : kind == 1 ? zct_lookup(f.nz, E, tile, &z)
                                        : (kind == 0 && z_for(E) && tile >= 1 &&
                                           6 * tile * (f.nz / 2 / E) <= 256);
            if (ok) f.zc = c;
        }
    }
    // The same for the strided passes A, B, D, E: NS_FORCE_STRIDED="kind,E,ct"
    // (kind 1 or 2) applies to each pass that has such a kernel compiled.
    if (const char *fs = getenv("NS_FORCE_STRIDED")) {
        int kind = -1, E = 0, ct = 0;
        if (sscanf(fs, "%d,%d,%d", &kind, &E, &ct) == 3 && (kind == 1 || kind == 2))
            for (int i = 0; i < 4; i++) {
                FzsKernel z;
                PassCfg ci;
                if (!cfg_from_triple(pass_len(f, i), kind, E, ct, false, ci)) continue;
                const bool ok = kind == 2 ? fzk_for(f, i, E, ct, &z)
                                          : fzs_lookup(i < 2 ? i : 2, pass_len(f, i), E, ct, &z);
                if (ok) f.sp[i] = ci;
            }
    }
    return cudaSuccess;
}

void fused_free(FusedRun &f) {
    void *ps[] = {f.a, f.a1, f.nl, f.abuf, f.bbuf, f.etab, f.etab_b, f.rp, f.part, f.series, f.counter, f.k2tab};
    for (void *p : ps)
        if (p) dev_free(p);
    f.a = f.a1 = f.nl = f.abuf = f.bbuf = nullptr;
    f.k2tab = nullptr;
    f.etab = f.etab_b = nullptr;
    f.rp = nullptr;
    f.part = f.series = nullptr;
    f.counter = nullptr;
}

static cudaError_t launch_update(FusedRun &f, const FzUpdate &u, cudaStream_t s) {
    if (f.cube) k_fused_update<false><<<dim3(f.nparts, f.nr), 256, 0, s>>>(f.a, f.a1, f.nl, f.etab, f.rp, u, f.part);
    else k_fused_update<true><<<dim3(f.nparts, f.nr), 256, 0, s>>>(f.a, f.a1, f.nl, f.etab, f.rp, u, f.part);
    return cudaGetLastError();
}

static cudaError_t launch_energy_final(FusedRun &f, int *flags, cudaStream_t s) {
    k_fz_energy_final<<<f.nr, 256, 0, s>>>(f.part, f.nparts, f.series, f.cap, f.counter, flags);
    return cudaGetLastError();
}

// The same pass on the magnetic block: input and output pointers shifted by
// the blocks' offsets.
static FzPass mag(FzPass p, long in_off, long out_off) {
    p.in += in_off;
    p.out += out_off;
    return p;
}

// One RK2 step of an MHD group: passes A, B on both blocks (u, w and b, j),
// the MHD pass C, passes D, E on both blocks, then the velocity update (with
// its energy partials) and the induction update.
static cudaError_t fused_step_mhd(FusedRun &f, int *flags, cudaStream_t s, Tracer *tr) {
    cudaError_t e;
    for (int stage = 1; stage <= 2; stage++) {
        FzPass A, B, D, Ep;
        pass_descs(f, stage == 1 ? f.a : f.a1, A, B, D, Ep);
        const FzPass Am = mag(A, f.blk_s, f.blk_A), Bm = mag(B, f.blk_A, f.blk_B),
                     Dm = mag(D, f.blk_B, f.blk_A), Em = mag(Ep, f.blk_A, f.blk_s);
        if ((e = NSK_TIMED(tr, "fused_A_x_inverse_curl", run_pass(f, 0, f.sp[0], A, s))) != cudaSuccess) return e;
        if ((e = NSK_TIMED(tr, "fused_A_x_inverse_curl", run_pass(f, 0, f.sp[0], Am, s))) != cudaSuccess) return e;
        if ((e = NSK_TIMED(tr, "fused_B_y_inverse", run_pass(f, 1, f.sp[1], B, s))) != cudaSuccess) return e;
        if ((e = NSK_TIMED(tr, "fused_B_y_inverse", run_pass(f, 1, f.sp[1], Bm, s))) != cudaSuccess) return e;
        if ((e = NSK_TIMED(tr, "fused_C_z_mhd", launch_zm(f, f.zm_E, f.zm_wpb, s))) != cudaSuccess) return e;
        if ((e = NSK_TIMED(tr, "fused_D_y_forward", run_pass(f, 2, f.sp[2], D, s))) != cudaSuccess) return e;
        if ((e = NSK_TIMED(tr, "fused_D_y_forward", run_pass(f, 2, f.sp[2], Dm, s))) != cudaSuccess) return e;
        if ((e = NSK_TIMED(tr, "fused_E_x_forward", run_pass(f, 3, f.sp[3], Ep, s))) != cudaSuccess) return e;
        if ((e = NSK_TIMED(tr, "fused_E_x_forward", run_pass(f, 3, f.sp[3], Em, s))) != cudaSuccess) return e;
        FzUpdate u = make_update(f, stage, f.nparts);
        if ((e = NSK_TIMED(tr, "fused_update", launch_update(f, u, s))) != cudaSuccess) return e;
        e = NSK_TIMED(tr, "fused_update_b",
                      (k_fused_update_b<<<dim3(f.nparts_upd, f.nr), 256, 0, s>>>(
                           f.a + f.blk_s, f.a1 + f.blk_s, f.nl + f.blk_s, f.etab_b, f.rp, u),
                       cudaGetLastError()));
        if (e != cudaSuccess) return e;
    }
    return NSK_TIMED(tr, "energy_final", launch_energy_final(f, flags, s));
}

cudaError_t fused_step(FusedRun &f, int *flags, cudaStream_t s, Tracer *tr) {
    f.flags = flags;
    if (f.mhd) return fused_step_mhd(f, flags, s, tr);
    cudaError_t e;
    for (int stage = 1; stage <= 2; stage++) {
        FzPass A, B, D, Ep;
        pass_descs(f, stage == 1 ? f.a : f.a1, A, B, D, Ep);
        e = NSK_TIMED(tr, "fused_A_x_inverse_curl", run_pass(f, 0, f.sp[0], A, s));
        if (e != cudaSuccess) return e;
        e = NSK_TIMED(tr, "fused_B_y_inverse", run_pass(f, 1, f.sp[1], B, s));
        if (e != cudaSuccess) return e;
        e = NSK_TIMED(tr, "fused_C_z_nonlinear", launch_z(f, f.zc, s));
        if (e != cudaSuccess) return e;
        e = NSK_TIMED(tr, "fused_D_y_forward", run_pass(f, 2, f.sp[2], D, s));
        if (e != cudaSuccess) return e;
        if (f.eu_E) {
            e = NSK_TIMED(tr, "fused_E_x_forward_update", launch_eu(f, f.eu_E, f.eu_ct, stage, s));
            if (e != cudaSuccess) return e;
            continue;
        }
        e = NSK_TIMED(tr, "fused_E_x_forward", run_pass(f, 3, f.sp[3], Ep, s));
        if (e != cudaSuccess) return e;
        FzUpdate u = make_update(f, stage, f.nparts);
        e = NSK_TIMED(tr, "fused_update", launch_update(f, u, s));
        if (e != cudaSuccess) return e;
    }
    return NSK_TIMED(tr, "energy_final", launch_energy_final(f, flags, s));
}

int fused_describe(const FusedRun &f, char *out, int len) {
    const char *names[4] = {"A_x_inverse_curl", "B_y_inverse", "D_y_forward", "E_x_forward"};
    int w = snprintf(out, len, "{");
    for (int i = 0; i < 4 && w < len; i++)
        w += snprintf(out + w, len - w,
                      "\"%s\": {\"kernel\": \"%s\", \"E\": %d, \"cols_per_cta\": %d}, ", names[i],
                      f.sp[i].kind == 2   ? "constant geometry"
                      : f.sp[i].kind == 1 ? "compile-time length"
                                          : "runtime length",
                      f.sp[i].pl.E,
                      f.sp[i].ct);
    if (w < len && f.mhd)
        w += snprintf(out + w, len - w, "\"C_z_mhd\": {\"E\": %d, \"warps_per_cta\": %d}, ", f.zm_E,
                      f.zm_wpb);
    if (w < len && f.eu_E)
        w += snprintf(out + w, len - w, "\"E_fused_with_update\": {\"E\": %d, \"cols_per_cta\": %d}, ",
                      f.eu_E, f.eu_ct);
    else if (w < len)
        w += snprintf(out + w, len - w, "\"E_fused_with_update\": null, ");
    if (w < len && f.zc.kind == 2)
        w += snprintf(out + w, len - w,
                      "\"C_z_nonlinear\": {\"kernel\": \"register-resident\", \"E\": %d, "
                      "\"warps_per_cta\": %d, \"parked_fields\": %d, \"loads\": \"%s\"}}",
                      f.zc.pl.E, (f.zc.ct % ZR_ASYNC) % ZR_PARK, (f.zc.ct % ZR_ASYNC) / ZR_PARK,
                      f.zc.ct / ZR_ASYNC == 2   ? "bulk copies, two fields ahead"
                      : f.zc.ct / ZR_ASYNC == 1 ? "per-lane asynchronous copies, two fields ahead"
                                                : "registers, one field ahead");
    else if (w < len && f.zc.kind == 1)
        w += snprintf(out + w, len - w,
                      "\"C_z_nonlinear\": {\"kernel\": \"compile-time length\", \"E\": %d, "
                      "\"warps_per_cta\": %d}}",
                      f.zc.pl.E, f.zc.ct);
    else if (w < len)
        w += snprintf(out + w, len - w,
                      "\"C_z_nonlinear\": {\"E\": %d, \"stages\": %d, \"lines_per_cta\": %d}}",
                      f.zc.pl.E, f.zc.pl.nst, f.zc.ct);
    return w;
}

cudaError_t fused_set_state(FusedRun &f, int run, int field, const double2 *src, int on_device, void *staging,
                            size_t staging_bytes, cudaStream_t s) {
    const int n = f.n, nh = f.nz / 2 + 1;
    const long plane = (long)f.ny * nh, M = (long)n * plane;
    const int pc = on_device ? n : (int)std::max<size_t>(1, staging_bytes / (plane * sizeof(double2)));
    if (field != 0 && !(field == 1 && f.mhd)) return cudaErrorInvalidValue;
    float2 *a = f.a + field * f.blk_s + (long)run * 3 * f.M;
    const int dealias = f.p[run].dealias;
    cudaError_t e;
    if ((e = cudaMemsetAsync(a, 0, 3 * f.M * sizeof(float2), s)) != cudaSuccess) return e;
    const int ranges[2][2] = {{0, f.K + 1}, {n - f.K, n}};
    for (int c = 0; c < 3; c++) {
        for (auto &r : ranges) {
            for (int kx0 = r[0]; kx0 < r[1]; kx0 += pc) {
                const int cnt = std::min(pc, r[1] - kx0);
                const double2 *p = src + c * M + (long)kx0 * plane;
                if (!on_device) {
                    if ((e = cudaMemcpyAsync(staging, p, cnt * plane * sizeof(double2),
                                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
                        return e;
                    p = (const double2 *)staging;
                }
                const long work = (long)cnt * f.My * f.Mz;
                k_fz_load<<<grid_of(work, 256, 152L * 16), 256, 0, s>>>(p, a + c * f.M, kx0, cnt, half_geom(f),
                                                                      dealias);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                if (!on_device && (e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}

cudaError_t fused_get_state(FusedRun &f, int run, int field, double2 *dst, int on_device, void *staging,
                            size_t staging_bytes, cudaStream_t s) {
    const int n = f.n, nh = f.nz / 2 + 1;
    const long plane = (long)f.ny * nh, M = (long)n * plane;
    const int pc = on_device ? n : (int)std::max<size_t>(1, staging_bytes / (plane * sizeof(double2)));
    if (field != 0 && !(field == 1 && f.mhd)) return cudaErrorInvalidValue;
    const float2 *a = f.a + field * f.blk_s + (long)run * 3 * f.M;
    cudaError_t e;
    for (int c = 0; c < 3; c++) {
        for (int kx0 = 0; kx0 < n; kx0 += pc) {
            const int cnt = std::min(pc, n - kx0);
            double2 *out = dst + c * M + (long)kx0 * plane;
            double2 *d = on_device ? out : (double2 *)staging;
            const long work = (long)cnt * plane;
            k_fz_store<double2><<<grid_of(work, 256, 152L * 16), 256, 0, s>>>(a + c * f.M, d, kx0, cnt,
                                                                            half_geom(f));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if (!on_device) {
                if ((e = cudaMemcpyAsync(out, staging, work * sizeof(double2), cudaMemcpyDeviceToHost,
                                         s)) != cudaSuccess)
                    return e;
                if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}

cudaError_t fused_expand(FusedRun &f, int run, int field, float2 *dst, cudaStream_t s) {
    if (field != 0 && !(field == 1 && f.mhd)) return cudaErrorInvalidValue;
    const float2 *a = f.a + field * f.blk_s + (long)run * 3 * f.M;
    const long M = (long)f.n * f.ny * (f.nz / 2 + 1);
    for (int c = 0; c < 3; c++) {
        k_fz_store<float2><<<grid_of(M, 256, 152L * 16), 256, 0, s>>>(a + c * f.M, dst + c * M, 0, f.n, half_geom(f));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t fused_spectrum(FusedRun &f, int run, int field, int nbins, double *spec, double *ens,
                           cudaStream_t s) {
    if (field != 0 && !(field == 1 && f.mhd)) return cudaErrorInvalidValue;
    CompactAcc acc{f.a + field * f.blk_s + (long)run * 3 * f.M, f.K, f.Mx, f.Mz, f.M};
    return shell_launch(k_shell_spectrum<CompactAcc>, nbins, spec, ens, s, acc, f.n, nbins);
}

cudaError_t fused_helicity(FusedRun &f, int run, int nbins, double *spec, double *aux, cudaStream_t s) {
    CompactHelAcc acc{f.a + (long)run * 3 * f.M, f.K, f.Mx, f.Mz, f.M};
    return shell_launch(k_shell_spectrum<CompactHelAcc>, nbins, spec, aux, s, acc, f.n, nbins);
}

}  // namespace nsk
