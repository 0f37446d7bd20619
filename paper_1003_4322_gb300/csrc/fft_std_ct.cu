// fft_std_ct.cu -- the standalone FP32 3D transforms (ns_fft_r2c, ns_fft_c2r,
// and their grid forms; Sec. 2, Fig. 1) on compile-time-length kernels, one
// length per axis: the strided x and y passes
// reuse the column machinery of the fused form with every row present (the y
// pass flattens (x, kz) into columns, so no tile is ragged), and the z pass is
// a warp-level r2c / c2r with the line in shared memory.
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>

#include "fft_ct.cuh"
#include "fused.h"
#include "fused_access.cuh"
#include "ns_internal.h"

namespace nsk {

template <int N, int E_> struct ZStdShape {
    static constexpr int n = N / 2;
    static constexpr int E = E_;
    static constexpr int T = n / E;
    static constexpr bool ok = n % E == 0 && ct_valid(n, E) && T >= 1 && T <= 32 && 32 % T == 0;
    static constexpr int LPW = ok ? 32 / T : 1;
    static constexpr int LS = ok ? ct_line_stride(n, E, 1) : 1;
};

// r2c of nlines lines of N reals into N/2+1 complex values each.
template <int N, int E, int WPB>
__global__ void __launch_bounds__(32 * WPB)
k_z_r2c_ct(const float *__restrict__ in, float2 *__restrict__ out, long nlines,
           const float2 *__restrict__ tw) {
    typedef ZStdShape<N, E> Z;
    constexpr int n = Z::n, T = Z::T, LPW = Z::LPW, LS = Z::LS;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ll = lane / T, slot = lane % T;
    const long line = ((long)blockIdx.x * WPB + warp) * LPW + ll;
    const bool valid = line < nlines;
    float2 *L = sm + (long)(warp * LPW + ll) * LS;
    auto sl = [&](int e) -> float2 { return L[ct_skew(e)]; };
    auto ss = [&](int e, float2 v) { L[ct_skew(e)] = v; };
    const float2 *src = reinterpret_cast<const float2 *>(in + line * N);
    float2 x[E];
#pragma unroll
    for (int j = 0; j < E; j++) x[j] = valid ? src[slot + j * T] : make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < E; j++) ss(slot + j * T, x[j]);
    __syncwarp();
    ct_fft_smem<n, E, -1, N>(slot, tw, sl, ss);
    if (!valid) return;
    float2 *dst = out + line * (n + 1);
    // X[k] = (Z[k] + conj Z[n-k])/2 - i W^k (Z[k] - conj Z[n-k])/2, k = 0..n
#pragma unroll
    for (int j = 0; j <= E; j++) {
        const int k = slot + j * T;
        if (k > n) break;
        const float2 zk = sl(k == n ? 0 : k);
        const float2 zc = cconj(sl(k == 0 || k == n ? 0 : n - k));
        const float2 ev = cscale(cadd(zk, zc), 0.5f);
        const float2 od = cmul_i<-1>(cscale(csub(zk, zc), 0.5f));
        dst[k] = cadd(ev, cmul(od, __ldg(tw + k)));
    }
}

// c2r of nlines lines of N/2+1 complex values into N reals each (real parts of
// the kz = 0 and N/2 entries).
template <int N, int E, int WPB>
__global__ void __launch_bounds__(32 * WPB)
k_z_c2r_ct(const float2 *__restrict__ in, float *__restrict__ out, long nlines,
           const float2 *__restrict__ tw) {
    typedef ZStdShape<N, E> Z;
    constexpr int n = Z::n, T = Z::T, LPW = Z::LPW, LS = Z::LS;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ll = lane / T, slot = lane % T;
    const long line = ((long)blockIdx.x * WPB + warp) * LPW + ll;
    const bool valid = line < nlines;
    float2 *L = sm + (long)(warp * LPW + ll) * LS;
    auto sl = [&](int e) -> float2 { return L[ct_skew(e)]; };
    auto ss = [&](int e, float2 v) { L[ct_skew(e)] = v; };
    const float2 *src = in + line * (n + 1);
    float2 xk[E], xm[E];
#pragma unroll
    for (int j = 0; j < E; j++) {
        const int k = slot + j * T;
        xk[j] = valid ? src[k] : make_float2(0.f, 0.f);
        xm[j] = valid ? src[n - k] : make_float2(0.f, 0.f);
    }
    // Z[k] = (X[k] + conj X[n-k]) + i W^{-k} (X[k] - conj X[n-k])
#pragma unroll
    for (int j = 0; j < E; j++) {
        const int k = slot + j * T;
        float2 a0 = xk[j], am = xm[j];
        if (k == 0) {
            a0.y = 0.f;
            am.y = 0.f;
        }
        const float2 xc = cconj(am);
        const float2 wb = cmulc(csub(a0, xc), __ldg(tw + k));
        ss(k, cadd(cadd(a0, xc), cmul_i<1>(wb)));
    }
    __syncwarp();
    ct_fft_smem<n, E, +1, N>(slot, tw, sl, ss);
    if (!valid) return;
    float2 *dst = reinterpret_cast<float2 *>(out + line * N);
#pragma unroll
    for (int j = 0; j < E; j++) dst[slot + j * T] = sl(slot + j * T);
}

template <int N, int E, int WPB> static bool zstd_entry(bool r2c, ZctKernel *o) {
    typedef ZStdShape<N, E> Z;
    if constexpr (!Z::ok) {
        return false;
    } else {
        o->k = r2c ? (const void *)k_z_r2c_ct<N, E, WPB> : (const void *)k_z_c2r_ct<N, E, WPB>;
        o->smem = (size_t)WPB * Z::LPW * Z::LS * sizeof(float2);
        o->lines_per_block = WPB * Z::LPW;
        o->threads = 32 * WPB;
        return true;
    }
}

template <int N> static bool zstd_by(bool r2c, int E, int wpb, ZctKernel *o) {
    constexpr bool three = (N / 2) % 3 == 0;
    constexpr int Ebig = three ? 12 : 16, Esmall = three ? 6 : 8;
    if (E == Ebig && wpb == 2) return zstd_entry<N, Ebig, 2>(r2c, o);
    if (E == Ebig && wpb == 4) return zstd_entry<N, Ebig, 4>(r2c, o);
    if (E == Esmall && wpb == 2) return zstd_entry<N, Esmall, 2>(r2c, o);
    if (E == Esmall && wpb == 4) return zstd_entry<N, Esmall, 4>(r2c, o);
    return false;
}

bool zstd_lookup(int N, bool r2c, int E, int wpb, ZctKernel *o) {
    switch (N) {
    case 64: return zstd_by<64>(r2c, E, wpb, o);
    case 96: return zstd_by<96>(r2c, E, wpb, o);
    case 128: return zstd_by<128>(r2c, E, wpb, o);
    case 192: return zstd_by<192>(r2c, E, wpb, o);
    case 256: return zstd_by<256>(r2c, E, wpb, o);
    case 384: return zstd_by<384>(r2c, E, wpb, o);
    case 512: return zstd_by<512>(r2c, E, wpb, o);
    case 768: return zstd_by<768>(r2c, E, wpb, o);
    case 1024: return zstd_by<1024>(r2c, E, wpb, o);
    }
    return false;
}

// ---------------------------------------------------------------- host side

static cudaError_t launch_zstd(const ZctKernel &z, const void *in, void *out, long nlines,
                               const float2 *tw, cudaStream_t s) {
    cudaError_t e = allow_smem(z.k, z.smem);
    if (e != cudaSuccess) return e;
    const long blocks = (nlines + z.lines_per_block - 1) / z.lines_per_block;
    void *args[] = {(void *)&in, (void *)&out, (void *)&nlines, (void *)&tw};
    return cudaLaunchKernel(z.k, dim3((unsigned)blocks), dim3(z.threads), args, z.smem, s);
}

static cudaError_t launch_col(const FzsKernel &k, const FzPass &ps, int ct, const float2 *tw,
                              cudaStream_t s) {
    cudaError_t e = allow_smem(k.k, k.smem);
    if (e != cudaSuccess) return e;
    const long blocks = (ps.ncols + ct - 1) / ct * ps.nfields;
    FzPass p = ps;
    void *args[] = {(void *)&p, (void *)&tw};
    return cudaLaunchKernel(k.k, dim3((unsigned)blocks), dim3(k.threads), args, k.smem, s);
}

// Tuned shapes of the standalone transform for one (N, direction): the x
// and y passes' (E, columns per CTA) and the z pass's (E, warps per CTA).
struct StdShapes {
    int ex = 0, cx = 0, ey = 0, cy = 0, ez = 0, wz = 0;
    int zreg = 0;      // z pass: 0 line in shared memory (zstd), 1 register-resident (zreg)
    bool ok = false;   // false: no compiled kernel for some axis (the caller falls back)
};

// Register-resident z-pass candidates (fft_std_reg.cu).
bool zreg_lookup(int N, bool r2c, int E, ZctKernel *o);

static bool z_kernel(const StdShapes &sh, int N, bool r2c, ZctKernel *z) {
    return sh.zreg ? zreg_lookup(N, r2c, sh.ez, z) : zstd_lookup(N, r2c, sh.ez, sh.wz, z);
}

static bool std_lookup_col(bool fwd, int N, int E, int CT, FzsKernel *k) {
    return fwd ? fzs_lookup_PF(N, E, CT, k) : fzs_lookup_PI(N, E, CT, k);
}

template <class F> static float std_time(F launch, cudaStream_t s) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.f;
    }
    float ms = -1.f;
    if (launch() == cudaSuccess && cudaEventRecord(a, s) == cudaSuccess) {
        bool ok = true;
        for (int i = 0; i < 3 && ok; i++) ok = launch() == cudaSuccess;
        if (ok && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
            ms /= 3;
        else
            ms = -1.f;
    }
    cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

// Column descriptors of the y and x passes over ncomp half-layout fields
// [c][x][y][kz] of an nx x ny x nz grid (kz < Nh = nz/2 + 1): y pass columns
// (x, kz), x pass columns (y, kz).
static void std_descs(const float2 *in, float2 *out, const StdGrid &g, int ncomp, FzPass &py, FzPass &px) {
    const long Nh = g.nz / 2 + 1, plane = (long)g.ny * Nh, M = (long)g.nx * plane;
    py = FzPass{in, out, (long)g.nx * Nh, M, Nh, M, Nh, plane, ncomp, (int)Nh, 0, 0, 0, 0, plane};
    px = FzPass{in, out, plane, M, plane, M, plane, Nh, ncomp, (int)Nh, 0, 0, 0, 0, Nh};
}

// Choose the shapes on the first call for (grid, direction), timing every
// compiled candidate on the call's own buffers (the passes run in place on
// `work`, whose contents the real transform then overwrites); kept for the
// life of the process.  NS_FORCE_STD_Z=smem, =reg or =pf restricts the z pass
// to one kernel family (so that tests can run each).
static bool std_shapes(const StdGrid &g, bool fwd, const void *zin, void *zout, float2 *work, int ncomp,
                       cudaStream_t s, StdShapes *out) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, bool, int>, StdShapes> cache;
    const char *fz = getenv("NS_FORCE_STD_Z");
    const bool try_smem = !fz || strcmp(fz, "smem") == 0, try_reg = !fz || strcmp(fz, "reg") == 0,
               try_pf = !fz || strcmp(fz, "pf") == 0;
    const auto key = std::make_tuple(g.nx, g.ny, g.nz, fwd, (int)try_smem + 2 * (int)try_reg + 4 * (int)try_pf);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *out = it->second;
            return out->ok;
        }
    }
    FzsKernel k;
    ZctKernel z;
    // every axis needs a compiled kernel before anything is launched (a miss is
    // remembered, so later calls, possibly inside a graph capture, launch nothing)
    {
        bool hx = false, hy = false, hz = false;
        const int Ec[] = {6, 8, 12, 16, 32, 106, 108, 112, 116};
        for (int E : Ec)
            for (int ct = 8; ct <= 16; ct *= 2) {
                hx = hx || std_lookup_col(fwd, g.nx, E, ct, &k);
                hy = hy || std_lookup_col(fwd, g.ny, E, ct, &k);
            }
        for (int E : Ec)
            for (int w = 2; w <= 4; w *= 2) hz = hz || zstd_lookup(g.nz, fwd, E, w, &z);
        for (int E : Ec) hz = hz || zreg_lookup(g.nz, fwd, E, &z);
        if (!hx || !hy || !hz) {
            std::lock_guard<std::mutex> lk(mu);
            cache[key] = StdShapes{};
            return false;
        }
    }
    const int Es[] = {8, 12, 16, 32};
    StdShapes best;
    float bx = -1.f, by = -1.f, bz = -1.f;
    FzPass py, px;
    std_descs(work, work, g, ncomp, py, px);
    for (int E : Es)
        for (int ct = 8; ct <= 16; ct *= 2) {
            if (std_lookup_col(fwd, g.ny, E, ct, &k)) {
                const float ty = std_time([&]() { return launch_col(k, py, ct, g.twy, s); }, s);
                if (ty > 0.f && (by < 0.f || ty < by)) { by = ty; best.ey = E; best.cy = ct; }
            }
            if (std_lookup_col(fwd, g.nx, E, ct, &k)) {
                const float tx = std_time([&]() { return launch_col(k, px, ct, g.twx, s); }, s);
                if (tx > 0.f && (bx < 0.f || tx < bx)) { bx = tx; best.ex = E; best.cx = ct; }
            }
        }
    const int Ezs[] = {16, 12, 8, 6};
    const long nlines = (long)(fwd ? ncomp : 1) * g.nx * g.ny;
    for (int E : Ezs)
        for (int w = 2; w <= 4 && try_smem; w *= 2) {
            if (!zstd_lookup(g.nz, fwd, E, w, &z)) continue;
            const float t = std_time([&]() { return launch_zstd(z, zin, zout, nlines, g.twz, s); }, s);
            if (t > 0.f && (bz < 0.f || t < bz)) { bz = t; best.ez = E; best.wz = w; best.zreg = 0; }
        }
    const int Eregs[] = {16, 12, 8, 6, 116, 112, 108, 106};   // E + 100: prefetching form
    for (int E : Eregs) {
        if (!(E < 100 ? try_reg : try_pf) || !zreg_lookup(g.nz, fwd, E, &z)) continue;
        const float t = std_time([&]() { return launch_zstd(z, zin, zout, nlines, g.twz, s); }, s);
        if (t > 0.f && (bz < 0.f || t < bz)) { bz = t; best.ez = E; best.wz = 4; best.zreg = 1; }
    }
    best.ok = bx >= 0.f && by >= 0.f && bz >= 0.f;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = best;
    *out = best;
    return best.ok;
}

bool std_r2c_fp32_grid(const float *in, float2 *out, const StdGrid &g, int ncomp, cudaStream_t s,
                       cudaError_t *err) {
    StdShapes sh;
    if (!std_shapes(g, true, in, out, out, ncomp, s, &sh)) return false;
    FzsKernel kx, ky;
    ZctKernel kz;
    if (!std_lookup_col(true, g.nx, sh.ex, sh.cx, &kx) || !std_lookup_col(true, g.ny, sh.ey, sh.cy, &ky) ||
        !z_kernel(sh, g.nz, true, &kz))
        return false;
    *err = launch_zstd(kz, in, out, (long)ncomp * g.nx * g.ny, g.twz, s);
    if (*err != cudaSuccess) return true;
    FzPass py, px;
    std_descs(out, out, g, ncomp, py, px);
    *err = launch_col(ky, py, sh.cy, g.twy, s);
    if (*err != cudaSuccess) return true;
    *err = launch_col(kx, px, sh.cx, g.twx, s);
    return true;
}

bool std_c2r_fp32_grid(const float2 *in, float2 *tmp, float *out, const StdGrid &g, cudaStream_t s,
                       cudaError_t *err) {
    StdShapes sh;
    if (!std_shapes(g, false, tmp, out, tmp, 1, s, &sh)) return false;
    FzsKernel kx, ky;
    ZctKernel kz;
    if (!std_lookup_col(false, g.nx, sh.ex, sh.cx, &kx) || !std_lookup_col(false, g.ny, sh.ey, sh.cy, &ky) ||
        !z_kernel(sh, g.nz, false, &kz))
        return false;
    FzPass py, px;
    std_descs(in, tmp, g, 1, py, px);
    *err = launch_col(kx, px, sh.cx, g.twx, s);
    if (*err != cudaSuccess) return true;
    std_descs(tmp, tmp, g, 1, py, px);
    *err = launch_col(ky, py, sh.cy, g.twy, s);
    if (*err != cudaSuccess) return true;
    *err = launch_zstd(kz, tmp, out, (long)g.nx * g.ny, g.twz, s);
    return true;
}

bool std_r2c_fp32(const float *in, float2 *out, int N, int ncomp, const float2 *tw, cudaStream_t s,
                  cudaError_t *err) {
    return std_r2c_fp32_grid(in, out, StdGrid{N, N, N, tw, tw, tw}, ncomp, s, err);
}

bool std_c2r_fp32(const float2 *in, float2 *tmp, float *out, int N, const float2 *tw, cudaStream_t s,
                  cudaError_t *err) {
    return std_c2r_fp32_grid(in, tmp, out, StdGrid{N, N, N, tw, tw, tw}, s, err);
}

}  // namespace nsk
