// fft_std_ct.cu -- the standalone FP32 3D transforms (ns_fft_r2c, ns_fft_c2r;
// Sec. 2, Fig. 1) on compile-time-length kernels: the strided x and y passes
// reuse the column machinery of the fused form with every row present (the y
// pass flattens (x, kz) into columns, so no tile is ragged), and the z pass is
// a warp-level r2c / c2r with the line in shared memory.
#include "fft_ct.cuh"
#include "fused.h"
#include "fused_access.cuh"

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

// Shapes of the standalone transform for grid size N: the strided passes'
// (E, columns per CTA) and the z pass's (E, warps per CTA).
static bool std_shapes(int N, bool fwd, FzsKernel *kx, FzsKernel *ky, int *ct, ZctKernel *kz) {
    const bool three = N % 3 == 0;
    const int Es = N == 1024 ? 32 : (three ? 12 : 16);
    const int Ez = three ? 12 : 16;
    *ct = 16;
    const bool okx = fwd ? fzs_lookup_PF(N, Es, 16, kx) : fzs_lookup_PI(N, Es, 16, kx);
    const bool oky = fwd ? fzs_lookup_PF(N, Es, 16, ky) : fzs_lookup_PI(N, Es, 16, ky);
    return okx && oky && zstd_lookup(N, fwd, Ez, 2, kz);
}

// Column descriptors of the y and x passes over ncomp half-layout fields
// [c][x][y][kz] (kz < Nh): y pass columns (x, kz), x pass columns (y, kz).
static void std_descs(const float2 *in, float2 *out, int N, int ncomp, FzPass &py, FzPass &px,
                      bool y_first_in) {
    const long Nh = N / 2 + 1, plane = (long)N * Nh, M = (long)N * plane;
    (void)y_first_in;
    py = FzPass{in, out, plane, M, Nh, M, Nh, plane, ncomp, (int)Nh, 0, 0, 0, 0, plane};
    px = FzPass{in, out, plane, M, plane, M, plane, Nh, ncomp, (int)Nh, 0, 0, 0, 0, Nh};
}

bool std_r2c_fp32(const float *in, float2 *out, int N, int ncomp, const float2 *tw, cudaStream_t s,
                  cudaError_t *err) {
    FzsKernel kx, ky;
    ZctKernel kz;
    int ct;
    if (!std_shapes(N, true, &kx, &ky, &ct, &kz)) return false;
    *err = launch_zstd(kz, in, out, (long)ncomp * N * N, tw, s);
    if (*err != cudaSuccess) return true;
    FzPass py, px;
    std_descs(out, out, N, ncomp, py, px, false);
    *err = launch_col(ky, py, ct, tw, s);
    if (*err != cudaSuccess) return true;
    *err = launch_col(kx, px, ct, tw, s);
    return true;
}

bool std_c2r_fp32(const float2 *in, float2 *tmp, float *out, int N, const float2 *tw, cudaStream_t s,
                  cudaError_t *err) {
    FzsKernel kx, ky;
    ZctKernel kz;
    int ct;
    if (!std_shapes(N, false, &kx, &ky, &ct, &kz)) return false;
    FzPass py, px;
    std_descs(in, tmp, N, 1, py, px, true);
    *err = launch_col(kx, px, ct, tw, s);
    if (*err != cudaSuccess) return true;
    std_descs(tmp, tmp, N, 1, py, px, false);
    *err = launch_col(ky, py, ct, tw, s);
    if (*err != cudaSuccess) return true;
    *err = launch_zstd(kz, tmp, out, (long)N * N, tw, s);
    return true;
}

}  // namespace nsk
