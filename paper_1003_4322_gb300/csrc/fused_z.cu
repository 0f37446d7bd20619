// fused_z.cu -- pass C of the fused form for compile-time grid sizes.
//
// Pass C (z c2r of u and w, the cross product u x w on the grid, z r2c of
// the product; Sec. 2, Eqs. 1-2) is the arithmetic-heaviest pass: nine
// length-N/2 transforms per (y, x) line for every 9 * N/3 complex values that
// cross HBM.  Here one warp owns whole lines (32 / T lines of T = N/2 / E
// threads each) and works through the six fields one after another, so the
// exchange between Stockham stages needs only __syncwarp, and with N fixed
// at compile time every index, stride and span is a constant.
#include "fft_ct.cuh"
#include "fused.h"

namespace nsk {

// Shape of pass C for grid size N with E elements per thread: T threads per
// line, 32 / T lines per warp.  `ok` is false when E does not suit N/2 or a
// line would not fit one warp.
template <int N, int E_> struct ZShape {
    static constexpr int n = N / 2;
    static constexpr int E = E_;
    static constexpr int T = n / E;
    static constexpr bool ok = n % E == 0 && ct_valid(n, E) && T >= 1 && T <= 32 && 32 % T == 0;
    static constexpr int LPW = ok ? 32 / T : 1;                 // lines per warp
    static constexpr int LS = ok ? ct_line_stride(n, E, 6) : 1; // elements per field line
};

template <int N, int E, int WPB>
__global__ void __launch_bounds__(32 * WPB)
k_fused_z_ct(float2 *buf, long fs, int Mz, long nlines, long brun, const float2 *__restrict__ tw) {
    typedef ZShape<N, E> Z;
    buf += blockIdx.y * brun;   // run of the group
    constexpr int n = Z::n, T = Z::T, LPW = Z::LPW, LS = Z::LS;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ll = lane / T, slot = lane % T;
    const long line = ((long)blockIdx.x * WPB + warp) * LPW + ll;
    const bool valid = line < nlines;
    float2 *L6 = sm + (long)(warp * LPW + ll) * 6 * LS;

    // Stage twiddles and the packing twiddles W^k, k = slot + j T, stay in
    // registers for all nine transforms of the line.
    CtTwiddles<n, E, N> twr;
    twr.load(slot, tw);
    float2 wk[E];
#pragma unroll
    for (int j = 0; j < E; j++) wk[j] = __ldg(tw + slot + j * T);

    // c2r of the six fields: Z[k] = (X[k] + conj X[n-k]) + i W^{-k} (X[k] - conj X[n-k]),
    // X[k] = 0 for k >= Mz, real parts of X[0] and X[n]; then one inverse
    // length-n FFT leaves the 2n real samples in natural order.  The loads of
    // field f + 1 are issued before the transform of field f.
    float2 xk[E], xm[E];
    auto fetch = [&](int f) {
        const float2 *src = buf + f * fs + line * Mz;
#pragma unroll
        for (int j = 0; j < E; j++) {
            const int k = slot + j * T;
            xk[j] = (valid && k < Mz) ? src[k] : make_float2(0.f, 0.f);
            xm[j] = (valid && n - k < Mz) ? src[n - k] : make_float2(0.f, 0.f);
        }
    };
    fetch(0);
    for (int f = 0; f < 6; f++) {
        float2 *Lf = L6 + f * LS;
        auto sl = [&](int e) -> float2 { return Lf[ct_skew(e)]; };
        auto ss = [&](int e, float2 v) { Lf[ct_skew(e)] = v; };
#pragma unroll
        for (int j = 0; j < E; j++) {
            const int k = slot + j * T;
            float2 a0 = xk[j], am = xm[j];
            if (k == 0) {
                a0.y = 0.f;
                am.y = 0.f;
            }
            const float2 xc = cconj(am);
            const float2 wb = cmulc(csub(a0, xc), wk[j]);
            ss(k, cadd(cadd(a0, xc), cmul_i<1>(wb)));
        }
        if (f < 5) fetch(f + 1);
        __syncwarp();
        ct_fft_smem_tw<n, E, +1, N>(slot, twr, sl, ss);
    }

    // u x w at the 2n points (complex element m holds points 2m and 2m + 1)
#pragma unroll
    for (int j = 0; j < E; j++) {
        float2 *b = L6 + ct_skew(slot + j * T);
        const float2 ux = b[0], uy = b[LS], uz = b[2 * LS];
        const float2 wx = b[3 * LS], wy = b[4 * LS], wz = b[5 * LS];
        b[0] = make_float2(uy.x * wz.x - uz.x * wy.x, uy.y * wz.y - uz.y * wy.y);
        b[LS] = make_float2(uz.x * wx.x - ux.x * wz.x, uz.y * wx.y - ux.y * wz.y);
        b[2 * LS] = make_float2(ux.x * wy.x - uy.x * wx.x, ux.y * wy.y - uy.y * wx.y);
    }
    __syncwarp();

    // r2c of the three products and the kept kz < Mz written over fields 0..2:
    // X[k] = (Z[k] + conj Z[n-k])/2 - i W^k (Z[k] - conj Z[n-k])/2
    for (int f = 0; f < 3; f++) {
        float2 *Lf = L6 + f * LS;
        auto sl = [&](int e) -> float2 { return Lf[ct_skew(e)]; };
        auto ss = [&](int e, float2 v) { Lf[ct_skew(e)] = v; };
        ct_fft_smem_tw<n, E, -1, N>(slot, twr, sl, ss);
        float2 *dst = buf + f * fs + line * Mz;
#pragma unroll
        for (int j = 0; j < E; j++) {
            const int k = slot + j * T;
            if (valid && k < Mz) {
                const float2 zk = sl(k);
                const float2 zc = cconj(sl(k == 0 ? 0 : n - k));
                const float2 ev = cscale(cadd(zk, zc), 0.5f);
                const float2 od = cmul_i<-1>(cscale(csub(zk, zc), 0.5f));
                dst[k] = cadd(ev, cmul(od, wk[j]));
            }
        }
    }
}

template <int N, int E, int WPB> static bool zct_entry(ZctKernel *o) {
    typedef ZShape<N, E> Z;
    if constexpr (!Z::ok) {
        return false;
    } else {
        o->k = (const void *)k_fused_z_ct<N, E, WPB>;
        o->smem = (size_t)WPB * Z::LPW * 6 * Z::LS * sizeof(float2);
        o->lines_per_block = WPB * Z::LPW;
        o->threads = 32 * WPB;
        return true;
    }
}

template <int N, int E> static bool zct_by_wpb(int wpb, ZctKernel *o) {
    switch (wpb) {
    case 1: return zct_entry<N, E, 1>(o);
    case 2: return zct_entry<N, E, 2>(o);
    case 4: return zct_entry<N, E, 4>(o);
    }
    return false;
}

// E = 16 (12 for N divisible by 3) or half of it (8, 6).
template <int N> static bool zct_by_e(int E, int wpb, ZctKernel *o) {
    constexpr bool three = (N / 2) % 3 == 0;
    constexpr int Ebig = three ? 12 : 16, Esmall = three ? 6 : 8;
    if (E == Ebig) return zct_by_wpb<N, Ebig>(wpb, o);
    if (E == Esmall) return zct_by_wpb<N, Esmall>(wpb, o);
    return false;
}

bool zct_lookup(int N, int E, int wpb, ZctKernel *o) {
    switch (N) {
    case 32: return zct_by_e<32>(E, wpb, o);
    case 64: return zct_by_e<64>(E, wpb, o);
    case 96: return zct_by_e<96>(E, wpb, o);
    case 128: return zct_by_e<128>(E, wpb, o);
    case 192: return zct_by_e<192>(E, wpb, o);
    case 256: return zct_by_e<256>(E, wpb, o);
    case 384: return zct_by_e<384>(E, wpb, o);
    case 512: return zct_by_e<512>(E, wpb, o);
    case 768: return zct_by_e<768>(E, wpb, o);
    case 1024: return zct_by_e<1024>(E, wpb, o);
    }
    return false;
}

}  // namespace nsk
