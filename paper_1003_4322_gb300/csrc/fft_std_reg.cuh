// fft_std_reg.cuh -- register-resident z passes of the standalone FP32
// transforms (ns_fft_r2c / ns_fft_c2r and their grid forms; Sec. 2, Fig. 1).
// A line of N reals is the complex line Z[m] = x[2m] + i x[2m+1] of length
// n = N/2, spread over T = n/E threads with E values each.  The length-n FFT
// runs in registers (ct_fft_reg), exchanging through shared memory only
// between stages, and the even/odd packing of the real transform pairs
// position k with n - k through a warp shuffle with the partner lane, so the
// line is read and written once, coalesced, and never staged whole in shared
// memory.  The candidates sit beside the shared-memory line kernels of
// fft_std_ct.cu; the transform's tuner times both.
#pragma once
#include "fused_zr.cuh"   // ct_fft_reg

namespace nsk {

template <int N, int E_> struct ZRegShape {
    static constexpr int n = N / 2;
    static constexpr int E = E_;
    static constexpr int T = n / E;
    static constexpr bool ok = n % E == 0 && ct_valid(n, E) && T >= 1 && T <= 32 && 32 % T == 0;
    static constexpr int LPW = ok ? 32 / T : 1;   // lines per warp
    static constexpr int NST = ok ? ct_nst(n, E) : 1;
    static constexpr int LS = (ok && NST > 1) ? ct_line_stride(n, E, 1) : 0;   // exchange buffer
};

// v of lane src (all 32 lanes take part).
NSK_DEV float2 zreg_shfl(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// r2c output of a transformed line Z (positions slot + jT in v):
// X[k] = (Z[k] + conj Z[n-k])/2 - i W^k (Z[k] - conj Z[n-k])/2 for k < n, and
// X[n] = Re Z[0] - Im Z[0]; Z[n-k] comes from the partner lane (register
// E-1-j), or from this lane's register (E-j) mod E when slot = 0.
template <int n, int E, int T>
NSK_DEV void zreg_r2c_store(const float2 (&v)[E], int slot, int partner, bool valid, float2 *dst,
                            const float2 *__restrict__ tw) {
#pragma unroll
    for (int j = 0; j < E; j++) {
        const int k = slot + j * T;
        float2 zm = zreg_shfl(v[E - 1 - j], partner);
        if (slot == 0) zm = v[(E - j) % E];   // n - jT = (E - j) T, and Z[n] = Z[0]
        const float2 zk = v[j], zc = cconj(zm);
        const float2 ev = cscale(cadd(zk, zc), 0.5f);
        const float2 od = cmul_i<-1>(cscale(csub(zk, zc), 0.5f));
        if (valid) dst[k] = cadd(ev, cmul(od, __ldg(tw + k)));
    }
    if (valid && slot == 0) dst[n] = make_float2(v[0].x - v[0].y, 0.f);
}

// c2r input of a line from X (positions slot + jT in x, X[n] in xn on slot 0):
// Z[k] = (X[k] + conj X[n-k]) + i W^{-k} (X[k] - conj X[n-k]), the imaginary
// parts of X[0] and X[n] dropped.
template <int n, int E, int T>
NSK_DEV void zreg_c2r_pack(const float2 (&x)[E], float2 xn, int slot, int partner, float2 (&v)[E],
                           const float2 *__restrict__ tw) {
#pragma unroll
    for (int j = 0; j < E; j++) {
        const int k = slot + j * T;
        float2 a0 = x[j];
        float2 am = zreg_shfl(x[E - 1 - j], partner);
        if (slot == 0) am = j > 0 ? x[(E - j) % E] : xn;
        if (k == 0) {
            a0.y = 0.f;
            am.y = 0.f;
        }
        const float2 xc = cconj(am);
        const float2 wb = cmulc(csub(a0, xc), __ldg(tw + k));
        v[j] = cadd(cadd(a0, xc), cmul_i<1>(wb));
    }
}

// r2c of nlines lines of N reals into N/2 + 1 complex values each (W = e^{-2 pi i/N}).
template <int N, int E, int WPB>
__global__ void __launch_bounds__(32 * WPB)
k_z_r2c_reg(const float *__restrict__ in, float2 *__restrict__ out, long nlines,
            const float2 *__restrict__ tw) {
    typedef ZRegShape<N, E> Z;
    constexpr int n = Z::n, T = Z::T, LPW = Z::LPW, LS = Z::LS;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ll = lane / T, slot = lane % T;
    const int partner = ll * T + (T - slot) % T;   // holds position n - k of this line
    const long line = ((long)blockIdx.x * WPB + warp) * LPW + ll;
    const bool valid = line < nlines;
    float2 *L = sm + (long)(warp * LPW + ll) * LS;
    auto sl = [&](int e) -> float2 { return L[ct_skew(e)]; };
    auto ss = [&](int e, float2 v) { L[ct_skew(e)] = v; };
    CtTwiddles<n, E, N> twr;
    twr.load(slot, tw);
    const float2 *src = reinterpret_cast<const float2 *>(in + (valid ? line : 0) * N);
    float2 v[E];
#pragma unroll
    for (int j = 0; j < E; j++) v[j] = valid ? src[slot + j * T] : make_float2(0.f, 0.f);
    ct_fft_reg<n, E, -1, N>(v, slot, twr, sl, ss);
    zreg_r2c_store<n, E, T>(v, slot, partner, valid, out + (valid ? line : 0) * (n + 1), tw);
}

// c2r of nlines lines of N/2 + 1 complex values into N reals each: the packed
// line, its inverse length-n FFT, complex element m holding the reals 2m, 2m + 1.
template <int N, int E, int WPB>
__global__ void __launch_bounds__(32 * WPB)
k_z_c2r_reg(const float2 *__restrict__ in, float *__restrict__ out, long nlines,
            const float2 *__restrict__ tw) {
    typedef ZRegShape<N, E> Z;
    constexpr int n = Z::n, T = Z::T, LPW = Z::LPW, LS = Z::LS;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ll = lane / T, slot = lane % T;
    const int partner = ll * T + (T - slot) % T;
    const long line = ((long)blockIdx.x * WPB + warp) * LPW + ll;
    const bool valid = line < nlines;
    float2 *L = sm + (long)(warp * LPW + ll) * LS;
    auto sl = [&](int e) -> float2 { return L[ct_skew(e)]; };
    auto ss = [&](int e, float2 v) { L[ct_skew(e)] = v; };
    CtTwiddles<n, E, N> twr;
    twr.load(slot, tw);
    const float2 *src = in + (valid ? line : 0) * (n + 1);
    float2 x[E];
#pragma unroll
    for (int j = 0; j < E; j++) x[j] = valid ? src[slot + j * T] : make_float2(0.f, 0.f);
    const float2 xn = valid && slot == 0 ? src[n] : make_float2(0.f, 0.f);
    float2 v[E];
    zreg_c2r_pack<n, E, T>(x, xn, slot, partner, v, tw);
    ct_fft_reg<n, E, +1, N>(v, slot, twr, sl, ss);
    if (!valid) return;
    float2 *dst = reinterpret_cast<float2 *>(out + line * N);
#pragma unroll
    for (int j = 0; j < E; j++) dst[slot + j * T] = v[j];
}

// The same two transforms with IT consecutive line groups per warp: the
// input of group i + 1 is loaded into registers while group i is
// transformed, so a warp keeps a line's loads in flight through its FFT, and
// the stage twiddles are loaded once per IT groups.
template <int N, int E, int WPB, int IT>
__global__ void __launch_bounds__(32 * WPB)
k_z_r2c_pf(const float *__restrict__ in, float2 *__restrict__ out, long nlines,
           const float2 *__restrict__ tw) {
    typedef ZRegShape<N, E> Z;
    constexpr int n = Z::n, T = Z::T, LPW = Z::LPW, LS = Z::LS;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ll = lane / T, slot = lane % T;
    const int partner = ll * T + (T - slot) % T;
    const long g0 = ((long)blockIdx.x * WPB + warp) * IT;   // first line group of the warp
    float2 *L = sm + (long)(warp * LPW + ll) * LS;
    auto sl = [&](int e) -> float2 { return L[ct_skew(e)]; };
    auto ss = [&](int e, float2 v) { L[ct_skew(e)] = v; };
    CtTwiddles<n, E, N> twr;
    twr.load(slot, tw);
    float2 nx[E];
    auto fetch = [&](long grp) {
        const long line = grp * LPW + ll;
        const bool ok = line < nlines;
        const float2 *src = reinterpret_cast<const float2 *>(in + (ok ? line : 0) * N);
#pragma unroll
        for (int j = 0; j < E; j++) nx[j] = ok ? src[slot + j * T] : make_float2(0.f, 0.f);
    };
    fetch(g0);
#pragma unroll 1
    for (int it = 0; it < IT; it++) {
        const long line = (g0 + it) * LPW + ll;
        const bool valid = line < nlines;
        float2 v[E];
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = nx[j];
        if (it + 1 < IT) fetch(g0 + it + 1);
        ct_fft_reg<n, E, -1, N>(v, slot, twr, sl, ss);
        zreg_r2c_store<n, E, T>(v, slot, partner, valid, out + (valid ? line : 0) * (n + 1), tw);
    }
}

template <int N, int E, int WPB, int IT>
__global__ void __launch_bounds__(32 * WPB)
k_z_c2r_pf(const float2 *__restrict__ in, float *__restrict__ out, long nlines,
           const float2 *__restrict__ tw) {
    typedef ZRegShape<N, E> Z;
    constexpr int n = Z::n, T = Z::T, LPW = Z::LPW, LS = Z::LS;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ll = lane / T, slot = lane % T;
    const int partner = ll * T + (T - slot) % T;
    const long g0 = ((long)blockIdx.x * WPB + warp) * IT;
    float2 *L = sm + (long)(warp * LPW + ll) * LS;
    auto sl = [&](int e) -> float2 { return L[ct_skew(e)]; };
    auto ss = [&](int e, float2 v) { L[ct_skew(e)] = v; };
    CtTwiddles<n, E, N> twr;
    twr.load(slot, tw);
    float2 nx[E], nn;
    auto fetch = [&](long grp) {
        const long line = grp * LPW + ll;
        const bool ok = line < nlines;
        const float2 *src = in + (ok ? line : 0) * (n + 1);
#pragma unroll
        for (int j = 0; j < E; j++) nx[j] = ok ? src[slot + j * T] : make_float2(0.f, 0.f);
        nn = ok && slot == 0 ? src[n] : make_float2(0.f, 0.f);
    };
    fetch(g0);
#pragma unroll 1
    for (int it = 0; it < IT; it++) {
        const long line = (g0 + it) * LPW + ll;
        const bool valid = line < nlines;
        float2 x[E];
#pragma unroll
        for (int j = 0; j < E; j++) x[j] = nx[j];
        const float2 xn = nn;
        if (it + 1 < IT) fetch(g0 + it + 1);
        float2 v[E];
        zreg_c2r_pack<n, E, T>(x, xn, slot, partner, v, tw);
        ct_fft_reg<n, E, +1, N>(v, slot, twr, sl, ss);
        if (valid) {
            float2 *dst = reinterpret_cast<float2 *>(out + line * N);
#pragma unroll
            for (int j = 0; j < E; j++) dst[slot + j * T] = v[j];
        }
    }
}

template <int N, int E, int WPB, int IT> bool zpf_entry(bool r2c, ZctKernel *o) {
    typedef ZRegShape<N, E> Z;
    if constexpr (!Z::ok) {
        return false;
    } else {
        o->k = r2c ? (const void *)k_z_r2c_pf<N, E, WPB, IT> : (const void *)k_z_c2r_pf<N, E, WPB, IT>;
        o->smem = (size_t)WPB * Z::LPW * (Z::LS > 0 ? Z::LS : 1) * sizeof(float2);
        o->lines_per_block = WPB * Z::LPW * IT;
        o->threads = 32 * WPB;
        return true;
    }
}

template <int N, int E, int WPB> bool zreg_entry(bool r2c, ZctKernel *o) {
    typedef ZRegShape<N, E> Z;
    if constexpr (!Z::ok) {
        return false;
    } else {
        o->k = r2c ? (const void *)k_z_r2c_reg<N, E, WPB> : (const void *)k_z_c2r_reg<N, E, WPB>;
        o->smem = (size_t)WPB * Z::LPW * (Z::LS > 0 ? Z::LS : 1) * sizeof(float2);
        o->lines_per_block = WPB * Z::LPW;
        o->threads = 32 * WPB;
        return true;
    }
}

}  // namespace nsk
