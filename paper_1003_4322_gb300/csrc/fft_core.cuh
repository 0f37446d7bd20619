// fft_core.cuh -- device building blocks of the batched 1D FFTs that make up
// every 3D transform of the solver (Sec. 2: FFTs along each direction of the
// N^3 box, with the axis change done in HBM instead of by an all-to-all).
//
// A line of length n is split over T = n/E threads, each holding E complex
// values in registers.  One stage of radix R (R divides E) lets every thread
// run E/R radix-R butterflies in registers; stages exchange data through
// shared memory in Stockham (self-sorting) order, so the result comes out in
// natural order with no bit reversal.  For a stage with span p (the product
// of the radices already applied), butterfly i (0 <= i < n/R) reads
// x[i + q n/R], q < R, multiplies input q by W_{pR}^{q (i mod p)}, applies
// the radix-R DFT and writes output q to position (i - i mod p) R + i mod p
// + q p.  The first stage reads through a load functor and the last writes
// through a store functor, so loads/stores to HBM (and any pre- or
// post-processing) happen straight from/to registers.
#pragma once
#include <cuda_runtime.h>

namespace nsk {

#define NSK_DEV __device__ __forceinline__

template <typename T> struct Cx;
template <> struct Cx<float> { typedef float2 type; };
template <> struct Cx<double> { typedef double2 type; };

NSK_DEV float2 mkc(float a, float b) { return make_float2(a, b); }
NSK_DEV double2 mkc(double a, double b) { return make_double2(a, b); }
template <typename C> NSK_DEV C cadd(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <typename C> NSK_DEV C csub(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
template <typename C> NSK_DEV C cneg(C a) { return mkc(-a.x, -a.y); }
template <typename C> NSK_DEV C cconj(C a) { return mkc(a.x, -a.y); }
template <typename C, typename T> NSK_DEV C cscale(C a, T s) { return mkc(a.x * s, a.y * s); }
// a * b
template <typename C> NSK_DEV C cmul(C a, C b) {
    return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> NSK_DEV C cmulc(C a, C b) {
    return mkc(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// a * (s i) for s = +1 / -1
template <int S, typename C> NSK_DEV C cmul_i(C a) {
    return S > 0 ? mkc(-a.y, a.x) : mkc(a.y, -a.x);
}
// a + S i b for S = +1 / -1 (one addition per part, no separate swap).
template <int S, typename C> NSK_DEV C cadd_i(C a, C b) {
    return S > 0 ? mkc(a.x - b.y, a.y + b.x) : mkc(a.x + b.y, a.y - b.x);
}

// Even/odd packing of a real transform of N points as a complex one of
// n = N/2 (w = W^k = exp(-2 pi i k / N)).  With f = a + b and g = a - b of
// the two modes k and n - k (four additions for both formulas):
//  c2r: Z[k] = (X[k] + conj X[n-k]) + i conj(w) (X[k] - conj X[n-k])
//       = (f.x, g.y) + i conj(w) (g.x, f.y);
//  r2c: X[k] = (Z[k] + conj Z[n-k]) / 2 - i w (Z[k] - conj Z[n-k]) / 2
//       = ((f.x, g.y) + w (f.y, -g.x)) / 2,
// ten arithmetic instructions per mode for r2c where the expanded form takes
// fourteen.  The plain form's z passes use them; the FP32 kernels of the
// fused form keep their own expressions, which suit their register budgets.
template <typename C> NSK_DEV C c2r_pack(C xk, C xm, C w) {
    const C f = cadd(xk, xm), g = csub(xk, xm);
    const auto bx = g.x * w.x + f.y * w.y, by = f.y * w.x - g.x * w.y;
    return mkc(f.x - by, g.y + bx);
}
template <typename C> NSK_DEV C r2c_unpack(C zk, C zm, C w) {
    typedef decltype(zk.x) T;
    const C f = cadd(zk, zm), g = csub(zk, zm);
    return cscale(mkc(f.x + f.y * w.x + g.x * w.y, g.y + f.y * w.y - g.x * w.x), (T)0.5);
}
template <typename C> NSK_DEV C czero() { C z; z.x = 0; z.y = 0; return z; }

// cos and sin of 2 pi key / 288 for the angles the register butterflies use
// (radices 2, 3, 4, 6, 8, 9, 12, 16, 32); values of the mathematical constants.
NSK_DEV void angle288(int key, double &c, double &s) {
    switch (key) {
    case 0: c = 1.0; s = 0.0; break;
    case 9: c = 0.9807852804032304; s = 0.19509032201612828; break;
    case 18: c = 0.9238795325112867; s = 0.3826834323650898; break;
    case 24: c = 0.8660254037844386; s = 0.5; break;
    case 27: c = 0.8314696123025452; s = 0.5555702330196022; break;
    case 32: c = 0.766044443118978; s = 0.6427876096865394; break;
    case 36: c = 0.7071067811865476; s = 0.7071067811865476; break;
    case 45: c = 0.5555702330196022; s = 0.8314696123025452; break;
    case 48: c = 0.5; s = 0.8660254037844386; break;
    case 54: c = 0.3826834323650898; s = 0.9238795325112867; break;
    case 63: c = 0.19509032201612828; s = 0.9807852804032304; break;
    case 64: c = 0.17364817766693036; s = 0.984807753012208; break;
    case 72: c = 0.0; s = 1.0; break;
    case 81: c = -0.19509032201612828; s = 0.9807852804032304; break;
    case 90: c = -0.3826834323650898; s = 0.9238795325112867; break;
    case 96: c = -0.5; s = 0.8660254037844386; break;
    case 99: c = -0.5555702330196022; s = 0.8314696123025452; break;
    case 108: c = -0.7071067811865476; s = 0.7071067811865476; break;
    case 117: c = -0.8314696123025452; s = 0.5555702330196022; break;
    case 120: c = -0.8660254037844386; s = 0.5; break;
    case 126: c = -0.9238795325112867; s = 0.3826834323650898; break;
    case 128: c = -0.9396926207859084; s = 0.3420201433256687; break;
    case 135: c = -0.9807852804032304; s = 0.19509032201612828; break;
    case 144: c = -1.0; s = 0.0; break;
    case 153: c = -0.9807852804032304; s = -0.19509032201612828; break;
    case 160: c = -0.9396926207859084; s = -0.3420201433256687; break;
    case 162: c = -0.9238795325112867; s = -0.3826834323650898; break;
    case 168: c = -0.8660254037844386; s = -0.5; break;
    case 171: c = -0.8314696123025452; s = -0.5555702330196022; break;
    case 180: c = -0.7071067811865476; s = -0.7071067811865476; break;
    case 189: c = -0.5555702330196022; s = -0.8314696123025452; break;
    case 192: c = -0.5; s = -0.8660254037844386; break;
    case 198: c = -0.3826834323650898; s = -0.9238795325112867; break;
    case 207: c = -0.19509032201612828; s = -0.9807852804032304; break;
    case 216: c = 0.0; s = -1.0; break;
    case 224: c = 0.17364817766693036; s = -0.984807753012208; break;
    case 225: c = 0.19509032201612828; s = -0.9807852804032304; break;
    case 234: c = 0.3826834323650898; s = -0.9238795325112867; break;
    case 240: c = 0.5; s = -0.8660254037844386; break;
    case 243: c = 0.5555702330196022; s = -0.8314696123025452; break;
    case 252: c = 0.7071067811865476; s = -0.7071067811865476; break;
    case 256: c = 0.766044443118978; s = -0.6427876096865394; break;
    case 261: c = 0.8314696123025452; s = -0.5555702330196022; break;
    case 264: c = 0.8660254037844386; s = -0.5; break;
    case 270: c = 0.9238795325112867; s = -0.3826834323650898; break;
    case 279: c = 0.9807852804032304; s = -0.19509032201612828; break;
    default: c = 1.0; s = 0.0; break;
    }
}

// v * W_R^m with W_R = exp(DIR 2 pi i / R); m is a compile-time constant once
// the butterflies are unrolled, so the branches and the table fold away.
template <int R, int DIR, typename C> NSK_DEV C twc(C v, int m) {
    m %= R;
    if (m == 0) return v;
    if (4 * m == R) return cmul_i<DIR>(v);
    if (2 * m == R) return cneg(v);
    if (4 * m == 3 * R) return cmul_i<-DIR>(v);
    double c, s;
    angle288(m * (288 / R), c, s);
    typedef decltype(v.x) T;
    const T cc = (T)c, ss = (T)(DIR * s);
    return mkc(v.x * cc - v.y * ss, v.x * ss + v.y * cc);
}

// In-register DFT of length R: a[k] <- sum_j a[j] exp(DIR 2 pi i j k / R).
template <int R, int DIR, typename C> struct Dft;

template <int DIR, typename C> struct Dft<2, DIR, C> {
    static NSK_DEV void run(C *a) {
        C t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    }
};

template <int DIR, typename C> struct Dft<3, DIR, C> {
    static NSK_DEV void run(C *a) {
        typedef decltype(a[0].x) T;
        const T h = (T)0.8660254037844386;  // sqrt(3)/2
        C t1 = cadd(a[1], a[2]);
        C t2 = csub(a[0], cscale(t1, (T)0.5));   // 0.5 t1 is exact
        C t3 = cscale(csub(a[1], a[2]), h);
        a[0] = cadd(a[0], t1);
        a[1] = cadd_i<DIR>(t2, t3);
        a[2] = cadd_i<-DIR>(t2, t3);
    }
};

template <int DIR, typename C> struct Dft<4, DIR, C> {
    static NSK_DEV void run(C *a) {
        C s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
        C s13 = cadd(a[1], a[3]), d13 = csub(a[1], a[3]);
        a[0] = cadd(s02, s13);
        a[2] = csub(s02, s13);
        a[1] = cadd_i<DIR>(d02, d13);
        a[3] = cadd_i<-DIR>(d02, d13);
    }
};

// R = R1 R2 with j = R2 j1 + j2 and k = k1 + R1 k2:
// A[k1 + R1 k2] = sum_j2 W_R2^{j2 k2} W_R^{j2 k1} sum_j1 W_R1^{j1 k1} a[R2 j1 + j2].
template <int R1, int R2, int DIR, typename C> struct DftComposite {
    static NSK_DEV void run(C *a) {
        constexpr int R = R1 * R2;
        C B[R];
#pragma unroll
        for (int j2 = 0; j2 < R2; j2++) {
            C b[R1];
#pragma unroll
            for (int j1 = 0; j1 < R1; j1++) b[j1] = a[R2 * j1 + j2];
            Dft<R1, DIR, C>::run(b);
#pragma unroll
            for (int k1 = 0; k1 < R1; k1++) B[j2 * R1 + k1] = twc<R, DIR>(b[k1], j2 * k1);
        }
#pragma unroll
        for (int k1 = 0; k1 < R1; k1++) {
            C c[R2];
#pragma unroll
            for (int j2 = 0; j2 < R2; j2++) c[j2] = B[j2 * R1 + k1];
            Dft<R2, DIR, C>::run(c);
#pragma unroll
            for (int k2 = 0; k2 < R2; k2++) a[k1 + R1 * k2] = c[k2];
        }
    }
};
template <int DIR, typename C> struct Dft<6, DIR, C> : DftComposite<2, 3, DIR, C> {};

NSK_DEV float fmac(float a, float b, float c) { return fmaf(a, b, c); }
NSK_DEV double fmac(double a, double b, double c) { return fma(a, b, c); }

// Radix 8 in FP64 as 2 x 4 (j = 4 j1 + j2, k = k1 + 2 k2) like the
// composite, with the odd outputs k1 = 1 regrouped: their inputs carry W^j2,
// W = exp(DIR 2 pi i / 8), and W^2 = DIR i, so the length-4 sums pair up as
// W (b1 +- DIR i b3) and W = (1 + DIR i) / sqrt(2).  The 1/sqrt(2) is applied
// by the fused multiply-adds of the last additions: 52 arithmetic
// instructions where the composite takes 56, which pays in the FP64 passes
// (bound by the FP64 pipe: 2-3 % per pass).  The FP32 passes, bound by
// memory, keep the composite: the regrouped form changed their register
// allocation and cost up to 10 % (pass A at 1024^3).
template <int DIR, typename C> struct Dft<8, DIR, C> : DftComposite<2, 4, DIR, C> {};
template <int DIR> struct Dft<8, DIR, double2> {
    typedef double2 C;
    static NSK_DEV void run(C *a) {
        typedef double T;
        const T h = (T)0.7071067811865476;   // 1 / sqrt(2)
        C b0[4], b1[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            b0[j] = cadd(a[j], a[4 + j]);
            b1[j] = csub(a[j], a[4 + j]);
        }
        Dft<4, DIR, C>::run(b0);
        a[0] = b0[0];
        a[2] = b0[1];
        a[4] = b0[2];
        a[6] = b0[3];
        const C s02 = cadd_i<DIR>(b1[0], b1[2]), d02 = cadd_i<-DIR>(b1[0], b1[2]);
        const C e = cadd_i<DIR>(b1[1], b1[3]), f = cadd_i<-DIR>(b1[1], b1[3]);
        // W e = h (pe, qe), W f = h (pf, qf)
        const T pe = DIR > 0 ? e.x - e.y : e.x + e.y, qe = DIR > 0 ? e.y + e.x : e.y - e.x;
        const T pf = DIR > 0 ? f.x - f.y : f.x + f.y, qf = DIR > 0 ? f.y + f.x : f.y - f.x;
        const T hd = DIR > 0 ? h : -h;
        a[1] = mkc(fmac(h, pe, s02.x), fmac(h, qe, s02.y));    // s02 + W e
        a[5] = mkc(fmac(-h, pe, s02.x), fmac(-h, qe, s02.y));  // s02 - W e
        a[3] = mkc(fmac(-hd, qf, d02.x), fmac(hd, pf, d02.y)); // d02 + DIR i W f
        a[7] = mkc(fmac(hd, qf, d02.x), fmac(-hd, pf, d02.y)); // d02 - DIR i W f
    }
};
template <int DIR, typename C> struct Dft<9, DIR, C> : DftComposite<3, 3, DIR, C> {};
template <int DIR, typename C> struct Dft<12, DIR, C> : DftComposite<4, 3, DIR, C> {};
template <int DIR, typename C> struct Dft<16, DIR, C> : DftComposite<4, 4, DIR, C> {};
template <int DIR, typename C> struct Dft<32, DIR, C> : DftComposite<4, 8, DIR, C> {};

// Radix plan of one line length: n = prod rad[s]; every radix divides E.
struct Plan {
    int n;                      // line length
    int E;                      // elements per thread
    int nst;                    // number of stages (<= 12)
    unsigned long long radix;   // radix of stage s in bits [5s, 5s + 5)
    __host__ __device__ int rad(int s) const { return (int)((radix >> (5 * s)) & 31u); }
};

template <typename C> NSK_DEV C ldg_c(const C *p) { return __ldg(p); }

// One Stockham stage of radix R (see the header comment).  tw holds
// exp(-2 pi i t / ntab), t < ntab, with n dividing ntab; the inverse
// direction uses its conjugate.
template <int R, int E, int DIR, typename C, class Ld, class St>
NSK_DEV void stage(C (&v)[E], int slot, int T, int n, int p, const C *__restrict__ tw,
                   int ntab, Ld ld, St st, bool sync_mid, bool active = true) {
    const int nR = n / R;
    if (active) {
#pragma unroll
        for (int b = 0; b < E / R; b++) {
            const int i = slot + b * T;
#pragma unroll
            for (int q = 0; q < R; q++) v[b * R + q] = ld(i + q * nR);
        }
        const int tstride = ntab / (p * R);
#pragma unroll
        for (int b = 0; b < E / R; b++) {
            if (p > 1) {
                const int k = (slot + b * T) % p;
#pragma unroll
                for (int q = 1; q < R; q++) {
                    const C w = ldg_c(tw + q * k * tstride);
                    v[b * R + q] = DIR < 0 ? cmul(v[b * R + q], w) : cmulc(v[b * R + q], w);
                }
            }
            Dft<R, DIR, C>::run(&v[b * R]);
        }
    }
    if (sync_mid) __syncthreads();
    if (active) {
#pragma unroll
        for (int b = 0; b < E / R; b++) {
            const int i = slot + b * T;
            const int k = i % p;
            const int j = (i - k) * R + k;
#pragma unroll
            for (int q = 0; q < R; q++) st(j + q * p, v[b * R + q]);
        }
    }
}

template <int E, int DIR, typename C, class Ld, class St>
NSK_DEV void stage_dispatch(int R, C (&v)[E], int slot, int T, int n, int p,
                            const C *__restrict__ tw, int ntab, Ld ld, St st, bool sync_mid,
                            bool active = true) {
    switch (R) {
    case 2: if constexpr (E % 2 == 0) stage<2, E, DIR>(v, slot, T, n, p, tw, ntab, ld, st, sync_mid, active); break;
    case 3: if constexpr (E % 3 == 0) stage<3, E, DIR>(v, slot, T, n, p, tw, ntab, ld, st, sync_mid, active); break;
    case 4: if constexpr (E % 4 == 0) stage<4, E, DIR>(v, slot, T, n, p, tw, ntab, ld, st, sync_mid, active); break;
    case 6: if constexpr (E % 6 == 0) stage<6, E, DIR>(v, slot, T, n, p, tw, ntab, ld, st, sync_mid, active); break;
    case 8: if constexpr (E % 8 == 0) stage<8, E, DIR>(v, slot, T, n, p, tw, ntab, ld, st, sync_mid, active); break;
    case 9: if constexpr (E % 9 == 0) stage<9, E, DIR>(v, slot, T, n, p, tw, ntab, ld, st, sync_mid, active); break;
    case 12: if constexpr (E % 12 == 0) stage<12, E, DIR>(v, slot, T, n, p, tw, ntab, ld, st, sync_mid, active); break;
    case 16: if constexpr (E % 16 == 0) stage<16, E, DIR>(v, slot, T, n, p, tw, ntab, ld, st, sync_mid, active); break;
    default: break;
    }
}

// Whole line FFT.  GL/GS: load of the first stage / store of the last stage.
// SL/SS: shared-memory exchange between stages.  FIRST_SMEM / LAST_SMEM say
// that GL reads or GS writes the same shared buffer (a stage that reads and
// writes shared memory must wait for every read before any write).  INPLACE
// says that GS overwrites what GL read (matters for a single-stage plan).
// The first radix of every plan is E (make_plan picks the largest radix
// first), so stage 0 is compiled for radix E with span 1 (no twiddles); the
// later stages share one dispatch whose store target (shared memory or GS)
// is a uniform runtime choice.  A thread with active == false skips every
// load, butterfly and store but takes every barrier, so blocks in which only
// some thread groups have a line stay in step.  Ends with the last stores
// issued and, if LAST_SMEM, synchronised.
template <int E, int DIR, bool FIRST_SMEM, bool LAST_SMEM, bool INPLACE, typename C,
          class GL, class SL, class SS, class GS>
NSK_DEV void fft_line_impl(bool active, const Plan &pl, int slot, const C *__restrict__ tw,
                           int ntab, GL gl, SL sl, SS ss, GS gs) {
    C v[E];
    const int T = pl.n / E;
    const int nst = pl.nst;
    {
        const bool last = nst == 1;
        auto st = [&](int e, C x) {
            if (last) gs(e, x);
            else ss(e, x);
        };
        const bool wr_smem = !last || LAST_SMEM;
        const bool mid = (FIRST_SMEM && wr_smem) || (last && INPLACE);
        stage<E, E, DIR>(v, slot, T, pl.n, 1, tw, ntab, gl, st, mid, active);
        if (wr_smem) __syncthreads();
    }
    int p = E;
    for (int s = 1; s < nst; s++) {
        const bool last = s == nst - 1;
        auto st = [&](int e, C x) {
            if (last) gs(e, x);
            else ss(e, x);
        };
        const bool wr_smem = !last || LAST_SMEM;
        const int R = pl.rad(s);
        stage_dispatch<E, DIR>(R, v, slot, T, pl.n, p, tw, ntab, sl, st, wr_smem, active);
        if (wr_smem) __syncthreads();
        p *= R;
    }
}

template <int E, int DIR, bool FIRST_SMEM, bool LAST_SMEM, bool INPLACE, typename C,
          class GL, class SL, class SS, class GS>
NSK_DEV void fft_line(const Plan &pl, int slot, const C *__restrict__ tw, int ntab, GL gl, SL sl,
                      SS ss, GS gs) {
    fft_line_impl<E, DIR, FIRST_SMEM, LAST_SMEM, INPLACE>(true, pl, slot, tw, ntab, gl, sl, ss, gs);
}

template <int E, int DIR, bool FIRST_SMEM, bool LAST_SMEM, typename C, class GL, class SL,
          class SS, class GS>
NSK_DEV void fft_line_masked(bool active, const Plan &pl, int slot, const C *__restrict__ tw,
                             int ntab, GL gl, SL sl, SS ss, GS gs) {
    fft_line_impl<E, DIR, FIRST_SMEM, LAST_SMEM, false>(active, pl, slot, tw, ntab, gl, sl, ss, gs);
}

}  // namespace nsk
