// fused_zr.cuh -- pass C of the fused form with each line held in registers.
//
// Pass C (z c2r of u and w, the cross product u x w on the grid, z r2c of
// the product; Sec. 2, Eqs. 1-2) is the pass with the most arithmetic per
// byte.  This form keeps a (y, x) line's six transformed fields in the
// registers of the T = N/2 / E threads that own it instead of in shared
// memory:
//
//  * the first Stockham stage of a length-n transform reads the elements
//    slot + j T of the line, which are exactly the ones a thread loads (or,
//    for the forward transform, holds after the cross product), and the last
//    stage leaves the thread the same set of positions, so the line crosses
//    shared memory only between stages (one exchange for a two-stage plan);
//  * the even/odd packing of the real transforms pairs element k with
//    element n - k, which the partner lane (T - slot) mod T holds in register
//    E - 1 - j: it arrives by warp shuffle;
//  * the cross product is taken in registers, with the fields transformed in
//    the order u_x, w_y, u_y, w_x, u_z, w_z so that at most five field arrays
//    are live; PARK of them (u_x, then u_y: the longest-lived) can be parked
//    in thread-private shared memory to leave room for longer lines.
// With N fixed at compile time the kept range kz < (N-1)/3 + 1 is a constant
// too, so the registers that only ever hold dealiased zeros fold away.
#pragma once
#include "fft_ct.cuh"
#include "fused.h"

namespace nsk {

// Length-n line FFT over the T = n/E threads of a line.  v enters holding
// positions slot + j T (j < E) and leaves holding the transform at the same
// positions; stages after the first exchange through the line's shared
// buffer (sl/ss).
template <int n, int E, int DIR, int NTAB, int S = 0, class SL, class SS>
NSK_DEV void ct_fft_reg(float2 (&v)[E], int slot, const CtTwiddles<n, E, NTAB> &twr, SL sl, SS ss) {
    constexpr int NST = ct_nst(n, E);
    constexpr int R = ct_radix(n, E, S), T = n / E, nR = n / R, p = ct_span(n, E, S);
    if constexpr (S > 0) {
#pragma unroll
        for (int b = 0; b < E / R; b++) {
            const int i = slot + b * T;
#pragma unroll
            for (int q = 0; q < R; q++) v[b * R + q] = sl(i + q * nR);
        }
    }
#pragma unroll
    for (int b = 0; b < E / R; b++) {
        if constexpr (S > 0) {
            constexpr int o = CtTwiddles<n, E, NTAB>::offset(S);
#pragma unroll
            for (int q = 1; q < R; q++) {
                const float2 w = twr.w[o + b * (R - 1) + q - 1];
                v[b * R + q] = DIR < 0 ? cmul(v[b * R + q], w) : cmulc(v[b * R + q], w);
            }
        }
        Dft<R, DIR, float2>::run(&v[b * R]);
    }
    if constexpr (S + 1 < NST) {
        __syncwarp();
#pragma unroll
        for (int b = 0; b < E / R; b++) {
            const int i = slot + b * T;
            const int k = i % p;
            const int j = (i - k) * R + k;
#pragma unroll
            for (int q = 0; q < R; q++) ss(j + q * p, v[b * R + q]);
        }
        __syncwarp();
        ct_fft_reg<n, E, DIR, NTAB, S + 1>(v, slot, twr, sl, ss);
    } else {
        // The last stage's butterfly b leaves output q at slot + T (b + q E/R).
        float2 t[E];
#pragma unroll
        for (int b = 0; b < E / R; b++)
#pragma unroll
            for (int q = 0; q < R; q++) t[b + q * (E / R)] = v[b * R + q];
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = t[j];
    }
}

// Shape of the register form for grid size N with E elements per thread.
template <int N, int E_> struct ZrShape {
    static constexpr int n = N / 2;
    static constexpr int E = E_;
    static constexpr int T = n / E;
    static constexpr bool ok = n % E == 0 && ct_valid(n, E) && T >= 1 && T <= 32 && 32 % T == 0;
    static constexpr int LPW = ok ? 32 / T : 1;                       // lines per warp
    static constexpr int NST = ok ? ct_nst(n, E) : 1;
    static constexpr int LS = (ok && NST > 1) ? ct_line_stride(n, E, 1) : 0;   // exchange buffer
    static constexpr int Mz = (N - 1) / 3 + 1;                        // kept kz
};

NSK_DEV float2 pmul(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }

// Asynchronous 8-byte copy global -> shared (zero-filled when ok is false;
// src is then not read), and the group commit / wait of such copies.
NSK_DEV void cp_async8(float2 *dst, const float2 *src, bool ok) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 8 : 0)
                 : "memory");
}
NSK_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING> NSK_DEV void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}
// Bulk copies global -> shared that complete on an mbarrier (the
// transaction count of the barrier's current phase), and the barrier's
// bounded wait.
NSK_DEV unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
NSK_DEV void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
NSK_DEV void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
// Shared memory read by generic loads before an asynchronous-proxy write.
NSK_DEV void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// bytes (a multiple of 16) from src to dst (both 16-byte aligned); one
// arrival on bar that expects them.
NSK_DEV void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
NSK_DEV bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// true once the phase of the given parity has completed; false after
// `cycles` clock cycles without it
NSK_DEV bool mbar_wait(unsigned long long *bar, unsigned parity, long long cycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > cycles) return false;
    return true;
}

NSK_DEV float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// A warp owns a group of LPW lines at a time and walks the groups
// warp * WPB * gridDim.x apart (the launch sizes the grid to what is
// resident at once); the first field of its next group is loaded while the
// current group's last three transforms run, so only a warp's first group
// waits for its loads.
// DEPTH > 0: the fields are copied into DEPTH per-warp shared buffers by
// asynchronous copies issued DEPTH fields ahead (the field order continues
// into the next group), so a load has DEPTH transforms' time to land instead
// of one, with no more registers; each thread copies and reads back only its
// own elements.  DEPTH divides the six fields of a group (2 or 3), so a
// field keeps its buffer from group to group.
// BULK (with DEPTH): one lane copies the warp's LPW lines of a field (they are
// contiguous, LPW Mz 8 bytes, a multiple of 16) with one bulk copy that
// completes on the buffer's mbarrier, and every lane reads its elements from
// the natural line layout; the warp syncs before a buffer is refilled.  A
// wait that runs out of ctl.wait_cycles raises bit 1 of *ctl.flags, the
// loads that follow read zeros, and the kernel still waits for the copies it
// issued before it exits.
template <int N, int E, int WPB, int PARK, int DEPTH = 0, bool BULK = false>
__global__ void __launch_bounds__(32 * WPB)
k_fused_zr(float2 *buf, long fs, long nlines, long brun, const float2 *__restrict__ tw, ZrCtl ctl) {
    static_assert(DEPTH == 0 || DEPTH == 2 || DEPTH == 3, "DEPTH divides 6");
    static_assert(!BULK || DEPTH > 0, "bulk copies run ahead");
    constexpr bool ASYNC = DEPTH > 0;
    typedef ZrShape<N, E> Z;
    constexpr int n = Z::n, T = Z::T, LPW = Z::LPW, LS = Z::LS, Mz = Z::Mz;
    buf += blockIdx.y * brun;   // run of the group
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ll = lane / T, slot = lane % T;
    const int partner = ll * T + (T - slot) % T;   // holds position n - k of this line
    const long ngroups = (nlines + LPW - 1) / LPW;
    const long gstride = (long)gridDim.x * WPB;
    long group = (long)blockIdx.x * WPB + warp;   // warp-uniform
    long line = group * LPW + ll;
    bool valid = line < nlines;
    float2 *L = sm + (long)(warp * LPW + ll) * LS;
    float2 *park0 = sm + (long)WPB * LPW * LS + (long)warp * PARK * E * 32 + lane;   // u_x
    float2 *park1 = park0 + E * 32;                                                   // u_y
    // ASYNC: [warp][DEPTH buffers][E][32 lanes] after the parked fields
    float2 *pfb = sm + (long)WPB * LPW * LS + (long)WPB * PARK * E * 32 + (long)warp * DEPTH * E * 32 + lane;
    // BULK: [warp][DEPTH buffers][BL] (16-byte aligned), then the warps'
    // mbarriers [warp][DEPTH]
    constexpr int BL = (LPW * Mz + 1) & ~1;
    constexpr long BB = ((long)WPB * LPW * LS + (long)WPB * PARK * E * 32 + 1) & ~1L;
    float2 *bb = sm + BB + (long)warp * DEPTH * BL;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(sm + BB + (long)WPB * DEPTH * BL) + warp * DEPTH;
    unsigned par = 0, pend = 0;   // BULK: phase parity and copy in flight, bit b for buffer b
    bool bad = false;             // BULK: a wait ran out
    bool first_copy = true;
    auto sl = [&](int e) -> float2 { return L[ct_skew(e)]; };
    auto ss = [&](int e, float2 v) { L[ct_skew(e)] = v; };

    CtTwiddles<n, E, N> twr;
    twr.load(slot, tw);
    float2 wk[E];   // W^k = exp(-2 pi i k / N), k = slot + j T
#pragma unroll
    for (int j = 0; j < E; j++) wk[j] = __ldg(tw + slot + j * T);

    float2 x[E];   // X[k], k = slot + j T, of the field being loaded
    auto fetch_at = [&](int f, long ln, bool ok) {
        const float2 *src = buf + f * fs + ln * Mz;
#pragma unroll
        for (int j = 0; j < E; j++) {
            const int k = slot + j * T;
            x[j] = make_float2(0.f, 0.f);
            if (j * T < Mz && ok && k < Mz) x[j] = src[k];
        }
    };
    auto fetch = [&](int f) { fetch_at(f, line, valid); };
    // ASYNC: field f of line ln into buffer b (one commit group), and the
    // buffer's contents into x once all but the latest group have landed
    auto issue_at = [&](int f, long ln, bool ok, int b) {
        const float2 *src = buf + f * fs + (ok ? ln : 0) * Mz;
#pragma unroll
        for (int j = 0; j < E; j++) {
            const int k = slot + j * T;
            if (j * T < Mz) cp_async8(pfb + (b * E + j) * 32, ok && k < Mz ? src + k : buf, ok && k < Mz);
        }
        cp_async_commit();
    };
    auto take = [&](int b) {
        cp_async_wait<(DEPTH > 0 ? DEPTH - 1 : 0)>();
#pragma unroll
        for (int j = 0; j < E; j++) x[j] = j * T < Mz ? pfb[(b * E + j) * 32] : make_float2(0.f, 0.f);
    };
    // BULK: field f of group g into buffer b (no copy past the last group)
    auto issue_bulk = [&](int f, long g, int b) {
        if (g >= ngroups || bad) return;
        __syncwarp();   // every lane has read buffer b
        if (lane == 0 && !(ctl.skip_first_copy && first_copy)) {
            fence_proxy_async_smem();
            bulk_g2s(bb + b * BL, buf + f * fs + g * LPW * Mz, LPW * Mz * 8, &bars[b]);
        }
        first_copy = false;
        pend |= 1u << b;
    };
    // BULK: wait for buffer b's copy (the phase stays current: a second wait
    // on it returns at once)
    auto wait_bulk = [&](int b) {
        if (bad || !(pend & (1u << b))) return;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars[b], (par >> b) & 1u, ctl.wait_cycles));
        if (!ok) {
            bad = true;
            pend &= ~(1u << b);
            if (lane == 0 && ctl.flags) atomicOr(ctl.flags, 2);
        }
    };
    auto take_bulk = [&](int b) {
        wait_bulk(b);
        const bool ok = !bad;
        if (ok && (pend & (1u << b))) {   // else a copy in flight stays pending for the exit
            par ^= 1u << b;
            pend &= ~(1u << b);
        }
        const float2 *src = bb + b * BL + ll * Mz;
#pragma unroll
        for (int j = 0; j < E; j++) {
            const int k = slot + j * T;
            x[j] = make_float2(0.f, 0.f);
            if (j * T < Mz && ok && k < Mz) x[j] = src[k];
        }
    };
    // the field DEPTH places after position i of the order u_x, w_y, u_y, w_x,
    // u_z, w_z (the last DEPTH positions reach into the next group), into the
    // buffer position i has just freed
    constexpr int kOrder[6] = {0, 4, 1, 3, 2, 5};
    auto issue_ahead = [&](int i) {
        if constexpr (BULK) {
            if (i + DEPTH < 6) issue_bulk(kOrder[i + DEPTH], group, i % DEPTH);
            else issue_bulk(kOrder[i + DEPTH - 6], group + gstride, i % DEPTH);
        } else if (i + DEPTH < 6) {
            issue_at(kOrder[i + DEPTH], line, valid, i % DEPTH);
        } else {
            const long nl = (group + gstride) * LPW + ll;
            issue_at(kOrder[i + DEPTH - 6], nl, group + gstride < ngroups && nl < nlines, i % DEPTH);
        }
    };
    // c2r: Z[k] = (X[k] + conj X[n-k]) + i W^{-k} (X[k] - conj X[n-k]) with
    // the imaginary parts of X[0] and X[n] dropped, then the inverse length-n
    // FFT; complex element m of the result holds the real points 2m, 2m + 1.
    // fnext: the field to load next (-1 none, -2 field 0 of the next group);
    // ASYNC: pos, the position of this field in the order (buffer pos % DEPTH).
    auto inverse = [&](float2 (&v)[E], int fnext, int pos) {
        if constexpr (BULK) take_bulk(pos % DEPTH);
        else if constexpr (ASYNC) take(pos % (DEPTH > 0 ? DEPTH : 1));
#pragma unroll
        for (int j = 0; j < E; j++) {
            const int k = slot + j * T;
            float2 a0 = x[j];
            float2 am = make_float2(0.f, 0.f);
            if ((E - 1 - j) * T < Mz) am = shfl2(x[E - 1 - j], partner);
            if (slot == 0) am = (j > 0 && (E - j) * T < Mz) ? x[(E - j) % E] : make_float2(0.f, 0.f);
            if (k == 0) {
                a0.y = 0.f;
                am.y = 0.f;
            }
            const float2 xc = cconj(am);
            const float2 wb = cmulc(csub(a0, xc), wk[j]);
            v[j] = cadd(cadd(a0, xc), cmul_i<1>(wb));
        }
        if constexpr (ASYNC) {
            issue_ahead(pos);
        } else {
            if (fnext >= 0) fetch(fnext);
            if (fnext == -2) {
                const long nl = (group + gstride) * LPW + ll;
                fetch_at(0, nl, group + gstride < ngroups && nl < nlines);
            }
        }
        ct_fft_reg<n, E, +1, N>(v, slot, twr, sl, ss);
    };
    // r2c of a product held as Z[m] = x[2m] + i x[2m+1]: forward length-n FFT,
    // then X[k] = (Z[k] + conj Z[n-k])/2 - i W^k (Z[k] - conj Z[n-k])/2 for
    // the kept k < Mz, written over field f of the line.
    auto forward_store = [&](float2 (&v)[E], int f) {
        ct_fft_reg<n, E, -1, N>(v, slot, twr, sl, ss);
        float2 *dst = buf + f * fs + line * Mz;
#pragma unroll
        for (int j = 0; j < E; j++) {
            if (j * T < Mz) {
                const int k = slot + j * T;
                float2 zm = shfl2(v[E - 1 - j], partner);
                if (slot == 0) zm = v[(E - j) % E];
                const float2 zk = v[j], zc = cconj(zm);
                const float2 ev = cscale(cadd(zk, zc), 0.5f);
                const float2 od = cmul_i<-1>(cscale(csub(zk, zc), 0.5f));
                if (valid && k < Mz) dst[k] = cadd(ev, cmul(od, wk[j]));
            }
        }
    };

    // fields: 0..2 = u_x, u_y, u_z; 3..5 = w_x, w_y, w_z; output over 0..2.
    // Order u_x, w_y, u_y, w_x (then (u x w)_z is complete), u_z, w_z: at
    // most five field arrays are live.  A thread stores only positions it
    // loaded itself, and its loads of a field precede its stores to it.
    float2 A[E], B[E], C[E], D[E], P[E];
    if constexpr (BULK) {
        if (lane == 0) {
#pragma unroll
            for (int b = 0; b < DEPTH; b++) mbar_init(&bars[b], 1);
            mbar_init_fence();
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < DEPTH; i++) issue_bulk(kOrder[i], group, i);
    } else if constexpr (ASYNC) {
#pragma unroll
        for (int i = 0; i < DEPTH; i++) issue_at(kOrder[i], line, valid, i);
    } else {
        fetch(0);
    }
    for (; group < ngroups; group += gstride) {
    inverse(A, 4, 0);   // u_x
    if constexpr (PARK >= 1) {
#pragma unroll
        for (int j = 0; j < E; j++) park0[j * 32] = A[j];
    }
    inverse(B, 1, 1);   // w_y
#pragma unroll
    for (int j = 0; j < E; j++) P[j] = pmul(PARK >= 1 ? park0[j * 32] : A[j], B[j]);   // u_x w_y
    inverse(C, 3, 2);   // u_y
    if constexpr (PARK >= 2) {
#pragma unroll
        for (int j = 0; j < E; j++) park1[j * 32] = C[j];
    }
    inverse(D, 2, 3);   // w_x
#pragma unroll
    for (int j = 0; j < E; j++) {
        const float2 t = pmul(PARK >= 2 ? park1[j * 32] : C[j], D[j]);   // u_y w_x
        P[j] = make_float2(P[j].x - t.x, P[j].y - t.y);
    }
    // ASYNC: the store over field 2 must not overtake the copy of u_z (field
    // 2, position 4); groups complete in order, and the copies issued after it
    // are those of positions 5 .. 3 + DEPTH.  BULK: wait for that copy.
    if constexpr (BULK) wait_bulk(4 % DEPTH);
    else if constexpr (ASYNC) cp_async_wait<(DEPTH > 0 ? DEPTH - 2 : 0)>();
    forward_store(P, 2);
    float2 px[E], py[E];
    inverse(P, 5, 4);   // u_z
#pragma unroll
    for (int j = 0; j < E; j++) {
        px[j] = pmul(P[j], B[j]);   // u_z w_y (subtracted below)
        py[j] = pmul(P[j], D[j]);   // u_z w_x
    }
    inverse(B, -2, 5);  // w_z; the next group's u_x starts loading
#pragma unroll
    for (int j = 0; j < E; j++) {
        const float2 a = PARK >= 1 ? park0[j * 32] : A[j];
        const float2 s = pmul(PARK >= 2 ? park1[j * 32] : C[j], B[j]);   // u_y w_z
        const float2 t = pmul(a, B[j]);      // u_x w_z
        px[j] = make_float2(s.x - px[j].x, s.y - px[j].y);
        py[j] = make_float2(py[j].x - t.x, py[j].y - t.y);
    }
    forward_store(px, 0);
    forward_store(py, 1);
    line += gstride * LPW;
    valid = line < nlines;
    }
    if constexpr (BULK) {   // no copy may land after the CTA exits
#pragma unroll
        for (int b = 0; b < DEPTH; b++)
            if (pend & (1u << b)) (void)mbar_wait(&bars[b], (par >> b) & 1u, ctl.wait_cycles);
    } else if constexpr (ASYNC) {
        cp_async_wait<0>();
    }
}

// Pass C of the MHD form (Alfven units): the group's B buffers form two
// blocks, bu = (u, w = curl u) and bb = (b, j = curl b), six fields each.
// Per (y, x) line: the c2r of the twelve fields, u x b written over b's
// slots (the induction term) and u x w + j x b over u's slots (the velocity
// term), as r2c of the kept kz.  u and b wait in thread-private shared
// memory; the products accumulate in registers while w and j stream through.
template <int N, int E, int WPB>
__global__ void __launch_bounds__(32 * WPB)
k_fused_zr_mhd(float2 *bu, float2 *bb, long fs, long nlines, long brun, const float2 *__restrict__ tw) {
    typedef ZrShape<N, E> Z;
    constexpr int n = Z::n, T = Z::T, LPW = Z::LPW, LS = Z::LS, Mz = Z::Mz;
    bu += blockIdx.y * brun;   // run of the group
    bb += blockIdx.y * brun;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ll = lane / T, slot = lane % T;
    const int partner = ll * T + (T - slot) % T;
    const long line = ((long)blockIdx.x * WPB + warp) * LPW + ll;
    const bool valid = line < nlines;
    float2 *L = sm + (long)(warp * LPW + ll) * LS;
    float2 *park = sm + (long)WPB * LPW * LS + (long)warp * 6 * E * 32 + lane;   // u, then b
    auto pk = [&](int c, int j) -> float2 & { return park[(c * E + j) * 32]; };
    auto sl = [&](int e) -> float2 { return L[ct_skew(e)]; };
    auto ss = [&](int e, float2 v) { L[ct_skew(e)] = v; };

    CtTwiddles<n, E, N> twr;
    twr.load(slot, tw);
    float2 wk[E];
#pragma unroll
    for (int j = 0; j < E; j++) wk[j] = __ldg(tw + slot + j * T);

    float2 x[E];
    auto fetch = [&](const float2 *field) {
        const float2 *src = field + line * Mz;
#pragma unroll
        for (int j = 0; j < E; j++) {
            const int k = slot + j * T;
            x[j] = make_float2(0.f, 0.f);
            if (j * T < Mz && valid && k < Mz) x[j] = src[k];
        }
    };
    auto inverse = [&](float2 (&v)[E], const float2 *next) {
#pragma unroll
        for (int j = 0; j < E; j++) {
            const int k = slot + j * T;
            float2 a0 = x[j];
            float2 am = make_float2(0.f, 0.f);
            if ((E - 1 - j) * T < Mz) am = shfl2(x[E - 1 - j], partner);
            if (slot == 0) am = (j > 0 && (E - j) * T < Mz) ? x[(E - j) % E] : make_float2(0.f, 0.f);
            if (k == 0) {
                a0.y = 0.f;
                am.y = 0.f;
            }
            const float2 xc = cconj(am);
            const float2 wb = cmulc(csub(a0, xc), wk[j]);
            v[j] = cadd(cadd(a0, xc), cmul_i<1>(wb));
        }
        if (next) fetch(next);
        ct_fft_reg<n, E, +1, N>(v, slot, twr, sl, ss);
    };
    auto forward_store = [&](float2 (&v)[E], float2 *field) {
        ct_fft_reg<n, E, -1, N>(v, slot, twr, sl, ss);
        float2 *dst = field + line * Mz;
#pragma unroll
        for (int j = 0; j < E; j++) {
            if (j * T < Mz) {
                const int k = slot + j * T;
                float2 zm = shfl2(v[E - 1 - j], partner);
                if (slot == 0) zm = v[(E - j) % E];
                const float2 zk = v[j], zc = cconj(zm);
                const float2 ev = cscale(cadd(zk, zc), 0.5f);
                const float2 od = cmul_i<-1>(cscale(csub(zk, zc), 0.5f));
                if (valid && k < Mz) dst[k] = cadd(ev, cmul(od, wk[j]));
            }
        }
    };
    auto acc = [&](float2 &p, float2 a, float2 b, float sgn) {
        p = make_float2(p.x + sgn * a.x * b.x, p.y + sgn * a.y * b.y);
    };

    // the twelve fields in transform order: u, b, w, j
    const float2 *seq[12] = {bu, bu + fs, bu + 2 * fs, bb, bb + fs, bb + 2 * fs,
                             bu + 3 * fs, bu + 4 * fs, bu + 5 * fs, bb + 3 * fs, bb + 4 * fs, bb + 5 * fs};
    float2 V[E];
    fetch(seq[0]);
    for (int c = 0; c < 6; c++) {   // u_x, u_y, u_z, b_x, b_y, b_z -> parked
        inverse(V, seq[c + 1]);
#pragma unroll
        for (int j = 0; j < E; j++) pk(c, j) = V[j];
    }
    // u x b, component by component, over b's slots
    for (int c = 0; c < 3; c++) {
        const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
#pragma unroll
        for (int j = 0; j < E; j++) {
            const float2 u1 = pk(c1, j), u2 = pk(c2, j), b1 = pk(3 + c1, j), b2 = pk(3 + c2, j);
            V[j] = make_float2(u1.x * b2.x - u2.x * b1.x, u1.y * b2.y - u2.y * b1.y);
        }
        forward_store(V, bb + c * fs);
    }
    // u x w + j x b, with w and j one component at a time
    float2 P0[E], P1[E], P2[E];
#pragma unroll
    for (int j = 0; j < E; j++) P0[j] = P1[j] = P2[j] = make_float2(0.f, 0.f);
    inverse(V, seq[7]);   // w_x: (u x w)_y += u_z w_x, (u x w)_z -= u_y w_x
#pragma unroll
    for (int j = 0; j < E; j++) {
        acc(P1[j], pk(2, j), V[j], 1.f);
        acc(P2[j], pk(1, j), V[j], -1.f);
    }
    inverse(V, seq[8]);   // w_y: (u x w)_z += u_x w_y, (u x w)_x -= u_z w_y
#pragma unroll
    for (int j = 0; j < E; j++) {
        acc(P2[j], pk(0, j), V[j], 1.f);
        acc(P0[j], pk(2, j), V[j], -1.f);
    }
    inverse(V, seq[9]);   // w_z: (u x w)_x += u_y w_z, (u x w)_y -= u_x w_z
#pragma unroll
    for (int j = 0; j < E; j++) {
        acc(P0[j], pk(1, j), V[j], 1.f);
        acc(P1[j], pk(0, j), V[j], -1.f);
    }
    inverse(V, seq[10]);  // j_x: (j x b)_y -= j_x b_z, (j x b)_z += j_x b_y
#pragma unroll
    for (int j = 0; j < E; j++) {
        acc(P1[j], V[j], pk(5, j), -1.f);
        acc(P2[j], V[j], pk(4, j), 1.f);
    }
    inverse(V, seq[11]);  // j_y: (j x b)_x += j_y b_z, (j x b)_z -= j_y b_x
#pragma unroll
    for (int j = 0; j < E; j++) {
        acc(P0[j], V[j], pk(5, j), 1.f);
        acc(P2[j], V[j], pk(3, j), -1.f);
    }
    inverse(V, nullptr);  // j_z: (j x b)_x -= j_z b_y, (j x b)_y += j_z b_x
#pragma unroll
    for (int j = 0; j < E; j++) {
        acc(P0[j], V[j], pk(4, j), -1.f);
        acc(P1[j], V[j], pk(3, j), 1.f);
    }
    forward_store(P0, bu);
    forward_store(P1, bu + fs);
    forward_store(P2, bu + 2 * fs);
}

template <int N, int E, int WPB> bool zrm_entry(ZctKernel *o) {
    typedef ZrShape<N, E> Z;
    if constexpr (!Z::ok) {
        return false;
    } else {
        o->k = (const void *)k_fused_zr_mhd<N, E, WPB>;
        o->smem = (size_t)WPB * (Z::LPW * Z::LS + 6 * E * 32) * sizeof(float2);
        o->lines_per_block = WPB * Z::LPW;
        o->threads = 32 * WPB;
        return true;
    }
}

template <int N, int E, int WPB, int PARK, int DEPTH = 0, bool BULK = false> bool zr_entry(ZctKernel *o) {
    typedef ZrShape<N, E> Z;
    // a bulk copy moves a warp's LPW lines of a field: a multiple of 16 bytes
    if constexpr (!Z::ok || (BULK && (Z::LPW * Z::Mz) % 2 != 0)) {
        return false;
    } else {
        o->k = (const void *)k_fused_zr<N, E, WPB, PARK, DEPTH, BULK>;
        if constexpr (BULK) {
            constexpr long BL = (Z::LPW * Z::Mz + 1) & ~1;
            constexpr long BB = ((long)WPB * Z::LPW * Z::LS + (long)WPB * PARK * E * 32 + 1) & ~1L;
            o->smem = (size_t)(BB + WPB * DEPTH * BL) * sizeof(float2) + WPB * DEPTH * sizeof(unsigned long long);
            o->bulk_bytes = Z::LPW * Z::Mz * (int)sizeof(float2);
        } else {
            o->smem = (size_t)WPB * (Z::LPW * Z::LS + PARK * E * 32 + DEPTH * E * 32) * sizeof(float2);
            o->bulk_bytes = 0;
        }
        o->lines_per_block = WPB * Z::LPW;
        o->threads = 32 * WPB;
        return true;
    }
}

// tile = warps per CTA (1 or 2) + ZR_PARK x the number of parked fields
// + ZR_ASYNC x the load mode (0 registers, 1 per-lane asynchronous copies, 2
// bulk copies; both copy forms two fields ahead).
template <int N, int E, int PARK, int DEPTH = 0, bool BULK = false> bool zr_by_tile(int tile, ZctKernel *o) {
    static_assert(DEPTH == 0 || DEPTH == 2, "the copy forms run two fields ahead");
    const int mode = tile / ZR_ASYNC;
    if (mode != (BULK ? 2 : DEPTH > 0 ? 1 : 0)) return false;
    tile %= ZR_ASYNC;
    if (tile / ZR_PARK != PARK) return false;
    switch (tile % ZR_PARK) {
    case 1: return zr_entry<N, E, 1, PARK, DEPTH, BULK>(o);
    case 2: return zr_entry<N, E, 2, PARK, DEPTH, BULK>(o);
    }
    return false;
}

// Lookups per family of grid sizes (fused_zr2.cu: powers of two, fused_zr3.cu:
// with a factor 3).
bool zr_lookup2(int N, int E, int tile, ZctKernel *o);
bool zr_lookup3(int N, int E, int tile, ZctKernel *o);
// The asynchronous-copy form for powers of two (fused_zr4.cu), and the
// bulk-copy form (fused_zr5.cu).
bool zr_lookup4(int N, int E, int tile, ZctKernel *o);
bool zr_lookup5(int N, int E, int tile, ZctKernel *o);

}  // namespace nsk
