// fft_ct.cuh -- line FFTs whose length is a compile-time constant.
//
// Same Stockham scheme as fft_core.cuh (T = n/E threads per line, radix-R
// butterflies in registers, exchange through shared memory), but the radix
// plan, every stride and every span are constants, so the index arithmetic
// folds away, and a line lives inside one warp so that stages are separated
// by __syncwarp instead of block barriers.
#pragma once
#include "fft_core.cuh"

namespace nsk {

constexpr int kCtRadices[9] = {32, 16, 12, 9, 8, 6, 4, 3, 2};

// Radix of stage s of the greedy plan of length n with E elements per thread
// (the largest radix dividing both E and what is left); 0 past the last stage.
constexpr int ct_radix(int n, int E, int s) {
    int m = n;
    for (int i = 0; i < 16; i++) {
        if (m <= 1) return 0;
        int R = 0;
        for (int j = 0; j < 9; j++) {
            const int r = kCtRadices[j];
            if (E % r == 0 && m % r == 0) {
                R = r;
                break;
            }
        }
        if (R == 0) return 0;
        if (i == s) return R;
        m /= R;
    }
    return 0;
}
constexpr int ct_nst(int n, int E) {
    int s = 0;
    while (ct_radix(n, E, s) != 0) s++;
    return s;
}
constexpr int ct_span(int n, int E, int s) {
    int p = 1;
    for (int i = 0; i < s; i++) p *= ct_radix(n, E, i);
    return p;
}
constexpr bool ct_valid(int n, int E) {
    return n % E == 0 && ct_radix(n, E, 0) == E && ct_span(n, E, ct_nst(n, E)) == n;
}

// Element e of a line sits at e + e/16 (one element of skew per 128 bytes).
constexpr int ct_skew(int e) { return e + (e >> 4); }

// Shared-memory cost of one warp access to 8-byte elements, served in two
// half-warp phases: in each phase, lanes that hit the same bank pair (word
// index mod 16) at different words serialise.  Lane l belongs to line l / T
// (lines LS elements apart, scaled by fields_apart) and slot l % T.
constexpr int ct_phase_cost(const int (&w)[32]) {
    int cost = 0;
    for (int h = 0; h < 2; h++) {
        int cnt[16] = {};
        for (int c = 16 * h; c < 16 * h + 16; c++) {
            bool first = true;
            for (int d = 16 * h; d < c; d++)
                if (w[d] == w[c]) first = false;
            if (first) cnt[w[c] & 15]++;
        }
        int worst = 1;
        for (int b = 0; b < 16; b++)
            if (cnt[b] > worst) worst = cnt[b];
        cost += worst;
    }
    return cost;
}

// Cost of the shared-memory accesses of an n-point plan when 32 / T lines
// share a warp, consecutive lines `stride` elements apart.  Butterfly b = 0
// and inputs q = 0 and R/2 stand for each stage (the others are shifts).
constexpr int ct_plan_cost(int n, int E, int stride) {
    const int T = n / E;
    const int nst = ct_nst(n, E);
    int total = 0;
    int p = 1;
    for (int s = 0; s < nst; s++) {
        const int R = ct_radix(n, E, s);
        for (int qi = 0; qi < 2; qi++) {
            const int q = qi * (R / 2);
            int wl[32] = {}, ws[32] = {};
            for (int l = 0; l < 32; l++) {
                const int line = l / T, slot = l % T;
                const int i = slot;
                const int k = i % p;
                const int j = (i - k) * R + k;
                wl[l] = line * stride + ct_skew(i + q * (n / R));
                ws[l] = line * stride + ct_skew(j + q * p);
            }
            total += ct_phase_cost(wl) + ct_phase_cost(ws);
        }
        p *= R;
    }
    return total;
}

// Smallest-cost line stride (in elements) for `fields` consecutive line
// buffers per line, at least ct_skew(n - 1) + 1 elements each.
constexpr int ct_line_stride(int n, int E, int fields) {
    const int lo = ct_skew(n - 1) + 1;
    int best = lo, best_cost = 1 << 30;
    for (int ls = lo; ls < lo + 16; ls++) {
        const int c = ct_plan_cost(n, E, fields * ls);
        if (c < best_cost) {
            best_cost = c;
            best = ls;
        }
    }
    return best;
}

// Stage twiddles of one thread, kept in registers across many transforms of
// the same length: W_{pR}^{q k} for stages s >= 1, k = (slot + b T) mod p.
template <int n, int E, int NTAB> struct CtTwiddles {
    static constexpr int offset(int s) {
        int o = 0;
        for (int i = 1; i < s; i++) o += (E / ct_radix(n, E, i)) * (ct_radix(n, E, i) - 1);
        return o;
    }
    static constexpr int count() { return offset(ct_nst(n, E)) > 0 ? offset(ct_nst(n, E)) : 1; }
    float2 w[count()];
    template <int S = 1> NSK_DEV void load(int slot, const float2 *__restrict__ tw) {
        if constexpr (S < ct_nst(n, E)) {
            constexpr int R = ct_radix(n, E, S), p = ct_span(n, E, S), T = n / E, o = offset(S);
#pragma unroll
            for (int b = 0; b < E / R; b++) {
                const int k = (slot + b * T) % p;
#pragma unroll
                for (int q = 1; q < R; q++) w[o + b * (R - 1) + q - 1] = __ldg(tw + q * k * (NTAB / (p * R)));
            }
            load<S + 1>(slot, tw);
        }
    }
};

// In-place FFT as ct_fft_smem, with the stage twiddles already in registers.
template <int n, int E, int DIR, int NTAB, int S = 0, class SL, class SS>
NSK_DEV void ct_fft_smem_tw(int slot, const CtTwiddles<n, E, NTAB> &twr, SL sl, SS ss) {
    constexpr int NST = ct_nst(n, E);
    if constexpr (S < NST) {
        constexpr int R = ct_radix(n, E, S), T = n / E, nR = n / R;
        constexpr int p = ct_span(n, E, S);
        float2 v[E];
#pragma unroll
        for (int b = 0; b < E / R; b++) {
            const int i = slot + b * T;
#pragma unroll
            for (int q = 0; q < R; q++) v[b * R + q] = sl(i + q * nR);
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
        ct_fft_smem_tw<n, E, DIR, NTAB, S + 1>(slot, twr, sl, ss);
    }
}

// In-place FFT of one line in shared memory (sl/ss read and write element e)
// by T = n/E threads of one warp, slot = the thread's index in its line.
// tw: exp(-2 pi i t / NTAB), t < NTAB, with n dividing NTAB.
template <int n, int E, int DIR, int NTAB, int S = 0, class SL, class SS>
NSK_DEV void ct_fft_smem(int slot, const float2 *__restrict__ tw, SL sl, SS ss) {
    constexpr int NST = ct_nst(n, E);
    if constexpr (S < NST) {
        constexpr int R = ct_radix(n, E, S), p = ct_span(n, E, S), T = n / E, nR = n / R;
        float2 v[E];
#pragma unroll
        for (int b = 0; b < E / R; b++) {
            const int i = slot + b * T;
#pragma unroll
            for (int q = 0; q < R; q++) v[b * R + q] = sl(i + q * nR);
        }
#pragma unroll
        for (int b = 0; b < E / R; b++) {
            if constexpr (p > 1) {
                const int k = (slot + b * T) % p;
#pragma unroll
                for (int q = 1; q < R; q++) {
                    const float2 w = __ldg(tw + q * k * (NTAB / (p * R)));
                    v[b * R + q] = DIR < 0 ? cmul(v[b * R + q], w) : cmulc(v[b * R + q], w);
                }
            }
            Dft<R, DIR, float2>::run(&v[b * R]);
        }
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
        ct_fft_smem<n, E, DIR, NTAB, S + 1>(slot, tw, sl, ss);
    }
}

// Line FFT by T = n/E threads of a block: the first stage loads through gl,
// the last stores through gs, the stages in between exchange through shared
// memory (sl/ss) with block barriers.  Out of place: gs never writes what gl
// reads.
template <int n, int E, int DIR, int NTAB, int S = 0, class GL, class SL, class SS, class GS>
NSK_DEV void ct_fft_block(int slot, const float2 *__restrict__ tw, GL gl, SL sl, SS ss, GS gs) {
    constexpr int NST = ct_nst(n, E);
    if constexpr (S < NST) {
        constexpr int R = ct_radix(n, E, S), p = ct_span(n, E, S), T = n / E, nR = n / R;
        constexpr bool first = S == 0, last = S == NST - 1;
        float2 v[E];
#pragma unroll
        for (int b = 0; b < E / R; b++) {
            const int i = slot + b * T;
#pragma unroll
            for (int q = 0; q < R; q++) {
                if constexpr (first) v[b * R + q] = gl(i + q * nR);
                else v[b * R + q] = sl(i + q * nR);
            }
        }
#pragma unroll
        for (int b = 0; b < E / R; b++) {
            if constexpr (p > 1) {
                const int k = (slot + b * T) % p;
#pragma unroll
                for (int q = 1; q < R; q++) {
                    const float2 w = __ldg(tw + q * k * (NTAB / (p * R)));
                    v[b * R + q] = DIR < 0 ? cmul(v[b * R + q], w) : cmulc(v[b * R + q], w);
                }
            }
            Dft<R, DIR, float2>::run(&v[b * R]);
        }
        if constexpr (!first && !last) __syncthreads();
#pragma unroll
        for (int b = 0; b < E / R; b++) {
            const int i = slot + b * T;
            const int k = i % p;
            const int j = (i - k) * R + k;
#pragma unroll
            for (int q = 0; q < R; q++) {
                if constexpr (last) gs(j + q * p, v[b * R + q]);
                else ss(j + q * p, v[b * R + q]);
            }
        }
        if constexpr (!last) __syncthreads();
        ct_fft_block<n, E, DIR, NTAB, S + 1>(slot, tw, gl, sl, ss, gs);
    }
}

// As ct_fft_block, but the last stage leaves the line in v instead of storing
// it: v[j] holds position slot + j T (T = n/E) afterwards, the same positions
// whatever the plan (the last stage's butterfly b writes output q at
// slot + T (b + q E/R)).  The caller separates two calls that share the
// shared-memory tile with a block barrier.
template <int n, int E, int DIR, int NTAB, int S = 0, class GL, class SL, class SS>
NSK_DEV void ct_fft_block_reg(float2 (&v)[E], int slot, const float2 *__restrict__ tw, GL gl, SL sl,
                              SS ss) {
    constexpr int NST = ct_nst(n, E);
    constexpr int R = ct_radix(n, E, S), p = ct_span(n, E, S), T = n / E, nR = n / R;
    constexpr bool first = S == 0, last = S == NST - 1;
#pragma unroll
    for (int b = 0; b < E / R; b++) {
        const int i = slot + b * T;
#pragma unroll
        for (int q = 0; q < R; q++) {
            if constexpr (first) v[b * R + q] = gl(i + q * nR);
            else v[b * R + q] = sl(i + q * nR);
        }
    }
#pragma unroll
    for (int b = 0; b < E / R; b++) {
        if constexpr (p > 1) {
            const int k = (slot + b * T) % p;
#pragma unroll
            for (int q = 1; q < R; q++) {
                const float2 w = __ldg(tw + q * k * (NTAB / (p * R)));
                v[b * R + q] = DIR < 0 ? cmul(v[b * R + q], w) : cmulc(v[b * R + q], w);
            }
        }
        Dft<R, DIR, float2>::run(&v[b * R]);
    }
    if constexpr (!last) {
        if constexpr (!first) __syncthreads();
#pragma unroll
        for (int b = 0; b < E / R; b++) {
            const int i = slot + b * T;
            const int k = i % p;
            const int j = (i - k) * R + k;
#pragma unroll
            for (int q = 0; q < R; q++) ss(j + q * p, v[b * R + q]);
        }
        __syncthreads();
        ct_fft_block_reg<n, E, DIR, NTAB, S + 1>(v, slot, tw, gl, sl, ss);
    } else {
        float2 t[E];
#pragma unroll
        for (int b = 0; b < E / R; b++)
#pragma unroll
            for (int q = 0; q < R; q++) t[b + q * (E / R)] = v[b * R + q];
#pragma unroll
        for (int j = 0; j < E; j++) v[j] = t[j];
    }
}

}  // namespace nsk
