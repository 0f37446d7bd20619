// fused_update.cuh -- the per-mode step of the fused form's update (1/N^3,
// Coriolis force, projection, forcing, IF-RK2 stage; Sec. 2, Eqs. 1-2) and
// the compensated accumulation of the energy partials, shared by the
// standalone update kernel (fused.cu) and the x-forward pass fused with the
// update (fused_keu.cu).
#pragma once
#include "fused.h"
#include "fused_access.cuh"

namespace nsk {

// 1/N^3, projection, forcing and the RK2 stage on the compact state; at
// stage 2 also the per-block energy and enstrophy partial sums of the new
// state, FP64 quality (grid-stride with a fixed grid: deterministic).  Grid y is the
// run of the group; each run has its own parameters and factor table.
struct FzUpdate {
    int n, K, Mx, Mz;
    int stage;
    long M;          // compact modes per component
    int nk2;         // entries of one run's factor table
    int nparts;      // partial sums per run
    // a grid or a box (fz_update_mode_grid): the y compaction, 1 / (N_x N_y
    // N_z), the wavenumber per grid index 1 / l_i, the sphere in integers
    // (D = lcm N_i, q_i = D / N_i); the factor table is then per axis by
    // compact index, [Mx | My | Mz]
    int My = 0, Ky = 0;
    float inv = 0.f;
    float sx = 1.f, sy = 1.f, sz = 1.f;
    long D = 0, qx = 0, qy = 0, qz = 0;
    // (m_i / l_i)^2 per axis by compact index as FP32 pairs hi + lo of the FP64
    // value, [Mx | My | Mz]: the enstrophy weight to FP64 accuracy
    const float2 *k2tab = nullptr;
};

__device__ __forceinline__ void fz_forcing(int kx, int ky, int kz, int kf, float F, float2 &fx,
                                           float2 &fy, float2 &fz) {
    const float h = 0.5f * F;
    if (kf <= 0) return;
    if (kx == 0 && ky == 0 && kz == kf) {
        fx = cadd(fx, make_float2(0.f, -h));
        fy = cadd(fy, make_float2(h, 0.f));
    }
    if (kx == 0 && kz == 0 && (ky == kf || ky == -kf)) {
        fx = cadd(fx, make_float2(h, 0.f));
        fz = cadd(fz, make_float2(0.f, ky > 0 ? -h : h));
    }
    if (ky == 0 && kz == 0 && (kx == kf || kx == -kf)) {
        fy = cadd(fy, make_float2(0.f, kx > 0 ? -h : h));
        fz = cadd(fz, make_float2(h, 0.f));
    }
}

// Compensated FP32 accumulator (value hi + lo) for the energy partials of
// the update.  A square of an FP32 value splits exactly into p + e with
// e = fma(x, x, -p), each addition keeps its rounding error (Knuth's TwoSum)
// and the pair is renormalised once per mode (Dekker's Fast2Sum), so a
// thread's few hundred terms sum to within a few units of 2^-48 relative --
// FP64-quality accumulation without FP64 instructions, which this GPU issues
// at 1/64 of the FP32 rate.  Block and final sums are FP64.
// The _rn intrinsics keep each rounding where it is written (no contraction
// into FMA), which the error terms rely on.
struct DfAcc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float b) {
        const float s = __fadd_rn(hi, b), bb = __fsub_rn(s, hi);
        lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
        hi = s;
    }
    __device__ __forceinline__ void add_sq(float x) {
        const float p = __fmul_rn(x, x);
        add(p);
        lo += fmaf(x, x, -p);
    }
    __device__ __forceinline__ void renorm() {
        const float s = __fadd_rn(hi, lo);
        lo = __fsub_rn(lo, __fsub_rn(s, hi));
        hi = s;
    }
    // += c * v for an exactly representable weight c (c * v.hi split exactly)
    __device__ __forceinline__ void add_scaled(const DfAcc &v, float c) {
        const float q = __fmul_rn(c, v.hi);
        add(q);
        lo += fmaf(c, v.hi, -q) + c * v.lo;
        renorm();
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// One mode of the update: N = P Pi (transform of u x w)/N^3 + f, then the
// IF-RK2 stage, from operands already loaded (b = a, c = a1, v = nl).
struct FzMode {
    float2 o0, o1, o2;
    int k2, kz;
    float k2f;          // grids and boxes: |k|^2 with the physical wavenumbers
    float k2hi, k2lo;   // the same as an unevaluated sum, to FP64 accuracy
};

// ABC forcing at the grid indices (mfx, mfy, mfz) of k_f along each axis.
__device__ __forceinline__ void fz_forcing_grid(int mx, int my, int mz, const FzRunParams &q, float2 &fx,
                                                float2 &fy, float2 &fz) {
    const float h = 0.5f * q.force_amp;
    if (q.force_k <= 0) return;
    if (mx == 0 && my == 0 && mz == q.mfz) {
        fx = cadd(fx, make_float2(0.f, -h));
        fy = cadd(fy, make_float2(h, 0.f));
    }
    if (mx == 0 && mz == 0 && (my == q.mfy || my == -q.mfy)) {
        fx = cadd(fx, make_float2(h, 0.f));
        fz = cadd(fz, make_float2(0.f, my > 0 ? -h : h));
    }
    if (my == 0 && mz == 0 && (mx == q.mfx || mx == -q.mfx)) {
        fy = cadd(fy, make_float2(0.f, mx > 0 ? -h : h));
        fz = cadd(fz, make_float2(h, 0.f));
    }
}

// The mode at flat compact index m = (ikx My + iky) Mz + kz of a grid or box
// state: physical wavenumbers m_i / l_i in the projection and |k|^2, the
// sphere of the spherical rule in grid indices, the factor as the product of
// the per-axis tables.
__device__ __forceinline__ FzMode fz_update_mode_grid(long m, const FzUpdate &u, const FzRunParams &q,
                                                      const float *__restrict__ etab, float2 vx, float2 vy,
                                                      float2 vz, float2 b0, float2 b1, float2 b2, float2 c0,
                                                      float2 c1, float2 c2) {
    const unsigned row = (unsigned)m / (unsigned)u.Mz;
    const int kz = (int)((unsigned)m - row * (unsigned)u.Mz);
    const int iky = (int)(row % (unsigned)u.My), ikx = (int)(row / (unsigned)u.My);
    const int mx = fz_compact_signed(ikx, u.Mx, u.K), my = fz_compact_signed(iky, u.My, u.Ky);
    FzMode r;
    r.kz = kz;
    r.k2 = 0;
    const float fkx = (float)mx * u.sx, fky = (float)my * u.sy, fkz = (float)kz * u.sz;
    r.k2f = fkx * fkx + fky * fky + fkz * fkz;
    {   // |k|^2 = sum of the three per-axis pairs (Knuth's TwoSum on the high parts)
        const float2 tx = u.k2tab[ikx], ty = u.k2tab[u.Mx + iky], tz = u.k2tab[u.Mx + u.My + kz];
        const float s1 = __fadd_rn(tx.x, ty.x), b1 = __fsub_rn(s1, tx.x);
        const float e1 = __fadd_rn(__fsub_rn(tx.x, __fsub_rn(s1, b1)), __fsub_rn(ty.x, b1));
        const float s2 = __fadd_rn(s1, tz.x), b2 = __fsub_rn(s2, s1);
        const float e2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, b2)), __fsub_rn(tz.x, b2));
        r.k2hi = s2;
        r.k2lo = e1 + e2 + tx.y + ty.y + tz.y;
    }
    bool keep = mx != 0 || my != 0 || kz != 0;
    if (q.dealias == 1) {
        const long ax = mx * u.qx, ay = my * u.qy, az = kz * u.qz;
        if (9 * (ax * ax + ay * ay + az * az) >= u.D * u.D) keep = false;
    }
    r.o0 = r.o1 = r.o2 = make_float2(0.f, 0.f);
    if (keep) {
        vx = cscale(vx, u.inv);
        vy = cscale(vy, u.inv);
        vz = cscale(vz, u.inv);
        if (q.rot != 0.f) {   // Coriolis -2 rot z x u of the stage's state, before P
            const float r2 = 2.f * q.rot;
            const float2 cx = u.stage == 1 ? b0 : c0, cy = u.stage == 1 ? b1 : c1;
            vx = cadd(vx, cscale(cy, r2));
            vy = csub(vy, cscale(cx, r2));
        }
        const float ik2 = 1.f / r.k2f;
        const float2 kv = cadd(cadd(cscale(vx, fkx), cscale(vy, fky)), cscale(vz, fkz));
        vx = csub(vx, cscale(kv, fkx * ik2));
        vy = csub(vy, cscale(kv, fky * ik2));
        vz = csub(vz, cscale(kv, fkz * ik2));
        fz_forcing_grid(mx, my, kz, q, vx, vy, vz);
        const float e = etab[ikx] * etab[u.Mx + iky] * etab[u.Mx + u.My + kz];
        if (u.stage == 1) {
            r.o0 = cscale(cadd(b0, cscale(vx, q.dt)), e);
            r.o1 = cscale(cadd(b1, cscale(vy, q.dt)), e);
            r.o2 = cscale(cadd(b2, cscale(vz, q.dt)), e);
        } else {
            const float he = 0.5f * e;
            r.o0 = cadd(cscale(b0, he), cscale(cadd(c0, cscale(vx, q.dt)), 0.5f));
            r.o1 = cadd(cscale(b1, he), cscale(cadd(c1, cscale(vy, q.dt)), 0.5f));
            r.o2 = cadd(cscale(b2, he), cscale(cadd(c2, cscale(vz, q.dt)), 0.5f));
        }
    }
    return r;
}

// The mode at wavenumbers (kx, ky, kz) of a compact state.
__device__ __forceinline__ FzMode fz_update_k(int kx, int ky, int kz, const FzUpdate &u,
                                              const FzRunParams &q, const float *__restrict__ etab,
                                              float inv, float2 vx, float2 vy, float2 vz, float2 b0,
                                              float2 b1, float2 b2, float2 c0, float2 c1, float2 c2) {
    FzMode r;
    r.kz = kz;
    r.k2 = kx * kx + ky * ky + kz * kz;
    bool keep = r.k2 > 0;
    if (q.dealias == 1 && 9L * r.k2 >= (long)u.n * u.n) keep = false;
    r.o0 = r.o1 = r.o2 = make_float2(0.f, 0.f);
    if (keep) {
        vx = cscale(vx, inv);
        vy = cscale(vy, inv);
        vz = cscale(vz, inv);
        if (q.rot != 0.f) {   // Coriolis -2 rot z x u of the stage's state, before P
            const float r2 = 2.f * q.rot;
            const float2 cx = u.stage == 1 ? b0 : c0, cy = u.stage == 1 ? b1 : c1;
            vx = cadd(vx, cscale(cy, r2));
            vy = csub(vy, cscale(cx, r2));
        }
        const float fkx = (float)kx, fky = (float)ky, fkz = (float)kz, ik2 = 1.f / (float)r.k2;
        const float2 kv = cadd(cadd(cscale(vx, fkx), cscale(vy, fky)), cscale(vz, fkz));
        vx = csub(vx, cscale(kv, fkx * ik2));
        vy = csub(vy, cscale(kv, fky * ik2));
        vz = csub(vz, cscale(kv, fkz * ik2));
        fz_forcing(kx, ky, kz, q.force_k, q.force_amp, vx, vy, vz);
        const float e = etab[r.k2];
        if (u.stage == 1) {
            r.o0 = cscale(cadd(b0, cscale(vx, q.dt)), e);
            r.o1 = cscale(cadd(b1, cscale(vy, q.dt)), e);
            r.o2 = cscale(cadd(b2, cscale(vz, q.dt)), e);
        } else {
            const float he = 0.5f * e;
            r.o0 = cadd(cscale(b0, he), cscale(cadd(c0, cscale(vx, q.dt)), 0.5f));
            r.o1 = cadd(cscale(b1, he), cscale(cadd(c1, cscale(vy, q.dt)), 0.5f));
            r.o2 = cadd(cscale(b2, he), cscale(cadd(c2, cscale(vz, q.dt)), 0.5f));
        }
    }
    return r;
}

// The mode at flat compact index m = (ikx Mx + iky) Mz + kz.
__device__ __forceinline__ FzMode fz_update_mode(long m, const FzUpdate &u, const FzRunParams &q,
                                                 const float *__restrict__ etab, float inv, float2 vx,
                                                 float2 vy, float2 vz, float2 b0, float2 b1, float2 b2,
                                                 float2 c0, float2 c1, float2 c2) {
    const unsigned Mz = (unsigned)u.Mz, Mx = (unsigned)u.Mx;   // M < 2^31 for every supported N
    const unsigned row = (unsigned)m / Mz;
    const int kz = (int)((unsigned)m - row * Mz);
    const int iky = (int)(row % Mx);
    const int ikx = (int)(row / Mx);
    return fz_update_k(fz_compact_signed(ikx, u.Mx, u.K), fz_compact_signed(iky, u.Mx, u.K), kz, u, q,
                       etab, inv, vx, vy, vz, b0, b1, b2, c0, c1, c2);
}

// Energy and enstrophy of one updated mode into a thread's accumulators
// (stage 2; weight 1/2 on the kz = 0 plane, the half-layout weight over 2).
__device__ __forceinline__ void fz_accumulate(const FzMode &r, DfAcc &e_acc, DfAcc &o_acc) {
    DfAcc me;   // |a(k)|^2 of this mode, exact up to the pair's rounding
    me.add_sq(r.o0.x);
    me.add_sq(r.o0.y);
    me.add_sq(r.o1.x);
    me.add_sq(r.o1.y);
    me.add_sq(r.o2.x);
    me.add_sq(r.o2.y);
    me.renorm();
    const float w = r.kz == 0 ? 0.5f : 1.0f;
    e_acc.add_scaled(me, w);
    o_acc.add_scaled(me, w * (float)r.k2);   // k2 <= 3 K^2 < 2^24: exact
}

// The same on a grid or box, with the physical |k|^2 as the pair hi + lo.
// The kz = N_z/2 plane is never kept, so kz = 0 is the only half weight.
__device__ __forceinline__ void fz_accumulate_grid(const FzMode &r, DfAcc &e_acc, DfAcc &o_acc) {
    DfAcc me;
    me.add_sq(r.o0.x);
    me.add_sq(r.o0.y);
    me.add_sq(r.o1.x);
    me.add_sq(r.o1.y);
    me.add_sq(r.o2.x);
    me.add_sq(r.o2.y);
    me.renorm();
    const float w = r.kz == 0 ? 0.5f : 1.0f;
    e_acc.add_scaled(me, w);
    o_acc.add_scaled(me, w * r.k2hi);
    o_acc.add_scaled(me, w * r.k2lo);
}

}  // namespace nsk
