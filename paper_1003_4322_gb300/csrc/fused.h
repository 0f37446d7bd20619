// fused.h -- the fused, pruned FP32 form of the solver step.
#pragma once
#include "../../include/ns.h"
#include "ns_internal.h"

namespace nsk {

// Launch configuration of one pass: its radix plan (elements per thread) and
// its tile (columns per CTA for a strided pass, lines per CTA for pass C).
struct PassCfg {
    Plan pl{};
    int ct = 16;
    int kind = 0;   // 0: runtime-length kernel; 1: compile-time-length kernel (ct = warps per CTA)
};

// A pass-C kernel specialised for one grid size (fused_z.cu).
struct ZctKernel {
    const void *k = nullptr;
    size_t smem = 0;
    int lines_per_block = 0;
    int threads = 0;
};
// Kernel for grid size N with wpb warps per CTA, if one was compiled.
bool zct_lookup(int N, int wpb, ZctKernel *out);

// A strided-pass kernel specialised for one (N, E, CT) shape (fused_s*.cu).
struct FzsKernel {
    const void *k = nullptr;
    size_t smem = 0;
    int threads = 0;
};
bool fzs_lookup_A(int N, int E, int CT, FzsKernel *out);    // x inverse + curl
bool fzs_lookup_B(int N, int E, int CT, FzsKernel *out);    // y inverse
bool fzs_lookup_DE(int N, int E, int CT, FzsKernel *out);   // y / x forward

// One run of the fused form.  Compact state layout [c][ikx][iky][kz] with
// ikx, iky in [0, Mx) (index k for k >= 0, k + Mx for k < 0) and kz in
// [0, Mz): only the modes the cubic 2/3 rule keeps, |kx|, |ky|, kz <= K.
struct FusedRun {
    ns_run_params p{};
    int n = 0, K = 0, Mx = 0, Mz = 0;
    long M = 0;                  // compact modes per component, Mx * Mx * Mz
    Plan plN{}, plH{};           // default plans of length n (x, y) and n/2 (z)
    PassCfg sp[4];               // passes A, B, D, E (chosen by the autotuner)
    PassCfg zc;                  // pass C
    const float2 *tw = nullptr;  // exp(-2 pi i t / n), t < n (owned by the context)
    float2 *a = nullptr;         // state
    float2 *a1 = nullptr;        // first-stage state
    float2 *nl = nullptr;        // unnormalised transform of u x w (compact)
    float2 *abuf = nullptr;      // pass A output (6 fields), reused for pass D (3)
    float2 *bbuf = nullptr;      // pass B output (6 fields), pass C in place (3)
    float *etab = nullptr;       // exp(-nu k^2 dt) by integer k^2 <= 3 K^2
    int nparts = 0;              // energy partial sums (update kernel blocks)
    double *part = nullptr;      // [nparts][2], owned by the context
};

bool fused_enabled();
cudaError_t fused_alloc(FusedRun &f, const ns_run_params &p, const float2 *tw, cudaStream_t s);
void fused_free(FusedRun &f);
cudaError_t fused_set_state(FusedRun &f, const double2 *src, int on_device, void *staging,
                            size_t staging_bytes, cudaStream_t s);
cudaError_t fused_get_state(FusedRun &f, double2 *dst, int on_device, void *staging,
                            size_t staging_bytes, cudaStream_t s);
cudaError_t fused_step(FusedRun &f, double *series, int cap, unsigned long long *counter,
                       int *flags, cudaStream_t s, Tracer *tr);
// JSON text describing the chosen per-pass configuration; returns its length.
int fused_describe(const FusedRun &f, char *out, int len);
cudaError_t fused_spectrum(FusedRun &f, int nbins, double *spec, double *ens, cudaStream_t s);

}  // namespace nsk
