// fused.h -- the fused, pruned FP32 form of the solver step.
#pragma once
#include "../../include/ns.h"
#include "ns_internal.h"

namespace nsk {

struct FusedRun {
    int n = 0;
    int nparts = 0;
    double *part = nullptr;
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
cudaError_t fused_spectrum(FusedRun &f, int nbins, double *spec, double *ens, cudaStream_t s);

}  // namespace nsk
