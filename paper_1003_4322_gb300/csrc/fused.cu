// fused.cu -- placeholder until the fused form lands.
#include "fused.h"

namespace nsk {
bool fused_enabled() { return false; }
cudaError_t fused_alloc(FusedRun &, const ns_run_params &, const float2 *, cudaStream_t) {
    return cudaErrorNotSupported;
}
void fused_free(FusedRun &) {}
cudaError_t fused_set_state(FusedRun &, const double2 *, int, void *, size_t, cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t fused_get_state(FusedRun &, double2 *, int, void *, size_t, cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t fused_step(FusedRun &, double *, int, unsigned long long *, int *, cudaStream_t, Tracer *) {
    return cudaErrorNotSupported;
}
cudaError_t fused_spectrum(FusedRun &, int, double *, double *, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace nsk
