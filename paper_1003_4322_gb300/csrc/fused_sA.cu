// fused_sA.cu -- compile-time-length kernels of pass A (x inverse + curl).
#include "fused_s.cuh"

namespace nsk {

bool fzs_lookup_A(int N, int E, int CT, FzsKernel *o) {
#define NSK_CASE(n_, e_, ct_)                          \
    if (N == n_ && E == e_ && CT == ct_) {             \
        fzs_fill<n_, e_, ct_, +1, true, false, true>(o);   \
        return true;                                   \
    }
    NSK_FZS_SHAPES(NSK_CASE)
#undef NSK_CASE
    return false;
}

}  // namespace nsk
