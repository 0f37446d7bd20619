// fused_sDE.cu -- compile-time-length kernels of passes D and E (y and x forward).
#include "fused_s.cuh"

namespace nsk {

bool fzs_lookup_DE(int N, int E, int CT, FzsKernel *o) {
#define NSK_CASE(n_, e_, ct_)                          \
    if (N == n_ && E == e_ && CT == ct_) {             \
        fzs_fill<n_, e_, ct_, -1, false, true, false>(o);   \
        return true;                                   \
    }
    NSK_FZS_SHAPES(NSK_CASE)
#undef NSK_CASE
    return false;
}

}  // namespace nsk
