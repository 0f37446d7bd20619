// fused_sPI.cu -- compile-time-length strided kernels of the standalone inverse transform (x and y passes):
// every row of the column stored and loaded (no compact rows, no curl).
#include "fused_s.cuh"

namespace nsk {

bool fzs_lookup_PI(int N, int E, int CT, FzsKernel *o) {
#define NSK_CASE(n_, e_, ct_)                          \
    if (N == n_ && E == e_ && CT == ct_) {             \
        fzs_fill<n_, e_, ct_, +1, false, false, false>(o);  \
        return true;                                   \
    }
    NSK_FZS_SHAPES(NSK_CASE)
#undef NSK_CASE
    return false;
}

}  // namespace nsk
