// fused_kA.cu -- constant-geometry kernels of pass A (x inverse + curl).
#include "fused_k.cuh"

namespace nsk {

bool fzk_lookup_A(int N, int E, int CT, FzsKernel *o) {
#define NSK_CASE(n_, e_, ct_)                          \
    if (N == n_ && E == e_ && CT == ct_) {             \
        fzk_fill<n_, e_, ct_, FZ_A>(o);               \
        return true;                                   \
    }
    NSK_FZS_SHAPES(NSK_CASE)
#undef NSK_CASE
    return false;
}

}  // namespace nsk
