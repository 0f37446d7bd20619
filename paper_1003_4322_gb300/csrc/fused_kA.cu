// fused_kA.cu -- constant-geometry kernels of pass A (x inverse + curl).
#include "fused_k.cuh"

namespace nsk {

bool fzk_lookup_A(int NX, int NY, int NZ, int E, int CT, FzsKernel *o) {
#define NSK_CASE(n_, e_, ct_)                                          \
    if (NX == n_ && NY == n_ && NZ == n_ && E == e_ && CT == ct_) {    \
        fzk_fill<n_, n_, n_, e_, ct_, FZ_A>(o);                      \
        return true;                                                   \
    }
    NSK_FZS_SHAPES(NSK_CASE)
#undef NSK_CASE
#define NSK_CASE(nx_, ny_, nz_, e_, ct_)                                 \
    if (NX == nx_ && NY == ny_ && NZ == nz_ && E == e_ && CT == ct_) {   \
        fzk_fill<nx_, ny_, nz_, e_, ct_, FZ_A>(o);                     \
        return true;                                                     \
    }
    NSK_FZK_GRIDS(NSK_CASE)
#undef NSK_CASE
    return false;
}

}  // namespace nsk
