// fused_zr3.cu -- register-resident pass C for grid sizes with a factor 3:
// E = 12 with u_x parked in shared memory, or E = 6.
#include "fused_zr.cuh"

namespace nsk {

template <int N> static bool zr_three(int E, int tile, ZctKernel *o) {
    if (E == 12) return zr_by_tile<N, 12, true>(tile, o);
    if (E == 6) return zr_by_tile<N, 6, false>(tile, o);
    return false;
}

bool zr_lookup3(int N, int E, int tile, ZctKernel *o) {
    switch (N) {
    case 96: return zr_three<96>(E, tile, o);
    case 192: return zr_three<192>(E, tile, o);
    case 384: return zr_three<384>(E, tile, o);
    case 768: return zr_three<768>(E, tile, o);
    }
    return false;
}

}  // namespace nsk
