// fused_zr3.cu -- register-resident pass C for grid sizes with a factor 3:
// E = 12 with one or two fields parked in shared memory, or E = 6.
#include "fused_zr.cuh"

namespace nsk {

template <int N> static bool zr_three(int E, int tile, ZctKernel *o) {
    if (E == 12) return zr_by_tile<N, 12, 1>(tile, o) || zr_by_tile<N, 12, 2>(tile, o);
    if (E == 6) return zr_by_tile<N, 6, 0>(tile, o);
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
