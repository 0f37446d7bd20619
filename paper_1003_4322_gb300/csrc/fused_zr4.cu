// fused_zr4.cu -- register-resident pass C with asynchronous copies of the
// fields two ahead (fused_zr.cuh, DEPTH = 2) for power-of-two grid sizes:
// E = 16 with one or two fields parked (N = 256 to 1024) and E = 8 (N <= 512).
// Depth 3 timed no faster than depth 2 at 512^3 and 1024^3 (pass C 1.052 vs
// 1.058 ms, 9.85 vs 9.67 ms) for 1.5x the copy buffers, so it is not compiled.
#include "fused_zr.cuh"

namespace nsk {

template <int N, int D> static bool zr_async_d(int E, int tile, ZctKernel *o) {
    if (E == 16) return zr_by_tile<N, 16, 1, D>(tile, o) || zr_by_tile<N, 16, 2, D>(tile, o);
    if constexpr (N <= 512)
        if (E == 8) return zr_by_tile<N, 8, 0, D>(tile, o);
    return false;
}
template <int N> static bool zr_async(int E, int tile, ZctKernel *o) { return zr_async_d<N, 2>(E, tile, o); }

bool zr_lookup4(int N, int E, int tile, ZctKernel *o) {
    switch (N) {
    case 256: return zr_async<256>(E, tile, o);
    case 512: return zr_async<512>(E, tile, o);
    case 1024: return zr_async<1024>(E, tile, o);
    }
    return false;
}

}  // namespace nsk
