// fused_zr5.cu -- register-resident pass C whose fields arrive by one bulk
// copy per warp and field (fused_zr.cuh, BULK), two fields ahead, for
// power-of-two grid sizes: E = 16 with one or two fields parked (N = 256 to
// 1024) and E = 8 at N = 256.  A warp's lines of a field are contiguous, and
// their LPW Mz complex values make a multiple of 16 bytes at these shapes
// (two lines of 171 at N = 512, one of 342 at 1024, four or two of 86 at 256).
#include "fused_zr.cuh"

namespace nsk {

template <int N> static bool zr_bulk(int E, int tile, ZctKernel *o) {
    if (E == 16) return zr_by_tile<N, 16, 1, 2, true>(tile, o) || zr_by_tile<N, 16, 2, 2, true>(tile, o);
    if constexpr (N == 256)
        if (E == 8) return zr_by_tile<N, 8, 0, 2, true>(tile, o);
    return false;
}

bool zr_lookup5(int N, int E, int tile, ZctKernel *o) {
    switch (N) {
    case 256: return zr_bulk<256>(E, tile, o);
    case 512: return zr_bulk<512>(E, tile, o);
    case 1024: return zr_bulk<1024>(E, tile, o);
    }
    return false;
}

}  // namespace nsk
