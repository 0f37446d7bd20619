// fused_zr2.cu -- register-resident pass C for power-of-two grid sizes:
// E = 8 or 4 elements per thread; E = 16 with one or two fields parked at
// N = 256 and 512 (a two-stage plan) and at N = 1024 (where E = 8 would need
// two warps per line).
#include "fused_zr.cuh"

namespace nsk {

template <int N> static bool zr_pow2(int E, int tile, ZctKernel *o) {
    if constexpr (N == 1024) {
        return E == 16 && (zr_by_tile<N, 16, 1>(tile, o) || zr_by_tile<N, 16, 2>(tile, o));
    } else {
        if (E == 8) return zr_by_tile<N, 8, 0>(tile, o);
        if (E == 4) return zr_by_tile<N, 4, 0>(tile, o);
        if constexpr (N == 256 || N == 512)
            if (E == 16) return zr_by_tile<N, 16, 1>(tile, o) || zr_by_tile<N, 16, 2>(tile, o);
        return false;
    }
}

bool zr_lookup2(int N, int E, int tile, ZctKernel *o) {
    switch (N) {
    case 32: return zr_pow2<32>(E, tile, o);
    case 64: return zr_pow2<64>(E, tile, o);
    case 128: return zr_pow2<128>(E, tile, o);
    case 256: return zr_pow2<256>(E, tile, o);
    case 512: return zr_pow2<512>(E, tile, o);
    case 1024: return zr_pow2<1024>(E, tile, o);
    }
    return false;
}

bool zr_lookup(int N, int E, int tile, ZctKernel *o) {
    return zr_lookup2(N, E, tile, o) || zr_lookup3(N, E, tile, o) || zr_lookup4(N, E, tile, o) ||
           zr_lookup5(N, E, tile, o);
}

}  // namespace nsk
