// fused_zm.cu -- pass C of the MHD form (fused_zr.cuh, k_fused_zr_mhd): E = 8
// (16 at N = 1024) for powers of two, 6 (12 at N = 768) with a factor 3; 1 or 2
// warps per CTA.
#include "fused_zr.cuh"

namespace nsk {

template <int N> static bool zrm_by(int E, int wpb, ZctKernel *o) {
    constexpr bool three = (N / 2) % 3 == 0;
    // the smaller E wherever a line fits one warp with it (fewer registers)
    constexpr int Ek = three ? (N == 768 ? 12 : 6) : (N == 1024 ? 16 : 8);
    if (E != Ek) return false;
    return wpb == 1 ? zrm_entry<N, Ek, 1>(o) : wpb == 2 && zrm_entry<N, Ek, 2>(o);
}

bool zrm_lookup(int N, int E, int wpb, ZctKernel *o) {
    switch (N) {
    case 32: return zrm_by<32>(E, wpb, o);
    case 64: return zrm_by<64>(E, wpb, o);
    case 96: return zrm_by<96>(E, wpb, o);
    case 128: return zrm_by<128>(E, wpb, o);
    case 192: return zrm_by<192>(E, wpb, o);
    case 256: return zrm_by<256>(E, wpb, o);
    case 384: return zrm_by<384>(E, wpb, o);
    case 512: return zrm_by<512>(E, wpb, o);
    case 768: return zrm_by<768>(E, wpb, o);
    case 1024: return zrm_by<1024>(E, wpb, o);
    }
    return false;
}

bool fused_mhd_supported(int N) {
    ZctKernel z;
    const int Es[] = {16, 12, 8, 6};
    for (int E : Es)
        if (zrm_lookup(N, E, 1, &z)) return true;
    return false;
}

}  // namespace nsk
