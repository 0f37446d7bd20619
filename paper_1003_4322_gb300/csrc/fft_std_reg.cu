// fft_std_reg.cu -- the compiled register-resident z-pass candidates of the
// standalone FP32 transforms (kernels in fft_std_reg.cuh), four warps per CTA.
#include "fft_std_reg.cuh"

namespace nsk {

template <int N, int E1, int E2> static bool zreg_by(bool r2c, int E, ZctKernel *o) {
    if (E == E1) return zreg_entry<N, E1, 4>(r2c, o);
    if (E2 > 0 && E == E2) return zreg_entry<N, (E2 > 0 ? E2 : E1), 4>(r2c, o);
    // E + 100: the prefetching form, four line groups per warp
    if (E == E1 + 100) return zpf_entry<N, E1, 4, 4>(r2c, o);
    if (E2 > 0 && E == E2 + 100) return zpf_entry<N, (E2 > 0 ? E2 : E1), 4, 4>(r2c, o);
    return false;
}

// Register-resident z kernel for line length N with E elements per thread
// (E + 100: its prefetching form), if one was compiled.
bool zreg_lookup(int N, bool r2c, int E, ZctKernel *o) {
    switch (N) {
    case 256: return zreg_by<256, 8, 16>(r2c, E, o);
    case 384: return zreg_by<384, 6, 12>(r2c, E, o);
    case 512: return zreg_by<512, 8, 16>(r2c, E, o);
    case 768: return zreg_by<768, 12, 0>(r2c, E, o);
    case 1024: return zreg_by<1024, 16, 0>(r2c, E, o);
    }
    return false;
}

}  // namespace nsk
