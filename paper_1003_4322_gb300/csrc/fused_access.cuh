// fused_access.cuh -- pass descriptors and per-column addressing of the
// strided passes of the fused form (A: x inverse + curl, B: y inverse,
// D: y forward, E: x forward), shared by the runtime-length and the
// compile-time-length kernels.
#pragma once
#include "fft_core.cuh"

namespace nsk {

__device__ __forceinline__ int fz_full_signed(int e, int n) { return 2 * e < n ? e : e - n; }
__device__ __forceinline__ int fz_compact_signed(int i, int Mx, int K) { return i <= K ? i : i - Mx; }
// full index e (0..n-1) -> compact index, or -1 when the wavenumber is not kept
__device__ __forceinline__ int fz_compact(int e, int n, int K, int Mx) {
    if (e <= K) return e;
    if (e >= n - K) return e - n + Mx;
    return -1;
}

struct FzPass {
    const float2 *in;
    float2 *out;
    long ncols;          // flattened columns per field plane
    long ifs, irs;       // input field / row strides (complex elements)
    long ofs, ors, obs;  // output field / row strides; outer stride of a column
    int nfields;         // output fields handled by the grid
    int Mz, K, Mx;       // kept kz; kept |k| and compact rows along the transform axis
    long irun, orun;     // input / output strides between the runs of a group (grid y)
    long ibs;            // input outer stride of a column (input element: ou * ibs + iz)
    // pass A of a grid or box: the compaction of the outer (y) index and the
    // wavenumber per grid index along x, y, z (1 / l_i) for the curl; Mo = 0:
    // the outer index is compacted like the rows (K, Mx) and the scales are 1
    int Ko = 0, Mo = 0;
    float sx = 1.f, sy = 1.f, sz = 1.f;
};

// One column of a strided pass: grid x is fields x tiles (field fastest),
// grid y the run of the group;
// column `col` of field f, its outer index ou = col / Mz and kz = col % Mz.
// IN_C: input rows are compact (only kept wavenumbers stored), the others
// read as zero.  OUT_C: only kept output rows are stored.  CURL: pass A,
// whose fields 3..5 are the vorticity i k x a of the three input components.
template <bool IN_C, bool OUT_C, bool CURL> struct FzColumn {
    int n, f;
    long col, ou, iz;
    bool valid;
    const float2 *in;
    float2 *out;
    __device__ __forceinline__ FzColumn(const FzPass &ps, int n_, int ct, int c) : n(n_) {
        in = ps.in + blockIdx.y * ps.irun;
        out = ps.out + blockIdx.y * ps.orun;
        f = blockIdx.x % ps.nfields;
        const long tile = blockIdx.x / ps.nfields;
        col = tile * ct + c;
        valid = col < ps.ncols;
        ou = valid ? col / ps.Mz : 0;
        iz = valid ? col % ps.Mz : 0;
    }
    __device__ __forceinline__ float2 load(const FzPass &ps, int e) const {
        const int r = IN_C ? fz_compact(e, n, ps.K, ps.Mx) : e;
        if (!valid || r < 0) return make_float2(0.f, 0.f);
        if constexpr (!CURL) {
            return in[f * ps.ifs + r * ps.irs + ou * ps.ibs + iz];
        } else {
            const float2 *b = in + r * ps.irs + ou * ps.ibs + iz;
            if (f < 3) return b[f * ps.ifs];
            float kx = (float)fz_full_signed(e, n);
            float ky = (float)fz_compact_signed((int)ou, ps.Mx, ps.K);
            float kz = (float)iz;
            if (ps.Mo) {   // a grid or a box
                kx *= ps.sx;
                ky = (float)fz_compact_signed((int)ou, ps.Mo, ps.Ko) * ps.sy;
                kz *= ps.sz;
            }
            float2 p, q;
            float sp, sq;
            if (f == 3) { p = b[2 * ps.ifs]; sp = ky; q = b[ps.ifs]; sq = kz; }   // i(ky az - kz ay)
            else if (f == 4) { p = b[0]; sp = kz; q = b[2 * ps.ifs]; sq = kx; }   // i(kz ax - kx az)
            else { p = b[ps.ifs]; sp = kx; q = b[0]; sq = ky; }                   // i(kx ay - ky ax)
            const float re = sp * p.x - sq * q.x, im = sp * p.y - sq * q.y;
            return make_float2(-im, re);
        }
    }
    __device__ __forceinline__ void store(const FzPass &ps, int e, float2 v) const {
        const int r = OUT_C ? fz_compact(e, n, ps.K, ps.Mx) : e;
        if (!valid || r < 0) return;
        out[f * ps.ofs + r * ps.ors + ou * ps.obs + iz] = v;
    }
};

}  // namespace nsk
