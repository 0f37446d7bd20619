// fused_k.cuh -- strided passes A, B, D and E of the fused form with the
// whole geometry fixed at compile time.
//
// For a grid of N_x x N_y x N_z points the pruned layouts are constants:
// K_i = (N_i - 1)/3 kept wavenumbers per side, Mx = 2K_x+1 and My = 2K_y+1
// kept rows along x and y, Mz = K_z+1 kept kz, and every field, row, column
// and run stride of every pass follows from them.  With those strides as
// constants, a column splits into (outer, kz) by a division by a constant,
// each thread forms its column's base pointers once, and the per-element
// offsets are 32-bit multiples of constants, which keeps the integer work of
// a load or store to a couple of instructions.  A cube (N_x = N_y = N_z) runs
// on the unit box; any other grid takes the wavenumber per grid index of its
// box (1 / l_i) for the curl of pass A as a kernel argument.
#pragma once
#include "fused_s.cuh"

namespace nsk {

enum { FZ_A = 0, FZ_B = 1, FZ_D = 2, FZ_E = 3 };

// Layouts (per run; runs of a group follow each other):
//   state      [3][ikx][iky][kz]   (M = Mx My Mz per component)
//   A out      [6][iky][x][kz]     (pass A: x inverse of u and w = i k x u)
//   B out      [6][y][x][kz]       (pass B: y inverse; pass C works in place)
//   D out      [3][x][iky][kz]     (pass D: y forward of u x w, kept ky)
//   E out      [3][ikx][iky][kz]   (pass E: x forward, kept kx)
template <int NX, int NY, int NZ, int PASS> struct FzGeom3 {
    static constexpr int Kx = (NX - 1) / 3, Ky = (NY - 1) / 3, Kz = (NZ - 1) / 3;
    static constexpr int Mx = 2 * Kx + 1, My = 2 * Ky + 1, Mz = Kz + 1;
    static constexpr long M = (long)Mx * My * Mz;
    static constexpr int MyMz = My * Mz, NMz = NX * Mz;
    static constexpr long sA = 6L * My * NX * Mz, sB = 6L * NY * NX * Mz, S3 = 3 * M;
    static constexpr bool in_c = PASS == FZ_A || PASS == FZ_B;    // input rows compact
    static constexpr bool out_c = PASS == FZ_D || PASS == FZ_E;   // output rows compact
    static constexpr bool curl = PASS == FZ_A;
    static constexpr bool along_x = PASS == FZ_A || PASS == FZ_E;
    static constexpr bool box = !(NX == NY && NY == NZ);          // scaled wavenumbers in the curl
    static constexpr int L = along_x ? NX : NY;                   // transform length
    static constexpr int K = along_x ? Kx : Ky, Ml = along_x ? Mx : My;   // rows along the line
    static constexpr int Ko = along_x ? Ky : 0, Mo = along_x ? My : 0;    // outer index (passes A, E: iky)
    static constexpr int DIR = in_c ? +1 : -1;
    static constexpr int nfields = in_c ? 6 : 3;
    static constexpr int ncols = along_x ? MyMz : NMz;
    static constexpr long ifs = PASS == FZ_A ? M : PASS == FZ_B ? (long)My * NMz
                              : PASS == FZ_D ? (long)NY * NMz : (long)NX * MyMz;
    static constexpr int irs = along_x ? MyMz : NMz;
    static constexpr long ofs = PASS == FZ_A ? (long)My * NMz : PASS == FZ_B ? (long)NY * NMz
                              : PASS == FZ_D ? (long)NX * MyMz : M;
    static constexpr int ors = PASS == FZ_A ? Mz : PASS == FZ_B ? NMz : PASS == FZ_D ? Mz : MyMz;
    static constexpr long obs = PASS == FZ_A ? NMz : PASS == FZ_B ? Mz : PASS == FZ_D ? MyMz : Mz;
    static constexpr long irun = PASS == FZ_A ? S3 : PASS == FZ_B ? sA : PASS == FZ_D ? sB : sA;
    static constexpr long orun = PASS == FZ_A ? sA : PASS == FZ_B ? sB : PASS == FZ_D ? sA : S3;
    // row offsets stay below 2^31 for every compiled grid
    static_assert((long)L * (irs > ors ? irs : ors) < (1L << 31), "32-bit row offsets");
};
template <int N, int PASS> using FzGeom = FzGeom3<N, N, N, PASS>;

// One column of a pass: grid x is fields x tiles (field fastest), grid y the
// run; column col of field f splits into the outer index ou and kz = iz.
// sc: the wavenumber per grid index along x, y, z (grids other than cubes).
template <int NX, int NY, int NZ, int PASS> struct FzColK {
    typedef FzGeom3<NX, NY, NZ, PASS> G;
    int f;
    bool valid;
    const float2 *ib;
    float2 *ob;
    float kx_s;     // pass A: scale of kx
    float ky, kz;   // pass A: wavenumbers of the column for the curl
    __device__ __forceinline__ FzColK(const float2 *in, float2 *out, int ct, int c, float3 sc) {
        f = blockIdx.x % G::nfields;
        const int tile = blockIdx.x / G::nfields;
        const int col = tile * ct + c;
        valid = col < G::ncols;
        const int cc = valid ? col : 0;
        const int ou = cc / G::Mz, iz = cc - (cc / G::Mz) * G::Mz;
        ib = in + blockIdx.y * G::irun + (long)ou * G::Mz + iz + (G::curl ? 0L : f * G::ifs);
        ob = out + blockIdx.y * G::orun + f * G::ofs + ou * G::obs + iz;
        ky = (float)(ou <= G::Ko ? ou : ou - G::Mo);
        kz = (float)iz;
        kx_s = sc.x;
        if constexpr (G::box) {
            ky *= sc.y;
            kz *= sc.z;
        }
    }
    __device__ __forceinline__ static int compact(int e) {
        return e <= G::K ? e : (e >= G::L - G::K ? e - G::L + G::Ml : -1);
    }
    __device__ __forceinline__ float2 load(int e) const {
        const int r = G::in_c ? compact(e) : e;
        if (!valid || r < 0) return make_float2(0.f, 0.f);
        const float2 *b = ib + r * G::irs;
        if constexpr (!G::curl) {
            return *b;
        } else {
            if (f < 3) return b[f * G::ifs];
            float kx = (float)(2 * e < NX ? e : e - NX);
            if constexpr (G::box) kx *= kx_s;
            float2 p, q;
            float sp, sq;
            if (f == 3) { p = b[2 * G::ifs]; sp = ky; q = b[G::ifs]; sq = kz; }   // i(ky az - kz ay)
            else if (f == 4) { p = b[0]; sp = kz; q = b[2 * G::ifs]; sq = kx; }   // i(kz ax - kx az)
            else { p = b[G::ifs]; sp = kx; q = b[0]; sq = ky; }                   // i(kx ay - ky ax)
            const float re = sp * p.x - sq * q.x, im = sp * p.y - sq * q.y;
            return make_float2(-im, re);
        }
    }
    __device__ __forceinline__ void store(int e, float2 v) const {
        const int r = G::out_c ? compact(e) : e;
        if (!valid || r < 0) return;
        ob[r * G::ors] = v;
    }
};

template <int NX, int NY, int NZ, int E, int CT, int PASS>
__global__ void __launch_bounds__(CT *(FzGeom3<NX, NY, NZ, PASS>::L / E))
k_fzk(const float2 *__restrict__ in, float2 *__restrict__ out, const float2 *__restrict__ tw, float3 sc) {
    typedef FzGeom3<NX, NY, NZ, PASS> G;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int c = threadIdx.x % CT, slot = threadIdx.x / CT;
    const FzColK<NX, NY, NZ, PASS> col(in, out, CT, c, sc);
    auto gl = [&](int e) -> float2 { return col.load(e); };
    auto gs = [&](int e, float2 v) { col.store(e, v); };
    auto sl = [&](int e) -> float2 { return sm[TileIndex<E, CT>::at(e, c)]; };
    auto ss = [&](int e, float2 v) { sm[TileIndex<E, CT>::at(e, c)] = v; };
    ct_fft_block<G::L, E, G::DIR, G::L>(slot, tw, gl, sl, ss, gs);
}

template <int NX, int NY, int NZ, int E, int CT, int PASS> static void fzk_fill(FzsKernel *o) {
    constexpr int L = FzGeom3<NX, NY, NZ, PASS>::L;
    o->k = (const void *)k_fzk<NX, NY, NZ, E, CT, PASS>;
    o->smem = (size_t)(L + 1) * TileIndex<E, CT>::rows_stride() * sizeof(float2);
    o->threads = CT * (L / E);
}

// Grids other than cubes with constant-geometry kernels, (N_x, N_y, N_z, E,
// CT): E and CT hold for the transforms along x and along y.
#define NSK_FZK_GRIDS(X)                                                                          \
    X(96, 96, 48, 12, 8) X(96, 96, 48, 12, 16)                                                    \
    X(512, 512, 256, 16, 8) X(512, 512, 256, 16, 16) X(512, 512, 256, 32, 8)                      \
    X(512, 512, 256, 32, 16) X(512, 512, 256, 8, 8)

// Per-pass lookups (fused_kA.cu, fused_kB.cu, fused_kD.cu, fused_kE.cu):
// the cube N x N x N (NY = NZ = N) or a grid of NSK_FZK_GRIDS.
bool fzk_lookup_A(int NX, int NY, int NZ, int E, int CT, FzsKernel *o);
bool fzk_lookup_B(int NX, int NY, int NZ, int E, int CT, FzsKernel *o);
bool fzk_lookup_D(int NX, int NY, int NZ, int E, int CT, FzsKernel *o);
bool fzk_lookup_E(int NX, int NY, int NZ, int E, int CT, FzsKernel *o);
// Pass E fused with the update (fused_keu.cu); grid x = ceil(Mx Mz / CT)
// column tiles, one energy partial per CTA.
bool fzeu_lookup(int N, int E, int CT, FzsKernel *o);

}  // namespace nsk
