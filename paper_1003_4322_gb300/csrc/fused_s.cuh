// fused_s.cuh -- strided passes of the fused form for compile-time grid
// sizes: the same columns and addressing as the runtime-length kernel
// (fused_access.cuh), with N, the radix split E and the columns per CTA CT
// fixed at compile time.  Instantiated per pass mode in fused_sA.cu,
// fused_sB.cu and fused_sDE.cu.
#pragma once
#include "fft_ct.cuh"
#include "fused.h"
#include "fused_access.cuh"

namespace nsk {

// Shared tile row of element e.  With 16 columns a half-warp covers one row,
// and a padded stride (17) keeps it conflict-free.  With 8 columns a
// half-warp covers two rows, which must fall in opposite bank halves: rows
// are 8 elements (half the banks) apart, and the row index is XORed with the
// parity of e / E so that the rows E apart written by the first stage also
// alternate (consecutive rows of one block of E alternate by themselves).
template <int E, int CT> struct TileIndex {
    static __device__ __forceinline__ int at(int e, int c) {
        if constexpr (CT == 8) return ((e ^ ((e / E) & 1)) << 3) + c;
        else return e * (CT + 1) + c;
    }
    static constexpr int rows_stride() { return CT == 8 ? 8 : CT + 1; }
};

template <int N, int E, int CT, int DIR, bool IN_C, bool OUT_C, bool CURL>
__global__ void __launch_bounds__(CT *(N / E))
k_fzs_ct(FzPass ps, const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int c = threadIdx.x % CT, slot = threadIdx.x / CT;
    const FzColumn<IN_C, OUT_C, CURL> col(ps, N, CT, c);
    auto gl = [&](int e) -> float2 { return col.load(ps, e); };
    auto gs = [&](int e, float2 v) { col.store(ps, e, v); };
    auto sl = [&](int e) -> float2 { return sm[TileIndex<E, CT>::at(e, c)]; };
    auto ss = [&](int e, float2 v) { sm[TileIndex<E, CT>::at(e, c)] = v; };
    ct_fft_block<N, E, DIR, N>(slot, tw, gl, sl, ss, gs);
}

// (N, E, CT) shapes compiled for every pass mode.
#define NSK_FZS_SHAPES(X)                                                                         \
    X(64, 16, 8) X(64, 16, 16) X(64, 8, 16)                                                       \
    X(96, 12, 8) X(96, 12, 16)                                                                    \
    X(128, 16, 8) X(128, 16, 16) X(128, 8, 16)                                                    \
    X(192, 12, 8) X(192, 12, 16)                                                                  \
    X(256, 16, 8) X(256, 16, 16) X(256, 32, 16) X(256, 8, 16)                                     \
    X(384, 12, 8) X(384, 12, 16)                                                                  \
    X(512, 16, 8) X(512, 16, 16) X(512, 32, 8) X(512, 32, 16) X(512, 8, 8)                        \
    X(768, 12, 8)                                                                                 \
    X(1024, 16, 8) X(1024, 32, 8) X(1024, 32, 16)

template <int N, int E, int CT, int DIR, bool IN_C, bool OUT_C, bool CURL>
static void fzs_fill(FzsKernel *o) {
    o->k = (const void *)k_fzs_ct<N, E, CT, DIR, IN_C, OUT_C, CURL>;
    o->smem = (size_t)(N + 1) * TileIndex<E, CT>::rows_stride() * sizeof(float2);
    o->threads = CT * (N / E);
}

}  // namespace nsk
