// fused_keu.cu -- pass E of the fused form fused with the update: the x
// forward FFT of the three components of u x w, then, for every kept mode,
// 1/N^3, the Coriolis force, the projection P(k), the forcing and the IF-RK2
// stage (Sec. 2, Eqs. 1-2), and at stage 2 the energy partials.
//
// A CTA owns CT columns (iky, kz) and transforms all three components of
// them one after another; after the last Stockham stage a thread holds the
// positions slot + j T of its column for every component, so it holds all
// three components of those modes and updates them in registers: the
// transform of u x w never returns to HBM.
#include "fused_k.cuh"
#include "fused_update.cuh"
#include "reduce.cuh"

namespace nsk {

template <int N, int E, int CT>
__global__ void __launch_bounds__(CT *(N / E))
k_fzeu(const float2 *__restrict__ din, float2 *__restrict__ a, float2 *__restrict__ a1,
       const float *__restrict__ etab, const FzRunParams *__restrict__ rp, FzUpdate u,
       const float2 *__restrict__ tw, double *__restrict__ part) {
    typedef FzGeom<N, FZ_E> G;
    constexpr int T = N / E;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    __shared__ double red[2 * CT * T];
    const int c = threadIdx.x % CT, slot = threadIdx.x / CT;
    const int run = blockIdx.y;
    const int col = blockIdx.x * CT + c;
    const bool valid = col < G::ncols;
    const int cc = valid ? col : 0;
    const float2 *src = din + run * G::irun + cc;
    auto sl = [&](int e) -> float2 { return sm[TileIndex<E, CT>::at(e, c)]; };
    auto ss = [&](int e, float2 v) { sm[TileIndex<E, CT>::at(e, c)] = v; };

    float2 X[3][E];
#pragma unroll
    for (int f = 0; f < 3; f++) {
        if (f > 0) __syncthreads();   // the previous transform's last reads of the tile
        auto gl = [&](int e) -> float2 {
            return valid ? src[f * G::ifs + e * G::irs] : make_float2(0.f, 0.f);
        };
        ct_fft_block_reg<N, E, -1, N>(X[f], slot, tw, gl, sl, ss);
    }

    const long M = G::M;
    a += run * 3 * M;
    a1 += run * 3 * M;
    etab += (long)run * u.nk2;
    const FzRunParams q = rp[run];
    const float inv = (float)(1.0 / ((double)N * N * N));
    const bool two = u.stage == 2;
    float2 *dst = two ? a : a1;
    const int iky = cc / G::Mz, kz = cc - (cc / G::Mz) * G::Mz;
    const int ky = iky <= G::Ky ? iky : iky - G::My;
    DfAcc e_acc, o_acc;
#pragma unroll
    for (int j = 0; j < E; j++) {
        const int e = slot + j * T;
        const int ikx = FzColK<N, N, N, FZ_E>::compact(e);
        if (!valid || ikx < 0) continue;
        const long m = (long)ikx * G::MyMz + cc;
        const float2 z = make_float2(0.f, 0.f);
        const float2 b0 = a[m], b1 = a[M + m], b2 = a[2 * M + m];
        const float2 c0 = two ? a1[m] : z, c1 = two ? a1[M + m] : z, c2 = two ? a1[2 * M + m] : z;
        const FzMode r = fz_update_k(2 * e < N ? e : e - N, ky, kz, u, q, etab, inv, X[0][j], X[1][j],
                                     X[2][j], b0, b1, b2, c0, c1, c2);
        dst[m] = r.o0;
        dst[M + m] = r.o1;
        dst[2 * M + m] = r.o2;
        if (two) fz_accumulate(r, e_acc, o_acc);
    }
    if (two) {
        double e = e_acc.value(), o = o_acc.value();
        block_sum2(e, o, red);
        if (threadIdx.x == 0) {
            double *pp = part + 2 * ((long)run * u.nparts + blockIdx.x);
            pp[0] = e;
            pp[1] = o;
        }
    }
}

template <int N, int E, int CT> static void fzeu_fill(FzsKernel *o) {
    o->k = (const void *)k_fzeu<N, E, CT>;
    o->smem = (size_t)(N + 1) * TileIndex<E, CT>::rows_stride() * sizeof(float2);
    o->threads = CT * (N / E);
}

bool fzeu_lookup(int N, int E, int CT, FzsKernel *o) {
#define NSK_CASE(n_, e_, ct_)                          \
    if (N == n_ && E == e_ && CT == ct_) {             \
        fzeu_fill<n_, e_, ct_>(o);                     \
        return true;                                   \
    }
    NSK_FZS_SHAPES(NSK_CASE)
#undef NSK_CASE
    return false;
}

}  // namespace nsk
