// fused.h -- the fused, pruned FP32 form of the solver step.
#pragma once
#include "../../include/ns.h"
#include "ns_internal.h"

#include <vector>

namespace nsk {

// Launch configuration of one pass: its radix plan (elements per thread) and
// its tile (columns per CTA for a strided pass, lines per CTA for pass C).
struct PassCfg {
    Plan pl{};
    int ct = 16;
    int kind = 0;   // 0: runtime-length kernel; 1: compile-time-length kernel (for pass C, ct = warps per CTA);
                    // 2: pass C register-resident kernel (ct = zr_lookup tile), passes A, B, D, E
                    //    constant-geometry kernel (fused_k.cuh)
};

// A pass-C kernel specialised for one grid size (fused_z.cu).
struct ZctKernel {
    const void *k = nullptr;
    size_t smem = 0;
    int lines_per_block = 0;
    int threads = 0;
    int bulk_bytes = 0;   // pass C with bulk copies: bytes of one copy (a warp's lines of one field)
};

// Control block of the register-resident pass C: the context's error word
// (bit 1 set when a bounded wait gave up), the clock-cycle limit of each
// wait, and a test switch that leaves a warp's first bulk copy unissued so
// that the wait for it runs out.
struct ZrCtl {
    int *flags;
    long long wait_cycles;
    int skip_first_copy;
};
// Kernel for grid size N, E elements per thread and wpb warps per CTA, if one
// was compiled (E in {16, 8} or {12, 6}; wpb in {1, 2, 4}).
bool zct_lookup(int N, int E, int wpb, ZctKernel *out);
// Register-resident pass-C kernel (fused_zr.cuh, fused_zr2.cu, fused_zr3.cu,
// fused_zr4.cu): tile = warps per CTA (1 or 2) + ZR_PARK x the number of
// fields parked in shared memory (0, 1: u_x, 2: u_x and u_y), + ZR_ASYNC x
// the load mode: 0 registers, 1 per-lane asynchronous copies two fields
// ahead, 2 one bulk copy per warp and field, two fields ahead.
constexpr int ZR_PARK = 8;
constexpr int ZR_ASYNC = 32;
bool zr_lookup(int N, int E, int tile, ZctKernel *out);
// Pass C of the MHD form (fused_zm.cu): E elements per thread, wpb warps per CTA.
bool zrm_lookup(int N, int E, int wpb, ZctKernel *out);
// Whether grid size N has a compiled MHD pass C (else MHD runs use the plain form).
bool fused_mhd_supported(int N);

// A strided-pass kernel specialised for one (N, E, CT) shape (fused_s*.cu).
struct FzsKernel {
    const void *k = nullptr;
    size_t smem = 0;
    int threads = 0;
};
bool fzs_lookup_A(int N, int E, int CT, FzsKernel *out);    // x inverse + curl
bool fzs_lookup_B(int N, int E, int CT, FzsKernel *out);    // y inverse
bool fzs_lookup_DE(int N, int E, int CT, FzsKernel *out);   // y / x forward
bool fzs_lookup_PF(int N, int E, int CT, FzsKernel *out);   // every row, forward
bool fzs_lookup_PI(int N, int E, int CT, FzsKernel *out);   // every row, inverse

// Standalone-transform z-pass kernel (fft_std_ct.cu).
bool zstd_lookup(int N, bool r2c, int E, int wpb, ZctKernel *out);
// FP32 standalone transforms on compile-time-length kernels.  Return false
// (and launch nothing) when N has no compiled kernels; otherwise *err holds
// the launch status.  c2r handles one field through the scratch tmp.
bool std_r2c_fp32(const float *in, float2 *out, int N, int ncomp, const float2 *tw, cudaStream_t s,
                  cudaError_t *err);
bool std_c2r_fp32(const float2 *in, float2 *tmp, float *out, int N, const float2 *tw, cudaStream_t s,
                  cudaError_t *err);

// Per-run parameters of the update kernel (device array, one per run).
struct FzRunParams {
    float dt, force_amp;
    int force_k, dealias;
    float rot;   // rotation rate about z (Coriolis -2 rot z x u)
    int mfx, mfy, mfz;   // grids and boxes: k_f as the grid index k_f l_i along each axis
};

// A group of nr runs of the fused form that share the grid (and box); their
// buffers are contiguous ([run][...]) so that one launch per pass (grid y =
// run) advances all of them.  Compact state layout [c][ikx][iky][kz] with
// ikx in [0, Mx), iky in [0, My) (index m for m >= 0, m + Mx or m + My for
// m < 0) and kz in [0, Mz): only the modes the 2/3 rule keeps along every
// axis, |m_x| <= K, |m_y| <= Ky, m_z <= Kz.  On the cube N_x = N_y = N_z = n,
// Ky = Kz = K and My = Mx.
struct FusedRun {
    int nr = 0;
    std::vector<ns_run_params> p;   // per run
    int n = 0, K = 0, Mx = 0, Mz = 0;   // n = N_x; K, Mx: along x
    int ny = 0, nz = 0, Ky = 0, Kz = 0, My = 0;
    bool cube = true;            // N_x = N_y = N_z on the unit box
    bool unit = true;            // the unit box: integer wavenumbers, factor table by k^2
    float sx = 1.f, sy = 1.f, sz = 1.f;   // wavenumber per grid index, 1 / l_i
    long D = 0, qx = 0, qy = 0, qz = 0;   // lcm(N_i) and D / N_i (the sphere in integers)
    long M = 0;                  // compact modes per component, Mx * My * Mz
    Plan plN{}, plH{};           // default plans of length n (x) and N_z / 2 (z)
    Plan plY{};                  // and of length N_y (y)
    const float2 *twy = nullptr, *twz = nullptr;   // tables of lengths N_y, N_z (tw: N_x)
    PassCfg sp[4];               // passes A, B, D, E (chosen by the autotuner)
    PassCfg zc;                  // pass C
    int eu_E = 0, eu_ct = 0;     // pass E fused with the update (fused_keu.cu); 0: separate kernels
    // MHD group: a, a1, nl, abuf and bbuf each hold a velocity block (u, w =
    // curl u) and then a magnetic block (b, j = curl b), both with the
    // per-run layout of the Navier-Stokes form; blk_* are the block offsets.
    bool mhd = false;
    long blk_s = 0, blk_A = 0, blk_B = 0;
    float *etab_b = nullptr;     // exp(-eta k^2 dt) by integer k^2       [nr][nk2]
    int zm_E = 0, zm_wpb = 0;    // MHD pass C (fused_zm.cu)
    int *flags = nullptr;        // the context's device error word (set by fused_step)
    int nparts_upd = 0;          // energy partials per run of the separate update kernel
    const float2 *tw = nullptr;  // exp(-2 pi i t / n), t < n (owned by the context)
    float2 *a = nullptr;         // state                       [nr][3][M]
    float2 *a1 = nullptr;        // first-stage state           [nr][3][M]
    float2 *nl = nullptr;        // transform of u x w (compact)[nr][3][M]
    float2 *abuf = nullptr;      // pass A output (6 fields), reused for pass D (3)   [nr][sA]
    float2 *bbuf = nullptr;      // pass B output (6 fields), pass C in place (3)     [nr][sB]
    long sA = 0, sB = 0;         // per-run elements of abuf and bbuf
    float *etab = nullptr;       // exp(-nu k^2 dt) by integer k^2 <= 3 K^2            [nr][nk2]
                                 // (a grid or box: per axis by compact index,        [nr][Mx + My + Mz])
    int nk2 = 0;
    float2 *k2tab = nullptr;     // a grid or box: (m_i / l_i)^2 as FP32 pairs hi + lo, [Mx + My + Mz]
    FzRunParams *rp = nullptr;   // [nr]
    int nparts = 0;              // energy partial sums per run (update kernel blocks)
    double *part = nullptr;      // [nr][nparts][2]
    double *series = nullptr;    // [nr][cap][2] energy / enstrophy ring buffers
    unsigned long long *counter = nullptr;   // [nr] steps recorded
    int cap = 0;
};

bool fused_enabled();
// Allocate a group for runs (all of the same N) and tune its passes.
// tw, twy, twz: the tables exp(-2 pi i t / N_i), t < N_i, of the three axes
// (the same table thrice on the cube).
cudaError_t fused_alloc(FusedRun &f, const std::vector<ns_run_params> &runs, const float2 *tw,
                        const float2 *twy, const float2 *twz, int series_cap, cudaStream_t s);
// Whether the fused form covers a run on a grid of N_x x N_y x N_z points on
// the box of sides 2 pi l_i (the cube always; a grid or box for the
// Navier-Stokes equations with the cubic or spherical 2/3 rule).
bool fused_grid_supported(const ns_run_params &p);
// The full FP32 half layout [3][N_x][N_y][N_z/2+1] of one run's field from
// the compact state (zeros outside the kept modes), into dst.
cudaError_t fused_expand(FusedRun &f, int run, int field, float2 *dst, cudaStream_t s);
void fused_free(FusedRun &f);
cudaError_t fused_set_state(FusedRun &f, int run, int field, const double2 *src, int on_device, void *staging,
                            size_t staging_bytes, cudaStream_t s);
cudaError_t fused_get_state(FusedRun &f, int run, int field, double2 *dst, int on_device, void *staging,
                            size_t staging_bytes, cudaStream_t s);
// One RK2 step of every run of the group.
cudaError_t fused_step(FusedRun &f, int *flags, cudaStream_t s, Tracer *tr);
// JSON text describing the chosen per-pass configuration; returns its length.
int fused_describe(const FusedRun &f, char *out, int len);
cudaError_t fused_spectrum(FusedRun &f, int run, int field, int nbins, double *spec, double *ens,
                           cudaStream_t s);
cudaError_t fused_helicity(FusedRun &f, int run, int nbins, double *spec, double *aux, cudaStream_t s);

}  // namespace nsk
