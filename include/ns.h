/*
 * ns.h -- C ABI of libns, the GB300 (sm_103a) hot path of the pseudospectral
 * incompressible Navier-Stokes solver of Mininni, Rosenberg, Reddy and
 * Pouquet, "A hybrid MPI-OpenMP scheme for scalable parallel pseudospectral
 * computations for fluid turbulence" (Sec. 2, Eqs. 1-2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Box and grid: the (2 pi)^3 periodic box sampled on N^3 points
 *   x_j = 2 pi j / N (Sec. 2).  Physical fields are [ncomp][N][N][N]
 *   (C order, z fastest).  A run may instead have N_x x N_y x N_z points on
 *   a box of sides 2 pi l_x, 2 pi l_y, 2 pi l_z (the domains of aspect ratio
 *   other than one that Sec. 5 says the scheme handles; fields
 *   [ncomp][N_x][N_y][N_z], spectra [ncomp][N_x][N_y][N_z/2+1]); index m
 *   along axis i then stands for the wavenumber m / l_i, and every rule
 *   below that names N holds per axis in grid indices (3 |m_i| < N_i; the
 *   spheres become the ellipsoids sum_i (3 m_i / N_i)^2 < 1 or < 2; the
 *   phase shift is half a grid spacing along every axis).
 * Spectral fields: the r2c half layout [ncomp][N][N][N/2+1] (kx, ky, kz with
 *   kz in [0, N/2] fastest), the C-order mirror of the (N/2+1) x N x M
 *   arrays of Sec. 2, Fig. 1.  Full index i stands for the wavenumber
 *   i (i < N/2) or i - N.  a(-k) = conj(a(k)) supplies the other half (the
 *   printed relation of Sec. 2 carries a spurious minus sign; this is its
 *   reading).  Complex numbers are interleaved (re, im).
 * Transforms: unnormalised both ways, forward exp(-i k.x), inverse
 *   exp(+i k.x).  The c2r direction treats the kz = 0 and kz = N/2 planes as
 *   given and returns the real part of the inverse, so it is exact for
 *   Hermitian-consistent input.
 * Solver state: normalised coefficients a(k) = FFT(u)(k) / N^3, so that
 *   u(x) = sum_k a(k) e^{ik.x}, restricted to the dealiased set Pi.
 * Equations (Sec. 2, Eqs. 1-2, rotational form):
 *   da/dt = -nu |k|^2 a + N(a),
 *   N(a)  = P(k) Pi FFT(u x w)/N^3 + f_hat,  u = IFFT(a), w = IFFT(i k x a),
 *   P(k) v = v - k (k.v)/|k|^2 (projection onto divergence-free fields),
 *   Pi: the 2/3 rule, keep iff 3 max|k_i| < N (dealias = 0) or also
 *   9|k|^2 < N^2 (dealias = 1); the Nyquist index is never kept.
 *   f = F (sin kf z + cos kf y, sin kf x + cos kf z, sin kf y + cos kf x).
 *   Time step: integrating-factor Heun (RK2), E = exp(-nu |k|^2 dt):
 *   a1 = E (a + dt N(a)),  a_next = E a / 2 + (a1 + dt N(a1)) / 2.
 * Supported N: 2^a 3^b with N >= 8, N even and N <= 1024; other N give
 *   NS_ERR_UNSUPPORTED_N.
 * Precision: NS_FP64 is the plain form (unfused, FP64 throughout, in the
 *   full half layout; its transforms skip the lines the dealiasing rule
 *   zeroes or discards, with the same result bit for bit).  NS_FP32 is the
 *   fused form (pruned FP32 transforms and nonlinear term); its twiddle and
 *   integrating-factor tables are generated in FP64 and rounded once, and its
 *   energy, enstrophy and spectrum sums accumulate in FP64.
 *
 * Ownership: the caller owns every pointer it passes; the context owns its
 *   internal device buffers and frees them in ns_destroy.  Nothing is kept
 *   from a caller pointer after a call returns.
 * Errors: every call returns a status; nothing is thrown across the ABI.
 *   CUDA errors are sticky per context: once a call has returned
 *   NS_ERR_CUDA, later calls on the context return it too.  A non-finite
 *   energy, found by ns_sync, ns_energy_spectrum or ns_get_state, returns
 *   NS_ERR_NONFINITE.
 * Streams: work is queued on the stream given to ns_init (NULL = the legacy
 *   default stream) and runs asynchronously unless a call says it syncs.
 * Threading: one context per host thread.
 */
#ifndef NS_H
#define NS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ns_ctx ns_ctx;

typedef enum {
    NS_OK = 0,
    NS_ERR_ARG = 1,            /* invalid argument (null pointer, range) */
    NS_ERR_CUDA = 2,           /* a CUDA runtime call or kernel failed */
    NS_ERR_OOM = 3,            /* device or host allocation failed */
    NS_ERR_UNSUPPORTED_N = 4,  /* N is not 2^a 3^b, even, >= 8, in range */
    NS_ERR_TIMEOUT = 5,        /* a bounded device wait gave up (the fused
                                  FP32 pass C waits at most about a second
                                  for each bulk copy of its input); reported,
                                  like NS_ERR_NONFINITE, by the next call
                                  that checks the context's error word */
    NS_ERR_NONFINITE = 6       /* the energy of a run is NaN or infinite */
} ns_status;

typedef enum { NS_FP64 = 0, NS_FP32 = 1 } ns_prec;

/* One run of the solver (the problem statement of Sec. 2, Eqs. 1-2). */
typedef struct {
    int n;             /* grid points per axis */
    double nu;         /* kinematic viscosity, >= 0 */
    double dt;         /* time step, > 0 */
    double force_amp;  /* ABC forcing amplitude F (0 = unforced) */
    int force_k;       /* ABC forcing wavenumber kf (0 = unforced) */
    int dealias;       /* 0 = cubic 2/3 rule, 1 = spherical 2/3 rule,
                          2 = phase shift: the product also on the grid
                          shifted by (pi/N)(1,1,1), the two averaged, with
                          the sphere 9|k|^2 < 2 N^2 (Navier-Stokes only;
                          twice the transforms; the dealiasing left open in
                          Sec. 2).  A context with a dealias = 2 run uses
                          the plain form in either precision. */
    double rot;        /* rotation rate about z (0 = inertial frame): the
                          Coriolis force -2 rot z x u of the rotating
                          equations (Sec. 5) joins u x w before the
                          projection; any finite value */
    double eta;        /* magnetic diffusivity, >= 0 (used when mhd = 1) */
    int mhd;           /* 1: the magnetohydrodynamic equations of the same
                          code (Sec. 5), Alfven units: a magnetic field b
                          joins the state, j = curl b, the Lorentz force
                          j x b joins u x w, and db/dt = curl(u x b) +
                          eta lap b; b(k = 0) is a constant mean field.
                          FP32 MHD runs use the fused form, unless one of
                          the context's MHD runs has an N without a
                          compiled fused MHD kernel (N other than 32, 64,
                          96, 128, 192, 256, 384, 512, 768, 1024): then the
                          context uses the plain FP32 form.  0:
                          Navier-Stokes. */
    int ny, nz;        /* grid points along y and z (0: n), each 2^a 3^b,
                          even, >= 8.  On a grid other than n^3 or a box
                          side other than 2 pi, FP32 Navier-Stokes runs with
                          dealias 0 or 1 keep the fused form; MHD and
                          dealias 2 there make the context use the plain
                          form */
    double lx, ly, lz; /* box sides in units of 2 pi (0: 1); with forcing,
                          every force_k * l_i must be an integer (the ABC
                          field periodic on the box) */
} ns_run_params;

/* Create a context for nruns independent runs (an ensemble when nruns > 1;
 * runs may have different N) in precision prec, queueing work on
 * cuda_stream (a cudaStream_t, or NULL).  Allocates every device buffer the
 * runs need; states start at zero.  *out receives the context, or NULL on
 * error.  Errors: NS_ERR_ARG (null pointer, nruns < 1, nu < 0, dt <= 0,
 * dealias not 0/1/2, force_k < 0, mhd not 0/1, mhd with dealias 2, eta < 0,
 * ny or nz < 0, a box side < 0 or > 1e6, forcing not periodic on the box,
 * a non-finite parameter), NS_ERR_UNSUPPORTED_N (an axis not supported, or
 * above 1024 points, or more points than 1024^3), NS_ERR_OOM (a plain FP64
 * 1024^3 run needs about 155 GB, an MHD one more than the GPU has),
 * NS_ERR_CUDA. */
ns_status ns_init(const ns_run_params *runs, int nruns, ns_prec prec,
                  void *cuda_stream, ns_ctx **out);

/* Load the state of one run from a full half-layout FP64 complex array
 * [3][N][N][N/2+1], [3][N_x][N_y][N_z/2+1] on other grids (host memory
 * if on_device = 0, device memory if 1).
 * Modes outside Pi are dropped (the Galerkin truncation of Sec. 2); the
 * context converts to its precision and layout.  Synchronous with respect to
 * the host buffer: it may be reused when the call returns.  A page-locked
 * host buffer (cudaHostAlloc'd or registered, 16-byte aligned) is read by the
 * conversion kernels directly; pageable memory is copied through a device
 * staging buffer.  Errors: NS_ERR_ARG (bad run index or null pointer),
 * NS_ERR_CUDA. */
ns_status ns_set_state(ns_ctx *ctx, int run, const void *uhat, int on_device);

/* ns_set_state of runs first .. first + count - 1 from uhats[0 .. count-1]
 * (all host or all device buffers, as on_device says), synchronising once at
 * the end for page-locked or device buffers: every buffer may be reused when
 * the call returns, after an error too.  Sets the velocity (field 0) of each
 * run; an MHD run's magnetic field is loaded with ns_set_field.  On an error
 * the runs before the failing one are loaded.  Errors as ns_set_state. */
ns_status ns_set_states(ns_ctx *ctx, int first, int count, const void *const *uhats, int on_device);

/* Store the state of one run into a full half-layout FP64 complex array
 * [3][N][N][N/2+1] ([3][N_x][N_y][N_z/2+1] on other grids; host if
 * on_device = 0, device if 1); modes outside Pi
 * are written as zero (directly into a page-locked host buffer, else through
 * a device staging buffer).  Synchronises the context's stream.  Errors:
 * NS_ERR_ARG, NS_ERR_CUDA, NS_ERR_NONFINITE. */
ns_status ns_get_state(ns_ctx *ctx, int run, void *uhat, int on_device);

/* ns_set_state / ns_get_state for one field of the state: field 0 is the
 * velocity (the same as those calls), field 1 the magnetic field of an MHD
 * run (same layout; its k = 0 mode is the mean field).  Errors as theirs,
 * and NS_ERR_ARG for field 1 of a Navier-Stokes run. */
ns_status ns_set_field(ns_ctx *ctx, int run, int field, const void *uhat, int on_device);
ns_status ns_get_field(ns_ctx *ctx, int run, int field, void *uhat, int on_device);

/* Advance every run by nsteps integrating-factor RK2 steps (Sec. 2,
 * Eqs. 1-2), queued asynchronously; each step also records the run's energy
 * and enstrophy (FP64) on the device.  Errors: NS_ERR_ARG (nsteps < 0),
 * NS_ERR_CUDA. */
ns_status ns_step(ns_ctx *ctx, int nsteps);

/* Unnormalised forward r2c transform (Sec. 2, Fig. 1) of ncomp real fields
 * [ncomp][n][n][n] at device pointer in, into the half layout
 * [ncomp][n][n][n/2+1] at device pointer out, in the context's precision
 * (float/double in, interleaved complex out).  in and out must not
 * overlap.  Asynchronous on the context's stream.  Errors: NS_ERR_ARG,
 * NS_ERR_UNSUPPORTED_N, NS_ERR_OOM (first call for a new n allocates its
 * tables), NS_ERR_CUDA. */
ns_status ns_fft_r2c(ns_ctx *ctx, int n, int ncomp, const void *in, void *out);

/* Unnormalised inverse c2r transform of ncomp half-layout complex fields at
 * device pointer in into real fields [ncomp][n][n][n] at device pointer out.
 * in is not modified; the context keeps one field of complex scratch per n
 * (allocated on the first call for that n).  Errors as ns_fft_r2c. */
ns_status ns_fft_c2r(ns_ctx *ctx, int n, int ncomp, const void *in, void *out);

/* ns_fft_r2c / ns_fft_c2r on a grid of nx x ny x nz points (each 2^a 3^b,
 * even, >= 8): real fields [ncomp][nx][ny][nz] <-> half-layout complex
 * fields [ncomp][nx][ny][nz/2+1], device pointers, unnormalised, the
 * exponent sum_i 2 pi m_i j_i / n_i (the transform of a field on any box
 * does not depend on its sides).  ncomp * nx <= 65535.  ns_fft_c2r_grid
 * keeps one field of complex scratch (grown to the largest grid asked for)
 * and synchronises the stream when it grows it.  Errors as ns_fft_r2c. */
ns_status ns_fft_r2c_grid(ns_ctx *ctx, int nx, int ny, int nz, int ncomp, const void *in, void *out);
ns_status ns_fft_c2r_grid(ns_ctx *ctx, int nx, int ny, int nz, int ncomp, const void *in, void *out);

/* FP32 inverse c2r transform, as ns_fft_c2r for a context of precision
 * NS_FP32, that allocates nothing.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc, such as applications
 * whose device memory is owned by a caching pool allocator (a raw cudaMalloc
 * can fail or fragment memory the pool holds) and real-time loops that forbid
 * allocation after start-up.  No context is needed.
 *   in:  device pointer, ncomp complex64 fields [ncomp][n][n][n/2+1];
 *   out: device pointer, ncomp float fields [ncomp][n][n][n];
 *   cuda_stream: a cudaStream_t, or NULL for the legacy default stream.
 * Scratch space (one complex field of 128^3 half layout, 8,519,680 bytes)
 * and the twiddle tables of every supported n up to 128 (716 complex64
 * entries) sit in fixed device arrays inside the library, which every GPU
 * that loads libns holds until the process exits; n above 128 (or an
 * unsupported n) returns NS_ERR_UNSUPPORTED_N.  The first call on a device
 * sets that device up: it looks up the arrays' device addresses, fills the
 * twiddle tables from host memory on cuda_stream and waits for that stream;
 * later calls only launch the transform kernels.  Make the first call on each
 * device before any stream capture, and at start-up, before a pool allocator
 * reserves its memory: loading the library's kernels onto the device (which
 * the CUDA driver may defer to first use) takes device memory, including the
 * fixed arrays.  Every call shares the same arrays and overwrites them: calls
 * whose work overlaps on the GPU (other streams, other threads) race and
 * give wrong results, so serialise them.  The function calls no cudaMalloc,
 * cudaFree or allocating library routine.  Asynchronous on cuda_stream after
 * the first call.  Errors: NS_ERR_ARG (null pointer, ncomp < 1),
 * NS_ERR_UNSUPPORTED_N, NS_ERR_CUDA.  It does not reset the CUDA runtime's
 * last-error state: an error raised by the caller's earlier work stays there
 * for the caller to read. */
ns_status ns_fft_c2r_noalloc(int n, int ncomp, const void *in, void *out, void *cuda_stream);

/* Energy E = 1/2 sum |a|^2, enstrophy Omega = 1/2 sum |k|^2 |a|^2 (sums
 * over the full spectrum) and the shell spectrum E(K), K = round-half-up
 * |k|, of one run's current state, accumulated in FP64 (the reductions for
 * global quantities and spectra of Sec. 3).  spec receives
 * min(nbins, ns_run_nbins(run)) shells (spec may be NULL when nbins = 0);
 * on other boxes the shells are round-half-up(|k| / k_min); energy
 * and enstrophy may be NULL.  Host outputs; synchronises the stream.
 * Errors: NS_ERR_ARG, NS_ERR_CUDA, NS_ERR_NONFINITE. */
ns_status ns_energy_spectrum(ns_ctx *ctx, int run, double *spec, int nbins,
                             double *energy, double *enstrophy);

/* ns_energy_spectrum of one field (0: velocity, as ns_energy_spectrum; 1:
 * the magnetic field of an MHD run, E_b = 1/2 sum |b|^2 and 1/2 sum |k|^2
 * |b|^2 = 1/2 <|j|^2>).  Errors as ns_energy_spectrum, and NS_ERR_ARG for
 * field 1 of a Navier-Stokes run. */
ns_status ns_field_spectrum(ns_ctx *ctx, int run, int field, double *spec, int nbins,
                            double *energy, double *enstrophy);

/* ns_energy_spectrum of runs first .. first + count - 1 with one
 * synchronisation (an ensemble's diagnostics in one round trip): spec
 * receives count rows of nbins doubles (row i: run first + i, its
 * ns_run_nbins shells, the rest of the row zeroed; spec may be NULL when
 * nbins = 0); energy and enstrophy receive count values each and may be
 * NULL.  Errors: NS_ERR_ARG (range, null pointer), NS_ERR_CUDA, NS_ERR_OOM,
 * NS_ERR_NONFINITE (some run's energy is not finite). */
ns_status ns_energy_spectra(ns_ctx *ctx, int first, int count, double *spec, int nbins,
                            double *energy, double *enstrophy);

/* Helicity H = 1/2 <u . w> = 1/2 sum Re(a . conj(i k x a)) over the full
 * spectrum and its shell spectrum H(K) (same shells and FP64 accumulation as
 * ns_energy_spectrum) of one run's current state.  The paper does not define
 * it: it is one more global quantity and spectrum of the kind Sec. 3 reduces,
 * the standard invariant of ideal 3D flow; a Beltrami (ABC) field with
 * w = k u has H = k E.  spec
 * receives min(nbins, ns_run_nbins(run)) shells; helicity may be NULL.  Host
 * outputs; synchronises the stream.  Errors: NS_ERR_ARG, NS_ERR_CUDA,
 * NS_ERR_NONFINITE (H is not finite). */
ns_status ns_helicity(ns_ctx *ctx, int run, double *spec, int nbins, double *helicity);

/* Number of shells of an N^3 grid: ceil(sqrt(3) N / 2) + 1. */
int ns_nbins(int n);

/* Number of shells of a run's grid and box: shell K = round-half-up(|k| /
 * k_min) with k_min = 1 / max_i l_i, K = 0 .. ceil(|k_corner| / k_min),
 * k_corner = (N_x / 2l_x, N_y / 2l_y, N_z / 2l_z); ns_nbins(N) on the
 * (2 pi)^3 cube.  0 for a null pointer or n < 2. */
int ns_run_nbins(const ns_run_params *p);

/* Energy and enstrophy recorded by the last `count` steps of one run
 * (oldest first, at most the ring size ns_series_capacity()); fewer are
 * written if fewer steps ran.  *written receives the count.  Host outputs;
 * synchronises the stream.  Errors: NS_ERR_ARG, NS_ERR_CUDA. */
ns_status ns_series(ns_ctx *ctx, int run, int count, double *energy,
                    double *enstrophy, int *written);
int ns_series_capacity(void);

/* Per-kernel timing (the profiling of Sec. 3's benchmarks, which time only
 * the main time-advance loop): runs nsteps steps of every run WITHOUT the
 * CUDA graph, bracketing each kernel launch with a pair of CUDA events on the
 * context's stream, and reports per kernel name the launch count and the
 * summed device time.  The state advances by nsteps steps.  out receives up
 * to max entries; *count receives the number of distinct kernels.
 * Synchronises the stream.  Errors: NS_ERR_ARG, NS_ERR_CUDA. */
typedef struct {
    char name[48];
    int launches;
    double total_ms;
} ns_kernel_time;
ns_status ns_kernel_census(ns_ctx *ctx, int nsteps, ns_kernel_time *out, int max, int *count);

/* Measured FMA rate of the current device, the ALU roof of the transforms
 * (the paper's timings are per step; a roofline needs the device's own
 * arithmetic peak, which for FP64 the specification sheet only estimates).
 * prec NS_FP64 times fma() on doubles, NS_FP32 fmaf() on floats: every thread
 * of a grid that fills each SM to its occupancy limit runs eight independent
 * chains x <- x a + b.  One calibration launch sizes the run to about ms
 * milliseconds per launch; the best of three timed launches (CUDA events on
 * cuda_stream, NULL for the legacy default stream) gives *flops_per_s, at two
 * flops per FMA, at whatever SM clock the device runs.  Synchronises the
 * stream.  Errors: NS_ERR_ARG (null pointer, unknown prec, ms outside
 * (0, 10000]), NS_ERR_CUDA. */
ns_status ns_alu_peak(int prec, double ms, double *flops_per_s, void *cuda_stream);

/* Wait for all queued work and report any sticky or device-side error. */
ns_status ns_sync(ns_ctx *ctx);

/* JSON description of how one run is executed: its form, sizes and, for the
 * fused form, the radix split and tile the autotuner chose for each pass
 * (ns_init runs each pass with a few candidate configurations on the run's
 * own buffers and keeps the fastest, per N, for the life of the process).
 * Writes at most len bytes including the terminating zero (2048 always
 * suffice).  Errors: NS_ERR_ARG (also when the text did not fit in len). */
ns_status ns_describe_run(ns_ctx *ctx, int run, char *out, int len);

/* Detail of the last CUDA failure the context recorded (CUDA error name,
 * message and source location), or "" if none.  Owned by the context. */
const char *ns_last_error(ns_ctx *ctx);

/* Static description of a status code. */
const char *ns_status_str(ns_status s);

/* Free the context and all its device buffers (NULL is accepted). */
void ns_destroy(ns_ctx *ctx);

/* Debug guard bands (no counterpart in the paper; a stand-in for a device
 * memory-error detector).  With NS_GUARD=1 in the environment when the library
 * makes its first allocation, every device buffer it allocates carries 4 KiB
 * of a fixed byte pattern on each side.  ns_guard_check synchronises the
 * device and stores in *bad_bytes how many guard bytes of all live buffers
 * no longer hold the pattern (a kernel wrote outside its buffer), or -1 when
 * guards are off.  ns_guard_selftest writes one byte into the guard of a
 * buffer of its own and stores the count ns_guard_check then reports for it
 * (1 when the scan detects it; -1 when guards are off).  Errors: NS_ERR_ARG
 * (null pointer), NS_ERR_OOM, NS_ERR_CUDA. */
ns_status ns_guard_check(long long *bad_bytes);
ns_status ns_guard_selftest(long long *detected);

#ifdef __cplusplus
}
#endif

#endif /* NS_H */
