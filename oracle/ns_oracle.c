/*
 * ns_oracle.c -- plain FP64 CPU oracle of the pseudospectral Navier-Stokes
 * hot path of Mininni, Rosenberg, Reddy and Pouquet, "A hybrid MPI-OpenMP
 * scheme for scalable parallel pseudospectral computations for fluid
 * turbulence" (Sec. 2, Eqs. 1-2).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * of the package entry file and the CPU-baseline / reference leg of the
 * benchmark may load this library.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * Everything here is the definition written out, in double precision, with no
 * blocking, fusion or reordering beyond what the definitions state:
 *
 *   grid        x_j = 2 pi j / N on the (2 pi)^3 periodic box (Sec. 2);
 *   transforms  unnormalised, forward exp(-i k.x), inverse exp(+i k.x); the
 *               r2c result is kept in the half layout [N][N][N/2+1] with the
 *               halved index fastest (Sec. 2, Fig. 1 caption);  a(-k) =
 *               conj(a(k)) is the symmetry that makes the half sufficient
 *               (the printed relation carries a spurious minus sign; this is
 *               its reading);
 *   state       a(k) = FFT(u)(k) / N^3, so that u(x) = sum_k a(k) e^{ik.x};
 *   Eqs. 1-2    d_t u = u x w - grad(p + |u|^2/2) + nu lap u + f, div u = 0,
 *               i.e. the convective form of Eq. 1 rewritten in rotational
 *               form, the gradient being removed by the projection;
 *   nonlinear   N(a) = P(k) Pi(k) FFT(u x w)/N^3 + f_hat, u = IFFT(Pi a),
 *               w = IFFT(i k x Pi a)  (Sec. 2: product in physical space,
 *               projection onto divergence-free fields, dealiasing);
 *   Pi          cubic 2/3 rule: keep iff 3 max|k_i| < N (dealias = 0), or the
 *               sphere 9|k|^2 < N^2 (dealias = 1);  the Nyquist index is
 *               never kept;
 *   phase shift (dealias = 2, Navier-Stokes only; the dealiasing the
 *               paper's Sec. 2 leaves open, in its phase-shift variant) the
 *               product is evaluated on the grid and on the grid shifted by
 *               D = (pi/N)(1,1,1), i.e. from a(k) e^{i k.D}, the second
 *               transform multiplied by e^{-i k.D}, and the two averaged:
 *               aliases k + N m with odd m_x + m_y + m_z cancel, and with
 *               Pi the sphere 9|k|^2 < 2 N^2 no other alias reaches a kept
 *               mode, so N equals the exact convolution on that sphere;
 *   P           P(k) v = v - k (k.v)/|k|^2, and N(k=0) = 0;
 *   forcing     ABC: f = F (sin kf z + cos kf y, sin kf x + cos kf z,
 *               sin kf y + cos kf x), constant in time, added inside N;
 *   rotation    frame rotating at rate rot about z (the rotating equations the
 *               same code integrates, Sec. 5): the Coriolis force -2 rot z x u
 *               = 2 rot (u_y, -u_x, 0) joins u x w before the projection,
 *               N(a) = P Pi [FFT(u x w)/N^3 + 2 rot (a_y, -a_x, 0)] + f_hat;
 *   MHD         (mhd = 1; the magnetohydrodynamic equations of the same code,
 *               Sec. 5) in Alfven units, state [u; b] of six components,
 *               j = curl b:  N_u = P Pi [FFT(u x w + j x b)/N^3 + Coriolis]
 *               + f_hat,  N_b = Pi [i k x FFT(u x b)/N^3];  b has its own
 *               factor exp(-eta |k|^2 dt), and its mean b(k = 0) is a
 *               constant of the motion;
 *   time step   integrating-factor Heun (RK2), E(k) = exp(-nu |k|^2 dt):
 *               a1 = E (a + dt N(a)),  a' = E a / 2 + (a1 + dt N(a1)) / 2;
 *   diagnostics E = 1/2 sum |a|^2, Omega = 1/2 sum |k|^2 |a|^2 over the full
 *               spectrum (half-layout weight 2 for 0 < kz < N/2, else 1), and
 *               the shell spectrum binned by round-half-up(|k|) (the
 *               reductions for global quantities and spectra of Sec. 3);
 *               helicity H = 1/2 <u . w> = 1/2 sum Re(a . conj(i k x a)) and
 *               its shell spectrum, with the same weights and bins.
 *
 * The paper leaves the dealiasing rule, the integrator, the form of the
 * nonlinear term and the shell binning unstated; the choices above are the
 * readings this oracle fixes.
 *
 * OpenMP pragmas parallelise the loops over independent lines and modes only
 * (the loop-level threading of Sec. 3); results do not depend on the thread
 * count.  Diagnostic sums run serially in a fixed order.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_OOM = 3 };

/* Same field list as the run parameters of the boundary (problem statement
 * of Sec. 2: N, nu, dt, forcing, dealiasing rule; rotation rate, Sec. 5). */
typedef struct {
    int n;
    double nu, dt;
    double force_amp;
    int force_k;
    int dealias;
    double rot;
    double eta;     /* magnetic diffusivity (MHD) */
    int mhd;        /* 1: state [u; b], 6 components */
} or_params;

static const double OR_TWO_PI = 6.283185307179586476925286766559;

int or_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* 1D discrete Fourier transform                                       */
/* ------------------------------------------------------------------ */

static int smallest_factor(int n)
{
    for (int r = 2; r * r <= n; r++)
        if (n % r == 0) return r;
    return n;
}

/* out[k] = sum_{j<n} in[j*is] * w[((j*k) mod n) * ws]  for k < n, where
 * w[t*ws] = exp(sign * 2 pi i t / n).  Decimation in time on the smallest
 * prime factor r of n (Cooley-Tukey): with m = n/r and Y_q the length-m DFT
 * of in[q + r j],  X[k + m s] = sum_q w^{q (k + m s)} Y_q[k].  A prime length
 * is the definition itself. */
static void dft_line(cplx *out, const cplx *in, int n, long is,
                     const cplx *w, int ws)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int r = smallest_factor(n);
    if (r == n) {
        for (int k = 0; k < n; k++) {
            cplx acc = 0;
            for (int j = 0; j < n; j++)
                acc += in[j * is] * w[(int)(((long)j * k) % n) * ws];
            out[k] = acc;
        }
        return;
    }
    int m = n / r;
    for (int q = 0; q < r; q++)
        dft_line(out + q * m, in + q * is, m, is * r, w, ws * r);
    cplx t[r], y[r];
    for (int k = 0; k < m; k++) {
        for (int q = 0; q < r; q++) t[q] = out[q * m + k];
        for (int s = 0; s < r; s++) {
            cplx acc = 0;
            for (int q = 0; q < r; q++)
                acc += t[q] * w[(int)(((long)q * (k + m * s)) % n) * ws];
            y[s] = acc;
        }
        for (int s = 0; s < r; s++) out[k + m * s] = y[s];
    }
}

/* Table w[t] = exp(sign * 2 pi i t / n), t < n, from libm in double. */
static cplx *twiddles(int n, int sign)
{
    cplx *w = malloc(sizeof(cplx) * (size_t)n);
    if (!w) return NULL;
    for (int t = 0; t < n; t++) {
        double a = OR_TWO_PI * (double)t / (double)n;
        w[t] = cos(a) + I * (sign * sin(a));
    }
    return w;
}

/* Transform every line of a full complex n^3 array (x slowest, z fastest)
 * along one axis (0 = x, 1 = y, 2 = z). */
static int fft3_axis(cplx *a, int n, int axis, int sign)
{
    cplx *w = twiddles(n, sign);
    if (!w) return OR_ERR_OOM;
    const long nn = (long)n * n;
    const long stride = axis == 0 ? nn : (axis == 1 ? n : 1);
    int err = 0;
#pragma omp parallel
    {
        cplx *buf = malloc(sizeof(cplx) * 2 * (size_t)n);
        if (!buf) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(static)
        for (long l = 0; l < nn; l++) {
            if (!buf) continue;
            long p = l / n, q = l % n;
            long base = axis == 0 ? l : (axis == 1 ? p * nn + q : p * nn + q * n);
            for (int j = 0; j < n; j++) buf[j] = a[base + j * stride];
            dft_line(buf + n, buf, n, 1, w, 1);
            for (int j = 0; j < n; j++) a[base + j * stride] = buf[n + j];
        }
        free(buf);
    }
    free(w);
    return err ? OR_ERR_OOM : OR_OK;
}

static int fft3_full(cplx *a, int n, int sign)
{
    for (int axis = 2; axis >= 0; axis--) {
        int e = fft3_axis(a, n, axis, sign);
        if (e) return e;
    }
    return OR_OK;
}

/* Forward r2c of ncomp real n^3 fields [c][x][y][z] into the half layout
 * [c][kx][ky][kz], kz <= n/2:  X(k) = sum_x u(x) exp(-i k.x). */
int or_fft3_r2c(int n, int ncomp, const double *in, cplx *out)
{
    if (n < 2 || ncomp < 1 || !in || !out) return OR_ERR_ARG;
    const long V = (long)n * n * n, nh = n / 2 + 1;
    cplx *a = malloc(sizeof(cplx) * (size_t)V);
    if (!a) return OR_ERR_OOM;
    for (int c = 0; c < ncomp; c++) {
        for (long i = 0; i < V; i++) a[i] = in[c * V + i];
        int e = fft3_full(a, n, -1);
        if (e) { free(a); return e; }
        cplx *o = out + (long)c * n * n * nh;
        for (long xy = 0; xy < (long)n * n; xy++)
            for (long kz = 0; kz < nh; kz++) o[xy * nh + kz] = a[xy * n + kz];
    }
    free(a);
    return OR_OK;
}

/* Inverse c2r: complete the half layout by a(kx,ky,kz) = conj(a(-kx,-ky,-kz))
 * for kz > n/2 (the kz = 0 and n/2 planes are taken as given), apply the
 * unnormalised inverse transform u(x) = sum_k a(k) exp(+i k.x) and keep the
 * real part. */
int or_fft3_c2r(int n, int ncomp, const cplx *in, double *out)
{
    if (n < 2 || ncomp < 1 || !in || !out) return OR_ERR_ARG;
    const long V = (long)n * n * n, nh = n / 2 + 1;
    cplx *a = malloc(sizeof(cplx) * (size_t)V);
    if (!a) return OR_ERR_OOM;
    for (int c = 0; c < ncomp; c++) {
        const cplx *h = in + (long)c * n * n * nh;
        for (long x = 0; x < n; x++)
            for (long y = 0; y < n; y++)
                for (long z = 0; z < n; z++) {
                    cplx v;
                    if (z < nh)
                        v = h[(x * n + y) * nh + z];
                    else
                        v = conj(h[(((n - x) % n) * n + (n - y) % n) * nh + (n - z)]);
                    a[(x * n + y) * n + z] = v;
                }
        int e = fft3_full(a, n, +1);
        if (e) { free(a); return e; }
        for (long i = 0; i < V; i++) out[c * V + i] = creal(a[i]);
    }
    free(a);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Spectral operators                                                  */
/* ------------------------------------------------------------------ */

/* Signed wavenumber of full index i (index n/2 maps to -n/2, the Nyquist). */
static int wavenumber(int i, int n) { return 2 * i < n ? i : i - n; }

/* Dealiasing mask Pi: 1 if the mode is kept. */
static int keep(int kx, int ky, int kz, int n, int dealias)
{
    int m = abs(kx);
    if (abs(ky) > m) m = abs(ky);
    if (abs(kz) > m) m = abs(kz);
    if (dealias == 2) return 2 * m < n && 9L * (kx * kx + ky * ky + kz * kz) < 2L * n * n;
    if (3 * m >= n) return 0;
    if (dealias == 1 && 9L * (kx * kx + ky * ky + kz * kz) >= (long)n * n) return 0;
    return 1;
}

/* Apply Pi and then P(k) v = v - k (k.v)/|k|^2 to a half-layout vector field
 * in place; the k = 0 mode is set to zero. */
int or_project(int n, int dealias, cplx *v)
{
    if (n < 2 || !v) return OR_ERR_ARG;
    const long nh = n / 2 + 1, M = (long)n * n * nh;
#pragma omp parallel for schedule(static)
    for (long ix = 0; ix < n; ix++) {
        int kx = wavenumber((int)ix, n);
        for (long iy = 0; iy < n; iy++) {
            int ky = wavenumber((int)iy, n);
            for (long kz = 0; kz < nh; kz++) {
                long m = (ix * n + iy) * nh + kz;
                double k2 = (double)kx * kx + (double)ky * ky + (double)kz * kz;
                if (!keep(kx, ky, (int)kz, n, dealias) || k2 == 0.0) {
                    v[m] = v[M + m] = v[2 * M + m] = 0;
                    continue;
                }
                cplx kv = kx * v[m] + ky * v[M + m] + (double)kz * v[2 * M + m];
                v[m] -= kx * kv / k2;
                v[M + m] -= ky * kv / k2;
                v[2 * M + m] -= (double)kz * kv / k2;
            }
        }
    }
    return OR_OK;
}

/* Apply Pi alone (zero every mode that is not kept). */
static void apply_mask(int n, int dealias, int ncomp, cplx *v)
{
    const long nh = n / 2 + 1, M = (long)n * n * nh;
    for (long ix = 0; ix < n; ix++)
        for (long iy = 0; iy < n; iy++)
            for (long kz = 0; kz < nh; kz++)
                if (!keep(wavenumber((int)ix, n), wavenumber((int)iy, n), (int)kz, n, dealias))
                    for (int c = 0; c < ncomp; c++) v[c * M + (ix * n + iy) * nh + kz] = 0;
}

/* Vorticity coefficients w = i k x a of a half-layout vector field. */
int or_curl(int n, const cplx *a, cplx *w)
{
    if (n < 2 || !a || !w) return OR_ERR_ARG;
    const long nh = n / 2 + 1, M = (long)n * n * nh;
#pragma omp parallel for schedule(static)
    for (long ix = 0; ix < n; ix++) {
        double kx = wavenumber((int)ix, n);
        for (long iy = 0; iy < n; iy++) {
            double ky = wavenumber((int)iy, n);
            for (long kz = 0; kz < nh; kz++) {
                long m = (ix * n + iy) * nh + kz;
                cplx ax = a[m], ay = a[M + m], az = a[2 * M + m];
                w[m] = I * (ky * az - (double)kz * ay);
                w[M + m] = I * ((double)kz * ax - kx * az);
                w[2 * M + m] = I * (kx * ay - ky * ax);
            }
        }
    }
    return OR_OK;
}

/* Coefficients of the ABC forcing, f_hat = FFT(f)/N^3 restricted to Pi,
 * with f sampled on the grid from its definition. */
int or_forcing(const or_params *p, cplx *fh)
{
    if (!p || !fh || p->n < 2) return OR_ERR_ARG;
    const int n = p->n;
    const long V = (long)n * n * n, nh = n / 2 + 1, M = (long)n * n * nh;
    memset(fh, 0, sizeof(cplx) * 3 * (size_t)M);
    if (p->force_k == 0 || p->force_amp == 0.0) return OR_OK;
    double *f = malloc(sizeof(double) * 3 * (size_t)V);
    if (!f) return OR_ERR_OOM;
    const double F = p->force_amp, kf = p->force_k;
    for (long ix = 0; ix < n; ix++)
        for (long iy = 0; iy < n; iy++)
            for (long iz = 0; iz < n; iz++) {
                double x = OR_TWO_PI * ix / n, y = OR_TWO_PI * iy / n, z = OR_TWO_PI * iz / n;
                long i = (ix * n + iy) * n + iz;
                f[i] = F * (sin(kf * z) + cos(kf * y));
                f[V + i] = F * (sin(kf * x) + cos(kf * z));
                f[2 * V + i] = F * (sin(kf * y) + cos(kf * x));
            }
    int e = or_fft3_r2c(n, 3, f, fh);
    free(f);
    if (e) return e;
    for (long i = 0; i < 3 * M; i++) fh[i] /= (double)V;
    apply_mask(n, p->dealias, 3, fh);
    return OR_OK;
}

/* Nonlinear term N(a) = P Pi FFT(u x w)/N^3 + f_hat (Sec. 2, Eqs. 1-2). */
static int nonlinear_mhd(const or_params *p, const cplx *a_in, cplx *out);

/* Velocity part of N from the transformed product already divided by N^3
 * (in out): the Coriolis force of the state a, then Pi and P, then f_hat. */
static int finish_velocity(const or_params *p, const cplx *a, cplx *out)
{
    const int n = p->n;
    const long M = (long)n * n * (n / 2 + 1);
    for (long i = 0; i < M; i++) {                   /* Coriolis -2 rot z x u */
        out[i] += 2.0 * p->rot * a[M + i];
        out[M + i] -= 2.0 * p->rot * a[i];
    }
    int e = or_project(n, p->dealias, out);          /* Pi, then P */
    if (e) return e;
    cplx *fh = malloc(sizeof(cplx) * 3 * (size_t)M);
    if (!fh) return OR_ERR_OOM;
    e = or_forcing(p, fh);
    if (!e)
        for (long i = 0; i < 3 * M; i++) out[i] += fh[i];
    free(fh);
    return e;
}

/* Multiply a half-layout vector field by exp(i sign k.D), D = (pi/N)(1,1,1):
 * its values on the grid shifted by D (sign +1), or back (sign -1). */
static void phase_shift(int n, int sign, cplx *v)
{
    const long nh = n / 2 + 1, M = (long)n * n * nh;
    for (long ix = 0; ix < n; ix++)
        for (long iy = 0; iy < n; iy++)
            for (long kz = 0; kz < nh; kz++) {
                const double t = sign * OR_TWO_PI * 0.5 *
                                 (wavenumber((int)ix, n) + wavenumber((int)iy, n) + (double)kz) / n;
                const cplx ph = cos(t) + I * sin(t);
                for (int c = 0; c < 3; c++) v[c * M + (ix * n + iy) * nh + kz] *= ph;
            }
}

static int product_ns(int n, const cplx *a, cplx *out);

int or_nonlinear(const or_params *p, const cplx *a_in, cplx *out)
{
    if (!p || !a_in || !out || p->n < 2) return OR_ERR_ARG;
    if (p->mhd) return p->dealias == 2 ? OR_ERR_ARG : nonlinear_mhd(p, a_in, out);
    const int n = p->n;
    const long M = (long)n * n * (n / 2 + 1);
    int e = OR_ERR_OOM;
    cplx *a = malloc(sizeof(cplx) * 3 * (size_t)M);
    cplx *as = malloc(sizeof(cplx) * 3 * (size_t)M);
    cplx *o2 = malloc(sizeof(cplx) * 3 * (size_t)M);
    if (!a || !as || !o2) goto done;
    memcpy(a, a_in, sizeof(cplx) * 3 * (size_t)M);
    apply_mask(n, p->dealias, 3, a);                 /* Galerkin truncation */
    if ((e = product_ns(n, a, out))) goto done;      /* FFT(u x w)/N^3 */
    if (p->dealias == 2) {                           /* and on the shifted grid */
        memcpy(as, a, sizeof(cplx) * 3 * (size_t)M);
        phase_shift(n, +1, as);
        if ((e = product_ns(n, as, o2))) goto done;
        phase_shift(n, -1, o2);
        for (long i = 0; i < 3 * M; i++) out[i] = 0.5 * (out[i] + o2[i]);
    }
    e = finish_velocity(p, a, out);
done:
    free(a); free(as); free(o2);
    return e;
}

/* FFT(u x w)/N^3 of a (truncated) half-layout velocity a. */
static int product_ns(int n, const cplx *a, cplx *out)
{
    const long V = (long)n * n * n, nh = n / 2 + 1, M = (long)n * n * nh;
    int e = OR_ERR_OOM;
    cplx *wh = malloc(sizeof(cplx) * 3 * (size_t)M);
    double *u = malloc(sizeof(double) * 3 * (size_t)V);
    double *w = malloc(sizeof(double) * 3 * (size_t)V);
    double *c = malloc(sizeof(double) * 3 * (size_t)V);
    if (!wh || !u || !w || !c) goto done;

    if ((e = or_curl(n, a, wh))) goto done;          /* w_hat = i k x a */
    if ((e = or_fft3_c2r(n, 3, a, u))) goto done;    /* u on the grid */
    if ((e = or_fft3_c2r(n, 3, wh, w))) goto done;   /* w on the grid */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; i++) {                   /* u x w, pointwise */
        c[i] = u[V + i] * w[2 * V + i] - u[2 * V + i] * w[V + i];
        c[V + i] = u[2 * V + i] * w[i] - u[i] * w[2 * V + i];
        c[2 * V + i] = u[i] * w[V + i] - u[V + i] * w[i];
    }
    if ((e = or_fft3_r2c(n, 3, c, out))) goto done;
    for (long i = 0; i < 3 * M; i++) out[i] /= (double)V;
    e = OR_OK;
done:
    free(wh); free(u); free(w); free(c);
    return e;
}

/* MHD nonlinear terms of the six-component state [u; b]. */
static int nonlinear_mhd(const or_params *p, const cplx *a_in, cplx *out)
{
    const int n = p->n;
    const long V = (long)n * n * n, nh = n / 2 + 1, M = (long)n * n * nh;
    int e = OR_ERR_OOM;
    cplx *a = malloc(sizeof(cplx) * 6 * (size_t)M);
    cplx *cw = malloc(sizeof(cplx) * 6 * (size_t)M);     /* curl u, curl b */
    cplx *tb = malloc(sizeof(cplx) * 3 * (size_t)M);
    double *g = malloc(sizeof(double) * 12 * (size_t)V);  /* u, w, b, j on the grid */
    double *c = malloc(sizeof(double) * 6 * (size_t)V);   /* u x w + j x b, u x b */
    if (!a || !cw || !tb || !g || !c) goto done;

    memcpy(a, a_in, sizeof(cplx) * 6 * (size_t)M);
    apply_mask(n, p->dealias, 6, a);                      /* Galerkin truncation */
    if ((e = or_curl(n, a, cw))) goto done;               /* w_hat = i k x u_hat */
    if ((e = or_curl(n, a + 3 * M, cw + 3 * M))) goto done;   /* j_hat = i k x b_hat */
    if ((e = or_fft3_c2r(n, 3, a, g))) goto done;
    if ((e = or_fft3_c2r(n, 3, cw, g + 3 * V))) goto done;
    if ((e = or_fft3_c2r(n, 3, a + 3 * M, g + 6 * V))) goto done;
    if ((e = or_fft3_c2r(n, 3, cw + 3 * M, g + 9 * V))) goto done;
    const double *u = g, *w = g + 3 * V, *b = g + 6 * V, *j = g + 9 * V;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; i++) {
        /* u x w + j x b */
        c[i] = u[V + i] * w[2 * V + i] - u[2 * V + i] * w[V + i]
             + j[V + i] * b[2 * V + i] - j[2 * V + i] * b[V + i];
        c[V + i] = u[2 * V + i] * w[i] - u[i] * w[2 * V + i]
                 + j[2 * V + i] * b[i] - j[i] * b[2 * V + i];
        c[2 * V + i] = u[i] * w[V + i] - u[V + i] * w[i]
                     + j[i] * b[V + i] - j[V + i] * b[i];
        /* u x b */
        c[3 * V + i] = u[V + i] * b[2 * V + i] - u[2 * V + i] * b[V + i];
        c[4 * V + i] = u[2 * V + i] * b[i] - u[i] * b[2 * V + i];
        c[5 * V + i] = u[i] * b[V + i] - u[V + i] * b[i];
    }
    if ((e = or_fft3_r2c(n, 3, c, out))) goto done;
    if ((e = or_fft3_r2c(n, 3, c + 3 * V, tb))) goto done;
    for (long i = 0; i < 3 * M; i++) {
        out[i] /= (double)V;
        tb[i] /= (double)V;
    }
    if ((e = finish_velocity(p, a, out))) goto done;
    if ((e = or_curl(n, tb, out + 3 * M))) goto done;    /* N_b = i k x FFT(u x b) */
    apply_mask(n, p->dealias, 3, out + 3 * M);
    e = OR_OK;
done:
    free(a); free(cw); free(tb); free(g); free(c);
    return e;
}

/* nsteps integrating-factor RK2 (Heun) steps of the state a, in place
 * (three components, or six [u; b] with mhd, b with the factor of eta).
 * The state is first restricted to Pi (the Galerkin space). */
int or_step(const or_params *p, cplx *a, int nsteps)
{
    if (!p || !a || p->n < 2 || nsteps < 0) return OR_ERR_ARG;
    const int n = p->n, nc = p->mhd ? 6 : 3;
    const long nh = n / 2 + 1, M = (long)n * n * nh;
    int e = OR_ERR_OOM;
    double *E = malloc(sizeof(double) * 2 * (size_t)M);   /* nu, then eta */
    cplx *N0 = malloc(sizeof(cplx) * nc * (size_t)M);
    cplx *a1 = malloc(sizeof(cplx) * nc * (size_t)M);
    if (!E || !N0 || !a1) goto done;
    for (long ix = 0; ix < n; ix++) {
        double kx = wavenumber((int)ix, n);
        for (long iy = 0; iy < n; iy++) {
            double ky = wavenumber((int)iy, n);
            for (long kz = 0; kz < nh; kz++) {
                const double k2 = kx * kx + ky * ky + (double)kz * kz;
                E[(ix * n + iy) * nh + kz] = exp(-p->nu * k2 * p->dt);
                E[M + (ix * n + iy) * nh + kz] = exp(-p->eta * k2 * p->dt);
            }
        }
    }
    apply_mask(n, p->dealias, nc, a);
    for (int s = 0; s < nsteps; s++) {
        if ((e = or_nonlinear(p, a, N0))) goto done;
        for (long i = 0; i < nc * M; i++) {
            const double Ei = E[(i >= 3 * M ? M : 0) + i % M];
            a1[i] = Ei * (a[i] + p->dt * N0[i]);
        }
        if ((e = or_nonlinear(p, a1, N0))) goto done;
        for (long i = 0; i < nc * M; i++) {
            const double Ei = E[(i >= 3 * M ? M : 0) + i % M];
            a[i] = 0.5 * Ei * a[i] + 0.5 * (a1[i] + p->dt * N0[i]);
        }
    }
    e = OR_OK;
done:
    free(E); free(N0); free(a1);
    return e;
}

/* Number of shells: K = 0 .. ceil(sqrt(3) n / 2). */
int or_nbins(int n) { return (int)ceil(sqrt(3.0) * n / 2.0) + 1; }

/* Energy, enstrophy and shell spectrum of a half-layout vector field. */
int or_diagnostics(int n, const cplx *a, double *energy, double *enstrophy,
                   double *spec, int nbins)
{
    if (n < 2 || !a) return OR_ERR_ARG;
    const long nh = n / 2 + 1, M = (long)n * n * nh;
    double e = 0.0, om = 0.0;
    if (spec) memset(spec, 0, sizeof(double) * (size_t)nbins);
    for (long ix = 0; ix < n; ix++) {
        double kx = wavenumber((int)ix, n);
        for (long iy = 0; iy < n; iy++) {
            double ky = wavenumber((int)iy, n);
            for (long kz = 0; kz < nh; kz++) {
                long m = (ix * n + iy) * nh + kz;
                double w = (kz == 0 || 2 * kz == n) ? 1.0 : 2.0;
                double k2 = kx * kx + ky * ky + (double)kz * kz;
                double a2 = 0.0;
                for (int c = 0; c < 3; c++) {
                    cplx v = a[c * M + m];
                    a2 += creal(v) * creal(v) + cimag(v) * cimag(v);
                }
                double de = 0.5 * w * a2;
                e += de;
                om += k2 * de;
                long K = (long)floor(sqrt(k2) + 0.5);
                if (spec && K < nbins) spec[K] += de;
            }
        }
    }
    if (energy) *energy = e;
    if (enstrophy) *enstrophy = om;
    return OR_OK;
}

/* Helicity H = 1/2 sum Re(a . conj(w)), w = i k x a, over the full spectrum,
 * and its shell spectrum (same weights and shells as or_diagnostics). */
int or_helicity(int n, const cplx *a, double *helicity, double *spec, int nbins)
{
    if (n < 2 || !a) return OR_ERR_ARG;
    const long nh = n / 2 + 1, M = (long)n * n * nh;
    cplx *w = malloc(sizeof(cplx) * 3 * (size_t)M);
    if (!w) return OR_ERR_OOM;
    or_curl(n, a, w);
    double h = 0.0;
    if (spec) memset(spec, 0, sizeof(double) * (size_t)nbins);
    for (long ix = 0; ix < n; ix++) {
        double kx = wavenumber((int)ix, n);
        for (long iy = 0; iy < n; iy++) {
            double ky = wavenumber((int)iy, n);
            for (long kz = 0; kz < nh; kz++) {
                long m = (ix * n + iy) * nh + kz;
                double wt = (kz == 0 || 2 * kz == n) ? 1.0 : 2.0;
                double s = 0.0;
                for (int c = 0; c < 3; c++) s += creal(a[c * M + m] * conj(w[c * M + m]));
                double dh = 0.5 * wt * s;
                h += dh;
                long K = (long)floor(sqrt(kx * kx + ky * ky + (double)kz * kz) + 0.5);
                if (spec && K < nbins) spec[K] += dh;
            }
        }
    }
    free(w);
    if (helicity) *helicity = h;
    return OR_OK;
}
