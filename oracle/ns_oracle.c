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
 *               more generally N_x x N_y x N_z points on a box of sides
 *               2 pi l_x, 2 pi l_y, 2 pi l_z (the domains of aspect ratio
 *               other than one that the conclusions, Sec. 5, say the scheme
 *               handles), where index m along axis i stands for the
 *               wavenumber k_i = m / l_i;
 *   transforms  unnormalised, forward exp(-i k.x), inverse exp(+i k.x); the
 *               r2c result is kept in the half layout [N_x][N_y][N_z/2+1]
 *               with the halved index fastest (Sec. 2, Fig. 1 caption);  a(-k) =
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
 *               never kept;  on an N_x x N_y x N_z grid the rules hold per
 *               axis in grid indices: 3 |m_i| < N_i for every i, and the
 *               ellipsoid sum_i (3 m_i / N_i)^2 < 1 for the sphere;
 *   phase shift (dealias = 2, Navier-Stokes only; the dealiasing the
 *               paper's Sec. 2 leaves open, in its phase-shift variant) the
 *               product is evaluated on the grid and on the grid shifted by
 *               D = (pi/N)(1,1,1), i.e. from a(k) e^{i k.D}, the second
 *               transform multiplied by e^{-i k.D}, and the two averaged:
 *               aliases k + N m with odd m_x + m_y + m_z cancel, and with
 *               Pi the sphere 9|k|^2 < 2 N^2 no other alias reaches a kept
 *               mode, so N equals the exact convolution on that sphere;
 *               on other grids and boxes the shift is half a grid spacing
 *               along every axis (k.D = pi sum_i m_i / N_i) and the sphere
 *               is the ellipsoid sum_i (3 m_i / N_i)^2 < 2;
 *   P           P(k) v = v - k (k.v)/|k|^2, and N(k=0) = 0;
 *   forcing     ABC: f = F (sin kf z + cos kf y, sin kf x + cos kf z,
 *               sin kf y + cos kf x), constant in time, added inside N
 *               (periodic on the box only if every kf l_i is an integer;
 *               other boxes are refused);
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
 *               reductions for global quantities and spectra of Sec. 3), on
 *               other boxes by round-half-up(|k| / k_min) with k_min =
 *               1 / max_i l_i the smallest nonzero wavenumber;
 *               helicity H = 1/2 <u . w> = 1/2 sum Re(a . conj(i k x a)) and
 *               its shell spectrum, with the same weights and bins.
 *
 * The paper leaves the dealiasing rule, the integrator, the form of the
 * nonlinear term, the shell binning and the treatment of boxes of other
 * aspect ratios unstated; the choices above are the readings this oracle
 * fixes.
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
 * of Sec. 2: N, nu, dt, forcing, dealiasing rule; rotation rate, MHD and the
 * box of other aspect ratios, Sec. 5). */
typedef struct {
    int n;          /* grid points along x (and along y, z when ny, nz are 0) */
    double nu, dt;
    double force_amp;
    int force_k;
    int dealias;
    double rot;
    double eta;     /* magnetic diffusivity (MHD) */
    int mhd;        /* 1: state [u; b], 6 components */
    int ny, nz;     /* grid points along y and z (0: n) */
    double lx, ly, lz;   /* box sides in units of 2 pi (0: 1) */
} or_params;

/* Grid and box of a run: points per axis, box sides / (2 pi), and the sizes
 * of the half layout [nx][ny][nz/2+1] and of a field on the grid. */
typedef struct {
    int n[3];
    double l[3];
    long nzh, M, V;
} grid;

static const double OR_TWO_PI = 6.283185307179586476925286766559;

static grid make_grid(int nx, int ny, int nz, double lx, double ly, double lz)
{
    grid g;
    g.n[0] = nx; g.n[1] = ny; g.n[2] = nz;
    g.l[0] = lx; g.l[1] = ly; g.l[2] = lz;
    g.nzh = nz / 2 + 1;
    g.M = (long)nx * ny * g.nzh;
    g.V = (long)nx * ny * nz;
    return g;
}

static grid cube(int n) { return make_grid(n, n, n, 1.0, 1.0, 1.0); }

static grid grid_of(const or_params *p)
{
    return make_grid(p->n, p->ny > 0 ? p->ny : p->n, p->nz > 0 ? p->nz : p->n,
                     p->lx > 0 ? p->lx : 1.0, p->ly > 0 ? p->ly : 1.0, p->lz > 0 ? p->lz : 1.0);
}

static int grid_ok(const grid *g)
{
    for (int i = 0; i < 3; i++)
        if (g->n[i] < 2 || g->n[i] % 2 || !(g->l[i] > 0.0) || !isfinite(g->l[i])) return 0;
    return 1;
}

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

/* Transform every line of a full complex nx x ny x nz array (x slowest, z
 * fastest) along one axis (0 = x, 1 = y, 2 = z). */
static int fft3_axis(cplx *a, const int d[3], int axis, int sign)
{
    const int n = d[axis];
    cplx *w = twiddles(n, sign);
    if (!w) return OR_ERR_OOM;
    const long sx = (long)d[1] * d[2], sy = d[2];
    const long stride = axis == 0 ? sx : (axis == 1 ? sy : 1);
    const long lines = (long)d[0] * d[1] * d[2] / n;
    int err = 0;
#pragma omp parallel
    {
        cplx *buf = malloc(sizeof(cplx) * 2 * (size_t)n);
        if (!buf) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(static)
        for (long l = 0; l < lines; l++) {
            if (!buf) continue;
            /* the line's fixed coordinates, in the order of the other axes */
            long base;
            if (axis == 0) base = l;                                /* (y, z) */
            else if (axis == 1) base = (l / d[2]) * sx + l % d[2];  /* (x, z) */
            else base = l * d[2];                                   /* (x, y) */
            for (int j = 0; j < n; j++) buf[j] = a[base + j * stride];
            dft_line(buf + n, buf, n, 1, w, 1);
            for (int j = 0; j < n; j++) a[base + j * stride] = buf[n + j];
        }
        free(buf);
    }
    free(w);
    return err ? OR_ERR_OOM : OR_OK;
}

static int fft3_full(cplx *a, const int d[3], int sign)
{
    for (int axis = 2; axis >= 0; axis--) {
        int e = fft3_axis(a, d, axis, sign);
        if (e) return e;
    }
    return OR_OK;
}

/* Forward r2c of ncomp real fields [c][x][y][z] (nx x ny x nz) into the half
 * layout [c][kx][ky][kz], kz <= nz/2:  X(k) = sum_x u(x) exp(-i k.x). */
int or_fft3_r2c_grid(int nx, int ny, int nz, int ncomp, const double *in, cplx *out)
{
    if (nx < 2 || ny < 2 || nz < 2 || ncomp < 1 || !in || !out) return OR_ERR_ARG;
    const int d[3] = {nx, ny, nz};
    const long V = (long)nx * ny * nz, nh = nz / 2 + 1;
    cplx *a = malloc(sizeof(cplx) * (size_t)V);
    if (!a) return OR_ERR_OOM;
    for (int c = 0; c < ncomp; c++) {
        for (long i = 0; i < V; i++) a[i] = in[c * V + i];
        int e = fft3_full(a, d, -1);
        if (e) { free(a); return e; }
        cplx *o = out + (long)c * nx * ny * nh;
        for (long xy = 0; xy < (long)nx * ny; xy++)
            for (long kz = 0; kz < nh; kz++) o[xy * nh + kz] = a[xy * nz + kz];
    }
    free(a);
    return OR_OK;
}

/* Inverse c2r: complete the half layout by a(kx,ky,kz) = conj(a(-kx,-ky,-kz))
 * for kz > nz/2 (the kz = 0 and nz/2 planes are taken as given), apply the
 * unnormalised inverse transform u(x) = sum_k a(k) exp(+i k.x) and keep the
 * real part. */
int or_fft3_c2r_grid(int nx, int ny, int nz, int ncomp, const cplx *in, double *out)
{
    if (nx < 2 || ny < 2 || nz < 2 || ncomp < 1 || !in || !out) return OR_ERR_ARG;
    const int d[3] = {nx, ny, nz};
    const long V = (long)nx * ny * nz, nh = nz / 2 + 1;
    cplx *a = malloc(sizeof(cplx) * (size_t)V);
    if (!a) return OR_ERR_OOM;
    for (int c = 0; c < ncomp; c++) {
        const cplx *h = in + (long)c * nx * ny * nh;
        for (long x = 0; x < nx; x++)
            for (long y = 0; y < ny; y++)
                for (long z = 0; z < nz; z++) {
                    cplx v;
                    if (z < nh)
                        v = h[(x * ny + y) * nh + z];
                    else
                        v = conj(h[(((nx - x) % nx) * ny + (ny - y) % ny) * nh + (nz - z)]);
                    a[(x * ny + y) * nz + z] = v;
                }
        int e = fft3_full(a, d, +1);
        if (e) { free(a); return e; }
        for (long i = 0; i < V; i++) out[c * V + i] = creal(a[i]);
    }
    free(a);
    return OR_OK;
}

int or_fft3_r2c(int n, int ncomp, const double *in, cplx *out)
{
    return or_fft3_r2c_grid(n, n, n, ncomp, in, out);
}

int or_fft3_c2r(int n, int ncomp, const cplx *in, double *out)
{
    return or_fft3_c2r_grid(n, n, n, ncomp, in, out);
}

/* ------------------------------------------------------------------ */
/* Spectral operators                                                  */
/* ------------------------------------------------------------------ */

/* Signed index of full index i (index n/2 maps to -n/2, the Nyquist). */
static int wavenumber(int i, int n) { return 2 * i < n ? i : i - n; }

/* Half-layout position m -> signed indices (mx, my, mz) and the physical
 * wavevector k_i = m_i / l_i. */
static void mode_of(const grid *g, long m, int mi[3], double k[3])
{
    const long kz = m % g->nzh, iy = (m / g->nzh) % g->n[1], ix = m / (g->nzh * g->n[1]);
    mi[0] = wavenumber((int)ix, g->n[0]);
    mi[1] = wavenumber((int)iy, g->n[1]);
    mi[2] = (int)kz;
    for (int i = 0; i < 3; i++) k[i] = mi[i] / g->l[i];
}

static long gcd_l(long a, long b) { return b ? gcd_l(b, a % b) : a; }

/* Dealiasing mask Pi: 1 if the mode with signed indices mi is kept.  The
 * ellipsoid sum_i (3 m_i / N_i)^2 < c is tested exactly in integers, over
 * the common denominator D = lcm(N_x, N_y, N_z). */
static int keep(const int mi[3], const grid *g, int dealias)
{
    long D = g->n[0];
    for (int i = 1; i < 3; i++) D = D / gcd_l(D, g->n[i]) * g->n[i];
    long s = 0;
    int cube_ok = 1, half_ok = 1;
    for (int i = 0; i < 3; i++) {
        const long mm = labs((long)mi[i]);
        if (3 * mm >= g->n[i]) cube_ok = 0;
        if (2 * mm >= g->n[i]) half_ok = 0;
        const long q = mm * (D / g->n[i]);
        s += q * q;
    }
    if (dealias == 2) return half_ok && 9 * s < 2 * D * D;
    if (!cube_ok) return 0;
    if (dealias == 1 && 9 * s >= D * D) return 0;
    return 1;
}

/* Apply Pi and then P(k) v = v - k (k.v)/|k|^2 to a half-layout vector field
 * in place; the k = 0 mode is set to zero. */
static void project_g(const grid *g, int dealias, cplx *v)
{
    const long M = g->M;
#pragma omp parallel for schedule(static)
    for (long m = 0; m < M; m++) {
        int mi[3];
        double k[3];
        mode_of(g, m, mi, k);
        const double kx = k[0], ky = k[1], kz = k[2];
        double k2 = kx * kx + ky * ky + kz * kz;
        if (!keep(mi, g, dealias) || k2 == 0.0) {
            v[m] = v[M + m] = v[2 * M + m] = 0;
            continue;
        }
        cplx kv = kx * v[m] + ky * v[M + m] + kz * v[2 * M + m];
        v[m] -= kx * kv / k2;
        v[M + m] -= ky * kv / k2;
        v[2 * M + m] -= kz * kv / k2;
    }
}

int or_project(int n, int dealias, cplx *v)
{
    if (n < 2 || !v) return OR_ERR_ARG;
    const grid g = cube(n);
    project_g(&g, dealias, v);
    return OR_OK;
}

int or_project_p(const or_params *p, cplx *v)
{
    if (!p || !v) return OR_ERR_ARG;
    const grid g = grid_of(p);
    if (!grid_ok(&g)) return OR_ERR_ARG;
    project_g(&g, p->dealias, v);
    return OR_OK;
}

/* Apply Pi alone (zero every mode that is not kept). */
static void apply_mask(const grid *g, int dealias, int ncomp, cplx *v)
{
    for (long m = 0; m < g->M; m++) {
        int mi[3];
        double k[3];
        mode_of(g, m, mi, k);
        if (!keep(mi, g, dealias))
            for (int c = 0; c < ncomp; c++) v[c * g->M + m] = 0;
    }
}

/* Vorticity coefficients w = i k x a of a half-layout vector field. */
static void curl_g(const grid *g, const cplx *a, cplx *w)
{
    const long M = g->M;
#pragma omp parallel for schedule(static)
    for (long m = 0; m < M; m++) {
        int mi[3];
        double k[3];
        mode_of(g, m, mi, k);
        const double kx = k[0], ky = k[1], kz = k[2];
        cplx ax = a[m], ay = a[M + m], az = a[2 * M + m];
        w[m] = I * (ky * az - kz * ay);
        w[M + m] = I * (kz * ax - kx * az);
        w[2 * M + m] = I * (kx * ay - ky * ax);
    }
}

int or_curl(int n, const cplx *a, cplx *w)
{
    if (n < 2 || !a || !w) return OR_ERR_ARG;
    const grid g = cube(n);
    curl_g(&g, a, w);
    return OR_OK;
}

int or_curl_p(const or_params *p, const cplx *a, cplx *w)
{
    if (!p || !a || !w) return OR_ERR_ARG;
    const grid g = grid_of(p);
    if (!grid_ok(&g)) return OR_ERR_ARG;
    curl_g(&g, a, w);
    return OR_OK;
}

/* Coefficients of the ABC forcing, f_hat = FFT(f)/V restricted to Pi, with
 * f sampled on the grid x_i = 2 pi l_i j / N_i from its definition. */
int or_forcing(const or_params *p, cplx *fh)
{
    if (!p || !fh) return OR_ERR_ARG;
    const grid g = grid_of(p);
    if (!grid_ok(&g)) return OR_ERR_ARG;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long V = g.V, M = g.M;
    memset(fh, 0, sizeof(cplx) * 3 * (size_t)M);
    if (p->force_k == 0 || p->force_amp == 0.0) return OR_OK;
    for (int i = 0; i < 3; i++) {      /* f must be periodic on the box */
        const double t = p->force_k * g.l[i];
        if (fabs(t - nearbyint(t)) > 1e-9 * t) return OR_ERR_ARG;
    }
    double *f = malloc(sizeof(double) * 3 * (size_t)V);
    if (!f) return OR_ERR_OOM;
    const double F = p->force_amp, kf = p->force_k;
    for (long ix = 0; ix < nx; ix++)
        for (long iy = 0; iy < ny; iy++)
            for (long iz = 0; iz < nz; iz++) {
                double x = OR_TWO_PI * g.l[0] * ix / nx, y = OR_TWO_PI * g.l[1] * iy / ny,
                       z = OR_TWO_PI * g.l[2] * iz / nz;
                long i = (ix * ny + iy) * nz + iz;
                f[i] = F * (sin(kf * z) + cos(kf * y));
                f[V + i] = F * (sin(kf * x) + cos(kf * z));
                f[2 * V + i] = F * (sin(kf * y) + cos(kf * x));
            }
    int e = or_fft3_r2c_grid(nx, ny, nz, 3, f, fh);
    free(f);
    if (e) return e;
    for (long i = 0; i < 3 * M; i++) fh[i] /= (double)V;
    apply_mask(&g, p->dealias, 3, fh);
    return OR_OK;
}

/* Nonlinear term N(a) = P Pi FFT(u x w)/V + f_hat (Sec. 2, Eqs. 1-2). */
static int nonlinear_mhd(const or_params *p, const cplx *a_in, cplx *out);

/* Velocity part of N from the transformed product already divided by V
 * (in out): the Coriolis force of the state a, then Pi and P, then f_hat. */
static int finish_velocity(const or_params *p, const cplx *a, cplx *out)
{
    const grid g = grid_of(p);
    const long M = g.M;
    for (long i = 0; i < M; i++) {                   /* Coriolis -2 rot z x u */
        out[i] += 2.0 * p->rot * a[M + i];
        out[M + i] -= 2.0 * p->rot * a[i];
    }
    project_g(&g, p->dealias, out);                  /* Pi, then P */
    cplx *fh = malloc(sizeof(cplx) * 3 * (size_t)M);
    if (!fh) return OR_ERR_OOM;
    int e = or_forcing(p, fh);
    if (!e)
        for (long i = 0; i < 3 * M; i++) out[i] += fh[i];
    free(fh);
    return e;
}

/* Multiply a half-layout vector field by exp(i sign k.D), D half a grid
 * spacing along every axis, k.D = pi (m_x/N_x + m_y/N_y + m_z/N_z): its
 * values on the shifted grid (sign +1), or back (sign -1). */
static void phase_shift(const grid *g, int sign, cplx *v)
{
    for (long m = 0; m < g->M; m++) {
        int mi[3];
        double k[3];
        mode_of(g, m, mi, k);
        const double t = sign * OR_TWO_PI * 0.5 *
                         ((double)mi[0] / g->n[0] + (double)mi[1] / g->n[1] + (double)mi[2] / g->n[2]);
        const cplx ph = cos(t) + I * sin(t);
        for (int c = 0; c < 3; c++) v[c * g->M + m] *= ph;
    }
}

static int product_ns(const grid *g, const cplx *a, cplx *out);

int or_nonlinear(const or_params *p, const cplx *a_in, cplx *out)
{
    if (!p || !a_in || !out) return OR_ERR_ARG;
    const grid g = grid_of(p);
    if (!grid_ok(&g)) return OR_ERR_ARG;
    if (p->mhd) return p->dealias == 2 ? OR_ERR_ARG : nonlinear_mhd(p, a_in, out);
    const long M = g.M;
    int e = OR_ERR_OOM;
    cplx *a = malloc(sizeof(cplx) * 3 * (size_t)M);
    cplx *as = malloc(sizeof(cplx) * 3 * (size_t)M);
    cplx *o2 = malloc(sizeof(cplx) * 3 * (size_t)M);
    if (!a || !as || !o2) goto done;
    memcpy(a, a_in, sizeof(cplx) * 3 * (size_t)M);
    apply_mask(&g, p->dealias, 3, a);                /* Galerkin truncation */
    if ((e = product_ns(&g, a, out))) goto done;     /* FFT(u x w)/V */
    if (p->dealias == 2) {                           /* and on the shifted grid */
        memcpy(as, a, sizeof(cplx) * 3 * (size_t)M);
        phase_shift(&g, +1, as);
        if ((e = product_ns(&g, as, o2))) goto done;
        phase_shift(&g, -1, o2);
        for (long i = 0; i < 3 * M; i++) out[i] = 0.5 * (out[i] + o2[i]);
    }
    e = finish_velocity(p, a, out);
done:
    free(a); free(as); free(o2);
    return e;
}

/* FFT(u x w)/V of a (truncated) half-layout velocity a. */
static int product_ns(const grid *g, const cplx *a, cplx *out)
{
    const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const long V = g->V, M = g->M;
    int e = OR_ERR_OOM;
    cplx *wh = malloc(sizeof(cplx) * 3 * (size_t)M);
    double *u = malloc(sizeof(double) * 3 * (size_t)V);
    double *w = malloc(sizeof(double) * 3 * (size_t)V);
    double *c = malloc(sizeof(double) * 3 * (size_t)V);
    if (!wh || !u || !w || !c) goto done;

    curl_g(g, a, wh);                                          /* w_hat = i k x a */
    if ((e = or_fft3_c2r_grid(nx, ny, nz, 3, a, u))) goto done;    /* u on the grid */
    if ((e = or_fft3_c2r_grid(nx, ny, nz, 3, wh, w))) goto done;   /* w on the grid */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; i++) {                   /* u x w, pointwise */
        c[i] = u[V + i] * w[2 * V + i] - u[2 * V + i] * w[V + i];
        c[V + i] = u[2 * V + i] * w[i] - u[i] * w[2 * V + i];
        c[2 * V + i] = u[i] * w[V + i] - u[V + i] * w[i];
    }
    if ((e = or_fft3_r2c_grid(nx, ny, nz, 3, c, out))) goto done;
    for (long i = 0; i < 3 * M; i++) out[i] /= (double)V;
    e = OR_OK;
done:
    free(wh); free(u); free(w); free(c);
    return e;
}

/* MHD nonlinear terms of the six-component state [u; b]. */
static int nonlinear_mhd(const or_params *p, const cplx *a_in, cplx *out)
{
    const grid g = grid_of(p);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long V = g.V, M = g.M;
    int e = OR_ERR_OOM;
    cplx *a = malloc(sizeof(cplx) * 6 * (size_t)M);
    cplx *cw = malloc(sizeof(cplx) * 6 * (size_t)M);     /* curl u, curl b */
    cplx *tb = malloc(sizeof(cplx) * 3 * (size_t)M);
    double *gr = malloc(sizeof(double) * 12 * (size_t)V);  /* u, w, b, j on the grid */
    double *c = malloc(sizeof(double) * 6 * (size_t)V);   /* u x w + j x b, u x b */
    if (!a || !cw || !tb || !gr || !c) goto done;

    memcpy(a, a_in, sizeof(cplx) * 6 * (size_t)M);
    apply_mask(&g, p->dealias, 6, a);                     /* Galerkin truncation */
    curl_g(&g, a, cw);                                    /* w_hat = i k x u_hat */
    curl_g(&g, a + 3 * M, cw + 3 * M);                    /* j_hat = i k x b_hat */
    if ((e = or_fft3_c2r_grid(nx, ny, nz, 3, a, gr))) goto done;
    if ((e = or_fft3_c2r_grid(nx, ny, nz, 3, cw, gr + 3 * V))) goto done;
    if ((e = or_fft3_c2r_grid(nx, ny, nz, 3, a + 3 * M, gr + 6 * V))) goto done;
    if ((e = or_fft3_c2r_grid(nx, ny, nz, 3, cw + 3 * M, gr + 9 * V))) goto done;
    const double *u = gr, *w = gr + 3 * V, *b = gr + 6 * V, *j = gr + 9 * V;
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
    if ((e = or_fft3_r2c_grid(nx, ny, nz, 3, c, out))) goto done;
    if ((e = or_fft3_r2c_grid(nx, ny, nz, 3, c + 3 * V, tb))) goto done;
    for (long i = 0; i < 3 * M; i++) {
        out[i] /= (double)V;
        tb[i] /= (double)V;
    }
    if ((e = finish_velocity(p, a, out))) goto done;
    curl_g(&g, tb, out + 3 * M);                          /* N_b = i k x FFT(u x b) */
    apply_mask(&g, p->dealias, 3, out + 3 * M);
    e = OR_OK;
done:
    free(a); free(cw); free(tb); free(gr); free(c);
    return e;
}

/* Time integrators.  The paper names none (Sec. 3 speaks only of the time
 * advance); OR_IF_HEUN is the reading every other part of the oracle and the
 * product use.  The other two are for comparison only:
 *   OR_IF_MIDPOINT  integrating factor with the midpoint rule, E_h =
 *                   exp(-nu |k|^2 dt / 2):  a_h = E_h (a + dt/2 N(a)),
 *                   a' = E a + dt E_h N(a_h);
 *   OR_RK2          Heun on da/dt = N(a) - nu |k|^2 a with the viscous
 *                   (and resistive) term explicit:  L(a) = N(a) - nu k^2 a,
 *                   a1 = a + dt L(a),  a' = a + dt/2 (L(a) + L(a1)). */
enum { OR_IF_HEUN = 0, OR_IF_MIDPOINT = 1, OR_RK2 = 2 };

int or_step_with(const or_params *p, int integrator, cplx *a, int nsteps)
{
    if (!p || !a || nsteps < 0 || integrator < OR_IF_HEUN || integrator > OR_RK2) return OR_ERR_ARG;
    const grid g = grid_of(p);
    if (!grid_ok(&g)) return OR_ERR_ARG;
    const int nc = p->mhd ? 6 : 3;
    const long M = g.M;
    int e = OR_ERR_OOM;
    double *E = malloc(sizeof(double) * 2 * (size_t)M);    /* full step: nu, then eta */
    double *Eh = malloc(sizeof(double) * 2 * (size_t)M);   /* half step */
    double *lam = malloc(sizeof(double) * 2 * (size_t)M);  /* nu |k|^2, then eta |k|^2 */
    cplx *N0 = malloc(sizeof(cplx) * nc * (size_t)M);
    cplx *N1 = malloc(sizeof(cplx) * nc * (size_t)M);
    cplx *a1 = malloc(sizeof(cplx) * nc * (size_t)M);
    if (!E || !Eh || !lam || !N0 || !N1 || !a1) goto done;
    for (long m = 0; m < M; m++) {
        int mi[3];
        double k[3];
        mode_of(&g, m, mi, k);
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        lam[m] = p->nu * k2;
        lam[M + m] = p->eta * k2;
        E[m] = exp(-lam[m] * p->dt);
        E[M + m] = exp(-lam[M + m] * p->dt);
        Eh[m] = exp(-lam[m] * p->dt / 2);
        Eh[M + m] = exp(-lam[M + m] * p->dt / 2);
    }
    apply_mask(&g, p->dealias, nc, a);
    for (int s = 0; s < nsteps; s++) {
        if ((e = or_nonlinear(p, a, N0))) goto done;
        for (long i = 0; i < nc * M; i++) {
            const long t = (i >= 3 * M ? M : 0) + i % M;
            if (integrator == OR_IF_HEUN) a1[i] = E[t] * (a[i] + p->dt * N0[i]);
            else if (integrator == OR_IF_MIDPOINT) a1[i] = Eh[t] * (a[i] + 0.5 * p->dt * N0[i]);
            else a1[i] = a[i] + p->dt * (N0[i] - lam[t] * a[i]);
        }
        if ((e = or_nonlinear(p, a1, N1))) goto done;
        for (long i = 0; i < nc * M; i++) {
            const long t = (i >= 3 * M ? M : 0) + i % M;
            if (integrator == OR_IF_HEUN) a[i] = 0.5 * E[t] * a[i] + 0.5 * (a1[i] + p->dt * N1[i]);
            else if (integrator == OR_IF_MIDPOINT) a[i] = E[t] * a[i] + p->dt * Eh[t] * N1[i];
            else a[i] = a[i] + 0.5 * p->dt * ((N0[i] - lam[t] * a[i]) + (N1[i] - lam[t] * a1[i]));
        }
    }
    e = OR_OK;
done:
    free(E); free(Eh); free(lam); free(N0); free(N1); free(a1);
    return e;
}

/* nsteps integrating-factor RK2 (Heun) steps of the state a, in place
 * (three components, or six [u; b] with mhd, b with the factor of eta).
 * The state is first restricted to Pi (the Galerkin space). */
int or_step(const or_params *p, cplx *a, int nsteps)
{
    if (!p || !a || nsteps < 0) return OR_ERR_ARG;
    const grid g = grid_of(p);
    if (!grid_ok(&g)) return OR_ERR_ARG;
    const int nc = p->mhd ? 6 : 3;
    const long M = g.M;
    int e = OR_ERR_OOM;
    double *E = malloc(sizeof(double) * 2 * (size_t)M);   /* nu, then eta */
    cplx *N0 = malloc(sizeof(cplx) * nc * (size_t)M);
    cplx *a1 = malloc(sizeof(cplx) * nc * (size_t)M);
    if (!E || !N0 || !a1) goto done;
    for (long m = 0; m < M; m++) {
        int mi[3];
        double k[3];
        mode_of(&g, m, mi, k);
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        E[m] = exp(-p->nu * k2 * p->dt);
        E[M + m] = exp(-p->eta * k2 * p->dt);
    }
    apply_mask(&g, p->dealias, nc, a);
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

/* Smallest nonzero wavenumber 1 / max_i l_i: the width of a shell. */
static double kmin_of(const grid *g)
{
    double lm = g->l[0];
    for (int i = 1; i < 3; i++)
        if (g->l[i] > lm) lm = g->l[i];
    return 1.0 / lm;
}

/* Number of shells: K = 0 .. ceil(|k|_max / k_min), |k|_max the corner
 * (N_x/2l_x, N_y/2l_y, N_z/2l_z); ceil(sqrt(3) n / 2) + 1 on the cube. */
static int nbins_g(const grid *g)
{
    if (g->n[0] == g->n[1] && g->n[1] == g->n[2] && g->l[0] == 1.0 && g->l[1] == 1.0 && g->l[2] == 1.0)
        return (int)ceil(sqrt(3.0) * g->n[0] / 2.0) + 1;
    double s = 0.0;
    for (int i = 0; i < 3; i++) {
        const double c = g->n[i] / 2 / g->l[i];
        s += c * c;
    }
    return (int)ceil(sqrt(s) / kmin_of(g)) + 1;
}

int or_nbins(int n)
{
    const grid g = cube(n);
    return nbins_g(&g);
}

int or_nbins_p(const or_params *p)
{
    if (!p) return 0;
    const grid g = grid_of(p);
    return grid_ok(&g) ? nbins_g(&g) : 0;
}

/* Energy, enstrophy and shell spectrum of a half-layout vector field: shell
 * K = round-half-up(|k| / k_min). */
static void diagnostics_g(const grid *g, const cplx *a, double *energy, double *enstrophy,
                          double *spec, int nbins)
{
    const long M = g->M;
    const double lmax = 1.0 / kmin_of(g);
    double e = 0.0, om = 0.0;
    if (spec) memset(spec, 0, sizeof(double) * (size_t)nbins);
    for (long m = 0; m < M; m++) {
        int mi[3];
        double k[3];
        mode_of(g, m, mi, k);
        double w = (mi[2] == 0 || 2 * mi[2] == g->n[2]) ? 1.0 : 2.0;
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double a2 = 0.0;
        for (int c = 0; c < 3; c++) {
            cplx v = a[c * M + m];
            a2 += creal(v) * creal(v) + cimag(v) * cimag(v);
        }
        double de = 0.5 * w * a2;
        e += de;
        om += k2 * de;
        long K = (long)floor(sqrt(k2) * lmax + 0.5);
        if (spec && K < nbins) spec[K] += de;
    }
    if (energy) *energy = e;
    if (enstrophy) *enstrophy = om;
}

int or_diagnostics(int n, const cplx *a, double *energy, double *enstrophy,
                   double *spec, int nbins)
{
    if (n < 2 || !a) return OR_ERR_ARG;
    const grid g = cube(n);
    diagnostics_g(&g, a, energy, enstrophy, spec, nbins);
    return OR_OK;
}

int or_diagnostics_p(const or_params *p, const cplx *a, double *energy, double *enstrophy,
                     double *spec, int nbins)
{
    if (!p || !a) return OR_ERR_ARG;
    const grid g = grid_of(p);
    if (!grid_ok(&g)) return OR_ERR_ARG;
    diagnostics_g(&g, a, energy, enstrophy, spec, nbins);
    return OR_OK;
}

/* Helicity H = 1/2 sum Re(a . conj(w)), w = i k x a, over the full spectrum,
 * and its shell spectrum (same weights and shells as the diagnostics). */
static int helicity_g(const grid *g, const cplx *a, double *helicity, double *spec, int nbins)
{
    const long M = g->M;
    const double lmax = 1.0 / kmin_of(g);
    cplx *w = malloc(sizeof(cplx) * 3 * (size_t)M);
    if (!w) return OR_ERR_OOM;
    curl_g(g, a, w);
    double h = 0.0;
    if (spec) memset(spec, 0, sizeof(double) * (size_t)nbins);
    for (long m = 0; m < M; m++) {
        int mi[3];
        double k[3];
        mode_of(g, m, mi, k);
        double wt = (mi[2] == 0 || 2 * mi[2] == g->n[2]) ? 1.0 : 2.0;
        double s = 0.0;
        for (int c = 0; c < 3; c++) s += creal(a[c * M + m] * conj(w[c * M + m]));
        double dh = 0.5 * wt * s;
        h += dh;
        long K = (long)floor(sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]) * lmax + 0.5);
        if (spec && K < nbins) spec[K] += dh;
    }
    free(w);
    if (helicity) *helicity = h;
    return OR_OK;
}

int or_helicity(int n, const cplx *a, double *helicity, double *spec, int nbins)
{
    if (n < 2 || !a) return OR_ERR_ARG;
    const grid g = cube(n);
    return helicity_g(&g, a, helicity, spec, nbins);
}

int or_helicity_p(const or_params *p, const cplx *a, double *helicity, double *spec, int nbins)
{
    if (!p || !a) return OR_ERR_ARG;
    const grid g = grid_of(p);
    if (!grid_ok(&g)) return OR_ERR_ARG;
    return helicity_g(&g, a, helicity, spec, nbins);
}
