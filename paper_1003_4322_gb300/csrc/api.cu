// api.cu -- the C ABI of libns (include/ns.h): context, state transfer,
// time stepping (captured once per context into a CUDA graph), standalone
// transforms and FP64 diagnostics.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <tuple>
#include <type_traits>
#include <map>
#include <mutex>
#include <memory>
#include <new>
#include <vector>

#include "../../include/ns.h"
#include "fused.h"
#include "ns_internal.h"
#include "plain.h"
#include "reduce.cuh"

using namespace nsk;

namespace {

const int kSeriesCap = 4096;

// Launch shapes of the plain form's transforms: radix splits of the x/y
// passes (inverse, forward) and of the z passes, columns per CTA of the x/y
// passes.  Defaults from make_plan / default_ct, replaced by the plain-form
// autotuner's choice (tune_plain) once per (N, precision) in the process.
struct PlainPlans {
    Plan inv{}, fwd{}, zc{}, zr{};
    int ct_inv = 0, ct_fwd = 0;
    bool tuned = false;
};

struct FftRes {
    int n = 0;
    Plan plN{}, plH{};
    PlainPlans pp;
    void *tw = nullptr;       // Cx<T>[n], exp(-2 pi i t / n)
    void *scratch = nullptr;  // one half-layout field (c2r)
};

// The largest |m_i| per axis that a run's dealiasing rule keeps: the plain
// form's transforms skip the lines beyond them (on = false: every line).
struct PlainPrune {
    bool on = false;
    int kx = 0, ky = 0, kz = 0;
};

struct Run {
    ns_run_params p{};
    int n = 0;    // N_x (the N of a cubic run)
    Grid g;       // grid and box
    PlainPlans gp[3];   // grid runs: the run's own plans for the x, y and z passes
    PlainPrune prune;   // lines of the step's transforms that are skipped
    long M = 0;   // modes per component, half layout
    long V = 0;   // grid points per component
    // plain form (full half layout)
    void *un = nullptr, *u1 = nullptr, *wn = nullptr, *work = nullptr, *phys = nullptr;
    void *sh = nullptr, *sh2 = nullptr;   // phase-shift dealiasing: shifted state, its product
    void *phtab = nullptr;                // per-axis shift factors exp(i pi m / N_i)
    void *etab = nullptr;   // exp(-nu k^2 dt) by integer k^2 (unit boxes)
    void *etab_b = nullptr; // MHD: exp(-eta k^2 dt); un, u1, wn then hold [u; b] (6 components)
    // fused form: the run is member gidx of group `group` of the context
    int group = -1, gidx = 0;
    // diagnostics (plain form owns them; fused runs point into their group)
    double *part = nullptr;
    double *series = nullptr;
    unsigned long long *counter = nullptr;
    int nparts = 0;
    bool owns_diag = true;
};

}  // namespace

struct ns_ctx {
    ns_prec prec = NS_FP64;
    cudaStream_t stream = nullptr;   // caller's stream
    cudaStream_t cap = nullptr;      // private stream for graph capture
    // independent units of a step (fused groups, or plain runs) are captured
    // on these streams, forked from and joined back to `cap`, so that the
    // graph runs them concurrently
    std::vector<cudaStream_t> par;
    std::vector<cudaEvent_t> fork_join;   // [0]: fork; [1 + i]: join of par[i]
    std::vector<Run> runs;
    std::vector<FusedRun> groups;   // fused form: runs grouped by N
    std::map<int, FftRes> fft;
    ns_status sticky = NS_OK;
    int *flags = nullptr;            // device error word (bit 0: non-finite energy, bit 1: a bounded
                                     // device wait gave up)
    double *spec = nullptr, *ens = nullptr;
    int spec_cap = 0;
    void *staging = nullptr;
    size_t staging_bytes = 0;
    bool plain_only = false;         // a run the fused form does not cover (MHD at a size
                                     // without a compiled kernel, phase-shift dealiasing,
                                     // or a grid or box other than the cube)
    void *gscratch = nullptr;        // c2r scratch of the grid transforms
    size_t gscratch_bytes = 0;
    double *bspec = nullptr;         // batched spectra: per run nbins results + partials, twice
    size_t bspec_runs = 0;
    cudaGraphExec_t graph = nullptr;
    char last_error[256] = {0};
};

namespace {

size_t elem_bytes(ns_prec p) { return p == NS_FP64 ? sizeof(double) : sizeof(float); }

// Grid and box of a run: ny, nz = 0 mean N; box sides 0 mean 2 pi.
Grid run_grid(const ns_run_params &p) {
    return make_grid(p.n, p.ny > 0 ? p.ny : p.n, p.nz > 0 ? p.nz : p.n, p.lx > 0 ? p.lx : 1.0,
                     p.ly > 0 ? p.ly : 1.0, p.lz > 0 ? p.lz : 1.0);
}

ns_status fail_cuda_at(ns_ctx *c, cudaError_t e, int line) {
    if (c)
        snprintf(c->last_error, sizeof(c->last_error), "%s (%s) at api.cu:%d", cudaGetErrorName(e),
                 cudaGetErrorString(e), line);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return NS_ERR_OOM;
    }
    if (c) c->sticky = NS_ERR_CUDA;
    return NS_ERR_CUDA;
}
#define fail_cuda(c, e) fail_cuda_at((c), (e), __LINE__)

#define NS_CK(expr)                                   \
    do {                                              \
        cudaError_t _e = (expr);                      \
        if (_e != cudaSuccess) return fail_cuda(c, _e); \
    } while (0)

template <typename P> cudaError_t dalloc(P **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    return dev_malloc((void **)p, bytes);
}

// Per-n transform resources (plans, twiddles, c2r scratch), created once.
ns_status get_fft(ns_ctx *c, int n, FftRes **out) {
    auto it = c->fft.find(n);
    if (it != c->fft.end()) {
        *out = &it->second;
        return NS_OK;
    }
    FftRes f;
    f.n = n;
    if (!make_plan(n, &f.plN) || !make_plan(n / 2, &f.plH)) return NS_ERR_UNSUPPORTED_N;
    f.pp.inv = f.pp.fwd = f.plN;
    f.pp.zc = f.pp.zr = f.plH;
    f.pp.ct_inv = f.pp.ct_fwd = default_ct(c->prec == NS_FP64 ? 16 : 8, n);
    cudaError_t e;
    if (c->prec == NS_FP64) f.tw = make_twiddles<double>(n, &e);
    else f.tw = make_twiddles<float>(n, &e);
    if (!f.tw) return fail_cuda(c, e);
    c->fft[n] = f;
    *out = &c->fft[n];
    return NS_OK;
}

// Transform resources of the three axes of a grid (the same entry thrice on
// the cube).
ns_status get_fft3(ns_ctx *c, const Grid &g, FftRes *f[3]) {
    const int n[3] = {g.nx, g.ny, g.nz};
    for (int i = 0; i < 3; i++) {
        ns_status st = get_fft(c, n[i], &f[i]);
        if (st != NS_OK) return st;
    }
    return NS_OK;
}

ns_status ensure_scratch(ns_ctx *c, FftRes *f) {
    if (f->scratch) return NS_OK;
    const size_t bytes = (size_t)f->n * f->n * (f->n / 2 + 1) * 2 * elem_bytes(c->prec);
    NS_CK(dalloc(&f->scratch, bytes));
    return NS_OK;
}

// ---------------------------------------------------------------- transforms

// Per-axis transform resources of a grid: x, y and z (all the same on the
// cube), and the plans of the x, y and z passes (those of the resources, or
// a grid run's own).
struct Fft3 {
    const FftRes *x = nullptr, *y = nullptr, *z = nullptr;
    const PlainPlans *px = nullptr, *py = nullptr, *pz = nullptr;
    Fft3() = default;
    Fft3(const FftRes *x_, const FftRes *y_, const FftRes *z_, const PlainPlans *px_, const PlainPlans *py_,
         const PlainPlans *pz_)
        : x(x_), y(y_), z(z_), px(px_), py(py_), pz(pz_) {}
};

// FP32 transforms of a grid whose axis lengths have compile-time kernels go
// through the tuned standalone path (fft_std_ct.cu); its shapes are chosen on
// the first call, which the plain form makes before any graph capture.
inline StdGrid std_grid(const Grid &g, const Fft3 &f) {
    return StdGrid{g.nx, g.ny, g.nz, (const float2 *)f.x->tw, (const float2 *)f.y->tw,
                   (const float2 *)f.z->tw};
}

// The lines of the x and y passes a pruned step transforms.  A field inside
// Pi is zero on every x line (fixed ky, kz) with |ky| > K_y or kz > K_z and on
// every y line with kz > K_z, and rows |kx| > K_x (x) and |ky| > K_y (y) of
// the others are zero; the forward passes need the same lines and rows only,
// because the update reads the transform inside Pi alone.  x pass: the plane
// [ky][kz] as N_y rows of N_z/2+1 columns, the kept ky rows and their first
// K_z + 1 columns, rows kx in the gap; y pass: the plane [kz] (one row), its
// first K_z + 1 columns, rows ky in the gap.
static void prune_sels(const Grid &g, const PlainPrune &p, StridedSel *sx, StridedSel *sy) {
    const long nh = g.nzh();
    sx->inner = nh;
    sx->nouter = g.ny;
    sx->keep = p.kz + 1;
    sx->o1 = p.ky + 1;
    sx->o2 = std::max(g.ny - p.ky, sx->o1);
    sx->gap_lo = p.kx + 1;
    sx->gap_hi = std::max(g.nx - p.kx, sx->gap_lo);
    sy->inner = nh;
    sy->nouter = 1;
    sy->keep = p.kz + 1;
    sy->o1 = sy->o2 = 1;
    sy->gap_lo = p.ky + 1;
    sy->gap_hi = std::max(g.ny - p.ky, sy->gap_lo);
}

// c2r of ncomp half fields [ncomp][N_x][N_y][N_z/2+1]: x pass (in -> tmp), y
// pass (tmp in place), z pass (tmp -> out [ncomp][N_x][N_y][N_z]).  FP32 on
// compiled lengths: the standalone kernels, one field at a time through tmp.
// pr (on): the fields lie inside the run's Pi, and only the lines that can be
// nonzero are transformed (the rest of tmp is neither read nor written).
template <typename T>
cudaError_t c2r_batch(const typename Cx<T>::type *in, typename Cx<T>::type *tmp, T *out, const Grid &g,
                      int ncomp, const Fft3 &f, cudaStream_t s, Tracer *tr = nullptr,
                      const PlainPrune *pr = nullptr) {
    typedef typename Cx<T>::type C;
    if constexpr (std::is_same<T, float>::value) {
        const StdGrid sg = std_grid(g, f);
        cudaError_t e = cudaSuccess;
        bool done = true;
        if (tr) tr->begin("fft_c2r_std");
        for (int k = 0; k < ncomp && done && e == cudaSuccess; k++)
            done = std_c2r_fp32_grid(in + k * g.M(), tmp, out + k * g.V(), sg, s, &e);
        if (tr) tr->end();
        if (done) return e;
    }
    const long nh = g.nzh(), plane = (long)g.ny * nh, M = (long)g.nx * plane;
    const PlainPlans &qx = *f.px, &qy = *f.py, &qz = *f.pz;
    const bool pruned = pr && pr->on;
    StridedSel sx, sy;
    if (pruned) prune_sels(g, *pr, &sx, &sy);
    cudaError_t e = NSK_TIMED(tr, "fft_x_inverse",
                              fft_strided<T>(in, tmp, plane, plane, M, M, ncomp, +1, qx.inv, (const C *)f.x->tw,
                                             g.nx, qx.ct_inv, s, pruned ? &sx : nullptr));
    if (e != cudaSuccess) return e;
    e = NSK_TIMED(tr, "fft_y_inverse",
                  fft_strided<T>(tmp, tmp, nh, nh, plane, plane, ncomp * g.nx, +1, qy.inv, (const C *)f.y->tw,
                                 g.ny, qy.ct_inv, s, pruned ? &sy : nullptr));
    if (e != cudaSuccess) return e;
    return NSK_TIMED(tr, "fft_z_c2r",
                     fft_z_c2r<T>(tmp, out, g.nz, (long)ncomp * g.nx * g.ny, qz.zc, (const C *)f.z->tw, s,
                                  pruned ? pr->kz + 1 : -1));
}

// r2c of ncomp real fields: z pass (in -> out), y and x passes in place.
// pr (on): only the modes inside the run's Pi are wanted; the others are left
// partly transformed or untouched.
template <typename T>
cudaError_t r2c_batch(const T *in, typename Cx<T>::type *out, const Grid &g, int ncomp, const Fft3 &f,
                      cudaStream_t s, Tracer *tr = nullptr, const PlainPrune *pr = nullptr) {
    typedef typename Cx<T>::type C;
    if constexpr (std::is_same<T, float>::value) {
        cudaError_t e = cudaSuccess;
        if (tr) tr->begin("fft_r2c_std");
        const bool done = std_r2c_fp32_grid(in, out, std_grid(g, f), ncomp, s, &e);
        if (tr) tr->end();
        if (done) return e;
    }
    const long nh = g.nzh(), plane = (long)g.ny * nh, M = (long)g.nx * plane;
    const PlainPlans &qx = *f.px, &qy = *f.py, &qz = *f.pz;
    const bool pruned = pr && pr->on;
    StridedSel sx, sy;
    if (pruned) prune_sels(g, *pr, &sx, &sy);
    cudaError_t e = NSK_TIMED(tr, "fft_z_r2c",
                              fft_z_r2c<T>(in, out, g.nz, (long)ncomp * g.nx * g.ny, qz.zr, (const C *)f.z->tw, s,
                                           pruned ? pr->kz + 1 : -1));
    if (e != cudaSuccess) return e;
    e = NSK_TIMED(tr, "fft_y_forward",
                  fft_strided<T>(out, out, nh, nh, plane, plane, ncomp * g.nx, -1, qy.fwd, (const C *)f.y->tw,
                                 g.ny, qy.ct_fwd, s, pruned ? &sy : nullptr));
    if (e != cudaSuccess) return e;
    return NSK_TIMED(tr, "fft_x_forward",
                     fft_strided<T>(out, out, plane, plane, M, M, ncomp, -1, qx.fwd, (const C *)f.x->tw, g.nx,
                                    qx.ct_fwd, s, pruned ? &sx : nullptr));
}

// The transforms of a run: the resources of its axis lengths with their plans
// (a cubic run), or with the run's own tuned plans (a grid run).
Fft3 run_fft3(const Run &r, FftRes *const f[3]) {
    if (r.g.cube) return Fft3{f[0], f[1], f[2], &f[0]->pp, &f[1]->pp, &f[2]->pp};
    return Fft3{f[0], f[1], f[2], &r.gp[0], &r.gp[1], &r.gp[2]};
}

ns_status fft3_of(ns_ctx *c, const Grid &g, Fft3 *out) {
    FftRes *f[3];
    ns_status st = get_fft3(c, g, f);
    if (st != NS_OK) return st;
    *out = Fft3{f[0], f[1], f[2], &f[0]->pp, &f[1]->pp, &f[2]->pp};
    return NS_OK;
}

// ---------------------------------------------------------------- state transfer

// dst (half layout, precision T) <- src (FP64 half layout) for modes
// [m0, m0 + cnt) of one component, zeroing modes outside Pi.
template <typename T>
__global__ void k_load_half(const double2 *__restrict__ src, typename Cx<T>::type *__restrict__ dst,
                            Grid g, long m0, long cnt, int dealias) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < cnt; i += (long)gridDim.x * blockDim.x) {
        const long m = m0 + i;
        typename Cx<T>::type v;
        if (kept(mode_at(m, g), g, dealias)) {
            v.x = (T)src[i].x;
            v.y = (T)src[i].y;
        } else {
            v.x = 0;
            v.y = 0;
        }
        dst[m] = v;
    }
}

template <typename T>
__global__ void k_store_half(const typename Cx<T>::type *__restrict__ src, double2 *__restrict__ dst,
                             long m0, long cnt) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < cnt; i += (long)gridDim.x * blockDim.x)
        dst[i] = make_double2((double)src[m0 + i].x, (double)src[m0 + i].y);
}

ns_status ensure_staging(ns_ctx *c, size_t bytes) {
    if (c->staging_bytes >= bytes) return NS_OK;
    if (c->staging) dev_free(c->staging);
    c->staging = nullptr;
    c->staging_bytes = 0;
    NS_CK(dalloc(&c->staging, bytes));
    c->staging_bytes = bytes;
    return NS_OK;
}

const size_t kStageChunk = 64u << 20;   // bytes of FP64 complex per host transfer

template <typename T>
ns_status plain_set_state(ns_ctx *c, Run &r, const double2 *src, int on_device, int field = 0) {
    typedef typename Cx<T>::type C;
    C *dst = (C *)r.un + (long)field * 3 * r.M;
    const long total = 3 * r.M;
    const long chunk = on_device ? total : (long)(kStageChunk / sizeof(double2));
    if (!on_device) {
        ns_status st = ensure_staging(c, (size_t)std::min(total, chunk) * sizeof(double2));
        if (st != NS_OK) return st;
    }
    for (long m0 = 0; m0 < total; m0 += chunk) {
        const long cnt = std::min(chunk, total - m0);
        const double2 *s = src + m0;
        if (!on_device) {
            NS_CK(cudaMemcpyAsync(c->staging, src + m0, cnt * sizeof(double2),
                                  cudaMemcpyHostToDevice, c->stream));
            s = (const double2 *)c->staging;
        }
        // component boundaries: mode index within the component
        long done = 0;
        while (done < cnt) {
            const long g = m0 + done;
            const int comp = (int)(g / r.M);
            const long mm = g % r.M;
            const long seg = std::min(cnt - done, r.M - mm);
            k_load_half<T><<<(unsigned)std::min<long>((seg + 255) / 256, 152 * 16), 256, 0, c->stream>>>(
                s + done, dst + (long)comp * r.M, r.g, mm, seg, r.p.dealias);
            NS_CK(cudaGetLastError());
            done += seg;
        }
        if (!on_device) NS_CK(cudaStreamSynchronize(c->stream));
    }
    return NS_OK;
}

template <typename T>
ns_status plain_get_state(ns_ctx *c, Run &r, double2 *dst, int on_device, int field = 0) {
    typedef typename Cx<T>::type C;
    const C *src = (const C *)r.un + (long)field * 3 * r.M;
    const long total = 3 * r.M;
    const long chunk = on_device ? total : (long)(kStageChunk / sizeof(double2));
    if (!on_device) {
        ns_status st = ensure_staging(c, (size_t)std::min(total, chunk) * sizeof(double2));
        if (st != NS_OK) return st;
    }
    for (long m0 = 0; m0 < total; m0 += chunk) {
        const long cnt = std::min(chunk, total - m0);
        double2 *d = on_device ? dst + m0 : (double2 *)c->staging;
        k_store_half<T><<<(unsigned)std::min<long>((cnt + 255) / 256, 152 * 16), 256, 0, c->stream>>>(
            src, d, m0, cnt);
        NS_CK(cudaGetLastError());
        if (!on_device) {
            NS_CK(cudaMemcpyAsync(dst + m0, c->staging, cnt * sizeof(double2), cudaMemcpyDeviceToHost,
                                  c->stream));
            NS_CK(cudaStreamSynchronize(c->stream));
        }
    }
    return NS_OK;
}

// ---------------------------------------------------------------- plain step

// Time `launch` after one warm-up: ms per launch over three, or -1.
template <class F> static float plain_time(F launch, cudaStream_t s) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.f;
    }
    float ms = -1.f;
    if (launch() == cudaSuccess && cudaEventRecord(a, s) == cudaSuccess) {
        bool ok = true;
        for (int i = 0; i < 3 && ok; i++) ok = launch() == cudaSuccess;
        if (ok && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
            ms /= 3;
        else
            ms = -1.f;
    }
    cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

// Plain-form autotuner: for the x/y inverse and forward passes and the z c2r
// and r2c passes, every radix split with at most four stages (and, for x/y,
// 2 to 32 columns per CTA within the kernel's thread bound) runs on the run's
// own buffers; the fastest is kept per (N, precision) for the life of the
// process.  Where nothing runs, the defaults stay.
// Plain-form plan cache file (environment variable NS_PLAIN_CACHE): one line
// per (N, bytes of the real type): "N bytes E_inv ct_inv E_fwd ct_fwd E_zc2r
// E_zr2c".  Entries found there are used as they are; newly tuned ones are
// written back, so that profiled runs execute the same kernels as plain ones.
static void plain_cache_read(std::map<std::pair<int, int>, PlainPlans> &cache) {
    const char *path = getenv("NS_PLAIN_CACHE");
    FILE *fp = path ? fopen(path, "r") : nullptr;
    if (!fp) return;
    int n, b, ei, ci, ef, cf, ec, er;
    while (fscanf(fp, "%d %d %d %d %d %d %d %d", &n, &b, &ei, &ci, &ef, &cf, &ec, &er) == 8) {
        PlainPlans q;
        // z plans: E, or E + 100 for a plan of length n (two lines per transform)
        auto zplan = [&](int code, Plan *pl) {
            return code >= 100 ? make_plan_e(n, code - 100, pl) : make_plan_e(n / 2, code, pl);
        };
        if (make_plan_e(n, ei, &q.inv) && make_plan_e(n, ef, &q.fwd) && zplan(ec, &q.zc) &&
            zplan(er, &q.zr) && ci > 0 && cf > 0) {
            q.ct_inv = ci;
            q.ct_fwd = cf;
            q.tuned = true;
            cache[std::make_pair(n, b)] = q;
        }
    }
    fclose(fp);
}

static void plain_cache_write(const std::map<std::pair<int, int>, PlainPlans> &cache) {
    const char *path = getenv("NS_PLAIN_CACHE");
    FILE *fp = path ? fopen(path, "w") : nullptr;
    if (!fp) return;
    for (const auto &kv : cache) {
        const PlainPlans &q = kv.second;
        const int n = kv.first.first;
        fprintf(fp, "%d %d %d %d %d %d %d %d\n", n, kv.first.second, q.inv.E, q.ct_inv, q.fwd.E, q.ct_fwd,
                q.zc.E + (q.zc.n == n ? 100 : 0), q.zr.E + (q.zr.n == n ? 100 : 0));
    }
    fclose(fp);
}

// Diagnostic restriction of the plain form's z-pass candidates,
// NS_PLAIN_Z=1 (one line per transform) or 2 (two lines per transform); with
// it set, tuning bypasses the plan caches.
static int plain_z_mode() {
    const char *v = getenv("NS_PLAIN_Z");
    return v && (v[0] == '1' || v[0] == '2') ? v[0] - '0' : 0;
}

template <typename T> ns_status tune_plain(ns_ctx *c, Run &r, FftRes *f) {
    typedef typename Cx<T>::type C;
    static std::mutex mu;
    static std::map<std::pair<int, int>, PlainPlans> cache;
    static bool loaded = false;
    const std::pair<int, int> key(r.n, (int)sizeof(T));
    const int zmode = plain_z_mode();
    if (!zmode) {
        std::lock_guard<std::mutex> g(mu);
        if (!loaded) {
            plain_cache_read(cache);
            loaded = true;
        }
        auto it = cache.find(key);
        if (it != cache.end()) {
            f->pp = it->second;
            return NS_OK;
        }
    }
    if (f->pp.tuned && !zmode) return NS_OK;
    const int n = r.n;
    const long nh = n / 2 + 1, plane = (long)n * nh, M = (long)n * plane, lines = 3L * n * n;
    const C *tw = (const C *)f->tw;
    cudaStream_t s = c->stream;
    C *in = (C *)r.un, *tmp = (C *)r.work, *half = (C *)r.wn;
    T *phys = (T *)r.phys;
    const int bound = sizeof(T) == 8 ? 384 : 512;
    PlainPlans best = f->pp;
    float bi = -1.f, bf = -1.f, bc = -1.f, br = -1.f;
    const int Es[] = {16, 12, 9, 8, 6, 4};
    for (int E : Es) {
        Plan pl;
        if (make_plan_e(n, E, &pl) && pl.nst <= 4) {
            const int Tn = n / E;
            for (int ct = 2; ct <= 32; ct *= 2) {
                if (ct * Tn > bound || ct * Tn < 32) continue;
                const float ti = plain_time([&]() {
                    return fft_strided<T>(in, tmp, plane, plane, M, M, 3, +1, pl, tw, n, ct, s);
                }, s);
                if (ti > 0.f && (bi < 0.f || ti < bi)) { bi = ti; best.inv = pl; best.ct_inv = ct; }
                const float tf = plain_time([&]() {
                    return fft_strided<T>(half, half, plane, plane, M, M, 3, -1, pl, tw, n, ct, s);
                }, s);
                if (tf > 0.f && (bf < 0.f || tf < bf)) { bf = tf; best.fwd = pl; best.ct_fwd = ct; }
            }
        }
        // z passes: one line per transform of length n/2 (even/odd packing), or
        // two lines per transform of length n
        for (int len : {n / 2, n}) {
            Plan ph;
            if ((zmode == 1 && len == n) || (zmode == 2 && len != n)) continue;
            if (!make_plan_e(len, E, &ph) || ph.nst > 4) continue;
            const float tc = plain_time([&]() { return fft_z_c2r<T>(tmp, phys, n, lines, ph, tw, s); }, s);
            if (tc > 0.f && (bc < 0.f || tc < bc)) { bc = tc; best.zc = ph; }
            const float tr = plain_time([&]() { return fft_z_r2c<T>(phys, half, n, lines, ph, tw, s); }, s);
            if (tr > 0.f && (br < 0.f || tr < br)) { br = tr; best.zr = ph; }
        }
    }
    NS_CK(cudaStreamSynchronize(s));
    best.tuned = true;
    f->pp = best;
    if (zmode) return NS_OK;
    std::lock_guard<std::mutex> g(mu);
    cache[key] = best;
    plain_cache_write(cache);
    return NS_OK;
}

// Grid runs: the same search per axis on the run's own geometry (the x, y
// and z passes of its grid), into the run's own plans, so that a run's
// transforms do not depend on the other runs of its context.  Kept per
// (grid, precision) for the life of the process; the cubic runs' plan cache
// is neither read nor written.
template <typename T> ns_status tune_plain_grid(ns_ctx *c, Run &r, FftRes *f[3]) {
    typedef typename Cx<T>::type C;
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int>, std::vector<PlainPlans>> cache;
    const Grid &g = r.g;
    const auto key = std::make_tuple(g.nx, g.ny, g.nz, (int)sizeof(T));
    const int zmode = plain_z_mode();
    if (!zmode) {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            for (int a = 0; a < 3; a++) r.gp[a] = it->second[a];
            return NS_OK;
        }
    }
    const long nh = g.nzh(), plane = (long)g.ny * nh, M = (long)g.nx * plane, lines = 3L * g.nx * g.ny;
    cudaStream_t s = c->stream;
    C *in = (C *)r.un, *tmp = (C *)r.work, *half = (C *)r.wn;
    T *phys = (T *)r.phys;
    const int bound = sizeof(T) == 8 ? 384 : 512;
    const int Es[] = {16, 12, 9, 8, 6, 4};
    for (int a = 0; a < 3; a++) r.gp[a] = f[a]->pp;
    for (int a = 0; a < 2; a++) {   // x pass, y pass
        const int n = a == 0 ? g.nx : g.ny;
        const C *tw = (const C *)f[a]->tw;
        auto pass = [&](const C *src, C *dst, int dir, const Plan &pl, int ct) {
            return a == 0 ? fft_strided<T>(src, dst, plane, plane, M, M, 3, dir, pl, tw, n, ct, s)
                          : fft_strided<T>(src, dst, nh, nh, plane, plane, 3 * g.nx, dir, pl, tw, n, ct, s);
        };
        PlainPlans &best = r.gp[a];
        float bi = -1.f, bf = -1.f;
        for (int E : Es) {
            Plan pl;
            if (!make_plan_e(n, E, &pl) || pl.nst > 4) continue;
            const int Tn = n / E;
            for (int ct = 2; ct <= 32; ct *= 2) {
                if (ct * Tn > bound || ct * Tn < 32) continue;
                const float ti = plain_time([&]() { return pass(a == 0 ? in : tmp, tmp, +1, pl, ct); }, s);
                if (ti > 0.f && (bi < 0.f || ti < bi)) { bi = ti; best.inv = pl; best.ct_inv = ct; }
                const float tf = plain_time([&]() { return pass(half, half, -1, pl, ct); }, s);
                if (tf > 0.f && (bf < 0.f || tf < bf)) { bf = tf; best.fwd = pl; best.ct_fwd = ct; }
            }
        }
    }
    {   // z passes
        const C *tw = (const C *)f[2]->tw;
        PlainPlans &best = r.gp[2];
        float bc = -1.f, br = -1.f;
        for (int E : Es)
            for (int len : {g.nz / 2, g.nz}) {
                Plan ph;
                if ((zmode == 1 && len == g.nz) || (zmode == 2 && len != g.nz)) continue;
                if (!make_plan_e(len, E, &ph) || ph.nst > 4) continue;
                const float tc = plain_time([&]() { return fft_z_c2r<T>(tmp, phys, g.nz, lines, ph, tw, s); }, s);
                if (tc > 0.f && (bc < 0.f || tc < bc)) { bc = tc; best.zc = ph; }
                const float tr = plain_time([&]() { return fft_z_r2c<T>(phys, half, g.nz, lines, ph, tw, s); }, s);
                if (tr > 0.f && (br < 0.f || tr < br)) { br = tr; best.zr = ph; }
            }
    }
    NS_CK(cudaStreamSynchronize(s));
    for (int a = 0; a < 3; a++) r.gp[a].tuned = true;
    if (zmode) return NS_OK;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = std::vector<PlainPlans>(r.gp, r.gp + 3);
    return NS_OK;
}

// Largest |m| along one axis that the dealiasing rule keeps.  The rule only
// loosens as any |m_i| shrinks, so no kept mode reaches beyond it.
static int axis_keep(const Grid &g, int axis, int dealias) {
    const int n = axis == 0 ? g.nx : axis == 1 ? g.ny : g.nz;
    int K = -1;
    for (int m = 0; 2 * m <= n; m++) {
        const Idx q{axis == 0 ? m : 0, axis == 1 ? m : 0, axis == 2 ? m : 0};
        if (kept(q, g, dealias)) K = m;
    }
    return K;
}

// NS_PLAIN_PRUNE=0 makes the plain form transform every line (the results
// inside Pi are the same bit for bit).
static bool plain_prune_enabled() {
    const char *v = getenv("NS_PLAIN_PRUNE");
    return !(v && v[0] == '0');
}

template <typename T> ns_status plain_alloc(ns_ctx *c, Run &r) {
    typedef typename Cx<T>::type C;
    r.prune.kx = axis_keep(r.g, 0, r.p.dealias);
    r.prune.ky = axis_keep(r.g, 1, r.p.dealias);
    r.prune.kz = axis_keep(r.g, 2, r.p.dealias);
    r.prune.on = plain_prune_enabled() && r.prune.kx >= 0 && r.prune.ky >= 0 && r.prune.kz >= 0;
    const size_t half = (size_t)r.M * sizeof(C), real = (size_t)r.V * sizeof(T);
    const int nc = r.p.mhd ? 6 : 3;   // state components: u, or u and b
    NS_CK(dalloc(&r.un, nc * half));
    NS_CK(dalloc(&r.u1, nc * half));
    NS_CK(dalloc(&r.wn, nc * half));
    NS_CK(dalloc(&r.work, 3 * half));
    NS_CK(dalloc(&r.phys, 2 * nc * real));
    if (r.p.dealias == 2) {
        NS_CK(dalloc(&r.sh, 3 * half));
        NS_CK(dalloc(&r.sh2, 3 * half));
    }
    NS_CK(cudaMemsetAsync(r.un, 0, nc * half, c->stream));
    NS_CK(cudaMemsetAsync(r.u1, 0, nc * half, c->stream));
    NS_CK(cudaMemsetAsync(r.wn, 0, nc * half, c->stream));   // modes a pruned curl never writes
    // factor tables, computed in FP64 and rounded once: by integer |k|^2 on a
    // unit box; elsewhere per axis by array position [N_x | N_y | N_z/2+1]
    auto factors = [&](double c, std::vector<T> &h) {
        if (r.g.unit) {
            h.resize(grid_max_k2(r.g) + 1);
            for (size_t k2 = 0; k2 < h.size(); k2++) h[k2] = (T)exp(-c * (double)k2 * r.p.dt);
            return;
        }
        const int n[3] = {r.g.nx, r.g.ny, r.g.nz};
        const double l[3] = {r.g.lx, r.g.ly, r.g.lz};
        h.clear();
        for (int a = 0; a < 3; a++) {
            const int cnt = a < 2 ? n[a] : n[a] / 2 + 1;
            for (int i = 0; i < cnt; i++) {
                const int m = a < 2 && 2 * i >= n[a] ? i - n[a] : i;
                const double k = (double)m / l[a];
                h.push_back((T)exp(-c * k * k * r.p.dt));
            }
        }
    };
    std::vector<T> h;
    factors(r.p.nu, h);
    NS_CK(dalloc(&r.etab, h.size() * sizeof(T)));
    NS_CK(cudaMemcpy(r.etab, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    if (r.p.mhd) {
        factors(r.p.eta, h);
        NS_CK(dalloc(&r.etab_b, h.size() * sizeof(T)));
        NS_CK(cudaMemcpy(r.etab_b, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    }
    if (r.p.dealias == 2) {   // per-axis shift factors exp(i pi m / N_i), FP64 rounded once
        const int n[3] = {r.g.nx, r.g.ny, r.g.nz};
        std::vector<C> ph;
        for (int a = 0; a < 3; a++) {
            const int cnt = a < 2 ? n[a] : n[a] / 2 + 1;
            for (int i = 0; i < cnt; i++) {
                const int m = a < 2 && 2 * i >= n[a] ? i - n[a] : i;
                const double t = M_PI * (double)m / (double)n[a];
                C v;
                v.x = (T)cos(t);
                v.y = (T)sin(t);
                ph.push_back(v);
            }
        }
        NS_CK(dalloc(&r.phtab, ph.size() * sizeof(C)));
        NS_CK(cudaMemcpy(r.phtab, ph.data(), ph.size() * sizeof(C), cudaMemcpyHostToDevice));
    }
    FftRes *f[3];
    ns_status st = get_fft3(c, r.g, f);
    if (st != NS_OK) return st;
    if ((st = r.g.cube ? tune_plain<T>(c, r, f[0]) : tune_plain_grid<T>(c, r, f)) != NS_OK) return st;
    if constexpr (std::is_same<T, float>::value) {
        // choose the standalone kernels' shapes now, outside any graph capture
        // (on the run's own buffers, whose contents the first step overwrites)
        const Fft3 f3 = run_fft3(r, f);
        NS_CK(r2c_batch<T>((const T *)r.phys, (C *)r.wn, r.g, 3, f3, c->stream));
        NS_CK(c2r_batch<T>((const C *)r.wn, (C *)r.work, (T *)r.phys, r.g, 3, f3, c->stream));
        NS_CK(cudaStreamSynchronize(c->stream));
    }
    return NS_OK;
}

// Update arguments of a stage: forcing index kf l_i along every axis.
UpdateArgs update_args(const Run &r, int stage) {
    UpdateArgs ua{};
    ua.stage = stage;
    ua.dt = r.p.dt;
    ua.force_amp = r.p.force_amp;
    ua.force_k = r.p.force_k;
    ua.mfx = (int)lround(r.p.force_k * r.g.lx);
    ua.mfy = (int)lround(r.p.force_k * r.g.ly);
    ua.mfz = (int)lround(r.p.force_k * r.g.lz);
    ua.dealias = r.p.dealias;
    ua.rot = r.p.rot;
    return ua;
}

template <typename T> ns_status plain_step(ns_ctx *c, Run &r, cudaStream_t s, Tracer *tr) {
    typedef typename Cx<T>::type C;
    FftRes *fr[3];
    ns_status st = get_fft3(c, r.g, fr);
    if (st != NS_OK) return st;
    const Fft3 f = run_fft3(r, fr);
    const Grid &g = r.g;
    T *phys = (T *)r.phys;
    const long M3 = 3 * r.M, V3 = 3 * r.V;
    // the pointwise kernels may skip the modes outside the kept rectangle only
    // where every transform that reads their output is pruned: the FP64 path
    // (FP32 transforms of compiled lengths read every mode)
    const Rect rc{r.prune.on && std::is_same<T, double>::value ? 1 : 0, r.prune.kx, r.prune.ky, r.prune.kz};
    for (int stage = 1; stage <= 2 && r.p.mhd; stage++) {
        // MHD (Alfven units): [u; b] -> w = curl u, j = curl b -> u, w, b, j on the
        // grid -> u x w + j x b, u x b -> their transforms -> the two updates
        C *src = (C *)(stage == 1 ? r.un : r.u1);
        C *wj = (C *)r.wn;
        NS_CK(NSK_TIMED(tr, "curl", plain_curl<T>(src, wj, g, rc, s)));
        NS_CK(NSK_TIMED(tr, "curl", plain_curl<T>(src + M3, wj + M3, g, rc, s)));
        NS_CK(c2r_batch<T>(src, (C *)r.work, phys, g, 3, f, s, tr, &r.prune));
        NS_CK(c2r_batch<T>(wj, (C *)r.work, phys + V3, g, 3, f, s, tr, &r.prune));
        NS_CK(c2r_batch<T>(src + M3, (C *)r.work, phys + 2 * V3, g, 3, f, s, tr, &r.prune));
        NS_CK(c2r_batch<T>(wj + M3, (C *)r.work, phys + 3 * V3, g, 3, f, s, tr, &r.prune));
        NS_CK(NSK_TIMED(tr, "cross_mhd", plain_cross_mhd<T>(phys, g, s)));
        NS_CK(r2c_batch<T>(phys, wj, g, 3, f, s, tr, &r.prune));
        NS_CK(r2c_batch<T>(phys + V3, wj + M3, g, 3, f, s, tr, &r.prune));
        const UpdateArgs ua = update_args(r, stage);
        NS_CK(NSK_TIMED(tr, "update",
                        plain_update<T>((C *)r.un, (C *)r.u1, (const C *)wj, (const T *)r.etab, g, ua, rc, s)));
        NS_CK(NSK_TIMED(tr, "update_b",
                        plain_update_b<T>((C *)r.un + M3, (C *)r.u1 + M3, (const C *)wj + M3,
                                          (const T *)r.etab_b, g, stage, r.p.dt,
                                          r.p.dealias, rc, s)));
    }
    for (int stage = 1; stage <= 2 && !r.p.mhd; stage++) {
        C *src = (C *)(stage == 1 ? r.un : r.u1);
        NS_CK(NSK_TIMED(tr, "curl", plain_curl<T>(src, (C *)r.wn, g, rc, s)));
        NS_CK(c2r_batch<T>(src, (C *)r.work, phys, g, 3, f, s, tr, &r.prune));
        NS_CK(c2r_batch<T>((C *)r.wn, (C *)r.work, phys + 3 * r.V, g, 3, f, s, tr, &r.prune));
        NS_CK(NSK_TIMED(tr, "cross", plain_cross<T>(phys, phys + 3 * r.V, g, s)));
        NS_CK(r2c_batch<T>(phys, (C *)r.wn, g, 3, f, s, tr, &r.prune));
        if (r.p.dealias == 2) {   // the same on the grid shifted by half a spacing, averaged
            C *sh = (C *)r.sh, *sh2 = (C *)r.sh2;
            NS_CK(NSK_TIMED(tr, "phase", plain_phase<T>(src, sh, (const C *)r.phtab, g, s)));
            NS_CK(NSK_TIMED(tr, "curl", plain_curl<T>(sh, sh2, g, rc, s)));
            NS_CK(c2r_batch<T>(sh, (C *)r.work, phys, g, 3, f, s, tr, &r.prune));
            NS_CK(c2r_batch<T>(sh2, (C *)r.work, phys + 3 * r.V, g, 3, f, s, tr, &r.prune));
            NS_CK(NSK_TIMED(tr, "cross", plain_cross<T>(phys, phys + 3 * r.V, g, s)));
            NS_CK(r2c_batch<T>(phys, sh2, g, 3, f, s, tr, &r.prune));
            NS_CK(NSK_TIMED(tr, "phase", plain_phase_avg<T>((C *)r.wn, sh2, (const C *)r.phtab, g, s)));
        }
        const UpdateArgs ua = update_args(r, stage);
        NS_CK(NSK_TIMED(tr, "update",
                        plain_update<T>((C *)r.un, (C *)r.u1, (const C *)r.wn, (const T *)r.etab, g, ua, rc, s)));
    }
    NS_CK(NSK_TIMED(tr, "energy_partials", plain_energy_partials<T>((const C *)r.un, g, r.part, rc, s)));
    NS_CK(NSK_TIMED(tr, "energy_final",
                    energy_final(r.part, r.nparts, r.series, kSeriesCap, r.counter, c->flags, s)));
    return NS_OK;
}

bool use_fused(const ns_ctx *c) { return c->prec == NS_FP32 && fused_enabled() && !c->plain_only; }

// One RK2 step of every run of the context: one batched sequence of launches
// per group of the fused form, or the plain sequence per run.
ns_status step_all(ns_ctx *c, cudaStream_t s, Tracer *tr) {
    if (use_fused(c)) {
        for (FusedRun &g : c->groups) {
            cudaError_t e = fused_step(g, c->flags, s, tr);
            if (e != cudaSuccess) return fail_cuda(c, e);
        }
        return NS_OK;
    }
    for (Run &r : c->runs) {
        ns_status st = c->prec == NS_FP64 ? plain_step<double>(c, r, s, tr) : plain_step<float>(c, r, s, tr);
        if (st != NS_OK) return st;
    }
    return NS_OK;
}

// The step with its independent units (fused groups, or plain runs) on the
// streams of c->par, forked from c->cap and joined back to it: captured, the
// units become parallel branches of the graph.  Unit u goes to stream
// u % par.size() (units on one stream stay in order).
ns_status step_all_forked(ns_ctx *c) {
    const int P = (int)c->par.size();
    NS_CK(cudaEventRecord(c->fork_join[0], c->cap));
    for (int q = 0; q < P; q++) NS_CK(cudaStreamWaitEvent(c->par[q], c->fork_join[0], 0));
    if (use_fused(c)) {
        for (size_t g = 0; g < c->groups.size(); g++) {
            cudaError_t e = fused_step(c->groups[g], c->flags, c->par[g % P], nullptr);
            if (e != cudaSuccess) return fail_cuda(c, e);
        }
    } else {
        for (size_t i = 0; i < c->runs.size(); i++) {
            Run &r = c->runs[i];
            cudaStream_t q = c->par[i % P];
            ns_status st = c->prec == NS_FP64 ? plain_step<double>(c, r, q, nullptr)
                                              : plain_step<float>(c, r, q, nullptr);
            if (st != NS_OK) return st;
        }
    }
    for (int q = 0; q < P; q++) {
        NS_CK(cudaEventRecord(c->fork_join[1 + q], c->par[q]));
        NS_CK(cudaStreamWaitEvent(c->cap, c->fork_join[1 + q], 0));
    }
    return NS_OK;
}

ns_status build_graph(ns_ctx *c) {
    if (c->graph) return NS_OK;
    // Resources the step needs must exist before capture (no allocation inside).
    for (Run &r : c->runs) {
        FftRes *f[3];
        ns_status st = get_fft3(c, r.g, f);
        if (st != NS_OK) return st;
    }
    NS_CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    ns_status st = c->par.empty() ? step_all(c, c->cap, nullptr) : step_all_forked(c);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap, &g);
    if (st != NS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail_cuda(c, e);
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail_cuda(c, e);
    return NS_OK;
}

void free_run(Run &r) {
    void *ps[] = {r.un, r.u1, r.wn, r.work, r.phys, r.etab, r.etab_b, r.sh, r.sh2, r.phtab};
    for (void *p : ps)
        if (p) dev_free(p);
    if (r.owns_diag) {
        void *qs[] = {r.part, r.series, r.counter};
        for (void *p : qs)
            if (p) dev_free(p);
    }
}

// Entry check: a null context is an argument error; a context that already
// failed stays failed.  A stale error left in the runtime's per-thread slot by
// some earlier, unrelated call is cleared so that the kernel launches of this
// call report only their own failures.
ns_status check_ctx(ns_ctx *c) {
    if (!c) return NS_ERR_ARG;
    if (c->sticky == NS_OK) (void)cudaGetLastError();
    return c->sticky;
}

// Energy spectrum (or, with hel, helicity spectrum) of a fused run on a grid
// or box: the compact state expanded into the full FP32 half layout in the
// group's pass-B buffer (the step is stream-ordered before it), then the
// plain form's shell kernels on the run's grid.
cudaError_t fused_grid_spectrum(ns_ctx *c, const Run &r, int field, int nb, double *spec, double *aux, bool hel) {
    FusedRun &g = c->groups[r.group];
    cudaError_t e = fused_expand(g, r.gidx, field, g.bbuf, c->stream);
    if (e != cudaSuccess) return e;
    return hel ? plain_helicity<float>(g.bbuf, r.g, nb, spec, aux, c->stream)
               : plain_spectrum<float>(g.bbuf, r.g, nb, spec, aux, c->stream);
}

ns_status check_flags(ns_ctx *c) {
    int h = 0;
    NS_CK(cudaMemcpy(&h, c->flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (h & 2) return NS_ERR_TIMEOUT;
    if (h & 1) return NS_ERR_NONFINITE;
    return NS_OK;
}

}  // namespace

// ================================================================ public ABI

extern "C" {

const char *ns_status_str(ns_status s) {
    switch (s) {
    case NS_OK: return "ok";
    case NS_ERR_ARG: return "invalid argument";
    case NS_ERR_CUDA: return "CUDA error";
    case NS_ERR_OOM: return "out of memory";
    case NS_ERR_UNSUPPORTED_N: return "unsupported grid size";
    case NS_ERR_TIMEOUT: return "device wait timed out";
    case NS_ERR_NONFINITE: return "non-finite energy";
    }
    return "unknown status";
}

int ns_nbins(int n) { return n < 1 ? 0 : (int)ceil(sqrt(3.0) * n / 2.0) + 1; }

int ns_series_capacity(void) { return kSeriesCap; }

const char *ns_last_error(ns_ctx *c) { return c ? c->last_error : ""; }

ns_status ns_describe_run(ns_ctx *c, int run, char *out, int len) {
    if (!c || run < 0 || run >= (int)c->runs.size() || !out || len < 1) return NS_ERR_ARG;
    const Run &r = c->runs[run];
    int w;
    if (use_fused(c)) {
        const FusedRun &g = c->groups[r.group];
        char tune[2048];
        if (fused_describe(g, tune, sizeof(tune)) >= (int)sizeof(tune)) return NS_ERR_ARG;
        w = snprintf(out, len,
                 "{\"form\": \"fused FP32\", \"equations\": \"%s\", \"n\": %d, \"grid\": [%d, %d, %d], "
                 "\"box\": [%.17g, %.17g, %.17g], \"K\": %d, \"K_yz\": [%d, %d], "
                 "\"state_modes\": %ld, \"runs_in_group\": %d, \"passes\": %s}",
                 g.mhd ? "MHD" : "Navier-Stokes", r.n, g.n, g.ny, g.nz, r.g.lx, r.g.ly, r.g.lz, g.K, g.Ky, g.Kz,
                 (g.mhd ? 6 : 3) * g.M, g.nr, tune);
    } else {
        // plans of the x pass (and the y pass of a cube) and of the z passes
        const auto it = c->fft.find(r.n);
        const PlainPlans qc = it != c->fft.end() ? it->second.pp : PlainPlans{};
        const PlainPlans &q = r.g.cube ? qc : r.gp[0], &qz = r.g.cube ? qc : r.gp[2];
        w = snprintf(out, len,
                 "{\"form\": \"plain %s\", \"equations\": \"%s\", \"n\": %d, \"grid\": [%d, %d, %d], "
                 "\"box\": [%.17g, %.17g, %.17g], \"tuned\": %s, "
                 "\"xy_inverse\": {\"E\": %d, \"cols_per_cta\": %d}, \"xy_forward\": {\"E\": %d, "
                 "\"cols_per_cta\": %d}, \"z_c2r\": {\"E\": %d, \"lines_per_transform\": %d}, "
                 "\"z_r2c\": {\"E\": %d, \"lines_per_transform\": %d}}",
                 c->prec == NS_FP64 ? "FP64" : "FP32", r.p.mhd ? "MHD" : "Navier-Stokes", r.n, r.g.nx, r.g.ny,
                 r.g.nz, r.g.lx, r.g.ly, r.g.lz, q.tuned ? "true" : "false", q.inv.E, q.ct_inv, q.fwd.E, q.ct_fwd,
                 qz.zc.E, qz.zc.n == r.g.nz ? 2 : 1, qz.zr.E, qz.zr.n == r.g.nz ? 2 : 1);
    }
    return w < len ? NS_OK : NS_ERR_ARG;   // the text did not fit in len bytes
}

ns_status ns_init(const ns_run_params *runs, int nruns, ns_prec prec, void *cuda_stream,
                  ns_ctx **out) {
    if (!out) return NS_ERR_ARG;
    *out = nullptr;
    if (!runs || nruns < 1 || (prec != NS_FP64 && prec != NS_FP32)) return NS_ERR_ARG;
    for (int i = 0; i < nruns; i++) {
        const ns_run_params &p = runs[i];
        if (!(p.nu >= 0.0) || !(p.dt > 0.0) || p.dealias < 0 || p.dealias > 2 ||
            p.force_k < 0 || !isfinite(p.force_amp) || !isfinite(p.nu) || !isfinite(p.dt) ||
            !isfinite(p.rot) || (p.mhd != 0 && p.mhd != 1) || !(p.eta >= 0.0) || !isfinite(p.eta) ||
            (p.dealias == 2 && p.mhd) || p.ny < 0 || p.nz < 0)
            return NS_ERR_ARG;
        const double l[3] = {p.lx, p.ly, p.lz};
        for (double li : l)
            if (!(li >= 0.0) || !(li <= 1e6)) return NS_ERR_ARG;
        const Grid g = run_grid(p);
        if (p.force_k > 0 && p.force_amp != 0.0) {   // the ABC field must be periodic on the box
            const double lg[3] = {g.lx, g.ly, g.lz};
            for (double li : lg) {
                const double t = p.force_k * li;
                if (fabs(t - nearbyint(t)) > 1e-9 * t) return NS_ERR_ARG;
            }
        }
        const int cap = 1024;
        const int ns[3] = {g.nx, g.ny, g.nz};
        for (int n : ns)
            if (!supported_n(n) || n > cap) return NS_ERR_UNSUPPORTED_N;
        if ((double)g.nx * g.ny * g.nz > (double)cap * cap * cap) return NS_ERR_UNSUPPORTED_N;
    }
    ns_ctx *c = new (std::nothrow) ns_ctx;
    if (!c) return NS_ERR_OOM;
    c->prec = prec;
    c->stream = (cudaStream_t)cuda_stream;
    for (int i = 0; i < nruns; i++)
        if ((runs[i].mhd && !fused_mhd_supported(runs[i].n)) || runs[i].dealias == 2 ||
            !fused_grid_supported(runs[i]))
            c->plain_only = true;
    ns_status st = NS_OK;
    auto bail = [&](ns_status s) {
        ns_destroy(c);
        return s;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(fail_cuda(nullptr, e));
    if ((e = prepare_fft_kernels()) != cudaSuccess) return bail(fail_cuda(nullptr, e));
    if ((e = dalloc(&c->flags, sizeof(int))) != cudaSuccess) return bail(fail_cuda(nullptr, e));
    cudaMemset(c->flags, 0, sizeof(int));
    c->runs.resize(nruns);
    int maxbins = 0;
    for (int i = 0; i < nruns; i++) {
        Run &r = c->runs[i];
        r.p = runs[i];
        r.n = r.p.n;
        r.g = run_grid(r.p);
        r.M = r.g.M();
        r.V = r.g.V();
        r.nparts = energy_nparts(r.M);
        maxbins = std::max(maxbins, grid_nbins(r.g));
        FftRes *f[3];
        if ((st = get_fft3(c, r.g, f)) != NS_OK) return bail(st);
        if (use_fused(c)) continue;   // grouped below
        st = prec == NS_FP64 ? plain_alloc<double>(c, r) : plain_alloc<float>(c, r);
        if (st != NS_OK) return bail(st);
        if ((e = dalloc(&r.part, sizeof(double) * 2 * std::max(r.nparts, 1))) != cudaSuccess ||
            (e = dalloc(&r.series, sizeof(double) * 2 * kSeriesCap)) != cudaSuccess ||
            (e = dalloc(&r.counter, sizeof(unsigned long long))) != cudaSuccess)
            return bail(fail_cuda(nullptr, e));
        cudaMemset(r.counter, 0, sizeof(unsigned long long));
    }
    if (use_fused(c)) {
        // runs of the same grid, box and equations form one group (in order of
        // first appearance); an MHD group carries a magnetic block beside the
        // velocity
        typedef std::tuple<int, int, int, double, double, double, int> GKey;
        std::vector<GKey> order;
        std::map<GKey, std::vector<int>> members;
        for (int i = 0; i < nruns; i++) {
            const Grid &g = c->runs[i].g;
            const GKey key(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, c->runs[i].p.mhd);
            if (!members.count(key)) order.push_back(key);
            members[key].push_back(i);
        }
        c->groups.resize(order.size());
        for (size_t gi = 0; gi < order.size(); gi++) {
            std::vector<ns_run_params> ps;
            for (int i : members[order[gi]]) ps.push_back(c->runs[i].p);
            FftRes *f[3];
            if ((st = get_fft3(c, c->runs[members[order[gi]][0]].g, f)) != NS_OK) return bail(st);
            e = fused_alloc(c->groups[gi], ps, (const float2 *)f[0]->tw, (const float2 *)f[1]->tw,
                            (const float2 *)f[2]->tw, kSeriesCap, c->stream);
            if (e != cudaSuccess) return bail(fail_cuda(nullptr, e));
            const std::vector<int> &mem = members[order[gi]];
            for (size_t j = 0; j < mem.size(); j++) {
                Run &r = c->runs[mem[j]];
                FusedRun &g = c->groups[gi];
                r.group = (int)gi;
                r.gidx = (int)j;
                r.owns_diag = false;
                r.series = g.series + (long)j * g.cap * 2;
                r.counter = g.counter + j;
            }
        }
    }
    // nbins results, then kShellParts partials per shell
    if ((e = dalloc(&c->spec, sizeof(double) * maxbins * (1 + kShellParts))) != cudaSuccess ||
        (e = dalloc(&c->ens, sizeof(double) * maxbins * (1 + kShellParts))) != cudaSuccess)
        return bail(fail_cuda(nullptr, e));
    c->spec_cap = maxbins;
    // streams for concurrent units of the step graph (ensembles)
    const size_t units = use_fused(c) ? c->groups.size() : c->runs.size();
    if (units > 1) {
        const int P = (int)std::min<size_t>(units, 8);
        c->par.resize(P, nullptr);
        c->fork_join.resize(P + 1, nullptr);
        for (int q = 0; q < P; q++)
            if ((e = cudaStreamCreateWithFlags(&c->par[q], cudaStreamNonBlocking)) != cudaSuccess)
                return bail(fail_cuda(nullptr, e));
        for (int q = 0; q <= P; q++)
            if ((e = cudaEventCreateWithFlags(&c->fork_join[q], cudaEventDisableTiming)) != cudaSuccess)
                return bail(fail_cuda(nullptr, e));
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(fail_cuda(nullptr, e));
    *out = c;
    return NS_OK;
}

void ns_destroy(ns_ctx *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (Run &r : c->runs) free_run(r);
    for (FusedRun &g : c->groups) fused_free(g);
    for (auto &kv : c->fft) {
        if (kv.second.tw) dev_free(kv.second.tw);
        if (kv.second.scratch) dev_free(kv.second.scratch);
    }
    if (c->flags) dev_free(c->flags);
    if (c->spec) dev_free(c->spec);
    if (c->ens) dev_free(c->ens);
    if (c->staging) dev_free(c->staging);
    if (c->gscratch) dev_free(c->gscratch);
    if (c->bspec) dev_free(c->bspec);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (cudaStream_t q : c->par) cudaStreamDestroy(q);
    for (cudaEvent_t ev : c->fork_join) cudaEventDestroy(ev);
    delete c;
}

// Device address of a host buffer the GPU can reach directly (page-locked
// memory: cudaHostAlloc'd or registered), 16-byte aligned, else null.  Such
// buffers are read and written by the conversion kernels themselves (over
// NVLink-C2C on Grace-Blackwell), without staging copies; pageable memory
// goes through the staging buffer.
static const void *mapped_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer || ((uintptr_t)a.devicePointer & 15)) return nullptr;
    return a.devicePointer;
}

ns_status ns_set_field(ns_ctx *c, int run, int field, const void *uhat, int on_device) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    if (run < 0 || run >= (int)c->runs.size() || !uhat) return NS_ERR_ARG;
    Run &r = c->runs[run];
    if (field != 0 && !(field == 1 && r.p.mhd)) return NS_ERR_ARG;
    if (!on_device) {
        if (const void *d = mapped_host(uhat)) {   // page-locked: no staging
            if ((st = ns_set_field(c, run, field, d, 1)) != NS_OK) return st;
            NS_CK(cudaStreamSynchronize(c->stream));   // the caller may reuse its buffer
            return NS_OK;
        }
    }
    if (use_fused(c)) {
        if (!on_device) {
            ns_status s2 = ensure_staging(c, kStageChunk);
            if (s2 != NS_OK) return s2;
        }
        cudaError_t e = fused_set_state(c->groups[r.group], r.gidx, field, (const double2 *)uhat, on_device,
                                        c->staging, kStageChunk, c->stream);
        if (e != cudaSuccess) return fail_cuda(c, e);
        return NS_OK;
    }
    return c->prec == NS_FP64 ? plain_set_state<double>(c, r, (const double2 *)uhat, on_device, field)
                              : plain_set_state<float>(c, r, (const double2 *)uhat, on_device, field);
}

ns_status ns_set_state(ns_ctx *c, int run, const void *uhat, int on_device) {
    return ns_set_field(c, run, 0, uhat, on_device);
}

ns_status ns_get_field(ns_ctx *c, int run, int field, void *uhat, int on_device) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    if (run < 0 || run >= (int)c->runs.size() || !uhat) return NS_ERR_ARG;
    Run &r = c->runs[run];
    if (field != 0 && !(field == 1 && r.p.mhd)) return NS_ERR_ARG;
    if (!on_device) {
        if (const void *d = mapped_host(uhat)) return ns_get_field(c, run, field, (void *)d, 1);
    }
    if (use_fused(c)) {
        if (!on_device) {
            ns_status s2 = ensure_staging(c, kStageChunk);
            if (s2 != NS_OK) return s2;
        }
        cudaError_t e = fused_get_state(c->groups[r.group], r.gidx, field, (double2 *)uhat, on_device,
                                        c->staging, kStageChunk, c->stream);
        if (e != cudaSuccess) return fail_cuda(c, e);
    } else {
        st = c->prec == NS_FP64 ? plain_get_state<double>(c, r, (double2 *)uhat, on_device, field)
                                : plain_get_state<float>(c, r, (double2 *)uhat, on_device, field);
        if (st != NS_OK) return st;
    }
    NS_CK(cudaStreamSynchronize(c->stream));
    return check_flags(c);
}

ns_status ns_get_state(ns_ctx *c, int run, void *uhat, int on_device) {
    return ns_get_field(c, run, 0, uhat, on_device);
}

ns_status ns_step(ns_ctx *c, int nsteps) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    if (nsteps < 0) return NS_ERR_ARG;
    if (nsteps == 0) return NS_OK;
    if ((st = build_graph(c)) != NS_OK) return st;
    for (int i = 0; i < nsteps; i++) NS_CK(cudaGraphLaunch(c->graph, c->stream));
    return NS_OK;
}

// Axis lengths of every entry point: those with transform plans, up to 1024
// points (the range the transforms are built, tuned and tested for).
static bool axis_ok(int n) { return n <= 1024 && supported_n(n); }

ns_status ns_fft_r2c(ns_ctx *c, int n, int ncomp, const void *in, void *out) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    if (!in || !out || ncomp < 1 || ncomp > 65535 / (n > 0 ? n : 1)) return NS_ERR_ARG;
    if (!axis_ok(n)) return NS_ERR_UNSUPPORTED_N;
    FftRes *f;
    if ((st = get_fft(c, n, &f)) != NS_OK) return st;
    const Grid g = make_grid(n, n, n, 1.0, 1.0, 1.0);
    const Fft3 f3{f, f, f, &f->pp, &f->pp, &f->pp};
    if (c->prec == NS_FP64) {
        NS_CK(r2c_batch<double>((const double *)in, (double2 *)out, g, ncomp, f3, c->stream));
    } else {
        cudaError_t e = cudaSuccess;
        if (std_r2c_fp32((const float *)in, (float2 *)out, n, ncomp, (const float2 *)f->tw, c->stream, &e))
            NS_CK(e);
        else
            NS_CK(r2c_batch<float>((const float *)in, (float2 *)out, g, ncomp, f3, c->stream));
    }
    return NS_OK;
}

ns_status ns_fft_c2r(ns_ctx *c, int n, int ncomp, const void *in, void *out) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    if (!in || !out || ncomp < 1) return NS_ERR_ARG;
    if (!axis_ok(n)) return NS_ERR_UNSUPPORTED_N;
    FftRes *f;
    if ((st = get_fft(c, n, &f)) != NS_OK) return st;
    if ((st = ensure_scratch(c, f)) != NS_OK) return st;
    const Grid g = make_grid(n, n, n, 1.0, 1.0, 1.0);
    const Fft3 f3{f, f, f, &f->pp, &f->pp, &f->pp};
    const long M = g.M(), V = g.V();
    for (int k = 0; k < ncomp; k++) {
        if (c->prec == NS_FP64)
            NS_CK(c2r_batch<double>((const double2 *)in + k * M, (double2 *)f->scratch,
                                    (double *)out + k * V, g, 1, f3, c->stream));
        else {
            cudaError_t e = cudaSuccess;
            if (std_c2r_fp32((const float2 *)in + k * M, (float2 *)f->scratch, (float *)out + k * V, n,
                             (const float2 *)f->tw, c->stream, &e))
                NS_CK(e);
            else
                NS_CK(c2r_batch<float>((const float2 *)in + k * M, (float2 *)f->scratch,
                                       (float *)out + k * V, g, 1, f3, c->stream));
        }
    }
    return NS_OK;
}

// The transforms of N_x x N_y x N_z grids (the three axes may differ).
static ns_status grid_fft_args(ns_ctx *c, int nx, int ny, int nz, int ncomp, const void *in, void *out,
                               Grid *g, Fft3 *f3) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    if (!in || !out || ncomp < 1 || ncomp > 65535 / (nx > 0 ? nx : 1)) return NS_ERR_ARG;
    if (!axis_ok(nx) || !axis_ok(ny) || !axis_ok(nz)) return NS_ERR_UNSUPPORTED_N;
    *g = make_grid(nx, ny, nz, 1.0, 1.0, 1.0);
    return fft3_of(c, *g, f3);
}

ns_status ns_fft_r2c_grid(ns_ctx *c, int nx, int ny, int nz, int ncomp, const void *in, void *out) {
    Grid g;
    Fft3 f3;
    ns_status st = grid_fft_args(c, nx, ny, nz, ncomp, in, out, &g, &f3);
    if (st != NS_OK) return st;
    if (c->prec == NS_FP64) {
        NS_CK(r2c_batch<double>((const double *)in, (double2 *)out, g, ncomp, f3, c->stream));
    } else {
        const StdGrid sg{nx, ny, nz, (const float2 *)f3.x->tw, (const float2 *)f3.y->tw,
                         (const float2 *)f3.z->tw};
        cudaError_t e = cudaSuccess;
        if (std_r2c_fp32_grid((const float *)in, (float2 *)out, sg, ncomp, c->stream, &e))
            NS_CK(e);
        else
            NS_CK(r2c_batch<float>((const float *)in, (float2 *)out, g, ncomp, f3, c->stream));
    }
    return NS_OK;
}

ns_status ns_fft_c2r_grid(ns_ctx *c, int nx, int ny, int nz, int ncomp, const void *in, void *out) {
    Grid g;
    Fft3 f3;
    ns_status st = grid_fft_args(c, nx, ny, nz, ncomp, in, out, &g, &f3);
    if (st != NS_OK) return st;
    const size_t bytes = (size_t)g.M() * 2 * elem_bytes(c->prec);
    if (c->gscratch_bytes < bytes) {
        NS_CK(cudaStreamSynchronize(c->stream));
        if (c->gscratch) dev_free(c->gscratch);
        c->gscratch = nullptr;
        c->gscratch_bytes = 0;
        NS_CK(dalloc(&c->gscratch, bytes));
        c->gscratch_bytes = bytes;
    }
    const long M = g.M(), V = g.V();
    const StdGrid sg{nx, ny, nz, (const float2 *)f3.x->tw, (const float2 *)f3.y->tw, (const float2 *)f3.z->tw};
    for (int k = 0; k < ncomp; k++) {
        if (c->prec == NS_FP64) {
            NS_CK(c2r_batch<double>((const double2 *)in + k * M, (double2 *)c->gscratch, (double *)out + k * V,
                                    g, 1, f3, c->stream));
        } else {
            cudaError_t e = cudaSuccess;
            if (std_c2r_fp32_grid((const float2 *)in + k * M, (float2 *)c->gscratch, (float *)out + k * V, sg,
                                  c->stream, &e))
                NS_CK(e);
            else
                NS_CK(c2r_batch<float>((const float2 *)in + k * M, (float2 *)c->gscratch, (float *)out + k * V,
                                       g, 1, f3, c->stream));
        }
    }
    return NS_OK;
}

int ns_run_nbins(const ns_run_params *p) {
    if (!p || p->n < 2) return 0;
    return grid_nbins(run_grid(*p));
}

ns_status ns_field_spectrum(ns_ctx *c, int run, int field, double *spec, int nbins, double *energy,
                            double *enstrophy) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    if (run < 0 || run >= (int)c->runs.size() || nbins < 0 || (nbins > 0 && !spec))
        return NS_ERR_ARG;
    Run &r = c->runs[run];
    if (field != 0 && !(field == 1 && r.p.mhd)) return NS_ERR_ARG;
    const int nb = grid_nbins(r.g);
    const long off = (long)field * 3 * r.M;
    if (use_fused(c) && c->groups[r.group].cube)
        NS_CK(fused_spectrum(c->groups[r.group], r.gidx, field, nb, c->spec, c->ens, c->stream));
    else if (use_fused(c))   // a grid or box: the shells of the plain form on the expanded state
        NS_CK(fused_grid_spectrum(c, r, field, nb, c->spec, c->ens, false));
    else if (c->prec == NS_FP64)
        NS_CK(plain_spectrum<double>((const double2 *)r.un + off, r.g, nb, c->spec, c->ens, c->stream));
    else
        NS_CK(plain_spectrum<float>((const float2 *)r.un + off, r.g, nb, c->spec, c->ens, c->stream));
    std::vector<double> hs(nb), he(nb);
    NS_CK(cudaMemcpyAsync(hs.data(), c->spec, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    NS_CK(cudaMemcpyAsync(he.data(), c->ens, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    NS_CK(cudaStreamSynchronize(c->stream));
    double e = 0.0, om = 0.0;
    for (int k = 0; k < nb; k++) {
        e += hs[k];
        om += he[k];
    }
    for (int k = 0; k < nbins && k < nb; k++) spec[k] = hs[k];
    if (energy) *energy = e;
    if (enstrophy) *enstrophy = om;
    if (!isfinite(e)) return NS_ERR_NONFINITE;
    return check_flags(c);
}

ns_status ns_energy_spectrum(ns_ctx *c, int run, double *spec, int nbins, double *energy,
                             double *enstrophy) {
    return ns_field_spectrum(c, run, 0, spec, nbins, energy, enstrophy);
}

ns_status ns_energy_spectra(ns_ctx *c, int first, int count, double *spec, int nbins, double *energy,
                            double *enstrophy) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    if (first < 0 || count < 1 || first + count > (int)c->runs.size() || nbins < 0 || (nbins > 0 && !spec))
        return NS_ERR_ARG;
    // one device slice per run: spec_cap results then partials, for spec and ens
    const size_t slice = (size_t)c->spec_cap * (1 + kShellParts);
    if (c->bspec_runs < (size_t)count) {
        NS_CK(cudaStreamSynchronize(c->stream));
        if (c->bspec) dev_free(c->bspec);
        c->bspec = nullptr;
        c->bspec_runs = 0;
        NS_CK(dalloc(&c->bspec, sizeof(double) * 2 * slice * count));
        c->bspec_runs = count;
    }
    for (int i = 0; i < count; i++) {
        Run &r = c->runs[first + i];
        const int nb = grid_nbins(r.g);
        double *sp = c->bspec + 2 * slice * i, *en = sp + slice;
        if (use_fused(c) && c->groups[r.group].cube)
            NS_CK(fused_spectrum(c->groups[r.group], r.gidx, 0, nb, sp, en, c->stream));
        else if (use_fused(c))
            NS_CK(fused_grid_spectrum(c, r, 0, nb, sp, en, false));
        else if (c->prec == NS_FP64)
            NS_CK(plain_spectrum<double>((const double2 *)r.un, r.g, nb, sp, en, c->stream));
        else
            NS_CK(plain_spectrum<float>((const float2 *)r.un, r.g, nb, sp, en, c->stream));
    }
    // the results of every run (spec, then ens, of each slice) in one copy
    std::vector<double> h((size_t)2 * count * c->spec_cap);
    NS_CK(cudaMemcpy2DAsync(h.data(), sizeof(double) * c->spec_cap, c->bspec, sizeof(double) * slice,
                            sizeof(double) * c->spec_cap, (size_t)2 * count, cudaMemcpyDeviceToHost,
                            c->stream));
    NS_CK(cudaStreamSynchronize(c->stream));
    bool finite = true;
    for (int i = 0; i < count; i++) {
        const int nb = grid_nbins(c->runs[first + i].g);
        const double *hs = h.data() + (size_t)2 * i * c->spec_cap, *he = hs + c->spec_cap;
        double e = 0.0, om = 0.0;
        for (int k = 0; k < nb; k++) {
            e += hs[k];
            om += he[k];
        }
        for (int k = 0; k < nbins; k++) spec[(size_t)i * nbins + k] = k < nb ? hs[k] : 0.0;
        if (energy) energy[i] = e;
        if (enstrophy) enstrophy[i] = om;
        finite = finite && isfinite(e);
    }
    if (!finite) return NS_ERR_NONFINITE;
    return check_flags(c);
}

ns_status ns_set_states(ns_ctx *c, int first, int count, const void *const *uhats, int on_device) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    if (first < 0 || count < 1 || first + count > (int)c->runs.size() || !uhats) return NS_ERR_ARG;
    for (int i = 0; i < count; i++)
        if (!uhats[i]) return NS_ERR_ARG;
    bool mapped = false;
    for (int i = 0; i < count; i++) {
        const void *p = uhats[i];
        int dev = on_device;
        if (!on_device) {
            if (const void *d = mapped_host(p)) {   // page-locked: read by the kernels, no staging
                p = d;
                dev = 1;
                mapped = true;
            }
        }
        if ((st = ns_set_field(c, first + i, 0, p, dev)) != NS_OK) break;
    }
    // the caller may reuse (or free) its buffers when the call returns, on
    // an error too: wait for the kernels that read the page-locked ones
    if (mapped) {
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        if (st == NS_OK && e != cudaSuccess) return fail_cuda(c, e);
    }
    return st;
}

ns_status ns_helicity(ns_ctx *c, int run, double *spec, int nbins, double *helicity) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    if (run < 0 || run >= (int)c->runs.size() || nbins < 0 || (nbins > 0 && !spec))
        return NS_ERR_ARG;
    Run &r = c->runs[run];
    const int nb = grid_nbins(r.g);
    if (use_fused(c) && c->groups[r.group].cube)
        NS_CK(fused_helicity(c->groups[r.group], r.gidx, nb, c->spec, c->ens, c->stream));
    else if (use_fused(c))
        NS_CK(fused_grid_spectrum(c, r, 0, nb, c->spec, c->ens, true));
    else if (c->prec == NS_FP64)
        NS_CK(plain_helicity<double>((const double2 *)r.un, r.g, nb, c->spec, c->ens, c->stream));
    else
        NS_CK(plain_helicity<float>((const float2 *)r.un, r.g, nb, c->spec, c->ens, c->stream));
    std::vector<double> hs(nb);
    NS_CK(cudaMemcpyAsync(hs.data(), c->spec, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    NS_CK(cudaStreamSynchronize(c->stream));
    double h = 0.0;
    for (int k = 0; k < nb; k++) h += hs[k];
    for (int k = 0; k < nbins && k < nb; k++) spec[k] = hs[k];
    if (helicity) *helicity = h;
    if (!isfinite(h)) return NS_ERR_NONFINITE;
    return check_flags(c);
}

ns_status ns_series(ns_ctx *c, int run, int count, double *energy, double *enstrophy,
                    int *written) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    if (run < 0 || run >= (int)c->runs.size() || count < 0 || !written ||
        (count > 0 && (!energy || !enstrophy)))
        return NS_ERR_ARG;
    Run &r = c->runs[run];
    std::vector<double> ring(2 * kSeriesCap);
    unsigned long long cnt = 0;
    NS_CK(cudaMemcpyAsync(ring.data(), r.series, ring.size() * sizeof(double),
                          cudaMemcpyDeviceToHost, c->stream));
    NS_CK(cudaMemcpyAsync(&cnt, r.counter, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    NS_CK(cudaStreamSynchronize(c->stream));
    unsigned long long avail = cnt < (unsigned long long)kSeriesCap ? cnt : kSeriesCap;
    int w = (int)std::min<unsigned long long>(avail, (unsigned long long)count);
    for (int i = 0; i < w; i++) {
        const unsigned long long idx = (cnt - w + i) % kSeriesCap;
        energy[i] = ring[2 * idx];
        enstrophy[i] = ring[2 * idx + 1];
    }
    *written = w;
    return NS_OK;
}

ns_status ns_kernel_census(ns_ctx *c, int nsteps, ns_kernel_time *out, int max, int *count) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    if (nsteps < 1 || max < 0 || !count || (max > 0 && !out)) return NS_ERR_ARG;
    for (Run &r : c->runs) {
        FftRes *f[3];
        if ((st = get_fft3(c, r.g, f)) != NS_OK) return st;
    }
    Tracer tr;
    tr.s = c->stream;
    for (int i = 0; i < nsteps; i++)
        if ((st = step_all(c, c->stream, &tr)) != NS_OK) return st;
    if (tr.err != cudaSuccess) return fail_cuda(c, tr.err);
    NS_CK(cudaStreamSynchronize(c->stream));
    std::vector<ns_kernel_time> agg;
    for (const Tracer::Rec &rec : tr.recs) {
        float ms = 0.f;
        NS_CK(cudaEventElapsedTime(&ms, rec.a, rec.b));
        size_t i = 0;
        while (i < agg.size() && strncmp(agg[i].name, rec.name, sizeof(agg[i].name)) != 0) i++;
        if (i == agg.size()) {
            ns_kernel_time k;
            memset(&k, 0, sizeof(k));
            strncpy(k.name, rec.name, sizeof(k.name) - 1);
            agg.push_back(k);
        }
        agg[i].launches++;
        agg[i].total_ms += ms;
    }
    int w = 0;
    for (size_t i = 0; i < agg.size() && w < max; i++) out[w++] = agg[i];
    *count = (int)agg.size();
    return check_flags(c);
}

ns_status ns_sync(ns_ctx *c) {
    ns_status st = check_ctx(c);
    if (st != NS_OK) return st;
    NS_CK(cudaStreamSynchronize(c->stream));
    NS_CK(cudaGetLastError());
    return check_flags(c);
}

}  // extern "C"
