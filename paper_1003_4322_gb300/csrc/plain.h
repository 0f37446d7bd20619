// plain.h -- launchers of the plain-form pointwise kernels and reductions.
#pragma once
#include "grid.cuh"
#include "ns_internal.h"

namespace nsk {

Grid make_grid(int nx, int ny, int nz, double lx, double ly, double lz);
// Shells K = 0 .. ceil(|k|_max lmax) (ceil(sqrt(3) N / 2) + 1 shells on the cube).
int grid_nbins(const Grid &g);
// Largest |k|^2 of the half layout on a unit box (size of the factor tables - 1).
long grid_max_k2(const Grid &g);

struct UpdateArgs {
    int stage;        // 1 or 2
    double dt;
    double force_amp;
    int force_k;      // 0: unforced
    int mfx, mfy, mfz;   // grid index of kf along each axis (kf l_i)
    int dealias;
    double rot;       // rotation rate about z (Coriolis -2 rot z x u)
};

// rc (the curl, both updates, the energy partials): the rectangle of the
// half layout outside which the state is zero and which alone the (pruned)
// transforms read; with rc.on the curl and the updates touch only its modes,
// and the partials load only its modes (in the same summation order).
template <typename T>
cudaError_t plain_curl(const typename Cx<T>::type *a, typename Cx<T>::type *w, const Grid &g, const Rect &rc,
                       cudaStream_t s);
template <typename T> cudaError_t plain_cross(T *u, const T *w, const Grid &g, cudaStream_t s);
// MHD: g = [u, w, b, j] on the grid -> g[0..3) = u x w + j x b, g[3..6) = u x b.
template <typename T> cudaError_t plain_cross_mhd(T *f, const Grid &g, cudaStream_t s);
// Phase-shift dealiasing: dst = src exp(i k.D) (the shifted grid's coefficients), and
// acc = (acc + sh exp(-i k.D)) / 2; D half a grid spacing along every axis,
// k.D = pi sum_i m_i / N_i, three components; ph = the per-axis factors
// exp(i pi m / N_i) by array position, [N_x | N_y | N_z/2+1].
template <typename T>
cudaError_t plain_phase(const typename Cx<T>::type *src, typename Cx<T>::type *dst,
                        const typename Cx<T>::type *ph, const Grid &g, cudaStream_t s);
template <typename T>
cudaError_t plain_phase_avg(typename Cx<T>::type *acc, const typename Cx<T>::type *sh,
                            const typename Cx<T>::type *ph, const Grid &g, cudaStream_t s);
// MHD induction update of b (stage 1: b1 = E (b + dt N_b); stage 2: b = E b/2 +
// (b1 + dt N_b)/2) from nb = transform of u x b.  Factor tables (etab here,
// and the update's): exp(-c k^2 dt) by integer |k|^2 on a unit box, else the
// per-axis factors exp(-c k_i^2 dt) by array position, [N_x | N_y | N_z/2+1].
template <typename T>
cudaError_t plain_update_b(typename Cx<T>::type *b, typename Cx<T>::type *b1,
                           const typename Cx<T>::type *nb, const T *etab, const Grid &g, int stage,
                           double dt, int dealias, const Rect &rc, cudaStream_t s);
template <typename T>
cudaError_t plain_update(typename Cx<T>::type *a, typename Cx<T>::type *a1,
                         const typename Cx<T>::type *nl, const T *etab, const Grid &g,
                         const UpdateArgs &ua, const Rect &rc, cudaStream_t s);
int energy_nparts(long M);
template <typename T>
cudaError_t plain_energy_partials(const typename Cx<T>::type *a, const Grid &g, double *part, const Rect &rc,
                                  cudaStream_t s);
template <typename T>
cudaError_t plain_spectrum(const typename Cx<T>::type *a, const Grid &g, int nbins, double *spec,
                           double *ens, cudaStream_t s);
template <typename T>
cudaError_t plain_helicity(const typename Cx<T>::type *a, const Grid &g, int nbins, double *spec,
                           double *aux, cudaStream_t s);
cudaError_t energy_final(const double *part, int nparts, double *series, int cap,
                         unsigned long long *counter, int *flags, cudaStream_t s);

}  // namespace nsk
