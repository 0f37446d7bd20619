// plain.h -- launchers of the plain-form pointwise kernels and reductions.
#pragma once
#include "ns_internal.h"

namespace nsk {

struct UpdateArgs {
    int stage;        // 1 or 2
    double dt;
    double force_amp;
    int force_k;
    int dealias;
    double rot;       // rotation rate about z (Coriolis -2 rot z x u)
};

template <typename T>
cudaError_t plain_curl(const typename Cx<T>::type *a, typename Cx<T>::type *w, int n, cudaStream_t s);
template <typename T> cudaError_t plain_cross(T *u, const T *w, int n, cudaStream_t s);
// MHD: g = [u, w, b, j] on the grid -> g[0..3) = u x w + j x b, g[3..6) = u x b.
template <typename T> cudaError_t plain_cross_mhd(T *g, int n, cudaStream_t s);
// Phase-shift dealiasing: dst = src exp(i k.D) (the shifted grid's coefficients), and
// acc = (acc + sh exp(-i k.D)) / 2; D = (pi/N)(1,1,1), three components.
template <typename T>
cudaError_t plain_phase(const typename Cx<T>::type *src, typename Cx<T>::type *dst, int n, cudaStream_t s);
template <typename T>
cudaError_t plain_phase_avg(typename Cx<T>::type *acc, const typename Cx<T>::type *sh, int n, cudaStream_t s);
// MHD induction update of b (stage 1: b1 = E (b + dt N_b); stage 2: b = E b/2 +
// (b1 + dt N_b)/2) from nb = transform of u x b; etab = exp(-eta k^2 dt).
template <typename T>
cudaError_t plain_update_b(typename Cx<T>::type *b, typename Cx<T>::type *b1,
                           const typename Cx<T>::type *nb, const T *etab, int n, int stage, double dt,
                           int dealias, cudaStream_t s);
template <typename T>
cudaError_t plain_update(typename Cx<T>::type *a, typename Cx<T>::type *a1,
                         const typename Cx<T>::type *nl, const T *etab, int n, const UpdateArgs &ua,
                         cudaStream_t s);
int energy_nparts(int n);
template <typename T>
cudaError_t plain_energy_partials(const typename Cx<T>::type *a, int n, double *part, cudaStream_t s);
template <typename T>
cudaError_t plain_spectrum(const typename Cx<T>::type *a, int n, int nbins, double *spec, double *ens,
                           cudaStream_t s);
template <typename T>
cudaError_t plain_helicity(const typename Cx<T>::type *a, int n, int nbins, double *spec, double *aux,
                           cudaStream_t s);
cudaError_t energy_final(const double *part, int nparts, double *series, int cap,
                         unsigned long long *counter, int *flags, cudaStream_t s);

}  // namespace nsk
