// Reaction-cross-diffusion (RCD) kernels: M coupled components per mode
// (Supplementary S4.1-S4.3).
#pragma once
#include "internal.h"

namespace spdba {

// Largest component count the RCD kernels take.
constexpr int kRcdMaxComponents = 64;

template <typename T> struct RcdArgs {
    cx_t<T>* u_hat;          // M * n transformed components (component-major)
    const cx_t<T>* g_hat;    // M * n: FFT of the reaction term
    const T* V;              // M x M eigenvectors of D, row-major V[i * M + j] (D = V diag(lam) V^T)
    const T* lam;            // M eigenvalues of D
    const T* k2ax[3];        // |k_a|^2 per axis (padded to 3 axes)
    const T* taper[3];       // transition taper per axis
    const uint8_t* states;
    const uint8_t* chi;
    const int32_t* list;
    const int32_t* count;
    T dt;
    int M;
    long long n;             // modes per component
    DevStats* stats;         // one (the plan's single run)
};

// R_i(u) = u_i (r - a u_i - sum_{j != i} alpha_ij u_j) at every grid point,
// in place on the inverse transform's output (real parts read, (R, 0) written).
template <typename T>
spdba_status launch_rcd_reaction(cx_t<T>* work, long long n, int M, T r, T a, T alpha, T beta, cudaStream_t st);

// Per block: maxsq[b] = max_{k in B} A(k)^2 with A(k)^2 = (1/M) sum_m |u_m(k)|^2
// (FP64-accurate: a double-float sum of exact squares for complex64, FP64 for
// complex128); gmax[0] = max over all k, gmax[1] = max over k != 0 (max-reduced:
// zero before).
template <typename T>
spdba_status launch_rcd_activity(const Geom& g, const cx_t<T>* u_hat, int M, double* maxsq, double* gmax,
                                 cudaStream_t st);

// The update (I + dt k^2 D)^{-1} [u_hat + dt g_hat] = V (I + dt k^2 Lambda)^{-1} V^T [...]
// on the listed blocks (dense = 0) or on every block (dense = 1); transition
// blocks blend with the taper.  Adds the step's non-frozen share to the stats.
template <typename T> spdba_status launch_rcd_update(const Geom& g, const RcdArgs<T>& a, int dense, cudaStream_t st);
// Sets the update kernel's shared-memory limit and records its launch shape
// for M components (once per process; call at plan creation).
template <typename T> spdba_status rcd_prepare(int M);

}  // namespace spdba
