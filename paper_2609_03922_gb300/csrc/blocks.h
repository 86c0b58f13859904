// Block geometry and the launchers of the activity / state / update kernels.
#pragma once
#include "internal.h"

namespace spdba {

spdba_status make_geom(Geom* g, int ndim, const int64_t* dims, const int32_t* block);
// `batch` equal fields of ndim <= 2 dims stacked along the leading padded axis.
spdba_status make_geom_batched(Geom* g, int ndim, const int64_t* dims, const int32_t* block, long long batch);

// maxsq / sumsq per block; per run r, gmax[2r] = max over all its modes and
// gmax[2r+1] = max over its modes k != 0.  gmax must be zeroed before the
// launch (the kernel max-reduces into it).
template <typename T>
spdba_status launch_block_activity(const Geom& g, const cx_t<T>* q, double* maxsq, double* sumsq, double* gmax,
                                   cudaStream_t st);
// Per run r: tau[r] = threshold (ABS) or threshold * sqrt(gmax[2r + exclude_dc])
// (REL_MAX); also records tau and the max amplitude in stats[r] (may be null).
spdba_status launch_tau(const double* gmax, int nruns, double threshold, int tau_rule, int exclude_dc, double* tau,
                        DevStats* stats, cudaStream_t st);
// States, frozen-neighbour bits and the ordered list of non-frozen blocks.
size_t classify_scratch_bytes(long long nb);
spdba_status launch_classify(const Geom& g, const double* msq, int msq_is_square, const double* tau, int force_dc,
                             int transitions, int all_active, uint8_t* active, uint8_t* states, uint8_t* chi,
                             int32_t* list, int32_t* count, void* scratch, DevStats* stats, cudaStream_t st);
// Classification straight from an activity scan's maxima (gmax, 2 per run):
// tau per run by launch_tau's rule, states, chi, list, counts; then gmax is
// zeroed for the next scan.  Three launches.
spdba_status launch_classify_from_scan(const Geom& g, const double* msq, int msq_is_square, double* gmax,
                                       double threshold, int tau_rule, int exclude_dc, int force_dc, int transitions,
                                       double* tau, uint8_t* active, uint8_t* states, uint8_t* chi, int32_t* list,
                                       int32_t* count, void* scratch, DevStats* stats, cudaStream_t st);

// Cahn-Hilliard update.  k2 tables: per axis (padded to 3 axes) |k_a|^2 in T.
template <typename T> struct CHUpdateArgs {
    cx_t<T>* c_hat;
    const cx_t<T>* g_hat;
    const T* k2ax[3];
    const T* taper[3];
    const uint8_t* states;
    const uint8_t* chi;
    const int32_t* list;
    const int32_t* count;
    T dt, dtkappa;
    DevStats* stats;   // one per run
};
template <typename T> spdba_status launch_ch_update(const Geom& g, const CHUpdateArgs<T>& a, int dense, cudaStream_t st);

// TMA form of the list-driven update (3-D complex64, 8^3 blocks, one run):
// tensor-map descriptors (128 bytes, 64-byte aligned) of c_hat and g_hat made
// once at plan creation; launch shape from tma_update_prepare.
bool tma_update_fits(const Geom& g);
spdba_status make_box_map(void* map_out, const void* base, const Geom& g);
// Tensor map (128 bytes at map_out, 64-byte aligned) over a 3-D array of 8-byte
// elements: dims = {x, y, z} extents (x fastest), row and plane strides in
// bytes, box = {x, y, z} extents of one copy (each <= 256; box x * 8 bytes a
// multiple of 16).  SPDBA_ERR_UNSUPPORTED where the driver has no encoder.
spdba_status tma_encode_3d(void* map_out, const void* base, const uint64_t dims[3], const uint64_t row_bytes,
                           const uint64_t plane_bytes, const uint32_t box[3]);
spdba_status tma_update_prepare(int* per_sm, int* nsm);
spdba_status launch_ch_update_tma(const void* map_c, const void* map_g, const Geom& g, const CHUpdateArgs<float>& a,
                                  long long grid, cudaStream_t st);

// Per-axis |k|^2 table and taper table, computed in FP64 on the host.
template <typename T> std::vector<T> k2_table(long long n, double dx);
template <typename T> std::vector<T> taper_table(int B);

}  // namespace spdba
