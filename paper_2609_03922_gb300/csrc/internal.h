// Host-side declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/spdba.h"
#include "fft_core.cuh"

namespace spdba {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
spdba_status fail(spdba_status s, const char* fmt, ...);
spdba_status cuda_fail(cudaError_t e, const char* what);
// Every device buffer of the library is allocated and freed here: the two
// count the live buffers, and dev_alloc fails one chosen allocation when told
// to (spdba_debug_fail_alloc), so the out-of-memory path can be tested on the
// host without exhausting a GPU.
cudaError_t dev_alloc(void** p, size_t bytes);
void dev_free(void* p);
// Iteration limit of a device wait on an mbarrier (the TMA kernels): the
// default, also the limit of the waits that let a timed-out kernel's copies in
// flight land before it returns; wait_limit() is the first waits' limit for
// kernels launched now (spdba_debug_set_wait_limit).
constexpr long long kWaitLimit = 1ll << 24;
long long wait_limit();
// Whether kernels launched now stall their first wait (spdba_debug_stall_waits).
int stall_waits();
#define SPDBA_CUDA(call)                                              \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ::spdba::cuda_fail(e_, #call);  \
    } while (0)

// ------------------------------------------------------------------ FFT passes
bool length_ok(int64_t n);              // 2^a 3^b
bool tile_length_supported(int64_t L);  // has a pass kernel

// Owner of device twiddle tables of one precision: exp(-2 pi i m / n), m < n,
// computed in FP64 on the device and rounded to the element type.
template <typename T> struct TwiddleCache {
    std::map<int64_t, cx_t<T>*> tables;
    cx_t<T>* get(int64_t n, cudaStream_t st, spdba_status* err);
    void release();
};

template <typename T> struct Pass {
    const void* func = nullptr;
    int nt = 0, smem = 0;
    int P = 0;           // pencils per tile
    long long grid = 0;
    PassParams<T> p{};
};

// Build a pass of length L over pencils (O, I) with the given strides.
template <typename T>
spdba_status make_pass(Pass<T>* out, int64_t L, int sign, int mode, long long O, long long I,
                       long long isO, long long isI, long long isJ, long long osO, long long osI,
                       long long osJ, TwiddleCache<T>& tw, cudaStream_t st);
template <typename T> spdba_status launch_pass(const Pass<T>& ps, const void* in, void* out, cudaStream_t st);

// A complete transform: list of passes (forward and inverse), scratch for the
// out-of-place four-step second pass.
template <typename T> struct FftEngine {
    int ndim = 0;
    int64_t dims[3] = {1, 1, 1};
    int64_t batch = 1;
    int64_t total = 0;  // elements per transform * batch
    std::vector<Pass<T>> fwd, inv;
    std::vector<int> fwd_scratch_out, inv_scratch_out;  // 1 if the pass writes to scratch
    cx_t<T>* scratch = nullptr;
    spdba_status init(int ndim, const int64_t* dims, int64_t batch, TwiddleCache<T>& tw, cudaStream_t st);
    spdba_status exec(const cx_t<T>* in, cx_t<T>* out, int direction, cudaStream_t st);
    void release();
};

// Half-spectrum pass of a 3-D complex64 field (PASS_HERM_INV, PASS_NL_HALF,
// PASS_MIRROR, PASS_UPD_HALF); the caller fills the update / mass fields.
spdba_status make_half_pass(Pass<float>* out, int mode, const HalfGeo& hg, TwiddleCache<float>& tw, cudaStream_t st);
// List the live tiles of a paired z forward pass (one with block states) into
// list[] (at most its tile count) and their number into *count.
spdba_status launch_pair_live_list(const Pass<float>& ps, int* list, int* count, cudaStream_t st);
// Live x-frequency columns of the half array for the paired z forward (one
// byte per column, NHP of them) from a single 3-D run's block states.

// Half-spectrum storage: live z pencils (zlive, N1 x NHP) and x columns (xlive,
// NHP) of the stored half under the half map's states (g: that map).
spdba_status launch_hs_live(const Geom& g, const uint8_t* states, uint8_t* zlive, uint8_t* xlive, cudaStream_t st);
spdba_status launch_half_col_live(const Geom& g, const uint8_t* states, int N2, int NHP, uint8_t* col_live,
                                  cudaStream_t st);
// Tiles of a paired z forward pass.
long long pair_tile_count(const Pass<float>& ps);
// Pencils per tile of the pass kernels of length L (0 if none).
template <typename T> int pass_tile_pencils(int64_t L);

// ------------------------------------------------------------------ TMA z inverse
// The Hermitian z inverse of the half-spectrum form with its tiles moved as
// tensor boxes (fft_herm_tma.cu): three tensor maps over c_hat (direct tile,
// mirror tile, the kx = 0 columns), the kernel, its shared memory and grid.
constexpr int kHermTmaNT = 256;
struct HermTma {
    alignas(64) unsigned char map[3][128];
    const void* func = nullptr;
    size_t smem = 0;
    long long grid = 0;
    bool ok = false;
};
// Fills ht for the z inverse pass zinv over c_hat; SPDBA_ERR_UNSUPPORTED (ht.ok
// false) where the shape has no TMA form (x rows not a whole number of tiles,
// lengths without a kernel, no tensor-map encoder).
spdba_status herm_tma_prepare(HermTma* ht, const Pass<float>& zinv, const void* c_hat);
// Same results as launch_pass(zinv, in, out) bit for bit; `in` must be the
// c_hat the maps were made for.  A wait that runs out adds 1 at *timeouts.
spdba_status launch_herm_inv_tma(const HermTma& ht, const Pass<float>& zinv, const void* in, void* out,
                                 unsigned long long* timeouts, cudaStream_t st);

// ------------------------------------------------------------------ multi-size passes
// One launch of a pass phase over every group of a batched complex64 plan: the
// groups' tiles form one queue (group after group) that the persistent CTAs of
// the launch walk in a fixed stride.
constexpr int kMultiMaxGroups = 8;
constexpr int kMultiNT = 256;
template <typename T> struct MultiGroup {
    PassParams<T> a;   // the group's pass with its input and output set (fu.dense 0, mass set)
    int L, P;          // pencil length, pencils per tile
    unsigned t0, nt;   // first tile in the queue's numbering, tile count
};
// Pencils per tile of length L in the multi-size table of `tile` elements per
// tile (4096 or 2048); 0 if the length has no multi-size kernel.
int multi_tile_pencils(int tile, int64_t L);
// Kernel, dynamic shared memory and resident CTAs (occupancy x SMs) of a
// multi-size pass: pfast = row-major tiles (PASS_PLAIN, PASS_CH_UPDATE), else
// pencil-major tiles (PASS_CH_NL).  Sets the kernel's shared-memory limit.
spdba_status multi_kernel(int tile, int sign, int mode, bool pfast, const void** func, int* smem,
                          long long* resident);
// One launch over `ng` groups (device array) and `total` queue positions.
// Bit g of dense_mask: group g updates every block this step; of mass_mask:
// group g accumulates its runs' mass (the nonlinearity pass).
spdba_status launch_multi(const void* func, int smem, long long grid, const MultiGroup<float>* groups, int ng,
                          unsigned total, unsigned dense_mask, unsigned mass_mask, cudaStream_t st);

// Pass along axis `axis` of `batch` contiguous arrays of shape dims (in place).
template <typename T>
spdba_status make_axis_pass(Pass<T>* out, int ndim, const int64_t* dims, int64_t batch, int axis, int sign,
                            int mode, TwiddleCache<T>& tw, cudaStream_t st);

}  // namespace spdba

struct spdba_predictor;
// Predicted states: features from (maxsq, tau, states) -> network -> measure_out = p (FP64).
spdba_status spdba_predictor_states_internal(spdba_predictor* pr, const double* maxsq, const double* tau,
                                             uint8_t* states, int32_t nmaps, void* x_scratch, double* measure_out,
                                             cudaStream_t st);
bool spdba_predictor_map_matches(const spdba_predictor* pr, long long nd, long long nh, long long nw);
