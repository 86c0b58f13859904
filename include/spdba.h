/*
 * spdba.h - C ABI of the GB300 (sm_103a) sp-DBA library, libspdba.so.
 *
 * sp-DBA (spectral dynamic block activation, arXiv 2609.03922) runs a
 * time-stepped transform-domain solver whose transformed field is cut into
 * fixed blocks.  Each block gets an activity measure that is compared with a
 * threshold; ACTIVE blocks run the model's update core, TRANSITION blocks
 * (neighbours of active blocks) apply a tapered increment, FROZEN blocks keep
 * their stored values (Methods; Supplementary S1.1).  The update sits between
 * a forward and an inverse FFT, both written here as CUDA kernels.
 *
 * Conventions for every entry point:
 *   - Return value: SPDBA_OK or an error code; no call aborts the process.
 *     spdba_last_error() returns a human-readable message for the calling
 *     thread's most recent failure.  A CUDA error seen by a plan is latched:
 *     every later call on that plan returns SPDBA_ERR_CUDA.
 *   - Arrays are row-major with the last axis fastest.  dims[0] is the slowest
 *     axis.  Complex values are interleaved (re, im) pairs of float (C64) or
 *     double (C128).
 *   - Caller buffers are never retained past the call.  "device" pointers
 *     must be CUDA device (or managed) memory on the current device; "host"
 *     pointers are ordinary host memory (pinned host memory makes the copy
 *     asynchronous with respect to the host thread up to the call's own sync).
 *   - Work is enqueued on the stream given in spdba_options.stream (or, for
 *     the kernel-level calls, the `stream` argument; NULL = legacy default).
 */
#ifndef SPDBA_H
#define SPDBA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPDBA_OK = 0,
    SPDBA_ERR_ARG = 1,          /* NULL pointer, bad enum value, size mismatch          */
    SPDBA_ERR_UNSUPPORTED = 2,  /* a length with a prime factor other than 2 or 3, a
                                   block edge that does not divide the grid, a length
                                   outside the supported range                           */
    SPDBA_ERR_CUDA = 3,         /* a CUDA runtime call or kernel failed (latched)        */
    SPDBA_ERR_OOM = 4,          /* device allocation failed                              */
    SPDBA_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out                    */
    SPDBA_ERR_STATE = 6         /* call not valid in the plan's current state            */
} spdba_status;

/* CH: Cahn-Hilliard-form semi-implicit step (S3.1, S4.2 with M = 1); NLS: split-step
   Fourier (S5.1-S5.2); RCD: M-component reaction-cross-diffusion (S4.1-S4.3). */
enum { SPDBA_MODEL_CH = 0, SPDBA_MODEL_NLS = 1, SPDBA_MODEL_RCD = 2 };
enum { SPDBA_C64 = 0, SPDBA_C128 = 1 };
/* spdba_apply(mode) of the paper (S2.1): 0 = Regular full update, 1 = sp-DBA */
enum { SPDBA_MODE_REGULAR = 0, SPDBA_MODE_ADAPTIVE = 1 };
/* Activation measure.  MAXAMP: A_B = max_{k in B} |q(k)| (S4.2, any-mode amplitude).
   ENERGY: ||q_B||_2 = sqrt(sum_{k in B} |q(k)|^2) (Results, PFC block energy). */
enum { SPDBA_MEASURE_MAXAMP = 0, SPDBA_MEASURE_ENERGY = 1 };
/* Threshold rule.  REL_MAX: tau = threshold * max_k |q(k)|, with k = 0 left out of
   the max for the conserved Cahn-Hilliard field.  ABS: tau = threshold. */
enum { SPDBA_TAU_REL_MAX = 0, SPDBA_TAU_ABS = 1 };
/* Block states as returned by spdba_get_mask (Methods). */
enum { SPDBA_FROZEN = 0, SPDBA_TRANSITION = 1, SPDBA_ACTIVE = 2 };
/* FFT direction: forward uses exp(-2 pi i n k / N), inverse exp(+...) and 1/N. */
enum { SPDBA_FORWARD = -1, SPDBA_INVERSE = 1 };

typedef struct spdba_options {
    int32_t model;          /* SPDBA_MODEL_CH or SPDBA_MODEL_NLS                          */
    int32_t precision;      /* SPDBA_C64 (FP32 bulk, FP64 norms) or SPDBA_C128 (FP64)     */
    int32_t mode;           /* SPDBA_MODE_REGULAR or SPDBA_MODE_ADAPTIVE                  */
    int32_t measure;        /* SPDBA_MEASURE_*                                            */
    int32_t tau_rule;       /* SPDBA_TAU_*                                                */
    int32_t transitions;    /* 1: transition blocks with boundary-aware smoothing (S1.1) */
    int32_t force_dc;       /* 1: the block holding k = 0 is always ACTIVE (S6.1)         */
    int32_t refresh_every;  /* F_refresh: all blocks ACTIVE every F steps, 0 = off (S1.3) */
    int32_t warmup_steps;   /* all blocks ACTIVE for the first steps (S3.2), 0 = none     */
    int32_t use_graph;      /* 1: replay captured CUDA graphs for runs of steps          */
    int32_t fuse_update;    /* CH: 1 = apply the update inside the last forward FFT pass;
                               0 = separate update kernel over the block list (staged)  */
    int32_t half_spectrum;  /* 3-D CH, complex64: 1 = run the transforms on x frequencies
                               0 .. N2/2 of the Hermitian part of c_hat (c = Re IFFT(c_hat)
                               is its inverse), 0 = full complex transforms; ignored where
                               no half-spectrum kernels exist for the shape                */
    double dt, kappa, dx;   /* Cahn-Hilliard: time step, gradient coefficient, spacing  */
    double beta2, gamma, h, dt_sample; /* NLS: ps^2/km, 1/(W km), km step, ps sample     */
    void* stream;           /* cudaStream_t the plan enqueues on                         */
    /* Dynamic threshold control (S1.3), adaptive plans without a predictor.  Every
       control_every steps (once the warm-up is over) each run compares its mean share
       r of non-frozen blocks over the adaptive steps since the last check with
       target_ratio: with q = r / target_ratio the threshold coefficient is doubled
       (q > 2), halved (q < 0.5), scaled by 1 + control_eta (q > 1 + eta) or
       1 - control_eta (q < 1 - eta), or kept; the check step itself runs with every
       block ACTIVE (the full-activation step that follows each check).  The
       coefficient is `threshold` of spdba_plan_create under either tau_rule. */
    double target_ratio;    /* 0 = control off (default)                                   */
    double control_eta;     /* relative deadband and step factor, default 0.05             */
    int32_t control_every;  /* control interval in steps, default 50                       */
    /* RCD (S4.1-S4.2): du/dt = D lap u + R(u) with M components, D symmetric circulant
       (D_ii = rcd_d_diag + 2 rcd_d_cross, -rcd_d_cross to the two periodic neighbour
       components), R_i = u_i (rcd_r - rcd_a u_i - sum_{j != i} alpha_ij u_j) with
       alpha_ij = rcd_beta + rcd_alpha for the neighbours and rcd_beta otherwise; per mode
       u_hat <- V (I + dt k^2 Lambda)^{-1} V^T [u_hat + dt FFT(R)] with D = V Lambda V^T
       (S4.3).  The activation measure is the component RMS amplitude
       A(k) = sqrt(mean_m |u_hat_m(k)|^2); one state per block for all components. */
    int32_t components;     /* M, 1..64, default 8                                          */
    double rcd_d_diag, rcd_d_cross, rcd_alpha, rcd_beta, rcd_r, rcd_a;  /* 0.5 0.05 1 0.3 1 1 */
    int32_t tma_update;     /* 1: the staged CH update of 3-D complex64 plans with 8^3 blocks
                               moves whole blocks as TMA boxes (same values bit for bit);
                               0 (default): per-warp loads.  spdba_plan_autotune may change it. */
    int32_t multi_pass;     /* batched 2-D complex64 CH plans of several run sizes (2..8 groups of
                               equal-size runs, sides of 64, 128, 192, 256, 384 or 512 points, the
                               update fused into the last forward pass):
                               1 or 2 = each pass phase of a step is ONE persistent launch over
                               every group's tiles (one queue, group after group, walked by the
                               launch's CTAs in a fixed stride; tiles of 4096 or 2048 elements
                               respectively), 0 (default) = one launch
                               per group and phase, groups on concurrent streams.  All forms give
                               bit-identical fields and block states (the FP64 mass statistic
                               differs in rounding).  Ignored (0 in force) where the plan does
                               not qualify; spdba_plan_autotune may change it. */
    int32_t tma_passes;     /* 1 (default): the z inverse of the half-spectrum form (3-D complex64)
                               loads its direct and mirror tiles as TMA tensor boxes where its x rows
                               are a whole number of tiles; 0: per-thread cp.async copies.  Same
                               values bit for bit.  A bounded wait that runs out makes
                               spdba_get_stats return SPDBA_ERR_TIMEOUT. */
    int32_t half_storage;   /* 3-D CH complex64 (each 3-D run is its own group), 2 B2 | N2:
                               1 = store the spectrum of the real field as its half
                               kx = 0 .. N2/2 (S1.2): the block map covers that half (N2/(2 B2) + 1
                               x-blocks, the last holding kx = N2/2 alone), an ACTIVE block's
                               neighbour in the omitted half is activated through its conjugate
                               counterpart X(-k) = conj X(k) (Eq. S.4; the other axes' block
                               indices mirrored, b -> nb - 1 - b, x-block 0 across kx = 0 and
                               x-block N2/(2 B2) - 1 past the Nyquist block), and every transform
                               and the update run on the stored half.  c is the complex-to-real
                               inverse of the stored half (the kx = 0 and N2/2 planes contribute
                               their Hermitian part).  spdba_get/set_spectrum then take
                               N0 x N1 x (N2/2 + 1) values and spdba_get_mask / spdba_get_activity
                               N0/B0 x N1/B1 x (N2/(2 B2) + 1) blocks.  0 (default) = full
                               spectrum.  SPDBA_ERR_UNSUPPORTED where the plan does not qualify. */
} spdba_options;

/* Per-run statistics, refreshed at each reassessment. */
typedef struct spdba_stats {
    int64_t step;            /* steps taken so far                                       */
    int64_t assessments;     /* reassessments done (block states set, exact or predicted) */
    int64_t nblocks;         /* blocks in the block map                                  */
    int64_t n_active;        /* ACTIVE blocks at the last reassessment                  */
    int64_t n_transition;    /* TRANSITION blocks at the last reassessment              */
    double tau;              /* threshold value used at the last reassessment           */
    double max_amp;          /* max |q(k)| at the last reassessment (k = 0 excluded, CH) */
    double mass;             /* CH: FP64 sum of the real field at the last reassessment;
                                NLS: FP64 sum |E(t)|^2                                    */
    double active_ratio_sum; /* sum over steps of (ACTIVE + TRANSITION) / nblocks        */
    int64_t predictions;     /* reassessments answered by an attached predictor            */
    int64_t missed_blocks;   /* blocks an exact judge found non-frozen that the prediction
                                in force had frozen (summed over judges)                  */
    double threshold;        /* threshold coefficient in force (moves under dynamic control) */
    int64_t controls;        /* dynamic-control decisions made                             */
} spdba_stats;

typedef struct spdba_plan spdba_plan;         /* opaque; owns all of its device buffers */
typedef struct spdba_fft_plan spdba_fft_plan; /* opaque; owns its twiddle tables        */

/* Fill *opt with the defaults: CH, C64, ADAPTIVE, MAXAMP, REL_MAX, transitions on,
   force_dc on (CH), refresh and warm-up off, graphs on, fused update on, dt = 0.01, kappa = 1,
   dx = 1, beta2 = -21.7, gamma = 1.3, h = 0.1, dt_sample = 1, default stream, threshold
   control off (target_ratio 0, control_eta 0.05, control_every 50). */
void spdba_options_default(spdba_options* opt);

/*
 * Create a plan for one field (spdba_init of S2.1).
 *   ndim        1, 2 or 3 (NLS: 1; CH: 2 or 3)
 *   dims[ndim]  grid extents; CH axes in {16, 32, 64, 128, 192, 256, 384, 512};
 *               NLS lengths 64..4096 (powers of two) and n1 * 512 with n1 in
 *               {16, 32, ..., 512} (up to 2^18); other lengths of the form
 *               2^a 3^b return SPDBA_ERR_UNSUPPORTED
 *   block[ndim] block edge per axis; must divide dims; the block map is
 *               dims[a]/block[a] per axis, row-major, slowest axis first
 *               (block b along an axis covers FFT indices [b*B, b*B + B - 1])
 *   threshold   see tau_rule; reassess  steps between block-state reassessments (>= 1)
 * The field starts at zero; set it with spdba_set_field.  *out receives the plan.
 * RCD plans (model SPDBA_MODEL_RCD) are 2-D or 3-D with opt->components fields;
 * their fields move in and out as components * prod(dims) reals, component-major.
 */
spdba_status spdba_plan_create(spdba_plan** out, int32_t ndim, const int64_t* dims,
                               const int32_t* block, double threshold, int32_t reassess,
                               const spdba_options* opt);

/*
 * Create one plan holding `nruns` independent fields of possibly different sizes
 * (an ensemble of CH runs or a batch of NLS signals) that step together.
 *   dims   nruns * ndim extents, run-major
 *   block  ndim block edges, or for NLS (block[0] <= 0) the block map has
 *          -block[0] blocks per signal (block edge = n / -block[0])
 */
spdba_status spdba_batch_create(spdba_plan** out, int32_t nruns, int32_t ndim,
                                const int64_t* dims, const int32_t* block, double threshold,
                                int32_t reassess, const spdba_options* opt);

/* Load run `run`'s field.  CH: real values (float for C64, double for C128),
   prod(dims) of them.  NLS: complex time-domain samples.  src_on_device selects
   a device or host source.  Resets the run's step counter, states and stats. */
spdba_status spdba_set_field(spdba_plan* plan, int32_t run, const void* src, int32_t src_on_device);

/* Advance every run by n steps (spdba_apply inside the time loop of S2.1).
   Asynchronous on the plan's stream; returns after enqueueing. */
spdba_status spdba_step(spdba_plan* plan, int64_t n);

/* Copy run `run`'s real-space field (CH: Re(IFFT(c_hat)) as real values; NLS:
   complex E(t)) to dst.  Synchronizes the plan's stream. */
spdba_status spdba_get_field(spdba_plan* plan, int32_t run, void* dst, int32_t dst_on_device);

/* Copy / overwrite run `run`'s transformed field (complex, full spectrum, FFT order).
   get synchronizes; set resets nothing but the cached block measures. */
spdba_status spdba_get_spectrum(spdba_plan* plan, int32_t run, void* dst, int32_t dst_on_device);
spdba_status spdba_set_spectrum(spdba_plan* plan, int32_t run, const void* src, int32_t src_on_device);

/* Copy run `run`'s block states at the last reassessment (uint8: 0 FROZEN,
   1 TRANSITION, 2 ACTIVE; nblocks entries) to host memory.  Synchronizes. */
spdba_status spdba_get_mask(spdba_plan* plan, int32_t run, uint8_t* dst, int64_t nblocks);

/* Statistics of run `run`.  Synchronizes. */
spdba_status spdba_get_stats(spdba_plan* plan, int32_t run, spdba_stats* out);

/* Copy run `run`'s per-block max |q(k)|^2 (FP64, nblocks values) and tau of the
   last exact reassessment, to device or host memory.  Synchronizes. */
spdba_status spdba_get_activity(spdba_plan* plan, int32_t run, double* maxsq, double* tau, int32_t dst_on_device);

/* Wait for all work enqueued by the plan. */
spdba_status spdba_sync(spdba_plan* plan);

/* Release the plan and its device memory (spdba_destroy of S2.1).  NULL is a no-op. */
void spdba_plan_destroy(spdba_plan* plan);

/* Kernel timing on the plan's stream (CUDA events around each launch of the
   step path), for roofline reporting.  begin clears the record; end waits for
   the stream and returns one entry per kernel kind (at most `capacity`), the
   number of entries in *n_out, and the number of kernels the plan launched
   since begin in *launches_out.  `bytes` is the algorithmic traffic of all
   recorded launches of that kind (bytes read + written by its definition). */
typedef struct spdba_kernel_time {
    char name[40];
    int64_t launches;
    double total_ms;
    double bytes;
} spdba_kernel_time;
/*
 * Autotuner (no counterpart in the paper).  Times `steps` steps of the plan
 * for every candidate launch configuration -- the CH update fused into the
 * last forward FFT pass or staged as its own kernel (when the plan was created
 * with fuse_update = 1), the staged update's block loads by warps or by TMA
 * boxes (3-D complex64 plans with 8^3 blocks), the 3-D transforms on the Hermitian half spectrum or
 * on the full one (when created with half_spectrum = 1 and the shape has half-
 * spectrum kernels), one launch per pass phase over all groups of a batched
 * 2-D complex64 plan with tiles of 4096 or 2048 elements (multi_pass, with the
 * fused update) or one per group, and reassessment segments replayed as a CUDA graph or
 * launched directly (graphs only on a non-legacy stream) -- each from the same
 * state after one warm-up segment, keeps the fastest for later spdba_step
 * calls, and restores the plan's fields, block states, statistics and step
 * count, so that the tuning leaves no trace in the results.  Both update forms
 * and both launch modes give bit-identical fields; the two transform forms
 * differ by rounding only.  Needs about one extra copy
 * of the plan's state in device memory for the duration of the call; not with
 * an attached predictor (SPDBA_ERR_STATE).  report may be NULL.  Synchronizes.
 */
#define SPDBA_TUNE_MAX 16
typedef struct spdba_tune_report {
    int32_t n_candidates;
    int32_t fuse_update[SPDBA_TUNE_MAX];
    int32_t use_graph[SPDBA_TUNE_MAX];
    int32_t half_spectrum[SPDBA_TUNE_MAX];
    int32_t tma_update[SPDBA_TUNE_MAX];  /* staged list update moved by TMA boxes (3-D complex64,
                                            8^3 blocks) instead of per-warp loads */
    double ms_per_step[SPDBA_TUNE_MAX];
    int32_t chosen;          /* index of the configuration in force afterwards */
    int32_t multi_pass[SPDBA_TUNE_MAX];  /* the candidate's multi_pass (see spdba_options) */
    int32_t cached;          /* 1: spdba_plan_autotune_cached applied a stored choice (no
                                timing; n_candidates = 1, ms_per_step[0] = the stored time) */
} spdba_tune_report;
spdba_status spdba_plan_autotune(spdba_plan* plan, int32_t steps, spdba_tune_report* report);
/*
 * Tuning cache (process-wide).  Every spdba_plan_autotune call stores its
 * choice under the plan's signature: precision, model, mode, dimensionality,
 * block edges, the run extents and run counts of its groups, the options that
 * enable candidates (fuse_update, half_spectrum) and the plan's stream kind
 * (graphs need a non-legacy stream).  spdba_plan_autotune_cached applies the
 * stored choice to a plan of the same signature without timing anything
 * (report->cached = 1), else it is spdba_plan_autotune.  The state a plan was
 * tuned in (its share of frozen blocks) is not part of the signature.  Not
 * for concurrent use from several threads.  spdba_tune_cache_clear empties it.
 */
spdba_status spdba_plan_autotune_cached(spdba_plan* plan, int32_t steps, spdba_tune_report* report);
void spdba_tune_cache_clear(void);
/*
 * The options in force (those the plan was created with, with the launch
 * configuration the autotuner chose): fuse_update, half_spectrum, tma_update
 * and tma_passes are 1 where some group uses that form, multi_pass is the form
 * in force (0, 1 or 2), use_graph as set.  Not a synchronizing call.
 */
spdba_status spdba_plan_get_config(const spdba_plan* plan, spdba_options* out);

spdba_status spdba_profile_begin(spdba_plan* plan);
/* As spdba_profile_begin, but records the kernels of one step in `every`
   (steps whose index is a multiple of `every`), so that the events disturb a
   long timed run little.  every >= 1, else SPDBA_ERR_ARG. */
spdba_status spdba_profile_begin_sampled(spdba_plan* plan, int32_t every);
spdba_status spdba_profile_end(spdba_plan* plan, spdba_kernel_time* out, int32_t capacity, int32_t* n_out,
                               int64_t* launches_out);

const char* spdba_last_error(void);
const char* spdba_status_string(spdba_status s);

/*
 * Host-side fault injection for the out-of-memory path (no counterpart in the
 * paper).  After spdba_debug_fail_alloc(k), the k-th device allocation the
 * library makes from then on (k >= 1; plans, FFT plans, predictors and the
 * autotuner's snapshot all count) fails as if the device were out of memory,
 * without calling cudaMalloc: the call that needed it returns SPDBA_ERR_OOM,
 * spdba_last_error() names the allocation, and everything the call had
 * allocated is freed.  k <= 0 switches the injection off; it also ends by
 * itself after the failing allocation.  spdba_debug_live_allocs() returns the
 * number of device buffers the library holds right now (a leak check).
 * Process-wide; not for concurrent use from several threads.
 */
void spdba_debug_fail_alloc(int64_t k);
int64_t spdba_debug_live_allocs(void);
/*
 * Host-side control of the device waits (no counterpart in the paper).  The
 * TMA kernels (the half form's z inverse, the TMA list update) wait on
 * mbarriers for their tile copies with an iteration limit; when a wait runs
 * out the kernel counts it in the run's statistics, lets its copies in flight
 * land (waiting again, with the default limit), and returns, and
 * spdba_get_stats then reports SPDBA_ERR_TIMEOUT.
 * spdba_debug_set_wait_limit(n): n >= 1 sets the first waits' limit to n
 * polls for kernels launched from then on, n <= 0 restores the default
 * (2^24 polls).  spdba_debug_stall_waits(1): the first wait of every CTA of
 * those kernels targets a barrier nothing arrives on, so it runs out (after
 * the limit, at most 4096 polls) while the real copies complete; 0 switches
 * this off.  Graph
 * segments captured earlier keep the settings they were captured with.
 * Process-wide; for tests of the timeout path.
 */
void spdba_debug_set_wait_limit(int64_t n);
void spdba_debug_stall_waits(int32_t on);

/* ------------------------------------------------------------------------------ */
/* Kernel-level entry points (device pointers, caller-owned buffers).               */
/* ------------------------------------------------------------------------------ */

/*
 * Batched multi-dimensional complex FFT (Stockham, shared-memory staged), the
 * transform that surrounds every sp-DBA update (Methods, Fig. 1b).
 * `batch` transforms of shape dims[0..ndim-1], contiguous one after another.
 * Supported lengths: axes of 2-D/3-D transforms in {16, 32, 64, 128, 192,
 * 256, 384, 512}; 1-D lengths in {16, ..., 4096} of that set plus 1024, 2048,
 * 4096, and n1 * 512 with n1 in {16, 32, 64, 128, 192, 256, 384, 512} (up to
 * 2^18); anything else returns SPDBA_ERR_UNSUPPORTED.  Twiddles are computed
 * in FP64 once, at plan creation.
 */
spdba_status spdba_fft_plan_create(spdba_fft_plan** out, int32_t precision, int32_t ndim,
                                   const int64_t* dims, int64_t batch);
/* in and out may alias (in-place); direction SPDBA_FORWARD or SPDBA_INVERSE. */
spdba_status spdba_fft_exec(spdba_fft_plan* plan, const void* in, void* out,
                            int32_t direction, void* stream);
void spdba_fft_plan_destroy(spdba_fft_plan* plan);

/*
 * Per-block activity of a transformed field q (device, complex, shape dims):
 *   maxsq[b] = max_{k in B_b} |q(k)|^2,  sumsq[b] = sum_{k in B_b} |q(k)|^2
 * and gmax[0] = max over all k, gmax[1] = max over k != 0 (FP64, device).
 * |q|^2 is formed in FP64 as re*re + im*im (Methods: activation measure;
 * Results 2.1 block energy; S4.2 any-mode amplitude).
 */
spdba_status spdba_block_activity(int32_t precision, int32_t ndim, const int64_t* dims,
                                  const int32_t* block, const void* q, double* maxsq,
                                  double* sumsq, double* gmax, void* stream);

/*
 * Block states and the compacted list of non-frozen blocks (Methods: state
 * preparation; S1.1 frozen-neighbour pattern).
 *   measure[nb]  block measure in amplitude units (device, FP64)
 *   tau          device FP64 scalar: ACTIVE iff measure >= tau
 *   force_dc     1: block 0 is ACTIVE regardless; transitions: 1 = dilate by face
 *                neighbours (periodic) into TRANSITION
 *   states[nb]   out: 0/1/2;   chi[nb]  out: bit (2a) set when the lower neighbour
 *                along axis a is FROZEN, bit (2a+1) for the upper one (axis 0 slowest)
 *   list[nb]     out: ids of non-frozen blocks in increasing order; count[0] their number
 *   scratch      device buffer of at least spdba_classify_scratch_bytes(nb) bytes
 */
size_t spdba_classify_scratch_bytes(int64_t nb);
spdba_status spdba_classify(int32_t ndim, const int64_t* nblocks, const double* measure,
                            const double* tau, int32_t force_dc, int32_t transitions,
                            uint8_t* states, uint8_t* chi, int32_t* list, int32_t* count,
                            void* scratch, void* stream);

/* ------------------------------------------------------------------------------ */
/* Learned block-activity predictor (no counterpart in the paper).                  */
/* ------------------------------------------------------------------------------ */
/*
 * A 3-D convolutional network over a block map of nd x nh x nw blocks that
 * predicts, per block, the probability that the block is non-frozen at any
 * reassessment within the next K steps:
 *   a1 = conv(x, W1) + b1, h1 = relu(a1)    2 -> 8 channels
 *   a2 = conv(h1, W2) + b2, h2 = relu(a2)   8 -> 16
 *   a3 = conv(h2, W3) + b3, h3 = relu(a3)   16 -> 8
 *   p  = sigmoid(h3 . wh + bh);  loss = mean binary cross-entropy
 * conv is a 3x3x3 convolution with periodic wrap (tap = 9(dz+1) + 3(dy+1) +
 * (dx+1)).  Input features x[v] = (clamp(log10(A_B / tau) / 8, -1, 1),
 * 1 if the block is not FROZEN).  Arrays are channels-last, maps contiguous.
 * Parameters: one FP32 vector of spdba_predictor_num_params() values in the
 * order W1 (8x27x2), b1, W2 (16x27x8), b2, W3 (8x27x16), b3, wh (8), bh (1),
 * each W indexed [out][tap][in].  Convolutions run on BF16 tensor cores with
 * FP32 accumulation; activations between layers and the backpropagated
 * pre-activation gradients are BF16; Adam keeps FP32 master weights.
 */
typedef struct spdba_predictor spdba_predictor;
int64_t spdba_predictor_num_params(void);
/* max_batch: most maps per call; init_params: host FP32 vector (copied). */
spdba_status spdba_predictor_create(spdba_predictor** out, int32_t nd, int32_t nh, int32_t nw,
                                    int32_t max_batch, const float* init_params);
void spdba_predictor_destroy(spdba_predictor* pr);
spdba_status spdba_predictor_get_params(spdba_predictor* pr, float* host_out);
spdba_status spdba_predictor_set_params(spdba_predictor* pr, const float* host_in);
/* x_bf16 (device, nmaps*V*2 bf16) from per-block max|q|^2 (device FP64, nmaps*V),
   per-map tau (device FP64, nmaps) and block states (device u8, nmaps*V). */
spdba_status spdba_predictor_features(spdba_predictor* pr, const double* maxsq, const double* tau,
                                      const uint8_t* states, int32_t nmaps, void* x_bf16, void* stream);
/* prob (device FP32, nmaps*V). */
spdba_status spdba_predictor_forward(spdba_predictor* pr, const void* x_bf16, int32_t nmaps, float* prob,
                                     void* stream);
/* Loss and gradients without an update; labels device FP32 in {0,1}; host outputs. Synchronizes. */
spdba_status spdba_predictor_gradients(spdba_predictor* pr, const void* x_bf16, const float* labels,
                                       int32_t nmaps, double* loss_out, float* grads_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr; loss_out may be NULL. */
spdba_status spdba_predictor_train_step(spdba_predictor* pr, const void* x_bf16, const float* labels,
                                        int32_t nmaps, float lr, double* loss_out, void* stream);
/*
 * Let `pr` answer most reassessments of a 3-D Cahn-Hilliard plan with one run
 * whose block map matches the predictor's.  States are then set every
 * `horizon` steps (instead of every reassess interval): at multiples of
 * `judge_every` (and at the first step) by the exact activity scan, in between
 * by the predictor (ACTIVE where p >= prob_threshold, then the usual
 * transition dilation and k = 0 forcing), fed with the last exact scan's
 * activity and the states in force.  Each exact judge counts the blocks it
 * finds non-frozen that the prediction in force had frozen (spdba_stats
 * missed_blocks) and replaces the prediction.  The plan does not own `pr`;
 * pass NULL to detach.
 */
spdba_status spdba_plan_attach_predictor(spdba_plan* plan, spdba_predictor* pr, int32_t horizon,
                                         int32_t judge_every, float prob_threshold);

/*
 * spdba_classify without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- for
 * example code that runs under a framework which owns every device buffer and
 * hands out only the inputs and outputs, or a fixed-footprint service loop
 * where any cudaMalloc is forbidden after start-up.
 *
 * Same arguments and results as spdba_classify, minus `scratch`: the scratch
 * is a fixed array of about 1 MiB compiled into the library (every GPU that
 * loads the library holds it until the process exits).  At most
 * SPDBA_CLASSIFY_STATIC_MAX_BLOCKS blocks; larger maps return
 * SPDBA_ERR_UNSUPPORTED.  Each call made outside stream capture looks up the
 * array's device address (cudaGetSymbolAddress) with the current device, so a
 * device reset between calls is harmless; a call made during capture reuses
 * the address of that device's last uncaptured call, so make one call on the
 * device before any stream capture (else SPDBA_ERR_STATE).  Calls never call cudaMalloc or
 * cudaFree.  All calls share the one array and it keeps the previous call's
 * contents (nothing in it needs to start at zero: each call writes what it
 * reads), so calls whose kernels overlap on the GPU (different streams, or
 * different host threads) race: serialize them.
 */
#define SPDBA_CLASSIFY_STATIC_MAX_BLOCKS (1 << 20)
spdba_status spdba_classify_static(int32_t ndim, const int64_t* nblocks, const double* measure,
                                   const double* tau, int32_t force_dc, int32_t transitions,
                                   uint8_t* states, uint8_t* chi, int32_t* list, int32_t* count,
                                   void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SPDBA_H */
