// State preparation of sp-DBA on the device: per-block activity (FP64 norms),
// the threshold, block states with transition dilation, the frozen-neighbour
// bits used by the smoothing weight, and the ordered compaction of the
// non-frozen block list (Methods: state preparation; S1.1).
#include <math.h>

#include "blocks.h"

namespace spdba {

spdba_status make_geom(Geom* g, int ndim, const int64_t* dims, const int32_t* block) {
    if (ndim < 1 || ndim > 3 || !dims || !block) return fail(SPDBA_ERR_ARG, "bad geometry arguments");
    Geom r;
    r.ndim = ndim;
    int off = 3 - ndim;
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] < 1 || block[a] < 1) return fail(SPDBA_ERR_ARG, "non-positive extent");
        if (dims[a] % block[a] != 0)
            return fail(SPDBA_ERR_UNSUPPORTED, "block edge %d does not divide %lld", block[a], (long long)dims[a]);
        r.n[off + a] = dims[a];
        r.b[off + a] = block[a];
        r.nb[off + a] = dims[a] / block[a];
    }
    *g = r;
    return SPDBA_OK;
}

spdba_status make_geom_batched(Geom* g, int ndim, const int64_t* dims, const int32_t* block, long long batch) {
    spdba_status s = make_geom(g, ndim, dims, block);
    if (s != SPDBA_OK) return s;
    if (batch < 1 || (batch > 1 && ndim > 2)) return fail(SPDBA_ERR_ARG, "batched geometry needs ndim <= 2");
    int ax = 2 - ndim;   // the padded axis just above the field's axes
    g->n[ax] = batch;
    g->nb[ax] = batch;
    return SPDBA_OK;
}

// ------------------------------------------------------------------ activity
// One warp per block.  The block max of |q|^2 is exact in FP64: an FP32 screen
// selects the few modes that can hold the max, and only those are evaluated
// exactly (re*re + im*im in FP64, the oracle's formula), so a mode that is
// skipped cannot be the max.  Non-negative doubles order like their bit
// patterns, so the warp max is two 32-bit integer reductions (high word, then
// low word among the lanes holding the high maximum) and costs no FP64
// instruction.  The ENERGY sum is accumulated per lane in FP64.
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    unsigned hi = (unsigned)(v >> 32), lo = (unsigned)v;
    unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
    unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
    return ((unsigned long long)mhi << 32) | mlo;
}
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

// The screen.  Any partition of a block's modes gives the block's exact max
// when every part yields its own exact max; a part is one lane's modes.  The
// lane keeps the running max S of p = fma(re, re, im * im) over its modes and
// evaluates exactly only the modes with p >= (1 - 2^-20) S, S taken after each
// chunk of modes has been folded in.  Below the FP32 overflow threshold,
// |p - |q|^2| <= 2^-23 |q|^2 + 2^-148, so the part's largest |q|^2 has
// p >= (1 - 2^-20) S whenever S >= 2^-99 (S bounds every p of the part, taken
// before or after it); below 2^-99 every nonzero mode is evaluated, and
// exactly-zero modes never need it.  The running max rises in few chunks, so
// about one mode in a chunk reaches the slow FP64 pipe; the rest costs two
// FP32 operations and a compare, and nothing crosses lanes until the end.  The
// field's k = 0 mode is kept out of the screen and taken apart, so that the
// max over k != 0 is exact as well.
__device__ __forceinline__ float screen_sq(float2 q) { return fmaf(q.x, q.x, q.y * q.y); }
constexpr float kScreen99 = 1.5777218104420236e-30f;   // 2^-99
__device__ __forceinline__ bool nonzero_mode(float2 v) {
    return ((__float_as_uint(v.x) | __float_as_uint(v.y)) << 1) != 0u;
}

template <typename T, bool ENERGY>
__global__ void __launch_bounds__(256) block_activity_kernel(Geom g, const cx_t<T>* __restrict__ q,
                                                             double* __restrict__ maxsq, double* __restrict__ sumsq,
                                                             double* __restrict__ gmax) {
    const int lane = threadIdx.x & 31;
    const long long blk = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (blk >= g.blocks()) return;   // whole warps leave together
    const long long b2 = blk % g.nb[2], b1 = (blk / g.nb[2]) % g.nb[1], b0 = blk / (g.nb[2] * g.nb[1]);
    const int B0 = g.b[0], B1 = g.b[1], B2 = g.b[2];
    const long long run = blk / g.bpr();
    const long long dc = run * g.fmodes();   // the field's k = 0 mode
    const long long base = ((b0 * B0) * g.n[1] + b1 * B1) * g.n[2] + b2 * B2;
    double mx = 0.0, mxnd = 0.0, sm = 0.0;
    if constexpr (sizeof(cx_t<T>) == 8) {
        // chunks of up to 16 modes per lane, as 8 16-byte loads of mode pairs along
        // the fast axis (B2 is even for every supported block), all issued before
        // use; the per-lane running screen of block_activity_rows_kernel (each
        // lane's modes are one part of the block), exact FP64 for its candidates
        const int H = B2 >> 1;
        const int npair = B0 * B1 * H;
        constexpr int K2 = 8;
        float S = 0.f;
        double Ddc = 0.0;   // |q(k = 0)|^2: pair 0 of the block holding it (lane 0)
        if (lane == 0 && base == dc) Ddc = mode_sq(q[dc]);
        for (int m0 = 0; m0 < npair; m0 += 32 * K2) {
            float4 w[K2];
            bool isdc[K2];
#pragma unroll
            for (int k = 0; k < K2; ++k) {
                const int m = m0 + k * 32 + lane;
                w[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                isdc[k] = false;
                if (m < npair) {
                    const int row = m / H, l2 = (m - row * H) * 2;
                    const int l1 = row % B1, l0 = row / B1;
                    const long long idx = base + ((long long)l0 * g.n[1] + l1) * g.n[2] + l2;
                    isdc[k] = idx == dc;
                    w[k] = *reinterpret_cast<const float4*>(q + idx);
                }
            }
            float2 v[2 * K2];
            float p32[2 * K2];
#pragma unroll
            for (int k = 0; k < K2; ++k) {
                v[2 * k] = make_float2(w[k].x, w[k].y);
                v[2 * k + 1] = make_float2(w[k].z, w[k].w);
                if (ENERGY) {
                    sm += mode_sq(v[2 * k]);
                    sm += mode_sq(v[2 * k + 1]);
                }
                if (isdc[k]) v[2 * k] = make_float2(0.f, 0.f);   // k = 0: out of the screen
            }
            float cm = S;
#pragma unroll
            for (int k = 0; k < 2 * K2; ++k) {
                p32[k] = screen_sq(v[k]);
                cm = fmaxf(cm, p32[k]);
            }
            S = cm;
            const float cut = S >= kScreen99 ? S * (1.0f - 9.5367431640625e-07f) : 0.f;
            unsigned mask = 0;
#pragma unroll
            for (int k = 0; k < 2 * K2; ++k)
                if (p32[k] >= cut && nonzero_mode(v[k])) mask |= 1u << k;   // exact zeros cannot raise the max
            while (mask) {
                const int i = __ffs(mask) - 1;
                mask &= mask - 1;
                float2 c = v[0];
#pragma unroll
                for (int k = 1; k < 2 * K2; ++k)
                    if (i == k) c = v[k];
                mxnd = fmax(mxnd, mode_sq(c));
            }
        }
        mx = fmax(mxnd, Ddc);
    } else {
        const int nmodes = B0 * B1 * B2;
        for (int m = lane; m < nmodes; m += 32) {
            int l2 = m % B2, r = m / B2;
            int l1 = r % B1, l0 = r / B1;
            long long idx = base + ((long long)l0 * g.n[1] + l1) * g.n[2] + l2;
            double e = mode_sq(q[idx]);
            if (ENERGY) sm += e;
            mx = fmax(mx, e);
            if (idx != dc) mxnd = fmax(mxnd, e);
        }
    }
    mx = bitsd(warp_max_u64(dbits(mx)));
    mxnd = bitsd(warp_max_u64(dbits(mxnd)));
    if (ENERGY) sm = warp_sum(sm);
    if (lane == 0) {
        maxsq[blk] = mx;
        if (ENERGY) sumsq[blk] = sm;
        atomic_max_nonneg(&gmax[2 * run], mx);
        atomic_max_nonneg(&gmax[2 * run + 1], mxnd);
    }
}

// complex64 fields whose rows are short (n2 / 2 <= 256 mode pairs): one CTA
// per row of blocks (b0, b1), reading its B0 * B1 whole rows of n2 modes in
// order (full-row 16-byte loads, the layout HBM streams best).  A thread keeps
// one mode pair column 2u, so it stays in one block bx = 2u / B2 throughout;
// its modes are one part of the block for the screen above.  The G = B2 / 2
// lanes of a block and the row groups combine at the end.
constexpr int ROWACT_NT = 256;
__global__ void __launch_bounds__(ROWACT_NT) block_activity_rows_kernel(Geom g, const float2* __restrict__ q,
                                                                         double* __restrict__ maxsq,
                                                                         double* __restrict__ gmax) {
    __shared__ unsigned long long s_mx[ROWACT_NT], s_mxnd[ROWACT_NT];
    const int n2 = (int)g.n[2], half = n2 >> 1;          // mode pairs per row
    const int rpi = ROWACT_NT / half;                      // rows per iteration (threads beyond rpi rows idle)
    const int u = threadIdx.x % half, rho = threadIdx.x / half;
    const int b0 = blockIdx.x / (int)g.nb[1], b1 = blockIdx.x - b0 * (int)g.nb[1];
    const int B0 = g.b[0], B1 = g.b[1], B2 = g.b[2];
    const int G = B2 >> 1;                                 // lanes per block (a power of two <= 32)
    const int rows = B0 * B1;
    const long long bpr = g.bpr();
    const long long blk0 = ((long long)b0 * g.nb[1] + b1) * g.nb[2];   // block id of bx = 0
    const long long run = blk0 / bpr;
    const long long dc = run * g.fmodes();
    const long long rowbase = ((long long)b0 * B0 * g.n[1] + (long long)b1 * B1) * n2 + 2 * u;
    float S = 0.f;        // running screen max of this lane's modes (k = 0 left out)
    double D = 0.0;       // exact max of this lane's k != 0 modes
    double Ddc = 0.0;     // |q(k = 0)|^2, in the lane that holds it (row 0, pair 0)
    if (rho == 0 && rowbase == dc) Ddc = mode_sq(q[dc]);
    constexpr int U = 8;
    for (int r0 = rho; rho < rpi && r0 < rows; r0 += U * rpi) {
        float4 w[U];
        bool isdc[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int r = r0 + k * rpi;
            w[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            isdc[k] = false;
            if (r < rows) {
                const int l0 = r / B1, l1 = r - l0 * B1;
                const long long idx = rowbase + ((long long)l0 * g.n[1] + l1) * n2;
                isdc[k] = idx == dc;
                w[k] = *reinterpret_cast<const float4*>(q + idx);
            }
        }
        float2 v[2 * U];
        float p[2 * U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            // the first mode of a pair may be k = 0: out of the screen (no FP64 here,
            // so none is evaluated speculatively)
            v[2 * k] = isdc[k] ? make_float2(0.f, 0.f) : make_float2(w[k].x, w[k].y);
            v[2 * k + 1] = make_float2(w[k].z, w[k].w);
        }
        float cm = S;
#pragma unroll
        for (int k = 0; k < 2 * U; ++k) {
            p[k] = screen_sq(v[k]);
            cm = fmaxf(cm, p[k]);
        }
        S = cm;
        const float cut = S >= kScreen99 ? S * (1.0f - 9.5367431640625e-07f) : 0.f;
        unsigned mask = 0;
#pragma unroll
        for (int k = 0; k < 2 * U; ++k)
            if (p[k] >= cut && nonzero_mode(v[k])) mask |= 1u << k;   // exact zeros (padding) cannot raise the max
        while (mask) {
            const int i = __ffs(mask) - 1;
            mask &= mask - 1;
            // select v[i] by compares (a dynamic index would move v to local memory)
            float2 c = v[0];
#pragma unroll
            for (int k = 1; k < 2 * U; ++k)
                if (i == k) c = v[k];
            D = fmax(D, mode_sq(c));
        }
    }
    // combine the G lanes of one block (aligned lane groups), then the row groups
    unsigned long long bm = dbits(fmax(D, Ddc)), bmnd = dbits(D);
    for (int o = G >> 1; o > 0; o >>= 1) {
        const unsigned long long om = __shfl_xor_sync(0xffffffffu, bm, o);
        const unsigned long long omnd = __shfl_xor_sync(0xffffffffu, bmnd, o);
        bm = om > bm ? om : bm;
        bmnd = omnd > bmnd ? omnd : bmnd;
    }
    s_mx[threadIdx.x] = bm;
    s_mxnd[threadIdx.x] = bmnd;
    __syncthreads();
    const int nbx = n2 / B2;
    if (threadIdx.x < nbx) {
        const int ul = threadIdx.x * G;   // first pair column of block bx
        unsigned long long a = 0, b = 0;
        for (int rr = 0; rr < rpi && rr < rows; ++rr) {
            a = s_mx[rr * half + ul] > a ? s_mx[rr * half + ul] : a;
            b = s_mxnd[rr * half + ul] > b ? s_mxnd[rr * half + ul] : b;
        }
        maxsq[blk0 + threadIdx.x] = bitsd(a);
        atomic_max_nonneg(&gmax[2 * run], bitsd(a));
        atomic_max_nonneg(&gmax[2 * run + 1], bitsd(b));
    }
}

static bool rows_kernel_fits(const Geom& g) {
    const long long n2 = g.n[2];
    if (n2 % 2 != 0 || n2 / 2 > ROWACT_NT) return false;
    const int B2 = g.b[2];
    if (B2 % 2 != 0) return false;
    const int G = B2 / 2;                                   // lanes per block
    if (G > 32 || (G & (G - 1)) != 0) return false;
    // one CTA per row of blocks: only where that gives a few waves of CTAs
    if (g.nb[0] * g.nb[1] < 608 || g.nb[0] * g.nb[1] >= 0x7fffffffLL) return false;
    return true;
}

template <typename T>
spdba_status launch_block_activity(const Geom& g, const cx_t<T>* q, double* maxsq, double* sumsq, double* gmax,
                                   cudaStream_t st) {
    long long nb = g.blocks();
    if constexpr (sizeof(cx_t<T>) == 8) {
        if (!sumsq && rows_kernel_fits(g)) {
            block_activity_rows_kernel<<<(unsigned)(g.nb[0] * g.nb[1]), ROWACT_NT, 0, st>>>(
                g, reinterpret_cast<const float2*>(q), maxsq, gmax);
            SPDBA_CUDA(cudaGetLastError());
            return SPDBA_OK;
        }
    }
    unsigned grid = (unsigned)((nb + 7) / 8);
    if (sumsq) block_activity_kernel<T, true><<<grid, 256, 0, st>>>(g, q, maxsq, sumsq, gmax);
    else block_activity_kernel<T, false><<<grid, 256, 0, st>>>(g, q, maxsq, nullptr, gmax);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}
template spdba_status launch_block_activity<float>(const Geom&, const float2*, double*, double*, double*,
                                                   cudaStream_t);
template spdba_status launch_block_activity<double>(const Geom&, const double2*, double*, double*, double*,
                                                    cudaStream_t);

// ------------------------------------------------------------------ threshold
__global__ void tau_kernel(const double* gmax, int nruns, double threshold, int tau_rule, int exclude_dc,
                           double* tau, DevStats* stats) {
    for (int r = threadIdx.x; r < nruns; r += blockDim.x) {
        double amax = sqrt(gmax[2 * r + (exclude_dc ? 1 : 0)]);
        double t = tau_rule == SPDBA_TAU_ABS ? threshold : threshold * amax;
        tau[r] = t;
        if (stats) {
            stats[r].tau = t;
            stats[r].max_amp = amax;
        }
    }
}

spdba_status launch_tau(const double* gmax, int nruns, double threshold, int tau_rule, int exclude_dc, double* tau,
                        DevStats* stats, cudaStream_t st) {
    tau_kernel<<<1, 256, 0, st>>>(gmax, nruns, threshold, tau_rule, exclude_dc, tau, stats);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

// ------------------------------------------------------------------ states
constexpr int CLS_NT = 1024;

// Block coordinates (32-bit: block maps hold fewer than 2^31 blocks).
struct BCoord {
    int c[3];
};
__device__ __forceinline__ BCoord bcoord(const Geom& g, int b) {
    const int n2 = (int)g.nb[2], n1 = (int)g.nb[1];
    BCoord r;
    const int q = b / n2;
    r.c[2] = b - q * n2;
    r.c[0] = q / n1;
    r.c[1] = q - r.c[0] * n1;
    return r;
}
__device__ __forceinline__ int bindex(const Geom& g, const BCoord& c) {
    return (c.c[0] * (int)g.nb[1] + c.c[1]) * (int)g.nb[2] + c.c[2];
}
// The block across the face of c along `axis` (dir -1 / +1): periodic wrap of
// the block index; on a half map (g.hx > 0) the x neighbour left of kx = 0 or
// right of the Nyquist block lies in the omitted half and is replaced by its
// conjugate counterpart, X(-k) = conj X(k) (S1.2, Eq. S.4): the other field
// axes' block indices mirrored (b -> nb - 1 - b), x-block 0 (across kx = 0,
// the symmetry boundary) or hx - 2 (whose modes are the conjugates of those
// right of kx = N/2).
__device__ __forceinline__ void mirror_other_axes(const Geom& g, BCoord& c) {
    for (int a = 3 - g.ndim; a < 2; ++a) c.c[a] = (int)g.nb[a] - 1 - c.c[a];
}
__device__ __forceinline__ BCoord bnbr(const Geom& g, BCoord c, int axis, int dir) {
    if (axis == 2 && g.hx > 0) {
        const int v = c.c[2] + dir;
        if (v >= 0 && v < g.hx) {
            c.c[2] = v;
        } else {
            mirror_other_axes(g, c);
            c.c[2] = v < 0 ? 0 : g.hx - 2;
        }
        return c;
    }
    const int n = (int)g.nb[axis];
    int v = c.c[axis] + dir;
    v = v < 0 ? v + n : (v >= n ? v - n : v);
    c.c[axis] = v;
    return c;
}

// ACTIVE iff the block's measure meets tau (>=), or forced.
// ACTIVE iff measure >= tau, with tau formed from the scan's maxima (tau_kernel's
// rule) by every thread; the first block of each run records tau and resets the
// run's counts (what tau_kernel and zero_counts_kernel do as separate launches).
__global__ void active_tau_kernel(Geom g, const double* __restrict__ msq, int msq_is_square, const double* gmax,
                                  double threshold, int tau_rule, int exclude_dc, int force_dc, double* tau,
                                  DevStats* stats, uint8_t* __restrict__ active) {
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long nb = g.blocks();
    if (b >= nb) return;
    const long long run = b / g.bpr();
    const double amax = sqrt(gmax[2 * run + (exclude_dc ? 1 : 0)]);
    // the run's coefficient in force (dynamic threshold control moves it)
    const double eps = stats ? stats[run].eps : threshold;
    const double t = tau_rule == SPDBA_TAU_ABS ? eps : eps * amax;
    double m = msq_is_square ? sqrt(msq[b]) : msq[b];
    bool a = (force_dc && b == run * g.bpr()) || (m >= t);
    active[b] = a ? 1 : 0;
    if (b == run * g.bpr()) {
        tau[run] = t;
        if (stats) {
            stats[run].tau = t;
            stats[run].max_amp = amax;
            stats[run].n_active = 0;
            stats[run].n_transition = 0;
            stats[run].assessments += 1;
        }
    }
}

__global__ void active_kernel(Geom g, const double* __restrict__ msq, int msq_is_square, const double* tau,
                              int force_dc, int all_active, uint8_t* __restrict__ active) {
    long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long nb = g.blocks();
    if (b >= nb) return;
    double m = msq_is_square ? sqrt(msq[b]) : msq[b];
    const long long run = b / g.bpr();
    bool a = all_active || (force_dc && b == run * g.bpr()) || (m >= tau[run]);
    active[b] = a ? 1 : 0;
}

// The face neighbours' flags are ORed without short-circuit, so that their
// loads are independent and in flight together (a chain of dependent loads per
// neighbour made the state kernel latency-bound).
//
// An ACTIVE block requests activation of the block across each of its faces
// (bnbr); c is TRANSITION when one of them requests it.  On a periodic map
// these are c's own face neighbours.  On a half map the x sources of a live
// block are: x - 1, or across kx = 0 its mirrored partner in x-block 0; x + 1
// below the Nyquist block (the Nyquist block's request goes to its conjugate
// counterpart instead); and, for x-block hx - 2, the mirrored Nyquist block,
// whose request past kx = N/2 lands there.
__device__ __forceinline__ bool has_active_nbr(const Geom& g, const uint8_t* active, const BCoord& c) {
    const int a0 = 3 - g.ndim;
    unsigned any = 0;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        if (ax < a0) continue;
        any |= active[bindex(g, bnbr(g, c, ax, -1))] | active[bindex(g, bnbr(g, c, ax, +1))];
    }
    if (g.hx > 0) {
        const int x = c.c[2];
        BCoord s = c;
        if (x > 0) {
            s.c[2] = x - 1;
        } else {
            mirror_other_axes(g, s);
            s.c[2] = 0;
        }
        any |= active[bindex(g, s)];
        if (x < g.hx - 1) {
            s = c;
            s.c[2] = x + 1;
            any |= active[bindex(g, s)];
        }
        if (x == g.hx - 2) {
            s = c;
            mirror_other_axes(g, s);
            s.c[2] = g.hx - 1;
            any |= active[bindex(g, s)];
        }
    } else {
        any |= active[bindex(g, bnbr(g, c, 2, -1))] | active[bindex(g, bnbr(g, c, 2, +1))];
    }
    return any != 0;
}

// TRANSITION iff not active and a face neighbour (periodic) is active; chi bit
// 2a / 2a+1 marks a FROZEN lower / upper neighbour along local axis a (axis 0
// = slowest axis of the field).  One CTA-sized count per CTA goes to scratch.
__global__ void __launch_bounds__(CLS_NT) state_kernel(Geom g, const uint8_t* __restrict__ active, int transitions,
                                                       uint8_t* __restrict__ states, uint8_t* __restrict__ chi,
                                                       int* __restrict__ cta_count, DevStats* stats,
                                                       double* gmax_reset, int nruns) {
    long long b = (long long)blockIdx.x * CLS_NT + threadIdx.x;
    long long nb = g.blocks();
    // the activity maxima were consumed by the previous kernel: zero them for the next scan
    if (gmax_reset != nullptr && blockIdx.x == 0)
        for (int r = threadIdx.x; r < 2 * nruns; r += CLS_NT) gmax_reset[r] = 0.0;
    int st = 0;
    uint8_t cb = 0;
    if (b < nb) {
        const BCoord c = bcoord(g, (int)b);
        const bool nbr_active = transitions && has_active_nbr(g, active, c);
        if (active[b]) st = SPDBA_ACTIVE;
        else if (nbr_active) st = SPDBA_TRANSITION;
        const int a0 = 3 - g.ndim;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            if (ax < a0) continue;
#pragma unroll
            for (int d = 0; d < 2; ++d) {
                const BCoord cn = bnbr(g, c, ax, d == 0 ? -1 : +1);
                // both loads issued unconditionally (transitions is uniform)
                const unsigned act_n = active[bindex(g, cn)];
                const bool nbr_n = transitions && has_active_nbr(g, active, cn);
                const bool frozen = act_n == 0 && !nbr_n;
                if (frozen) cb |= (uint8_t)(1u << (2 * (ax - a0) + d));
            }
        }
        if (g.hx > 0 && c.c[2] >= g.hx) st = 0, cb = 0;   // padding x-blocks of a half map
        states[b] = (uint8_t)st;
        chi[b] = cb;
    }
    unsigned nf = __ballot_sync(0xffffffffu, st != 0);
    unsigned na = __ballot_sync(0xffffffffu, st == SPDBA_ACTIVE);
    unsigned nt = __ballot_sync(0xffffffffu, st == SPDBA_TRANSITION);
    __shared__ int s_nf, s_na, s_nt;
    if (threadIdx.x == 0) s_nf = s_na = s_nt = 0;
    __syncthreads();
    const long long bpr = g.bpr();
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_nf, __popc(nf));
    if (stats) {
        // per-run counts: one atomic per CTA when a CTA never straddles runs (the
        // counters of a run are one address: per-warp atomics would queue on it),
        // else one per warp when a warp never straddles runs
        if (bpr % CLS_NT == 0) {
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(&s_na, __popc(na));
                atomicAdd(&s_nt, __popc(nt));
            }
            __syncthreads();
            const long long b0 = (long long)blockIdx.x * CLS_NT;
            if (threadIdx.x == 0 && b0 < nb) {
                const long long run = b0 / bpr;
                if (s_na) atomicAdd(&stats[run].n_active, (unsigned long long)s_na);
                if (s_nt) atomicAdd(&stats[run].n_transition, (unsigned long long)s_nt);
            }
        } else if (bpr % 32 == 0) {
            if ((threadIdx.x & 31) == 0 && b < nb) {
                long long run = b / bpr;
                if (na) atomicAdd(&stats[run].n_active, (unsigned long long)__popc(na));
                if (nt) atomicAdd(&stats[run].n_transition, (unsigned long long)__popc(nt));
            }
        } else if (b < nb) {
            long long run = b / bpr;
            if (st == SPDBA_ACTIVE) atomicAdd(&stats[run].n_active, 1ull);
            if (st == SPDBA_TRANSITION) atomicAdd(&stats[run].n_transition, 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) cta_count[blockIdx.x] = s_nf;
}

// Ordered compaction: CTA c starts at the sum of the counts of CTAs before it
// and places its non-frozen ids with a warp-ballot prefix and a block scan.
__global__ void __launch_bounds__(CLS_NT) compact_kernel(Geom g, const uint8_t* __restrict__ states,
                                                         const int* __restrict__ cta_count, int ncta,
                                                         int32_t* __restrict__ list, int32_t* __restrict__ count) {
    __shared__ int s_base;
    __shared__ int s_warp[CLS_NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w == 0) {
        int acc = 0;
        for (int c = lane; c < (int)blockIdx.x; c += 32) acc += cta_count[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_base = acc;
    }
    long long b = (long long)blockIdx.x * CLS_NT + threadIdx.x;
    bool keep = b < g.blocks() && states[b] != 0;
    unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_warp[w] = __popc(m);
    __syncthreads();
    if (w == 0) {
        int v = lane < CLS_NT / 32 ? s_warp[lane] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane < CLS_NT / 32) s_warp[lane] = incl - v;
        if (blockIdx.x == (unsigned)(ncta - 1) && lane == 31) *count = s_base + incl;
    }
    __syncthreads();
    if (keep) {
        int pos = s_base + s_warp[w] + __popc(m & ((1u << lane) - 1u));
        list[pos] = (int32_t)b;
    }
}

__global__ void zero_counts_kernel(DevStats* stats, long long nruns) {
    for (long long r = threadIdx.x; r < nruns; r += blockDim.x) {
        stats[r].n_active = 0;
        stats[r].n_transition = 0;
        stats[r].assessments += 1;
    }
}

size_t classify_scratch_bytes(long long nb) { return sizeof(int) * (size_t)((nb + CLS_NT - 1) / CLS_NT); }

spdba_status launch_classify(const Geom& g, const double* msq, int msq_is_square, const double* tau, int force_dc,
                             int transitions, int all_active, uint8_t* active, uint8_t* states, uint8_t* chi,
                             int32_t* list, int32_t* count, void* scratch, DevStats* stats, cudaStream_t st) {
    long long nb = g.blocks();
    int ncta = (int)((nb + CLS_NT - 1) / CLS_NT);
    if (stats) zero_counts_kernel<<<1, 256, 0, st>>>(stats, g.runs());
    active_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(g, msq, msq_is_square, tau, force_dc, all_active,
                                                                 active);
    state_kernel<<<ncta, CLS_NT, 0, st>>>(g, active, transitions, states, chi, (int*)scratch, stats, nullptr, 0);
    compact_kernel<<<ncta, CLS_NT, 0, st>>>(g, states, (const int*)scratch, ncta, list, count);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

spdba_status launch_classify_from_scan(const Geom& g, const double* msq, int msq_is_square, double* gmax,
                                       double threshold, int tau_rule, int exclude_dc, int force_dc, int transitions,
                                       double* tau, uint8_t* active, uint8_t* states, uint8_t* chi, int32_t* list,
                                       int32_t* count, void* scratch, DevStats* stats, cudaStream_t st) {
    long long nb = g.blocks();
    int ncta = (int)((nb + CLS_NT - 1) / CLS_NT);
    active_tau_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(g, msq, msq_is_square, gmax, threshold, tau_rule,
                                                                      exclude_dc, force_dc, tau, stats, active);
    state_kernel<<<ncta, CLS_NT, 0, st>>>(g, active, transitions, states, chi, (int*)scratch, stats, gmax,
                                          (int)g.runs());
    compact_kernel<<<ncta, CLS_NT, 0, st>>>(g, states, (const int*)scratch, ncta, list, count);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

}  // namespace spdba

// ------------------------------------------------------------------ C ABI
using namespace spdba;

extern "C" spdba_status spdba_block_activity(int32_t precision, int32_t ndim, const int64_t* dims,
                                             const int32_t* block, const void* q, double* maxsq, double* sumsq,
                                             double* gmax, void* stream) {
    if (!q || !maxsq || !gmax) return fail(SPDBA_ERR_ARG, "spdba_block_activity: NULL buffer");
    Geom g;
    spdba_status s = make_geom(&g, ndim, dims, block);
    if (s != SPDBA_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    SPDBA_CUDA(cudaMemsetAsync(gmax, 0, 2 * sizeof(double), st));
    if (precision == SPDBA_C64) return launch_block_activity<float>(g, (const float2*)q, maxsq, sumsq, gmax, st);
    if (precision == SPDBA_C128) return launch_block_activity<double>(g, (const double2*)q, maxsq, sumsq, gmax, st);
    return fail(SPDBA_ERR_ARG, "bad precision %d", precision);
}

extern "C" size_t spdba_classify_scratch_bytes(int64_t nb) { return classify_scratch_bytes(nb) + (size_t)nb; }

extern "C" spdba_status spdba_classify(int32_t ndim, const int64_t* nblocks, const double* measure,
                                       const double* tau, int32_t force_dc, int32_t transitions, uint8_t* states,
                                       uint8_t* chi, int32_t* list, int32_t* count, void* scratch, void* stream) {
    if (!nblocks || !measure || !tau || !states || !chi || !list || !count || !scratch)
        return fail(SPDBA_ERR_ARG, "spdba_classify: NULL argument");
    int64_t dims[3];
    int32_t one[3] = {1, 1, 1};
    for (int a = 0; a < ndim && a < 3; ++a) dims[a] = nblocks[a];
    Geom g;
    spdba_status s = make_geom(&g, ndim, dims, one);
    if (s != SPDBA_OK) return s;
    // scratch layout: per-CTA counts, then one active flag per block
    size_t cbytes = classify_scratch_bytes(g.blocks());
    uint8_t* active = (uint8_t*)scratch + cbytes;
    return launch_classify(g, measure, 0, tau, force_dc, transitions, 0, active, states, chi, list, count, scratch,
                           nullptr, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ classify without allocation
// Variant of spdba_classify whose scratch (per-CTA counts and one flag per
// block) lives in a fixed array compiled into the library, for callers that
// cannot allocate device memory.  The array is a file-scope __device__
// variable; host code obtains its device address with cudaGetSymbolAddress
// once per device (the name itself is only a host-side stand-in).
#include <mutex>

#define SPDBA_STATIC_SCRATCH_BYTES ((size_t)SPDBA_CLASSIFY_STATIC_MAX_BLOCKS + \
                                    sizeof(int) * (size_t)(SPDBA_CLASSIFY_STATIC_MAX_BLOCKS / 1024))

static __device__ __align__(256) unsigned char g_classify_scratch[SPDBA_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {nullptr};
}  // namespace

// The array's device address on the current device.  Outside stream capture it
// is looked up on every call (a host-side table lookup), so that a context
// torn down and re-created (cudaDeviceReset) never leaves a stale address
// behind; during capture, where the lookup may not be issued, the address
// of the device's last uncaptured call is used.
static spdba_status static_scratch_for_current_device(cudaStream_t st, void** out) {
    int dev = 0;
    SPDBA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(SPDBA_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    SPDBA_CUDA(cudaStreamIsCapturing(st, &cap));
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_classify_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(classify scratch)");
        g_static_ptr[dev] = p;
    } else if (!g_static_ptr[dev]) {
        return fail(SPDBA_ERR_STATE, "spdba_classify_static: first call on device %d made during stream capture", dev);
    }
    *out = g_static_ptr[dev];
    return SPDBA_OK;
}

extern "C" spdba_status spdba_classify_static(int32_t ndim, const int64_t* nblocks, const double* measure,
                                              const double* tau, int32_t force_dc, int32_t transitions,
                                              uint8_t* states, uint8_t* chi, int32_t* list, int32_t* count,
                                              void* stream) {
    if (!nblocks || !measure || !tau || !states || !chi || !list || !count)
        return fail(SPDBA_ERR_ARG, "spdba_classify_static: NULL argument");
    int64_t dims[3];
    int32_t one[3] = {1, 1, 1};
    for (int a = 0; a < ndim && a < 3; ++a) dims[a] = nblocks[a];
    Geom g;
    spdba_status s = make_geom(&g, ndim, dims, one);
    if (s != SPDBA_OK) return s;
    if (g.blocks() > SPDBA_CLASSIFY_STATIC_MAX_BLOCKS)
        return fail(SPDBA_ERR_UNSUPPORTED, "spdba_classify_static: %lld blocks exceed the fixed capacity of %d",
                    g.blocks(), SPDBA_CLASSIFY_STATIC_MAX_BLOCKS);
    void* scratch = nullptr;
    if ((s = static_scratch_for_current_device((cudaStream_t)stream, &scratch)) != SPDBA_OK) return s;
    // layout as in spdba_classify: per-CTA counts first, then one flag per block;
    // every byte a call reads is written earlier in the same call
    size_t cbytes = classify_scratch_bytes(g.blocks());
    uint8_t* active = (uint8_t*)scratch + cbytes;
    return launch_classify(g, measure, 0, tau, force_dc, transitions, 0, active, states, chi, list, count, scratch,
                           nullptr, (cudaStream_t)stream);
}
