// sp-DBA plan: owns the device buffers of one or more runs and drives the time
// loop of the paper's solver integration (S2.1): per step the pre-update
// (model terms and transforms), the update dispatched by mode (Regular: every
// mode; sp-DBA: state preparation at each reassessment, then the blockwise
// update of the non-frozen blocks), and the post-update transforms.
//
// Runs of equal size are stored contiguously as one "group" and step together
// with one launch per kernel per group: the batched form of an ensemble of
// Cahn-Hilliard fields or of a set of NLS signals.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <memory>
#include <vector>

#include "blocks.h"
#include "nls.h"
#include "rcd.h"

namespace spdba {

// ------------------------------------------------------------------ small kernels
template <typename T> __global__ void real_to_complex_kernel(const T* __restrict__ r, cx_t<T>* __restrict__ c, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c[i] = mk<cx_t<T>>(r[i], (T)0);
}
// Full spectrum (N0 x N1 x N2) of a half-stored one (kx = 0 .. N2/2 in rows of
// NHP entries): kx > N2/2 from X(k) = conj X(-k) (Eq. S.4).
template <typename T>
__global__ void half_storage_extend_kernel(const cx_t<T>* __restrict__ h, cx_t<T>* __restrict__ full, int N0, int N1,
                                           int N2, int NHP) {
    const long long n = (long long)N0 * N1 * N2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % N2);
        const long long zy = i / N2;
        const int y = (int)(zy % N1), z = (int)(zy / N1);
        cx_t<T> v;
        if (x <= N2 / 2) {
            v = h[zy * NHP + x];
        } else {
            const int my = y == 0 ? 0 : N1 - y, mz = z == 0 ? 0 : N0 - z;
            v = h[((long long)mz * N1 + my) * NHP + (N2 - x)];
            v.y = -v.y;
        }
        full[i] = v;
    }
}

template <typename T> __global__ void complex_real_part_kernel(const cx_t<T>* __restrict__ c, T* __restrict__ r, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        r[i] = c[i].x;
}
__global__ void zero_strided_kernel(double* p, long long n, int stride) {
    for (long long i = threadIdx.x; i < n; i += blockDim.x) p[i * stride] = 0.0;
}
// per-run share of non-frozen blocks for one step (1 on all-active steps)
__global__ void ratio_kernel(DevStats* stats, long long nruns, long long bpr, long long bmodes, int dense) {
    for (long long r = threadIdx.x; r < nruns; r += blockDim.x) {
        double nf = dense ? (double)bpr : (double)(stats[r].n_active + stats[r].n_transition);
        stats[r].ratio_sum += nf / (double)bpr;
        if (!dense) {
            stats[r].list_modes += nf * (double)bmodes;
            stats[r].ctl_nf += stats[r].n_active + stats[r].n_transition;   // control interval
            stats[r].ctl_steps += 1;
        }
    }
}
// Statistics of runs [0, n) reset, with the threshold coefficient in force set to eps.
__global__ void stats_reset_kernel(DevStats* stats, long long n, double eps) {
    for (long long r = threadIdx.x; r < n; r += blockDim.x) {
        stats[r] = DevStats{};
        stats[r].eps = eps;
    }
}

// Dynamic threshold control (S1.3): with q = r / r_tar the coefficient is
// doubled (q > 2) or halved (q < 0.5), else scaled by 1 + eta or 1 - eta
// outside the relative deadband, else kept.
__device__ __forceinline__ double control_decision(double eps, double r, double r_tar, double eta) {
    const double q = r / r_tar;
    if (q > 2.0) return eps * 2.0;
    if (q < 0.5) return eps * 0.5;
    if (q > 1.0 + eta) return eps * (1.0 + eta);
    if (q < 1.0 - eta) return eps * (1.0 - eta);
    return eps;
}
// One decision per run from the control interval's mean non-frozen share
// r = ctl_nf / (ctl_steps * blocks per run) (exact integer counts, one
// rounding in the quotient); the interval restarts.  Runs without an adaptive
// step in the interval keep their coefficient.
__global__ void control_kernel(DevStats* stats, long long nruns, long long bpr, double r_tar, double eta) {
    for (long long r = threadIdx.x; r < nruns; r += blockDim.x) {
        DevStats& s = stats[r];
        if (s.ctl_steps == 0) continue;
        const double ratio = (double)s.ctl_nf / ((double)s.ctl_steps * (double)bpr);
        s.eps = control_decision(s.eps, ratio, r_tar, eta);
        s.ctl_nf = 0;
        s.ctl_steps = 0;
        s.controls += 1;
    }
}

static unsigned grid_for(long long n, int nt) {
    long long g = (n + nt - 1) / nt;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// ------------------------------------------------------------------ one group of equal runs
template <typename T> struct Group {
    using C = cx_t<T>;
    Geom g;                 // block geometry of the group (runs stacked on a padded axis)
    Geom gT;                // long NLS signals: block geometry in the transposed storage order
    int ndim = 0;
    int64_t dims[3] = {1, 1, 1};
    long long batch = 1;
    long long n = 0;        // modes per run
    bool long_nls = false;
    long long n1 = 0;
    C* c_hat = nullptr;     // transformed fields (the solver state), batch * n
    C* work = nullptr;      // transform workspace, batch * n
    T* real = nullptr;      // real-space staging of one run (CH)
    double* maxsq = nullptr;
    double* sumsq = nullptr;
    double* gmax = nullptr; // 2 per run
    double* tau = nullptr;  // 1 per run
    uint8_t* active = nullptr;
    uint8_t* states = nullptr;
    uint8_t* chi = nullptr;
    int32_t* list = nullptr;
    int32_t* count = nullptr;
    void* scratch = nullptr;
    DevStats* stats = nullptr;  // 1 per run
    // CH
    T* k2ax[3] = {nullptr, nullptr, nullptr};
    T* taper[3] = {nullptr, nullptr, nullptr};
    std::vector<Pass<T>> pre_inv;   // inverse passes before the fused one (first reads c_hat)
    Pass<T> fused;                  // inverse + nonlinearity + forward along the fast axis
    std::vector<Pass<T>> pre_fwd;   // remaining forward passes
    // Hermitian half-spectrum form (3-D complex64): the transforms between c_hat
    // and the update run on x frequencies 0 .. N2/2 in `half`
    bool use_half = false;          // in use (has_half: passes built)
    bool has_half = false;
    C* half = nullptr;
    long long half_n = 0;           // elements of the half array
    Pass<T> h_inv_z, h_inv_y, h_nl, h_fwd_y, h_mirror, h_upd;
    int* pair_list = nullptr;       // live tiles of the paired z forward (with block states)
    uint8_t* col_live = nullptr;    // live x-frequency columns of the half array (the y forward skips the rest)
    int* pair_count = nullptr;
    long long pair_list_n = 0;      // capacity of pair_list
    HermTma herm_tma;               // the half form's z inverse with TMA tile copies (complex64)
    bool use_herm_tma = false;
    // Half-spectrum storage (3-D complex64 CH, S1.2): c_hat holds the stored half
    // kx = 0 .. N2/2 of the real field's spectrum in rows of hs_nhp entries (the
    // rest zero), g is the half map (g.hx live x-blocks); the passes run
    // h_inv_z, h_inv_y, h_nl, h_fwd_y and h_upd (fused) or h_mirror (plain z
    // forward) + the staged update, all in `work`
    bool hs = false;
    long long hs_n = 0;             // elements of the stored half (N0 * N1 * hs_nhp)
    int64_t hs_nhp = 0;
    uint8_t* hs_zlive = nullptr;    // live z pencils (N1 * hs_nhp) and x columns (hs_nhp) under the states:
    uint8_t* hs_xlive = nullptr;    // the z and y forward passes skip the rest on adaptive steps
    bool fused_update = false;      // the last forward pass carries the update (upd_pass)
    bool has_fused = false;         // upd_pass exists (else only the staged form)
    Pass<T> upd_pass;               // forward pass of the first axis with the update fused
    FftEngine<T> fft1;              // one run's transforms for set/get_field
    // NLS
    HPair<T>* H = nullptr;
    T* ntaper = nullptr;
    const C* tw_row = nullptr;      // stage twiddles: n (short) or 512 (long rows)
    const C* tw_col = nullptr;      // stage twiddles of n1 (long columns)
    const C* tw4 = nullptr;         // exp(-2 pi i m / n)
    C* tw2 = nullptr;               // exp(-2 pi i a b / n) at a * 512 + b (long NLS signals)
    int B = 1, nblk = 1;
    NLSLaunch nl;                   // NLS launch shapes (fixed at creation)
    // RCD: ncomp components per field, component-major in c_hat, work and real
    long long ncomp = 1;
    T* rcd_V = nullptr;             // eigenvectors of D, row-major V[i * M + j]
    T* rcd_lam = nullptr;           // eigenvalues of D
    FftEngine<T> rcd_fft;           // transforms of the ncomp fields (one batch)
    // TMA form of the list-driven update (3-D complex64, 8^3 blocks): tensor maps of c_hat and work
    alignas(64) unsigned char tma_map_c[128] = {};
    alignas(64) unsigned char tma_map_g[128] = {};
    bool tma_ok = false;            // the TMA kernel exists for this group
    bool use_tma = false;           // ... and is in use (the autotuner's choice)
    long long tma_grid = 0;
    // predictor (3-D CH runs): last exact activity, prediction in force, scratch
    double* snap_maxsq = nullptr;
    double* snap_tau = nullptr;
    double* pmeasure = nullptr;
    double* pthr = nullptr;
    uint8_t* pstates = nullptr;
    void* px = nullptr;
    bool has_snap = false, has_pred = false;
    int64_t step = 0;
    bool assessed = false;
    std::vector<void*> allocs;

    template <typename P> spdba_status alloc(P** p, size_t bytes) {
        void* q = nullptr;
        cudaError_t e = dev_alloc(&q, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "device allocation (plan buffer)");
        allocs.push_back(q);
        *p = (P*)q;
        return SPDBA_OK;
    }
    void release() {
        for (void* p : allocs) dev_free(p);
        allocs.clear();
        fft1.release();
        rcd_fft.release();
    }
};

}  // namespace spdba

using namespace spdba;

enum ProfKind { K_FFT_PASS = 0, K_FUSED_NL, K_UPDATE_DENSE, K_UPDATE_LIST, K_ASSESS, K_NLS_STEP, K_NLS_ROW, K_NLS_COL,
                K_FFT_UPDATE, K_FFT_ZFWD, K_RCD_FFT, K_RCD_REACTION, K_FFT_YFWD, K_PREDICT, K_COUNT };
static const char* kProfName[K_COUNT] = {"fft_pass", "fft_fused_nl", "update_dense", "update_list", "assess",
                                         "nls_step", "nls_row", "nls_col", "fft_update", "fft_z_forward",
                                         "rcd_fft", "rcd_reaction", "fft_y_forward_pruned", "predict"};

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double bytes;
};

struct RunRef {
    int group;
    long long sub;
};

struct RcdParams {
    double r, a, alpha, beta;
};

// One pass phase of the multi-size form: a single launch over every group's tiles.
struct MultiPhase {
    const void* func = nullptr;
    int smem = 0;
    long long grid = 0;
    spdba::MultiGroup<float>* groups = nullptr;   // device array, ng entries
    int ng = 0;
    unsigned total = 0;                           // tiles of all groups
};
// The multi-size form of a batched 2-D complex64 CH plan (one per tile table).
struct MultiForm {
    bool ok = false;
    MultiPhase inv, nl, upd;   // inverse along axis 0; nonlinearity along axis 1; forward + update along axis 0
};

struct spdba_plan {
    spdba_options opt;
    MultiForm multi[2];     // tile tables of 4096 and 2048 elements
    int multi_sel = 0;      // form in force: 0 = per group, 1 / 2 = multi[0] / multi[1]
    std::vector<void*> multi_bufs;   // device buffers of the multi-size forms
    RcdParams rcd{1.0, 1.0, 1.0, 0.3};
    bool prof = false;
    int prof_every = 1;     // record the kernels of one step in `prof_every`
    bool prof_on = false;   // recording the current step
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    long long launches = 0;
    double prof_list_bytes0 = 0;
    long long list_updates = 0;    // list-driven update launches so far (graph replays included)
    long long prof_list0 = 0;      // list_updates when the profile began
    double threshold = 0;
    int reassess = 1;
    int precision = SPDBA_C64;
    cudaStream_t st = 0;
    spdba_status latched = SPDBA_OK;
    std::vector<std::unique_ptr<Group<float>>> g32;
    std::vector<std::unique_ptr<Group<double>>> g64;
    std::vector<RunRef> runs;
    TwiddleCache<float> tw32;
    TwiddleCache<double> tw64;
    cudaGraphExec_t seg_exec = nullptr;   // one reassessment segment (R steps of every group)
    spdba_predictor* pred = nullptr;
    int horizon = 0, judge_every = 0;
    float prob_thr = 0.5f;
    long long seg_launches = 0;
    long long seg_list_updates = 0;   // list-driven updates in one captured segment
    // groups step concurrently on their own streams, forked from and joined to st
    std::vector<cudaStream_t> gstreams;
    std::vector<cudaEvent_t> gevents;
    cudaEvent_t fork_ev = nullptr;
    int nruns() const { return (int)runs.size(); }
};

namespace spdba {

static cudaEvent_t ev_get(spdba_plan* p) {
    if (p->ev_used < p->ev_pool.size()) return p->ev_pool[p->ev_used++];
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    p->ev_pool.push_back(e);
    p->ev_used++;
    return e;
}

// Records a start event now and a stop event when it goes out of scope.
struct ProfScope {
    spdba_plan* p;
    int kind;
    double bytes;
    cudaEvent_t a = nullptr;
    ProfScope(spdba_plan* pp, int k, double by) : p(pp), kind(k), bytes(by) {
        if (p->prof && p->prof_on && (a = ev_get(p)) != nullptr) cudaEventRecord(a, p->st);
    }
    ~ProfScope() {
        if (!a) return;
        cudaEvent_t b = ev_get(p);
        if (!b) return;
        cudaEventRecord(b, p->st);
        p->prof_recs.push_back(ProfRec{kind, a, b, bytes});
    }
};

template <typename T> static std::vector<std::unique_ptr<Group<T>>>& groups(spdba_plan* p);
template <> std::vector<std::unique_ptr<Group<float>>>& groups<float>(spdba_plan* p) { return p->g32; }
template <> std::vector<std::unique_ptr<Group<double>>>& groups<double>(spdba_plan* p) { return p->g64; }
template <typename T> static TwiddleCache<T>& twc(spdba_plan* p);
template <> TwiddleCache<float>& twc<float>(spdba_plan* p) { return p->tw32; }
template <> TwiddleCache<double>& twc<double>(spdba_plan* p) { return p->tw64; }

template <typename T, typename V>
static spdba_status upload(Group<T>& r, V** dst, const std::vector<V>& v, cudaStream_t st) {
    spdba_status s = r.alloc(dst, sizeof(V) * v.size());
    if (s != SPDBA_OK) return s;
    SPDBA_CUDA(cudaMemcpyAsync(*dst, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice, st));
    SPDBA_CUDA(cudaStreamSynchronize(st));   // v is a temporary
    return SPDBA_OK;
}

// H(w) = exp(i beta2 w^2 h / 4) per bin in FP64, split into hi + lo of type T
template <typename T> static std::vector<HPair<T>> half_step_table(long long n, double beta2, double h, double dts) {
    std::vector<HPair<T>> v((size_t)n);
    const double two_pi = 6.283185307179586476925286766559;
    for (long long k = 0; k < n; ++k) {
        long long kk = k <= n / 2 ? k : k - n;
        double w = two_pi * (double)kk / ((double)n * dts);
        double phi = beta2 * w * w * h / 4.0;
        double c = cos(phi), s = sin(phi);
        HPair<T> e;
        e.hi.x = (T)c;
        e.hi.y = (T)s;
        e.lo.x = (T)(c - (double)e.hi.x);
        e.lo.y = (T)(s - (double)e.hi.y);
        v[(size_t)k] = e;
    }
    return v;
}

// Common buffers of a group.
template <typename T> static spdba_status group_buffers(spdba_plan* p, Group<T>& r) {
    cudaStream_t st = p->st;
    spdba_status s;
    const long long nb = r.g.blocks();
    const long long tot = r.batch * r.n * r.ncomp;
    if ((s = r.alloc(&r.c_hat, sizeof(cx_t<T>) * tot)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.work, sizeof(cx_t<T>) * tot)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.real, sizeof(T) * r.n * r.ncomp)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.maxsq, sizeof(double) * nb)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.sumsq, sizeof(double) * nb)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.gmax, sizeof(double) * 2 * r.batch)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.tau, sizeof(double) * r.batch)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.active, nb)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.states, nb)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.chi, nb)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.list, sizeof(int32_t) * nb)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.count, sizeof(int32_t) * 2)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.scratch, classify_scratch_bytes(nb))) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.stats, sizeof(DevStats) * r.batch)) != SPDBA_OK) return s;
    SPDBA_CUDA(cudaMemsetAsync(r.c_hat, 0, sizeof(cx_t<T>) * tot, st));
    stats_reset_kernel<<<1, 256, 0, st>>>(r.stats, r.batch, p->threshold);
    SPDBA_CUDA(cudaGetLastError());
    SPDBA_CUDA(cudaMemsetAsync(r.gmax, 0, sizeof(double) * 2 * r.batch, st));
    SPDBA_CUDA(cudaMemsetAsync(r.states, SPDBA_ACTIVE, nb, st));
    SPDBA_CUDA(cudaMemsetAsync(r.chi, 0, nb, st));
    return SPDBA_OK;
}

// The update's view of a CH group (states, tables, divisors) for the kernels
// that fuse the update or skip frozen blocks.
template <typename T> static void fill_fuse(const spdba_plan* p, const Group<T>& r, CHFuse<T>& f) {
    f.c_hat = r.c_hat;
    for (int ax = 0; ax < 3; ++ax) { f.k2ax[ax] = r.k2ax[ax]; f.taper[ax] = r.taper[ax]; }
    f.states = r.states;
    f.chi = r.chi;
    f.dt = (T)p->opt.dt;
    f.dtkappa = (T)(p->opt.dt * p->opt.kappa);
    f.dense = 1;
    f.stats = r.stats;
    f.g = r.g;
    f.fd_bp.init((uint32_t)(r.g.ndim == 3 ? r.g.b[0] : r.g.b[1]));
    f.fd_b2.init((uint32_t)r.g.b[2]);
    f.fd_b1.init((uint32_t)r.g.b[1]);
    f.fd_n2.init((uint32_t)r.g.n[2]);
}

// Half-spectrum passes of a 3-D complex64 group; SPDBA_ERR_UNSUPPORTED (and
// no change) where the shape has no half-spectrum kernels or gains nothing.
static spdba_status setup_half(spdba_plan* p, Group<float>& r, const int64_t* dims) {
    cudaStream_t st = p->st;
    const int64_t N0 = dims[0], N1 = dims[1], N2 = dims[2];
    if (N2 % 2 != 0 || N0 > 4096 || N1 > 4096 || N2 > 4096) return SPDBA_ERR_UNSUPPORTED;
    const int Py = pass_tile_pencils<float>(N1);
    if (Py == 0) return SPDBA_ERR_UNSUPPORTED;
    const int64_t M = N2 / 2;
    const int64_t NHP = ((M + 1 + Py - 1) / Py) * Py;
    if (4 * NHP > 3 * N2) return SPDBA_ERR_UNSUPPORTED;   // under a quarter saved: keep the full form
    HalfGeo hg;
    hg.N0 = (int)N0; hg.N1 = (int)N1; hg.N2 = (int)N2; hg.NHP = (int)NHP;
    hg.fd_N2.init((uint32_t)N2);
    hg.fd_NHP.init((uint32_t)NHP);
    hg.fd_M.init((uint32_t)M);
    TwiddleCache<float>& tw = p->tw32;
    Pass<float> hz, hy_inv, hnl, hy_fwd, hmir, hupd;
    spdba_status s;
    if ((s = make_half_pass(&hz, PASS_HERM_INV, hg, tw, st)) != SPDBA_OK) return s;
    if ((s = make_half_pass(&hnl, PASS_NL_HALF, hg, tw, st)) != SPDBA_OK) return s;
    // z forward of the staged form: one transform per half pencil for kx and
    // N2 - kx where the paired tiles fit, else one per full pencil (the fused
    // update pass transforms every full pencil: with the update in the same
    // kernel, pairing saved less than it cost)
    const bool paired = make_half_pass(&hmir, PASS_PAIR_MIRROR, hg, tw, st) == SPDBA_OK;
    if (!paired) {
        if ((s = make_half_pass(&hmir, PASS_MIRROR, hg, tw, st)) != SPDBA_OK) return s;
        if (N2 % hmir.P != 0) return SPDBA_ERR_UNSUPPORTED;   // z tiles must stay within one x row
    } else if (r.g.nb[0] * upd_table_cols(hmir.P, r.g.b[2]) <= kPairTable) {
        // the paired pass skips frozen tiles and stores g_hat of non-frozen blocks only
        // (the staged update reads no other); without states it stores everything.
        // Its live tiles are listed at every state setting.
        fill_fuse<float>(p, r, hmir.p.fu);
        r.pair_list_n = pair_tile_count(hmir);
        if ((s = r.alloc(&r.pair_list, sizeof(int) * (size_t)r.pair_list_n)) != SPDBA_OK) return s;
        if ((s = r.alloc(&r.pair_count, sizeof(int))) != SPDBA_OK) return s;
        SPDBA_CUDA(cudaMemsetAsync(r.pair_count, 0, sizeof(int), st));
        hmir.p.live_tiles = r.pair_list;
        hmir.p.live_count = r.pair_count;
        if (r.g.nb[2] <= 64) {
            if ((s = r.alloc(&r.col_live, (size_t)NHP)) != SPDBA_OK) return s;
            SPDBA_CUDA(cudaMemsetAsync(r.col_live, 1, (size_t)NHP, st));
        }
    }
    const int64_t dh[3] = {N0, N1, NHP};
    if ((s = make_axis_pass<float>(&hy_inv, 3, dh, 1, 1, +1, PASS_PLAIN, tw, st)) != SPDBA_OK) return s;
    if ((s = make_axis_pass<float>(&hy_fwd, 3, dh, 1, 1, -1, PASS_PLAIN, tw, st)) != SPDBA_OK) return s;
    if (r.has_fused) {
        if ((s = make_half_pass(&hupd, PASS_UPD_HALF, hg, tw, st)) != SPDBA_OK) return s;
        const PassParams<float> keep = hupd.p;
        hupd.p.fu = r.upd_pass.p.fu;   // the same update (states, tables, divisors) as the full form
        hupd.p.hg = keep.hg;
    }
    r.half_n = N0 * N1 * NHP;
    if ((s = r.alloc(&r.half, sizeof(cx_t<float>) * (size_t)r.half_n)) != SPDBA_OK) return s;
    SPDBA_CUDA(cudaMemsetAsync(r.half, 0, sizeof(cx_t<float>) * (size_t)r.half_n, st));
    hnl.p.mass_stride = (int)(sizeof(DevStats) / sizeof(double));
    r.h_inv_z = hz;
    if (p->opt.tma_passes) {
        // where the x rows are whole tiles the z inverse moves its tiles as tensor boxes
        s = herm_tma_prepare(&r.herm_tma, hz, r.c_hat);
        if (s == SPDBA_OK) r.use_herm_tma = true;
        else if (s != SPDBA_ERR_UNSUPPORTED) return s;
    }
    r.h_inv_y = hy_inv;
    r.h_nl = hnl;
    r.h_fwd_y = hy_fwd;
    r.h_mirror = hmir;
    r.h_upd = hupd;
    r.has_half = true;
    r.use_half = true;
    return SPDBA_OK;
}

// A 3-D complex64 CH run with half-spectrum storage: the stored half of the
// spectrum, its block map with conjugate neighbours (S1.2, Eq. S.4), and the
// transforms between the stored half and the update, all on x frequencies
// 0 .. N2/2 (rows padded to NHP, a multiple of the y pass tile and of B2).
static spdba_status group_init_ch_hs(spdba_plan* p, Group<float>& r, const int64_t* dims, const int32_t* block) {
    cudaStream_t st = p->st;
    spdba_status s;
    const int64_t N0 = dims[0], N1 = dims[1], N2 = dims[2];
    const int B2 = block[2];
    if (B2 < 1 || N2 % (2 * B2) != 0)
        return fail(SPDBA_ERR_UNSUPPORTED, "half-spectrum storage needs 2 B2 | N2 (B2 = %d, N2 = %lld)", B2,
                    (long long)N2);
    const int Py = pass_tile_pencils<float>(N1);
    if (Py == 0) return fail(SPDBA_ERR_UNSUPPORTED, "no y pass for %lld points", (long long)N1);
    int64_t q = Py;
    while (q % B2 != 0) q += Py;   // a multiple of both
    const int64_t M = N2 / 2;
    const int64_t NHP = ((M + 1 + q - 1) / q) * q;
    const int64_t dh[3] = {N0, N1, NHP};
    if ((s = make_geom(&r.g, 3, dh, block)) != SPDBA_OK) return s;
    r.g.hx = (int)(M / B2 + 1);
    r.ndim = 3;
    r.batch = 1;
    r.n = N0 * N1 * N2;
    for (int a = 0; a < 3; ++a) r.dims[a] = dims[a];
    r.hs = true;
    r.hs_nhp = NHP;
    r.hs_n = N0 * N1 * NHP;
    if (r.hs_n >= 0x7fffffffLL) return fail(SPDBA_ERR_UNSUPPORTED, "half-spectrum storage over 2^31 modes");
    if ((s = group_buffers<float>(p, r)) != SPDBA_OK) return s;
    for (int ax = 0; ax < 3; ++ax) {
        std::vector<float> k2 = k2_table<float>(dims[ax], p->opt.dx);
        if (ax == 2) k2.resize((size_t)NHP, 0.f);   // x frequencies 0 .. N2/2, then padding
        if ((s = upload(r, &r.k2ax[ax], k2, st)) != SPDBA_OK) return s;
        if ((s = upload(r, &r.taper[ax], taper_table<float>(r.g.b[ax]), st)) != SPDBA_OK) return s;
    }
    TwiddleCache<float>& tw = p->tw32;
    if ((s = r.fft1.init(3, dims, 1, tw, st)) != SPDBA_OK) return s;
    HalfGeo hg;
    hg.N0 = (int)N0; hg.N1 = (int)N1; hg.N2 = (int)N2; hg.NHP = (int)NHP;
    hg.fd_N2.init((uint32_t)N2);
    hg.fd_NHP.init((uint32_t)NHP);
    hg.fd_M.init((uint32_t)M);
    hg.r2c = 1;
    if ((s = make_axis_pass<float>(&r.h_inv_z, 3, dh, 1, 0, +1, PASS_PLAIN, tw, st)) != SPDBA_OK) return s;
    if ((s = make_axis_pass<float>(&r.h_inv_y, 3, dh, 1, 1, +1, PASS_PLAIN, tw, st)) != SPDBA_OK) return s;
    if ((s = make_half_pass(&r.h_nl, PASS_NL_HALF, hg, tw, st)) != SPDBA_OK) return s;
    r.h_nl.p.mass_stride = (int)(sizeof(DevStats) / sizeof(double));
    if ((s = make_axis_pass<float>(&r.h_fwd_y, 3, dh, 1, 1, -1, PASS_PLAIN, tw, st)) != SPDBA_OK) return s;
    if ((s = make_axis_pass<float>(&r.h_mirror, 3, dh, 1, 0, -1, PASS_PLAIN, tw, st)) != SPDBA_OK) return s;
    Pass<float> up;
    s = make_axis_pass<float>(&up, 3, dh, 1, 0, -1, PASS_CH_UPDATE, tw, st);
    // the fused update's tiles must lie within one x row, and its state table fit
    if (s == SPDBA_OK && NHP % up.P == 0 && (N0 / r.g.b[0]) * (int64_t)upd_table_cols(up.P, r.g.b[2]) <= kUpdTable) {
        fill_fuse<float>(p, r, up.p.fu);
        r.h_upd = up;
        r.has_fused = true;
        r.fused_update = p->opt.fuse_update != 0;
    } else if (s != SPDBA_OK && s != SPDBA_ERR_UNSUPPORTED) {
        return s;
    }
    if ((s = r.alloc(&r.hs_zlive, (size_t)(N1 * NHP))) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.hs_xlive, (size_t)NHP)) != SPDBA_OK) return s;
    SPDBA_CUDA(cudaMemsetAsync(r.hs_zlive, 1, (size_t)(N1 * NHP), st));
    SPDBA_CUDA(cudaMemsetAsync(r.hs_xlive, 1, (size_t)NHP, st));
    if (tma_update_fits(r.g)) {
        int per_sm = 0, nsm = 0;
        if ((s = make_box_map(r.tma_map_c, r.c_hat, r.g)) != SPDBA_OK) return s;
        if ((s = make_box_map(r.tma_map_g, r.work, r.g)) != SPDBA_OK) return s;
        if ((s = tma_update_prepare(&per_sm, &nsm)) != SPDBA_OK) return s;
        r.tma_grid = (long long)per_sm * nsm;
        r.tma_ok = true;
        r.use_tma = p->opt.tma_update != 0;
    }
    return SPDBA_OK;
}

template <typename T>
static spdba_status group_init_ch(spdba_plan* p, Group<T>& r, int ndim, const int64_t* dims, const int32_t* block,
                                  long long batch) {
    if (p->opt.half_storage) {
        if constexpr (std::is_same<T, float>::value) {
            if (ndim != 3 || batch != 1)
                return fail(SPDBA_ERR_UNSUPPORTED, "half-spectrum storage is built for 3-D runs");
            return group_init_ch_hs(p, r, dims, block);
        }
        return fail(SPDBA_ERR_UNSUPPORTED, "half-spectrum storage is built for complex64");
    }
    cudaStream_t st = p->st;
    spdba_status s = ndim == 3 ? make_geom(&r.g, ndim, dims, block)
                               : make_geom_batched(&r.g, ndim, dims, block, batch);
    if (s != SPDBA_OK) return s;
    r.ndim = ndim;
    r.batch = batch;
    r.n = 1;
    for (int a = 0; a < ndim; ++a) { r.dims[a] = dims[a]; r.n *= dims[a]; }
    if ((s = group_buffers<T>(p, r)) != SPDBA_OK) return s;
    const int a0 = 3 - ndim;
    for (int ax = 0; ax < 3; ++ax) {
        std::vector<T> k2 = ax < a0 ? std::vector<T>((size_t)r.g.n[ax], (T)0) : k2_table<T>(r.g.n[ax], p->opt.dx);
        if ((s = upload(r, &r.k2ax[ax], k2, st)) != SPDBA_OK) return s;
        if ((s = upload(r, &r.taper[ax], taper_table<T>(r.g.b[ax]), st)) != SPDBA_OK) return s;
    }
    TwiddleCache<T>& tw = twc<T>(p);
    if ((s = r.fft1.init(ndim, dims, 1, tw, st)) != SPDBA_OK) return s;
    // inverse along axes 0..d-2, fused inverse/NL/forward along d-1, forward d-2..0
    for (int a = 0; a < ndim - 1; ++a) {
        Pass<T> ps;
        if ((s = make_axis_pass<T>(&ps, ndim, dims, batch, a, +1, PASS_PLAIN, tw, st)) != SPDBA_OK) return s;
        r.pre_inv.push_back(ps);
    }
    if ((s = make_axis_pass<T>(&r.fused, ndim, dims, batch, ndim - 1, -1, PASS_CH_NL, tw, st)) != SPDBA_OK) return s;
    r.fused.p.nl_scale = (T)(1.0 / (double)r.n);
    r.fused.p.mass_stride = (int)(sizeof(DevStats) / sizeof(double));
    r.fused.p.mass_ppr = r.n / dims[ndim - 1];
    for (int a = ndim - 2; a >= 0; --a) {
        Pass<T> ps;
        spdba_status sf = SPDBA_ERR_UNSUPPORTED;
        if (a == 0 && p->opt.fuse_update) {
            // the pass along the first axis also applies the update (when a kernel exists for it)
            sf = make_axis_pass<T>(&ps, ndim, dims, batch, a, -1, PASS_CH_UPDATE, tw, st);
            // the tile's (row, x-block) state table must fit the kernel's shared table
            const int64_t bpass = ndim == 3 ? r.g.b[0] : r.g.b[1];
            if (sf == SPDBA_OK && (dims[0] / bpass) * (int64_t)upd_table_cols(ps.P, (int)r.g.b[2]) > kUpdTable)
                sf = SPDBA_ERR_UNSUPPORTED;
            // 32-bit mode indices inside the kernel
            if (sf == SPDBA_OK && r.batch * r.n >= 0x7fffffffLL) sf = SPDBA_ERR_UNSUPPORTED;
            if (sf == SPDBA_OK) {
                fill_fuse<T>(p, r, ps.p.fu);
                r.upd_pass = ps;
                r.has_fused = true;
                r.fused_update = true;
            } else if (sf != SPDBA_ERR_UNSUPPORTED) {
                return sf;
            }
        }
        // the plain pass is kept in every case: the staged form uses it
        if ((s = make_axis_pass<T>(&ps, ndim, dims, batch, a, -1, PASS_PLAIN, tw, st)) != SPDBA_OK) return s;
        r.pre_fwd.push_back(ps);
    }
    if constexpr (std::is_same<T, float>::value) {
        if (ndim == 3 && batch == 1 && p->opt.half_spectrum) {
            s = setup_half(p, r, dims);
            if (s != SPDBA_OK && s != SPDBA_ERR_UNSUPPORTED) return s;
        }
        if (tma_update_fits(r.g)) {
            // the list-driven update moves whole 8^3 blocks as TMA boxes
            int per_sm = 0, nsm = 0;
            if ((s = make_box_map(r.tma_map_c, r.c_hat, r.g)) != SPDBA_OK) return s;
            if ((s = make_box_map(r.tma_map_g, r.work, r.g)) != SPDBA_OK) return s;
            if ((s = tma_update_prepare(&per_sm, &nsm)) != SPDBA_OK) return s;
            r.tma_grid = (long long)per_sm * nsm;
            r.tma_ok = true;
            r.use_tma = p->opt.tma_update != 0;
        }
    }
    return SPDBA_OK;
}

template <typename T>
static spdba_status group_init_nls(spdba_plan* p, Group<T>& r, long long n, int nblk, long long batch) {
    cudaStream_t st = p->st;
    if (nblk < 1 || n % nblk != 0) return fail(SPDBA_ERR_UNSUPPORTED, "%d blocks do not divide %lld bins", nblk, n);
    const int64_t d[1] = {n};
    const int32_t b[1] = {(int32_t)(n / nblk)};
    spdba_status s = make_geom_batched(&r.g, 1, d, b, batch);
    if (s != SPDBA_OK) return s;
    r.ndim = 1;
    r.dims[0] = n;
    r.batch = batch;
    r.n = n;
    r.B = (int)(n / nblk);
    r.nblk = nblk;
    r.long_nls = n > 4096;
    TwiddleCache<T>& tw = twc<T>(p);
    if (r.long_nls) {
        if (n % 512 != 0 || 512 % nblk != 0)
            return fail(SPDBA_ERR_UNSUPPORTED, "NLS length %lld / %d blocks not supported", n, nblk);
        r.n1 = n / 512;
        if (!(r.n1 == 16 || r.n1 == 32 || r.n1 == 64 || r.n1 == 128 || r.n1 == 256 || r.n1 == 512))
            return fail(SPDBA_ERR_UNSUPPORTED, "NLS length %lld not supported", n);
        const int64_t dT[2] = {r.n1, 512};
        const int32_t bT[2] = {(int32_t)r.n1, 512 / nblk};
        if ((s = make_geom_batched(&r.gT, 2, dT, bT, batch)) != SPDBA_OK) return s;
        s = SPDBA_OK;
        if (!(r.tw_row = tw.get(512, st, &s))) return s;
        if (!(r.tw_col = tw.get(r.n1, st, &s))) return s;
        if (!(r.tw4 = tw.get(n, st, &s))) return s;
    } else {
        if (!(n == 64 || n == 128 || n == 256 || n == 512 || n == 1024 || n == 2048 || n == 4096))
            return fail(SPDBA_ERR_UNSUPPORTED, "NLS length %lld not supported", n);
        s = SPDBA_OK;
        if (!(r.tw_row = tw.get(n, st, &s))) return s;
        if ((s = r.fft1.init(1, d, 1, tw, st)) != SPDBA_OK) return s;
    }
    if ((s = group_buffers<T>(p, r)) != SPDBA_OK) return s;
    if ((s = nls_prepare<T>(n, r.n1, batch, &r.nl)) != SPDBA_OK) return s;
    std::vector<HPair<T>> H = half_step_table<T>(n, p->opt.beta2, p->opt.h, p->opt.dt_sample);
    if (r.long_nls) {
        // the row pass reads H(k1 + n1 m) at k1 * 512 + m: store it in that order
        std::vector<HPair<T>> HT(H.size());
        for (long long k1 = 0; k1 < r.n1; ++k1)
            for (long long m = 0; m < 512; ++m) HT[(size_t)(k1 * 512 + m)] = H[(size_t)(k1 + r.n1 * m)];
        H.swap(HT);
        // four-step twiddles W_n^{a b} (a < n1, b < 512) at a * 512 + b
        if ((s = r.alloc(&r.tw2, sizeof(cx_t<T>) * (size_t)n)) != SPDBA_OK) return s;
        if ((s = nls_twiddle2<T>(r.tw4, r.tw2, n, st)) != SPDBA_OK) return s;
    }
    if ((s = upload(r, &r.H, H, st)) != SPDBA_OK) return s;
    if ((s = upload(r, &r.ntaper, taper_table<T>(r.B), st)) != SPDBA_OK) return s;
    return SPDBA_OK;
}

// Eigendecomposition D = V diag(lam) V^T of the symmetric circulant
// cross-diffusion matrix (S4.1, S4.3), in FP64 from its closed form: the real
// Fourier vectors diagonalise every symmetric circulant matrix, with
// eigenvalue d + 2c - 2c cos(2 pi k / M) for frequency k (first row d + 2c,
// -c, 0, ..., -c); for M = 2 the single off-diagonal entry -c gives d + c
// (vector (1, 1)) and d + 3c (vector (1, -1)).  V[i * M + j] is component i
// of eigenvector j.
static void rcd_eigen_host(int M, double d, double c, std::vector<double>& V, std::vector<double>& lam) {
    V.assign((size_t)M * M, 0.0);
    lam.assign((size_t)M, 0.0);
    if (M == 1) {
        V[0] = 1.0;
        lam[0] = d + 2.0 * c;
        return;
    }
    if (M == 2) {
        const double h = sqrt(0.5);
        V[0] = h; V[1] = h; V[2] = h; V[3] = -h;
        lam[0] = d + c;
        lam[1] = d + 3.0 * c;
        return;
    }
    const double two_pi = 6.283185307179586476925286766559;
    const double s0 = 1.0 / sqrt((double)M), s1 = sqrt(2.0 / (double)M);
    int col = 0;
    for (int i = 0; i < M; ++i) V[(size_t)i * M + col] = s0;
    lam[col++] = d;
    for (int k = 1; 2 * k < M; ++k) {
        const double l = d + 2.0 * c - 2.0 * c * cos(two_pi * (double)k / (double)M);
        for (int i = 0; i < M; ++i) {
            const double ang = two_pi * (double)((long long)k * i % M) / (double)M;   // reduced before the multiply
            V[(size_t)i * M + col] = s1 * cos(ang);
            V[(size_t)i * M + col + 1] = s1 * sin(ang);
        }
        lam[col] = l;
        lam[col + 1] = l;
        col += 2;
    }
    if (M % 2 == 0) {
        for (int i = 0; i < M; ++i) V[(size_t)i * M + col] = (i % 2 ? -s0 : s0);
        lam[col] = d + 4.0 * c;
    }
}

template <typename T>
static spdba_status group_init_rcd(spdba_plan* p, Group<T>& r, int ndim, const int64_t* dims, const int32_t* block) {
    cudaStream_t st = p->st;
    spdba_status s = make_geom(&r.g, ndim, dims, block);
    if (s != SPDBA_OK) return s;
    const int M = p->opt.components;
    r.ndim = ndim;
    r.batch = 1;
    r.ncomp = M;
    r.n = 1;
    for (int a = 0; a < ndim; ++a) { r.dims[a] = dims[a]; r.n *= dims[a]; }
    if ((s = group_buffers<T>(p, r)) != SPDBA_OK) return s;
    const int a0 = 3 - ndim;
    for (int ax = 0; ax < 3; ++ax) {
        std::vector<T> k2 = ax < a0 ? std::vector<T>((size_t)r.g.n[ax], (T)0) : k2_table<T>(r.g.n[ax], p->opt.dx);
        if ((s = upload(r, &r.k2ax[ax], k2, st)) != SPDBA_OK) return s;
        if ((s = upload(r, &r.taper[ax], taper_table<T>(r.g.b[ax]), st)) != SPDBA_OK) return s;
    }
    if ((s = r.rcd_fft.init(ndim, dims, M, twc<T>(p), st)) != SPDBA_OK) return s;
    std::vector<double> V, lam;
    rcd_eigen_host(M, p->opt.rcd_d_diag, p->opt.rcd_d_cross, V, lam);
    if ((s = upload(r, &r.rcd_V, std::vector<T>(V.begin(), V.end()), st)) != SPDBA_OK) return s;
    if ((s = upload(r, &r.rcd_lam, std::vector<T>(lam.begin(), lam.end()), st)) != SPDBA_OK) return s;
    return rcd_prepare<T>(M);
}

// State preparation (Methods): activity, threshold, states, list.
template <typename T> static spdba_status group_assess(spdba_plan* p, Group<T>& r) {
    cudaStream_t st = p->st;
    spdba_status s;
    ProfScope ps(p, K_ASSESS, (double)sizeof(cx_t<T>) * (double)(r.hs ? r.hs_n : r.batch * r.n));
    const bool ch = p->opt.model == SPDBA_MODEL_CH;
    // gmax is zero here: it starts zeroed and every classification zeroes it after use
    double* sumsq = p->opt.measure == SPDBA_MEASURE_ENERGY ? r.sumsq : nullptr;
    const Geom& ga = r.long_nls ? r.gT : r.g;   // same block numbering in both orders
    if ((s = launch_block_activity<T>(ga, r.c_hat, r.maxsq, sumsq, r.gmax, st)) != SPDBA_OK) return s;
    const double* msq = sumsq ? r.sumsq : r.maxsq;
    const int force_dc = ch ? p->opt.force_dc : 0;
    if ((s = launch_classify_from_scan(r.g, msq, 1, r.gmax, p->threshold, p->opt.tau_rule, ch ? 1 : 0, force_dc,
                                       p->opt.transitions, r.tau, r.active, r.states, r.chi, r.list, r.count,
                                       r.scratch, r.stats, st)) != SPDBA_OK)
        return s;
    p->launches += 4;
    r.assessed = true;
    return SPDBA_OK;
}

// blocks the exact states mark non-frozen while the prediction in force had them frozen
__global__ void missed_kernel(const uint8_t* __restrict__ exact, const uint8_t* __restrict__ pred, long long nb,
                              DevStats* stats) {
    unsigned long long c = 0;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (long long)gridDim.x * blockDim.x)
        c += (exact[b] != 0 && pred[b] == 0) ? 1ull : 0ull;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&stats->missed, c);
}
__global__ void count_prediction_kernel(DevStats* stats) { stats->predictions += 1; }

// Reassessment with an attached predictor (3-D CH, one run): exact judge or prediction.
template <typename T> static spdba_status group_assess_predicted(spdba_plan* p, Group<T>& r) {
    cudaStream_t st = p->st;
    spdba_status s;
    const long long nb = r.g.blocks();
    const bool judge = !r.has_snap || r.step % p->judge_every == 0;
    if (judge) {
        if ((s = group_assess<T>(p, r)) != SPDBA_OK) return s;
        if (r.has_pred) {
            missed_kernel<<<grid_for(nb, 256), 256, 0, st>>>(r.states, r.pstates, nb, r.stats);
            p->launches += 1;
        }
        SPDBA_CUDA(cudaMemcpyAsync(r.snap_maxsq, r.maxsq, sizeof(double) * nb, cudaMemcpyDeviceToDevice, st));
        SPDBA_CUDA(cudaMemcpyAsync(r.snap_tau, r.tau, sizeof(double), cudaMemcpyDeviceToDevice, st));
        r.has_snap = true;
        r.has_pred = false;
        return SPDBA_OK;
    }
    ProfScope ps(p, K_PREDICT, 0.0);
    if ((s = spdba_predictor_states_internal(p->pred, r.snap_maxsq, r.snap_tau, r.states, 1, r.px, r.pmeasure, st)) !=
        SPDBA_OK)
        return s;
    if ((s = launch_classify(r.g, r.pmeasure, 0, r.pthr, p->opt.force_dc, p->opt.transitions, 0, r.active, r.states,
                             r.chi, r.list, r.count, r.scratch, r.stats, st)) != SPDBA_OK)
        return s;
    SPDBA_CUDA(cudaMemcpyAsync(r.pstates, r.states, nb, cudaMemcpyDeviceToDevice, st));
    count_prediction_kernel<<<1, 1, 0, st>>>(r.stats);
    p->launches += 10;
    r.has_pred = true;
    r.assessed = true;
    return SPDBA_OK;
}

// A dynamic-control check happens at the start of this step (S1.3): every
// control_every steps once the warm-up is over.
static bool control_step(const spdba_plan* p, int64_t step) {
    return p->opt.mode == SPDBA_MODE_ADAPTIVE && p->opt.target_ratio > 0 && step > p->opt.warmup_steps &&
           step % p->opt.control_every == 0;
}

// Warm-up, refresh and control steps update every block.
static bool all_active_step(const spdba_plan* p, int64_t step) {
    return step < p->opt.warmup_steps || (p->opt.refresh_every > 0 && step > 0 && step % p->opt.refresh_every == 0) ||
           control_step(p, step);
}

// The control decision of a group's runs, before the step's reassessment.
template <typename T> static spdba_status group_control(spdba_plan* p, Group<T>& r) {
    control_kernel<<<1, 256, 0, p->st>>>(r.stats, r.batch, r.g.live_bpr(), p->opt.target_ratio, p->opt.control_eta);
    SPDBA_CUDA(cudaGetLastError());
    p->launches += 1;
    return SPDBA_OK;
}

// Whether the kernels of step `step` are recorded by an active profile.
static void prof_select(spdba_plan* p, long long step) {
    p->prof_on = p->prof && (p->prof_every <= 1 || step % p->prof_every == 0);
}

template <typename T> static spdba_status ch_staged_update(spdba_plan* p, Group<T>& r, int dense);

template <typename T> static spdba_status group_ch_step(spdba_plan* p, Group<T>& r) {
    cudaStream_t st = p->st;
    spdba_status s;
    prof_select(p, r.step);
    const bool adaptive = p->opt.mode == SPDBA_MODE_ADAPTIVE;
    const int interval = p->pred ? p->horizon : p->reassess;
    const bool reassess = adaptive && (!r.assessed || r.step % interval == 0);
    if (control_step(p, r.step) && (s = group_control<T>(p, r)) != SPDBA_OK) return s;
    if (reassess) {
        s = p->pred ? group_assess_predicted<T>(p, r) : group_assess<T>(p, r);
        if (s != SPDBA_OK) return s;
        if constexpr (std::is_same<T, float>::value) {
            if (r.pair_list) {
                if ((s = launch_pair_live_list(r.h_mirror, r.pair_list, r.pair_count, st)) != SPDBA_OK) return s;
                p->launches += 1;
            }
            if (r.col_live) {
                if ((s = launch_half_col_live(r.g, r.states, (int)r.g.n[2], (int)r.h_fwd_y.p.I, r.col_live, st)) !=
                    SPDBA_OK)
                    return s;
                p->launches += 1;
            }
            if (r.hs_zlive) {
                if ((s = launch_hs_live(r.g, r.states, r.hs_zlive, r.hs_xlive, st)) != SPDBA_OK) return s;
                p->launches += 1;
            }
        }
    }
    const int dense = !adaptive || all_active_step(p, r.step);
    if (r.hs) {
        // half-spectrum storage: z, y inverse, x (nonlinearity), y and z forward on
        // the stored half, then the update (fused into the z forward or staged).
        // Profiled bytes are algorithmic: x frequencies 0 .. N2/2.
        const double hb = sizeof(cx_t<T>) * (double)(r.dims[0] * r.dims[1] * (r.dims[2] / 2 + 1));
        {
            ProfScope pr(p, K_FFT_PASS, 2.0 * hb);
            if ((s = launch_pass<T>(r.h_inv_z, r.c_hat, r.work, st)) != SPDBA_OK) return s;
        }
        {
            ProfScope pr(p, K_FFT_PASS, 2.0 * hb);
            if ((s = launch_pass<T>(r.h_inv_y, r.work, r.work, st)) != SPDBA_OK) return s;
        }
        Pass<T> nl = r.h_nl;
        if (reassess) {
            nl.p.mass = &r.stats[0].mass;
            zero_strided_kernel<<<1, 256, 0, st>>>(&r.stats[0].mass, r.batch, nl.p.mass_stride);
            p->launches += 1;
        }
        {
            ProfScope pr(p, K_FUSED_NL, 2.0 * hb);
            if ((s = launch_pass<T>(nl, r.work, r.work, st)) != SPDBA_OK) return s;
        }
        {
            // adaptive steps: the y forward skips the x columns and the z forward
            // the z pencils that no non-frozen block reads (outputs never used)
            Pass<T> yf = r.h_fwd_y;
            if (!dense) yf.p.col_live = r.hs_xlive;
            ProfScope pr(p, dense ? K_FFT_PASS : K_FFT_YFWD, 2.0 * hb);
            if ((s = launch_pass<T>(yf, r.work, r.work, st)) != SPDBA_OK) return s;
        }
        p->launches += 5;
        if (r.fused_update) {
            Pass<T> ps = r.h_upd;
            ps.p.fu.dense = dense;
            ProfScope pr(p, K_FFT_UPDATE, 3.0 * hb);
            if ((s = launch_pass<T>(ps, r.work, r.work, st)) != SPDBA_OK) return s;
            r.step += 1;
            return SPDBA_OK;
        }
        {
            Pass<T> zf = r.h_mirror;
            if (!dense) zf.p.col_live = r.hs_zlive;
            ProfScope pr(p, K_FFT_ZFWD, 2.0 * hb);
            if ((s = launch_pass<T>(zf, r.work, r.work, st)) != SPDBA_OK) return s;
        }
        return ch_staged_update<T>(p, r, dense);
    }
    if (r.use_half) {
        // Hermitian half-spectrum form: z (from c_hat), y, x (nonlinearity), y, z (update).
        // Profiled bytes are algorithmic: x frequencies 0 .. N2/2 of the half array
        // (its padding columns excluded).
        const double full_b = sizeof(cx_t<T>) * (double)(r.batch * r.n);
        const double half_b = full_b * (double)(r.g.n[2] / 2 + 1) / (double)r.g.n[2];
        {
            ProfScope pr(p, K_FFT_PASS, full_b + half_b);
            bool tma = false;
            if constexpr (std::is_same<T, float>::value) {
                if (r.use_herm_tma) {
                    tma = true;
                    s = launch_herm_inv_tma(r.herm_tma, r.h_inv_z, r.c_hat, r.half, &r.stats[0].timeouts, st);
                }
            }
            if (!tma) s = launch_pass<T>(r.h_inv_z, r.c_hat, r.half, st);
            if (s != SPDBA_OK) return s;
        }
        {
            ProfScope pr(p, K_FFT_PASS, 2.0 * half_b);
            if ((s = launch_pass<T>(r.h_inv_y, r.half, r.half, st)) != SPDBA_OK) return s;
        }
        Pass<T> nl = r.h_nl;
        if (reassess) {
            nl.p.mass = &r.stats[0].mass;
            zero_strided_kernel<<<1, 256, 0, st>>>(&r.stats[0].mass, r.batch, nl.p.mass_stride);
            p->launches += 1;
        }
        {
            ProfScope pr(p, K_FUSED_NL, 2.0 * half_b);
            if ((s = launch_pass<T>(nl, r.half, r.half, st)) != SPDBA_OK) return s;
        }
        {
            // the staged form's y forward skips the x-frequency columns that no
            // live z-forward tile reads (their outputs are never used)
            Pass<T> yf = r.h_fwd_y;
            const bool prune = !r.fused_update && !dense && r.col_live != nullptr;
            if (prune) yf.p.col_live = r.col_live;
            ProfScope pr(p, prune ? K_FFT_YFWD : K_FFT_PASS, 2.0 * half_b);
            if ((s = launch_pass<T>(yf, r.half, r.half, st)) != SPDBA_OK) return s;
        }
        p->launches += 4;
        if (r.fused_update) {
            Pass<T> ps = r.h_upd;
            ps.p.fu.dense = dense;
            ProfScope pr(p, K_FFT_UPDATE, half_b + 2.0 * full_b);
            if ((s = launch_pass<T>(ps, r.half, r.work, st)) != SPDBA_OK) return s;
            p->launches += 1;
            r.step += 1;
            return SPDBA_OK;
        }
        {
            Pass<T> ps = r.h_mirror;
            ps.p.fu.dense = dense;
            ProfScope pr(p, K_FFT_ZFWD, half_b + full_b);
            if ((s = launch_pass<T>(ps, r.half, r.work, st)) != SPDBA_OK) return s;
            p->launches += 1;
        }
        return ch_staged_update<T>(p, r, dense);
    }
    // pre-update: c = Re(IFFT(c_hat)), g = c^3 - c, g_hat = FFT(g)
    const double pass_bytes = 2.0 * sizeof(cx_t<T>) * (double)(r.batch * r.n);
    const cx_t<T>* src = r.c_hat;
    for (auto& ps : r.pre_inv) {
        ProfScope pr(p, K_FFT_PASS, pass_bytes);
        if ((s = launch_pass<T>(ps, src, r.work, st)) != SPDBA_OK) return s;
        p->launches += 1;
        src = r.work;
    }
    Pass<T> fused = r.fused;
    if (reassess) {
        fused.p.mass = &r.stats[0].mass;
        zero_strided_kernel<<<1, 256, 0, st>>>(&r.stats[0].mass, r.batch, fused.p.mass_stride);
        p->launches += 1;
    }
    {
        ProfScope pr(p, K_FUSED_NL, pass_bytes);
        if ((s = launch_pass<T>(fused, src, r.work, st)) != SPDBA_OK) return s;
        p->launches += 1;
    }
    for (size_t k = 0; k < r.pre_fwd.size(); ++k) {
        const bool last_fused = r.fused_update && k + 1 == r.pre_fwd.size();
        if (last_fused) {
            // forward transform of the first axis + update; traffic depends on the states
            Pass<T> ps = r.upd_pass;
            ps.p.fu.dense = dense;
            ProfScope pr(p, K_FFT_UPDATE, pass_bytes + sizeof(cx_t<T>) * (double)(r.batch * r.n));
            if ((s = launch_pass<T>(ps, r.work, r.work, st)) != SPDBA_OK) return s;
        } else {
            ProfScope pr(p, K_FFT_PASS, pass_bytes);
            if ((s = launch_pass<T>(r.pre_fwd[k], r.work, r.work, st)) != SPDBA_OK) return s;
        }
        p->launches += 1;
    }
    if (r.fused_update) {
        r.step += 1;
        return SPDBA_OK;
    }
    return ch_staged_update<T>(p, r, dense);
}

// The staged update: list-driven (or dense) update kernel reading g_hat from work.
template <typename T> static spdba_status ch_staged_update(spdba_plan* p, Group<T>& r, int dense) {
    cudaStream_t st = p->st;
    spdba_status s;
    CHUpdateArgs<T> a;
    a.c_hat = r.c_hat;
    a.g_hat = r.work;
    for (int ax = 0; ax < 3; ++ax) { a.k2ax[ax] = r.k2ax[ax]; a.taper[ax] = r.taper[ax]; }
    a.states = r.states;
    a.chi = r.chi;
    a.list = r.list;
    a.count = r.count;
    a.dt = (T)p->opt.dt;
    a.dtkappa = (T)(p->opt.dt * p->opt.kappa);
    a.stats = r.stats;
    {
        // list-update traffic is known only on the device; it is added at profile end
        ProfScope pr(p, dense ? K_UPDATE_DENSE : K_UPDATE_LIST,
                     dense ? 3.0 * sizeof(cx_t<T>) * (double)(r.batch * r.n) : 0.0);
        bool tma = false;
        if constexpr (std::is_same<T, float>::value) tma = r.use_tma && !dense;
        if (tma) {
            if constexpr (std::is_same<T, float>::value)
                if ((s = launch_ch_update_tma(r.tma_map_c, r.tma_map_g, r.g, a, r.tma_grid, st)) != SPDBA_OK) return s;
        } else if ((s = launch_ch_update<T>(r.g, a, dense, st)) != SPDBA_OK) {
            return s;
        }
        p->launches += 1;
        if (!dense) p->list_updates += 1;
    }
    r.step += 1;
    return SPDBA_OK;
}

template <typename T> static NLSArgs<T> nls_args(spdba_plan* p, Group<T>& r, cx_t<T>* S, long long batch, int dense) {
    NLSArgs<T> a{};
    a.S = S;
    a.H = r.H;
    a.states = r.states;
    a.chi = r.chi;
    a.taper = r.ntaper;
    a.tw = r.tw_row;
    a.tw4 = r.tw2;
    a.n = r.n;
    a.n1 = r.n1;
    a.batch = batch;
    a.B = r.B;
    a.nblk = r.nblk;
    a.fd_B.init((uint32_t)r.B);
    a.mb_shift = 0;
    if (r.long_nls)
        while ((512 >> a.mb_shift) > r.nblk) ++a.mb_shift;
    a.dense = dense;
    a.gamma_h = (T)(p->opt.gamma * p->opt.h);
    a.inv_n = (T)(1.0 / (double)r.n);
    a.power = nullptr;
    a.power_stride = (int)(sizeof(DevStats) / sizeof(double));
    return a;
}

template <typename T>
static spdba_status row_pass(spdba_plan* p, Group<T>& r, NLSArgs<T> a, int fwd, int close, int open, int inv) {
    a.do_fwd = fwd; a.do_close = close; a.do_open = open; a.do_inv = inv;
    ProfScope pr(p, K_NLS_ROW, 2.0 * sizeof(cx_t<T>) * (double)(a.batch * a.n));
    p->launches += 1;
    return nls_row_pass<T>(a, r.nl, p->st);
}
template <typename T> static spdba_status col_pass(spdba_plan* p, Group<T>& r, NLSArgs<T> a, int inv, int kerr, int fwd) {
    a.do_inv = inv; a.do_kerr = kerr; a.do_fwd = fwd;
    ProfScope pr(p, K_NLS_COL, 2.0 * sizeof(cx_t<T>) * (double)(a.batch * a.n));
    p->launches += 1;
    return nls_col_pass<T>(a, r.nl, p->st);
}

// n steps of an NLS group.  Between calls S is the spectrum at a step boundary.
template <typename T> static spdba_status group_nls_steps(spdba_plan* p, Group<T>& r, int64_t nsteps) {
    cudaStream_t st = p->st;
    spdba_status s;
    const bool adaptive = p->opt.mode == SPDBA_MODE_ADAPTIVE;
    int prev_dense = 1;
    for (int64_t i = 0; i < nsteps; ++i) {
        prof_select(p, r.step);
        const bool reassess = adaptive && (!r.assessed || r.step % p->reassess == 0);
        const int dense = !adaptive || all_active_step(p, r.step);
        if (control_step(p, r.step) && (s = group_control<T>(p, r)) != SPDBA_OK) return s;
        NLSArgs<T> a = nls_args<T>(p, r, r.c_hat, r.batch, dense);
        if (r.long_nls) {
            // close the previous step unless this step's row pass can take it over
            const bool merge = i > 0 && !reassess && prev_dense == dense;
            if (i > 0 && !merge) {
                NLSArgs<T> c = nls_args<T>(p, r, r.c_hat, r.batch, prev_dense);
                if ((s = row_pass<T>(p, r, c, 1, 1, 0, 0)) != SPDBA_OK) return s;
            }
            if (reassess && (s = group_assess<T>(p, r)) != SPDBA_OK) return s;
            if ((s = row_pass<T>(p, r, a, merge ? 1 : 0, merge ? 1 : 0, 1, 1)) != SPDBA_OK) return s;
            NLSArgs<T> c = a;
            c.tw = r.tw_col;
            if (reassess) {
                zero_strided_kernel<<<1, 256, 0, st>>>(&r.stats[0].mass, r.batch, a.power_stride);
                c.power = &r.stats[0].mass;
            }
            if ((s = col_pass<T>(p, r, c, 1, 1, 1)) != SPDBA_OK) return s;
        } else {
            if (reassess && (s = group_assess<T>(p, r)) != SPDBA_OK) return s;
            if (reassess) {
                zero_strided_kernel<<<1, 256, 0, st>>>(&r.stats[0].mass, r.batch, a.power_stride);
                a.power = &r.stats[0].mass;
            }
            ProfScope pr(p, K_NLS_STEP, 2.0 * sizeof(cx_t<T>) * (double)(r.batch * r.n));
            if ((s = nls_small_step<T>(a, r.nl, st)) != SPDBA_OK) return s;
            p->launches += 1;
        }
        ratio_kernel<<<1, 256, 0, st>>>(r.stats, r.batch, r.g.bpr(), r.g.block_modes(), dense);
        SPDBA_CUDA(cudaGetLastError());
        p->launches += 1;
        prev_dense = dense;
        r.step += 1;
    }
    if (r.long_nls && nsteps > 0) {
        NLSArgs<T> c = nls_args<T>(p, r, r.c_hat, r.batch, prev_dense);
        if ((s = row_pass<T>(p, r, c, 1, 1, 0, 0)) != SPDBA_OK) return s;
    }
    return SPDBA_OK;
}

// One RCD step (S4.2): state preparation at reassessments (component RMS
// amplitude), u = IFFT(u_hat) of the M components, R(u) in real space, its
// FFT, then the per-mode coupled update on the listed blocks (or every block).
template <typename T> static spdba_status group_rcd_step(spdba_plan* p, Group<T>& r) {
    cudaStream_t st = p->st;
    spdba_status s;
    prof_select(p, r.step);
    const bool adaptive = p->opt.mode == SPDBA_MODE_ADAPTIVE;
    const bool reassess = adaptive && (!r.assessed || r.step % p->reassess == 0);
    const int M = (int)r.ncomp;
    const double field_b = sizeof(cx_t<T>) * (double)(M * r.n);
    if (control_step(p, r.step) && (s = group_control<T>(p, r)) != SPDBA_OK) return s;
    if (reassess) {
        ProfScope ps(p, K_ASSESS, field_b);
        if ((s = launch_rcd_activity<T>(r.g, r.c_hat, M, r.maxsq, r.gmax, st)) != SPDBA_OK) return s;
        if ((s = launch_classify_from_scan(r.g, r.maxsq, 1, r.gmax, p->threshold, p->opt.tau_rule, 1, p->opt.force_dc,
                                           p->opt.transitions, r.tau, r.active, r.states, r.chi, r.list, r.count,
                                           r.scratch, r.stats, st)) != SPDBA_OK)
            return s;
        p->launches += 4;
        r.assessed = true;
    }
    const int dense = !adaptive || all_active_step(p, r.step);
    {
        ProfScope pr(p, K_RCD_FFT, 2.0 * r.ndim * field_b);
        if ((s = r.rcd_fft.exec(r.c_hat, r.work, SPDBA_INVERSE, st)) != SPDBA_OK) return s;
    }
    {
        ProfScope pr(p, K_RCD_REACTION, 2.0 * field_b);
        const RcdParams& q = p->rcd;
        if ((s = launch_rcd_reaction<T>(r.work, r.n, M, (T)q.r, (T)q.a, (T)q.alpha, (T)q.beta, st)) != SPDBA_OK)
            return s;
    }
    {
        ProfScope pr(p, K_RCD_FFT, 2.0 * r.ndim * field_b);
        if ((s = r.rcd_fft.exec(r.work, r.work, SPDBA_FORWARD, st)) != SPDBA_OK) return s;
    }
    p->launches += 2 * r.ndim + 1;
    RcdArgs<T> a;
    a.u_hat = r.c_hat;
    a.g_hat = r.work;
    a.V = r.rcd_V;
    a.lam = r.rcd_lam;
    for (int ax = 0; ax < 3; ++ax) { a.k2ax[ax] = r.k2ax[ax]; a.taper[ax] = r.taper[ax]; }
    a.states = r.states;
    a.chi = r.chi;
    a.list = r.list;
    a.count = r.count;
    a.dt = (T)p->opt.dt;
    a.M = M;
    a.n = r.n;
    a.stats = r.stats;
    {
        // list-driven traffic is known only on the device; it is added at profile end
        ProfScope pr(p, dense ? K_UPDATE_DENSE : K_UPDATE_LIST, dense ? 3.0 * field_b : 0.0);
        if ((s = launch_rcd_update<T>(r.g, a, dense, st)) != SPDBA_OK) return s;
        p->launches += 1;
        if (!dense) p->list_updates += 1;
    }
    r.step += 1;
    return SPDBA_OK;
}

// ------------------------------------------------------------------ multi-size form
// Builds the multi-size form of a batched 2-D complex64 CH plan for one tile
// table (mf.ok stays false where some group does not qualify).
static spdba_status build_multi(spdba_plan* p, int tile, MultiForm& mf) {
    auto& gs = groups<float>(p);
    mf.ok = false;
    if (p->opt.model != SPDBA_MODEL_CH || gs.size() < 2 || gs.size() > (size_t)kMultiMaxGroups) return SPDBA_OK;
    std::vector<MultiGroup<float>> hv[3];
    unsigned tot[3] = {0, 0, 0};
    // the phase's pass of one group: length L along the pass axis, in -> out
    auto add = [&](int ph, const Pass<float>& ps, int64_t L, const void* in, void* out) {
        const int P = multi_tile_pencils(tile, L);
        const long long np = ps.p.O * ps.p.I;
        if (P == 0 || ps.p.generic || ps.p.I % P != 0 || np / P + tot[ph] >= 0x7fffffffLL) return false;
        MultiGroup<float> m;
        m.a = ps.p;
        m.a.in = reinterpret_cast<const cx_t<float>*>(in);
        m.a.out = reinterpret_cast<cx_t<float>*>(out);
        m.L = (int)L;
        m.P = P;
        m.t0 = tot[ph];
        m.nt = (unsigned)(np / P);
        tot[ph] += m.nt;
        hv[ph].push_back(m);
        return true;
    };
    for (auto& gp : gs) {
        Group<float>& r = *gp;
        if (r.ndim != 2 || r.pre_inv.size() != 1 || r.pre_fwd.size() != 1 || !r.has_fused) return SPDBA_OK;
        // the update's per-tile state table must fit with this table's tile width
        const int P0 = multi_tile_pencils(tile, r.dims[0]);
        if (P0 == 0 || (r.dims[0] / r.g.b[1]) * (int64_t)upd_table_cols(P0, r.g.b[2]) > kUpdTable) return SPDBA_OK;
        if (!add(0, r.pre_inv[0], r.dims[0], r.c_hat, r.work)) return SPDBA_OK;
        Pass<float> nl = r.fused;
        nl.p.mass = &r.stats[0].mass;   // the kernel clears it on steps without a reassessment
        if (!add(1, nl, r.dims[1], r.work, r.work)) return SPDBA_OK;
        Pass<float> up = r.upd_pass;
        up.p.fu.dense = 0;              // set per launch
        if (!add(2, up, r.dims[0], r.work, r.work)) return SPDBA_OK;
    }
    MultiPhase* ph[3] = {&mf.inv, &mf.nl, &mf.upd};
    const int sign[3] = {+1, -1, -1};
    const int mode[3] = {PASS_PLAIN, PASS_CH_NL, PASS_CH_UPDATE};
    const bool pfast[3] = {true, false, true};
    cudaStream_t st = p->st;
    for (int k = 0; k < 3; ++k) {
        MultiPhase& m = *ph[k];
        long long resident = 0;
        spdba_status s = multi_kernel(tile, sign[k], mode[k], pfast[k], &m.func, &m.smem, &resident);
        if (s != SPDBA_OK) return s;
        void* g = nullptr;
        cudaError_t e = dev_alloc(&g, sizeof(MultiGroup<float>) * hv[k].size());
        if (e != cudaSuccess) return cuda_fail(e, "device allocation (multi-size groups)");
        p->multi_bufs.push_back(g);
        SPDBA_CUDA(cudaMemcpyAsync(g, hv[k].data(), sizeof(MultiGroup<float>) * hv[k].size(), cudaMemcpyHostToDevice, st));
        m.groups = reinterpret_cast<MultiGroup<float>*>(g);
        m.ng = (int)hv[k].size();
        m.total = tot[k];
        m.grid = resident < (long long)tot[k] ? resident : (long long)tot[k];
    }
    SPDBA_CUDA(cudaStreamSynchronize(st));   // the host arrays are temporaries
    mf.ok = true;
    return SPDBA_OK;
}

// One step of every group in the multi-size form: per group the control
// check and the reassessment (when due), then three launches over all groups.
static spdba_status multi_ch_step(spdba_plan* p, const MultiForm& mf) {
    auto& gs = groups<float>(p);
    cudaStream_t st = p->st;
    spdba_status s;
    const bool adaptive = p->opt.mode == SPDBA_MODE_ADAPTIVE;
    unsigned dense_mask = 0, mass_mask = 0;
    double pass_bytes = 0, upd_bytes = 0;
    prof_select(p, gs[0]->step);
    for (size_t i = 0; i < gs.size(); ++i) {
        Group<float>& r = *gs[i];
        const bool reassess = adaptive && (!r.assessed || r.step % p->reassess == 0);
        if (control_step(p, r.step) && (s = group_control<float>(p, r)) != SPDBA_OK) return s;
        if (reassess) {
            if ((s = group_assess<float>(p, r)) != SPDBA_OK) return s;
            zero_strided_kernel<<<1, 256, 0, st>>>(&r.stats[0].mass, r.batch, r.fused.p.mass_stride);
            p->launches += 1;
            mass_mask |= 1u << i;
        }
        if (!adaptive || all_active_step(p, r.step)) dense_mask |= 1u << i;
        const double b = sizeof(cx_t<float>) * (double)(r.batch * r.n);
        pass_bytes += 2.0 * b;
        upd_bytes += 3.0 * b;
    }
    {
        ProfScope pr(p, K_FFT_PASS, pass_bytes);
        if ((s = launch_multi(mf.inv.func, mf.inv.smem, mf.inv.grid, mf.inv.groups, mf.inv.ng, mf.inv.total, 0u, 0u,
                              st)) != SPDBA_OK)
            return s;
    }
    {
        ProfScope pr(p, K_FUSED_NL, pass_bytes);
        if ((s = launch_multi(mf.nl.func, mf.nl.smem, mf.nl.grid, mf.nl.groups, mf.nl.ng, mf.nl.total, 0u,
                              mass_mask, st)) != SPDBA_OK)
            return s;
    }
    {
        // forward transform + update; traffic depends on the states (dense-equivalent bytes)
        ProfScope pr(p, K_FFT_UPDATE, upd_bytes);
        if ((s = launch_multi(mf.upd.func, mf.upd.smem, mf.upd.grid, mf.upd.groups, mf.upd.ng, mf.upd.total,
                              dense_mask, 0u, st)) != SPDBA_OK)
            return s;
    }
    p->launches += 3;
    for (auto& g : gs) g->step += 1;
    return SPDBA_OK;
}

template <typename T> static spdba_status group_steps(spdba_plan* p, Group<T>& g, int64_t n) {
    if (p->opt.model == SPDBA_MODEL_NLS) return group_nls_steps<T>(p, g, n);
    for (int64_t i = 0; i < n; ++i) {
        spdba_status s = p->opt.model == SPDBA_MODEL_RCD ? group_rcd_step<T>(p, g) : group_ch_step<T>(p, g);
        if (s != SPDBA_OK) return s;
    }
    return SPDBA_OK;
}

// Streams and events for running the groups concurrently (created once).
static spdba_status ensure_group_streams(spdba_plan* p, size_t ngroups) {
    if (p->gstreams.size() >= ngroups) return SPDBA_OK;
    if (!p->fork_ev) SPDBA_CUDA(cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming));
    while (p->gstreams.size() < ngroups) {
        cudaStream_t s = nullptr;
        SPDBA_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        p->gstreams.push_back(s);
        cudaEvent_t e = nullptr;
        SPDBA_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p->gevents.push_back(e);
    }
    return SPDBA_OK;
}

template <typename T> static spdba_status direct_steps(spdba_plan* p, int64_t n) {
    auto& gs = groups<T>(p);
    if constexpr (std::is_same<T, float>::value) {
        if (p->multi_sel > 0 && p->opt.model == SPDBA_MODEL_CH) {
            const MultiForm& mf = p->multi[p->multi_sel - 1];
            for (int64_t i = 0; i < n; ++i) {
                spdba_status s = multi_ch_step(p, mf);
                if (s != SPDBA_OK) return s;
            }
            return SPDBA_OK;
        }
    }
    if (gs.size() > 1 && !p->prof) {
        // groups share nothing during steps: each runs its n steps on its own
        // stream, forked from the plan's stream and joined back to it (inside a
        // graph capture the forked streams join the capture)
        spdba_status s = ensure_group_streams(p, gs.size());
        if (s != SPDBA_OK) return s;
        const cudaStream_t main = p->st;
        SPDBA_CUDA(cudaEventRecord(p->fork_ev, main));
        for (size_t i = 0; i < gs.size() && s == SPDBA_OK; ++i) {
            SPDBA_CUDA(cudaStreamWaitEvent(p->gstreams[i], p->fork_ev, 0));
            p->st = p->gstreams[i];
            s = group_steps<T>(p, *gs[i], n);
            p->st = main;
            cudaError_t e = cudaEventRecord(p->gevents[i], p->gstreams[i]);
            if (s == SPDBA_OK && e != cudaSuccess) s = cuda_fail(e, "cudaEventRecord(group)");
            if (s == SPDBA_OK) {
                e = cudaStreamWaitEvent(main, p->gevents[i], 0);
                if (e != cudaSuccess) s = cuda_fail(e, "cudaStreamWaitEvent(join)");
            }
        }
        p->st = main;
        return s;
    }
    if (p->opt.model == SPDBA_MODEL_NLS) {
        for (auto& g : gs) {
            spdba_status s = group_nls_steps<T>(p, *g, n);
            if (s != SPDBA_OK) return s;
        }
        return SPDBA_OK;
    }
    for (int64_t i = 0; i < n; ++i) {
        for (auto& g : gs) {
            spdba_status s = p->opt.model == SPDBA_MODEL_RCD ? group_rcd_step<T>(p, *g) : group_ch_step<T>(p, *g);
            if (s != SPDBA_OK) return s;
        }
    }
    return SPDBA_OK;
}

// A segment is R steps starting at a reassessment step with no all-active step
// inside: its launch sequence is the same every time, so it is captured once
// into a CUDA graph and replayed.
template <typename T> static bool segment_ready(spdba_plan* p) {
    if (p->pred) return false;   // judge/prediction alternate: the launch sequence varies
    for (auto& g : groups<T>(p)) {
        if (g->step % p->reassess != 0) return false;
        for (int64_t s = g->step; s < g->step + p->reassess; ++s) {
            if (all_active_step(p, s)) return false;
            // a sampled profile records events on its steps: those run directly
            if (p->prof && s % p->prof_every == 0) return false;
        }
    }
    return true;
}

template <typename T> static spdba_status plan_step(spdba_plan* p, int64_t n) {
    // graphs need a capturable (non-legacy) stream; a profile of every step records
    // events per kernel (a sampled one keeps graphs for unsampled segments)
    if (!p->opt.use_graph || (p->prof && p->prof_every <= 1) || p->st == 0) return direct_steps<T>(p, n);
    const int R = p->reassess;
    int64_t i = 0;
    while (i < n) {
        if (n - i >= R && segment_ready<T>(p)) {
            if (!p->seg_exec) {
                const long long l0 = p->launches, u0 = p->list_updates;
                SPDBA_CUDA(cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal));
                spdba_status s = direct_steps<T>(p, R);
                cudaGraph_t graph = nullptr;
                cudaError_t e = cudaStreamEndCapture(p->st, &graph);
                if (s != SPDBA_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return s;
                }
                if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&p->seg_exec, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) {
                    p->seg_exec = nullptr;
                    return cuda_fail(e, "cudaGraphInstantiate");
                }
                p->seg_launches = p->launches - l0;
                p->seg_list_updates = p->list_updates - u0;
                // the capture advanced the host-side step counters; run what it recorded
                SPDBA_CUDA(cudaGraphLaunch(p->seg_exec, p->st));
            } else {
                SPDBA_CUDA(cudaGraphLaunch(p->seg_exec, p->st));
                for (auto& g : groups<T>(p)) {
                    g->step += R;
                    if (p->opt.mode == SPDBA_MODE_ADAPTIVE) g->assessed = true;
                }
                p->launches += p->seg_launches;
                p->list_updates += p->seg_list_updates;
            }
            i += R;
        } else {
            spdba_status s = direct_steps<T>(p, 1);
            if (s != SPDBA_OK) return s;
            ++i;
        }
    }
    return SPDBA_OK;
}

template <typename T>
static spdba_status run_set_field(spdba_plan* p, Group<T>& r, long long sub, const void* src, int on_dev) {
    cudaStream_t st = p->st;
    spdba_status s;
    cx_t<T>* slot = r.c_hat + sub * r.n;
    cx_t<T>* wslot = r.work + sub * r.n;
    const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (p->opt.model == SPDBA_MODEL_RCD) {
        const long long tot = r.n * r.ncomp;
        SPDBA_CUDA(cudaMemcpyAsync(r.real, src, sizeof(T) * tot, kind, st));
        real_to_complex_kernel<T><<<grid_for(tot, 256), 256, 0, st>>>(r.real, r.work, tot);
        if ((s = r.rcd_fft.exec(r.work, r.c_hat, SPDBA_FORWARD, st)) != SPDBA_OK) return s;
    } else if (p->opt.model == SPDBA_MODEL_CH) {
        SPDBA_CUDA(cudaMemcpyAsync(r.real, src, sizeof(T) * r.n, kind, st));
        real_to_complex_kernel<T><<<grid_for(r.n, 256), 256, 0, st>>>(r.real, wslot, r.n);
        if ((s = r.fft1.exec(wslot, slot, SPDBA_FORWARD, st)) != SPDBA_OK) return s;
        if (r.hs) {
            // keep the half kx = 0 .. N2/2 of the full spectrum, rows padded with zeros
            const size_t es = sizeof(cx_t<T>);
            const int64_t N2 = r.dims[2];
            SPDBA_CUDA(cudaMemsetAsync(r.work, 0, es * (size_t)r.hs_n, st));
            SPDBA_CUDA(cudaMemcpy2DAsync(r.work, es * (size_t)r.hs_nhp, r.c_hat, es * (size_t)N2,
                                         es * (size_t)(N2 / 2 + 1), (size_t)(r.dims[0] * r.dims[1]),
                                         cudaMemcpyDeviceToDevice, st));
            SPDBA_CUDA(cudaMemcpyAsync(r.c_hat, r.work, es * (size_t)r.hs_n, cudaMemcpyDeviceToDevice, st));
        }
    } else if (!r.long_nls) {
        SPDBA_CUDA(cudaMemcpyAsync(wslot, src, sizeof(cx_t<T>) * r.n, kind, st));
        if ((s = r.fft1.exec(wslot, slot, SPDBA_FORWARD, st)) != SPDBA_OK) return s;
    } else {
        // E (natural time order) -> column pass (forward) -> row pass (forward): S in transposed order
        SPDBA_CUDA(cudaMemcpyAsync(slot, src, sizeof(cx_t<T>) * r.n, kind, st));
        NLSArgs<T> a = nls_args<T>(p, r, slot, 1, 1);
        a.tw = r.tw_col;
        a.do_inv = 0; a.do_kerr = 0; a.do_fwd = 1;
        if ((s = nls_col_pass<T>(a, r.nl, st)) != SPDBA_OK) return s;
        a.tw = r.tw_row;
        a.do_fwd = 1; a.do_close = 0; a.do_open = 0; a.do_inv = 0;
        if ((s = nls_row_pass<T>(a, r.nl, st)) != SPDBA_OK) return s;
    }
    r.step = 0;
    r.assessed = false;
    r.has_snap = false;
    r.has_pred = false;
    stats_reset_kernel<<<1, 32, 0, st>>>(r.stats + sub, 1, p->threshold);
    SPDBA_CUDA(cudaGetLastError());
    SPDBA_CUDA(cudaMemsetAsync(r.states + sub * r.g.bpr(), SPDBA_ACTIVE, r.g.bpr(), st));
    return SPDBA_OK;
}

template <typename T>
static spdba_status run_get_field(spdba_plan* p, Group<T>& r, long long sub, void* dst, int on_dev) {
    cudaStream_t st = p->st;
    spdba_status s;
    cx_t<T>* slot = r.c_hat + sub * r.n;
    cx_t<T>* wslot = r.work + sub * r.n;
    const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (p->opt.model == SPDBA_MODEL_RCD) {
        const long long tot = r.n * r.ncomp;
        if ((s = r.rcd_fft.exec(r.c_hat, r.work, SPDBA_INVERSE, st)) != SPDBA_OK) return s;
        complex_real_part_kernel<T><<<grid_for(tot, 256), 256, 0, st>>>(r.work, r.real, tot);
        SPDBA_CUDA(cudaMemcpyAsync(dst, r.real, sizeof(T) * tot, kind, st));
    } else if (p->opt.model == SPDBA_MODEL_CH) {
        if (r.hs) {
            half_storage_extend_kernel<T><<<grid_for(r.n, 256), 256, 0, st>>>(
                r.c_hat, r.work, (int)r.dims[0], (int)r.dims[1], (int)r.dims[2], (int)r.hs_nhp);
            if ((s = r.fft1.exec(r.work, wslot, SPDBA_INVERSE, st)) != SPDBA_OK) return s;
        } else if ((s = r.fft1.exec(slot, wslot, SPDBA_INVERSE, st)) != SPDBA_OK) {
            return s;
        }
        complex_real_part_kernel<T><<<grid_for(r.n, 256), 256, 0, st>>>(wslot, r.real, r.n);
        SPDBA_CUDA(cudaMemcpyAsync(dst, r.real, sizeof(T) * r.n, kind, st));
    } else if (!r.long_nls) {
        if ((s = r.fft1.exec(slot, wslot, SPDBA_INVERSE, st)) != SPDBA_OK) return s;
        SPDBA_CUDA(cudaMemcpyAsync(dst, wslot, sizeof(cx_t<T>) * r.n, kind, st));
    } else {
        SPDBA_CUDA(cudaMemcpyAsync(wslot, slot, sizeof(cx_t<T>) * r.n, cudaMemcpyDeviceToDevice, st));
        NLSArgs<T> a = nls_args<T>(p, r, wslot, 1, 1);
        a.tw = r.tw_row;
        a.do_fwd = 0; a.do_close = 0; a.do_open = 0; a.do_inv = 1;
        if ((s = nls_row_pass<T>(a, r.nl, st)) != SPDBA_OK) return s;
        a.tw = r.tw_col;
        a.do_inv = 1; a.do_kerr = 0; a.do_fwd = 0;
        if ((s = nls_col_pass<T>(a, r.nl, st)) != SPDBA_OK) return s;
        SPDBA_CUDA(cudaMemcpyAsync(dst, wslot, sizeof(cx_t<T>) * r.n, kind, st));
    }
    SPDBA_CUDA(cudaStreamSynchronize(st));
    return SPDBA_OK;
}

template <typename T>
static spdba_status copy_spectrum(spdba_plan* p, Group<T>& r, long long sub, void* buf, int on_dev, bool get) {
    cudaStream_t st = p->st;
    size_t bytes = sizeof(cx_t<T>) * (size_t)(r.n * r.ncomp);
    cx_t<T>* slot = r.c_hat + sub * r.n;
    cx_t<T>* wslot = r.work + sub * r.n;
    spdba_status s;
    if (r.hs) {
        // the stored half, N0 * N1 rows of N2/2 + 1 entries (rows of hs_nhp on the device)
        const size_t es = sizeof(cx_t<T>);
        const size_t w = es * (size_t)(r.dims[2] / 2 + 1), pitch = es * (size_t)r.hs_nhp;
        const size_t rows = (size_t)(r.dims[0] * r.dims[1]);
        if (get) {
            SPDBA_CUDA(cudaMemcpy2DAsync(buf, w, r.c_hat, pitch, w, rows,
                                         on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
            SPDBA_CUDA(cudaStreamSynchronize(st));
        } else {
            SPDBA_CUDA(cudaMemsetAsync(r.c_hat, 0, es * (size_t)r.hs_n, st));
            SPDBA_CUDA(cudaMemcpy2DAsync(r.c_hat, pitch, buf, w, w, rows,
                                         on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
            r.assessed = false;
        }
        return SPDBA_OK;
    }
    if (get) {
        const cx_t<T>* from = slot;
        if (r.long_nls) {
            if ((s = nls_permute<T>(slot, wslot, r.n, r.n1, 1, 1, st)) != SPDBA_OK) return s;
            from = wslot;
        }
        SPDBA_CUDA(cudaMemcpyAsync(buf, from, bytes, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        SPDBA_CUDA(cudaStreamSynchronize(st));
    } else {
        cx_t<T>* to = r.long_nls ? wslot : slot;
        SPDBA_CUDA(cudaMemcpyAsync(to, buf, bytes, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        if (r.long_nls && (s = nls_permute<T>(wslot, slot, r.n, r.n1, 1, 0, st)) != SPDBA_OK) return s;
        r.assessed = false;
    }
    return SPDBA_OK;
}

}  // namespace spdba

// ------------------------------------------------------------------ C ABI
static spdba_status latch(spdba_plan* p, spdba_status s) {
    if (s == SPDBA_ERR_CUDA && p) p->latched = s;
    return s;
}
#define PLAN_CHECK(p)                                                                             \
    do {                                                                                          \
        if (!(p)) return fail(SPDBA_ERR_ARG, "NULL plan");                                        \
        if ((p)->latched != SPDBA_OK) return fail((p)->latched, "plan has a latched CUDA error"); \
    } while (0)

extern "C" void spdba_options_default(spdba_options* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->model = SPDBA_MODEL_CH;
    o->precision = SPDBA_C64;
    o->mode = SPDBA_MODE_ADAPTIVE;
    o->measure = SPDBA_MEASURE_MAXAMP;
    o->tau_rule = SPDBA_TAU_REL_MAX;
    o->transitions = 1;
    o->force_dc = 1;
    o->refresh_every = 0;
    o->warmup_steps = 0;
    o->use_graph = 1;
    o->fuse_update = 1;
    o->half_spectrum = 1;
    o->tma_passes = 1;
    o->dt = 0.01;
    o->kappa = 1.0;
    o->dx = 1.0;
    o->beta2 = -21.7;
    o->gamma = 1.3;
    o->h = 0.1;
    o->dt_sample = 1.0;
    o->stream = nullptr;
    o->target_ratio = 0.0;
    o->control_eta = 0.05;
    o->control_every = 50;
    o->components = 8;
    o->rcd_d_diag = 0.5;
    o->rcd_d_cross = 0.05;
    o->rcd_alpha = 1.0;
    o->rcd_beta = 0.3;
    o->rcd_r = 1.0;
    o->rcd_a = 1.0;
}

static spdba_status check_opts(const spdba_options* o, int ndim) {
    if (!(o->target_ratio >= 0.0 && o->target_ratio <= 1.0))
        return fail(SPDBA_ERR_ARG, "target_ratio must lie in [0, 1]");
    if (o->target_ratio > 0 && (!(o->control_eta > 0.0 && o->control_eta < 1.0) || o->control_every < 1))
        return fail(SPDBA_ERR_ARG, "threshold control needs 0 < control_eta < 1 and control_every >= 1");
    if (o->model != SPDBA_MODEL_CH && o->model != SPDBA_MODEL_NLS && o->model != SPDBA_MODEL_RCD)
        return fail(SPDBA_ERR_ARG, "bad model %d", o->model);
    if (o->model == SPDBA_MODEL_RCD) {
        if (ndim < 2 || ndim > 3) return fail(SPDBA_ERR_UNSUPPORTED, "RCD plans are 2-D or 3-D");
        if (o->components < 1 || o->components > kRcdMaxComponents)
            return fail(SPDBA_ERR_UNSUPPORTED, "RCD with %d components (1..%d)", o->components, kRcdMaxComponents);
        if (o->measure != SPDBA_MEASURE_MAXAMP)
            return fail(SPDBA_ERR_ARG, "RCD activation uses the component RMS amplitude (SPDBA_MEASURE_MAXAMP)");
    }
    if (o->precision != SPDBA_C64 && o->precision != SPDBA_C128)
        return fail(SPDBA_ERR_ARG, "bad precision %d", o->precision);
    if (o->mode != SPDBA_MODE_REGULAR && o->mode != SPDBA_MODE_ADAPTIVE) return fail(SPDBA_ERR_ARG, "bad mode %d", o->mode);
    if (o->measure != SPDBA_MEASURE_MAXAMP && o->measure != SPDBA_MEASURE_ENERGY) return fail(SPDBA_ERR_ARG, "bad measure");
    if (o->tau_rule != SPDBA_TAU_REL_MAX && o->tau_rule != SPDBA_TAU_ABS) return fail(SPDBA_ERR_ARG, "bad tau rule");
    if (o->refresh_every < 0 || o->warmup_steps < 0) return fail(SPDBA_ERR_ARG, "negative refresh/warm-up");
    if (o->multi_pass < 0 || o->multi_pass > 2) return fail(SPDBA_ERR_ARG, "multi_pass must be 0, 1 or 2");
    if (o->half_storage < 0 || o->half_storage > 1) return fail(SPDBA_ERR_ARG, "half_storage must be 0 or 1");
    if (o->half_storage && (o->model != SPDBA_MODEL_CH || ndim != 3))
        return fail(SPDBA_ERR_UNSUPPORTED, "half-spectrum storage is built for 3-D Cahn-Hilliard plans");
    if (o->model == SPDBA_MODEL_CH && (ndim < 2 || ndim > 3)) return fail(SPDBA_ERR_UNSUPPORTED, "CH plans are 2-D or 3-D");
    if (o->model == SPDBA_MODEL_NLS && ndim != 1) return fail(SPDBA_ERR_UNSUPPORTED, "NLS plans are 1-D");
    return SPDBA_OK;
}

template <typename T>
static spdba_status build_groups(spdba_plan* p, int nruns, int ndim, const int64_t* dims, const int32_t* block) {
    auto& gs = groups<T>(p);
    // runs of equal extents share a group (3-D CH fields stay alone)
    std::vector<std::vector<int>> members;
    for (int r = 0; r < nruns; ++r) {
        const int64_t* d = dims + (size_t)r * ndim;
        int found = -1;
        if (!(p->opt.model == SPDBA_MODEL_CH && ndim == 3)) {
            for (size_t gi = 0; gi < members.size(); ++gi) {
                const int64_t* e = dims + (size_t)members[gi][0] * ndim;
                bool same = true;
                for (int a = 0; a < ndim; ++a) same = same && d[a] == e[a];
                if (same) { found = (int)gi; break; }
            }
        }
        if (found < 0) {
            found = (int)members.size();
            members.push_back({});
        }
        members[found].push_back(r);
    }
    p->runs.assign(nruns, RunRef{0, 0});
    for (size_t gi = 0; gi < members.size(); ++gi) {
        const int64_t* d = dims + (size_t)members[gi][0] * ndim;
        long long batch = (long long)members[gi].size();
        gs.emplace_back(new Group<T>());
        spdba_status s;
        if (p->opt.model == SPDBA_MODEL_RCD) {
            if (nruns != 1) return fail(SPDBA_ERR_UNSUPPORTED, "an RCD plan holds one field of M components");
            s = group_init_rcd<T>(p, *gs.back(), ndim, d, block);
        } else if (p->opt.model == SPDBA_MODEL_NLS) {
            if (block[0] > 0 && d[0] % block[0] != 0)
                return fail(SPDBA_ERR_UNSUPPORTED, "block edge %d does not divide %lld", block[0], (long long)d[0]);
            int nblk = block[0] <= 0 ? -block[0] : (int)(d[0] / block[0]);
            s = group_init_nls<T>(p, *gs.back(), d[0], nblk, batch);
        } else {
            s = group_init_ch<T>(p, *gs.back(), ndim, d, block, batch);
        }
        if (s != SPDBA_OK) return s;
        for (size_t k = 0; k < members[gi].size(); ++k) p->runs[members[gi][k]] = RunRef{(int)gi, (long long)k};
    }
    return SPDBA_OK;
}

extern "C" spdba_status spdba_batch_create(spdba_plan** out, int32_t nruns, int32_t ndim, const int64_t* dims,
                                           const int32_t* block, double threshold, int32_t reassess,
                                           const spdba_options* opt) {
    if (!out || !dims || !block || nruns < 1 || ndim < 1 || ndim > 3 || reassess < 1)
        return fail(SPDBA_ERR_ARG, "spdba_batch_create: bad arguments");
    spdba_options o;
    if (opt) o = *opt; else spdba_options_default(&o);
    spdba_status s = check_opts(&o, ndim);
    if (s != SPDBA_OK) return s;
    if (!(threshold >= 0)) return fail(SPDBA_ERR_ARG, "threshold must be >= 0");
    for (int r = 0; r < nruns; ++r)
        for (int a = 0; a < ndim; ++a) {
            int64_t d = dims[(size_t)r * ndim + a];
            if (!length_ok(d)) return fail(SPDBA_ERR_UNSUPPORTED, "length %lld is not 2^a 3^b", (long long)d);
        }
    spdba_plan* p = new spdba_plan();
    p->opt = o;
    p->rcd = RcdParams{o.rcd_r, o.rcd_a, o.rcd_alpha, o.rcd_beta};
    p->threshold = threshold;
    p->reassess = reassess;
    p->precision = o.precision;
    p->st = (cudaStream_t)o.stream;
    s = p->precision == SPDBA_C64 ? build_groups<float>(p, nruns, ndim, dims, block)
                                  : build_groups<double>(p, nruns, ndim, dims, block);
    if (s == SPDBA_OK && p->precision == SPDBA_C64 && ndim == 2) {
        // multi-size forms (tile tables of 4096 and 2048 elements)
        for (int k = 0; k < 2 && s == SPDBA_OK; ++k) s = build_multi(p, k == 0 ? 4096 : 2048, p->multi[k]);
        if (s == SPDBA_OK && o.multi_pass > 0 && o.fuse_update && p->multi[o.multi_pass - 1].ok)
            p->multi_sel = o.multi_pass;
    }
    p->opt.multi_pass = p->multi_sel;
    if (s == SPDBA_OK) {
        cudaError_t e = cudaStreamSynchronize(p->st);
        if (e != cudaSuccess) s = cuda_fail(e, "plan setup");
    }
    if (s != SPDBA_OK) {
        spdba_plan_destroy(p);
        return s;
    }
    *out = p;
    return SPDBA_OK;
}

extern "C" spdba_status spdba_plan_create(spdba_plan** out, int32_t ndim, const int64_t* dims, const int32_t* block,
                                          double threshold, int32_t reassess, const spdba_options* opt) {
    return spdba_batch_create(out, 1, ndim, dims, block, threshold, reassess, opt);
}

extern "C" void spdba_plan_destroy(spdba_plan* p) {
    if (!p) return;
    cudaStreamSynchronize(p->st);
    for (auto& g : p->g32) g->release();
    for (auto& g : p->g64) g->release();
    p->tw32.release();
    p->tw64.release();
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    if (p->seg_exec) cudaGraphExecDestroy(p->seg_exec);
    for (cudaStream_t gs : p->gstreams) {
        cudaStreamSynchronize(gs);
        cudaStreamDestroy(gs);
    }
    for (cudaEvent_t e : p->gevents) cudaEventDestroy(e);
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    for (void* b : p->multi_bufs) dev_free(b);
    delete p;
}

static bool run_ok(spdba_plan* p, int32_t run) { return run >= 0 && run < p->nruns(); }

// Calls F(group, sub) with the run's group of the plan's precision.
template <typename F> static spdba_status with_run(spdba_plan* p, int32_t run, F f) {
    const RunRef& rr = p->runs[run];
    if (p->precision == SPDBA_C64) return f(*p->g32[rr.group], rr.sub);
    return f(*p->g64[rr.group], rr.sub);
}

extern "C" spdba_status spdba_set_field(spdba_plan* p, int32_t run, const void* src, int32_t on_dev) {
    PLAN_CHECK(p);
    if (!src || !run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_set_field: bad arguments");
    return latch(p, with_run(p, run, [&](auto& G, long long sub) { return run_set_field(p, G, sub, src, on_dev); }));
}

extern "C" spdba_status spdba_step(spdba_plan* p, int64_t n) {
    PLAN_CHECK(p);
    if (n < 0) return fail(SPDBA_ERR_ARG, "negative step count");
    spdba_status s = p->precision == SPDBA_C64 ? plan_step<float>(p, n) : plan_step<double>(p, n);
    return latch(p, s);
}

// ------------------------------------------------------------------ autotuner
// Device state of a group copied aside, so that trial steps can be undone.
struct GroupSnap {
    std::vector<std::pair<void*, size_t>> bufs;   // (source, bytes)
    std::vector<void*> copies;
    int64_t step = 0;
    bool assessed = false;
    void release() {
        for (void* q : copies) dev_free(q);
        copies.clear();
    }
};

template <typename T> static spdba_status snap_take(spdba_plan* p, Group<T>& r, GroupSnap& sn) {
    const long long nb = r.g.blocks();
    sn.bufs = {{r.c_hat, sizeof(cx_t<T>) * (size_t)(r.batch * r.n * r.ncomp)},
               {r.stats, sizeof(DevStats) * (size_t)r.batch},
               {r.maxsq, sizeof(double) * (size_t)nb},
               {r.sumsq, sizeof(double) * (size_t)nb},
               {r.gmax, sizeof(double) * 2 * (size_t)r.batch},
               {r.tau, sizeof(double) * (size_t)r.batch},
               {r.active, (size_t)nb},
               {r.states, (size_t)nb},
               {r.chi, (size_t)nb},
               {r.list, sizeof(int32_t) * (size_t)nb},
               {r.count, sizeof(int32_t) * 2}};
    if (r.pair_list) {
        sn.bufs.push_back({r.pair_list, sizeof(int) * (size_t)r.pair_list_n});
        sn.bufs.push_back({r.pair_count, sizeof(int)});
    }
    // the forward passes' liveness follows the states in force: a tuning started
    // between reassessments resumes with the states of the snapshot, so their
    // liveness is restored with them
    if (r.col_live) sn.bufs.push_back({r.col_live, (size_t)r.h_fwd_y.p.I});
    if (r.hs_zlive) {
        sn.bufs.push_back({r.hs_zlive, (size_t)(r.g.n[1] * r.g.n[2])});
        sn.bufs.push_back({r.hs_xlive, (size_t)r.g.n[2]});
    }
    for (auto& b : sn.bufs) {
        void* q = nullptr;
        cudaError_t e = dev_alloc(&q, b.second);
        if (e != cudaSuccess) { sn.release(); return cuda_fail(e, "device allocation (autotune snapshot)"); }
        sn.copies.push_back(q);
        SPDBA_CUDA(cudaMemcpyAsync(q, b.first, b.second, cudaMemcpyDeviceToDevice, p->st));
    }
    sn.step = r.step;
    sn.assessed = r.assessed;
    return SPDBA_OK;
}

template <typename T> static spdba_status snap_restore(spdba_plan* p, Group<T>& r, const GroupSnap& sn) {
    for (size_t i = 0; i < sn.bufs.size(); ++i)
        SPDBA_CUDA(cudaMemcpyAsync(sn.bufs[i].first, sn.copies[i], sn.bufs[i].second, cudaMemcpyDeviceToDevice, p->st));
    r.step = sn.step;
    r.assessed = sn.assessed;
    return SPDBA_OK;
}

template <typename T> static void apply_config(spdba_plan* p, int fuse, int graph, int half, int tma, int multi) {
    for (auto& g : groups<T>(p)) {
        g->fused_update = fuse && g->has_fused;
        g->use_half = half && g->has_half;
        g->use_tma = tma && g->tma_ok;
    }
    p->multi_sel = (multi > 0 && fuse && p->multi[multi - 1].ok) ? multi : 0;
    p->opt.multi_pass = p->multi_sel;
    p->opt.use_graph = graph;
    if (p->seg_exec) {
        cudaGraphExecDestroy(p->seg_exec);
        p->seg_exec = nullptr;
    }
}

// ------------------------------------------------------------------ tuning cache
struct TunedConfig {
    int fuse, graph, half, tma, multi;
    double ms;
};
static std::map<std::string, TunedConfig>& tune_cache() {
    static std::map<std::string, TunedConfig> m;
    return m;
}
// What the candidate set and their timings depend on: precision, model, mode,
// dimensionality, block edges, each group's run extents and run count, the
// options that enable candidates and whether graphs are possible.
static std::string plan_signature(spdba_plan* p) {
    std::string k;
    char buf[96];
    snprintf(buf, sizeof buf, "p%d m%d md%d f%d h%d hs%d s%d|", p->precision, p->opt.model, p->opt.mode,
             p->opt.fuse_update, p->opt.half_spectrum, p->opt.half_storage, p->st == 0 ? 0 : 1);
    k += buf;
    auto add_groups = [&](auto& gs) {
        for (auto& g : gs) {
            snprintf(buf, sizeof buf, "d%d:%lld,%lld,%lld b%d,%d,%d x%lld;", g->ndim, (long long)g->dims[0],
                     (long long)g->dims[1], (long long)g->dims[2], g->g.b[0], g->g.b[1], g->g.b[2],
                     (long long)g->batch);
            k += buf;
        }
    };
    add_groups(p->g32);
    add_groups(p->g64);
    return k;
}

// Times `steps` steps (after a warm-up segment that also captures a graph)
// for every candidate (update form x graph replay) from the same state, then
// keeps the fastest and restores the state.
template <typename T> static spdba_status autotune_t(spdba_plan* p, int32_t steps, spdba_tune_report* rep) {
    auto& gs = groups<T>(p);
    bool any_fused = false, any_half = false, any_tma = false;
    for (auto& g : gs) {
        any_fused |= g->has_fused;
        any_half |= g->has_half;
        any_tma |= g->tma_ok;
    }
    struct Cand { int fuse, graph, half, tma, multi; };
    std::vector<Cand> cand;
    for (int hf : {1, 0}) {
        if (hf && !any_half) continue;
        for (int f : {1, 0}) {
            if (f && !any_fused) continue;
            for (int gr : {1, 0}) {
                if (gr && p->st == 0) continue;   // graphs need a non-legacy stream
                // the staged form's list-driven update: warp kernel or TMA kernel
                for (int tm : {0, 1}) {
                    if (tm && (f || !any_tma)) continue;
                    cand.push_back({f, gr, hf, tm, 0});
                }
                // the fused form of a batched 2-D plan: one launch per phase over all groups
                for (int mu : {1, 2})
                    if (f && !hf && p->multi[mu - 1].ok) cand.push_back({f, gr, hf, 0, mu});
            }
        }
    }
    if ((int)cand.size() > SPDBA_TUNE_MAX) cand.resize(SPDBA_TUNE_MAX);
    std::vector<GroupSnap> snaps(gs.size());
    spdba_status s = SPDBA_OK;
    for (size_t i = 0; i < gs.size() && s == SPDBA_OK; ++i) s = snap_take<T>(p, *gs[i], snaps[i]);
    const long long launches0 = p->launches;
    const int R = p->reassess;
    std::vector<double> ms(cand.size(), 0.0);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (s == SPDBA_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        s = fail(SPDBA_ERR_CUDA, "autotune: cudaEventCreate failed");
    for (size_t c = 0; c < cand.size() && s == SPDBA_OK; ++c) {
        apply_config<T>(p, cand[c].fuse, cand[c].graph, cand[c].half, cand[c].tma, cand[c].multi);
        if ((s = plan_step<T>(p, R)) != SPDBA_OK) break;   // warm-up (graph capture)
        for (size_t i = 0; i < gs.size() && s == SPDBA_OK; ++i) s = snap_restore<T>(p, *gs[i], snaps[i]);
        if (s != SPDBA_OK) break;
        cudaEventRecord(e0, p->st);
        if ((s = plan_step<T>(p, steps)) != SPDBA_OK) break;
        cudaEventRecord(e1, p->st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { s = cuda_fail(e, "autotune sync"); break; }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms[c] = t / (double)steps;
        for (size_t i = 0; i < gs.size() && s == SPDBA_OK; ++i) s = snap_restore<T>(p, *gs[i], snaps[i]);
    }
    size_t best = 0;
    for (size_t c = 1; c < cand.size(); ++c)
        if (ms[c] < ms[best]) best = c;
    if (s == SPDBA_OK && !cand.empty())
        apply_config<T>(p, cand[best].fuse, cand[best].graph, cand[best].half, cand[best].tma, cand[best].multi);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaError_t e = cudaStreamSynchronize(p->st);
    for (auto& sn : snaps) sn.release();
    p->launches = launches0;
    if (s != SPDBA_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "autotune sync");
    if (rep) {
        memset(rep, 0, sizeof *rep);
        rep->n_candidates = (int32_t)cand.size();
        for (size_t c = 0; c < cand.size(); ++c) {
            rep->fuse_update[c] = cand[c].fuse;
            rep->use_graph[c] = cand[c].graph;
            rep->half_spectrum[c] = cand[c].half;
            rep->tma_update[c] = cand[c].tma;
            rep->multi_pass[c] = cand[c].multi;
            rep->ms_per_step[c] = ms[c];
        }
        rep->chosen = (int32_t)best;
    }
    if (!cand.empty()) {
        const Cand& b = cand[best];
        tune_cache()[plan_signature(p)] = TunedConfig{b.fuse, b.graph, b.half, b.tma, b.multi, ms[best]};
    }
    return SPDBA_OK;
}

extern "C" spdba_status spdba_plan_autotune(spdba_plan* p, int32_t steps, spdba_tune_report* report) {
    PLAN_CHECK(p);
    if (steps < 1) return fail(SPDBA_ERR_ARG, "spdba_plan_autotune: steps must be >= 1");
    if (p->pred) return fail(SPDBA_ERR_STATE, "spdba_plan_autotune: detach the predictor first");
    if (p->prof) return fail(SPDBA_ERR_STATE, "spdba_plan_autotune: a profile is open");
    spdba_status s = p->precision == SPDBA_C64 ? autotune_t<float>(p, steps, report) : autotune_t<double>(p, steps, report);
    return latch(p, s);
}

extern "C" spdba_status spdba_plan_autotune_cached(spdba_plan* p, int32_t steps, spdba_tune_report* report) {
    PLAN_CHECK(p);
    if (steps < 1) return fail(SPDBA_ERR_ARG, "spdba_plan_autotune_cached: steps must be >= 1");
    if (p->pred) return fail(SPDBA_ERR_STATE, "spdba_plan_autotune_cached: detach the predictor first");
    if (p->prof) return fail(SPDBA_ERR_STATE, "spdba_plan_autotune_cached: a profile is open");
    auto it = tune_cache().find(plan_signature(p));
    if (it == tune_cache().end()) return spdba_plan_autotune(p, steps, report);
    const TunedConfig& c = it->second;
    if (p->precision == SPDBA_C64) apply_config<float>(p, c.fuse, c.graph, c.half, c.tma, c.multi);
    else apply_config<double>(p, c.fuse, c.graph, c.half, c.tma, c.multi);
    if (report) {
        memset(report, 0, sizeof *report);
        report->n_candidates = 1;
        report->fuse_update[0] = c.fuse;
        report->use_graph[0] = c.graph;
        report->half_spectrum[0] = c.half;
        report->tma_update[0] = c.tma;
        report->multi_pass[0] = c.multi;
        report->ms_per_step[0] = c.ms;
        report->chosen = 0;
        report->cached = 1;
    }
    return SPDBA_OK;
}

extern "C" void spdba_tune_cache_clear(void) { tune_cache().clear(); }

extern "C" spdba_status spdba_plan_get_config(const spdba_plan* p, spdba_options* out) {
    if (!p || !out) return fail(SPDBA_ERR_ARG, "spdba_plan_get_config: bad arguments");
    *out = p->opt;
    int fuse = 0, half = 0, tma = 0, tmap = 0;
    auto scan = [&](auto& gs) {
        for (auto& g : gs) {
            fuse |= g->fused_update ? 1 : 0;
            half |= g->use_half ? 1 : 0;
            tma |= g->use_tma ? 1 : 0;
            tmap |= g->use_half && g->use_herm_tma ? 1 : 0;
        }
    };
    scan(p->g32);
    scan(p->g64);
    out->fuse_update = fuse;
    out->half_spectrum = half;
    out->tma_update = tma;
    out->tma_passes = tmap;
    int hs = 0;
    for (auto& g : p->g32) hs |= g->hs ? 1 : 0;
    out->half_storage = hs;
    out->multi_pass = p->multi_sel;
    return SPDBA_OK;
}

extern "C" spdba_status spdba_get_field(spdba_plan* p, int32_t run, void* dst, int32_t on_dev) {
    PLAN_CHECK(p);
    if (!dst || !run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_get_field: bad arguments");
    return latch(p, with_run(p, run, [&](auto& G, long long sub) { return run_get_field(p, G, sub, dst, on_dev); }));
}

extern "C" spdba_status spdba_get_spectrum(spdba_plan* p, int32_t run, void* dst, int32_t on_dev) {
    PLAN_CHECK(p);
    if (!dst || !run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_get_spectrum: bad arguments");
    return latch(p, with_run(p, run, [&](auto& G, long long sub) { return copy_spectrum(p, G, sub, dst, on_dev, true); }));
}

extern "C" spdba_status spdba_set_spectrum(spdba_plan* p, int32_t run, const void* src, int32_t on_dev) {
    PLAN_CHECK(p);
    if (!src || !run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_set_spectrum: bad arguments");
    return latch(p, with_run(p, run,
                             [&](auto& G, long long sub) { return copy_spectrum(p, G, sub, (void*)src, on_dev, false); }));
}

template <typename T>
static spdba_status get_mask_t(spdba_plan* p, Group<T>& r, long long sub, uint8_t* dst, int64_t nb) {
    if (r.hs) {
        // the half map's live x-blocks, row by row
        if (nb != r.g.live_bpr())
            return fail(SPDBA_ERR_ARG, "mask size %lld != %lld blocks", (long long)nb, r.g.live_bpr());
        SPDBA_CUDA(cudaMemcpy2DAsync(dst, (size_t)r.g.hx, r.states, (size_t)r.g.nb[2], (size_t)r.g.hx,
                                     (size_t)(r.g.nb[0] * r.g.nb[1]), cudaMemcpyDeviceToHost, p->st));
        SPDBA_CUDA(cudaStreamSynchronize(p->st));
        return SPDBA_OK;
    }
    if (nb != r.g.bpr()) return fail(SPDBA_ERR_ARG, "mask size %lld != %lld blocks", (long long)nb, r.g.bpr());
    SPDBA_CUDA(cudaMemcpyAsync(dst, r.states + sub * r.g.bpr(), (size_t)nb, cudaMemcpyDeviceToHost, p->st));
    SPDBA_CUDA(cudaStreamSynchronize(p->st));
    return SPDBA_OK;
}

extern "C" spdba_status spdba_get_mask(spdba_plan* p, int32_t run, uint8_t* dst, int64_t nb) {
    PLAN_CHECK(p);
    if (!dst || !run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_get_mask: bad arguments");
    return latch(p, with_run(p, run, [&](auto& G, long long sub) { return get_mask_t(p, G, sub, dst, nb); }));
}

template <typename T> static spdba_status get_stats_t(spdba_plan* p, Group<T>& r, long long sub, spdba_stats* out) {
    DevStats d;
    SPDBA_CUDA(cudaMemcpyAsync(&d, r.stats + sub, sizeof d, cudaMemcpyDeviceToHost, p->st));
    SPDBA_CUDA(cudaStreamSynchronize(p->st));
    out->step = r.step;
    out->assessments = (int64_t)d.assessments;
    out->nblocks = r.g.live_bpr();
    out->n_active = (int64_t)d.n_active;
    out->n_transition = (int64_t)d.n_transition;
    out->tau = d.tau;
    out->max_amp = d.max_amp;
    out->mass = d.mass;
    out->active_ratio_sum = d.ratio_sum;
    out->predictions = (int64_t)d.predictions;
    out->missed_blocks = (int64_t)d.missed;
    out->threshold = d.eps;
    out->controls = (int64_t)d.controls;
    if (d.timeouts) return fail(SPDBA_ERR_TIMEOUT, "a bounded device wait ran out (%llu times)", d.timeouts);
    return SPDBA_OK;
}

extern "C" spdba_status spdba_get_stats(spdba_plan* p, int32_t run, spdba_stats* out) {
    PLAN_CHECK(p);
    if (!out || !run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_get_stats: bad arguments");
    return latch(p, with_run(p, run, [&](auto& G, long long sub) { return get_stats_t(p, G, sub, out); }));
}

template <typename T> static spdba_status list_bytes_now(spdba_plan* p, double* out) {
    *out = 0;
    for (auto& g : groups<T>(p)) {
        std::vector<DevStats> d((size_t)g->batch);
        SPDBA_CUDA(cudaMemcpyAsync(d.data(), g->stats, sizeof(DevStats) * d.size(), cudaMemcpyDeviceToHost, p->st));
        SPDBA_CUDA(cudaStreamSynchronize(p->st));
        for (auto& x : d) *out += 3.0 * sizeof(cx_t<T>) * x.list_modes;
    }
    return SPDBA_OK;
}

extern "C" spdba_status spdba_profile_begin(spdba_plan* p) { return spdba_profile_begin_sampled(p, 1); }

extern "C" spdba_status spdba_profile_begin_sampled(spdba_plan* p, int32_t every) {
    PLAN_CHECK(p);
    if (every < 1) return fail(SPDBA_ERR_ARG, "profile sampling interval must be >= 1");
    p->prof_every = every;
    p->prof_on = every == 1;
    p->prof_recs.clear();
    p->ev_used = 0;
    p->launches = 0;
    p->prof_list0 = p->list_updates;
    spdba_status s = p->precision == SPDBA_C64 ? list_bytes_now<float>(p, &p->prof_list_bytes0)
                                               : list_bytes_now<double>(p, &p->prof_list_bytes0);
    if (s != SPDBA_OK) return latch(p, s);
    p->prof = true;
    return SPDBA_OK;
}

extern "C" spdba_status spdba_profile_end(spdba_plan* p, spdba_kernel_time* out, int32_t capacity, int32_t* n_out,
                                          int64_t* launches_out) {
    PLAN_CHECK(p);
    if (!p->prof) return fail(SPDBA_ERR_STATE, "profiling was not started");
    p->prof = false;
    p->prof_on = false;
    cudaError_t e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) return latch(p, cuda_fail(e, "profile sync"));
    spdba_kernel_time agg[K_COUNT];
    memset(agg, 0, sizeof agg);
    for (int k = 0; k < K_COUNT; ++k) snprintf(agg[k].name, sizeof agg[k].name, "%s", kProfName[k]);
    for (auto& r : p->prof_recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
        agg[r.kind].launches += 1;
        agg[r.kind].total_ms += ms;
        agg[r.kind].bytes += r.bytes;
    }
    double lb = 0;
    spdba_status s = p->precision == SPDBA_C64 ? list_bytes_now<float>(p, &lb) : list_bytes_now<double>(p, &lb);
    if (s != SPDBA_OK) return latch(p, s);
    // the device counts the list traffic of every step; keep the timed (sampled) steps' share
    const long long all_list = p->list_updates - p->prof_list0;
    if (all_list > 0)
        agg[K_UPDATE_LIST].bytes += (lb - p->prof_list_bytes0) * (double)agg[K_UPDATE_LIST].launches / (double)all_list;
    int n = 0;
    for (int k = 0; k < K_COUNT && n < capacity; ++k)
        if (agg[k].launches > 0 && out) out[n++] = agg[k];
    if (n_out) *n_out = n;
    if (launches_out) *launches_out = p->launches;
    return SPDBA_OK;
}

template <typename T>
static spdba_status get_activity_t(spdba_plan* p, Group<T>& r, long long sub, double* maxsq, double* tau, int on_dev) {
    const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const long long bpr = r.g.bpr();
    // with a predictor attached, the last exact scan is kept in the snapshot
    const double* src = r.has_snap ? r.snap_maxsq : r.maxsq;
    const double* tsrc = r.has_snap ? r.snap_tau : r.tau;
    if (maxsq && r.hs) {
        // the half map's live x-blocks, row by row
        const size_t es = sizeof(double);
        SPDBA_CUDA(cudaMemcpy2DAsync(maxsq, es * (size_t)r.g.hx, src, es * (size_t)r.g.nb[2], es * (size_t)r.g.hx,
                                     (size_t)(r.g.nb[0] * r.g.nb[1]), kind, p->st));
        maxsq = nullptr;
    }
    if (maxsq) SPDBA_CUDA(cudaMemcpyAsync(maxsq, src + sub * bpr, sizeof(double) * bpr, kind, p->st));
    if (tau) SPDBA_CUDA(cudaMemcpyAsync(tau, tsrc + sub, sizeof(double), kind, p->st));
    SPDBA_CUDA(cudaStreamSynchronize(p->st));
    return SPDBA_OK;
}

extern "C" spdba_status spdba_get_activity(spdba_plan* p, int32_t run, double* maxsq, double* tau, int32_t on_dev) {
    PLAN_CHECK(p);
    if (!run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_get_activity: bad run");
    return latch(p, with_run(p, run, [&](auto& G, long long sub) { return get_activity_t(p, G, sub, maxsq, tau, on_dev); }));
}

template <typename T> static spdba_status attach_t(spdba_plan* p, spdba_predictor* pr) {
    auto& gs = groups<T>(p);
    if (gs.size() != 1 || gs[0]->ndim != 3 || gs[0]->batch != 1 || p->opt.model != SPDBA_MODEL_CH)
        return fail(SPDBA_ERR_UNSUPPORTED, "a predictor attaches to a 3-D Cahn-Hilliard plan with one run");
    if (p->opt.target_ratio > 0)
        return fail(SPDBA_ERR_STATE, "a predictor does not attach to a plan under dynamic threshold control");
    Group<T>& r = *gs[0];
    if (r.hs) return fail(SPDBA_ERR_UNSUPPORTED, "a predictor attaches to a plan with full-spectrum storage");
    if (!spdba_predictor_map_matches(pr, r.g.nb[0], r.g.nb[1], r.g.nb[2]))
        return fail(SPDBA_ERR_ARG, "predictor block map does not match the plan's");
    const long long nb = r.g.blocks();
    spdba_status s;
    if (!r.snap_maxsq) {
        if ((s = r.alloc(&r.snap_maxsq, sizeof(double) * nb)) != SPDBA_OK) return s;
        if ((s = r.alloc(&r.snap_tau, sizeof(double))) != SPDBA_OK) return s;
        if ((s = r.alloc(&r.pmeasure, sizeof(double) * nb)) != SPDBA_OK) return s;
        if ((s = r.alloc(&r.pthr, sizeof(double))) != SPDBA_OK) return s;
        if ((s = r.alloc(&r.pstates, nb)) != SPDBA_OK) return s;
        if ((s = r.alloc(&r.px, 2 * 2 * nb)) != SPDBA_OK) return s;   // bf16 x 2 channels
    }
    double thr = (double)p->prob_thr;
    SPDBA_CUDA(cudaMemcpy(r.pthr, &thr, sizeof(double), cudaMemcpyHostToDevice));
    r.has_snap = false;
    r.has_pred = false;
    r.assessed = false;
    return SPDBA_OK;
}

extern "C" spdba_status spdba_plan_attach_predictor(spdba_plan* p, spdba_predictor* pr, int32_t horizon,
                                                   int32_t judge_every, float prob_threshold) {
    PLAN_CHECK(p);
    if (!pr) {
        p->pred = nullptr;
        return SPDBA_OK;
    }
    if (horizon < 1 || judge_every < horizon || judge_every % horizon != 0 || !(prob_threshold > 0.f))
        return fail(SPDBA_ERR_ARG, "attach: need horizon >= 1, judge_every a multiple of horizon, threshold > 0");
    p->horizon = horizon;
    p->judge_every = judge_every;
    p->prob_thr = prob_threshold;
    spdba_status s = p->precision == SPDBA_C64 ? attach_t<float>(p, pr) : attach_t<double>(p, pr);
    if (s != SPDBA_OK) return latch(p, s);
    p->pred = pr;
    return SPDBA_OK;
}

extern "C" spdba_status spdba_sync(spdba_plan* p) {
    PLAN_CHECK(p);
    cudaError_t e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) return latch(p, cuda_fail(e, "cudaStreamSynchronize"));
    return SPDBA_OK;
}
