// sp-DBA plan: owns the device buffers of one or more fields and runs the
// time loop of the paper's solver integration (S2.1): per step a pre-update
// (inverse transform, real-space nonlinearity, forward transform), then the
// update dispatched by mode (Regular: every mode; sp-DBA: state preparation at
// each reassessment, then the blockwise update of the listed blocks).
#include <stdio.h>
#include <string.h>

#include <memory>
#include <vector>

#include "blocks.h"

namespace spdba {

// ------------------------------------------------------------------ small kernels
template <typename T> __global__ void real_to_complex_kernel(const T* __restrict__ r, cx_t<T>* __restrict__ c, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c[i] = mk<cx_t<T>>(r[i], (T)0);
}
template <typename T> __global__ void complex_real_part_kernel(const cx_t<T>* __restrict__ c, T* __restrict__ r, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        r[i] = c[i].x;
}
__global__ void zero_double_kernel(double* p, int n) {
    if ((int)threadIdx.x < n) p[threadIdx.x] = 0.0;
}

static unsigned grid_for(long long n, int nt) {
    long long g = (n + nt - 1) / nt;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// ------------------------------------------------------------------ one field
template <typename T> struct Run {
    using C = cx_t<T>;
    Geom g;
    int ndim = 0;
    int64_t dims[3] = {1, 1, 1};
    long long n = 0;
    C* c_hat = nullptr;     // transformed field (the solver state)
    C* work = nullptr;      // transform workspace: c, g, g_hat
    T* real = nullptr;      // real-space staging for set/get_field
    double* maxsq = nullptr;
    double* sumsq = nullptr;
    double* dbl = nullptr;  // gmax[2], tau
    uint8_t* active = nullptr;
    uint8_t* states = nullptr;
    uint8_t* chi = nullptr;
    int32_t* list = nullptr;
    int32_t* count = nullptr;
    void* scratch = nullptr;
    DevStats* stats = nullptr;
    T* k2ax[3] = {nullptr, nullptr, nullptr};
    T* taper[3] = {nullptr, nullptr, nullptr};
    // CH pre-update passes
    std::vector<Pass<T>> pre_inv;   // inverse passes before the fused one (first reads c_hat)
    Pass<T> fused;                  // inverse + nonlinearity + forward along the fast axis
    std::vector<Pass<T>> pre_fwd;   // remaining forward passes
    FftEngine<T> fft;               // full transforms for set/get_field
    int64_t step = 0;
    bool assessed = false;
    std::vector<void*> allocs;

    template <typename P> spdba_status alloc(P** p, size_t bytes) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        allocs.push_back(q);
        *p = (P*)q;
        return SPDBA_OK;
    }
    void release() {
        for (void* p : allocs) cudaFree(p);
        allocs.clear();
        fft.release();
    }
};

}  // namespace spdba

using namespace spdba;

enum ProfKind { K_FFT_PASS = 0, K_FUSED_NL, K_UPDATE_DENSE, K_UPDATE_LIST, K_ASSESS, K_COUNT };
static const char* kProfName[K_COUNT] = {"fft_pass", "fft_fused_nl", "update_dense", "update_list", "assess"};

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double bytes;
};

struct spdba_plan {
    spdba_options opt;
    bool prof = false;
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    long long launches = 0;
    std::vector<double> prof_list_modes0;
    double threshold = 0;
    int reassess = 1;
    int precision = SPDBA_C64;
    cudaStream_t st = 0;
    spdba_status latched = SPDBA_OK;
    std::vector<std::unique_ptr<Run<float>>> r32;
    std::vector<std::unique_ptr<Run<double>>> r64;
    TwiddleCache<float> tw32;
    TwiddleCache<double> tw64;
    int nruns() const { return precision == SPDBA_C64 ? (int)r32.size() : (int)r64.size(); }
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
        if (p->prof && (a = ev_get(p)) != nullptr) cudaEventRecord(a, p->st);
    }
    ~ProfScope() {
        if (!p->prof || !a) return;
        cudaEvent_t b = ev_get(p);
        if (!b) return;
        cudaEventRecord(b, p->st);
        p->prof_recs.push_back(ProfRec{kind, a, b, bytes});
    }
};

template <typename T> static std::vector<std::unique_ptr<Run<T>>>& runs(spdba_plan* p);
template <> std::vector<std::unique_ptr<Run<float>>>& runs<float>(spdba_plan* p) { return p->r32; }
template <> std::vector<std::unique_ptr<Run<double>>>& runs<double>(spdba_plan* p) { return p->r64; }
template <typename T> static TwiddleCache<T>& twc(spdba_plan* p);
template <> TwiddleCache<float>& twc<float>(spdba_plan* p) { return p->tw32; }
template <> TwiddleCache<double>& twc<double>(spdba_plan* p) { return p->tw64; }

template <typename T>
static spdba_status upload(Run<T>& r, T** dst, const std::vector<T>& v, cudaStream_t st) {
    spdba_status s = r.alloc(dst, sizeof(T) * v.size());
    if (s != SPDBA_OK) return s;
    SPDBA_CUDA(cudaMemcpyAsync(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
    return SPDBA_OK;
}

template <typename T>
static spdba_status run_init(spdba_plan* p, Run<T>& r, int ndim, const int64_t* dims, const int32_t* block) {
    cudaStream_t st = p->st;
    spdba_status s = make_geom(&r.g, ndim, dims, block);
    if (s != SPDBA_OK) return s;
    r.ndim = ndim;
    r.n = 1;
    for (int a = 0; a < ndim; ++a) { r.dims[a] = dims[a]; r.n *= dims[a]; }
    const long long nb = r.g.blocks();
    if ((s = r.alloc(&r.c_hat, sizeof(cx_t<T>) * r.n)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.work, sizeof(cx_t<T>) * r.n)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.real, sizeof(T) * r.n)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.maxsq, sizeof(double) * nb)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.sumsq, sizeof(double) * nb)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.dbl, sizeof(double) * 4)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.active, nb)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.states, nb)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.chi, nb)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.list, sizeof(int32_t) * nb)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.count, sizeof(int32_t) * 2)) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.scratch, classify_scratch_bytes(nb))) != SPDBA_OK) return s;
    if ((s = r.alloc(&r.stats, sizeof(DevStats))) != SPDBA_OK) return s;
    SPDBA_CUDA(cudaMemsetAsync(r.c_hat, 0, sizeof(cx_t<T>) * r.n, st));
    SPDBA_CUDA(cudaMemsetAsync(r.stats, 0, sizeof(DevStats), st));
    SPDBA_CUDA(cudaMemsetAsync(r.states, SPDBA_ACTIVE, nb, st));
    for (int ax = 0; ax < 3; ++ax) {
        if ((s = upload<T>(r, &r.k2ax[ax], k2_table<T>(r.g.n[ax], p->opt.dx), st)) != SPDBA_OK) return s;
        if ((s = upload<T>(r, &r.taper[ax], taper_table<T>(r.g.b[ax]), st)) != SPDBA_OK) return s;
    }
    TwiddleCache<T>& tw = twc<T>(p);
    if ((s = r.fft.init(ndim, dims, 1, tw, st)) != SPDBA_OK) return s;
    if (p->opt.model == SPDBA_MODEL_CH) {
        // inverse along axes 0..d-2, fused inverse/NL/forward along d-1, forward d-2..0
        for (int a = 0; a < ndim - 1; ++a) {
            Pass<T> ps;
            if ((s = make_axis_pass<T>(&ps, ndim, dims, 1, a, +1, PASS_PLAIN, tw, st)) != SPDBA_OK) return s;
            r.pre_inv.push_back(ps);
        }
        if ((s = make_axis_pass<T>(&r.fused, ndim, dims, 1, ndim - 1, -1, PASS_CH_NL, tw, st)) != SPDBA_OK) return s;
        r.fused.p.nl_scale = (T)(1.0 / (double)r.n);
        for (int a = ndim - 2; a >= 0; --a) {
            Pass<T> ps;
            if ((s = make_axis_pass<T>(&ps, ndim, dims, 1, a, -1, PASS_PLAIN, tw, st)) != SPDBA_OK) return s;
            r.pre_fwd.push_back(ps);
        }
    }
    return SPDBA_OK;
}

// State preparation (Methods): activity, threshold, states, list.
template <typename T> static spdba_status run_assess(spdba_plan* p, Run<T>& r) {
    cudaStream_t st = p->st;
    spdba_status s;
    ProfScope ps(p, K_ASSESS, (double)sizeof(cx_t<T>) * (double)r.n);
    p->launches += 7;
    double* gmax = r.dbl;
    double* tau = r.dbl + 2;
    zero_double_kernel<<<1, 32, 0, st>>>(gmax, 2);
    double* sumsq = p->opt.measure == SPDBA_MEASURE_ENERGY ? r.sumsq : nullptr;
    if ((s = launch_block_activity<T>(r.g, r.c_hat, r.maxsq, sumsq, gmax, st)) != SPDBA_OK) return s;
    int exclude_dc = p->opt.model == SPDBA_MODEL_CH ? 1 : 0;
    if ((s = launch_tau(gmax, p->threshold, p->opt.tau_rule, exclude_dc, tau, r.stats, st)) != SPDBA_OK) return s;
    const double* msq = p->opt.measure == SPDBA_MEASURE_ENERGY ? r.sumsq : r.maxsq;
    return launch_classify(r.g, msq, 1, tau, p->opt.force_dc, p->opt.transitions, 0, r.active, r.states, r.chi,
                           r.list, r.count, r.scratch, r.stats, st);
}

template <typename T> static spdba_status run_ch_step(spdba_plan* p, Run<T>& r) {
    cudaStream_t st = p->st;
    spdba_status s;
    const bool adaptive = p->opt.mode == SPDBA_MODE_ADAPTIVE;
    const bool reassess = adaptive && (!r.assessed || r.step % p->reassess == 0);
    const bool all_active = r.step < p->opt.warmup_steps ||
                            (p->opt.refresh_every > 0 && r.step > 0 && r.step % p->opt.refresh_every == 0);
    if (reassess) {
        if ((s = run_assess<T>(p, r)) != SPDBA_OK) return s;
        r.assessed = true;
    }
    // pre-update: c = Re(IFFT(c_hat)), g = c^3 - c, g_hat = FFT(g)
    const double pass_bytes = 2.0 * sizeof(cx_t<T>) * (double)r.n;
    const cx_t<T>* src = r.c_hat;
    for (auto& ps : r.pre_inv) {
        ProfScope pr(p, K_FFT_PASS, pass_bytes);
        if ((s = launch_pass<T>(ps, src, r.work, st)) != SPDBA_OK) return s;
        p->launches += 1;
        src = r.work;
    }
    Pass<T> fused = r.fused;
    if (reassess) {
        fused.p.mass = &r.stats->mass;
        zero_double_kernel<<<1, 32, 0, st>>>(&r.stats->mass, 1);
        p->launches += 1;
    }
    {
        ProfScope pr(p, K_FUSED_NL, pass_bytes);
        if ((s = launch_pass<T>(fused, src, r.work, st)) != SPDBA_OK) return s;
        p->launches += 1;
    }
    for (auto& ps : r.pre_fwd) {
        ProfScope pr(p, K_FFT_PASS, pass_bytes);
        if ((s = launch_pass<T>(ps, r.work, r.work, st)) != SPDBA_OK) return s;
        p->launches += 1;
    }
    // update
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
    a.inv_nblocks = 1.0 / (double)r.g.blocks();
    const int dense = !adaptive || all_active;
    {
        // list-update traffic is known only on the device; it is added at profile end
        ProfScope pr(p, dense ? K_UPDATE_DENSE : K_UPDATE_LIST, dense ? 3.0 * sizeof(cx_t<T>) * (double)r.n : 0.0);
        if ((s = launch_ch_update<T>(r.g, a, dense, st)) != SPDBA_OK) return s;
        p->launches += 1;
    }
    r.step += 1;
    return SPDBA_OK;
}

template <typename T> static spdba_status plan_step(spdba_plan* p, int64_t n) {
    auto& rs = runs<T>(p);
    for (int64_t i = 0; i < n; ++i) {
        for (auto& r : rs) {
            spdba_status s = SPDBA_OK;
            if (p->opt.model == SPDBA_MODEL_CH) s = run_ch_step<T>(p, *r);
            else s = fail(SPDBA_ERR_UNSUPPORTED, "model %d not built", p->opt.model);
            if (s != SPDBA_OK) return s;
        }
    }
    return SPDBA_OK;
}

template <typename T> static spdba_status run_set_field(spdba_plan* p, Run<T>& r, const void* src, int on_dev) {
    cudaStream_t st = p->st;
    if (p->opt.model == SPDBA_MODEL_CH) {
        SPDBA_CUDA(cudaMemcpyAsync(r.real, src, sizeof(T) * r.n, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        real_to_complex_kernel<T><<<grid_for(r.n, 256), 256, 0, st>>>(r.real, r.work, r.n);
        spdba_status s = r.fft.exec(r.work, r.c_hat, SPDBA_FORWARD, st);
        if (s != SPDBA_OK) return s;
    } else {
        SPDBA_CUDA(cudaMemcpyAsync(r.work, src, sizeof(cx_t<T>) * r.n, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        spdba_status s = r.fft.exec(r.work, r.c_hat, SPDBA_FORWARD, st);
        if (s != SPDBA_OK) return s;
    }
    r.step = 0;
    r.assessed = false;
    SPDBA_CUDA(cudaMemsetAsync(r.stats, 0, sizeof(DevStats), st));
    SPDBA_CUDA(cudaMemsetAsync(r.states, SPDBA_ACTIVE, r.g.blocks(), st));
    return SPDBA_OK;
}

template <typename T> static spdba_status run_get_field(spdba_plan* p, Run<T>& r, void* dst, int on_dev) {
    cudaStream_t st = p->st;
    spdba_status s = r.fft.exec(r.c_hat, r.work, SPDBA_INVERSE, st);
    if (s != SPDBA_OK) return s;
    if (p->opt.model == SPDBA_MODEL_CH) {
        complex_real_part_kernel<T><<<grid_for(r.n, 256), 256, 0, st>>>(r.work, r.real, r.n);
        SPDBA_CUDA(cudaMemcpyAsync(dst, r.real, sizeof(T) * r.n, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    } else {
        SPDBA_CUDA(cudaMemcpyAsync(dst, r.work, sizeof(cx_t<T>) * r.n, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    SPDBA_CUDA(cudaStreamSynchronize(st));
    return SPDBA_OK;
}

}  // namespace spdba

// ------------------------------------------------------------------ C ABI
static spdba_status latch(spdba_plan* p, spdba_status s) {
    if (s == SPDBA_ERR_CUDA && p) p->latched = s;
    return s;
}
#define PLAN_CHECK(p)                                                                  \
    do {                                                                               \
        if (!(p)) return fail(SPDBA_ERR_ARG, "NULL plan");                             \
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
    o->dt = 0.01;
    o->kappa = 1.0;
    o->dx = 1.0;
    o->beta2 = -21.7;
    o->gamma = 1.3;
    o->h = 0.1;
    o->dt_sample = 1.0;
    o->stream = nullptr;
}

static spdba_status check_opts(const spdba_options* o, int ndim) {
    if (o->model != SPDBA_MODEL_CH && o->model != SPDBA_MODEL_NLS) return fail(SPDBA_ERR_ARG, "bad model %d", o->model);
    if (o->precision != SPDBA_C64 && o->precision != SPDBA_C128) return fail(SPDBA_ERR_ARG, "bad precision %d", o->precision);
    if (o->mode != SPDBA_MODE_REGULAR && o->mode != SPDBA_MODE_ADAPTIVE) return fail(SPDBA_ERR_ARG, "bad mode %d", o->mode);
    if (o->measure != SPDBA_MEASURE_MAXAMP && o->measure != SPDBA_MEASURE_ENERGY) return fail(SPDBA_ERR_ARG, "bad measure");
    if (o->tau_rule != SPDBA_TAU_REL_MAX && o->tau_rule != SPDBA_TAU_ABS) return fail(SPDBA_ERR_ARG, "bad tau rule");
    if (o->refresh_every < 0 || o->warmup_steps < 0) return fail(SPDBA_ERR_ARG, "negative refresh/warm-up");
    if (o->model == SPDBA_MODEL_CH && (ndim < 2 || ndim > 3)) return fail(SPDBA_ERR_UNSUPPORTED, "CH plans are 2-D or 3-D");
    if (o->model == SPDBA_MODEL_NLS && ndim != 1) return fail(SPDBA_ERR_UNSUPPORTED, "NLS plans are 1-D");
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
    p->threshold = threshold;
    p->reassess = reassess;
    p->precision = o.precision;
    p->st = (cudaStream_t)o.stream;
    for (int r = 0; r < nruns && s == SPDBA_OK; ++r) {
        const int64_t* d = dims + (size_t)r * ndim;
        int32_t blk[3];
        for (int a = 0; a < ndim; ++a) blk[a] = block[a];
        if (o.model == SPDBA_MODEL_NLS && block[0] <= 0) blk[0] = (int32_t)(d[0] / (-block[0]));
        if (p->precision == SPDBA_C64) {
            p->r32.emplace_back(new Run<float>());
            s = run_init<float>(p, *p->r32.back(), ndim, d, blk);
        } else {
            p->r64.emplace_back(new Run<double>());
            s = run_init<double>(p, *p->r64.back(), ndim, d, blk);
        }
    }
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
    for (auto& r : p->r32) r->release();
    for (auto& r : p->r64) r->release();
    p->tw32.release();
    p->tw64.release();
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    delete p;
}

static bool run_ok(spdba_plan* p, int32_t run) { return run >= 0 && run < p->nruns(); }

extern "C" spdba_status spdba_set_field(spdba_plan* p, int32_t run, const void* src, int32_t on_dev) {
    PLAN_CHECK(p);
    if (!src || !run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_set_field: bad arguments");
    spdba_status s = p->precision == SPDBA_C64 ? run_set_field<float>(p, *p->r32[run], src, on_dev)
                                               : run_set_field<double>(p, *p->r64[run], src, on_dev);
    return latch(p, s);
}

extern "C" spdba_status spdba_step(spdba_plan* p, int64_t n) {
    PLAN_CHECK(p);
    if (n < 0) return fail(SPDBA_ERR_ARG, "negative step count");
    spdba_status s = p->precision == SPDBA_C64 ? plan_step<float>(p, n) : plan_step<double>(p, n);
    return latch(p, s);
}

extern "C" spdba_status spdba_get_field(spdba_plan* p, int32_t run, void* dst, int32_t on_dev) {
    PLAN_CHECK(p);
    if (!dst || !run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_get_field: bad arguments");
    spdba_status s = p->precision == SPDBA_C64 ? run_get_field<float>(p, *p->r32[run], dst, on_dev)
                                               : run_get_field<double>(p, *p->r64[run], dst, on_dev);
    return latch(p, s);
}

template <typename T> static spdba_status copy_spectrum(spdba_plan* p, Run<T>& r, void* buf, int on_dev, bool get) {
    size_t bytes = sizeof(cx_t<T>) * (size_t)r.n;
    if (get) {
        SPDBA_CUDA(cudaMemcpyAsync(buf, r.c_hat, bytes, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->st));
        SPDBA_CUDA(cudaStreamSynchronize(p->st));
    } else {
        SPDBA_CUDA(cudaMemcpyAsync(r.c_hat, buf, bytes, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->st));
        r.assessed = false;
    }
    return SPDBA_OK;
}

extern "C" spdba_status spdba_get_spectrum(spdba_plan* p, int32_t run, void* dst, int32_t on_dev) {
    PLAN_CHECK(p);
    if (!dst || !run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_get_spectrum: bad arguments");
    spdba_status s = p->precision == SPDBA_C64 ? copy_spectrum<float>(p, *p->r32[run], dst, on_dev, true)
                                               : copy_spectrum<double>(p, *p->r64[run], dst, on_dev, true);
    return latch(p, s);
}

extern "C" spdba_status spdba_set_spectrum(spdba_plan* p, int32_t run, const void* src, int32_t on_dev) {
    PLAN_CHECK(p);
    if (!src || !run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_set_spectrum: bad arguments");
    spdba_status s = p->precision == SPDBA_C64 ? copy_spectrum<float>(p, *p->r32[run], (void*)src, on_dev, false)
                                               : copy_spectrum<double>(p, *p->r64[run], (void*)src, on_dev, false);
    return latch(p, s);
}

template <typename T> static spdba_status get_mask_t(spdba_plan* p, Run<T>& r, uint8_t* dst, int64_t nb) {
    if (nb != r.g.blocks()) return fail(SPDBA_ERR_ARG, "mask size %lld != %lld blocks", (long long)nb, r.g.blocks());
    SPDBA_CUDA(cudaMemcpyAsync(dst, r.states, (size_t)nb, cudaMemcpyDeviceToHost, p->st));
    SPDBA_CUDA(cudaStreamSynchronize(p->st));
    return SPDBA_OK;
}

extern "C" spdba_status spdba_get_mask(spdba_plan* p, int32_t run, uint8_t* dst, int64_t nb) {
    PLAN_CHECK(p);
    if (!dst || !run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_get_mask: bad arguments");
    spdba_status s = p->precision == SPDBA_C64 ? get_mask_t<float>(p, *p->r32[run], dst, nb)
                                               : get_mask_t<double>(p, *p->r64[run], dst, nb);
    return latch(p, s);
}

template <typename T> static spdba_status get_stats_t(spdba_plan* p, Run<T>& r, spdba_stats* out) {
    DevStats d;
    SPDBA_CUDA(cudaMemcpyAsync(&d, r.stats, sizeof d, cudaMemcpyDeviceToHost, p->st));
    SPDBA_CUDA(cudaStreamSynchronize(p->st));
    out->step = r.step;
    out->assessments = (int64_t)d.assessments;
    out->nblocks = r.g.blocks();
    out->n_active = (int64_t)d.n_active;
    out->n_transition = (int64_t)d.n_transition;
    out->tau = d.tau;
    out->max_amp = d.max_amp;
    out->mass = d.mass;
    out->active_ratio_sum = d.ratio_sum;
    return SPDBA_OK;
}

extern "C" spdba_status spdba_get_stats(spdba_plan* p, int32_t run, spdba_stats* out) {
    PLAN_CHECK(p);
    if (!out || !run_ok(p, run)) return fail(SPDBA_ERR_ARG, "spdba_get_stats: bad arguments");
    spdba_status s = p->precision == SPDBA_C64 ? get_stats_t<float>(p, *p->r32[run], out)
                                               : get_stats_t<double>(p, *p->r64[run], out);
    return latch(p, s);
}

template <typename T> static spdba_status list_modes_now(spdba_plan* p, std::vector<double>* out) {
    out->clear();
    for (auto& r : runs<T>(p)) {
        DevStats d;
        SPDBA_CUDA(cudaMemcpyAsync(&d, r->stats, sizeof d, cudaMemcpyDeviceToHost, p->st));
        SPDBA_CUDA(cudaStreamSynchronize(p->st));
        out->push_back(d.list_modes);
    }
    return SPDBA_OK;
}

extern "C" spdba_status spdba_profile_begin(spdba_plan* p) {
    PLAN_CHECK(p);
    p->prof_recs.clear();
    p->ev_used = 0;
    p->launches = 0;
    spdba_status s = p->precision == SPDBA_C64 ? list_modes_now<float>(p, &p->prof_list_modes0)
                                               : list_modes_now<double>(p, &p->prof_list_modes0);
    if (s != SPDBA_OK) return latch(p, s);
    p->prof = true;
    return SPDBA_OK;
}

extern "C" spdba_status spdba_profile_end(spdba_plan* p, spdba_kernel_time* out, int32_t capacity, int32_t* n_out,
                                          int64_t* launches_out) {
    PLAN_CHECK(p);
    if (!p->prof) return fail(SPDBA_ERR_STATE, "profiling was not started");
    p->prof = false;
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
    std::vector<double> lm;
    spdba_status s = p->precision == SPDBA_C64 ? list_modes_now<float>(p, &lm) : list_modes_now<double>(p, &lm);
    if (s != SPDBA_OK) return latch(p, s);
    double esz = p->precision == SPDBA_C64 ? 8.0 : 16.0;
    for (size_t i = 0; i < lm.size() && i < p->prof_list_modes0.size(); ++i)
        agg[K_UPDATE_LIST].bytes += 3.0 * esz * (lm[i] - p->prof_list_modes0[i]);
    int n = 0;
    for (int k = 0; k < K_COUNT && n < capacity; ++k)
        if (agg[k].launches > 0 && out) out[n++] = agg[k];
    if (n_out) *n_out = n;
    if (launches_out) *launches_out = p->launches;
    return SPDBA_OK;
}

extern "C" spdba_status spdba_sync(spdba_plan* p) {
    PLAN_CHECK(p);
    cudaError_t e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) return latch(p, cuda_fail(e, "cudaStreamSynchronize"));
    return SPDBA_OK;
}
