// Host side of the Stockham FFT: FP64 twiddle tables, pass planning, the
// kernel-level FFT entry points, and the library's error reporting.
#include <atomic>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>
#include <map>
#include <set>

#include <algorithm>

#include "internal.h"
#include "kernel_table.h"

namespace spdba {

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}
spdba_status fail(spdba_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}
spdba_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SPDBA_ERR_OOM : SPDBA_ERR_CUDA;
}

// ------------------------------------------------------------------ device allocations
static std::atomic<long long> g_live_allocs{0};
static std::atomic<long long> g_fail_countdown{0};

cudaError_t dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (g_fail_countdown.load() > 0 && g_fail_countdown.fetch_sub(1) == 1) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) g_live_allocs.fetch_add(1);
    else *p = nullptr;
    return e;
}
void dev_free(void* p) {
    if (!p) return;
    cudaFree(p);
    g_live_allocs.fetch_sub(1);
}

bool length_ok(int64_t n) {
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

bool tile_length_supported(int64_t L) {
    switch (L) {
        case 16: case 32: case 64: case 128: case 192: case 256: case 384: case 512:
        case 1024: case 2048: case 4096: return true;
        default: return false;
    }
}

// ------------------------------------------------------------------ twiddles
template <typename T> __global__ void twiddle_kernel(cx_t<T>* t, long long n) {
    long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m < n) {
        double s, c;
        sincospi(2.0 * (double)m / (double)n, &s, &c);   // FP64: angle 2 pi m / n
        t[m] = mk<cx_t<T>>((T)c, (T)(-s));
    }
}

template <typename T> cx_t<T>* TwiddleCache<T>::get(int64_t n, cudaStream_t st, spdba_status* err) {
    auto it = tables.find(n);
    if (it != tables.end()) return it->second;
    cx_t<T>* p = nullptr;
    cudaError_t e = dev_alloc((void**)&p, sizeof(cx_t<T>) * (size_t)n);
    if (e != cudaSuccess) { *err = cuda_fail(e, "device allocation (twiddle table)"); return nullptr; }
    twiddle_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, (long long)n);
    e = cudaGetLastError();
    if (e != cudaSuccess) { dev_free(p); *err = cuda_fail(e, "twiddle_kernel"); return nullptr; }
    tables[n] = p;
    return p;
}
template <typename T> void TwiddleCache<T>::release() {
    for (auto& kv : tables) dev_free(kv.second);
    tables.clear();
}

// ------------------------------------------------------------------ passes
static std::mutex g_attr_mu;
static std::map<const void*, int> g_attr_smem;   // dynamic shared-memory limit set per kernel
// Raises a kernel's dynamic shared-memory limit to `smem` (the size of some
// kernels depends on the shape, so a later plan may need more than an earlier one).
static spdba_status ensure_smem_attr(const void* f, int smem, bool max_carveout) {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto it = g_attr_smem.find(f);
    if (it != g_attr_smem.end() && it->second >= smem) return SPDBA_OK;
    // always raise the dynamic limit: some kernels also carry static shared memory
    SPDBA_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    // pipelined tiles stream through shared memory only; give them the whole
    // carveout so that the compiled CTAs per SM fit
    if (max_carveout) SPDBA_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    g_attr_smem[f] = smem;
    return SPDBA_OK;
}

template <typename T>
spdba_status make_pass(Pass<T>* out, int64_t L, int sign, int mode, long long O, long long I, long long isO,
                       long long isI, long long isJ, long long osO, long long osI, long long osJ,
                       TwiddleCache<T>& tw, cudaStream_t st) {
    bool loadp = (isJ != 1), storep = (osJ != 1);
    if (loadp && isI != 1) return fail(SPDBA_ERR_UNSUPPORTED, "pass without a unit-stride input direction");
    if (storep && osI != 1) return fail(SPDBA_ERR_UNSUPPORTED, "pass without a unit-stride output direction");
    // pencil indices and offsets within one tile are 32-bit in the kernels
    if (O * I >= 0x7fffffffLL) return fail(SPDBA_ERR_UNSUPPORTED, "FFT pass over 2^31 pencils or more");
    if ((L - 1) * (isJ > osJ ? isJ : osJ) + 4096 * (isI > osI ? isI : osI) > 0x7fffffffLL)
        return fail(SPDBA_ERR_UNSUPPORTED, "FFT pass with a tile span beyond 2^31 elements");
    KernelInfo ki;
    // the tile size depends only on (T, L); ask once to learn P
    if (!get_pass_kernel<T>(L, sign, mode, loadp, storep, true, &ki))
        return fail(SPDBA_ERR_UNSUPPORTED, "no FFT pass kernel for length %lld (mode %d)", (long long)L, mode);
    const bool generic = (I % ki.P) != 0;
    if (!get_pass_kernel<T>(L, sign, mode, loadp, storep, generic, &ki))
        return fail(SPDBA_ERR_UNSUPPORTED, "no FFT pass kernel for length %lld (mode %d)", (long long)L, mode);
    spdba_status s = ensure_smem_attr(ki.func, ki.smem, ki.pipe);
    if (s != SPDBA_OK) return s;
    long long ntiles = (O * I + ki.P - 1) / ki.P;
    long long grid = ntiles;
    if (ki.pipe) {
        int per_sm = 0, nsm = 0, dev = 0;
        SPDBA_CUDA(cudaGetDevice(&dev));
        SPDBA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        SPDBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ki.func, ki.NT, ki.smem));
        if (per_sm < 1) per_sm = 1;
        long long resident = (long long)per_sm * nsm;
        if (grid > resident) grid = resident;
    }
    s = SPDBA_OK;
    cx_t<T>* t = tw.get(L, st, &s);
    if (!t) return s;
    Pass<T> ps;
    ps.func = ki.func;
    ps.nt = ki.NT;
    ps.P = ki.P;
    ps.smem = ki.smem;
    ps.grid = grid;
    ps.p.O = O; ps.p.I = I;
    ps.p.isO = isO; ps.p.isI = isI; ps.p.isJ = isJ;
    ps.p.osO = osO; ps.p.osI = osI; ps.p.osJ = osJ;
    ps.p.tw = t;
    ps.p.tw4 = nullptr;
    ps.p.n4 = 1;
    ps.p.scale = (T)1;
    ps.p.generic = generic;
    ps.p.fd_I.init((uint32_t)I);
    ps.p.nl_scale = (T)1;
    ps.p.mass = nullptr;
    *out = ps;
    return SPDBA_OK;
}

template <typename T> spdba_status launch_pass(const Pass<T>& ps, const void* in, void* out, cudaStream_t st) {
    PassParams<T> p = ps.p;
    p.in = reinterpret_cast<const cx_t<T>*>(in);
    p.out = reinterpret_cast<cx_t<T>*>(out);
    void* args[] = {&p};
    SPDBA_CUDA(cudaLaunchKernel(ps.func, dim3((unsigned)ps.grid), dim3(ps.nt), args, (size_t)ps.smem, st));
    return SPDBA_OK;
}

template <typename T>
spdba_status make_axis_pass(Pass<T>* out, int ndim, const int64_t* dims, int64_t batch, int axis, int sign,
                            int mode, TwiddleCache<T>& tw, cudaStream_t st) {
    long long L = dims[axis];
    long long O = batch, I = 1;
    for (int a = 0; a < axis; ++a) O *= dims[a];
    for (int a = axis + 1; a < ndim; ++a) I *= dims[a];
    if (I == 1) {
        // contiguous pencils: index them as the inner direction
        return make_pass<T>(out, L, sign, mode, 1, O, 0, L, 1, 0, L, 1, tw, st);
    }
    return make_pass<T>(out, L, sign, mode, O, I, L * I, 1, I, L * I, 1, I, tw, st);
}

// ------------------------------------------------------------------ engine
template <typename T>
spdba_status FftEngine<T>::init(int nd, const int64_t* d, int64_t b, TwiddleCache<T>& tw, cudaStream_t st) {
    ndim = nd;
    batch = b;
    total = b;
    for (int a = 0; a < nd; ++a) { dims[a] = d[a]; total *= d[a]; }
    fwd.clear(); inv.clear(); fwd_scratch_out.clear(); inv_scratch_out.clear();
    spdba_status s;
    if (nd == 1 && d[0] > 4096) {
        // four-step: n = n1 * n2, pass 1 over n1 (stride n2) with twiddles, pass 2 over n2
        long long n = d[0];
        long long n2 = 512, n1 = n / n2;
        if (n % 512 != 0 || !tile_length_supported(n1) || n1 > 512)
            return fail(SPDBA_ERR_UNSUPPORTED, "1-D length %lld not supported", n);
        s = SPDBA_OK;
        cx_t<T>* t4 = tw.get(n, st, &s);
        if (!t4) return s;
        for (int dir = 0; dir < 2; ++dir) {
            int sign = dir == 0 ? -1 : +1;
            Pass<T> p1, p2;
            s = make_pass<T>(&p1, n1, sign, PASS_PLAIN, b, n2, n, 1, n2, n, 1, n2, tw, st);
            if (s != SPDBA_OK) return s;
            p1.p.tw4 = t4;
            p1.p.n4 = n;
            s = make_pass<T>(&p2, n2, sign, PASS_PLAIN, b, n1, n, n2, 1, n, 1, n1, tw, st);
            if (s != SPDBA_OK) return s;
            if (sign > 0) p2.p.scale = (T)(1.0 / (double)n);
            auto& v = dir == 0 ? fwd : inv;
            auto& so = dir == 0 ? fwd_scratch_out : inv_scratch_out;
            v.push_back(p1); so.push_back(1);
            v.push_back(p2); so.push_back(0);
        }
        if (!scratch) {
            cudaError_t e = dev_alloc((void**)&scratch, sizeof(cx_t<T>) * (size_t)total);
            if (e != cudaSuccess) return cuda_fail(e, "device allocation (FFT scratch)");
        }
        return SPDBA_OK;
    }
    for (int a = 0; a < nd; ++a) {
        if (!tile_length_supported(d[a]) || (nd > 1 && d[a] > 512))
            return fail(SPDBA_ERR_UNSUPPORTED, "axis length %lld not supported", (long long)d[a]);
    }
    // forward: fastest axis first; inverse: slowest axis first, 1/N on the last pass
    for (int a = nd - 1; a >= 0; --a) {
        Pass<T> p;
        s = make_axis_pass<T>(&p, nd, d, b, a, -1, PASS_PLAIN, tw, st);
        if (s != SPDBA_OK) return s;
        fwd.push_back(p); fwd_scratch_out.push_back(0);
    }
    for (int a = 0; a < nd; ++a) {
        Pass<T> p;
        s = make_axis_pass<T>(&p, nd, d, b, a, +1, PASS_PLAIN, tw, st);
        if (s != SPDBA_OK) return s;
        if (a == nd - 1) p.p.scale = (T)(1.0 / (double)(total / b));
        inv.push_back(p); inv_scratch_out.push_back(0);
    }
    return SPDBA_OK;
}

template <typename T>
spdba_status FftEngine<T>::exec(const cx_t<T>* in, cx_t<T>* out, int direction, cudaStream_t st) {
    auto& v = direction < 0 ? fwd : inv;
    auto& so = direction < 0 ? fwd_scratch_out : inv_scratch_out;
    const cx_t<T>* src = in;
    for (size_t k = 0; k < v.size(); ++k) {
        cx_t<T>* dst = so[k] ? scratch : out;
        spdba_status s = launch_pass<T>(v[k], src, dst, st);
        if (s != SPDBA_OK) return s;
        src = dst;
    }
    return SPDBA_OK;
}

template <typename T> void FftEngine<T>::release() {
    if (scratch) dev_free(scratch);
    scratch = nullptr;
}

template struct TwiddleCache<float>;
template struct TwiddleCache<double>;
template struct FftEngine<float>;
template struct FftEngine<double>;
template spdba_status make_pass<float>(Pass<float>*, int64_t, int, int, long long, long long, long long, long long,
                                       long long, long long, long long, long long, TwiddleCache<float>&,
                                       cudaStream_t);
template spdba_status make_pass<double>(Pass<double>*, int64_t, int, int, long long, long long, long long, long long,
                                        long long, long long, long long, long long, TwiddleCache<double>&,
                                        cudaStream_t);
// Half-spectrum passes of a 3-D complex64 field (see fft_half.cuh).
spdba_status make_half_pass(Pass<float>* out, int mode, const HalfGeo& hg, TwiddleCache<float>& tw, cudaStream_t st) {
    const bool rows = mode == PASS_NL_HALF;
    const int64_t L = rows ? hg.N2 : hg.N0;
    KernelInfo ki;
    if (!get_half_kernel(L, mode, hg.NHP, &ki)) {
        // no message for the paired pass: the caller then takes the unpaired one
        if (mode == PASS_PAIR_MIRROR) return SPDBA_ERR_UNSUPPORTED;
        return fail(SPDBA_ERR_UNSUPPORTED, "no half-spectrum kernel for length %lld (mode %d)", (long long)L, mode);
    }
    Pass<float> ps;
    PassParams<float>& a = ps.p;
    a.fu = CHFuse<float>{};   // no states: the paired z forward then stores every mode
    if (rows) {
        a.O = hg.N0;
        a.I = hg.N1;
    } else {
        a.O = 1;
        a.I = (long long)hg.N1 * (mode == PASS_HERM_INV ? hg.NHP : hg.N2);
        a.osO = 0;
        a.osI = 1;
        a.osJ = a.I;
    }
    const bool pair = mode == PASS_PAIR_MIRROR;
    long long ntiles = a.O * a.I / ki.P;
    if (pair) {
        // tiles of P x frequencies below N2/2 within one half row, then the
        // column N2/2 in tiles of P rows; 16-byte pencil pairs need an even row pitch
        const long long M = hg.N2 / 2;
        if (M % ki.P != 0 || hg.N1 % ki.P != 0 || hg.NHP % 2 != 0)
            return SPDBA_ERR_UNSUPPORTED;
        a.I = (long long)hg.N1 * (M + 1);
        a.osJ = (long long)hg.N1 * hg.N2;
        ntiles = a.I / ki.P;
    } else if ((a.O * a.I) % ki.P != 0) {
        return fail(SPDBA_ERR_UNSUPPORTED, "half-spectrum tiles do not divide the pencils");
    }
    spdba_status s = ensure_smem_attr(ki.func, ki.smem, true);
    if (s != SPDBA_OK) return s;
    int per_sm = 0, nsm = 0, dev = 0;
    SPDBA_CUDA(cudaGetDevice(&dev));
    SPDBA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SPDBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ki.func, ki.NT, ki.smem));
    if (per_sm < 1) return fail(SPDBA_ERR_UNSUPPORTED, "half-spectrum kernel does not fit an SM");
    ps.grid = std::min<long long>(ntiles, (long long)per_sm * nsm);
    ps.func = ki.func;
    ps.nt = ki.NT;
    ps.P = ki.P;
    ps.smem = ki.smem;
    s = SPDBA_OK;
    if (!(a.tw = tw.get(L, st, &s))) return s;
    a.tw4 = nullptr;

    a.n4 = 1;
    a.scale = 1.f;
    a.generic = 0;
    a.nl_scale = (float)(1.0 / ((double)hg.N0 * hg.N1 * hg.N2));
    a.mass = nullptr;
    a.mass_ppr = (long long)hg.N0 * hg.N1;
    a.fd_I.init((uint32_t)a.I);
    a.hg = hg;
    *out = ps;
    return SPDBA_OK;
}

template spdba_status launch_pass<float>(const Pass<float>&, const void*, void*, cudaStream_t);
template spdba_status launch_pass<double>(const Pass<double>&, const void*, void*, cudaStream_t);
template spdba_status make_axis_pass<float>(Pass<float>*, int, const int64_t*, int64_t, int, int, int,
                                            TwiddleCache<float>&, cudaStream_t);
template spdba_status make_axis_pass<double>(Pass<double>*, int, const int64_t*, int64_t, int, int, int,
                                             TwiddleCache<double>&, cudaStream_t);

}  // namespace spdba

// ------------------------------------------------------------------ C ABI: FFT
using namespace spdba;

struct spdba_fft_plan {
    int precision;
    TwiddleCache<float> tw32;
    TwiddleCache<double> tw64;
    FftEngine<float> e32;
    FftEngine<double> e64;
};

extern "C" spdba_status spdba_fft_plan_create(spdba_fft_plan** out, int32_t precision, int32_t ndim,
                                              const int64_t* dims, int64_t batch) {
    if (!out || !dims || ndim < 1 || ndim > 3 || batch < 1) return fail(SPDBA_ERR_ARG, "spdba_fft_plan_create: bad arguments");
    if (precision != SPDBA_C64 && precision != SPDBA_C128) return fail(SPDBA_ERR_ARG, "bad precision %d", precision);
    for (int a = 0; a < ndim; ++a)
        if (!length_ok(dims[a])) return fail(SPDBA_ERR_UNSUPPORTED, "length %lld is not 2^a 3^b", (long long)dims[a]);
    spdba_fft_plan* p = new spdba_fft_plan();
    p->precision = precision;
    spdba_status s = precision == SPDBA_C64 ? p->e32.init(ndim, dims, batch, p->tw32, 0)
                                            : p->e64.init(ndim, dims, batch, p->tw64, 0);
    if (s == SPDBA_OK) {
        cudaError_t e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) s = cuda_fail(e, "fft plan setup");
    }
    if (s != SPDBA_OK) {
        spdba_fft_plan_destroy(p);
        return s;
    }
    *out = p;
    return SPDBA_OK;
}

extern "C" spdba_status spdba_fft_exec(spdba_fft_plan* p, const void* in, void* out, int32_t direction, void* stream) {
    if (!p || !in || !out || (direction != SPDBA_FORWARD && direction != SPDBA_INVERSE))
        return fail(SPDBA_ERR_ARG, "spdba_fft_exec: bad arguments");
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return fail(SPDBA_ERR_ARG, "spdba_fft_exec: buffers must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    if (p->precision == SPDBA_C64)
        return p->e32.exec((const float2*)in, (float2*)out, direction, st);
    return p->e64.exec((const double2*)in, (double2*)out, direction, st);
}

extern "C" void spdba_fft_plan_destroy(spdba_fft_plan* p) {
    if (!p) return;
    p->e32.release();
    p->e64.release();
    p->tw32.release();
    p->tw64.release();
    delete p;
}

extern "C" const char* spdba_last_error(void) { return g_err; }

extern "C" const char* spdba_status_string(spdba_status s) {
    switch (s) {
        case SPDBA_OK: return "ok";
        case SPDBA_ERR_ARG: return "invalid argument";
        case SPDBA_ERR_UNSUPPORTED: return "unsupported size";
        case SPDBA_ERR_CUDA: return "CUDA error";
        case SPDBA_ERR_OOM: return "out of device memory";
        case SPDBA_ERR_TIMEOUT: return "device wait timed out";
        case SPDBA_ERR_STATE: return "invalid state";
        default: return "unknown status";
    }
}

extern "C" void spdba_debug_fail_alloc(int64_t k) { spdba::g_fail_countdown.store(k > 0 ? (long long)k : 0); }

extern "C" int64_t spdba_debug_live_allocs(void) { return (int64_t)spdba::g_live_allocs.load(); }

namespace spdba {
static std::atomic<long long> g_wait_limit{0};   // 0: the default
long long wait_limit() {
    const long long n = g_wait_limit.load();
    return n > 0 ? n : kWaitLimit;
}
}  // namespace spdba

namespace spdba {
static std::atomic<int> g_stall_waits{0};
int stall_waits() { return g_stall_waits.load(); }
}  // namespace spdba

extern "C" void spdba_debug_set_wait_limit(int64_t n) { spdba::g_wait_limit.store(n > 0 ? (long long)n : 0); }
extern "C" void spdba_debug_stall_waits(int32_t on) { spdba::g_stall_waits.store(on ? 1 : 0); }
