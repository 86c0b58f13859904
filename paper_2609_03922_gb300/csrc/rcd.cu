// Reaction-cross-diffusion kernels (Supplementary S4.1-S4.3).
//
// The per-mode coupled update is two small dense contractions with the
// constant eigenbasis V of the cross-diffusion matrix: z = V^T b, z_j /=
// 1 + dt k^2 lambda_j, x = V z (S4.3), for b = u_hat + dt FFT(R(u)).  A CTA
// takes tiles of 64 modes of one block: the tile's M x 64 complex values sit
// in shared memory as M rows of 128 real columns; each thread keeps one real
// column in registers and forms its share of the output rows from V's rows in
// shared memory (warp-uniform rows: broadcast reads), so both contractions run
// at FP32 (or FP64) FMA rate without leaving the SM.
#include "rcd.h"

namespace spdba {

// ------------------------------------------------------------------ reaction
// One thread per grid point; its M component values are staged in a
// shared-memory column (su[m * NT + tid], conflict-free), so that the sum over
// components and the two periodic neighbours of each component need one read
// of the field each.
constexpr int RCD_RX_NT = 256;

template <typename T>
__global__ void __launch_bounds__(RCD_RX_NT) rcd_reaction_kernel(cx_t<T>* __restrict__ w, long long n, int M, T r, T a,
                                                                 T alpha, T beta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);
    const int tid = threadIdx.x;
    for (long long x = (long long)blockIdx.x * blockDim.x + tid; x < n; x += (long long)gridDim.x * blockDim.x) {
        T S = (T)0;
        for (int m = 0; m < M; ++m) {
            const T v = w[(long long)m * n + x].x;
            su[m * RCD_RX_NT + tid] = v;
            S += v;
        }
        for (int m = 0; m < M; ++m) {
            const T um = su[m * RCD_RX_NT + tid];
            // sum_{j != i} alpha_ij u_j: beta + alpha for the two periodic
            // neighbours (the one other component when M = 2), beta otherwise
            T inter;
            if (M >= 3) {
                const T prev = su[(m == 0 ? M - 1 : m - 1) * RCD_RX_NT + tid];
                const T next = su[(m + 1 == M ? 0 : m + 1) * RCD_RX_NT + tid];
                inter = beta * (S - um) + alpha * (prev + next);
            } else {
                inter = (beta + alpha) * (S - um);
            }
            w[(long long)m * n + x] = mk<cx_t<T>>(um * (r - a * um - inter), (T)0);
        }
    }
}

template <typename T>
spdba_status launch_rcd_reaction(cx_t<T>* work, long long n, int M, T r, T a, T alpha, T beta, cudaStream_t st) {
    if (M < 1 || M > kRcdMaxComponents)
        return fail(SPDBA_ERR_UNSUPPORTED, "RCD with %d components (at most %d)", M, kRcdMaxComponents);
    const int smem = M * RCD_RX_NT * (int)sizeof(T);
    long long grid = (n + RCD_RX_NT - 1) / RCD_RX_NT;
    if (grid > 152 * 8) grid = 152 * 8;
    rcd_reaction_kernel<T><<<(unsigned)grid, RCD_RX_NT, smem, st>>>(work, n, M, r, a, alpha, beta);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

// ------------------------------------------------------------------ activity
// One warp per block.  A(k)^2 = (1/M) sum_m (re^2 + im^2).  GB300's FP64 rate
// is a small fraction of its FP32 rate, so the sum runs in double-float: each
// square is split exactly into p + e with an FMA (Dekker's two-product), the
// large parts are added with Knuth's two-sum into (hi, lo), and hi + lo is
// converted to FP64 once per mode.  The result carries about 2^-44 relative
// error (squares of |x| < 2^-63 fall below FP32's range and count as zero:
// such values lie far below any threshold in use), so the block maximum and
// the global maxima are FP64-accurate.  Non-negative doubles order like their
// bit patterns: the global maxima are integer atomicMax on the bits.
__device__ __forceinline__ void rcd_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void rcd_acc_sq(float x, float& hi, float& lo) {
    const float p = __fmul_rn(x, x);
    const float pe = __fmaf_rn(x, x, -p);   // x^2 = p + pe exactly
    float s, e;
    rcd_two_sum(hi, p, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
}
template <typename C> __device__ __forceinline__ double rcd_mode_sq(const C* __restrict__ q, long long n, long long e,
                                                                    int M);
template <> __device__ __forceinline__ double rcd_mode_sq<float2>(const float2* __restrict__ q, long long n,
                                                                   long long e, int M) {
    float hi = 0.f, lo = 0.f;
    // the component loads of a group of 8 are issued before any is used
    int m = 0;
    for (; m + 8 <= M; m += 8) {
        float2 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = q[(long long)(m + k) * n + e];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            rcd_acc_sq(v[k].x, hi, lo);
            rcd_acc_sq(v[k].y, hi, lo);
        }
    }
    for (; m < M; ++m) {
        const float2 v = q[(long long)m * n + e];
        rcd_acc_sq(v.x, hi, lo);
        rcd_acc_sq(v.y, hi, lo);
    }
    return __ddiv_rn(__dadd_rn((double)hi, (double)lo), (double)M);
}
template <> __device__ __forceinline__ double rcd_mode_sq<double2>(const double2* __restrict__ q, long long n,
                                                                    long long e, int M) {
    double s = 0.0;
    for (int m = 0; m < M; ++m) {
        const double2 v = q[(long long)m * n + e];
        s = __dadd_rn(s, __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)));
    }
    return __ddiv_rn(s, (double)M);
}

template <typename T>
__global__ void rcd_activity_kernel(Geom g, const cx_t<T>* __restrict__ q, int M, long long n, double* maxsq,
                                    double* gmax) {
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long nb = g.blocks();
    const int B0 = g.b[0], B1 = g.b[1], B2 = g.b[2];
    const long long bm = (long long)B0 * B1 * B2;
    double gall = 0.0, gnz = 0.0;
    for (long long blk = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; blk < nb; blk += nwarps) {
        const long long b2 = blk % g.nb[2], b1 = (blk / g.nb[2]) % g.nb[1], b0 = blk / (g.nb[2] * g.nb[1]);
        double bmax = 0.0;
        for (long long o = lane; o < bm; o += 32) {
            const int d2 = (int)(o % B2);
            const long long rr = o / B2;
            const int d1 = (int)(rr % B1), d0 = (int)(rr / B1);
            const long long e = ((b0 * B0 + d0) * g.n[1] + (b1 * B1 + d1)) * g.n[2] + (b2 * B2 + d2);
            const double a2 = rcd_mode_sq(q, n, e, M);
            bmax = fmax(bmax, a2);
            gall = fmax(gall, a2);
            if (e != 0) gnz = fmax(gnz, a2);
        }
        for (int off = 16; off > 0; off >>= 1) bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, off));
        if (lane == 0) maxsq[blk] = bmax;
    }
    for (int off = 16; off > 0; off >>= 1) {
        gall = fmax(gall, __shfl_xor_sync(0xffffffffu, gall, off));
        gnz = fmax(gnz, __shfl_xor_sync(0xffffffffu, gnz, off));
    }
    if (lane == 0) {
        if (gall > 0.0) atomicMax(reinterpret_cast<unsigned long long*>(gmax), (unsigned long long)__double_as_longlong(gall));
        if (gnz > 0.0) atomicMax(reinterpret_cast<unsigned long long*>(gmax + 1), (unsigned long long)__double_as_longlong(gnz));
    }
}

template <typename T>
spdba_status launch_rcd_activity(const Geom& g, const cx_t<T>* u_hat, int M, double* maxsq, double* gmax,
                                 cudaStream_t st) {
    const long long nb = g.blocks();
    long long grid = (nb + 7) / 8;
    if (grid > 152 * 16) grid = 152 * 16;
    rcd_activity_kernel<T><<<(unsigned)grid, 256, 0, st>>>(g, u_hat, M, g.modes(), maxsq, gmax);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

// ------------------------------------------------------------------ update
constexpr int RCD_TM = 64;             // modes per tile
constexpr int RCD_COLS = 2 * RCD_TM;   // real columns per tile
constexpr int RCD_NT = 256;            // threads: two threads per real column
constexpr int RCD_RG = RCD_NT / RCD_COLS;

template <int MM> __host__ __device__ constexpr int rcd_smem_elems() { return 2 * MM * MM + 2 * MM * RCD_COLS; }

// acc += dot(row[0 .. MM), col[0 .. MM)) with 16-byte row reads
// (two partial sums: half the dependent FMA chain)
template <int MM>
__device__ __forceinline__ float rcd_dot(const float* __restrict__ row, const float (&col)[MM]) {
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int i = 0; i < MM; i += 4) {
        const float4 v = *reinterpret_cast<const float4*>(row + i);
        a0 = fmaf(v.x, col[i], a0);
        a1 = fmaf(v.y, col[i + 1], a1);
        a0 = fmaf(v.z, col[i + 2], a0);
        a1 = fmaf(v.w, col[i + 3], a1);
    }
    return a0 + a1;
}
template <int MM>
__device__ __forceinline__ double rcd_dot(const double* __restrict__ row, const double (&col)[MM]) {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < MM; i += 2) {
        const double2 v = *reinterpret_cast<const double2*>(row + i);
        acc = fma(v.x, col[i], acc);
        acc = fma(v.y, col[i + 1], acc);
    }
    return acc;
}

// CTAs per SM the update kernel is compiled for: three for complex64 up to 48
// components (shared memory 67.6 KB at 48), else as registers allow
template <typename T, int MM> struct RcdOcc {
    static constexpr int value = sizeof(T) == 4 ? (MM <= 48 ? 3 : 2) : 1;
};

template <typename T, int MM>
__global__ void __launch_bounds__(RCD_NT, RcdOcc<T, MM>::value) rcd_update_kernel(Geom g, RcdArgs<T> a, int dense) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sVt = reinterpret_cast<T*>(smem_raw);   // sVt[j * MM + i] = V[i][j] (zero padded)
    T* sV = sVt + MM * MM;                     // sV[i * MM + j] = V[i][j]
    T* sU = sV + MM * MM;                      // u_hat tile: row m, column 2 t + part
    T* sY = sU + MM * RCD_COLS;                // b, then z, then the result
    const int M = a.M;
    const long long n = a.n;
    for (int e = threadIdx.x; e < MM * MM; e += RCD_NT) {
        const int i = e / MM, j = e - (e / MM) * MM;
        const T v = (i < M && j < M) ? a.V[i * M + j] : (T)0;
        sV[i * MM + j] = v;
        sVt[j * MM + i] = v;
    }
    const int B0 = g.b[0], B1 = g.b[1], B2 = g.b[2];
    const int bm = B0 * B1 * B2;
    const int tpb = (bm + RCD_TM - 1) / RCD_TM;
    const long long nblk = dense ? g.blocks() : (long long)*a.count;
    const long long items = nblk * tpb;
    if (blockIdx.x == 0 && a.stats) {
        // the step's share of non-frozen blocks (one run), as the CH update kernels
        if (threadIdx.x == 0) {
            DevStats& s = a.stats[0];
            if (dense) {
                s.ratio_sum += 1.0;
            } else {
                const unsigned long long nfi = s.n_active + s.n_transition;
                s.ratio_sum += (double)nfi * (1.0 / (double)g.bpr());
                s.list_modes += (double)nfi * (double)bm * (double)a.M;   // modes of every component
                s.ctl_nf += nfi;
                s.ctl_steps += 1;
            }
        }
    }
    const int c = threadIdx.x % RCD_COLS;   // this thread's real column
    const int rg = threadIdx.x / RCD_COLS;  // its row group
    const int tm = c >> 1;                  // the column's mode in the tile
    for (long long w = blockIdx.x; w < items; w += gridDim.x) {
        const long long blk = dense ? w / tpb : (long long)a.list[w / tpb];
        const int ti = (int)(w % tpb);
        const long long b2 = blk % g.nb[2], b1 = (blk / g.nb[2]) % g.nb[1], b0 = blk / (g.nb[2] * g.nb[1]);
        __syncthreads();   // the previous tile's stores have read sY
        // load u_hat and b = u_hat + dt g_hat of the tile's modes: thread e handles
        // mode t = e % RCD_TM of components m = e / RCD_TM, e / RCD_TM + RCD_NT / RCD_TM, ...
        constexpr int LSTEP = RCD_NT / RCD_TM;   // components per pass of the CTA
        constexpr int LPER = (MM + LSTEP - 1) / LSTEP;
        const int lt = threadIdx.x % RCD_TM, lm0 = threadIdx.x / RCD_TM;
        const int lo = ti * RCD_TM + lt;
        const bool lvalid = lo < bm;
        long long lidx = 0;
        if (lvalid) {
            const int d2 = lo % B2, d1 = (lo / B2) % B1, d0 = lo / (B2 * B1);
            lidx = ((b0 * B0 + d0) * g.n[1] + (b1 * B1 + d1)) * g.n[2] + (b2 * B2 + d2);
        }
        {
            cx_t<T> u[LPER], gg[LPER];
#pragma unroll
            for (int k = 0; k < LPER; ++k) {
                const int m = lm0 + LSTEP * k;
                u[k] = mk<cx_t<T>>((T)0, (T)0);
                gg[k] = u[k];
                if (m < M && lvalid) {
                    u[k] = a.u_hat[(long long)m * n + lidx];
                    gg[k] = a.g_hat[(long long)m * n + lidx];
                }
            }
#pragma unroll
            for (int k = 0; k < LPER; ++k) {
                const int m = lm0 + LSTEP * k;
                if (m < MM) {
                    sU[m * RCD_COLS + 2 * lt] = u[k].x;
                    sU[m * RCD_COLS + 2 * lt + 1] = u[k].y;
                    sY[m * RCD_COLS + 2 * lt] = u[k].x + a.dt * gg[k].x;
                    sY[m * RCD_COLS + 2 * lt + 1] = u[k].y + a.dt * gg[k].y;
                }
            }
        }
        __syncthreads();
        // this column's mode: |k|^2 and (transition blocks) the taper weight
        const int o = ti * RCD_TM + tm;
        const bool valid = o < bm;
        const int d2 = o % B2, d1 = (o / B2) % B1, d0 = o / (B2 * B1);
        const long long z = b0 * B0 + d0, y = b1 * B1 + d1, x = b2 * B2 + d2;
        const T k2 = valid ? a.k2ax[0][z] + a.k2ax[1][y] + a.k2ax[2][x] : (T)0;
        const int st = dense ? SPDBA_ACTIVE : a.states[blk];
        T sg = (T)1;
        if (st == SPDBA_TRANSITION) {
            const unsigned ch = a.chi[blk];
            const int a0 = 3 - g.ndim;
            const int l[3] = {d0, d1, d2};
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                if (ax < a0) continue;
                if ((ch >> (2 * (ax - a0))) & 1u) sg *= a.taper[ax][l[ax]];
                if ((ch >> (2 * (ax - a0) + 1)) & 1u) sg *= a.taper[ax][g.b[ax] - 1 - l[ax]];
            }
        }
        // z = V^T b, scaled by 1 / (1 + dt k^2 lambda_j)
        T col[MM];
#pragma unroll
        for (int i = 0; i < MM; ++i) col[i] = sY[i * RCD_COLS + c];
        __syncthreads();
        for (int j = rg; j < M; j += RCD_RG) {
            const T zj = rcd_dot<MM>(sVt + j * MM, col);
            sY[j * RCD_COLS + c] = zj / ((T)1 + a.dt * k2 * a.lam[j]);
        }
        __syncthreads();
        // x = V z, then the state's rule: ACTIVE x, TRANSITION u + sigma (x - u)
#pragma unroll
        for (int j = 0; j < MM; ++j) col[j] = sY[j * RCD_COLS + c];
        __syncthreads();
        for (int i = rg; i < M; i += RCD_RG) {
            const T xi = rcd_dot<MM>(sV + i * MM, col);
            const T ui = sU[i * RCD_COLS + c];
            sY[i * RCD_COLS + c] = st == SPDBA_ACTIVE ? xi : ui + sg * (xi - ui);
        }
        __syncthreads();
        if (lvalid) {
#pragma unroll
            for (int k = 0; k < LPER; ++k) {
                const int m = lm0 + LSTEP * k;
                if (m < M)
                    a.u_hat[(long long)m * n + lidx] =
                        mk<cx_t<T>>(sY[m * RCD_COLS + 2 * lt], sY[m * RCD_COLS + 2 * lt + 1]);
            }
        }
    }
}

// Launch shape of one update kernel instantiation: fixed by the kernel, set up
// once per process by rcd_prepare (at plan creation, outside any capture).
template <typename T, int MM> struct RcdShape {
    static int per_sm;
    static int nsm;
};
template <typename T, int MM> int RcdShape<T, MM>::per_sm = 0;
template <typename T, int MM> int RcdShape<T, MM>::nsm = 0;

template <typename T, int MM> static spdba_status prepare_mm() {
    if (RcdShape<T, MM>::per_sm > 0) return SPDBA_OK;
    const int smem = rcd_smem_elems<MM>() * (int)sizeof(T);
    const void* f = (const void*)rcd_update_kernel<T, MM>;
    if (smem > 48 * 1024) SPDBA_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int k = 0, dev = 0, nsm = 0;
    SPDBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, f, RCD_NT, smem));
    SPDBA_CUDA(cudaGetDevice(&dev));
    SPDBA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    RcdShape<T, MM>::nsm = nsm < 1 ? 1 : nsm;
    RcdShape<T, MM>::per_sm = k < 1 ? 1 : k;
    return SPDBA_OK;
}

template <typename T, int MM> static spdba_status update_go(const Geom& g, const RcdArgs<T>& a, int dense,
                                                            cudaStream_t st) {
    if (RcdShape<T, MM>::per_sm == 0) return fail(SPDBA_ERR_STATE, "RCD update kernel not prepared");
    const int smem = rcd_smem_elems<MM>() * (int)sizeof(T);
    const int bm = g.b[0] * g.b[1] * g.b[2];
    const long long items = g.blocks() * ((bm + RCD_TM - 1) / RCD_TM);
    long long grid = (long long)RcdShape<T, MM>::per_sm * RcdShape<T, MM>::nsm;
    if (grid > items) grid = items;
    if (grid < 1) grid = 1;
    rcd_update_kernel<T, MM><<<(unsigned)grid, RCD_NT, smem, st>>>(g, a, dense);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

template <typename T> spdba_status rcd_prepare(int M) {
    if (M < 1) return fail(SPDBA_ERR_ARG, "RCD needs at least one component");
    {
        // the reaction kernel's staging column: M values per thread
        const int smem = kRcdMaxComponents * RCD_RX_NT * (int)sizeof(T);
        if (smem > 48 * 1024)
            SPDBA_CUDA(cudaFuncSetAttribute((const void*)rcd_reaction_kernel<T>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    }
    if (M <= 4) return prepare_mm<T, 4>();
    if (M <= 8) return prepare_mm<T, 8>();
    if (M <= 16) return prepare_mm<T, 16>();
    if (M <= 32) return prepare_mm<T, 32>();
    if (M <= 48) return prepare_mm<T, 48>();
    if (M <= 64) return prepare_mm<T, 64>();
    return fail(SPDBA_ERR_UNSUPPORTED, "RCD with %d components (at most %d)", M, kRcdMaxComponents);
}

template <typename T> spdba_status launch_rcd_update(const Geom& g, const RcdArgs<T>& a, int dense, cudaStream_t st) {
    const int M = a.M;
    if (M <= 4) return update_go<T, 4>(g, a, dense, st);
    if (M <= 8) return update_go<T, 8>(g, a, dense, st);
    if (M <= 16) return update_go<T, 16>(g, a, dense, st);
    if (M <= 32) return update_go<T, 32>(g, a, dense, st);
    if (M <= 48) return update_go<T, 48>(g, a, dense, st);
    if (M <= 64) return update_go<T, 64>(g, a, dense, st);
    return fail(SPDBA_ERR_UNSUPPORTED, "RCD with %d components (at most %d)", M, kRcdMaxComponents);
}

template spdba_status launch_rcd_reaction<float>(float2*, long long, int, float, float, float, float, cudaStream_t);
template spdba_status launch_rcd_reaction<double>(double2*, long long, int, double, double, double, double,
                                                  cudaStream_t);
template spdba_status launch_rcd_activity<float>(const Geom&, const float2*, int, double*, double*, cudaStream_t);
template spdba_status launch_rcd_activity<double>(const Geom&, const double2*, int, double*, double*, cudaStream_t);
template spdba_status launch_rcd_update<float>(const Geom&, const RcdArgs<float>&, int, cudaStream_t);
template spdba_status launch_rcd_update<double>(const Geom&, const RcdArgs<double>&, int, cudaStream_t);
template spdba_status rcd_prepare<float>(int);
template spdba_status rcd_prepare<double>(int);

}  // namespace spdba
