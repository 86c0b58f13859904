// Cahn-Hilliard semi-implicit Fourier update (conserved CH-form dynamics of
// S3.1, semi-implicit update of S4.2 with M = 1):
//     new(k) = (c_hat(k) - dt k^2 g_hat(k)) / (1 + dt kappa k^4)
// Regular mode runs it on every mode; sp-DBA mode runs it only on the listed
// (non-frozen) blocks: ACTIVE modes take new(k), TRANSITION modes take
// c_hat + sigma(k) (new - c_hat) (S1.1, Eq. S.1), FROZEN modes are never read.
#include <math.h>

#include <type_traits>

#include "blocks.h"
#include "ch_math.cuh"

namespace spdba {

template <typename T> std::vector<T> k2_table(long long n, double dx) {
    std::vector<T> v((size_t)n);
    const double two_pi = 6.283185307179586476925286766559;
    for (long long j = 0; j < n; ++j) {
        long long jj = j <= n / 2 ? j : j - n;
        double k = two_pi * (double)jj / ((double)n * dx);
        v[(size_t)j] = (T)(k * k);
    }
    return v;
}
template <typename T> std::vector<T> taper_table(int B) {
    std::vector<T> v((size_t)B);
    const double pi = 3.14159265358979323846264338327950288;
    for (int i = 0; i < B; ++i) v[(size_t)i] = B < 2 ? (T)1 : (T)(0.5 * (1.0 - std::cos(pi * i / (double)(B - 1))));
    return v;
}
template std::vector<float> k2_table<float>(long long, double);
template std::vector<double> k2_table<double>(long long, double);
template std::vector<float> taper_table<float>(int);
template std::vector<double> taper_table<double>(int);

// Two consecutive modes along the fast axis move together (one 16-byte access
// for complex64).
__device__ __forceinline__ void load2(const float2* p, float2& a, float2& b) {
    float4 v = *reinterpret_cast<const float4*>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void store2(float2* p, float2 a, float2 b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void load2(const double2* p, double2& a, double2& b) { a = p[0]; b = p[1]; }
__device__ __forceinline__ void store2(double2* p, double2 a, double2 b) { p[0] = a; p[1] = b; }

// Regular: every mode, two consecutive modes per thread along the fast axis.
template <typename T>
__global__ void ch_dense_kernel(Geom g, CHUpdateArgs<T> a) {
    const long long npairs = g.modes() / 2;
    if (blockIdx.x == 0 && a.stats)
        for (long long r = threadIdx.x; r < g.runs(); r += blockDim.x) a.stats[r].ratio_sum += 1.0;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < npairs;
         u += (long long)gridDim.x * blockDim.x) {
        long long e = 2 * u;
        long long x = e % g.n[2];
        long long r = e / g.n[2];
        long long y = r % g.n[1], z = r / g.n[1];
        T kzy = a.k2ax[0][z] + a.k2ax[1][y];
        cx_t<T> c0, c1, g0, g1;
        load2(a.c_hat + e, c0, c1);
        load2(a.g_hat + e, g0, g1);
        c0 = ch_new(c0, g0, kzy + a.k2ax[2][x], a.dt, a.dtkappa);
        c1 = ch_new(c1, g1, kzy + a.k2ax[2][x + 1], a.dt, a.dtkappa);
        store2(a.c_hat + e, c0, c1);
    }
}

// sp-DBA: one warp per listed block, mode pairs along the fast axis.  Block
// and mode coordinates are 32-bit (block maps and fields of a group hold
// fewer than 2^31 entries along each axis product used here) and divided by
// precomputed multiplicative inverses (fd_h: pairs per block row, fd_b1: the
// block edge along axis 1; fd_nb2, fd_nb1: the block map's extents).
template <typename T>
__global__ void ch_list_kernel(Geom g, CHUpdateArgs<T> a, FastDiv fd_h, FastDiv fd_b1, FastDiv fd_nb2,
                               FastDiv fd_nb1) {
    const int lane = threadIdx.x & 31;
    const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int cnt = *a.count;
    const int B0 = g.b[0], B1 = g.b[1], B2 = g.b[2];
    const long long nmodes = (long long)B0 * B1 * B2;
    if (blockIdx.x == 0 && a.stats) {
        const double inv = 1.0 / (double)g.live_bpr();
        for (long long r = threadIdx.x; r < g.runs(); r += blockDim.x) {
            const unsigned long long nfi = a.stats[r].n_active + a.stats[r].n_transition;
            double nf = (double)nfi;
            a.stats[r].ratio_sum += nf * inv;
            a.stats[r].list_modes += nf * (double)nmodes;
            a.stats[r].ctl_nf += nfi;       // an adaptive step of the control interval
            a.stats[r].ctl_steps += 1;
        }
    }
    const int H = B2 / 2;
    const int npair = (int)(nmodes / 2);
    const long long n1 = g.n[1], n2 = g.n[2];
    for (long long w = warp0; w < cnt; w += nwarps) {
        const int blk = a.list[w];
        const int st = a.states[blk];
        const unsigned ch = a.chi[blk];
        const int q = (int)fd_nb2.div((uint32_t)blk);
        const int b2 = blk - q * (int)g.nb[2];
        const int b0 = (int)fd_nb1.div((uint32_t)q), b1 = q - b0 * (int)g.nb[1];
        for (int m = lane; m < npair; m += 32) {
            const int rr = (int)fd_h.div((uint32_t)m);
            const int l2 = (m - rr * H) * 2;
            const int l0 = (int)fd_b1.div((uint32_t)rr), l1 = rr - l0 * B1;
            const int z = b0 * B0 + l0, y = b1 * B1 + l1, x = b2 * B2 + l2;
            const long long e = ((long long)z * n1 + y) * n2 + x;
            T kzy = a.k2ax[0][z] + a.k2ax[1][y];
            cx_t<T> c0, c1, g0, g1;
            load2(a.c_hat + e, c0, c1);
            load2(a.g_hat + e, g0, g1);
            cx_t<T> n0 = ch_new(c0, g0, kzy + a.k2ax[2][x], a.dt, a.dtkappa);
            cx_t<T> n1v = ch_new(c1, g1, kzy + a.k2ax[2][x + 1], a.dt, a.dtkappa);
            if (st == SPDBA_TRANSITION) {
                n0 = ch_blend<T>(c0, n0, a.taper, g, ch, l0, l1, l2);
                n1v = ch_blend<T>(c1, n1v, a.taper, g, ch, l0, l1, l2 + 1);
            }
            store2(a.c_hat + e, n0, n1v);
        }
    }
}

// sp-DBA, complex64, 8^3 blocks of a single 3-D field: the warp-per-block
// update with the block shape fixed at compile time.  Lane l keeps the mode
// pair (x = 2 (l % 4), y = l / 4) of every z plane of the block, so its x and y
// wavenumbers and transition coordinates are fixed, the eight planes are eight
// independent row loads of ĉ and ĝ at a fixed stride, and no index is divided
// at run time.  The same arithmetic as ch_list_kernel, bit for bit.
__global__ void __launch_bounds__(256) ch_list8_kernel(Geom g, CHUpdateArgs<float> a) {
    constexpr int B = 8;
    const int lane = threadIdx.x & 31;
    const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int cnt = *a.count;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats) {
        const unsigned long long nfi = a.stats[0].n_active + a.stats[0].n_transition;
        const double nf = (double)nfi;
        a.stats[0].ratio_sum += nf * (1.0 / (double)g.live_bpr());
        a.stats[0].list_modes += nf * (double)(B * B * B);
        a.stats[0].ctl_nf += nfi;       // an adaptive step of the control interval
        a.stats[0].ctl_steps += 1;
    }
    const int l2 = (lane & 3) * 2, l1 = lane >> 2;
    const int nb2 = (int)g.nb[2], nb1 = (int)g.nb[1];
    const long long n2 = g.n[2], plane = g.n[1] * g.n[2];
    for (long long w = warp0; w < cnt; w += nwarps) {
        const int blk = a.list[w];
        const int st = a.states[blk];
        const unsigned ch = a.chi[blk];
        const int q = blk / nb2;
        const int b2 = blk - q * nb2, b0 = q / nb1, b1 = q - b0 * nb1;
        const int x = b2 * B + l2, y = b1 * B + l1, z0 = b0 * B;
        const float ky = a.k2ax[1][y], kx0 = a.k2ax[2][x], kx1 = a.k2ax[2][x + 1];
        float2* cp = a.c_hat + (long long)z0 * plane + (long long)y * n2 + x;
        const float2* gp = a.g_hat + (long long)z0 * plane + (long long)y * n2 + x;
        // the block's sixteen 16-byte loads of this lane are all issued before any store
        float4 cvs[B], gvs[B];
#pragma unroll
        for (int l0 = 0; l0 < B; ++l0) {
            cvs[l0] = *reinterpret_cast<const float4*>(cp + l0 * plane);
            gvs[l0] = *reinterpret_cast<const float4*>(gp + l0 * plane);
        }
#pragma unroll
        for (int l0 = 0; l0 < B; ++l0) {
            const float4 cv = cvs[l0], gv = gvs[l0];
            const float kzy = a.k2ax[0][z0 + l0] + ky;
            const float2 c0 = make_float2(cv.x, cv.y), c1 = make_float2(cv.z, cv.w);
            float2 n0 = ch_new(c0, make_float2(gv.x, gv.y), kzy + kx0, a.dt, a.dtkappa);
            float2 n1 = ch_new(c1, make_float2(gv.z, gv.w), kzy + kx1, a.dt, a.dtkappa);
            if (st == SPDBA_TRANSITION) {
                n0 = ch_blend<float>(c0, n0, a.taper, g, ch, l0, l1, l2);
                n1 = ch_blend<float>(c1, n1, a.taper, g, ch, l0, l1, l2 + 1);
            }
            *reinterpret_cast<float4*>(cp + l0 * plane) = make_float4(n0.x, n0.y, n1.x, n1.y);
        }
    }
}

template <typename T> spdba_status launch_ch_update(const Geom& g, const CHUpdateArgs<T>& a, int dense, cudaStream_t st) {
    if (dense) {
        long long npairs = g.modes() / 2;
        long long grid = (npairs + 255) / 256;
        if (grid > 152 * 16) grid = 152 * 16;
        ch_dense_kernel<T><<<(unsigned)grid, 256, 0, st>>>(g, a);
    } else {
        long long nb = g.blocks();
        long long grid = (nb * 32 + 255) / 256;
        if (grid > 152 * 16) grid = 152 * 16;
        bool fixed8 = false;
        if constexpr (std::is_same<T, float>::value) {
            fixed8 = g.ndim == 3 && g.runs() == 1 && g.b[0] == 8 && g.b[1] == 8 && g.b[2] == 8 &&
                     g.blocks() < 0x7fffffffLL;
            if (fixed8) ch_list8_kernel<<<(unsigned)grid, 256, 0, st>>>(g, a);
        }
        if (!fixed8) {
            FastDiv fd_h, fd_b1, fd_nb2, fd_nb1;
            fd_h.init((uint32_t)(g.b[2] / 2));
            fd_b1.init((uint32_t)g.b[1]);
            fd_nb2.init((uint32_t)g.nb[2]);
            fd_nb1.init((uint32_t)g.nb[1]);
            ch_list_kernel<T><<<(unsigned)grid, 256, 0, st>>>(g, a, fd_h, fd_b1, fd_nb2, fd_nb1);
        }
    }
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}
template spdba_status launch_ch_update<float>(const Geom&, const CHUpdateArgs<float>&, int, cudaStream_t);
template spdba_status launch_ch_update<double>(const Geom&, const CHUpdateArgs<double>&, int, cudaStream_t);

}  // namespace spdba
