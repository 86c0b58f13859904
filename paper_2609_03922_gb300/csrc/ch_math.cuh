// Cahn-Hilliard semi-implicit update of one mode and the transition blend
// (S3.1 conserved dynamics, S4.2 semi-implicit form with M = 1; S1.1 Eq. S.1).
#pragma once
#include "common.cuh"
#include "geom.cuh"

namespace spdba {

// Evaluation order is pinned with explicit fma so that the Regular and the
// sp-DBA kernels produce bit-identical values for the same mode.  The FP32
// reciprocal is the hardware approximation (at most 2 ulp), far inside the
// FP32 path's tolerance; every FP32 update kernel shares this function.
__device__ __forceinline__ float2 ch_new(float2 c, float2 g, float k2, float dt, float dtkappa) {
    float den = __fmaf_rn(dtkappa, __fmul_rn(k2, k2), 1.0f);
    float inv = __fdividef(1.0f, den);
    float a = __fmul_rn(dt, k2);
    return make_float2(__fmul_rn(__fmaf_rn(-a, g.x, c.x), inv), __fmul_rn(__fmaf_rn(-a, g.y, c.y), inv));
}
__device__ __forceinline__ double2 ch_new(double2 c, double2 g, double k2, double dt, double dtkappa) {
    double den = __fma_rn(dtkappa, __dmul_rn(k2, k2), 1.0);
    double a = __dmul_rn(dt, k2);
    return make_double2(__ddiv_rn(__fma_rn(-a, g.x, c.x), den), __ddiv_rn(__fma_rn(-a, g.y, c.y), den));
}

template <typename T>
__device__ __forceinline__ cx_t<T> ch_blend(cx_t<T> c, cx_t<T> nw, const T* const* taper, const Geom& g,
                                            unsigned ch, int l0, int l1, int l2) {
    const int a0 = 3 - g.ndim;
    int l[3] = {l0, l1, l2};
    T sg = (T)1;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (ax < a0) continue;
        unsigned lo = (ch >> (2 * (ax - a0))) & 1u, hi = (ch >> (2 * (ax - a0) + 1)) & 1u;
        if (lo) sg *= taper[ax][l[ax]];
        if (hi) sg *= taper[ax][g.b[ax] - 1 - l[ax]];
    }
    return mk<cx_t<T>>(fma_rn(sg, nw.x - c.x, c.x), fma_rn(sg, nw.y - c.y, c.y));
}

}  // namespace spdba
