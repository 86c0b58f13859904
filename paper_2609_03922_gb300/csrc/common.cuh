// Shared device helpers for the sp-DBA kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace spdba {

// Complex value types: interleaved (re, im).
template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };
template <typename T> using cx_t = typename Cx<T>::type;

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
    C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
// Rounded multiply and fused multiply-add with the rounding pinned: every
// transform kernel evaluates a product the same way, whatever the compiler
// would contract in its context, so the launch forms of a pass (one group per
// launch or many; any tile width) give bit-identical values.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return mk<C>(fma_rn(a.x, b.x, -mul_rn(a.y, b.y)), fma_rn(a.x, b.y, mul_rn(a.y, b.x)));
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) {
    return mk<C>(mul_rn(a.x, s), mul_rn(a.y, s));
}
// multiply by s*i for s = +-1
template <int S, typename C> __device__ __forceinline__ C cmul_si(C a) {
    return S > 0 ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}

// cos and sin of 2*pi*m/16, m = 0..15, from the closed forms
// cos(pi/8) = sqrt(2 + sqrt 2)/2, sin(pi/8) = sqrt(2 - sqrt 2)/2, cos(pi/4) = sqrt(2)/2.
__host__ __device__ constexpr double cos16(int m) {
    constexpr double C1 = 0.92387953251128674, S1 = 0.38268343236508977, R2 = 0.70710678118654752;
    switch (m & 15) {
        case 0: return 1.0;  case 1: return C1;  case 2: return R2;  case 3: return S1;
        case 4: return 0.0;  case 5: return -S1; case 6: return -R2; case 7: return -C1;
        case 8: return -1.0; case 9: return -C1; case 10: return -R2; case 11: return -S1;
        case 12: return 0.0; case 13: return S1; case 14: return R2; default: return C1;
    }
}
__host__ __device__ constexpr double sin16(int m) { return cos16(m - 4); }

// x * exp(SIGN * 2 pi i m / 16) with compile-time m (exact for multiples of 4)
template <int M, int SIGN, typename C> __device__ __forceinline__ C twiddle16(C x) {
    using T = decltype(C::x);
    constexpr int m = M & 15;
    if constexpr (m == 0) return x;
    else if constexpr (m == 4) return cmul_si<SIGN>(x);
    else if constexpr (m == 8) return mk<C>(-x.x, -x.y);
    else if constexpr (m == 12) return cmul_si<-SIGN>(x);
    else {
        constexpr T c = (T)cos16(m);
        constexpr T s = (T)(SIGN * sin16(m));
        return mk<C>(fma_rn(x.x, c, -mul_rn(x.y, s)), fma_rn(x.x, s, mul_rn(x.y, c)));
    }
}

// In-register DFT of length R with kernel exp(SIGN * 2 pi i n k / R), natural order in and out.
template <int R, int SIGN, typename C> struct Dft;

template <int SIGN, typename C> struct Dft<2, SIGN, C> {
    static __device__ __forceinline__ void run(C* v) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b); v[1] = csub(a, b);
    }
};
template <int SIGN, typename C> struct Dft<3, SIGN, C> {
    static __device__ __forceinline__ void run(C* v) {
        using T = decltype(C::x);
        const T h = (T)0.5;
        const T r3 = (T)(SIGN * 0.86602540378443865);   // SIGN * sqrt(3)/2
        C t1 = cadd(v[1], v[2]);
        C t2 = mk<C>(fma_rn(-h, t1.x, v[0].x), fma_rn(-h, t1.y, v[0].y));
        C d = csub(v[1], v[2]);
        C t3 = mk<C>(mul_rn(-r3, d.y), mul_rn(r3, d.x));   // i * r3 * (v1 - v2)
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    }
};
template <int SIGN, typename C> struct Dft<4, SIGN, C> {
    static __device__ __forceinline__ void run(C* v) {
        C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        C t2 = cadd(v[1], v[3]), t3 = cmul_si<SIGN>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3); v[3] = csub(t1, t3);
    }
};

// R = A * B by the four-step factorisation, all indices compile-time.
template <int A, int B, int SIGN, typename C> struct DftAB {
    static constexpr int R = A * B;
    template <int b, int k1> static __device__ __forceinline__ C tw(C x) {
        return twiddle16<(b * k1) * (16 / R), SIGN>(x);
    }
    template <int b> static __device__ __forceinline__ void step1(const C* v, C* u) {
        if constexpr (b < B) {
            C t[A];
#pragma unroll
            for (int a = 0; a < A; ++a) t[a] = v[b + B * a];
            Dft<A, SIGN, C>::run(t);
            step1_tw<b, 0>(t, u);
            step1<b + 1>(v, u);
        }
    }
    template <int b, int k1> static __device__ __forceinline__ void step1_tw(const C* t, C* u) {
        if constexpr (k1 < A) {
            u[b + B * k1] = tw<b, k1>(t[k1]);
            step1_tw<b, k1 + 1>(t, u);
        }
    }
    static __device__ __forceinline__ void run(C* v) {
        C u[R];
        step1<0>(v, u);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
            C t[B];
#pragma unroll
            for (int b = 0; b < B; ++b) t[b] = u[b + B * k1];
            Dft<B, SIGN, C>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = t[k2];
        }
    }
};
template <int SIGN, typename C> struct Dft<8, SIGN, C> {
    static __device__ __forceinline__ void run(C* v) { DftAB<2, 4, SIGN, C>::run(v); }
};
template <int SIGN, typename C> struct Dft<16, SIGN, C> {
    static __device__ __forceinline__ void run(C* v) { DftAB<4, 4, SIGN, C>::run(v); }
};

// Division of 0 <= x < 2^31 by a divisor 1 <= d < 2^31 fixed at plan time:
// q = floor(x * m / 2^p) with p = 31 + ceil(log2 d), m = ceil(2^p / d) (the
// round-up method of Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994); exact because x < 2^31 <= 2^p / d.
struct FastDiv {
    uint32_t d = 1, m = 0;   // m = 0: d == 1
    int s = 0;               // p - 32
    __host__ __device__ void init(uint32_t dd) {
        d = dd;
        if (d <= 1) { d = 1; m = 0; s = 0; return; }
        int l = 0;
        while ((1ull << l) < (unsigned long long)d) ++l;
        const int p = 31 + l;
        m = (uint32_t)(((1ull << p) + d - 1) / d);
        s = p - 32;
    }
    __device__ __forceinline__ uint32_t div(uint32_t x) const { return m ? (__umulhi(x, m) >> s) : x; }
};

// FP64 max over warp lanes
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// atomic max of a non-negative double through its bit pattern; the atomic is
// skipped when a plain read already shows a value at least as large (the max
// only grows), which keeps many CTAs from serializing on one address.
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    if (v <= *reinterpret_cast<volatile double*>(addr)) return;
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// |q|^2 in FP64 as re*re + im*im with each product rounded, then the sum rounded
// (no contraction), the same evaluation the oracle uses.
__device__ __forceinline__ double mode_sq(float2 q) {
    double re = (double)q.x, im = (double)q.y;
    return __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
}
__device__ __forceinline__ double mode_sq(double2 q) {
    return __dadd_rn(__dmul_rn(q.x, q.x), __dmul_rn(q.y, q.y));
}

}  // namespace spdba
