// Batched Stockham FFT pass: one CTA transforms a tile of P pencils of length L
// staged in shared memory.  A "pass" transforms one axis of a batch of arrays;
// a multi-dimensional FFT is one pass per axis (an axis of a 1-D signal longer
// than one tile is split four-step into two passes).
//
// Pencil q of a pass (q in [0, O*I)) has its element j at
//     o*sO + i*sI + j*sJ,   o = q / I, i = q % I
// for the input and (with its own strides) the output.  A tile holds P
// consecutive pencils.  When I % P == 0 a tile shares one o and its pencils
// are sI apart; global loads run along whichever of sJ or sI is 1, so rows of
// the tile are read as contiguous 16-byte vectors.
#pragma once
#include "common.cuh"

namespace spdba {

// Radix schedule per pencil length (product of radices == L).
template <int L> struct Radices;
template <int... R> struct RList {};
template <> struct Radices<16> { using type = RList<16>; };
template <> struct Radices<32> { using type = RList<8, 4>; };
template <> struct Radices<64> { using type = RList<8, 8>; };
template <> struct Radices<128> { using type = RList<16, 8>; };
template <> struct Radices<192> { using type = RList<16, 4, 3>; };
template <> struct Radices<256> { using type = RList<16, 16>; };
template <> struct Radices<384> { using type = RList<16, 8, 3>; };
template <> struct Radices<512> { using type = RList<8, 8, 8>; };
template <> struct Radices<1024> { using type = RList<16, 16, 4>; };
template <> struct Radices<2048> { using type = RList<16, 16, 8>; };
template <> struct Radices<4096> { using type = RList<16, 16, 16>; };

// Shared-memory index of element j of pencil p: one pad element every 16 keeps
// the radix-R scatter of the first stage conflict-free, and an odd pencil
// stride keeps transposed (pencil-fastest) row loads conflict-free.
template <int L> struct SmemLayout {
    static constexpr int PSTR = L + L / 16 + 1;
    static __device__ __forceinline__ int idx(int p, int j) { return p * PSTR + j + (j >> 4); }
};

template <typename T> struct PassParams {
    const cx_t<T>* in;
    cx_t<T>* out;
    long long O, I;                       // pencil grid
    long long isO, isI, isJ;              // input strides (elements)
    long long osO, osI, osJ;              // output strides
    const cx_t<T>* tw;                    // exp(-2 pi i m / L), m < L
    const cx_t<T>* tw4;                   // four-step twiddles exp(-2 pi i m / N4), or null
    long long n4;
    T scale;                              // multiply on store (1 = none)
    int generic;                          // 1: I % P != 0, per-pencil address arithmetic
    // CH nonlinearity fused between the inverse and forward x transforms
    T nl_scale;                           // 1 / (number of grid points)
    double* mass;                         // FP64 sum of c, or null
};

// Address of element (p, j) of the tile starting at pencil q0.
template <int P> __device__ __forceinline__ long long tile_addr(long long q0, int p, int j, long long O,
                                                                 long long I, long long sO, long long sI,
                                                                 long long sJ, int generic) {
    if (!generic) {
        long long o = q0 / I, i0 = q0 - o * I;
        return o * sO + (i0 + p) * sI + (long long)j * sJ;
    }
    long long q = q0 + p;
    long long o = q / I, i = q - o * I;
    return o * sO + i * sI + (long long)j * sJ;
}

// ---------------------------------------------------------------- tile load/store
// PFAST: pencils are the unit-stride direction; otherwise elements are.
template <typename T, int L, int P, int NT, bool PFAST>
__device__ __forceinline__ void load_tile(cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
    using SL = SmemLayout<L>;
    const long long npencil = a.O * a.I;
    if constexpr (sizeof(C) == 8) {
        // float2: move pairs as float4
        constexpr int UNITS = P * L / 2;
        constexpr int PER = (UNITS + NT - 1) / NT;
        float4 r[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            int u = threadIdx.x + k * NT;
            if (UNITS % NT == 0 || u < UNITS) {
                int p, j;
                if constexpr (PFAST) { j = u / (P / 2); p = (u % (P / 2)) * 2; }
                else { p = u / (L / 2); j = (u % (L / 2)) * 2; }
                if (q0 + p < npencil) {
                    long long ad = tile_addr<P>(q0, p, j, a.O, a.I, a.isO, a.isI, a.isJ, a.generic);
                    r[k] = __ldg(reinterpret_cast<const float4*>(a.in + ad));
                } else {
                    r[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            int u = threadIdx.x + k * NT;
            if (UNITS % NT == 0 || u < UNITS) {
                int p, j;
                if constexpr (PFAST) {
                    j = u / (P / 2); p = (u % (P / 2)) * 2;
                    sm[SL::idx(p, j)] = mk<C>(r[k].x, r[k].y);
                    sm[SL::idx(p + 1, j)] = mk<C>(r[k].z, r[k].w);
                } else {
                    p = u / (L / 2); j = (u % (L / 2)) * 2;
                    sm[SL::idx(p, j)] = mk<C>(r[k].x, r[k].y);
                    sm[SL::idx(p, j + 1)] = mk<C>(r[k].z, r[k].w);
                }
            }
        }
    } else {
        constexpr int UNITS = P * L;
        constexpr int PER = (UNITS + NT - 1) / NT;
        C r[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            int u = threadIdx.x + k * NT;
            if (UNITS % NT == 0 || u < UNITS) {
                int p, j;
                if constexpr (PFAST) { j = u / P; p = u % P; }
                else { p = u / L; j = u % L; }
                if (q0 + p < npencil) {
                    long long ad = tile_addr<P>(q0, p, j, a.O, a.I, a.isO, a.isI, a.isJ, a.generic);
                    r[k] = __ldg(a.in + ad);
                } else {
                    r[k] = mk<C>(0, 0);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            int u = threadIdx.x + k * NT;
            if (UNITS % NT == 0 || u < UNITS) {
                int p, j;
                if constexpr (PFAST) { j = u / P; p = u % P; }
                else { p = u / L; j = u % L; }
                sm[SL::idx(p, j)] = r[k];
            }
        }
    }
}

template <typename T, int L, int P, int NT, bool PFAST>
__device__ __forceinline__ void store_tile(const cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
    using SL = SmemLayout<L>;
    const long long npencil = a.O * a.I;
    const T s = a.scale;
    if constexpr (sizeof(C) == 8) {
        constexpr int UNITS = P * L / 2;
        constexpr int PER = (UNITS + NT - 1) / NT;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            int u = threadIdx.x + k * NT;
            if (UNITS % NT == 0 || u < UNITS) {
                int p, j;
                C v0, v1;
                if constexpr (PFAST) {
                    j = u / (P / 2); p = (u % (P / 2)) * 2;
                    v0 = sm[SL::idx(p, j)]; v1 = sm[SL::idx(p + 1, j)];
                } else {
                    p = u / (L / 2); j = (u % (L / 2)) * 2;
                    v0 = sm[SL::idx(p, j)]; v1 = sm[SL::idx(p, j + 1)];
                }
                if (q0 + p < npencil) {
                    long long ad = tile_addr<P>(q0, p, j, a.O, a.I, a.osO, a.osI, a.osJ, a.generic);
                    *reinterpret_cast<float4*>(a.out + ad) = make_float4(v0.x * s, v0.y * s, v1.x * s, v1.y * s);
                }
            }
        }
    } else {
        constexpr int UNITS = P * L;
        constexpr int PER = (UNITS + NT - 1) / NT;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            int u = threadIdx.x + k * NT;
            if (UNITS % NT == 0 || u < UNITS) {
                int p, j;
                if constexpr (PFAST) { j = u / P; p = u % P; }
                else { p = u / L; j = u % L; }
                if (q0 + p < npencil) {
                    long long ad = tile_addr<P>(q0, p, j, a.O, a.I, a.osO, a.osI, a.osJ, a.generic);
                    a.out[ad] = cscale(sm[SL::idx(p, j)], s);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- Stockham stages
// One radix-R stage over all P pencils in shared memory.  NS = product of the
// radices already applied.  Butterfly j of a pencil reads elements j + r L/R,
// multiplies element r by W_{NS R}^{r (j mod NS)}, runs a length-R DFT and writes
// to (j / NS) NS R + (j mod NS) + r NS (autosorting; natural order after the
// last stage).
template <typename T, int L, int P, int NT, int SIGN, int NS, int R>
__device__ __forceinline__ void stockham_stage(cx_t<T>* sm, const cx_t<T>* __restrict__ tw) {
    using C = cx_t<T>;
    using SL = SmemLayout<L>;
    constexpr int Q = L / R;
    constexpr int NB = P * Q;
    constexpr int PER = (NB + NT - 1) / NT;
    C v[PER][R];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int b = threadIdx.x + k * NT;
        if (NB % NT == 0 || b < NB) {
            int p = b / Q, j = b % Q;
#pragma unroll
            for (int r = 0; r < R; ++r) v[k][r] = sm[SL::idx(p, j + r * Q)];
            if constexpr (NS > 1) {
                int jm = j % NS;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C w = __ldg(tw + r * jm * (L / (NS * R)));
                    if constexpr (SIGN > 0) w.y = -w.y;
                    v[k][r] = cmul(v[k][r], w);
                }
            }
            Dft<R, SIGN, C>::run(v[k]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int b = threadIdx.x + k * NT;
        if (NB % NT == 0 || b < NB) {
            int p = b / Q, j = b % Q;
            int jm = j % NS;
            int d = (j / NS) * NS * R + jm;
#pragma unroll
            for (int r = 0; r < R; ++r) sm[SL::idx(p, d + r * NS)] = v[k][r];
        }
    }
    __syncthreads();
}

template <typename T, int L, int P, int NT, int SIGN, int NS, int R, int... Rest>
__device__ __forceinline__ void run_stages_impl(cx_t<T>* sm, const cx_t<T>* tw) {
    stockham_stage<T, L, P, NT, SIGN, NS, R>(sm, tw);
    if constexpr (sizeof...(Rest) > 0) run_stages_impl<T, L, P, NT, SIGN, NS * R, Rest...>(sm, tw);
}
template <typename T, int L, int P, int NT, int SIGN, int... Rs>
__device__ __forceinline__ void run_stages_list(cx_t<T>* sm, const cx_t<T>* tw, RList<Rs...>) {
    run_stages_impl<T, L, P, NT, SIGN, 1, Rs...>(sm, tw);
}
// All stages of a length-L transform with kernel exp(SIGN 2 pi i n k / L).
template <typename T, int L, int P, int NT, int SIGN>
__device__ __forceinline__ void run_stages(cx_t<T>* sm, const cx_t<T>* tw) {
    run_stages_list<T, L, P, NT, SIGN>(sm, tw, typename Radices<L>::type{});
}

// Four-step twiddle: element (pencil i, output index j) *= W_N^{i j}.
template <typename T, int L, int P, int NT, int SIGN>
__device__ __forceinline__ void apply_fourstep_twiddle(cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
    using SL = SmemLayout<L>;
    for (int e = threadIdx.x; e < P * L; e += NT) {
        int p = e / L, j = e % L;
        long long q = q0 + p;
        long long i = q % a.I;
        long long m = (i * (long long)j) % a.n4;
        C w = __ldg(a.tw4 + m);
        if constexpr (SIGN > 0) w.y = -w.y;
        sm[SL::idx(p, j)] = cmul(sm[SL::idx(p, j)], w);
    }
    __syncthreads();
}

// Pass modes
enum PassMode : int {
    PASS_PLAIN = 0,      // transform, optional four-step twiddle, scaled store
    PASS_CH_NL = 1,      // inverse transform, c = Re(.)/N, g = c^3 - c, forward transform
};

template <typename T, int L, int P, int NT, int SIGN, int MODE, bool LOADP, bool STOREP>
__global__ void __launch_bounds__(NT) fft_pass_kernel(PassParams<T> a) {
    using C = cx_t<T>;
    using SL = SmemLayout<L>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const long long q0 = (long long)blockIdx.x * P;

    load_tile<T, L, P, NT, LOADP>(sm, a, q0);
    __syncthreads();

    if constexpr (MODE == PASS_PLAIN) {
        run_stages<T, L, P, NT, SIGN>(sm, a.tw);
        if (a.tw4 != nullptr) apply_fourstep_twiddle<T, L, P, NT, SIGN>(sm, a, q0);
    } else if constexpr (MODE == PASS_CH_NL) {
        // inverse transform along this axis completes c = IFFT(c_hat) (scaled by nl_scale)
        run_stages<T, L, P, NT, +1>(sm, a.tw);
        T msum = 0;
        for (int e = threadIdx.x; e < P * L; e += NT) {
            int p = e / L, j = e % L;
            C v = sm[SL::idx(p, j)];
            T c = v.x * a.nl_scale;
            msum += c;
            sm[SL::idx(p, j)] = mk<C>(c * c * c - c, (T)0);
        }
        if (a.mass != nullptr) {
            double ms = (double)msum;
            ms = warp_sum(ms);
            if ((threadIdx.x & 31) == 0) atomicAdd(a.mass, ms);
        }
        __syncthreads();
        run_stages<T, L, P, NT, -1>(sm, a.tw);
    }
    store_tile<T, L, P, NT, STOREP>(sm, a, q0);
}

template <int L> constexpr int smem_bytes_for(int P, int elem) { return P * SmemLayout<L>::PSTR * elem; }

}  // namespace spdba
