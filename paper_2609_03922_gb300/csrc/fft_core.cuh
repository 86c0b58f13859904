// Batched Stockham FFT pass: one CTA transforms a tile of P pencils of length L
// staged in shared memory.  A "pass" transforms one axis of a batch of arrays;
// a multi-dimensional FFT is one pass per axis (a 1-D signal longer than one
// tile is split four-step into two passes).
//
// Pencil q of a pass (q in [0, O*I)) has its element j at
//     o*sO + i*sI + j*sJ,   o = q / I, i = q % I
// for the input and (with its own strides) the output.  A tile holds P
// consecutive pencils.  When I % P == 0 a tile shares one o and its pencils
// are sI apart; global traffic runs along whichever of sJ or sI is 1, so rows
// of the tile move as contiguous 16-byte vectors.
//
// Two shared-memory layouts:
//   A (pencil-major, padded): element (p, j) at p*PSTR + j + j/16.  Used when
//     pencils are contiguous in memory (sJ == 1).  Butterflies are assigned
//     with j fastest; the pad keeps the strided scatter of a stage spread
//     over the banks.
//   B (row-major): element (p, j) at j*P + p.  Used when pencils are the unit-
//     stride direction (sI == 1): a tile row in memory is a row in shared
//     memory.  Butterflies are assigned with p fastest, so every stage access
//     of a warp touches 16 consecutive elements per half-warp (conflict-free).
#pragma once
#include <type_traits>

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

// Layout A; ODD selects an odd pencil stride (needed when pencils are read
// transposed, pencil-fastest), otherwise the stride stays even so that a pair
// (j, j+1) is one aligned 16-byte shared-memory word.
template <int L, int P, bool ODD> struct LayoutA {
    static constexpr int PSTR = L + L / 16 + (ODD ? 1 : 0);
    static constexpr int SIZE = P * PSTR;
    static constexpr bool PMAP = false;
    static __device__ __forceinline__ int idx(int p, int j) { return p * PSTR + j + (j >> 4); }
};
template <int L, int P> struct LayoutB {
    static constexpr int SIZE = P * L;
    static constexpr bool PMAP = true;
    static __device__ __forceinline__ int idx(int p, int j) { return j * P + p; }
};
// Kept for the simple (non-pipelined) kernel.
template <int L> struct SmemLayout {
    static constexpr int PSTR = L + L / 16 + 1;
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
    T nl_scale;                           // 1 / (number of grid points of one field)
    double* mass;                         // FP64 sum of c per field (strided), or null
    int mass_stride;                      // doubles between consecutive fields' accumulators
    long long mass_ppr;                   // pencils per field
};

// Address of element (p, j) of the tile starting at pencil q0.
__device__ __forceinline__ long long tile_addr(long long q0, int p, int j, long long I, long long sO, long long sI,
                                               long long sJ, int generic) {
    if (!generic) {
        long long o = q0 / I, i0 = q0 - o * I;
        return o * sO + (i0 + p) * sI + (long long)j * sJ;
    }
    long long q = q0 + p;
    long long o = q / I, i = q - o * I;
    return o * sO + i * sI + (long long)j * sJ;
}

// ---------------------------------------------------------------- cp.async
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------- tile load/store
// Synchronous load (used by the simple kernel and for uneven tiles).
template <typename T, int L, int P, int NT, bool PFAST, class LY>
__device__ __forceinline__ void load_tile(cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
    const long long npencil = a.O * a.I;
    if constexpr (sizeof(C) == 8) {
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
                    long long ad = tile_addr(q0, p, j, a.I, a.isO, a.isI, a.isJ, a.generic);
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
                    sm[LY::idx(p, j)] = mk<C>(r[k].x, r[k].y);
                    sm[LY::idx(p + 1, j)] = mk<C>(r[k].z, r[k].w);
                } else {
                    p = u / (L / 2); j = (u % (L / 2)) * 2;
                    sm[LY::idx(p, j)] = mk<C>(r[k].x, r[k].y);
                    sm[LY::idx(p, j + 1)] = mk<C>(r[k].z, r[k].w);
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
                    long long ad = tile_addr(q0, p, j, a.I, a.isO, a.isI, a.isJ, a.generic);
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
                sm[LY::idx(p, j)] = r[k];
            }
        }
    }
}

// Asynchronous load of a full tile (I % P == 0).  Layout B keeps a pencil
// pair of a row contiguous, so complex64 moves in 16-byte pieces; the padded
// layout A moves complex64 one element (8 bytes) at a time.
template <typename T, int L, int P, int NT, bool PFAST, class LY>
__device__ __forceinline__ void issue_tile(cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
    const long long o = q0 / a.I, i0 = q0 - o * a.I;
    const C* base = a.in + o * a.isO + i0 * a.isI;
    if constexpr (sizeof(C) == 8 && PFAST) {
        constexpr int UNITS = P * L / 2;
#pragma unroll 4
        for (int u = threadIdx.x; u < UNITS; u += NT) {
            int j = u / (P / 2), p = (u % (P / 2)) * 2;
            cp_async16(sm + LY::idx(p, j), base + (long long)p * a.isI + (long long)j * a.isJ);
        }
    } else if constexpr (sizeof(C) == 8) {
        constexpr int UNITS = P * L;
#pragma unroll 4
        for (int u = threadIdx.x; u < UNITS; u += NT) {
            int p = u / L, j = u % L;
            cp_async8(sm + LY::idx(p, j), base + (long long)p * a.isI + (long long)j * a.isJ);
        }
    } else {
        constexpr int UNITS = P * L;
#pragma unroll 4
        for (int u = threadIdx.x; u < UNITS; u += NT) {
            int p, j;
            if constexpr (PFAST) { j = u / P; p = u % P; }
            else { p = u / L; j = u % L; }
            cp_async16(sm + LY::idx(p, j), base + (long long)p * a.isI + (long long)j * a.isJ);
        }
    }
}

template <typename T, int L, int P, int NT, bool PFAST, class LY>
__device__ __forceinline__ void store_tile(const cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
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
                    v0 = sm[LY::idx(p, j)]; v1 = sm[LY::idx(p + 1, j)];
                } else {
                    p = u / (L / 2); j = (u % (L / 2)) * 2;
                    v0 = sm[LY::idx(p, j)]; v1 = sm[LY::idx(p, j + 1)];
                }
                if (q0 + p < npencil) {
                    long long ad = tile_addr(q0, p, j, a.I, a.osO, a.osI, a.osJ, a.generic);
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
                    long long ad = tile_addr(q0, p, j, a.I, a.osO, a.osI, a.osJ, a.generic);
                    a.out[ad] = cscale(sm[LY::idx(p, j)], s);
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
template <typename T, int L, int P, int NT, int SIGN, int NS, int R, class LY>
__device__ __forceinline__ void stockham_stage(cx_t<T>* sm, const cx_t<T>* __restrict__ tw) {
    using C = cx_t<T>;
    constexpr int Q = L / R;
    constexpr int NB = P * Q;
    constexpr int PER = (NB + NT - 1) / NT;
    C v[PER][R];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int b = threadIdx.x + k * NT;
        if (NB % NT == 0 || b < NB) {
            int p, j;
            if constexpr (LY::PMAP) { p = b % P; j = b / P; }
            else { p = b / Q; j = b % Q; }
#pragma unroll
            for (int r = 0; r < R; ++r) v[k][r] = sm[LY::idx(p, j + r * Q)];
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
            int p, j;
            if constexpr (LY::PMAP) { p = b % P; j = b / P; }
            else { p = b / Q; j = b % Q; }
            int jm = j % NS;
            int d = (j / NS) * NS * R + jm;
#pragma unroll
            for (int r = 0; r < R; ++r) sm[LY::idx(p, d + r * NS)] = v[k][r];
        }
    }
    __syncthreads();
}

template <typename T, int L, int P, int NT, int SIGN, class LY, int NS, int R, int... Rest>
__device__ __forceinline__ void run_stages_impl(cx_t<T>* sm, const cx_t<T>* tw) {
    stockham_stage<T, L, P, NT, SIGN, NS, R, LY>(sm, tw);
    if constexpr (sizeof...(Rest) > 0) run_stages_impl<T, L, P, NT, SIGN, LY, NS * R, Rest...>(sm, tw);
}
template <typename T, int L, int P, int NT, int SIGN, class LY, int... Rs>
__device__ __forceinline__ void run_stages_list(cx_t<T>* sm, const cx_t<T>* tw, RList<Rs...>) {
    run_stages_impl<T, L, P, NT, SIGN, LY, 1, Rs...>(sm, tw);
}
// All stages of a length-L transform with kernel exp(SIGN 2 pi i n k / L).
template <typename T, int L, int P, int NT, int SIGN, class LY>
__device__ __forceinline__ void run_stages(cx_t<T>* sm, const cx_t<T>* tw) {
    run_stages_list<T, L, P, NT, SIGN, LY>(sm, tw, typename Radices<L>::type{});
}

// Four-step twiddle: element (pencil i, output index j) *= W_N^{i j}.
template <typename T, int L, int P, int NT, int SIGN, class LY>
__device__ __forceinline__ void apply_fourstep_twiddle(cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
    for (int e = threadIdx.x; e < P * L; e += NT) {
        int p, j;
        if constexpr (LY::PMAP) { p = e % P; j = e / P; }
        else { p = e / L; j = e % L; }
        long long q = q0 + p;
        long long i = q % a.I;
        long long m = (i * (long long)j) % a.n4;
        C w = __ldg(a.tw4 + m);
        if constexpr (SIGN > 0) w.y = -w.y;
        sm[LY::idx(p, j)] = cmul(sm[LY::idx(p, j)], w);
    }
    __syncthreads();
}

// Pass modes
enum PassMode : int {
    PASS_PLAIN = 0,      // transform, optional four-step twiddle, scaled store
    PASS_CH_NL = 1,      // inverse transform, c = Re(.)/N, g = c^3 - c, forward transform
};

// Body shared by both kernels: transform the tile in shared memory.
template <typename T, int L, int P, int NT, int SIGN, int MODE, class LY>
__device__ __forceinline__ void tile_body(cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
    if constexpr (MODE == PASS_PLAIN) {
        run_stages<T, L, P, NT, SIGN, LY>(sm, a.tw);
        if (a.tw4 != nullptr) apply_fourstep_twiddle<T, L, P, NT, SIGN, LY>(sm, a, q0);
    } else if constexpr (MODE == PASS_CH_NL) {
        // inverse transform along this axis completes c = IFFT(c_hat) (scaled by nl_scale)
        run_stages<T, L, P, NT, +1, LY>(sm, a.tw);
        T msum = 0;
        for (int e = threadIdx.x; e < P * L; e += NT) {
            int p, j;
            if constexpr (LY::PMAP) { p = e % P; j = e / P; }
            else { p = e / L; j = e % L; }
            C v = sm[LY::idx(p, j)];
            T c = v.x * a.nl_scale;
            msum += c;
            sm[LY::idx(p, j)] = mk<C>(c * c * c - c, (T)0);
        }
        if (a.mass != nullptr) {
            double ms = (double)msum;
            ms = warp_sum(ms);
            if ((threadIdx.x & 31) == 0) atomicAdd(a.mass + (q0 / a.mass_ppr) * a.mass_stride, ms);
        }
        __syncthreads();
        run_stages<T, L, P, NT, -1, LY>(sm, a.tw);
    }
}

// Simple kernel: one tile per CTA, synchronous loads; handles uneven tiles
// (generic addressing) and the transposing store of the four-step second pass.
template <typename T, int L, int P, int NT, int SIGN, int MODE, bool LOADP, bool STOREP>
__global__ void __launch_bounds__(NT) fft_pass_kernel(PassParams<T> a) {
    using C = cx_t<T>;
    using LY = LayoutA<L, P, true>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const long long q0 = (long long)blockIdx.x * P;
    load_tile<T, L, P, NT, LOADP, LY>(sm, a, q0);
    __syncthreads();
    tile_body<T, L, P, NT, SIGN, MODE, LY>(sm, a, q0);
    store_tile<T, L, P, NT, STOREP, LY>(sm, a, q0);
}

// Pipelined kernel: persistent CTAs walk the tiles; the next tile streams into
// the second shared buffer with cp.async while the current one is transformed.
// Requires I % P == 0 and in/out with the same orientation.
// Resident CTAs per SM the pipelined kernel is compiled for (register budget).
template <typename T, int L, int MODE> struct PipeOcc {
    static constexpr int value = (sizeof(T) == 4 && L <= 256 && MODE == PASS_PLAIN) ? 3 : 1;
};

template <typename T, int L, int P, int NT, int SIGN, int MODE, bool PFAST>
__global__ void __launch_bounds__(NT, PipeOcc<T, L, MODE>::value) fft_pass_pipe_kernel(PassParams<T> a) {
    using C = cx_t<T>;
    using LY = typename std::conditional<PFAST, LayoutB<L, P>, LayoutA<L, P, true>>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm0 = reinterpret_cast<C*>(smem_raw);
    C* sm1 = sm0 + LY::SIZE;
    const long long ntiles = (a.O * a.I) / P;
    long long t = blockIdx.x;
    if (t < ntiles) issue_tile<T, L, P, NT, PFAST, LY>(sm0, a, t * P);
    cp_async_commit();
    int buf = 0;
    for (; t < ntiles; t += gridDim.x) {
        const long long tn = t + gridDim.x;
        if (tn < ntiles) issue_tile<T, L, P, NT, PFAST, LY>(buf ? sm0 : sm1, a, tn * P);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        C* sm = buf ? sm1 : sm0;
        tile_body<T, L, P, NT, SIGN, MODE, LY>(sm, a, t * P);
        store_tile<T, L, P, NT, PFAST, LY>(sm, a, t * P);
        __syncthreads();
        buf ^= 1;
    }
    cp_async_wait<0>();
}

}  // namespace spdba
