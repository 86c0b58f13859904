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

#include "ch_math.cuh"
#include "common.cuh"

namespace spdba {

// Twiddle load: from a CTA's shared copy of the table (the compiler sees the
// shared address space after inlining) or through the read-only cache.
template <class C> __device__ __forceinline__ C tw_load(const C* p) { return __isShared(p) ? *p : __ldg(p); }

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

template <class RL> struct LastOf;
template <int R0> struct LastOf<RList<R0>> { static constexpr int value = R0; };
template <int R0, int R1, int... Rs> struct LastOf<RList<R0, R1, Rs...>> {
    static constexpr int value = LastOf<RList<R1, Rs...>>::value;
};
template <class RL> struct CountOf;
template <int... Rs> struct CountOf<RList<Rs...>> { static constexpr int value = sizeof...(Rs); };
template <int L> struct NSTAGES { static constexpr int value = CountOf<typename Radices<L>::type>::value; };
template <class RL> struct RArr;
template <int... Rs> struct RArr<RList<Rs...>> {
    static constexpr int n = sizeof...(Rs);
    static constexpr int v[sizeof...(Rs)] = {Rs...};
};
// i-th radix of a length and the product of the radices before it
template <int L> __host__ __device__ constexpr int radix_at(int i) { return RArr<typename Radices<L>::type>::v[i]; }
template <int L> __host__ __device__ constexpr int ns_at(int i) {
    int p = 1;
    for (int k = 0; k < i; ++k) p *= radix_at<L>(k);
    return p;
}
template <int L> struct Radices_last { static constexpr int value = LastOf<typename Radices<L>::type>::value; };

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

// Cahn-Hilliard update fused into the last forward pass (the pass along the
// field's first axis): per mode new = (c_hat - dt k^2 g_hat) / (1 + dt kappa k^4)
// on ACTIVE blocks, the transition blend on TRANSITION blocks, nothing on
// FROZEN blocks; tiles whose blocks are all frozen are skipped entirely.
template <typename T> struct CHFuse {
    cx_t<T>* c_hat;
    const T* k2ax[3];
    const T* taper[3];
    const uint8_t* states;
    const uint8_t* chi;
    T dt, dtkappa;
    int dense;
    DevStats* stats;   // one per run
    Geom g;
    // divisors of the per-tile geometry (pass-axis block edge, x block edge,
    // outer block edge (3-D), row length (3-D))
    FastDiv fd_bp, fd_b2, fd_b1, fd_n2;
};

// Half-spectrum geometry of a 3-D field N0 x N1 x N2 (N2 even): the half array
// holds x frequencies 0 .. N2/2 in rows of NHP >= N2/2 + 1 entries (the rest 0).
struct HalfGeo {
    int N0 = 1, N1 = 1, N2 = 2, NHP = 2;
    // the half array is the stored spectrum itself (half-spectrum storage):
    // the x pass keeps only the real parts of the kx = 0 and kx = N2/2 entries,
    // as a complex-to-real transform does (their planes need not be
    // conjugate-symmetric within themselves)
    int r2c = 0;
    FastDiv fd_N2, fd_NHP, fd_M;   // fd_M: division by N2 / 2
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
    CHFuse<T> fu;                         // PASS_CH_UPDATE only
    FastDiv fd_I;                         // division by I (pipelined kernel, O * I < 2^31)
    HalfGeo hg;                           // half-spectrum passes only
    // paired z forward with block states: its live tiles (any order) and their count
    const int* live_tiles = nullptr;
    const int* live_count = nullptr;
    // plain passes whose tiles are P consecutive columns i of the pencil grid: a
    // tile is skipped when none of its columns is marked (the outputs of
    // unmarked columns are never read), or null to transform every tile
    const uint8_t* col_live = nullptr;
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
    const long long o = a.fd_I.div((uint32_t)q0), i0 = q0 - o * a.I;
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

// Asynchronous load of a z-pencil tile of a 3-D field from its half array
// (PASS_MIRROR / PASS_UPD_HALF): pencil (ky, kx) of the full field is the half
// array's pencil (ky, kx) for kx <= N2/2 and, for kx > N2/2, the conjugate
// mirror ((-ky) mod N1, N2 - kx) (the transform of a real field along y and x
// satisfies D(z, ky, kx) = conj(D(z, -ky, -kx))); the caller applies the
// conjugation and the index reversal to the transform's outputs.
template <typename T, int L, int P, int NT, class LY>
__device__ __forceinline__ void issue_tile_half(cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
    const HalfGeo& h = a.hg;
    const int M = h.N2 >> 1;
    static_assert(NT % P == 0, "each thread keeps one pencil");
    const int p = (int)(threadIdx.x % P);
    const int q = (int)q0 + p;                       // full pencil index ky * N2 + kx (one field)
    const int ky = (int)h.fd_N2.div((uint32_t)q), kx = q - ky * h.N2;
    const bool mir = kx > M;
    const int sy = mir ? (ky == 0 ? 0 : h.N1 - ky) : ky;
    const int sx = mir ? h.N2 - kx : kx;
    const C* src = a.in + ((long long)sy * h.NHP + sx);
    const long long zs = (long long)h.N1 * h.NHP;   // z stride of the half array
    // direct pencil pairs (p, p + 1), p even, are one 16-byte copy by pencil p
    // (kx and NHP even keep it aligned; P even keeps kx's parity that of p)
    const bool pair = !mir && (p & 1) == 0 && kx + 1 <= M;
    const bool covered = !mir && (p & 1) == 1;        // kx odd <= M: copied with pencil p - 1
    if (pair) {
#pragma unroll 4
        for (int j = (int)(threadIdx.x / P); j < L; j += NT / P) cp_async16(sm + LY::idx(p, j), src + j * zs);
    } else if (!covered) {
#pragma unroll 4
        for (int j = (int)(threadIdx.x / P); j < L; j += NT / P) cp_async8(sm + LY::idx(p, j), src + j * zs);
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
                if constexpr (PFAST && LY::PMAP) {
                    // layout B keeps (p, p+1) adjacent and 16-byte aligned
                    j = u / (P / 2); p = (u % (P / 2)) * 2;
                    float4 t = *reinterpret_cast<const float4*>(sm + LY::idx(p, j));
                    v0 = make_float2(t.x, t.y); v1 = make_float2(t.z, t.w);
                } else if constexpr (PFAST) {
                    // pencils are the unit stride: (p, j) and (p + 1, j) are adjacent in memory
                    j = u / (P / 2); p = (u % (P / 2)) * 2;
                    v0 = sm[LY::idx(p, j)]; v1 = sm[LY::idx(p + 1, j)];
                } else {
                    // elements are the unit stride: (p, j) and (p, j + 1), j even
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
// Reader of a stage's input element m of pencil p: the tile itself by default.
template <typename T, class LY> struct SmemIn {
    const cx_t<T>* sm;
    __device__ __forceinline__ cx_t<T> operator()(int p, int m) const { return sm[LY::idx(p, m)]; }
};

template <typename T, int L, int P, int NT, int SIGN, int NS, int R, class LY, class IN>
__device__ __forceinline__ void stockham_stage_in(cx_t<T>* sm, const cx_t<T>* __restrict__ tw, const IN& in) {
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
            for (int r = 0; r < R; ++r) v[k][r] = in(p, j + r * Q);
            if constexpr (NS > 1) {
                int jm = j % NS;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C w = tw_load(tw + r * jm * (L / (NS * R)));
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

template <typename T, int L, int P, int NT, int SIGN, int NS, int R, class LY>
__device__ __forceinline__ void stockham_stage(cx_t<T>* sm, const cx_t<T>* __restrict__ tw) {
    stockham_stage_in<T, L, P, NT, SIGN, NS, R, LY>(sm, tw, SmemIn<T, LY>{sm});
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

// Last stage with its outputs handed to `out` instead of written back to
// shared memory.  For the last stage NS * R == L, so butterfly j of pencil p
// produces outputs j + r NS, r = 0..R-1.  out.begin(k, p, j) runs before the
// stage reads its inputs (so that loads the outputs need are in flight during
// the butterflies); out.emit(k, p, j, v) receives the R outputs.  An output
// that writes shared memory sets OUT::SYNC (all reads finish first).
template <typename T, int L, int P, int NT, int SIGN, int NS, int R, class LY, class OUT>
__device__ __forceinline__ void stockham_stage_out(cx_t<T>* sm, const cx_t<T>* __restrict__ tw, OUT& out) {
    using C = cx_t<T>;
    static_assert(NS * R == L, "direct output is for the last stage");
    constexpr int Q = L / R;
    constexpr int NB = P * Q;
    constexpr int PER = (NB + NT - 1) / NT;
    out.pre();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int b = threadIdx.x + k * NT;
        if (NB % NT == 0 || b < NB) {
            int p, j;
            if constexpr (LY::PMAP) { p = b % P; j = b / P; }
            else { p = b / Q; j = b % Q; }
            out.begin(k, p, j);
        }
    }
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
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C w = tw_load(tw + r * j);
                    if constexpr (SIGN > 0) w.y = -w.y;
                    v[k][r] = cmul(v[k][r], w);
                }
            }
            Dft<R, SIGN, C>::run(v[k]);
        }
    }
    if constexpr (OUT::SYNC) __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int b = threadIdx.x + k * NT;
        if (NB % NT == 0 || b < NB) {
            int p, j;
            if constexpr (LY::PMAP) { p = b % P; j = b / P; }
            else { p = b / Q; j = b % Q; }
            out.emit(k, p, j, v[k]);
        }
    }
}

template <typename T, int L, int P, int NT, int SIGN, class LY, class OUT, int NS, int R, int... Rest>
__device__ __forceinline__ void run_stages_out_impl(cx_t<T>* sm, const cx_t<T>* tw, OUT& out) {
    if constexpr (sizeof...(Rest) == 0) {
        stockham_stage_out<T, L, P, NT, SIGN, NS, R, LY, OUT>(sm, tw, out);
    } else {
        stockham_stage<T, L, P, NT, SIGN, NS, R, LY>(sm, tw);
        run_stages_out_impl<T, L, P, NT, SIGN, LY, OUT, NS * R, Rest...>(sm, tw, out);
    }
}
template <typename T, int L, int P, int NT, int SIGN, class LY, class OUT, int... Rs>
__device__ __forceinline__ void run_stages_out_list(cx_t<T>* sm, const cx_t<T>* tw, OUT& out, RList<Rs...>) {
    run_stages_out_impl<T, L, P, NT, SIGN, LY, OUT, 1, Rs...>(sm, tw, out);
}
// All stages of a length-L transform, the last one emitting through `out`.
template <typename T, int L, int P, int NT, int SIGN, class LY, class OUT>
__device__ __forceinline__ void run_stages_out(cx_t<T>* sm, const cx_t<T>* tw, OUT& out) {
    run_stages_out_list<T, L, P, NT, SIGN, LY, OUT>(sm, tw, out, typename Radices<L>::type{});
}

// Last-stage outputs passed through an elementwise step and written back to
// shared memory in natural order.
template <typename T, int L, class LY, class MID> struct MidOut {
    using C = cx_t<T>;
    static constexpr bool SYNC = true;
    C* sm;
    MID& mid;
    __device__ __forceinline__ void pre() {}
    __device__ __forceinline__ void begin(int, int, int) {}
    template <int R> __device__ __forceinline__ void emit(int, int p, int j, C (&v)[R]) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = j + r * (L / R);
            sm[LY::idx(p, m)] = mid(p, m, v[r]);
        }
    }
};

// c = Re(x) / N, g = c^3 - c (the CH nonlinearity), with the sum of c kept.
template <typename T> struct ChNlMid {
    T scale, msum;
    __device__ __forceinline__ cx_t<T> operator()(int, int, cx_t<T> x) {
        const T c = mul_rn(x.x, scale);
        msum += c;
        return mk<cx_t<T>>(fma_rn(mul_rn(c, c), c, -c), (T)0);
    }
};

// Stages I .. E-1 of a length-L transform (in shared memory).
template <typename T, int L, int P, int NT, int SIGN, class LY, int I, int E>
__device__ __forceinline__ void run_stage_range(cx_t<T>* sm, const cx_t<T>* tw) {
    if constexpr (I < E) {
        stockham_stage<T, L, P, NT, SIGN, ns_at<L>(I), radix_at<L>(I), LY>(sm, tw);
        run_stage_range<T, L, P, NT, SIGN, LY, I + 1, E>(sm, tw);
    }
}

// Plain store of a z-transform from the half array (PASS_MIRROR): outputs of
// a mirrored pencil go, conjugated, to frequency -m.
template <typename T, int L, int P> struct MirrorPlainOut {
    using C = cx_t<T>;
    static constexpr bool SYNC = false;
    C* po;        // this thread's pencil, output element 0
    int osJ;
    bool mir;
    __device__ __forceinline__ MirrorPlainOut(const PassParams<T>& a, long long q0) {
        const int p = (int)(threadIdx.x % P);
        const long long o = a.fd_I.div((uint32_t)q0);
        po = a.out + (o * a.osO + (q0 - o * a.I + p) * a.osI);
        osJ = (int)a.osJ;
        const int q = (int)(q0 - o * a.I) + p;
        const int ky = (int)a.hg.fd_N2.div((uint32_t)q);
        mir = q - ky * a.hg.N2 > (a.hg.N2 >> 1);
    }
    __device__ __forceinline__ void pre() {}
    __device__ __forceinline__ void begin(int, int, int) {}
    template <int R> __device__ __forceinline__ void emit(int, int, int j, C (&v)[R]) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = j + r * (L / R);
            C x = v[r];
            int kz = m;
            if (mir) {
                x.y = -x.y;
                kz = m == 0 ? 0 : L - m;
            }
            po[kz * osJ] = x;
        }
    }
};

// Outputs of a first stage (NS = 1): butterfly j writes j R + r.
template <typename T, int L, int R, class LY> struct FirstStageOut {
    using C = cx_t<T>;
    static constexpr bool SYNC = true;
    C* sm;
    __device__ __forceinline__ void pre() {}
    __device__ __forceinline__ void begin(int, int, int) {}
    __device__ __forceinline__ void emit(int, int p, int j, C (&v)[R]) {
#pragma unroll
        for (int r = 0; r < R; ++r) sm[LY::idx(p, j * R + r)] = v[r];
    }
};

// The last stage of one transform (sign SA, span NS = L / R) and the first
// stage of the next (sign SB) of the same pencil, when both have radix R: the
// first's butterfly j yields exactly the elements j + r L/R (natural order)
// that the second's butterfly j reads, so both butterflies and an elementwise
// step between them (mid(p, m, x) for element m) run in registers.  The
// second stage's outputs go to `out` (j R + r for a stage that others follow).
template <typename T, int L, int P, int NT, int SA, int SB, int NS, int R, class LY, class MID, class OUT>
__device__ __forceinline__ void fused_mid_stage(cx_t<T>* sm, const cx_t<T>* __restrict__ tw, MID& mid, OUT& out) {
    using C = cx_t<T>;
    static_assert(NS * R == L, "the first of the two stages closes its transform");
    constexpr int Q = L / R;
    constexpr int NB = P * Q;
    constexpr int PER = (NB + NT - 1) / NT;
    out.pre();
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
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C w = tw_load(tw + r * j);
                    if constexpr (SA > 0) w.y = -w.y;
                    v[k][r] = cmul(v[k][r], w);
                }
            }
            Dft<R, SA, C>::run(v[k]);
#pragma unroll
            for (int r = 0; r < R; ++r) v[k][r] = mid(p, j + r * Q, v[k][r]);
            Dft<R, SB, C>::run(v[k]);
        }
    }
    if constexpr (OUT::SYNC) __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int b = threadIdx.x + k * NT;
        if (NB % NT == 0 || b < NB) {
            int p, j;
            if constexpr (LY::PMAP) { p = b % P; j = b / P; }
            else { p = b / Q; j = b % Q; }
            out.emit(k, p, j, v[k]);
        }
    }
}

// Two transforms of the tile with an elementwise step between them: SA then
// SB, the second's last stage emitting through `out`.  When the first's last
// radix equals the second's first, the two meeting stages run fused in
// registers (fused_mid_stage); otherwise `mid` rides in the first's last stage.
// One transform whose first stage reads through `in` and whose last stage
// emits through `out` (at least two stages).
template <typename T, int L, int P, int NT, int SIGN, class LY, class IN, class OUT>
__device__ __forceinline__ void run_stages_in_out(cx_t<T>* sm, const cx_t<T>* tw, const IN& in, OUT& out) {
    constexpr int NST = NSTAGES<L>::value;
    static_assert(NST >= 2, "a separate first and last stage");
    stockham_stage_in<T, L, P, NT, SIGN, 1, radix_at<L>(0), LY>(sm, tw, in);
    run_stage_range<T, L, P, NT, SIGN, LY, 1, NST - 1>(sm, tw);
    stockham_stage_out<T, L, P, NT, SIGN, ns_at<L>(NST - 1), radix_at<L>(NST - 1), LY>(sm, tw, out);
}

template <typename T, int L, int P, int NT, int SA, int SB, class LY, class MID, class OUT>
__device__ __forceinline__ void transform_pair(cx_t<T>* sm, const cx_t<T>* tw, MID& mid, OUT& out);

// transform_pair whose first stage reads its inputs through `in` (an
// elementwise preparation folded into the first stage's loads); at least
// three stages in all.
template <typename T, int L, int P, int NT, int SA, int SB, class LY, class IN, class MID, class OUT>
__device__ __forceinline__ void transform_pair_in(cx_t<T>* sm, const cx_t<T>* tw, const IN& in, MID& mid, OUT& out) {
    constexpr int NST = NSTAGES<L>::value;
    constexpr int R0 = radix_at<L>(0), RL = radix_at<L>(NST - 1);
    static_assert(NST >= 2, "the first stage must not be the meeting stage");
    stockham_stage_in<T, L, P, NT, SA, 1, R0, LY>(sm, tw, in);
    if constexpr (R0 == RL) {
        run_stage_range<T, L, P, NT, SA, LY, 1, NST - 1>(sm, tw);
        FirstStageOut<T, L, R0, LY> fo{sm};
        fused_mid_stage<T, L, P, NT, SA, SB, L / R0, R0, LY>(sm, tw, mid, fo);
        __syncthreads();
        run_stage_range<T, L, P, NT, SB, LY, 1, NST - 1>(sm, tw);
        stockham_stage_out<T, L, P, NT, SB, ns_at<L>(NST - 1), RL, LY>(sm, tw, out);
    } else {
        run_stage_range<T, L, P, NT, SA, LY, 1, NST - 1>(sm, tw);
        MidOut<T, L, LY, MID> mo{sm, mid};
        stockham_stage_out<T, L, P, NT, SA, ns_at<L>(NST - 1), RL, LY>(sm, tw, mo);
        __syncthreads();
        run_stages_out<T, L, P, NT, SB, LY>(sm, tw, out);
    }
}

template <typename T, int L, int P, int NT, int SA, int SB, class LY, class MID, class OUT>
__device__ __forceinline__ void transform_pair(cx_t<T>* sm, const cx_t<T>* tw, MID& mid, OUT& out) {
    constexpr int NST = NSTAGES<L>::value;
    constexpr int R0 = radix_at<L>(0), RL = radix_at<L>(NST - 1);
    if constexpr (R0 == RL) {
        run_stage_range<T, L, P, NT, SA, LY, 0, NST - 1>(sm, tw);
        if constexpr (NST == 1) {
            fused_mid_stage<T, L, P, NT, SA, SB, 1, R0, LY>(sm, tw, mid, out);
        } else {
            FirstStageOut<T, L, R0, LY> fo{sm};
            fused_mid_stage<T, L, P, NT, SA, SB, L / R0, R0, LY>(sm, tw, mid, fo);
            __syncthreads();
            run_stage_range<T, L, P, NT, SB, LY, 1, NST - 1>(sm, tw);
            stockham_stage_out<T, L, P, NT, SB, ns_at<L>(NST - 1), RL, LY>(sm, tw, out);
        }
    } else {
        MidOut<T, L, LY, MID> mo{sm, mid};
        run_stages_out<T, L, P, NT, SA, LY>(sm, tw, mo);
        __syncthreads();
        run_stages_out<T, L, P, NT, SB, LY>(sm, tw, out);
    }
}

// Hand a transformed tile in shared memory to `out` as if it came from a
// last stage of radix R2 (outputs j + r L/R2 of butterfly j): the same output
// code at lower register pressure than the fused last stage.
template <typename T, int L, int P, int NT, int R2, class LY, class OUT>
__device__ __forceinline__ void drain_tile(const cx_t<T>* sm, OUT& out) {
    using C = cx_t<T>;
    constexpr int Q = L / R2;
    constexpr int NB = P * Q;
    constexpr int PER = (NB + NT - 1) / NT;
    out.pre();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        int b = threadIdx.x + k * NT;
        if (NB % NT == 0 || b < NB) {
            int p, j;
            if constexpr (LY::PMAP) { p = b % P; j = b / P; }
            else { p = b / Q; j = b % Q; }
            out.begin(k, p, j);
            C v[R2];
#pragma unroll
            for (int r = 0; r < R2; ++r) v[r] = sm[LY::idx(p, j + r * Q)];
            out.emit(k, p, j, v);
        }
    }
}

// Plain pass output: scaled store of every output straight from registers.
// Consecutive threads hold consecutive unit-stride outputs (pencils for
// row-major tiles, elements for pencil-major tiles), so warp stores coalesce.
template <typename T, int L> struct PlainOut {
    using C = cx_t<T>;
    static constexpr bool SYNC = false;
    C* base;      // output (p = 0, j = 0) of the tile
    int osI, osJ;  // strides within a tile fit 32 bits (checked at plan time)
    T scale;
    __device__ __forceinline__ PlainOut(const PassParams<T>& a, long long q0) {
        const long long o = a.fd_I.div((uint32_t)q0);
        base = a.out + (o * a.osO + (q0 - o * a.I) * a.osI);
        osI = (int)a.osI;
        osJ = (int)a.osJ;
        scale = a.scale;
    }
    __device__ __forceinline__ void pre() {}
    __device__ __forceinline__ void begin(int, int, int) {}
    template <int R> __device__ __forceinline__ void emit(int, int p, int j, C (&v)[R]) {
        C* po = base + (p * osI + j * osJ);
#pragma unroll
        for (int r = 0; r < R; ++r) po[r * (L / R) * osJ] = cscale(v[r], scale);
    }
};


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
    PASS_CH_UPDATE = 2,  // forward transform, then the CH update of c_hat (no store of the transform)
    // Hermitian half-spectrum passes of a 3-D field (x frequencies 0 .. N2/2 kept)
    PASS_HERM_INV = 3,   // inverse z-transform of (c_hat(k) + conj(c_hat(-k))) / 2 into the half array
    PASS_NL_HALF = 4,    // x rows: half spectrum -> real -> g = c^3 - c -> half spectrum
    PASS_MIRROR = 5,     // forward z-transform of the half array, stored for every x frequency
    PASS_UPD_HALF = 6,   // forward z-transform of the half array, then the CH update of c_hat
    // PASS_MIRROR with one transform per half pencil for x frequencies kx and N2 - kx
    PASS_PAIR_MIRROR = 7,
};
constexpr bool is_update_mode(int m) { return m == PASS_CH_UPDATE || m == PASS_UPD_HALF; }
constexpr bool reads_half(int m) { return m == PASS_MIRROR || m == PASS_UPD_HALF; }

// Padded (axis 0, 1, 2) coordinates of element (p, j) of the tile at pencil q0
// of the pass along the field's first axis: 3-D fields (z = j, (y, x) from the
// pencil), 2-D groups ((run, y = j, x) with the run as the pencil's outer index).
template <typename T>
__device__ __forceinline__ void fuse_coords(const PassParams<T>& a, long long q0, int p, int j, long long& c0,
                                            long long& c1, long long& c2) {
    const Geom& g = a.fu.g;
    long long o = q0 / a.I, i = q0 - o * a.I + p;
    if (g.ndim == 3) { c0 = j; c1 = i / g.n[2]; c2 = i - c1 * g.n[2]; }
    else { c0 = o; c1 = j; c2 = i; }
}
__device__ __forceinline__ long long block_id(const Geom& g, long long c0, long long c1, long long c2) {
    return ((c0 / g.b[0]) * g.nb[1] + c1 / g.b[1]) * g.nb[2] + c2 / g.b[2];
}

// Per-tile constants of the fused update (32-bit; every thread derives the
// same values).  The tile holds pencils x0 .. x0 + P - 1 of one row cy of the
// outer axis (3-D: y; 2-D group: the run), unless `rows` (the tile spans
// several rows of a small 3-D grid).
struct UpdTile {
    int o, i0, cy, x0, bx0, nbx, l_out;
    long long boff;   // block id offset of (block row 0, x-block bx0)
    int bstride;      // block id step per block row of the pass axis
    bool rows;
};
template <typename T, int P>
__device__ __forceinline__ UpdTile upd_tile(const PassParams<T>& a, int q0) {
    const CHFuse<T>& f = a.fu;
    const Geom& g = f.g;
    UpdTile u;
    u.o = (int)a.fd_I.div((uint32_t)q0);
    u.i0 = q0 - u.o * (int)a.I;
    const bool d3 = g.ndim == 3;
    if (d3) {
        u.cy = (int)f.fd_n2.div((uint32_t)u.i0);
        u.x0 = u.i0 - u.cy * (int)g.n[2];
    } else {
        u.cy = u.o;
        u.x0 = u.i0;
    }
    u.rows = d3 && u.x0 + P > (int)g.n[2];
    u.bx0 = (int)f.fd_b2.div((uint32_t)u.x0);
    u.nbx = (int)f.fd_b2.div((uint32_t)(u.x0 + P - 1)) - u.bx0 + 1;
    if (d3) {
        const int by = (int)f.fd_b1.div((uint32_t)u.cy);
        u.l_out = u.cy - by * g.b[1];
        u.boff = (long long)by * g.nb[2] + u.bx0;
        u.bstride = (int)(g.nb[1] * g.nb[2]);
    } else {
        u.l_out = 0;
        u.boff = (long long)u.cy * g.nb[1] * g.nb[2] + u.bx0;
        u.bstride = (int)g.nb[2];
    }
    return u;
}

// A tile is live when any block its modes belong to is not FROZEN.  Every warp
// evaluates this independently (no block-wide synchronisation needed).
template <typename T, int P, int MODE>
__device__ __forceinline__ bool tile_live(const PassParams<T>& a, long long q0) {
    if constexpr (MODE == PASS_PLAIN) {
        if (a.col_live == nullptr) return true;
        const long long i0 = q0 - (long long)a.fd_I.div((uint32_t)q0) * a.I;
        bool live = false;
#pragma unroll
        for (int p = 0; p < P; ++p) live |= a.col_live[i0 + p] != 0;
        return live;
    } else if constexpr (!is_update_mode(MODE)) {
        return true;
    } else {
        if (a.fu.dense) return true;
        const UpdTile u = upd_tile<T, P>(a, (int)q0);
        if (u.rows) return true;
        const int npass = (int)(a.fu.g.ndim == 3 ? a.fu.g.nb[0] : a.fu.g.nb[1]);
        bool live = false;
        for (int bp = threadIdx.x & 31; bp < npass && !live; bp += 32)
            for (int bx = 0; bx < u.nbx; ++bx) live |= a.fu.states[u.boff + (long long)bp * u.bstride + bx] != 0;
        return __any_sync(0xffffffffu, live);
    }
}

// Per-run share of non-frozen blocks for this step (CTA 0, once per launch);
// dense: every block is updated this step.
template <typename T, int NT> __device__ __forceinline__ void ch_update_stats(const CHFuse<T>& f, int dense) {
    const Geom& g = f.g;
    if (blockIdx.x != 0 || !f.stats) return;
    const double inv = 1.0 / (double)g.live_bpr();
    const long long bm = g.block_modes();
    for (long long r = threadIdx.x; r < g.runs(); r += NT) {
        double nf = dense ? (double)g.live_bpr() : (double)(f.stats[r].n_active + f.stats[r].n_transition);
        f.stats[r].ratio_sum += nf * inv;
        if (!dense) {
            f.stats[r].list_modes += nf * (double)bm;
            f.stats[r].ctl_nf += f.stats[r].n_active + f.stats[r].n_transition;   // control interval
            f.stats[r].ctl_steps += 1;
        }
    }
}

// Update of a tile that spans several rows of a small grid (P > row length):
// g_hat of the tile is in shared memory; per-mode coordinates and states.
template <typename T, int L, int P, int NT, class LY>
__device__ __forceinline__ void ch_update_tile_rows(const cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
    const CHFuse<T>& f = a.fu;
    const Geom& g = f.g;
    constexpr int UN = P * L;
    for (int u = threadIdx.x; u < UN; u += NT) {
        const int j = u / P, p = u % P;
        long long c0, c1, c2;
        fuse_coords<T>(a, q0, p, j, c0, c1, c2);
        const long long id = block_id(g, c0, c1, c2);
        const int st = f.dense ? SPDBA_ACTIVE : f.states[id];
        if (st == SPDBA_FROZEN) continue;
        const long long ad = tile_addr(q0, p, j, a.I, a.osO, a.osI, a.osJ, 0);
        C cv = f.c_hat[ad];
        C nv = ch_new(cv, sm[LY::idx(p, j)], (f.k2ax[0][c0] + f.k2ax[1][c1]) + f.k2ax[2][c2], f.dt, f.dtkappa);
        if (st == SPDBA_TRANSITION)
            nv = ch_blend<T>(cv, nv, f.taper, g, f.chi[id], (int)(c0 % g.b[0]), (int)(c1 % g.b[1]),
                             (int)(c2 % g.b[2]));
        f.c_hat[ad] = nv;
    }
}

// Per-tile table of the update: entry (bp, bx) = state | chi << 2 of the block
// in block row bp of the pass axis and x-block bx0 + bx (bytes).
constexpr int kUpdTable = 4096;
// Capacity of each of the two state tables of a paired z tile (direct and mirror columns).
constexpr int kPairTable = 1024;
__host__ __device__ __forceinline__ int upd_table_cols(int P, int bx) { return (P + bx - 2) / bx + 1; }
// The update pass stages c_hat in a third tile buffer for row-major tiles of
// L <= 256 whose last stage emits directly (not the radix-3 tail of 192).
template <typename T, int L> __host__ __device__ constexpr bool upd_stages_chat() {
    return L <= 256 && Radices_last<L>::value != 3;
}

// Update emitted from the forward transform's last stage (tile within one row):
// each output is updated and stored from registers.  With CS the tile's
// non-frozen c_hat rows were staged in shared memory (layout LY) by cp.async
// during the transform; otherwise a butterfly's c_hat loads are issued before
// its arithmetic.
template <typename T, int L, int P, int NT, int R, bool CS, class LY, bool HALF = false> struct UpdOut {
    using C = cx_t<T>;
    static constexpr bool SYNC = false;
    static constexpr int NS = L / R;
    static constexpr int PER = (P * NS + NT - 1) / NT;
    static_assert(NT % P == 0, "each thread keeps one pencil");
    const PassParams<T>& a;
    const uint8_t* tab;   // shared per-tile table
    const T* kp;          // shared |k|^2 table of the pass axis
    const C* cs;          // staged c_hat tile (CS)
    int nbx, bxs, lx, l_out;
    bool mir;             // HALF: this pencil's transform is the conjugate mirror's
    C* cb;                // c_hat of (p, j = 0)
    int osJ;
    T kx, kc;
    C cv[CS ? 1 : PER][CS ? 1 : R];
    __device__ __forceinline__ UpdOut(const PassParams<T>& a_, const UpdTile& u, const uint8_t* tab_, const T* kp_,
                                      const C* cs_)
        : a(a_), tab(tab_), kp(kp_), cs(cs_) {
        const CHFuse<T>& f = a.fu;
        const bool d3 = f.g.ndim == 3;
        nbx = u.nbx;
        const int x = u.x0 + (int)(threadIdx.x % P);
        const int bx = (int)f.fd_b2.div((uint32_t)x);
        bxs = bx - u.bx0;
        lx = x - bx * f.g.b[2];
        kx = f.k2ax[2][x];
        kc = d3 ? f.k2ax[1][u.cy] : f.k2ax[0][u.cy];
        l_out = u.l_out;
        cb = f.c_hat + ((long long)u.o * a.osO + (long long)(u.i0 + (int)(threadIdx.x % P)) * a.osI);
        osJ = (int)a.osJ;
        mir = HALF && x > (a.hg.N2 >> 1);
    }
    // output index of transform output m: the mirror's output m is frequency -m
    __device__ __forceinline__ int kz_of(int m) const {
        if constexpr (HALF) return (mir && m != 0) ? L - m : m;
        else return m;
    }
    // before the last stage: the staged c_hat must have landed and be visible
    __device__ __forceinline__ void pre() {
        if constexpr (CS) {
            cp_async_wait<0>();
            __syncthreads();
        }
    }
    __device__ __forceinline__ unsigned entry(int jj) const { return tab[(int)a.fu.fd_bp.div((uint32_t)jj) * nbx + bxs]; }
    __device__ __forceinline__ void begin(int k, int, int j) {
        if constexpr (!CS) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int jj = kz_of(j + r * NS);
                if ((entry(jj) & 3u) != SPDBA_FROZEN) cv[k][r] = cb[jj * osJ];
            }
        }
    }
    __device__ __forceinline__ void emit(int k, int p, int j, C (&v)[R]) {
        const CHFuse<T>& f = a.fu;
        const bool d3 = f.g.ndim == 3;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int jj = kz_of(j + r * NS);
            const int bp = (int)f.fd_bp.div((uint32_t)jj);
            const unsigned e = tab[bp * nbx + bxs];
            const int st = (int)(e & 3u);
            if (st == SPDBA_FROZEN) continue;
            C c;
            if constexpr (CS) c = cs[LY::idx(p, jj)];
            else c = cv[k][r];
            C gv = v[r];
            if constexpr (HALF) {
                if (mir) gv.y = -gv.y;
            }
            // same association as the staged kernels: (k_outer + k_pass) then + k_x
            const T k01 = d3 ? kp[jj] + kc : kc + kp[jj];
            C nv = ch_new(c, gv, k01 + kx, f.dt, f.dtkappa);
            if (st == SPDBA_TRANSITION) {
                const int lj = jj - bp * (d3 ? f.g.b[0] : f.g.b[1]);
                nv = d3 ? ch_blend<T>(c, nv, f.taper, f.g, e >> 2, lj, l_out, lx)
                        : ch_blend<T>(c, nv, f.taper, f.g, e >> 2, 0, lj, lx);
            }
            cb[jj * osJ] = nv;
        }
    }
};

// Fill the per-tile table (visible after the next barrier).
template <typename T, int L, int P, int NT>
__device__ __forceinline__ void ch_update_table(uint8_t* tab, const PassParams<T>& a, const UpdTile& u) {
    const CHFuse<T>& f = a.fu;
    const int npass = (int)(f.g.ndim == 3 ? f.g.nb[0] : f.g.nb[1]);
    for (int k = threadIdx.x; k < npass * u.nbx; k += NT) {
        const int bp = k / u.nbx, bx = k - bp * u.nbx;
        const long long id = u.boff + (long long)bp * u.bstride + bx;
        tab[k] = f.dense ? (uint8_t)SPDBA_ACTIVE : (uint8_t)(f.states[id] | (f.chi[id] << 2));
    }
}

// Stage the tile's non-frozen c_hat rows into shared memory (row-major tile,
// one cp.async group).  The table must be visible to every thread.
template <typename T, int L, int P, int NT, class LY>
__device__ __forceinline__ void issue_chat(cx_t<T>* cs, const PassParams<T>& a, const UpdTile& u, const uint8_t* tab) {
    using C = cx_t<T>;
    const CHFuse<T>& f = a.fu;
    const C* base = f.c_hat + ((long long)u.o * a.osO + (long long)u.i0 * a.osI);
    const int osJ = (int)a.osJ;
    if constexpr (sizeof(C) == 8) {
        // pencil pairs (p, p + 1): 16 bytes; copied when either block is non-frozen
        static_assert(NT % (P / 2) == 0, "each thread keeps one pencil pair");
        constexpr int UNITS = P * L / 2;
        const int p = (int)(threadIdx.x % (P / 2)) * 2;
        const int b0 = (int)f.fd_b2.div((uint32_t)(u.x0 + p)) - u.bx0;
        const int b1 = (int)f.fd_b2.div((uint32_t)(u.x0 + p + 1)) - u.bx0;
#pragma unroll 4
        for (int w = threadIdx.x; w < UNITS; w += NT) {
            const int j = w / (P / 2);
            const int row = (int)f.fd_bp.div((uint32_t)j) * u.nbx;
            if ((tab[row + b0] & 3) != SPDBA_FROZEN || (tab[row + b1] & 3) != SPDBA_FROZEN)
                cp_async16(cs + LY::idx(p, j), base + (p + j * osJ));
        }
    } else {
        static_assert(NT % P == 0, "each thread keeps one pencil");
        constexpr int UNITS = P * L;
        const int p = (int)(threadIdx.x % P);
        const int b0 = (int)f.fd_b2.div((uint32_t)(u.x0 + p)) - u.bx0;
#pragma unroll 4
        for (int w = threadIdx.x; w < UNITS; w += NT) {
            const int j = w / P;
            if ((tab[(int)f.fd_bp.div((uint32_t)j) * u.nbx + b0] & 3) != SPDBA_FROZEN)
                cp_async16(cs + LY::idx(p, j), base + (p + j * osJ));
        }
    }
    cp_async_commit();
}

// Body shared by both kernels: transform the tile in shared memory.
template <typename T, int L, int P, int NT, int SIGN, int MODE, class LY>
__device__ __forceinline__ void tile_body(cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
    if constexpr (MODE == PASS_PLAIN) {
        run_stages<T, L, P, NT, SIGN, LY>(sm, a.tw);
        if (a.tw4 != nullptr) apply_fourstep_twiddle<T, L, P, NT, SIGN, LY>(sm, a, q0);
    } else if constexpr (MODE == PASS_CH_UPDATE) {
        run_stages<T, L, P, NT, -1, LY>(sm, a.tw);
    } else if constexpr (MODE == PASS_CH_NL) {
      {
        // one pencil at a time: inverse transform, c = Re(.)/N, g = c^3 - c, forward
        run_stages<T, L, P, NT, +1, LY>(sm, a.tw);
        T msum = 0;
        for (int e = threadIdx.x; e < P * L; e += NT) {
            int p, j;
            if constexpr (LY::PMAP) { p = e % P; j = e / P; }
            else { p = e / L; j = e % L; }
            C v = sm[LY::idx(p, j)];
            T c = mul_rn(v.x, a.nl_scale);
            msum += c;
            sm[LY::idx(p, j)] = mk<C>(fma_rn(mul_rn(c, c), c, -c), (T)0);
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
// (chosen from the compiler's register counts: the largest count of CTAs at
// which the kernel does not spill)
template <typename T, int L, int MODE, bool PFAST> struct PipeOcc {
    static constexpr bool PLAINISH = MODE == PASS_PLAIN || MODE == PASS_MIRROR;
    static constexpr int value = sizeof(T) != 4 || L > 512     ? 1
                                 : L == 384 || L == 512        ? ((PLAINISH && (PFAST || L == 512)) ? 2 : 1)
                                 : L == 192                    ? (MODE == PASS_CH_NL ? 1 : 2)
                                 : is_update_mode(MODE)        ? 2
                                                               : 3;
};

// Shared-memory layout of the pipelined kernels' tiles.
template <int L, int P, bool PFAST>
using PipeLayout = typename std::conditional<PFAST, LayoutB<L, P>, LayoutA<L, P, true>>::type;

// Start the asynchronous load of the tile at pencil q0 (one cp.async group is
// committed by the caller).
template <typename T, int L, int P, int NT, int MODE, bool PFAST>
__device__ __forceinline__ void pipe_issue(cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using LY = PipeLayout<L, P, PFAST>;
    if constexpr (reads_half(MODE)) issue_tile_half<T, L, P, NT, LY>(sm, a, q0);
    else issue_tile<T, L, P, NT, PFAST, LY>(sm, a, q0);
}

// Transform the tile at pencil q0, resident in `sm`, and store it (or apply
// the update).  chat: the tile-sized buffer that receives staged c_hat rows
// (update passes that stage them); tab: the per-tile state table (update
// passes); kp: |k|^2 of the pass axis; tw: the length-L twiddle table.  Ends
// with the tile's results issued; the caller synchronises before reusing
// shared memory.
template <typename T, int L, int P, int NT, int SIGN, int MODE, bool PFAST>
__device__ __forceinline__ void pipe_tile(cx_t<T>* sm, cx_t<T>* chat, const PassParams<T>& a, long long q0,
                                          uint8_t* tab, const T* kp, const cx_t<T>* tw) {
    using C = cx_t<T>;
    using LY = PipeLayout<L, P, PFAST>;
    // direct stores from the last stage stay coalesced when a warp's lanes
    // cover at least 32 contiguous bytes of each output row
    // (the radix-3 tails of 192 and 384 hold too many registers to emit directly)
    constexpr bool DIRECT = (LY::PMAP || (L / Radices_last<L>::value) * (int)sizeof(C) >= 32) &&
                            Radices_last<L>::value != 3;
    if constexpr (MODE == PASS_MIRROR) {
        MirrorPlainOut<T, L, P> out(a, q0);
        run_stages_out<T, L, P, NT, SIGN, LY>(sm, tw, out);
    } else if constexpr (!is_update_mode(MODE) && !DIRECT) {
        // short pencil-major pencils: the staged store keeps 16-byte coalesced writes
        tile_body<T, L, P, NT, SIGN, MODE, LY>(sm, a, q0);
        store_tile<T, L, P, NT, PFAST, LY>(sm, a, q0);
    } else if constexpr (MODE == PASS_PLAIN) {
        if (a.tw4 != nullptr) {
            // first pass of a four-step transform: twiddle in shared memory
            tile_body<T, L, P, NT, SIGN, MODE, LY>(sm, a, q0);
            store_tile<T, L, P, NT, PFAST, LY>(sm, a, q0);
        } else {
            PlainOut<T, L> out(a, q0);
            run_stages_out<T, L, P, NT, SIGN, LY>(sm, tw, out);
        }
    } else if constexpr (MODE == PASS_CH_NL) {
        // inverse transform, the nonlinearity, forward transform (last stage storing)
        ChNlMid<T> mid{a.nl_scale, (T)0};
        PlainOut<T, L> out(a, q0);
        transform_pair<T, L, P, NT, +1, -1, LY>(sm, tw, mid, out);
        const T msum = mid.msum;
        if (a.mass != nullptr) {
            double ms = warp_sum((double)msum);
            if ((threadIdx.x & 31) == 0) atomicAdd(a.mass + (q0 / a.mass_ppr) * a.mass_stride, ms);
        }
    } else {
        const UpdTile u = upd_tile<T, P>(a, (int)q0);
        if (u.rows) {
            // the tile spans several rows of a small grid
            run_stages<T, L, P, NT, -1, LY>(sm, tw);
            ch_update_tile_rows<T, L, P, NT, LY>(sm, a, q0);
        } else if constexpr (upd_stages_chat<T, L>()) {
            // c_hat of the tile's non-frozen rows streams in during the transform
            ch_update_table<T, L, P, NT>(tab, a, u);
            __syncthreads();
            issue_chat<T, L, P, NT, LY>(chat, a, u, tab);
            UpdOut<T, L, P, NT, Radices_last<L>::value, true, LY, MODE == PASS_UPD_HALF> out(a, u, tab, kp, chat);
            run_stages_out<T, L, P, NT, -1, LY>(sm, tw, out);
        } else {
            ch_update_table<T, L, P, NT>(tab, a, u);
            run_stages<T, L, P, NT, -1, LY>(sm, tw);
            UpdOut<T, L, P, NT, 4, false, LY, MODE == PASS_UPD_HALF> out(a, u, tab, kp, nullptr);
            drain_tile<T, L, P, NT, 4, LY>(sm, out);
        }
    }
}

template <typename T, int L, int P, int NT, int SIGN, int MODE, bool PFAST>
__global__ void __launch_bounds__(NT, PipeOcc<T, L, MODE, PFAST>::value) fft_pass_pipe_kernel(PassParams<T> a) {
    using C = cx_t<T>;
    using LY = PipeLayout<L, P, PFAST>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm0 = reinterpret_cast<C*>(smem_raw);
    C* sm1 = sm0 + LY::SIZE;
    __shared__ uint8_t s_tab[is_update_mode(MODE) ? kUpdTable : 1];
    __shared__ T s_kp[is_update_mode(MODE) ? L : 1];   // |k|^2 of the pass axis
    if constexpr (is_update_mode(MODE)) {
        const T* kpg = a.fu.g.ndim == 3 ? a.fu.k2ax[0] : a.fu.k2ax[1];
        for (int j = threadIdx.x; j < L; j += NT) s_kp[j] = kpg[j];   // visible after the loop's first barrier
    }
    // complex64 passes up to 512 points keep the twiddle table in shared memory
    constexpr bool STW = sizeof(T) == 4 && L <= 512;
    __shared__ C s_tw[STW ? L : 1];
    if constexpr (STW)
        for (int j = threadIdx.x; j < L; j += NT) s_tw[j] = a.tw[j];   // visible after the loop's first barrier
    const C* const tw = STW ? s_tw : a.tw;
    const long long ntiles = (a.O * a.I) / P;
    if constexpr (is_update_mode(MODE)) ch_update_stats<T, NT>(a.fu, a.fu.dense);
    long long t = blockIdx.x;
    while (t < ntiles && !tile_live<T, P, MODE>(a, t * P)) t += gridDim.x;
    if (t < ntiles) pipe_issue<T, L, P, NT, MODE, PFAST>(sm0, a, t * P);
    cp_async_commit();
    int buf = 0;
    while (t < ntiles) {
        long long tn = t + gridDim.x;
        while (tn < ntiles && !tile_live<T, P, MODE>(a, tn * P)) tn += gridDim.x;
        if (tn < ntiles) pipe_issue<T, L, P, NT, MODE, PFAST>(buf ? sm0 : sm1, a, tn * P);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        pipe_tile<T, L, P, NT, SIGN, MODE, PFAST>(buf ? sm1 : sm0, sm0 + 2 * LY::SIZE, a, t * P, s_tab, s_kp, tw);
        __syncthreads();
        buf ^= 1;
        t = tn;
    }
    cp_async_wait<0>();
}

}  // namespace spdba
