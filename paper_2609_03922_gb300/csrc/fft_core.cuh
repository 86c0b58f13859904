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
// Every second pencil of a layout-A tile (pencil m at slot 2m): the packed
// pencils of the two-real-signals transforms.
template <int L, int P> struct LayoutA2 {
    static constexpr int PSTR = 2 * (L + L / 16 + 1);
    static constexpr bool PMAP = false;
    static __device__ __forceinline__ int idx(int m, int j) { return m * PSTR + j + (j >> 4); }
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
    PASS_CH_UPDATE = 2,  // forward transform, then the CH update of c_hat (no store of the transform)
};

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

// A tile is live when any block its modes belong to is not FROZEN.  Every warp
// evaluates this independently (no block-wide synchronisation needed).
template <typename T, int P, int MODE>
__device__ __forceinline__ bool tile_live(const PassParams<T>& a, long long q0) {
    if constexpr (MODE != PASS_CH_UPDATE) return true;
    else {
        if (a.fu.dense) return true;
        const Geom& g = a.fu.g;
        long long c0, c1, c2;
        fuse_coords<T>(a, q0, 0, 0, c0, c1, c2);
        const long long bx0 = c2 / g.b[2], bx1 = (c2 + P - 1) / g.b[2];
        const long long nbx = bx1 - bx0 + 1;
        // blocks along the pass axis: all of them
        const long long npass = g.ndim == 3 ? g.nb[0] : g.nb[1];
        const long long total = npass * nbx;
        bool live = false;
        for (long long k = threadIdx.x & 31; k < total && !live; k += 32) {
            long long bp = k / nbx, bx = bx0 + k % nbx;
            long long id = g.ndim == 3 ? (bp * g.nb[1] + c1 / g.b[1]) * g.nb[2] + bx
                                       : (c0 * g.nb[1] + bp) * g.nb[2] + bx;
            live = a.fu.states[id] != 0;
        }
        return __any_sync(0xffffffffu, live);
    }
}

// Per-run share of non-frozen blocks for this step (CTA 0, once per launch).
template <typename T, int NT> __device__ __forceinline__ void ch_update_stats(const CHFuse<T>& f) {
    const Geom& g = f.g;
    if (blockIdx.x != 0 || !f.stats) return;
    const double inv = 1.0 / (double)g.bpr();
    const long long bm = g.block_modes();
    for (long long r = threadIdx.x; r < g.runs(); r += NT) {
        double nf = f.dense ? (double)g.bpr() : (double)(f.stats[r].n_active + f.stats[r].n_transition);
        f.stats[r].ratio_sum += nf * inv;
        if (!f.dense) f.stats[r].list_modes += nf * (double)bm;
    }
}

// Update epilogue: g_hat of the tile is in shared memory (layout B).  The
// tile's block states and chi bits are staged in shared memory once; every
// thread issues its c_hat loads (non-frozen rows only) before using any.
template <typename T, int L, int P, int NT, class LY>
__device__ __forceinline__ void ch_update_tile(const cx_t<T>* sm, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
    const CHFuse<T>& f = a.fu;
    const Geom& g = f.g;
    constexpr int MAXB = 256;
    __shared__ uint8_t s_st[MAXB], s_chi[MAXB];
    // tile-constant coordinates: 3-D (z = j, y, x0 + p); 2-D group (run, y = j, x0 + p)
    const long long o = q0 / a.I, i0 = q0 - o * a.I;
    const bool d3 = g.ndim == 3;
    if (d3 && (i0 % g.n[2]) + P > g.n[2]) {
        // the tile spans several rows of a small grid: per-mode coordinates and states
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
        return;
    }
    const long long cy = d3 ? i0 / g.n[2] : o;        // coordinate on the non-pass outer axis
    const long long x0 = d3 ? i0 - cy * g.n[2] : i0;
    const int Bp = d3 ? g.b[0] : g.b[1];               // block edge along the pass axis
    const long long npass = d3 ? g.nb[0] : g.nb[1];
    const long long bx0 = x0 / g.b[2];
    const int nbx = (int)((x0 + P - 1) / g.b[2] - bx0 + 1);
    const int nst = (int)(npass * nbx);
    for (int k = threadIdx.x; k < nst; k += NT) {
        long long bp = k / nbx, bx = bx0 + k % nbx;
        long long id = d3 ? (bp * g.nb[1] + cy / g.b[1]) * g.nb[2] + bx : (cy * g.nb[1] + bp) * g.nb[2] + bx;
        s_st[k] = f.dense ? (uint8_t)SPDBA_ACTIVE : f.states[id];
        s_chi[k] = f.dense ? (uint8_t)0 : f.chi[id];
    }
    __syncthreads();
    const T* __restrict__ kp = d3 ? f.k2ax[0] : f.k2ax[1];   // |k|^2 table of the pass axis
    const T kc = d3 ? f.k2ax[1][cy] : f.k2ax[0][cy];         // fixed outer axis (0 for a group's run axis)
    const int l_out = (int)(d3 ? cy % g.b[1] : 0);
    constexpr int E = sizeof(C) == 8 ? 2 : 1;   // modes per 16-byte access
    constexpr int UPR = P / E;                   // units per row of the tile
    static_assert(NT % UPR == 0, "threads must cover whole rows");
    constexpr int JSTEP = NT / UPR;              // rows advanced per unit step
    constexpr int PER = L / JSTEP;               // units per thread
    // this thread's pencil offset and first row never change within the tile
    const int p = (threadIdx.x % UPR) * E;
    const int j0 = threadIdx.x / UPR;
    const long long x = x0 + p;
    const int bxs = (int)(x / g.b[2] - bx0);
    const int lx = (int)(x % g.b[2]);
    T kx[E];
#pragma unroll
    for (int e = 0; e < E; ++e) kx[e] = f.k2ax[2][x + e];
    const long long o2 = (q0 / a.I) * a.osO + (i0 + p) * a.osI;   // address of (p, j = 0)
    C cv[PER][E];
    int stv[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int j = j0 + k * JSTEP;
        stv[k] = s_st[(j / Bp) * nbx + bxs];
        if (stv[k] == SPDBA_FROZEN) continue;
        const long long ad = o2 + (long long)j * a.osJ;
        if constexpr (E == 2) {
            float4 t = *reinterpret_cast<const float4*>(f.c_hat + ad);
            cv[k][0] = make_float2(t.x, t.y);
            cv[k][1] = make_float2(t.z, t.w);
        } else {
            cv[k][0] = f.c_hat[ad];
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (stv[k] == SPDBA_FROZEN) continue;
        const int j = j0 + k * JSTEP;
        const long long ad = o2 + (long long)j * a.osJ;
        // same association as the staged kernels: (k_outer + k_pass) then + k_x
        const T k01 = d3 ? kp[j] + kc : kc + kp[j];
        C nv[E];
#pragma unroll
        for (int e = 0; e < E; ++e) nv[e] = ch_new(cv[k][e], sm[LY::idx(p + e, j)], k01 + kx[e], f.dt, f.dtkappa);
        if (stv[k] == SPDBA_TRANSITION) {
            const unsigned chi = s_chi[(j / Bp) * nbx + bxs];
            const int lj = j % Bp;
#pragma unroll
            for (int e = 0; e < E; ++e)
                nv[e] = d3 ? ch_blend<T>(cv[k][e], nv[e], f.taper, g, chi, lj, l_out, lx + e)
                           : ch_blend<T>(cv[k][e], nv[e], f.taper, g, chi, 0, lj, lx + e);
        }
        if constexpr (E == 2) {
            *reinterpret_cast<float4*>(f.c_hat + ad) = make_float4(nv[0].x, nv[0].y, nv[1].x, nv[1].y);
        } else {
            f.c_hat[ad] = nv[0];
        }
    }
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
        // c = Re(IFFT_x(w)) equals IFFT_x of w's Hermitian part H(w)(k) = (w(k) + conj(w(-k)))/2,
        // which lies in the same pencil.  Two Hermitian pencils a, b go through one
        // complex transform as H(a) + i H(b): the real and imaginary parts of the result
        // are the two real fields; g = c^3 - c of both is packed as g_a + i g_b, transformed
        // forward once, and separated by symmetry (G_a(k) = (Z(k) + conj Z(-k))/2,
        // G_b(k) = (Z(k) - conj Z(-k))/(2i)).
      if constexpr (P % 2 == 0 && !LY::PMAP) {
        using L2 = LayoutA2<L, P>;
        constexpr int H = L / 2 + 1;   // k = 0 .. L/2 (each with its mirror L - k)
        for (int e = threadIdx.x; e < (P / 2) * H; e += NT) {
            const int m = e / H, k = e % H, kr = (L - k) % L;
            const C a0 = sm[LY::idx(2 * m, k)], a1 = sm[LY::idx(2 * m, kr)];
            const C b0 = sm[LY::idx(2 * m + 1, k)], b1 = sm[LY::idx(2 * m + 1, kr)];
            const T h = (T)0.5;
            // H(a)(k) and H(b)(k); H(x)(-k) = conj(H(x)(k))
            const C ha = mk<C>(h * (a0.x + a1.x), h * (a0.y - a1.y));
            const C hb = mk<C>(h * (b0.x + b1.x), h * (b0.y - b1.y));
            sm[LY::idx(2 * m, k)] = mk<C>(ha.x - hb.y, ha.y + hb.x);      // H(a) + i H(b) at k
            sm[LY::idx(2 * m, kr)] = mk<C>(ha.x + hb.y, -ha.y + hb.x);    // at -k
        }
        __syncthreads();
        run_stages<T, L, P / 2, NT, +1, L2>(sm, a.tw);
        T msum = 0;
        for (int e = threadIdx.x; e < (P / 2) * L; e += NT) {
            const int m = e / L, j = e % L;
            const C v = sm[L2::idx(m, j)];
            const T ca = v.x * a.nl_scale, cb = v.y * a.nl_scale;
            msum += ca + cb;
            sm[L2::idx(m, j)] = mk<C>(ca * ca * ca - ca, cb * cb * cb - cb);
        }
        if (a.mass != nullptr) {
            double ms = (double)msum;
            ms = warp_sum(ms);
            if ((threadIdx.x & 31) == 0) atomicAdd(a.mass + (q0 / a.mass_ppr) * a.mass_stride, ms);
        }
        __syncthreads();
        run_stages<T, L, P / 2, NT, -1, L2>(sm, a.tw);
        for (int e = threadIdx.x; e < (P / 2) * H; e += NT) {
            const int m = e / H, k = e % H, kr = (L - k) % L;
            const C z0 = sm[LY::idx(2 * m, k)], z1 = sm[LY::idx(2 * m, kr)];
            const T h = (T)0.5;
            const C ga = mk<C>(h * (z0.x + z1.x), h * (z0.y - z1.y));     // (Z(k) + conj Z(-k))/2
            const C gb = mk<C>(h * (z0.y + z1.y), h * (z1.x - z0.x));     // (Z(k) - conj Z(-k))/(2i)
            sm[LY::idx(2 * m, k)] = ga;
            sm[LY::idx(2 * m, kr)] = mk<C>(ga.x, -ga.y);
            sm[LY::idx(2 * m + 1, k)] = gb;
            sm[LY::idx(2 * m + 1, kr)] = mk<C>(gb.x, -gb.y);
        }
        __syncthreads();
      } else {
        // one pencil at a time: inverse transform, c = Re(.)/N, g = c^3 - c, forward
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
    static constexpr int value = (sizeof(T) == 4 && L <= 256) ? (MODE == PASS_PLAIN ? 3 : MODE == PASS_CH_UPDATE ? 2 : 1) : 1;
};

template <typename T, int L, int P, int NT, int SIGN, int MODE, bool PFAST>
__global__ void __launch_bounds__(NT, PipeOcc<T, L, MODE>::value) fft_pass_pipe_kernel(PassParams<T> a) {
    using C = cx_t<T>;
    using LY = typename std::conditional<PFAST, LayoutB<L, P>, LayoutA<L, P, true>>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm0 = reinterpret_cast<C*>(smem_raw);
    C* sm1 = sm0 + LY::SIZE;
    const long long ntiles = (a.O * a.I) / P;
    if constexpr (MODE == PASS_CH_UPDATE) ch_update_stats<T, NT>(a.fu);
    long long t = blockIdx.x;
    while (t < ntiles && !tile_live<T, P, MODE>(a, t * P)) t += gridDim.x;
    if (t < ntiles) issue_tile<T, L, P, NT, PFAST, LY>(sm0, a, t * P);
    cp_async_commit();
    int buf = 0;
    while (t < ntiles) {
        long long tn = t + gridDim.x;
        while (tn < ntiles && !tile_live<T, P, MODE>(a, tn * P)) tn += gridDim.x;
        if (tn < ntiles) issue_tile<T, L, P, NT, PFAST, LY>(buf ? sm0 : sm1, a, tn * P);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        C* sm = buf ? sm1 : sm0;
        tile_body<T, L, P, NT, SIGN, MODE, LY>(sm, a, t * P);
        if constexpr (MODE == PASS_CH_UPDATE) ch_update_tile<T, L, P, NT, LY>(sm, a, t * P);
        else store_tile<T, L, P, NT, PFAST, LY>(sm, a, t * P);
        __syncthreads();
        buf ^= 1;
        t = tn;
    }
    cp_async_wait<0>();
}

}  // namespace spdba
