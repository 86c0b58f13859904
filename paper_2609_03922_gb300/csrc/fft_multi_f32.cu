// Multi-size persistent pass kernels (complex64): one launch of a pass phase
// (the inverse transform along the first axis, the fused nonlinearity along the
// last, the forward transform with the update along the first) serves every
// group of a batched plan, whatever its run size.  The groups' tiles form one
// queue, numbered group after group; the persistent CTAs of the launch walk it
// in a fixed stride (CTA c takes positions c, c + grid, ...; frozen tiles of an
// update pass are passed over), so a large group and a small one share the
// machine within one launch instead of one launch (or one stream) each.  Each tile runs exactly the code of the
// one-group pipelined kernel for its length (pipe_issue / pipe_tile), with the
// group's pass parameters staged in shared memory.
#include "internal.h"
#include "kernel_table.h"

namespace spdba {

// Pencils per tile in the table of TILE elements per tile: the largest power
// of two P <= 64 with P * L <= TILE (at least 2), so that one pair of tile
// buffers fits every length.
template <int TILE, int L> struct MultiP {
    static constexpr int q = TILE / L;
    static constexpr int value = q >= 64 ? 64 : q >= 32 ? 32 : q >= 16 ? 16 : q >= 8 ? 8 : q >= 4 ? 4 : 2;
};

// Calls f(std::integral_constant<int, L>) for the lengths with multi-size kernels.
template <class F> __device__ __forceinline__ void with_length(int L, F&& f) {
    switch (L) {
        case 64: f(std::integral_constant<int, 64>()); break;
        case 128: f(std::integral_constant<int, 128>()); break;
        case 192: f(std::integral_constant<int, 192>()); break;
        case 256: f(std::integral_constant<int, 256>()); break;
        case 384: f(std::integral_constant<int, 384>()); break;
        case 512: f(std::integral_constant<int, 512>()); break;
        default: break;
    }
}
static bool multi_length(int64_t L) {
    return L == 64 || L == 128 || L == 192 || L == 256 || L == 384 || L == 512;
}

constexpr int cmax(int a, int b) { return a > b ? a : b; }
// Elements of one tile buffer: the largest tile layout over the lengths.
template <int TILE, bool PFAST> struct MultiBuf {
    template <int L> static constexpr int sz() { return PipeLayout<L, MultiP<TILE, L>::value, PFAST>::SIZE; }
    static constexpr int SIZE =
        cmax(cmax(cmax(sz<64>(), sz<128>()), cmax(sz<192>(), sz<256>())), cmax(sz<384>(), sz<512>()));
};

// Group of queue position t (groups in queue order, ng >= 1).
template <typename T>
__device__ __forceinline__ int multi_group_of(const MultiGroup<T>* __restrict__ gs, int ng, unsigned t) {
    int g = 0;
    while (g + 1 < ng && t >= gs[g + 1].t0) ++g;
    return g;
}

// Resident CTAs per SM the kernels are compiled for (128 registers a thread
// at 256 threads).  The tile functions of 192 and 384 points spill a few
// hundred bytes at this budget; one CTA per SM (no spills) measured slower
// (the ensemble's nonlinearity pass 115 against 94 us, its update pass 170
// against 111 us).
template <int MODE> struct MultiOcc { static constexpr int value = 2; };

// One tile of length L (queue position `lt` within its group).  Not inlined:
// each length gets its own register allocation, the launch the largest.
template <typename T, int TILE, int L, int SIGN, int MODE, bool PFAST>
__device__ __noinline__ void multi_tile(cx_t<T>* sm, cx_t<T>* chat, const PassParams<T>& a, unsigned lt,
                                        uint8_t* tab) {
    constexpr int P = MultiP<TILE, L>::value;
    const T* kp = nullptr;
    if constexpr (is_update_mode(MODE)) kp = a.fu.g.ndim == 3 ? a.fu.k2ax[0] : a.fu.k2ax[1];
    pipe_tile<T, L, P, kMultiNT, SIGN, MODE, PFAST>(sm, chat, a, (long long)lt * P, tab, kp, a.tw);
}

template <typename T, int TILE, int SIGN, int MODE, bool PFAST>
__global__ void __launch_bounds__(kMultiNT, MultiOcc<MODE>::value)
    fft_multi_kernel(const MultiGroup<T>* __restrict__ gs, int ng, unsigned total, unsigned dense_mask,
                     unsigned mass_mask) {
    using C = cx_t<T>;
    constexpr int NT = kMultiNT;
    constexpr int BUF = MultiBuf<TILE, PFAST>::SIZE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm0 = reinterpret_cast<C*>(smem_raw);
    C* sm1 = sm0 + BUF;
    C* chat = sm0 + 2 * BUF;   // update passes: staged c_hat rows
    static_assert(sizeof(PassParams<T>) % 8 == 0, "pass parameters copy as 8-byte words");
    constexpr int PW = (int)(sizeof(PassParams<T>) / 8);
    __shared__ unsigned long long s_par[2][PW];   // the pass parameters of the two buffered tiles
    __shared__ uint8_t s_tab[is_update_mode(MODE) ? kUpdTable : 1];

    if constexpr (is_update_mode(MODE)) {
        for (int g = 0; g < ng; ++g) ch_update_stats<T, NT>(gs[g].a.fu, (int)((dense_mask >> g) & 1u));
    }
    // the first live queue position at or after t in this CTA's share (t,
    // t + gridDim.x, ...), total when none is left; every warp finds the same
    auto next_live = [&](unsigned t) -> unsigned {
        for (; t < total; t += gridDim.x) {
            if constexpr (is_update_mode(MODE)) {
                const int g = multi_group_of(gs, ng, t);
                if ((dense_mask >> g) & 1u) return t;
                const MultiGroup<T>& G = gs[g];
                bool live = true;
                with_length(G.L, [&](auto lc) {
                    constexpr int L = decltype(lc)::value;
                    constexpr int P = MultiP<TILE, L>::value;
                    live = tile_live<T, P, MODE>(G.a, (long long)(t - G.t0) * P);
                });
                if (live) return t;
            } else {
                return t;
            }
        }
        return total;
    };
    // stage group g's parameters for a buffered tile; patched after the next barrier
    auto load_par = [&](int slot, int g) {
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&gs[g].a);
        for (int w = threadIdx.x; w < PW; w += NT) s_par[slot][w] = src[w];
    };
    auto patch_par = [&](int slot, int g) {
        PassParams<T>& a = *reinterpret_cast<PassParams<T>*>(s_par[slot]);
        a.fu.dense = (int)((dense_mask >> g) & 1u);
        if (!((mass_mask >> g) & 1u)) a.mass = nullptr;
    };
    auto issue = [&](C* sm, int g, unsigned t) {
        const MultiGroup<T>& G = gs[g];
        with_length(G.L, [&](auto lc) {
            constexpr int L = decltype(lc)::value;
            constexpr int P = MultiP<TILE, L>::value;
            pipe_issue<T, L, P, NT, MODE, PFAST>(sm, G.a, (long long)(t - G.t0) * P);
        });
    };

    unsigned t = next_live(blockIdx.x);
    int g = t < total ? multi_group_of(gs, ng, t) : 0;
    if (t < total) {
        load_par(0, g);
        issue(sm0, g, t);
    }
    cp_async_commit();
    __syncthreads();
    if (t < total && threadIdx.x == 0) patch_par(0, g);
    int buf = 0;
    while (t < total) {
        const unsigned tn = next_live(t + gridDim.x);
        const int gn = tn < total ? multi_group_of(gs, ng, tn) : 0;
        if (tn < total) {
            load_par(buf ^ 1, gn);
            issue(buf ? sm0 : sm1, gn, tn);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();   // tile t has landed; its parameters are patched; the next tile's are copied
        if (tn < total && threadIdx.x == 0) patch_par(buf ^ 1, gn);   // read after the next barrier
        const PassParams<T>& a = *reinterpret_cast<const PassParams<T>*>(s_par[buf]);
        with_length(gs[g].L, [&](auto lc) {
            constexpr int L = decltype(lc)::value;
            multi_tile<T, TILE, L, SIGN, MODE, PFAST>(buf ? sm1 : sm0, chat, a, t - gs[g].t0, s_tab);
        });
        __syncthreads();
        buf ^= 1;
        t = tn;
        g = gn;
    }
    cp_async_wait<0>();
}

int multi_tile_pencils(int tile, int64_t L) {
    if (!multi_length(L)) return 0;
    const int64_t q = tile / L;
    return q >= 64 ? 64 : q >= 32 ? 32 : q >= 16 ? 16 : q >= 8 ? 8 : q >= 4 ? 4 : 2;
}

template <int TILE> static bool pick_multi(int sign, int mode, bool pfast, const void** func, int* smem) {
    using C = cx_t<float>;
    const void* f = nullptr;
    int nbuf = 2;
    if (pfast) {
        if (mode == PASS_PLAIN)
            f = sign < 0 ? (const void*)fft_multi_kernel<float, TILE, -1, PASS_PLAIN, true>
                         : (const void*)fft_multi_kernel<float, TILE, +1, PASS_PLAIN, true>;
        else if (mode == PASS_CH_UPDATE) {
            f = (const void*)fft_multi_kernel<float, TILE, -1, PASS_CH_UPDATE, true>;
            nbuf = 3;
        }
        *smem = nbuf * MultiBuf<TILE, true>::SIZE * (int)sizeof(C);
    } else {
        if (mode == PASS_CH_NL) f = (const void*)fft_multi_kernel<float, TILE, -1, PASS_CH_NL, false>;
        *smem = nbuf * MultiBuf<TILE, false>::SIZE * (int)sizeof(C);
    }
    *func = f;
    return f != nullptr;
}

spdba_status multi_kernel(int tile, int sign, int mode, bool pfast, const void** func, int* smem,
                          long long* resident) {
    bool ok = false;
    if (tile == 4096) ok = pick_multi<4096>(sign, mode, pfast, func, smem);
    else if (tile == 2048) ok = pick_multi<2048>(sign, mode, pfast, func, smem);
    if (!ok) return fail(SPDBA_ERR_UNSUPPORTED, "no multi-size pass kernel (tile %d, mode %d)", tile, mode);
    SPDBA_CUDA(cudaFuncSetAttribute(*func, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem));
    SPDBA_CUDA(cudaFuncSetAttribute(*func, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per_sm = 0, nsm = 0, dev = 0;
    SPDBA_CUDA(cudaGetDevice(&dev));
    SPDBA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SPDBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, *func, kMultiNT, *smem));
    if (per_sm < 1) return fail(SPDBA_ERR_UNSUPPORTED, "multi-size pass kernel does not fit an SM");
    *resident = (long long)per_sm * nsm;
    return SPDBA_OK;
}

spdba_status launch_multi(const void* func, int smem, long long grid, const MultiGroup<float>* groups, int ng,
                          unsigned total, unsigned dense_mask, unsigned mass_mask, cudaStream_t st) {
    if (total == 0 || grid < 1) return SPDBA_OK;
    void* args[] = {&groups, &ng, &total, &dense_mask, &mass_mask};
    SPDBA_CUDA(cudaLaunchKernel(func, dim3((unsigned)grid), dim3(kMultiNT), args, (size_t)smem, st));
    return SPDBA_OK;
}

}  // namespace spdba
