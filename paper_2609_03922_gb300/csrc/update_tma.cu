// List-driven Cahn-Hilliard update of 3-D complex64 fields with 8^3 blocks,
// moved by the Tensor Memory Accelerator (S1.1 Eq. S.1 blend, S4.2 semi-implicit
// update with M = 1; the same arithmetic as ch_list_kernel, bit for bit).
//
// A block of 8^3 complex64 modes is one 3-D TMA box (8 x 8 x 8 elements of 8
// bytes; rows of 64 bytes).  Each CTA walks its share of the block list with
// TMA_STAGES boxes of c_hat and g_hat in flight: one thread issues the box
// loads (cp.async.bulk.tensor, completion counted on a per-stage mbarrier),
// every thread updates the stage's modes into one of two output boxes once
// the barrier flips, and the same thread stores that box with a bulk tensor
// store and refills the input stage at once (the store reads the output box,
// not the stage).
// Block rows of 64 bytes scattered over the field leave a per-warp load path
// latency-bound; with the boxes in flight per SM the copy engine keeps enough
// bytes outstanding to cover HBM latency.  Every wait is bounded: on timeout
// the kernel records it in the run statistics and returns.
#include "blocks.h"
#include "ch_math.cuh"
#include "tma.cuh"

namespace spdba {

constexpr int TMA_NT = 128;
constexpr int TMA_STAGES = 5;
constexpr int TMA_BOX = 8;
constexpr int TMA_BOX_MODES = TMA_BOX * TMA_BOX * TMA_BOX;           // 512
constexpr unsigned TMA_BOX_BYTES = TMA_BOX_MODES * sizeof(float2);   // 4096

struct TmaStage {
    float2 c[TMA_BOX_MODES];
    float2 g[TMA_BOX_MODES];
};

__global__ void __launch_bounds__(TMA_NT) ch_list_tma_kernel(const __grid_constant__ CUtensorMap map_c,
                                                             const __grid_constant__ CUtensorMap map_g, Geom g,
                                                             CHUpdateArgs<float> a, long long spin_limit,
                                                             int stall) {
    extern __shared__ __align__(128) unsigned char smem_tma[];
    // input stages (128-byte aligned), then two output boxes, then the barriers
    TmaStage* stage = reinterpret_cast<TmaStage*>(smem_tma);
    float2* outb = reinterpret_cast<float2*>(smem_tma + TMA_STAGES * sizeof(TmaStage));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_tma + TMA_STAGES * sizeof(TmaStage) + 2 * TMA_BOX_BYTES);
    __shared__ int s_abort;
    __shared__ uint64_t s_never;   // a barrier nothing arrives on (stall: the timeout path under test)
    const int cnt = *a.count;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats) {
        const unsigned long long nfi = a.stats[0].n_active + a.stats[0].n_transition;
        const double nf = (double)nfi;
        a.stats[0].ratio_sum += nf * (1.0 / (double)g.live_bpr());
        a.stats[0].list_modes += nf * (double)TMA_BOX_MODES;
        a.stats[0].ctl_nf += nfi;
        a.stats[0].ctl_steps += 1;
    }
    const long long nb1 = g.nb[1], nb2 = g.nb[2];
    auto issue = [&](int s, long long w) {
        const long long blk = a.list[w];
        const int bx = (int)(blk % nb2), by = (int)((blk / nb2) % nb1), bz = (int)(blk / (nb2 * nb1));
        mbar_expect_tx(&full[s], 2 * TMA_BOX_BYTES);
        tma_load_box(stage[s].c, &map_c, bx * TMA_BOX, by * TMA_BOX, bz * TMA_BOX, &full[s]);
        tma_load_box(stage[s].g, &map_g, bx * TMA_BOX, by * TMA_BOX, bz * TMA_BOX, &full[s]);
    };
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < TMA_STAGES; ++s) mbar_init(&full[s], 1);
        mbar_init(&s_never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int s = 0; s < TMA_STAGES; ++s) {
            const long long w = blockIdx.x + (long long)s * gridDim.x;
            if (w < cnt) issue(s, w);
        }
    }
    __syncthreads();
    // this thread's modes of a box: m = threadIdx.x + TMA_NT * i share l1 and l2
    constexpr int PER = TMA_BOX_MODES / TMA_NT;   // 4
    const int l2 = threadIdx.x & 7, l1 = (threadIdx.x >> 3) & 7, l0base = threadIdx.x >> 6;
    long long it = 0, it_abort = -1;
    for (long long w = blockIdx.x; w < cnt; w += gridDim.x, ++it) {
        const int s = (int)(it % TMA_STAGES);
        const unsigned parity = (unsigned)((it / TMA_STAGES) & 1);
        float2* ob = outb + (it & 1) * TMA_BOX_MODES;
        // the block's states and |k|^2 values are read before waiting for its
        // boxes, so that their latency overlaps the transfer
        const long long blk = a.list[w];
        const int st = a.states[blk];
        const unsigned ch = a.chi[blk];
        const long long b2 = blk % nb2, b1 = (blk / nb2) % nb1, b0 = blk / (nb2 * nb1);
        const float kyx0 = a.k2ax[1][b1 * TMA_BOX + l1];
        const float kx = a.k2ax[2][b2 * TMA_BOX + l2];
        float kz[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) kz[i] = a.k2ax[0][b0 * TMA_BOX + l0base + 2 * i];
        if (threadIdx.x == 0) {
            // the output box written two iterations ago has been read by its store
            bulk_wait_read_but_newest();
            // bounded wait for the stage's two boxes
            if (!(stall ? mbar_wait_bounded(&s_never, 0u, spin_limit < 4096 ? spin_limit : 4096)
                        : mbar_wait_bounded(&full[s], parity, spin_limit)))
                s_abort = 1;
        }
        __syncthreads();
        if (s_abort) {
            it_abort = it;
            break;
        }
        const float2* c = stage[s].c;
        const float2* gg = stage[s].g;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int m = threadIdx.x + TMA_NT * i;
            const int l0 = l0base + 2 * i;
            const float k2 = (kz[i] + kyx0) + kx;
            const float2 c0 = c[m];
            float2 n0 = ch_new(c0, gg[m], k2, a.dt, a.dtkappa);
            if (st == SPDBA_TRANSITION) n0 = ch_blend<float>(c0, n0, a.taper, g, ch, l0, l1, l2);
            ob[m] = n0;
        }
        // the async proxy (the bulk store) must see the generic-proxy writes
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tma_store_box(&map_c, (int)(b2 * TMA_BOX), (int)(b1 * TMA_BOX), (int)(b0 * TMA_BOX), ob);
            bulk_commit();
            // the input stage is free as soon as the update has read it
            const long long wn = w + (long long)TMA_STAGES * gridDim.x;
            if (wn < cnt) issue(s, wn);
        }
    }
    if (threadIdx.x == 0) {
        bulk_wait_all();
        if (it_abort >= 0) {
            // let the loads still in flight land (bounded) before the CTA leaves:
            // iterations it_abort .. it_abort + TMA_STAGES - 1 had theirs issued
            for (int k = 0; k < TMA_STAGES; ++k) {
                const long long it2 = it_abort + k;
                if (blockIdx.x + it2 * gridDim.x < cnt)
                    mbar_wait_bounded(&full[it2 % TMA_STAGES], (unsigned)((it2 / TMA_STAGES) & 1), kWaitLimit);
            }
            if (a.stats) atomicAdd(&a.stats[0].timeouts, 1ull);
        }
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

spdba_status tma_encode_3d(void* map_out, const void* base, const uint64_t dims[3], const uint64_t row_bytes,
                           const uint64_t plane_bytes, const uint32_t box[3]) {
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(SPDBA_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
        encode = (EncodeTiledFn)fn;
    }
    if (((uintptr_t)base & 15) != 0) return fail(SPDBA_ERR_ARG, "TMA base address not 16-byte aligned");
    // 8-byte elements (one complex64 each); the innermost box row must be a multiple of 16 bytes
    if ((box[0] * 8) % 16 != 0) return fail(SPDBA_ERR_ARG, "TMA box row not a multiple of 16 bytes");
    const cuuint64_t d[3] = {(cuuint64_t)dims[0], (cuuint64_t)dims[1], (cuuint64_t)dims[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)row_bytes, (cuuint64_t)plane_bytes};
    const cuuint32_t b[3] = {box[0], box[1], box[2]};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_UINT64, 3,
                        const_cast<void*>(base), d, strides, b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SPDBA_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return SPDBA_OK;
}

spdba_status make_box_map(void* map_out, const void* base, const Geom& g) {
    const uint64_t dims[3] = {(uint64_t)g.n[2], (uint64_t)g.n[1], (uint64_t)g.n[0]};
    const uint32_t box[3] = {TMA_BOX, TMA_BOX, TMA_BOX};
    return tma_encode_3d(map_out, base, dims, (uint64_t)g.n[2] * 8, (uint64_t)(g.n[2] * g.n[1]) * 8, box);
}

bool tma_update_fits(const Geom& g) {
    return g.ndim == 3 && g.b[0] == TMA_BOX && g.b[1] == TMA_BOX && g.b[2] == TMA_BOX && g.runs() == 1 &&
           g.n[2] % TMA_BOX == 0;
}

size_t tma_update_smem() {
    return TMA_STAGES * sizeof(TmaStage) + 2 * TMA_BOX_BYTES + TMA_STAGES * sizeof(uint64_t);
}

spdba_status tma_update_prepare(int* per_sm, int* nsm) {
    const int smem = (int)tma_update_smem();
    SPDBA_CUDA(cudaFuncSetAttribute((const void*)ch_list_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int k = 0, dev = 0, n = 0;
    SPDBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, (const void*)ch_list_tma_kernel, TMA_NT, smem));
    SPDBA_CUDA(cudaGetDevice(&dev));
    SPDBA_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    *per_sm = k < 1 ? 1 : k;
    *nsm = n < 1 ? 1 : n;
    return SPDBA_OK;
}

spdba_status launch_ch_update_tma(const void* map_c, const void* map_g, const Geom& g, const CHUpdateArgs<float>& a,
                                  long long grid, cudaStream_t st) {
    const long long cap = g.blocks();
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    ch_list_tma_kernel<<<(unsigned)grid, TMA_NT, tma_update_smem(), st>>>(
        *reinterpret_cast<const CUtensorMap*>(map_c), *reinterpret_cast<const CUtensorMap*>(map_g), g, a,
        wait_limit(), stall_waits());
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

}  // namespace spdba
