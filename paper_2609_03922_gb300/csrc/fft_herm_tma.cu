// z inverse of the Hermitian half-spectrum form (3-D complex64) with its
// tiles moved by the Tensor Memory Accelerator: the same transform as
// fft_herm_inv_kernel (fft_half.cuh), bit for bit, with the per-thread
// cp.async copies of the direct and mirror tiles replaced by a few tensor-box
// copies that one thread issues.
//
// Tile t: P consecutive pencils (ky, kx0 .. kx0 + P - 1) of the half array
// (NHP % P == 0: a tile stays in one x row).  Its boxes over c_hat (x fastest):
//   direct: x = kx0 .. kx0 + P - 1, y = ky, all z: lands as [z][p], the
//           row-major tile layout of the transform;
//   mirror: x = N2 - kx0 - P .. N2 - kx0 + 1 (P + 2 columns from an even
//           start), y = -ky mod N1, all z: pencil p's mirror column N2 - kx
//           sits at slot P - p of each row, and z = -kz mod N0 is read at kz;
//   for kx0 = 0 also x = 0, 1 of row -ky (the kx = 0 pencil mirrors onto
//           itself; columns N2, N2 + 1 of the mirror box lie beyond the array
//           and read as zero).
// Columns past N2/2 (padding pencils) are zeroed by the reader.  Boxes hold at
// most 256 z; longer pencils take two boxes per tile.  One thread issues the
// copies and waits on the tile's mbarriers (bounded: on timeout the kernel
// counts it, lets the copies in flight land, bounded again, and returns).
#include "fft_half.cuh"
#include "blocks.h"
#include "internal.h"
#include "tma.cuh"

namespace spdba {


// (direct + conj(mirror)) / 2 of element m of pencil p, from the tensor-box tiles
template <int L, int P> struct HermInBox {
    const float2* a;    // direct tile, row-major [z][p]
    const float2* b;    // mirror tile, [z][P + 2]
    const float2* c;    // kx = 0 columns of row -ky, [z][2] (tiles with kx0 = 0)
    int kx0, M;
    __device__ __forceinline__ float2 operator()(int p, int m) const {
        if (kx0 + p > M) return make_float2(0.f, 0.f);
        const int mz = m == 0 ? 0 : L - m;
        const float2 x = a[m * P + p];
        const float2 y = (kx0 + p == 0) ? c[mz * 2] : b[mz * (P + 2) + (P - p)];
        return make_float2(0.5f * (x.x + y.x), 0.5f * (x.y - y.y));
    }
};

template <int L, int P, int NT>
__global__ void __launch_bounds__(NT, 2)
    fft_herm_inv_tma_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                            const __grid_constant__ CUtensorMap map_c, PassParams<float> a,
                            unsigned long long* timeouts, long long spin_limit, int stall) {
    using C = float2;
    using LY = LayoutB<L, P>;
    constexpr int ZB = L <= 256 ? L : L / 2;   // z extent of one box
    constexpr int NZB = L / ZB;
    extern __shared__ __align__(128) unsigned char smem_herm[];
    C* smA0 = reinterpret_cast<C*>(smem_herm);
    C* smA1 = smA0 + LY::SIZE;
    C* smB = smA1 + LY::SIZE;
    C* smC = smB + L * (P + 2);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smC + 2 * L);   // fullA[0], fullA[1], fullB
    __shared__ C s_tw[L];
    __shared__ int s_abort;
    __shared__ uint64_t s_never;   // a barrier nothing arrives on (stall: the timeout path under test)
    for (int j = threadIdx.x; j < L; j += NT) s_tw[j] = a.tw[j];   // visible after the loop's first barrier
    const HalfGeo& h = a.hg;
    const int M = h.N2 >> 1;
    const long long ntiles = (a.O * a.I) / P;
    constexpr unsigned BYTES_A = (unsigned)(P * L * sizeof(C));
    constexpr unsigned BYTES_B = (unsigned)((P + 2) * L * sizeof(C));
    constexpr unsigned BYTES_C = (unsigned)(2 * L * sizeof(C));
    auto tile_pos = [&](long long t, int& ky, int& kx0) {
        const int q = (int)(t * P);
        ky = (int)h.fd_NHP.div((uint32_t)q);
        kx0 = q - ky * h.NHP;
    };
    auto issue_a = [&](C* dst, uint64_t* br, long long t) {
        int ky, kx0;
        tile_pos(t, ky, kx0);
        mbar_expect_tx(br, BYTES_A);
#pragma unroll
        for (int zb = 0; zb < NZB; ++zb) tma_load_box(dst + zb * ZB * P, &map_a, kx0, ky, zb * ZB, br);
    };
    auto issue_b = [&](long long t) {
        int ky, kx0;
        tile_pos(t, ky, kx0);
        const int my = ky == 0 ? 0 : h.N1 - ky;
        mbar_expect_tx(&bar[2], BYTES_B + (kx0 == 0 ? BYTES_C : 0u));
#pragma unroll
        for (int zb = 0; zb < NZB; ++zb) {
            tma_load_box(smB + zb * ZB * (P + 2), &map_b, h.N2 - kx0 - P, my, zb * ZB, &bar[2]);
            if (kx0 == 0) tma_load_box(smC + zb * ZB * 2, &map_c, 0, my, zb * ZB, &bar[2]);
        }
    };
    // thread 0: phase parity to wait for next, and whether a copy is in flight, per barrier
    unsigned ph_a[2] = {0u, 0u}, ph_b = 0u;
    bool out_a[2] = {false, false}, out_b = false;
    long long t = blockIdx.x;
    if (threadIdx.x == 0) {
        s_abort = 0;
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        mbar_init(&s_never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (t < ntiles) {
            issue_a(smA0, &bar[0], t);
            issue_b(t);
            out_a[0] = out_b = true;
        }
    }
    __syncthreads();
    int buf = 0;
    while (t < ntiles) {
        const long long tn = t + gridDim.x;
        if (threadIdx.x == 0) {
            if (tn < ntiles) {
                // the other buffer's last reads ended at the previous iteration's barrier
                fence_async_smem();
                issue_a(buf ? smA0 : smA1, &bar[buf ^ 1], tn);
                out_a[buf ^ 1] = true;
            }
            // the direct and mirror tiles of t
            bool ok = stall ? mbar_wait_bounded(&s_never, 0u, spin_limit < 4096 ? spin_limit : 4096)
                            : mbar_wait_bounded(&bar[buf], ph_a[buf], spin_limit);
            if (ok) {
                ph_a[buf] ^= 1u;
                out_a[buf] = false;
                ok = mbar_wait_bounded(&bar[2], ph_b, spin_limit);
                if (ok) {
                    ph_b ^= 1u;
                    out_b = false;
                }
            }
            if (!ok) s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;
        C* sm = buf ? smA1 : smA0;
        int ky, kx0;
        tile_pos(t, ky, kx0);
        PlainOut<float, L> out(a, t * P);
        HermInBox<L, P> in{sm, smB, smC, kx0, M};
        // the first stage reads the direct and mirror tiles; its barrier between
        // reads and writes frees the mirror buffer for the next tile's copy
        stockham_stage_in<float, L, P, NT, +1, 1, radix_at<L>(0), LY>(sm, s_tw, in);
        if (threadIdx.x == 0 && tn < ntiles) {
            fence_async_smem();
            issue_b(tn);
            out_b = true;
        }
        run_stage_range<float, L, P, NT, +1, LY, 1, NSTAGES<L>::value - 1>(sm, s_tw);
        stockham_stage_out<float, L, P, NT, +1, ns_at<L>(NSTAGES<L>::value - 1), radix_at<L>(NSTAGES<L>::value - 1),
                           LY>(sm, s_tw, out);
        __syncthreads();
        buf ^= 1;
        t = tn;
    }
    if (threadIdx.x == 0 && s_abort) {
        // copies still in flight land before the CTA leaves (bounded)
        for (int k = 0; k < 2; ++k)
            if (out_a[k]) mbar_wait_bounded(&bar[k], ph_a[k], kWaitLimit);
        if (out_b) mbar_wait_bounded(&bar[2], ph_b, kWaitLimit);
        if (timeouts) atomicAdd(timeouts, 1ull);
    }
}

template <int L, int P> static size_t herm_tma_smem() {
    return (2 * LayoutB<L, P>::SIZE + L * (P + 2) + 2 * L) * sizeof(float2) + 3 * sizeof(uint64_t);
}

template <int L, int P> static spdba_status herm_tma_kernel_info(const void** f, size_t* smem) {
    *f = (const void*)fft_herm_inv_tma_kernel<L, P, kHermTmaNT>;
    *smem = herm_tma_smem<L, P>();
    return SPDBA_OK;
}

static spdba_status herm_tma_kernel(int L, int P, const void** f, size_t* smem) {
    if (L == 64 && P == 64) return herm_tma_kernel_info<64, 64>(f, smem);
    if (L == 128 && P == 32) return herm_tma_kernel_info<128, 32>(f, smem);
    if (L == 256 && P == 16) return herm_tma_kernel_info<256, 16>(f, smem);
    if (L == 384 && P == 8) return herm_tma_kernel_info<384, 8>(f, smem);
    if (L == 512 && P == 16) return herm_tma_kernel_info<512, 16>(f, smem);
    return SPDBA_ERR_UNSUPPORTED;
}

spdba_status herm_tma_prepare(HermTma* ht, const Pass<float>& zinv, const void* c_hat) {
    const HalfGeo& h = zinv.p.hg;
    const int L = h.N0, P = zinv.P;
    ht->ok = false;
    if (zinv.nt != kHermTmaNT || h.NHP % P != 0 || (L > 256 && L % 2 != 0)) return SPDBA_ERR_UNSUPPORTED;
    const void* f = nullptr;
    size_t smem = 0;
    spdba_status s = herm_tma_kernel(L, P, &f, &smem);
    if (s != SPDBA_OK) return s;
    const uint32_t zb = (uint32_t)(L <= 256 ? L : L / 2);
    const uint64_t dims[3] = {(uint64_t)h.N2, (uint64_t)h.N1, (uint64_t)h.N0};
    const uint64_t row = (uint64_t)h.N2 * 8, plane = (uint64_t)h.N1 * h.N2 * 8;
    const uint32_t box_a[3] = {(uint32_t)P, 1, zb}, box_b[3] = {(uint32_t)P + 2, 1, zb}, box_c[3] = {2, 1, zb};
    if ((s = tma_encode_3d(ht->map[0], c_hat, dims, row, plane, box_a)) != SPDBA_OK) return s;
    if ((s = tma_encode_3d(ht->map[1], c_hat, dims, row, plane, box_b)) != SPDBA_OK) return s;
    if ((s = tma_encode_3d(ht->map[2], c_hat, dims, row, plane, box_c)) != SPDBA_OK) return s;
    SPDBA_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, nsm = 0, dev = 0;
    SPDBA_CUDA(cudaGetDevice(&dev));
    SPDBA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SPDBA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kHermTmaNT, smem));
    if (per_sm < 1) return SPDBA_ERR_UNSUPPORTED;
    const long long ntiles = (zinv.p.O * zinv.p.I) / P;
    ht->func = f;
    ht->smem = smem;
    ht->grid = (long long)per_sm * nsm < ntiles ? (long long)per_sm * nsm : ntiles;
    ht->ok = true;
    return SPDBA_OK;
}

spdba_status launch_herm_inv_tma(const HermTma& ht, const Pass<float>& zinv, const void* in, void* out,
                                 unsigned long long* timeouts, cudaStream_t st) {
    PassParams<float> p = zinv.p;
    p.in = reinterpret_cast<const float2*>(in);
    p.out = reinterpret_cast<float2*>(out);
    long long spin = wait_limit();
    int stall = stall_waits();
    void* args[] = {(void*)&ht.map[0], (void*)&ht.map[1], (void*)&ht.map[2], &p, &timeouts, &spin, &stall};
    SPDBA_CUDA(cudaLaunchKernel(ht.func, dim3((unsigned)ht.grid), dim3(kHermTmaNT), args, ht.smem, st));
    return SPDBA_OK;
}

}  // namespace spdba
