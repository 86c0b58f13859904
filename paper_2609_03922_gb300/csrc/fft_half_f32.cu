// Half-spectrum pass kernels of 3-D complex64 Cahn-Hilliard steps.
#include "fft_half.cuh"
#include "internal.h"
#include "kernel_table.h"

namespace spdba {

// pencils per tile of the z passes (row-major tiles), threads per CTA
template <int L> struct HalfTile;
template <> struct HalfTile<64> { static constexpr int P = 64; };
template <> struct HalfTile<128> { static constexpr int P = 32; };
template <> struct HalfTile<256> { static constexpr int P = 16; };
template <> struct HalfTile<384> { static constexpr int P = 8; };
template <> struct HalfTile<512> { static constexpr int P = 16; };
constexpr int kHalfNT = 256;
template <int L> static bool pick_z(int mode, KernelInfo* ki) {
    constexpr int P = HalfTile<L>::P, NT = kHalfNT;
    using C = cx_t<float>;
    ki->P = P;
    ki->NT = NT;
    ki->pipe = true;
    const int tile = LayoutB<L, P>::SIZE * (int)sizeof(C);
    switch (mode) {
        case PASS_HERM_INV:
            ki->func = (const void*)fft_herm_inv_kernel<float, L, P, NT>;
            ki->smem = 2 * tile + MirLay<L, P>::SIZE * (int)sizeof(C);
            return true;
        case PASS_MIRROR:
            ki->func = (const void*)fft_pass_pipe_kernel<float, L, P, NT, -1, PASS_MIRROR, true>;
            ki->smem = 2 * tile;
            return true;
        case PASS_UPD_HALF:
            ki->func = (const void*)fft_pass_pipe_kernel<float, L, P, NT, -1, PASS_UPD_HALF, true>;
            ki->smem = (upd_stages_chat<float, L>() ? 3 : 2) * tile;
            return true;
        default:
            return false;
    }
}

// pencils per tile and threads per CTA of the paired z forward pass (one
// butterfly per thread in the radix-16 stages; three tile buffers)
template <int L> struct PairTileP;
template <> struct PairTileP<64> { static constexpr int P = 16, NT = 128; };
template <> struct PairTileP<128> { static constexpr int P = 16, NT = 128; };
template <> struct PairTileP<256> { static constexpr int P = 8, NT = 128; };
template <int L> static bool pick_pair(KernelInfo* ki) {
    constexpr int P = PairTileP<L>::P, NT = PairTileP<L>::NT;
    ki->P = P;
    ki->NT = NT;
    ki->pipe = true;
    ki->func = (const void*)fft_pair_kernel<float, L, P, NT>;
    ki->smem = kPairBufs * LayoutBP<L, P>::SIZE * (int)sizeof(cx_t<float>);
    return true;
}

// real rows per tile of the x pass (two rows per transform pencil)
template <int N2> struct NlHalfRows { static constexpr int value = N2 <= 256 ? 4096 / N2 : 16; };

template <int N2> static bool pick_x(int nhp, KernelInfo* ki) {
    constexpr int P = NlHalfRows<N2>::value, NT = N2 <= 256 ? 128 : 256;
    ki->P = P;
    ki->NT = NT;
    ki->pipe = true;
    ki->func = (const void*)fft_nl_half_kernel<float, N2, P, NT>;
    ki->smem = (2 * P * nhp + LayoutA<N2, P / 2, true>::SIZE) * (int)sizeof(cx_t<float>);
    return true;
}

bool get_half_kernel(int64_t L, int mode, int nhp, KernelInfo* ki) {
    if (mode == PASS_NL_HALF) {   // L = N2, the full row length
        switch (L) {
            case 64: return pick_x<64>(nhp, ki);
            case 128: return pick_x<128>(nhp, ki);
            case 256: return pick_x<256>(nhp, ki);
            case 384: return pick_x<384>(nhp, ki);
            case 512: return pick_x<512>(nhp, ki);
            default: return false;
        }
    }
    if (mode == PASS_PAIR_MIRROR) {
        switch (L) {
            case 64: return pick_pair<64>(ki);
            case 128: return pick_pair<128>(ki);
            case 256: return pick_pair<256>(ki);
            default: return false;
        }
    }
    switch (L) {
        case 64: return pick_z<64>(mode, ki);
        case 128: return pick_z<128>(mode, ki);
        case 256: return pick_z<256>(mode, ki);
        case 384: return pick_z<384>(mode, ki);
        case 512: return pick_z<512>(mode, ki);
        default: return false;
    }
}

long long pair_tile_count(const Pass<float>& ps) {
    const HalfGeo& h = ps.p.hg;
    return (long long)h.N1 * (h.N2 / 2) / ps.P + h.N1 / ps.P;
}

spdba_status launch_pair_live_list(const Pass<float>& ps, int* list, int* count, cudaStream_t st) {
    const long long nt = pair_tile_count(ps);
    const unsigned grid = (unsigned)((nt + 7) / 8);   // a warp per tile, 8 per CTA
    SPDBA_CUDA(cudaMemsetAsync(count, 0, sizeof(int), st));
    switch (ps.P) {
        case 8: pair_live_list_kernel<float, 8><<<grid, 256, 0, st>>>(ps.p, list, count); break;
        case 16: pair_live_list_kernel<float, 16><<<grid, 256, 0, st>>>(ps.p, list, count); break;
        default: return SPDBA_ERR_UNSUPPORTED;
    }
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

}  // namespace spdba

namespace spdba {
// x frequencies 0 .. NHP-1 of the half array whose columns some paired z
// forward tile reads: column kx (kx <= N2/2) serves half pencils (ky, kx) for
// x frequencies kx and N2 - kx, so it is live when any block of block column
// kx / B2 or (N2 - kx) / B2 (over all kz, ky) is non-frozen; padding columns
// are never read.
__global__ void __launch_bounds__(1024) half_col_live_kernel(const uint8_t* __restrict__ states, int nrows, int nb2,
                                                             int B2, int N2, int NHP, uint8_t* __restrict__ col_live) {
    __shared__ uint8_t s_col[64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int bx = warp; bx < nb2; bx += 32) {
        // no early exit: the loads are independent, so several stay in flight
        unsigned live = 0;
#pragma unroll 8
        for (int r = lane; r < nrows; r += 32) live |= states[(long long)r * nb2 + bx];
        const unsigned any = __ballot_sync(0xffffffffu, live != 0);
        if (lane == 0) s_col[bx] = any != 0;
    }
    __syncthreads();
    for (int kx = threadIdx.x; kx < NHP; kx += blockDim.x) {
        uint8_t v = 0;
        if (kx <= N2 / 2) v = s_col[kx / B2] | (kx > 0 ? s_col[(N2 - kx) / B2] : (uint8_t)0);
        col_live[kx] = v;
    }
}

// Pencil liveness of the half-spectrum storage form under the half map's
// states: zlive[y * NHP + x] = some block of z pencil (y, x) is not FROZEN
// (the z forward's outputs are read only by the update of non-frozen blocks);
// xlive[x] = some z pencil of column x is live (the y forward's outputs in the
// other columns are read by no live z pencil).  xlive is zero on entry.
__global__ void __launch_bounds__(256) hs_live_kernel(const uint8_t* __restrict__ states, int nb0, int nb1, int nb2,
                                                      int B1, int B2, int N1, int NHP, uint8_t* __restrict__ zlive,
                                                      uint8_t* __restrict__ xlive) {
    const long long n = (long long)N1 * NHP;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / NHP), x = (int)(i - (long long)y * NHP);
        const long long b0 = (long long)(y / B1) * nb2 + x / B2;
        unsigned live = 0;
#pragma unroll 8
        for (int bz = 0; bz < nb0; ++bz) live |= states[(long long)bz * nb1 * nb2 + b0];
        zlive[i] = live != 0;
        if (live) xlive[x] = 1;
    }
}

spdba_status launch_hs_live(const Geom& g, const uint8_t* states, uint8_t* zlive, uint8_t* xlive, cudaStream_t st) {
    const long long n = g.n[1] * g.n[2];
    SPDBA_CUDA(cudaMemsetAsync(xlive, 0, (size_t)g.n[2], st));
    const long long grid = std::min<long long>((n + 255) / 256, 152 * 8);
    hs_live_kernel<<<(unsigned)grid, 256, 0, st>>>(states, (int)g.nb[0], (int)g.nb[1], (int)g.nb[2], g.b[1], g.b[2],
                                                   (int)g.n[1], (int)g.n[2], zlive, xlive);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

spdba_status launch_half_col_live(const Geom& g, const uint8_t* states, int N2, int NHP, uint8_t* col_live,
                                  cudaStream_t st) {
    if (g.nb[2] > 64) return fail(SPDBA_ERR_UNSUPPORTED, "more than 64 block columns");
    half_col_live_kernel<<<1, 1024, 0, st>>>(states, (int)(g.nb[0] * g.nb[1]), (int)g.nb[2], g.b[2], N2, NHP,
                                             col_live);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}
}  // namespace spdba
