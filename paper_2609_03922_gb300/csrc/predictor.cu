// Learned block-activity predictor (no counterpart in the paper): a small 3-D
// convolutional network over the block map that predicts which blocks will be
// non-frozen over the next K steps, so that most exact activity scans can be
// skipped (the exact scan stays as a periodic judge).
//
//   a1 = conv(x, W1) + b1, h1 = relu(a1)    2 -> 8 channels, 3x3x3, periodic
//   a2 = conv(h1, W2) + b2, h2 = relu(a2)   8 -> 16
//   a3 = conv(h2, W3) + b3, h3 = relu(a3)   16 -> 8
//   z = h3 . wh + bh, p = sigmoid(z);  loss = mean BCE(p, y)
//
// Convolutions are implicit GEMMs on the BF16 tensor cores (mma.sync m16n8k16,
// FP32 accumulate): forward and input-gradient use M = voxels, N = output
// channels, K = 27 x input channels; the weight gradient uses M = output
// channels, N = 27 x input channels, K = voxels.  Activations are channels-
// last, stored as BF16 between layers; master weights and Adam state are FP32.
// The GEMM shapes are tiny (N = 8 or 16), so these kernels are latency-bound.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "blocks.h"

namespace spdba {

typedef __nv_bfloat16 bf16;

constexpr int NPARAM = 8 * 27 * 2 + 8 + 16 * 27 * 8 + 16 + 8 * 27 * 16 + 8 + 8 + 1;
// offsets of the flat parameter vector: W1, b1, W2, b2, W3, b3, wh, bh
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + 8 * 27 * 2, OFF_W2 = OFF_B1 + 8, OFF_B2 = OFF_W2 + 16 * 27 * 8,
              OFF_W3 = OFF_B2 + 16, OFF_B3 = OFF_W3 + 8 * 27 * 16, OFF_WH = OFF_B3 + 8, OFF_BH = OFF_WH + 8;
static_assert(OFF_BH + 1 == NPARAM, "parameter layout");

__host__ __device__ constexpr int kpad(int k) { return (k + 15) / 16 * 16; }

struct MapDims {
    int D, H, W;
    long long V;  // voxels per map
};

__device__ __forceinline__ long long neighbor(const MapDims& m, long long v, int tap) {
    const long long per = v / m.V, r = v - per * m.V;
    int z = (int)(r / ((long long)m.H * m.W)), y = (int)((r / m.W) % m.H), x = (int)(r % m.W);
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    z = (z + dz + m.D) % m.D;
    y = (y + dy + m.H) % m.H;
    x = (x + dx + m.W) % m.W;
    return per * m.V + ((long long)z * m.H + y) * m.W + x;
}

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ------------------------------------------------------------------ conv (forward / input gradient)
enum ConvMode { CONV_FWD = 0, CONV_DGRAD = 1 };

// A tile of 16 voxels per warp.  Wt: [COUT][kpad(27 CIN)] bf16 (zero padded).
// FWD: out_pre = acc + bias (FP32), out = bf16(relu(out_pre)).
// DGRAD: out = bf16(acc * (mask_pre > 0)).
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(128) conv_kernel(MapDims m, long long nvox, const bf16* __restrict__ X,
                                                   const bf16* __restrict__ Wt, const float* __restrict__ bias,
                                                   float* __restrict__ out_pre, const float* __restrict__ mask_pre,
                                                   bf16* __restrict__ out) {
    constexpr int K = 27 * CIN, KP = kpad(K), NT = COUT / 8;
    __shared__ __align__(16) bf16 sW[COUT * KP];
    for (int i = threadIdx.x; i < COUT * KP; i += blockDim.x) sW[i] = Wt[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long ntile = (nvox + 15) / 16;
    for (long long tile = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < ntile;
         tile += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long v0 = tile * 16 + g, v1 = v0 + 8;
        const bool ok0 = v0 < nvox, ok1 = v1 < nvox;
        float acc[NT][4];
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll 1
        for (int k0 = 0; k0 < KP; k0 += 16) {
            // A: rows v0/v1, columns k0 + 2t (+8); a column pair shares one tap (CIN even)
            const int ka = k0 + 2 * t, kb = ka + 8;
            uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
            if (ka < K) {
                const int tap = ka / CIN, ci = ka % CIN;
                if (ok0) a0 = ld_pair(X + neighbor(m, v0, tap) * CIN + ci);
                if (ok1) a1 = ld_pair(X + neighbor(m, v1, tap) * CIN + ci);
            }
            if (kb < K) {
                const int tap = kb / CIN, ci = kb % CIN;
                if (ok0) a2 = ld_pair(X + neighbor(m, v0, tap) * CIN + ci);
                if (ok1) a3 = ld_pair(X + neighbor(m, v1, tap) * CIN + ci);
            }
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const bf16* wr = sW + (n * 8 + g) * KP;
                uint32_t b0 = ld_pair(wr + ka), b1 = ld_pair(wr + kb);
                mma16816(acc[n], a0, a1, a2, a3, b0, b1);
            }
        }
        // D: rows v0 / v1, columns co = n*8 + 2t, +1
#pragma unroll
        for (int n = 0; n < NT; ++n) {
            const int co = n * 8 + 2 * t;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long v = h ? v1 : v0;
                if (!(h ? ok1 : ok0)) continue;
                float x0 = acc[n][2 * h], x1 = acc[n][2 * h + 1];
                if (MODE == CONV_FWD) {
                    x0 += bias[co];
                    x1 += bias[co + 1];
                    out_pre[v * COUT + co] = x0;
                    out_pre[v * COUT + co + 1] = x1;
                    x0 = fmaxf(x0, 0.f);
                    x1 = fmaxf(x1, 0.f);
                } else {
                    if (!(mask_pre[v * COUT + co] > 0.f)) x0 = 0.f;
                    if (!(mask_pre[v * COUT + co + 1] > 0.f)) x1 = 0.f;
                }
                *reinterpret_cast<uint32_t*>(out + v * COUT + co) =
                    pack2(__float2bfloat16_rn(x0), __float2bfloat16_rn(x1));
            }
        }
    }
}

// ------------------------------------------------------------------ weight gradient
// dW[co][k] += sum_v dA[v][co] X[neighbour(v, tap(k))][ci(k)], k < 27 CIN, on
// the tensor cores: A = dA^T (rows co, padded to 16), B = im2col(X) (rows =
// voxels, columns = 8 k), reduction over 16 voxels per mma.  Each warp owns
// TPW column tiles and a slice of the voxels, then adds its partial into dW.
template <int CIN, int COUT, int TPW>
__global__ void __launch_bounds__(128) wgrad_kernel(MapDims m, long long nvox, const bf16* __restrict__ dA,
                                                    const bf16* __restrict__ X, float* __restrict__ dW,
                                                    float* __restrict__ dbias, long long vox_per_warp) {
    constexpr int K = 27 * CIN, NTILES = (K + 7) / 8;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int tile_groups = (NTILES + TPW - 1) / TPW;
    const int tg = (int)(warp % tile_groups);
    const long long slice = warp / tile_groups;
    const long long vbeg = slice * vox_per_warp;
    if (vbeg >= nvox) return;
    const long long vend = vbeg + vox_per_warp < nvox ? vbeg + vox_per_warp : nvox;
    float acc[TPW][4];
#pragma unroll
    for (int n = 0; n < TPW; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    float bsum0 = 0.f, bsum1 = 0.f;   // bias gradient of channel g (and g + 8)
    const bf16 zero = __float2bfloat16_rn(0.f);
    for (long long vb = vbeg; vb < vend; vb += 16) {
        // A fragment: A[co][vv] = dA[vb + vv][co]; rows g (and g + 8 for COUT = 16)
        const long long va = vb + 2 * t, vc = va + 8;
        auto dA_at = [&](long long v, int co) -> bf16 {
            return (v < vend && co < COUT) ? dA[v * COUT + co] : zero;
        };
        uint32_t a0 = pack2(dA_at(va, g), dA_at(va + 1, g));
        uint32_t a1 = pack2(dA_at(va, g + 8), dA_at(va + 1, g + 8));
        uint32_t a2 = pack2(dA_at(vc, g), dA_at(vc + 1, g));
        uint32_t a3 = pack2(dA_at(vc, g + 8), dA_at(vc + 1, g + 8));
        if (tg == 0) {
            bsum0 += __bfloat162float(dA_at(va, g)) + __bfloat162float(dA_at(va + 1, g)) +
                     __bfloat162float(dA_at(vc, g)) + __bfloat162float(dA_at(vc + 1, g));
            bsum1 += __bfloat162float(dA_at(va, g + 8)) + __bfloat162float(dA_at(va + 1, g + 8)) +
                     __bfloat162float(dA_at(vc, g + 8)) + __bfloat162float(dA_at(vc + 1, g + 8));
        }
#pragma unroll
        for (int n = 0; n < TPW; ++n) {
            const int kcol = (tg * TPW + n) * 8 + g;   // this lane's B column
            uint32_t b0 = 0, b1 = 0;
            if (kcol < K) {
                const int tap = kcol / CIN, ci = kcol % CIN;
                auto x_at = [&](long long v) -> bf16 { return v < vend ? X[neighbor(m, v, tap) * CIN + ci] : zero; };
                b0 = pack2(x_at(va), x_at(va + 1));
                b1 = pack2(x_at(vc), x_at(vc + 1));
            }
            mma16816(acc[n], a0, a1, a2, a3, b0, b1);
        }
    }
#pragma unroll
    for (int n = 0; n < TPW; ++n) {
        const int kc = (tg * TPW + n) * 8 + 2 * t;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int co = g + 8 * h;
            if (co >= COUT) continue;
            if (kc < K) atomicAdd(&dW[co * K + kc], acc[n][2 * h]);
            if (kc + 1 < K) atomicAdd(&dW[co * K + kc + 1], acc[n][2 * h + 1]);
        }
    }
    if (tg == 0) {
        // lanes with equal g hold partial sums of the same channel
        bsum0 += __shfl_xor_sync(0xffffffffu, bsum0, 1);
        bsum0 += __shfl_xor_sync(0xffffffffu, bsum0, 2);
        bsum1 += __shfl_xor_sync(0xffffffffu, bsum1, 1);
        bsum1 += __shfl_xor_sync(0xffffffffu, bsum1, 2);
        if (t == 0) {
            atomicAdd(&dbias[g], bsum0);
            if (g + 8 < COUT) atomicAdd(&dbias[g + 8], bsum1);
        }
    }
}

// ------------------------------------------------------------------ head, loss and its gradient
// z = h3 . wh + bh, p = sigmoid(z).  With labels: loss += BCE / n, dz = (p - y) / n,
// dwh += dz h3, dbh += dz, da3 = bf16(dz wh * (a3 > 0)).
__global__ void head_kernel(long long nvox, const bf16* __restrict__ h3, const float* __restrict__ a3,
                            const float* __restrict__ params, float* __restrict__ prob,
                            const float* __restrict__ labels, double inv_n, bf16* __restrict__ da3,
                            float* __restrict__ grads, double* __restrict__ loss) {
    const float* wh = params + OFF_WH;
    const float bh = params[OFF_BH];
    float gw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float gb = 0.f;
    double ls = 0.0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        float hv[8];
        float z = bh;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            hv[c] = __bfloat162float(h3[v * 8 + c]);
            z = fmaf(hv[c], wh[c], z);
        }
        const float p = 1.f / (1.f + expf(-z));
        if (prob) prob[v] = p;
        if (labels) {
            const float y = labels[v];
            const float eps = 1e-12f;
            ls -= (double)(y * logf(p + eps) + (1.f - y) * logf(1.f - p + eps));
            const float dz = (float)((double)(p - y) * inv_n);
            gb += dz;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                gw[c] = fmaf(dz, hv[c], gw[c]);
                const float d = a3[v * 8 + c] > 0.f ? dz * wh[c] : 0.f;
                da3[v * 8 + c] = __float2bfloat16_rn(d);
            }
        }
    }
    if (!labels) return;
#pragma unroll
    for (int c = 0; c < 8; ++c) gw[c] = warp_sumf(gw[c]);
    gb = warp_sumf(gb);
    ls = warp_sum(ls);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) atomicAdd(&grads[OFF_WH + c], gw[c]);
        atomicAdd(&grads[OFF_BH], gb);
        atomicAdd(loss, ls * inv_n);
    }
}

// ------------------------------------------------------------------ weights, features, Adam
// FP32 master -> BF16 forward layout Wt[co][k] (k = tap*CIN + ci, zero padded) and
// input-gradient layout Wd[ci][k'] (k' = tap'*COUT + co, tap' = 26 - tap).
__global__ void convert_weights_kernel(const float* __restrict__ P, int off, int cin, int cout, bf16* __restrict__ Wt,
                                       bf16* __restrict__ Wd) {
    const int K = 27 * cin, KP = kpad(K), Kd = 27 * cout, KPd = kpad(Kd);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cout * KP; i += gridDim.x * blockDim.x) {
        int co = i / KP, k = i % KP;
        Wt[i] = __float2bfloat16_rn(k < K ? P[off + co * K + k] : 0.f);
    }
    if (!Wd) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cin * KPd; i += gridDim.x * blockDim.x) {
        int ci = i / KPd, k = i % KPd;
        float w = 0.f;
        if (k < Kd) {
            int tapd = k / cout, co = k % cout;
            int tap = 26 - tapd;
            w = P[off + co * K + tap * cin + ci];
        }
        Wd[i] = __float2bfloat16_rn(w);
    }
}

// x[v][0] = clamp(log10(A_B / tau) / 8, -1, 1), x[v][1] = 1 if the block is not FROZEN.
__global__ void features_kernel(long long V, int nmaps, const double* __restrict__ maxsq, const double* __restrict__ tau,
                                const uint8_t* __restrict__ states, bf16* __restrict__ x) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V * nmaps;
         i += (long long)gridDim.x * blockDim.x) {
        const long long mp = i / V;
        const double a = sqrt(maxsq[i]);
        const double tv = tau[mp];
        double f = (a > 0 && tv > 0) ? log10(a / tv) / 8.0 : (a > 0 ? 1.0 : -1.0);
        f = f < -1.0 ? -1.0 : (f > 1.0 ? 1.0 : f);
        x[2 * i] = __float2bfloat16_rn((float)f);
        x[2 * i + 1] = __float2bfloat16_rn(states[i] != 0 ? 1.f : 0.f);
    }
}

__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                            float* __restrict__ Vv, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float g = G[i];
        float m = b1 * M[i] + (1.f - b1) * g;
        float v = b2 * Vv[i] + (1.f - b2) * g * g;
        M[i] = m;
        Vv[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

__global__ void prob_to_measure_kernel(const float* __restrict__ p, double* __restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)p[i];
}

}  // namespace spdba

using namespace spdba;

struct spdba_predictor {
    MapDims m;
    int max_batch;
    float *P, *G, *M, *Vv, *prob, *a1, *a2, *a3, *labels;
    bf16 *W1t, *W2t, *W3t, *W2d, *W3d, *h1, *h2, *h3, *da1, *da2, *da3;
    double* loss;
    long long adam_t;
    std::vector<void*> allocs;
    template <typename Q> spdba_status alloc(Q** p, size_t bytes) {
        void* q = nullptr;
        cudaError_t e = spdba::dev_alloc(&q, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "device allocation (predictor buffer)");
        allocs.push_back(q);
        *p = (Q*)q;
        return SPDBA_OK;
    }
};

namespace spdba {

static unsigned grid_of(long long n, int nt) {
    long long g = (n + nt - 1) / nt;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)(g < 1 ? 1 : g);
}

static spdba_status refresh_weights(spdba_predictor* pr, cudaStream_t st) {
    convert_weights_kernel<<<32, 256, 0, st>>>(pr->P, OFF_W1, 2, 8, pr->W1t, nullptr);
    convert_weights_kernel<<<32, 256, 0, st>>>(pr->P, OFF_W2, 8, 16, pr->W2t, pr->W2d);
    convert_weights_kernel<<<32, 256, 0, st>>>(pr->P, OFF_W3, 16, 8, pr->W3t, pr->W3d);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

static spdba_status forward(spdba_predictor* pr, const bf16* x, long long nvox, cudaStream_t st) {
    const unsigned g = grid_of((nvox + 15) / 16 * 32, 128);
    conv_kernel<2, 8, CONV_FWD><<<g, 128, 0, st>>>(pr->m, nvox, x, pr->W1t, pr->P + OFF_B1, pr->a1, nullptr, pr->h1);
    conv_kernel<8, 16, CONV_FWD><<<g, 128, 0, st>>>(pr->m, nvox, pr->h1, pr->W2t, pr->P + OFF_B2, pr->a2, nullptr, pr->h2);
    conv_kernel<16, 8, CONV_FWD><<<g, 128, 0, st>>>(pr->m, nvox, pr->h2, pr->W3t, pr->P + OFF_B3, pr->a3, nullptr, pr->h3);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

template <int CIN, int COUT>
static void wgrad(spdba_predictor* pr, long long nvox, const bf16* dA, const bf16* X, int offW, int offB, cudaStream_t st) {
    constexpr int TPW = 4;
    constexpr int NTILES = (27 * CIN + 7) / 8;
    const int tile_groups = (NTILES + TPW - 1) / TPW;
    const long long vpw = 1024;
    const long long slices = (nvox + vpw - 1) / vpw;
    const long long warps = slices * tile_groups;
    wgrad_kernel<CIN, COUT, TPW><<<(unsigned)((warps * 32 + 127) / 128), 128, 0, st>>>(pr->m, nvox, dA, X, pr->G + offW,
                                                                                      pr->G + offB, vpw);
}

static spdba_status backward(spdba_predictor* pr, const bf16* x, const float* labels, long long nvox, cudaStream_t st) {
    SPDBA_CUDA(cudaMemsetAsync(pr->G, 0, sizeof(float) * NPARAM, st));
    SPDBA_CUDA(cudaMemsetAsync(pr->loss, 0, sizeof(double), st));
    head_kernel<<<grid_of(nvox, 256), 256, 0, st>>>(nvox, pr->h3, pr->a3, pr->P, pr->prob, labels, 1.0 / (double)nvox,
                                                    pr->da3, pr->G, pr->loss);
    const unsigned g = grid_of((nvox + 15) / 16 * 32, 128);
    wgrad<16, 8>(pr, nvox, pr->da3, pr->h2, OFF_W3, OFF_B3, st);
    conv_kernel<8, 16, CONV_DGRAD><<<g, 128, 0, st>>>(pr->m, nvox, pr->da3, pr->W3d, nullptr, nullptr, pr->a2, pr->da2);
    wgrad<8, 16>(pr, nvox, pr->da2, pr->h1, OFF_W2, OFF_B2, st);
    conv_kernel<16, 8, CONV_DGRAD><<<g, 128, 0, st>>>(pr->m, nvox, pr->da2, pr->W2d, nullptr, nullptr, pr->a1, pr->da1);
    wgrad<2, 8>(pr, nvox, pr->da1, x, OFF_W1, OFF_B1, st);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

}  // namespace spdba

// ------------------------------------------------------------------ C ABI
extern "C" int64_t spdba_predictor_num_params(void) { return NPARAM; }

extern "C" void spdba_predictor_destroy(spdba_predictor* pr) {
    if (!pr) return;
    cudaDeviceSynchronize();
    for (void* p : pr->allocs) spdba::dev_free(p);
    delete pr;
}

extern "C" spdba_status spdba_predictor_create(spdba_predictor** out, int32_t nd, int32_t nh, int32_t nw,
                                               int32_t max_batch, const float* init_params) {
    if (!out || nd < 3 || nh < 3 || nw < 3 || max_batch < 1 || !init_params)
        return fail(SPDBA_ERR_ARG, "spdba_predictor_create: bad arguments");
    spdba_predictor* pr = new spdba_predictor();
    pr->m = MapDims{nd, nh, nw, (long long)nd * nh * nw};
    pr->max_batch = max_batch;
    pr->adam_t = 0;
    const long long nv = pr->m.V * max_batch;
    spdba_status s = SPDBA_OK;
#define A(ptr, bytes) \
    if (s == SPDBA_OK) s = pr->alloc(&pr->ptr, bytes)
    A(P, sizeof(float) * NPARAM);
    A(G, sizeof(float) * NPARAM);
    A(M, sizeof(float) * NPARAM);
    A(Vv, sizeof(float) * NPARAM);
    A(prob, sizeof(float) * nv);
    A(labels, sizeof(float) * nv);
    A(a1, sizeof(float) * nv * 8);
    A(a2, sizeof(float) * nv * 16);
    A(a3, sizeof(float) * nv * 8);
    A(W1t, sizeof(bf16) * 8 * kpad(54));
    A(W2t, sizeof(bf16) * 16 * kpad(216));
    A(W3t, sizeof(bf16) * 8 * kpad(432));
    A(W2d, sizeof(bf16) * 8 * kpad(27 * 16));
    A(W3d, sizeof(bf16) * 16 * kpad(27 * 8));
    A(h1, sizeof(bf16) * nv * 8);
    A(h2, sizeof(bf16) * nv * 16);
    A(h3, sizeof(bf16) * nv * 8);
    A(da1, sizeof(bf16) * nv * 8);
    A(da2, sizeof(bf16) * nv * 16);
    A(da3, sizeof(bf16) * nv * 8);
    A(loss, sizeof(double));
#undef A
    if (s == SPDBA_OK) {
        cudaError_t e = cudaMemcpy(pr->P, init_params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(pr->M, 0, sizeof(float) * NPARAM);
        if (e == cudaSuccess) e = cudaMemset(pr->Vv, 0, sizeof(float) * NPARAM);
        if (e != cudaSuccess) s = cuda_fail(e, "predictor init");
    }
    if (s == SPDBA_OK) s = refresh_weights(pr, 0);
    if (s == SPDBA_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) s = cuda_fail(e, "predictor init");
    }
    if (s != SPDBA_OK) {
        spdba_predictor_destroy(pr);
        return s;
    }
    *out = pr;
    return SPDBA_OK;
}

extern "C" spdba_status spdba_predictor_get_params(spdba_predictor* pr, float* host_out) {
    if (!pr || !host_out) return fail(SPDBA_ERR_ARG, "spdba_predictor_get_params: NULL");
    SPDBA_CUDA(cudaMemcpy(host_out, pr->P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    return SPDBA_OK;
}

extern "C" spdba_status spdba_predictor_set_params(spdba_predictor* pr, const float* host_in) {
    if (!pr || !host_in) return fail(SPDBA_ERR_ARG, "spdba_predictor_set_params: NULL");
    SPDBA_CUDA(cudaMemcpy(pr->P, host_in, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
    spdba_status s = refresh_weights(pr, 0);
    if (s != SPDBA_OK) return s;
    SPDBA_CUDA(cudaDeviceSynchronize());
    return SPDBA_OK;
}

extern "C" spdba_status spdba_predictor_features(spdba_predictor* pr, const double* maxsq, const double* tau,
                                                 const uint8_t* states, int32_t nmaps, void* x_bf16, void* stream) {
    if (!pr || !maxsq || !tau || !states || !x_bf16 || nmaps < 1 || nmaps > pr->max_batch)
        return fail(SPDBA_ERR_ARG, "spdba_predictor_features: bad arguments");
    features_kernel<<<grid_of(pr->m.V * nmaps, 256), 256, 0, (cudaStream_t)stream>>>(pr->m.V, nmaps, maxsq, tau, states,
                                                                                      (bf16*)x_bf16);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

extern "C" spdba_status spdba_predictor_forward(spdba_predictor* pr, const void* x_bf16, int32_t nmaps, float* prob,
                                                void* stream) {
    if (!pr || !x_bf16 || !prob || nmaps < 1 || nmaps > pr->max_batch)
        return fail(SPDBA_ERR_ARG, "spdba_predictor_forward: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const long long nvox = pr->m.V * nmaps;
    spdba_status s = forward(pr, (const bf16*)x_bf16, nvox, st);
    if (s != SPDBA_OK) return s;
    head_kernel<<<grid_of(nvox, 256), 256, 0, st>>>(nvox, pr->h3, pr->a3, pr->P, prob, nullptr, 0.0, nullptr, nullptr,
                                                    nullptr);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

extern "C" spdba_status spdba_predictor_gradients(spdba_predictor* pr, const void* x_bf16, const float* labels,
                                                  int32_t nmaps, double* loss_out, float* grads_host) {
    if (!pr || !x_bf16 || !labels || nmaps < 1 || nmaps > pr->max_batch)
        return fail(SPDBA_ERR_ARG, "spdba_predictor_gradients: bad arguments");
    const long long nvox = pr->m.V * nmaps;
    spdba_status s = forward(pr, (const bf16*)x_bf16, nvox, 0);
    if (s == SPDBA_OK) s = backward(pr, (const bf16*)x_bf16, labels, nvox, 0);
    if (s != SPDBA_OK) return s;
    SPDBA_CUDA(cudaDeviceSynchronize());
    if (loss_out) SPDBA_CUDA(cudaMemcpy(loss_out, pr->loss, sizeof(double), cudaMemcpyDeviceToHost));
    if (grads_host) SPDBA_CUDA(cudaMemcpy(grads_host, pr->G, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    return SPDBA_OK;
}

extern "C" spdba_status spdba_predictor_train_step(spdba_predictor* pr, const void* x_bf16, const float* labels,
                                                   int32_t nmaps, float lr, double* loss_out, void* stream) {
    if (!pr || !x_bf16 || !labels || nmaps < 1 || nmaps > pr->max_batch || !(lr > 0))
        return fail(SPDBA_ERR_ARG, "spdba_predictor_train_step: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const long long nvox = pr->m.V * nmaps;
    spdba_status s = forward(pr, (const bf16*)x_bf16, nvox, st);
    if (s == SPDBA_OK) s = backward(pr, (const bf16*)x_bf16, labels, nvox, st);
    if (s != SPDBA_OK) return s;
    pr->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)pr->adam_t), c2 = 1.f - powf(b2, (float)pr->adam_t);
    adam_kernel<<<grid_of(NPARAM, 256), 256, 0, st>>>(pr->P, pr->G, pr->M, pr->Vv, NPARAM, lr, b1, b2, 1e-8f, c1, c2);
    SPDBA_CUDA(cudaGetLastError());
    if ((s = refresh_weights(pr, st)) != SPDBA_OK) return s;
    if (loss_out) {
        SPDBA_CUDA(cudaMemcpyAsync(loss_out, pr->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        SPDBA_CUDA(cudaStreamSynchronize(st));
    }
    return SPDBA_OK;
}

// Predicted states: measure = p (as FP64) for the classifier, tau = prob_threshold.
spdba_status spdba_predictor_states_internal(spdba_predictor* pr, const double* maxsq, const double* tau,
                                             uint8_t* states, int32_t nmaps, void* x_scratch, double* measure_out,
                                             cudaStream_t st) {
    spdba_status s = spdba_predictor_features(pr, maxsq, tau, states, nmaps, x_scratch, st);
    if (s != SPDBA_OK) return s;
    if ((s = spdba_predictor_forward(pr, x_scratch, nmaps, pr->prob, st)) != SPDBA_OK) return s;
    const long long n = pr->m.V * nmaps;
    prob_to_measure_kernel<<<grid_of(n, 256), 256, 0, st>>>(pr->prob, measure_out, n);
    SPDBA_CUDA(cudaGetLastError());
    return SPDBA_OK;
}

bool spdba_predictor_map_matches(const spdba_predictor* pr, long long nd, long long nh, long long nw) {
    return pr && pr->m.D == nd && pr->m.H == nh && pr->m.W == nw;
}
