// Hermitian half-spectrum passes of a 3-D Cahn-Hilliard step (complex64).
//
// c = Re(IFFT(c_hat)) equals the inverse transform of the Hermitian part
// h(k) = (c_hat(k) + conj(c_hat(-k))) / 2, and every intermediate of that
// inverse (and of the forward transform of the real g) is Hermitian along x
// once y and z are in real space.  So the transforms run on x frequencies
// 0 .. N2/2 only (the "half array", rows of NHP >= N2/2 + 1 entries):
//   z: inverse of h, from the full c_hat (PASS_HERM_INV, this file)
//   y: plain inverse pass on the half array
//   x: half spectrum -> real row -> g = c^3 - c -> half spectrum (PASS_NL_HALF)
//   y: plain forward pass on the half array
//   z: forward pass of the half array for every x frequency, the mirrored
//      ones from D(z, ky, kx) = conj(D(z, -ky, -kx)) (PASS_UPD_HALF with the
//      update, PASS_MIRROR as a plain store), in fft_core.cuh.
// The x rows use the standard length-N2/2 complex transform of a real row of
// N2 samples: even and odd samples as real and imaginary parts, with the
// split / merge twiddles exp(-+2 pi i k / N2).
#pragma once
#include "fft_core.cuh"

namespace spdba {

// ---------------------------------------------------------------- z inverse
// Tile: P consecutive pencils (ky, kx) of the half array (pencil index
// ky * NHP + kx), j = kz.  Element (p, j) is h(kz, ky, kx), formed from the
// direct element c_hat(kz, ky, kx) (buffer A) and the mirror element
// c_hat(-kz, -ky, -kx) (buffer B, loaded at index j).  Padding pencils
// (kx > N2/2) are zero.
template <typename T, int L, int P, int NT, class LY>
__device__ __forceinline__ void issue_herm(cx_t<T>* sm, const PassParams<T>& a, long long q0, bool mirror) {
    using C = cx_t<T>;
    const HalfGeo& h = a.hg;
    const int M = h.N2 >> 1;
    static_assert(NT % P == 0, "each thread keeps one pencil");
    const int p = (int)(threadIdx.x % P);
    const int q = (int)q0 + p;
    const int ky = (int)h.fd_NHP.div((uint32_t)q), kx = q - ky * h.NHP;
    const long long plane = (long long)h.N1 * h.N2;
    if (kx > M) {
        for (int j = (int)(threadIdx.x / P); j < L; j += NT / P) sm[LY::idx(p, j)] = mk<C>((T)0, (T)0);
        return;
    }
    if (!mirror) {
        const C* src = a.in + ((long long)ky * h.N2 + kx);
        // pencil pairs (p, p + 1) of one row: one 16-byte copy by the even pencil
        const bool pair = (p & 1) == 0 && kx + 1 <= M && (kx & 1) == 0;
        const bool covered = (p & 1) == 1 && kx >= 1 && ((kx - 1) & 1) == 0;   // copied by pencil p - 1
        if (pair) {
#pragma unroll 4
            for (int j = (int)(threadIdx.x / P); j < L; j += NT / P) cp_async16(sm + LY::idx(p, j), src + j * plane);
        } else if (!covered) {
#pragma unroll 4
            for (int j = (int)(threadIdx.x / P); j < L; j += NT / P) cp_async8(sm + LY::idx(p, j), src + j * plane);
        }
    } else {
        const int my = ky == 0 ? 0 : h.N1 - ky, mx = kx == 0 ? 0 : h.N2 - kx;
        const C* src = a.in + ((long long)my * h.N2 + mx);
#pragma unroll 4
        for (int j = (int)(threadIdx.x / P); j < L; j += NT / P)
            cp_async8(sm + LY::idx(p, j), src + (j == 0 ? 0 : L - j) * plane);
    }
}

template <typename T, int L, int P, int NT>
__global__ void __launch_bounds__(NT, 2) fft_herm_inv_kernel(PassParams<T> a) {
    using C = cx_t<T>;
    using LY = LayoutB<L, P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smA0 = reinterpret_cast<C*>(smem_raw);
    C* smA1 = smA0 + LY::SIZE;
    C* smB = smA1 + LY::SIZE;
    const long long ntiles = (a.O * a.I) / P;
    long long t = blockIdx.x;
    if (t < ntiles) {
        issue_herm<T, L, P, NT, LY>(smA0, a, t * P, false);
        issue_herm<T, L, P, NT, LY>(smB, a, t * P, true);
    }
    cp_async_commit();
    int buf = 0;
    while (t < ntiles) {
        const long long tn = t + gridDim.x;
        if (tn < ntiles) issue_herm<T, L, P, NT, LY>(buf ? smA0 : smA1, a, tn * P, false);
        cp_async_commit();
        cp_async_wait<1>();   // the direct and mirror tiles of t have landed
        __syncthreads();
        C* sm = buf ? smA1 : smA0;
        for (int e = threadIdx.x; e < P * L; e += NT) {
            const C x = sm[e], y = smB[e];
            sm[e] = mk<C>((T)0.5 * (x.x + y.x), (T)0.5 * (x.y - y.y));
        }
        __syncthreads();
        // the mirror tile of the next tile streams in during this tile's transform
        if (tn < ntiles) issue_herm<T, L, P, NT, LY>(smB, a, tn * P, true);
        cp_async_commit();
        PlainOut<T, L> out(a, t * P);
        run_stages_out<T, L, P, NT, +1, LY>(sm, a.tw, out);
        __syncthreads();
        buf ^= 1;
        t = tn;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------- x rows
// Real-row split (inverse): Z[k] = (X[k] + conj X[M-k]) + i w^k (X[k] - conj X[M-k]),
// w = exp(2 pi i / N2), k < M = N2/2; the length-M inverse of Z holds the real row's
// even and odd samples as real and imaginary parts.
// Merge (forward): with U the length-M transform of u = g_even + i g_odd,
// G[k] = (U[k] + conj U[-k]) / 2 - i w^-k (U[k] - conj U[-k]) / 2 for k < M,
// G[M] = Re U[0] - Im U[0].
template <typename T> struct ChNlPairMid {
    T scale, msum;
    __device__ __forceinline__ cx_t<T> operator()(int, int, cx_t<T> x) {
        const T c0 = x.x * scale, c1 = x.y * scale;
        msum += c0 + c1;
        return mk<cx_t<T>>(c0 * c0 * c0 - c0, c1 * c1 * c1 - c1);
    }
};

// Natural-order store of the forward transform's outputs to shared memory.
template <typename T, int L, class LY> struct SmemOut {
    using C = cx_t<T>;
    static constexpr bool SYNC = true;
    C* sm;
    __device__ __forceinline__ void pre() {}
    __device__ __forceinline__ void begin(int, int, int) {}
    template <int R> __device__ __forceinline__ void emit(int, int p, int j, C (&v)[R]) {
#pragma unroll
        for (int r = 0; r < R; ++r) sm[LY::idx(p, j + r * (L / R))] = v[r];
    }
};

// L = M = N2 / 2 (transform length); rows of NHP entries, P rows per tile.
// a.tw: stage twiddles of M; a.tw4: exp(-2 pi i m / N2), m < N2.
template <typename T, int L, int P, int NT>
__global__ void __launch_bounds__(NT, 2) fft_nl_half_kernel(PassParams<T> a) {
    using C = cx_t<T>;
    using LY = LayoutA<L, P, true>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NHP = a.hg.NHP;
    C* rows0 = reinterpret_cast<C*>(smem_raw);
    C* rows1 = rows0 + P * NHP;
    C* tb = rows1 + P * NHP;                      // transform buffer (layout A)
    const long long nrows = a.O * a.I;
    const long long ntiles = nrows / P;
    const int units = P * NHP / 2;                // 16-byte units per tile
    auto issue = [&](C* dst, long long q0) {
        const C* src = a.in + q0 * NHP;
        for (int u = threadIdx.x; u < units; u += NT) cp_async16(dst + 2 * u, src + 2 * u);
    };
    long long t = blockIdx.x;
    if (t < ntiles) issue(rows0, t * P);
    cp_async_commit();
    int buf = 0;
    while (t < ntiles) {
        const long long tn = t + gridDim.x;
        if (tn < ntiles) issue(buf ? rows0 : rows1, tn * P);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        C* rw = buf ? rows1 : rows0;
        const long long q0 = t * P;
        // split into the length-M inverse input
        for (int e = threadIdx.x; e < P * L; e += NT) {
            const int p = e / L, k = e - p * L;
            const C x = rw[p * NHP + k];
            C y = rw[p * NHP + (L - k)];
            y.y = -y.y;
            C w = __ldg(a.tw4 + k);
            w.y = -w.y;                           // exp(+2 pi i k / N2)
            const C d = cmul(w, csub(x, y));
            tb[LY::idx(p, k)] = mk<C>(x.x + y.x - d.y, x.y + y.y + d.x);
        }
        __syncthreads();
        // inverse, c = Re / N and g = c^3 - c on both samples of each pair, forward
        ChNlPairMid<T> mid{a.nl_scale, (T)0};
        SmemOut<T, L, LY> so{tb};
        transform_pair<T, L, P, NT, +1, -1, LY>(tb, a.tw, mid, so);
        __syncthreads();
        // merge into the half spectrum of g (padding entries zero)
        for (int e = threadIdx.x; e < P * NHP; e += NT) {
            const int p = e / NHP, k = e - p * NHP;
            C g = mk<C>((T)0, (T)0);
            if (k < L) {
                const C u1 = tb[LY::idx(p, k)];
                C u2 = tb[LY::idx(p, k == 0 ? 0 : L - k)];
                u2.y = -u2.y;
                const C ev = mk<C>((T)0.5 * (u1.x + u2.x), (T)0.5 * (u1.y + u2.y));
                const C od = mk<C>((T)0.5 * (u1.y - u2.y), (T)-0.5 * (u1.x - u2.x));   // (u1 - u2) / (2i)
                const C w = __ldg(a.tw4 + k);                                             // exp(-2 pi i k / N2)
                const C wo = cmul(w, od);
                g = mk<C>(ev.x + wo.x, ev.y + wo.y);
            } else if (k == L) {
                const C u0 = tb[LY::idx(p, 0)];
                g = mk<C>(u0.x - u0.y, (T)0);
            }
            rw[e] = g;
        }
        __syncthreads();
        {
            C* dst = a.out + q0 * NHP;
            for (int u = threadIdx.x; u < units; u += NT)
                *reinterpret_cast<float4*>(dst + 2 * u) = *reinterpret_cast<const float4*>(rw + 2 * u);
        }
        if (a.mass != nullptr) {
            const double ms = warp_sum((double)mid.msum);
            if ((threadIdx.x & 31) == 0) atomicAdd(a.mass + (q0 / a.mass_ppr) * a.mass_stride, ms);
        }
        __syncthreads();
        buf ^= 1;
        t = tn;
    }
    cp_async_wait<0>();
}

}  // namespace spdba
