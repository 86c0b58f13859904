// Hermitian half-spectrum passes of a 3-D Cahn-Hilliard step (complex64).
//
// c = Re(IFFT(c_hat)) equals the inverse transform of the Hermitian part
// h(k) = (c_hat(k) + conj(c_hat(-k))) / 2, and every intermediate of that
// inverse (and of the forward transform of the real g) is Hermitian along x
// once y and z are in real space.  So the transforms run on x frequencies
// 0 .. N2/2 only (the "half array", rows of NHP >= N2/2 + 1 entries):
//   z: inverse of h, from the full c_hat (PASS_HERM_INV, this file)
//   y: plain inverse pass on the half array
//   x: half spectrum -> real row -> g = c^3 - c -> half spectrum, two rows per
//      complex transform (PASS_NL_HALF)
//   y: plain forward pass on the half array
//   z: forward pass of the half array for every x frequency, the mirrored
//      ones from D(z, ky, kx) = conj(D(z, -ky, -kx)): with the update
//      (PASS_UPD_HALF, fft_core.cuh), or stored for the separate update, one
//      transform per half pencil for kx and N2 - kx (PASS_PAIR_MIRROR, this
//      file; PASS_MIRROR in fft_core.cuh where the paired tiles do not fit).
#pragma once
#include "fft_core.cuh"

namespace spdba {

// ---------------------------------------------------------------- z inverse
// Tile: P consecutive pencils (ky, kx) of the half array (pencil index
// ky * NHP + kx), j = kz.  Element (p, j) is h(kz, ky, kx), formed from the
// direct element c_hat(kz, ky, kx) (buffer A) and the mirror element
// c_hat(-kz, -ky, -kx) (buffer B, loaded at index j).  Padding pencils
// (kx > N2/2) are zero.
// Layout of the mirror tile: pencil p at slot P - p of rows of P + 2 slots.
// Mirror columns N2 - kx descend as p rises, so an odd pencil p whose kx is odd
// copies the 16-byte unit (N2 - kx - 1, N2 - kx) = (pencil p + 1, pencil p)
// into slots (P - p - 1, P - p); pencil 0 copies its own column and a spare one
// into slots (P, P + 1).  Slot 0 (reached from p = P - 1) and slot P + 1 hold
// spares only; every other pencil copies its own column.
template <int L, int P> struct MirLay {
    static_assert(P % 2 == 0, "16-byte units need an even pencil count");
    static constexpr int SIZE = L * (P + 2);
    static __device__ __forceinline__ int idx(int p, int j) { return j * (P + 2) + (P - p); }
};

template <typename T, int L, int P, int NT, class LY>
__device__ __forceinline__ void issue_herm(cx_t<T>* sm, const PassParams<T>& a, long long q0) {
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
    const C* src = a.in + ((long long)ky * h.N2 + kx);
    // pencil pairs (p, p + 1), p even, of one row: one 16-byte copy by the even pencil
    const bool pair = (p & 1) == 0 && kx + 1 <= M && (kx & 1) == 0;
    const bool covered = (p & 1) == 1 && kx >= 1 && ((kx - 1) & 1) == 0;   // copied by pencil p - 1
    if (pair) {
#pragma unroll 4
        for (int j = (int)(threadIdx.x / P); j < L; j += NT / P) cp_async16(sm + LY::idx(p, j), src + j * plane);
    } else if (!covered) {
#pragma unroll 4
        for (int j = (int)(threadIdx.x / P); j < L; j += NT / P) cp_async8(sm + LY::idx(p, j), src + j * plane);
    }
}

// Mirror tile: element (p, j) = c_hat(-j, -ky, -kx) of pencil p = (ky, kx).
// A tile may cross an x row, so pairing is decided per pencil: a 16-byte copy
// needs an odd p (aligned slot) and an odd kx (aligned column), and pencil
// p + 1 must be the next pencil of the same row and not padding, or absent.
template <typename T, int L, int P, int NT>
__device__ __forceinline__ void issue_herm_mirror(cx_t<T>* smb, const PassParams<T>& a, long long q0) {
    using C = cx_t<T>;
    using ML = MirLay<L, P>;
    const HalfGeo& h = a.hg;
    const int M = h.N2 >> 1;
    const int p = (int)(threadIdx.x % P);
    const int q = (int)q0 + p;
    const int ky = (int)h.fd_NHP.div((uint32_t)q), kx = q - ky * h.NHP;
    const long long plane = (long long)h.N1 * h.N2;
    if (kx > M) {   // never reached by a neighbour's copy: that needs kx <= M here
        for (int j = (int)(threadIdx.x / P); j < L; j += NT / P) smb[ML::idx(p, j)] = mk<C>((T)0, (T)0);
        return;
    }
    const int c = kx == 0 ? 0 : h.N2 - kx;   // this pencil's mirror column
    const bool odd_p = (p & 1) != 0, odd_k = (kx & 1) != 0;
    const C* src = a.in + (long long)(ky == 0 ? 0 : h.N1 - ky) * h.N2;
    if (odd_p && odd_k && (p + 1 == P || kx + 1 <= M)) {
#pragma unroll 4
        for (int j = (int)(threadIdx.x / P); j < L; j += NT / P)
            cp_async16(smb + ML::idx(p + 1, j), src + (c - 1) + (j == 0 ? 0 : L - j) * plane);
    } else if (p == 0 && (c & 1) == 0) {
#pragma unroll 4
        for (int j = (int)(threadIdx.x / P); j < L; j += NT / P)
            cp_async16(smb + ML::idx(0, j), src + c + (j == 0 ? 0 : L - j) * plane);
    } else if (!odd_p && p >= 2 && !odd_k && kx >= 2) {
        return;   // copied by pencil p - 1 (odd p - 1, odd kx - 1, kx <= M)
    } else {
#pragma unroll 4
        for (int j = (int)(threadIdx.x / P); j < L; j += NT / P)
            cp_async8(smb + ML::idx(p, j), src + c + (j == 0 ? 0 : L - j) * plane);
    }
}

// (direct + conj(mirror)) / 2 of element m of pencil p
template <typename T, int L, int P, class LY> struct HermIn {
    const cx_t<T>* a;
    const cx_t<T>* b;
    __device__ __forceinline__ cx_t<T> operator()(int p, int m) const {
        const cx_t<T> x = a[LY::idx(p, m)], y = b[MirLay<L, P>::idx(p, m)];
        return mk<cx_t<T>>((T)0.5 * (x.x + y.x), (T)0.5 * (x.y - y.y));
    }
};

template <typename T, int L, int P, int NT>
__global__ void __launch_bounds__(NT, 2) fft_herm_inv_kernel(PassParams<T> a) {
    using C = cx_t<T>;
    using LY = LayoutB<L, P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smA0 = reinterpret_cast<C*>(smem_raw);
    C* smA1 = smA0 + LY::SIZE;
    C* smB = smA1 + LY::SIZE;
    // complex64 passes up to 512 points keep the twiddle table in shared memory
    constexpr bool STW = sizeof(T) == 4 && L <= 512;
    __shared__ C s_tw[STW ? L : 1];
    if constexpr (STW)
        for (int j = threadIdx.x; j < L; j += NT) s_tw[j] = a.tw[j];   // visible after the loop's first barrier
    const C* const tw = STW ? s_tw : a.tw;
    const long long ntiles = (a.O * a.I) / P;
    long long t = blockIdx.x;
    if (t < ntiles) {
        issue_herm<T, L, P, NT, LY>(smA0, a, t * P);
        issue_herm_mirror<T, L, P, NT>(smB, a, t * P);
    }
    cp_async_commit();
    int buf = 0;
    while (t < ntiles) {
        const long long tn = t + gridDim.x;
        if (tn < ntiles) issue_herm<T, L, P, NT, LY>(buf ? smA0 : smA1, a, tn * P);
        cp_async_commit();
        cp_async_wait<1>();   // the direct and mirror tiles of t have landed
        __syncthreads();
        C* sm = buf ? smA1 : smA0;
        // the first stage reads (direct + conj(mirror)) / 2; the stage's barrier
        // between its reads and writes frees the mirror buffer
        PlainOut<T, L> out(a, t * P);
        HermIn<T, L, P, LY> in{sm, smB};
        stockham_stage_in<T, L, P, NT, +1, 1, radix_at<L>(0), LY>(sm, tw, in);
        // the mirror tile of the next tile streams in during the rest of the transform
        if (tn < ntiles) issue_herm_mirror<T, L, P, NT>(smB, a, tn * P);
        cp_async_commit();
        run_stage_range<T, L, P, NT, +1, LY, 1, NSTAGES<L>::value - 1>(sm, tw);
        stockham_stage_out<T, L, P, NT, +1, ns_at<L>(NSTAGES<L>::value - 1), radix_at<L>(NSTAGES<L>::value - 1), LY>(
            sm, tw, out);
        __syncthreads();
        buf ^= 1;
        t = tn;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------- x rows
// Two real rows r1, r2 (half spectra X1, X2, x frequencies 0 .. N2/2) share one
// complex transform of the full length N2: Z[k] = X1[k] + i X2[k], extended to
// k > N2/2 by Z[k] = conj(X1[N2-k]) + i conj(X2[N2-k]), whose inverse is
// x1 + i x2.  The nonlinearity acts on real and imaginary parts, and the
// forward transform W of g1 + i g2 separates into
// G1[k] = (W[k] + conj W[-k]) / 2, G2[k] = (W[k] - conj W[-k]) / (2i), k <= N2/2.
template <typename T> struct ChNlPairMid {
    T scale, msum;
    __device__ __forceinline__ cx_t<T> operator()(int, int, cx_t<T> x) {
        const T c0 = mul_rn(x.x, scale), c1 = mul_rn(x.y, scale);
        msum += c0 + c1;
        return mk<cx_t<T>>(fma_rn(mul_rn(c0, c0), c0, -c0), fma_rn(mul_rn(c1, c1), c1, -c1));
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

// Packed input element k of transform pencil pp: X1[k] + i X2[k] from rows
// 2 pp and 2 pp + 1, extended past N2/2 by conjugate symmetry (with r2c, the
// imaginary parts at k = 0 and N2/2 dropped).
template <typename T, int L> struct PairPackIn {
    const cx_t<T>* rw;
    int nhp;
    bool r2c;
    __device__ __forceinline__ cx_t<T> operator()(int pp, int k) const {
        const cx_t<T>* r1 = rw + (2 * pp) * nhp;
        const cx_t<T>* r2 = r1 + nhp;
        cx_t<T> x1, x2;
        if (k <= L / 2) {
            x1 = r1[k];
            x2 = r2[k];
            if (r2c && (k == 0 || k == L / 2)) x1.y = x2.y = (T)0;
        } else {
            x1 = r1[L - k];
            x2 = r2[L - k];
            x1.y = -x1.y;
            x2.y = -x2.y;
        }
        return mk<cx_t<T>>(x1.x - x2.y, x1.y + x2.x);
    }
};

// L = N2 (transform length), P real rows per tile (P / 2 transform pencils),
// rows of NHP entries.  a.tw: stage twiddles of N2.
template <typename T, int L, int P, int NT>
__global__ void __launch_bounds__(NT, L == 384 ? 1 : 512 / NT) fft_nl_half_kernel(PassParams<T> a) {
    using C = cx_t<T>;
    constexpr int PP = P / 2;
    constexpr int M = L / 2;
    using LY = LayoutA<L, PP, true>;
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
        // inverse (its first stage packing the row pairs), c = Re / N and
        // g = c^3 - c on both rows, forward
        ChNlPairMid<T> mid{a.nl_scale, (T)0};
        SmemOut<T, L, LY> so{tb};
        PairPackIn<T, L> in{rw, NHP, a.hg.r2c != 0};
        transform_pair_in<T, L, PP, NT, +1, -1, LY>(tb, a.tw, in, mid, so);
        __syncthreads();
        // separate the two rows' half spectra (padding entries zero), straight
        // to the output rows: one loop over all (pair, entry) items, so that
        // every trip keeps all threads busy (consecutive threads, consecutive
        // entries of a row)
        {
            C* dst = a.out + q0 * NHP;
            for (int it = threadIdx.x; it < PP * NHP; it += NT) {
                const int pp = (int)a.hg.fd_NHP.div((uint32_t)it);
                const int k = it - pp * NHP;
                C g1 = mk<C>((T)0, (T)0), g2 = g1;
                if (k <= M) {
                    const C w = tb[LY::idx(pp, k)];
                    C v = tb[LY::idx(pp, k == 0 ? 0 : L - k)];
                    v.y = -v.y;                                               // conj W[-k]
                    g1 = mk<C>((T)0.5 * (w.x + v.x), (T)0.5 * (w.y + v.y));
                    g2 = mk<C>((T)0.5 * (w.y - v.y), (T)-0.5 * (w.x - v.x));  // (w - v) / (2i)
                }
                dst[(2 * pp) * NHP + k] = g1;
                dst[(2 * pp + 1) * NHP + k] = g2;
            }
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

// ---------------------------------------------------------------- z forward, paired
// The forward z-transform of half pencil (ky, kx) gives D(kz, ky, kx) and, by
// D(z, -ky, -kx) = conj(D(z, ky, kx)), also D(-kz, -ky, N2 - kx) =
// conj(D(kz, ky, kx)): one transform serves both x frequencies kx and N2 - kx
// (PASS_PAIR_MIRROR: the full z-transform stored for the separate update).
// Tiles of P pencils kx = x0 .. x0 + P - 1 (x0 < N2/2) of one half row ky emit
// both; the column kx = N2/2 (its own mirror) runs as tiles of P pencils along
// y after them.  Requires (N2/2) % P == 0, N1 % P == 0 and an even NHP.

// Row-major tile (element j of pencil p at j * P + p); with P < 16 every 16
// rows are followed by P pad slots, so that the rows j R + r that a first
// stage's lanes write fall on alternating halves of the banks.
template <int L, int P> struct LayoutBP {
    static constexpr int PAD = P < 16 ? P : 0;
    static constexpr int SIZE = P * L + PAD * (L / 16);
    static constexpr bool PMAP = true;
    static __device__ __forceinline__ int idx(int p, int j) { return j * P + p + PAD * (j >> 4); }
};

// Half-array tile of tile t: paired tiles as 16-byte pencil pairs of one row,
// column tiles (kx = N2/2, P rows of y) element by element.
template <typename T, int L, int P, int NT, class LY>
__device__ __forceinline__ void issue_pair_half(cx_t<T>* sm, const PassParams<T>& a, int t, int ntm) {
    const HalfGeo& h = a.hg;
    const int M = h.N2 >> 1;
    const long long zs = (long long)h.N1 * h.NHP;
    if (t < ntm) {
        const int q0 = t * P;
        const int ky = (int)h.fd_M.div((uint32_t)q0), x0 = q0 - ky * M;
        const cx_t<T>* base = a.in + ((long long)ky * h.NHP + x0);
        constexpr int UNITS = P * L / 2;
#pragma unroll 4
        for (int w = threadIdx.x; w < UNITS; w += NT) {
            const int j = w / (P / 2), pp = (w % (P / 2)) * 2;
            cp_async16(sm + LY::idx(pp, j), base + (j * zs + pp));
        }
    } else {
        const int ky0 = (t - ntm) * P;
        const cx_t<T>* base = a.in + ((long long)ky0 * h.NHP + M);
        constexpr int UNITS = P * L;
#pragma unroll 4
        for (int w = threadIdx.x; w < UNITS; w += NT) {
            const int j = w / P, p = w % P;
            cp_async8(sm + LY::idx(p, j), base + (j * zs + (long long)p * h.NHP));
        }
    }
}

// Blocks of a paired tile (32-bit; every thread derives the same values):
// x-blocks of the direct columns x0 .. x0 + P - 1 in row ky and of the mirror
// columns N2 - x0 - P + 1 .. N2 - x0 (column N2 excluded: x0 = 0 has no mirror
// of column 0) in row my.
struct PairBlocks {
    int bxd0, nbxd, bxm0, nbxm;
    long long boffd, boffm;   // block ids of (z block row 0, first x-block) in rows ky and my
    int bstride;              // block id step per z block row
};
template <typename T, int P>
__device__ __forceinline__ PairBlocks pair_blocks(const PassParams<T>& a, int t) {
    const HalfGeo& h = a.hg;
    const CHFuse<T>& f = a.fu;
    const Geom& g = f.g;
    const int q0 = t * P;
    const int ky = (int)h.fd_M.div((uint32_t)q0), x0 = q0 - ky * (h.N2 >> 1);
    const int my = ky == 0 ? 0 : h.N1 - ky;
    PairBlocks u;
    u.bxd0 = (int)f.fd_b2.div((uint32_t)x0);
    u.nbxd = (int)f.fd_b2.div((uint32_t)(x0 + P - 1)) - u.bxd0 + 1;
    const int mlo = h.N2 - x0 - (P - 1), mhi = x0 == 0 ? h.N2 - 1 : h.N2 - x0;
    u.bxm0 = (int)f.fd_b2.div((uint32_t)mlo);
    u.nbxm = (int)f.fd_b2.div((uint32_t)mhi) - u.bxm0 + 1;
    u.boffd = (long long)f.fd_b1.div((uint32_t)ky) * g.nb[2] + u.bxd0;
    u.boffm = (long long)f.fd_b1.div((uint32_t)my) * g.nb[2] + u.bxm0;
    u.bstride = (int)(g.nb[1] * g.nb[2]);
    return u;
}

// With block states (masked): a paired tile is live when any block of its
// direct or mirror columns is not FROZEN (warp-uniform); column tiles always.
template <typename T, int P>
__device__ __forceinline__ bool pair_live(const PassParams<T>& a, bool masked, int t, int ntm) {
    if (!masked || t >= ntm) return true;
    const PairBlocks u = pair_blocks<T, P>(a, t);
    const int npass = (int)a.fu.g.nb[0];
    const uint8_t* st = a.fu.states;
    bool live = false;
    for (int bp = threadIdx.x & 31; bp < npass && !live; bp += 32) {
        const long long r = (long long)bp * u.bstride;
        for (int bx = 0; bx < u.nbxd; ++bx) live |= st[u.boffd + r + bx] != SPDBA_FROZEN;
        for (int bx = 0; bx < u.nbxm; ++bx) live |= st[u.boffm + r + bx] != SPDBA_FROZEN;
    }
    return __any_sync(0xffffffffu, live);
}
// Live tiles of the paired z forward under the block states, in any order:
// one warp per tile, appended to list[]; *count must be zero on entry.  Run
// once per state setting, so that the pass deals equal shares of live tiles
// to its CTAs (liveness clusters in the spectrum).
template <typename T, int P>
__global__ void __launch_bounds__(256) pair_live_list_kernel(PassParams<T> a, int* list, int* count) {
    const int ntm = a.hg.N1 * (a.hg.N2 >> 1) / P, nt = ntm + a.hg.N1 / P;
    const int t = (int)(blockIdx.x * 8 + (threadIdx.x >> 5));
    if (t >= nt) return;   // warp-uniform
    if (pair_live<T, P>(a, true, t, ntm) && (threadIdx.x & 31) == 0) list[atomicAdd(count, 1)] = t;
}

// Per-tile state tables (masked): tabd[bp * nbxd + bx], tabm[bp * nbxm + bx]
// for z block row bp.  Visible after the next barrier.
template <typename T, int NT>
__device__ __forceinline__ void pair_tables(uint8_t* tabd, uint8_t* tabm, const PassParams<T>& a,
                                            const PairBlocks& u) {
    const int npass = (int)a.fu.g.nb[0];
    const uint8_t* st = a.fu.states;
    for (int k = threadIdx.x; k < npass * u.nbxd; k += NT) {
        const int bp = k / u.nbxd;
        tabd[k] = st[u.boffd + (long long)bp * u.bstride + (k - bp * u.nbxd)];
    }
    for (int k = threadIdx.x; k < npass * u.nbxm; k += NT) {
        const int bp = k / u.nbxm;
        tabm[k] = st[u.boffm + (long long)bp * u.bstride + (k - bp * u.nbxm)];
    }
}

// Outputs of a paired tile's last stage stored as the full z-transform:
// D(kz, ky, x0 + p) and conj(D) at (-kz, -ky, N2 - x0 - p); masked, only the
// modes of non-FROZEN blocks (the staged update reads no others).
template <typename T, int L, int P, int R> struct PairPlainOut {
    using C = cx_t<T>;
    static constexpr bool SYNC = false;
    static constexpr int NS = L / R;
    C* pd;
    C* pm;
    bool has_m, masked;
    int osJ;
    const uint8_t* tabd;
    const uint8_t* tabm;
    int nbxd, nbxm, bxsd, bxsm;
    FastDiv fd_bp;
    // z block rows of the outputs without a division per output: with NS a
    // multiple of the z block edge bz, output m = j + r NS lies in row
    // j / bz + r NS / bz and its mirror -m in row L / bz - r NS / bz - ceil(j / bz)
    bool aligned;
    int nsb, lb, bz;
    __device__ __forceinline__ PairPlainOut(const PassParams<T>& a, int t, bool masked_, const uint8_t* td,
                                            const uint8_t* tm)
        : masked(masked_), tabd(td), tabm(tm) {
        const HalfGeo& h = a.hg;
        const int q0 = t * P;
        const int ky = (int)h.fd_M.div((uint32_t)q0), x0 = q0 - ky * (h.N2 >> 1);
        const int my = ky == 0 ? 0 : h.N1 - ky;
        const int xd = x0 + (int)(threadIdx.x % P);
        has_m = xd != 0;   // column 0 is its own mirror
        const int xm = has_m ? h.N2 - xd : 0;
        pd = a.out + ((long long)ky * h.N2 + xd);
        pm = a.out + ((long long)my * h.N2 + xm);
        osJ = h.N1 * h.N2;
        if (masked) {
            const PairBlocks u = pair_blocks<T, P>(a, t);
            const CHFuse<T>& f = a.fu;
            nbxd = u.nbxd;
            nbxm = u.nbxm;
            bxsd = (int)f.fd_b2.div((uint32_t)xd) - u.bxd0;
            bxsm = (int)f.fd_b2.div((uint32_t)xm) - u.bxm0;
            fd_bp = f.fd_bp;
            bz = (int)f.fd_bp.d;
            aligned = NS % bz == 0;
            nsb = NS / bz;
            lb = L / bz;
        }
    }
    __device__ __forceinline__ void pre() {}
    __device__ __forceinline__ void begin(int, int, int) {}
    __device__ __forceinline__ void emit(int, int, int j, C (&v)[R]) {
        if (masked && aligned) {
            const int bj = (int)fd_bp.div((uint32_t)j), cj = (int)fd_bp.div((uint32_t)(j + bz - 1));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int m = j + r * NS;
                if (tabd[(bj + r * nsb) * nbxd + bxsd] != SPDBA_FROZEN) pd[m * osJ] = v[r];
                if (has_m) {
                    const int mz = m == 0 ? 0 : L - m;
                    const int bm = m == 0 ? 0 : lb - r * nsb - cj;
                    if (tabm[bm * nbxm + bxsm] != SPDBA_FROZEN) pm[mz * osJ] = mk<C>(v[r].x, -v[r].y);
                }
            }
            return;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = j + r * NS;
            if (!masked || tabd[(int)fd_bp.div((uint32_t)m) * nbxd + bxsd] != SPDBA_FROZEN) pd[m * osJ] = v[r];
            if (has_m) {
                const int mz = m == 0 ? 0 : L - m;
                if (!masked || tabm[(int)fd_bp.div((uint32_t)mz) * nbxm + bxsm] != SPDBA_FROZEN)
                    pm[mz * osJ] = mk<C>(v[r].x, -v[r].y);
            }
        }
    }
};

// Column kx = N2/2 (tile of pencils ky0 .. ky0 + P - 1, transform in shared
// memory): plain store of every element.
template <typename T, int L, int P, int NT, class LY>
__device__ __forceinline__ void pair_column(const cx_t<T>* sm, const PassParams<T>& a, int ky0) {
    const HalfGeo& h = a.hg;
    const int M = h.N2 >> 1;
    const long long plane = (long long)h.N1 * h.N2;
    for (int w = threadIdx.x; w < P * L; w += NT) {
        const int j = w / P, p = w % P;
        a.out[(long long)j * plane + (long long)(ky0 + p) * h.N2 + M] = sm[LY::idx(p, j)];
    }
}

// Persistent CTAs walk the tiles t = blockIdx.x + k gridDim.x (masked: the
// live ones) with a three-deep cp.async pipeline: the tile two steps ahead
// streams in while one is transformed (a tile's own compute is too short to
// hide one load).
constexpr int kPairBufs = 3;
template <typename T, int L, int P, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) fft_pair_kernel(PassParams<T> a) {
    using C = cx_t<T>;
    using LY = LayoutBP<L, P>;
    static_assert(NT % P == 0 && NT % (P / 2) == 0, "each thread keeps one pencil");
    static_assert(Radices_last<L>::value != 3, "the last stage emits directly");
    static_assert(kPairBufs == 3, "the loop keeps two tiles in flight");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // complex64 passes up to 512 points keep the twiddle table in shared memory
    constexpr bool STW = sizeof(T) == 4 && L <= 512;
    __shared__ C s_tw[STW ? L : 1];
    if constexpr (STW)
        for (int j = threadIdx.x; j < L; j += NT) s_tw[j] = a.tw[j];   // visible after the loop's first barrier
    const C* const tw = STW ? s_tw : a.tw;
    __shared__ uint8_t s_tab[2 * kPairTable];
    C* const smb = reinterpret_cast<C*>(smem_raw);
    const int ntm = a.hg.N1 * (a.hg.N2 >> 1) / P, nt = ntm + a.hg.N1 / P;
    const bool masked = a.fu.states != nullptr && !a.fu.dense;
    // this CTA's k-th tile: every tile in turn, or (masked) every live one from the list
    const int G = (int)gridDim.x;
    const int nlist = masked ? *a.live_count : 0;
    auto tile_at = [&](int k) -> int {
        const int i = (int)blockIdx.x + k * G;
        if (masked) return i < nlist ? a.live_tiles[i] : nt;
        return i < nt ? i : nt;
    };
    int t = tile_at(0);
    if (t < nt) issue_pair_half<T, L, P, NT, LY>(smb, a, t, ntm);
    cp_async_commit();
    int t1 = tile_at(1);
    if (t1 < nt) issue_pair_half<T, L, P, NT, LY>(smb + LY::SIZE, a, t1, ntm);
    cp_async_commit();
    int tn = tile_at(2);   // the tile to issue at the next iteration's start
    int slot = 0;
    for (int k = 3; t < nt; ++k) {
        const int t2 = tn;
        tn = tile_at(k);   // in flight during this tile's work
        const int s2 = slot == 0 ? 2 : slot - 1;   // (slot + 2) mod 3: freed by the previous tile
        if (t2 < nt) issue_pair_half<T, L, P, NT, LY>(smb + s2 * LY::SIZE, a, t2, ntm);
        cp_async_commit();
        if (masked && t < ntm) pair_tables<T, NT>(s_tab, s_tab + kPairTable, a, pair_blocks<T, P>(a, t));
        cp_async_wait<2>();   // tile t (the oldest pending group) has landed
        __syncthreads();
        C* sm = smb + slot * LY::SIZE;
        if (t < ntm) {
            PairPlainOut<T, L, P, Radices_last<L>::value> out(a, t, masked, s_tab, s_tab + kPairTable);
            run_stages_out<T, L, P, NT, -1, LY>(sm, tw, out);
        } else {
            run_stages<T, L, P, NT, -1, LY>(sm, tw);
            pair_column<T, L, P, NT, LY>(sm, a, (t - ntm) * P);
        }
        __syncthreads();   // buffer `slot` and the tables are free again
        t = t1;
        t1 = t2;
        slot = slot == 2 ? 0 : slot + 1;
    }
    cp_async_wait<0>();
}

}  // namespace spdba
