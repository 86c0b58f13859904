// NLS split-step kernels: arguments and launchers.
#pragma once
#include "internal.h"

namespace spdba {

// Linear half-step factor H(w) as a pair hi + lo whose sum carries FP64
// accuracy (lo = 0 for the FP64 path), so that the per-step FP32 rounding of
// H does not accumulate into a systematic phase drift.
template <typename T> struct HPair {
    cx_t<T> hi, lo;
};

template <typename T> struct NLSArgs {
    cx_t<T>* S;                 // spectra of `batch` signals of n samples
    const HPair<T>* H;          // n entries: natural order (short), H(k1 + n1 m) at k1 * 512 + m (long)
    const uint8_t* states;      // batch * nblk
    const uint8_t* chi;
    const T* taper;             // B entries
    const cx_t<T>* tw;          // stage twiddles of the pass length
    const cx_t<T>* tw4;         // long signals: exp(-2 pi i a b / n) at a * 512 + b, a < n1, b < 512
    long long n, n1;            // n = n1 * 512 for long signals
    long long batch;
    int B, nblk;                // block edge (bins) and blocks per signal
    FastDiv fd_B;               // division by B (short signals)
    int mb_shift;               // long signals: log2(512 / nblk), element m of a row is in block m >> mb_shift
    int dense;                  // 1: every bin ACTIVE (Regular)
    T gamma_h, inv_n;
    double* power;              // per-signal FP64 sum |E|^2 accumulators (strided) or null
    int power_stride;
    int do_fwd, do_close, do_open, do_inv, do_kerr;
};

// Launch shapes of the three NLS kernels for one group, fixed at plan creation
// (function attributes and occupancy are queried there, never during a step).
struct NLSLaunch {
    long long small_grid = 0, row_grid = 0, col_grid = 0;
    int small_smem = 0, row_smem = 0, col_smem = 0;
};
template <typename T> spdba_status nls_prepare(long long n, long long n1, long long batch, NLSLaunch* out);
template <typename T> spdba_status nls_small_step(const NLSArgs<T>& a, const NLSLaunch& l, cudaStream_t st);
template <typename T> spdba_status nls_row_pass(const NLSArgs<T>& a, const NLSLaunch& l, cudaStream_t st);
template <typename T> spdba_status nls_col_pass(const NLSArgs<T>& a, const NLSLaunch& l, cudaStream_t st);
// tw2[a * 512 + b] = tw4[a * b] for a < n / 512, b < 512.
template <typename T> spdba_status nls_twiddle2(const cx_t<T>* tw4, cx_t<T>* tw2, long long n, cudaStream_t st);
template <typename T>
spdba_status nls_permute(const cx_t<T>* in, cx_t<T>* out, long long n, long long n1, long long batch, int to_natural,
                         cudaStream_t st);

}  // namespace spdba
