// FFT pass kernels, complex64 (FP32 arithmetic, FP64-computed twiddles).
#define SPDBA_T float
#include "fft_kernels.inc"
