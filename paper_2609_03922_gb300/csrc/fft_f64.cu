// FFT pass kernels, complex128 (FP64 arithmetic).
#define SPDBA_T double
#include "fft_kernels.inc"
