// NLS split-step kernels, complex64.
#define SPDBA_T float
#include "nls_kernels.inc"
