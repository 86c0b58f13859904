// NLS split-step kernels, complex128.
#define SPDBA_T double
#include "nls_kernels.inc"
