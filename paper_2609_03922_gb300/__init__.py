"""GB300 (sm_103a) implementation of sp-DBA, spectral dynamic block activation.

The compute path is libspdba.so (CUDA kernels + C ABI in include/spdba.h);
`paper_2609_03922_gb300.spdba` is its thin ctypes binding.
"""
