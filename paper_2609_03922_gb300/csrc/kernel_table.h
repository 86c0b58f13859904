// Lookup of compiled pass kernels by (length, direction, mode, orientation).
#pragma once
#include <stdint.h>

namespace spdba {
struct KernelInfo {
    const void* func = nullptr;
    int P = 0, NT = 0, smem = 0;
    bool pipe = false;  // persistent, double-buffered kernel: grid = resident CTAs
};
// generic: the pencil count is not a multiple of the tile (simple kernel only)
template <typename T>
bool get_pass_kernel(int64_t L, int sign, int mode, bool loadp, bool storep, bool generic, KernelInfo* ki);
// complex64 half-spectrum passes (PASS_HERM_INV, PASS_NL_HALF, PASS_MIRROR,
// PASS_UPD_HALF); nhp = half row length (PASS_NL_HALF shared memory)
bool get_half_kernel(int64_t L, int mode, int nhp, KernelInfo* ki);
// pencils per tile of the pass kernels of length L (0 if none)
template <typename T> int pass_tile_pencils(int64_t L);
}  // namespace spdba
