// Block geometry and per-run device statistics, shared by every kernel family.
#pragma once
#include <stdint.h>

#include "../../include/spdba.h"

namespace spdba {

// Grid and block map padded to three axes (axis 0 slowest); unused leading
// axes have extent 1.
struct Geom {
    int ndim = 0;
    long long n[3] = {1, 1, 1};
    int b[3] = {1, 1, 1};
    // Half map (hx > 0): the blocks of the stored half kx = 0 .. N/2 of a real
    // field's spectrum, hx x-blocks of it (the last holding the column kx =
    // N/2), any x-blocks past them padding; neighbours in the omitted half are
    // conjugate counterparts (S1.2).  hx = 0: a full, periodic map.
    int hx = 0;
    long long nb[3] = {1, 1, 1};
    __host__ __device__ long long modes() const { return n[0] * n[1] * n[2]; }
    __host__ __device__ long long blocks() const { return nb[0] * nb[1] * nb[2]; }
    __host__ __device__ long long block_modes() const { return (long long)b[0] * b[1] * b[2]; }
    // A group stores several equal fields along the unused leading axis (or
    // axes): blocks [r*bpr, (r+1)*bpr) and modes [r*fmodes, (r+1)*fmodes)
    // belong to run r.  Neighbour relations never cross runs.
    __host__ __device__ long long bpr() const {
        return ndim == 3 ? nb[0] * nb[1] * nb[2] : ndim == 2 ? nb[1] * nb[2] : nb[2];
    }
    __host__ __device__ long long fmodes() const {
        return ndim == 3 ? n[0] * n[1] * n[2] : ndim == 2 ? n[1] * n[2] : n[2];
    }
    __host__ __device__ long long runs() const { return blocks() / bpr(); }
    // blocks of a run that hold modes (the padding x-blocks of a half map excluded)
    __host__ __device__ long long live_bpr() const { return hx > 0 ? bpr() / nb[2] * hx : bpr(); }
};
// Device statistics of one run (mirrors spdba_stats, accumulated on the device).
struct DevStats {
    double tau;
    double max_amp;
    double mass;
    double ratio_sum;
    unsigned long long n_active;
    unsigned long long n_transition;
    unsigned long long assessments;
    double list_modes;   // modes touched by list-driven updates (for traffic accounting)
    unsigned long long predictions;
    unsigned long long missed;
    double eps;                     // threshold coefficient in force (dynamic control moves it)
    unsigned long long ctl_nf;      // non-frozen blocks summed over the control interval's adaptive steps
    unsigned long long ctl_steps;   // adaptive steps in the control interval
    unsigned long long controls;    // control decisions made
    unsigned long long timeouts;    // bounded device waits that ran out (SPDBA_ERR_TIMEOUT)
};

}  // namespace spdba
