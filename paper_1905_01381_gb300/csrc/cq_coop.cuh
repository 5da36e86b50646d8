// Warp-cooperative ERI + J/K kernel driven by generated instruction tables
// (gen_coop.py).  One warp evaluates one contracted shell quartet:
//   1. lanes compute the per-primitive-quartet coefficients (prefactor,
//      Boys values, PA, QC, W-P, W-Q, exponent ratios) of up to 32 primitive
//      quartets in parallel, into shared memory;
//   2. for each primitive quartet the lanes walk the vertical-recurrence
//      table level by level, 32 independent nodes at a time, with values in a
//      per-warp shared-memory buffer, and add the [e0|f0] targets to
//      accumulators spread over the lanes' registers;
//   3. the horizontal-recurrence table turns the contracted [e0|f0] into the
//      (ab|cd) block in shared memory;
//   4. digestion is output-stationary: every lane owns whole elements of the
//      six J'/K' blocks of the quartet (a full contraction over the other two
//      indices), so no cross-lane reduction is needed before the adds.
#pragma once
#include "cq_jk.cuh"

namespace cq {

constexpr int NQC_COOP = 21;
constexpr int COOP_WARPS = 2;
constexpr int COOP_THREADS = 32 * COOP_WARPS;
constexpr int COOP_NCOEF = 26;
constexpr int COOP_MAXACC = 31;   // ceil(961 / 32)

struct CoopClass {
    int la, lb, lc, ld, L, nacc, N, nslots, nvg, nhg;
    const int4* vgrp;
    const int4* vdesc;
    const int4* hgrp;
    const int4* hdesc;
    const unsigned short* tgt;
};

// per-class slot counts for shared-memory sizing on the host
struct CoopSize {
    int nslots, nacc, N;
    int vslots, hslots;   // slots of the vertical and of the horizontal recurrence
};

// Slots of a warp's region in the cooperative kernel: the coefficient and
// Boys buffers (32 primitive quartets) followed by the vertical recurrence's
// slots; the horizontal recurrence and the digestion, which need neither
// buffer, reuse the whole region.
constexpr int COOP_BUF_SLOTS = 32 * COOP_NCOEF + 32 * (LTOT_MAX + 1);
__host__ __device__ constexpr int coop_region_slots(int vslots, int hslots)
{
    return COOP_BUF_SLOTS + vslots > hslots ? COOP_BUF_SLOTS + vslots : hslots;
}

// bytes of a warp: region, density blocks, AB and CD
template <typename R>
__host__ __device__ constexpr size_t coop_warp_bytes(int region_slots)
{
    return (size_t)(region_slots + 6 * 36 + 8) * sizeof(R);
}

}  // namespace cq
