// Launcher of the warp-cooperative ERI + J/K kernel; the instruction tables
// (coop_tables.cuh, written by gen_coop.py) live in this translation unit.
#include "cq_internal.h"
#include "cq_coop.cuh"
#include "coop_tables.cuh"
#include "cq_coop_kernel.cuh"

namespace cq {

template <typename R>
static void launch_coop_t(const JKArgs& a, int qc, cudaStream_t s)
{
    static int attr_done = 0;
    const int nslots = COOP_SIZES[qc].nslots;
    const size_t bytes = (size_t)COOP_WARPS * coop_warp_bytes<R>(nslots);
    if (!attr_done) {
        cudaFuncSetAttribute(jk_coop_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr_done = 1;
    }
    const int blocks = (a.ntasks + COOP_WARPS - 1) / COOP_WARPS;
    if (blocks == 0) return;
    jk_coop_kernel<R><<<blocks, COOP_THREADS, bytes, s>>>(a, qc, nslots);
}

void launch_coop(const JKArgs& a, int qc, int fp32, cudaStream_t s)
{
    if (fp32) launch_coop_t<float>(a, qc, s);
    else launch_coop_t<double>(a, qc, s);
}

size_t coop_smem_bytes(int qc, int fp32)
{
    const int nslots = COOP_SIZES[qc].nslots;
    return (size_t)COOP_WARPS * (fp32 ? coop_warp_bytes<float>(nslots) : coop_warp_bytes<double>(nslots));
}

}  // namespace cq
