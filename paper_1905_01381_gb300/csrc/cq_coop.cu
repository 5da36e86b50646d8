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
    const int wslots = coop_region_slots(COOP_SIZES[qc].vslots, COOP_SIZES[qc].hslots);
    const size_t bytes = (size_t)COOP_WARPS * coop_warp_bytes<R>(wslots);
    if (!attr_done) {
        cudaFuncSetAttribute(jk_coop_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr_done = 1;
    }
    const long long tasks = (long long)a.ntasks * (a.coop_list ? a.coop_split : 1);
    long long blocks = (tasks + COOP_WARPS - 1) / COOP_WARPS;
    if (blocks == 0) return;
    const long long cap = jk_grid_cap();
    if (a.coop_list && blocks > cap) blocks = cap;   // warps stride over the list
    jk_coop_kernel<R><<<(unsigned)blocks, COOP_THREADS, bytes, s>>>(a, qc, wslots);
}

// prec: 0 FP64, 1 FP32, 2 double-float
void launch_coop(const JKArgs& a, int qc, int prec, cudaStream_t s)
{
    if (prec == 1) launch_coop_t<float>(a, qc, s);
    else if (prec == 2) launch_coop_t<df>(a, qc, s);
    else launch_coop_t<double>(a, qc, s);
}

size_t coop_smem_bytes(int qc, int prec)
{
    const int wslots = coop_region_slots(COOP_SIZES[qc].vslots, COOP_SIZES[qc].hslots);
    return (size_t)COOP_WARPS * (prec == 1 ? coop_warp_bytes<float>(wslots) : coop_warp_bytes<double>(wslots));
}

}  // namespace cq
