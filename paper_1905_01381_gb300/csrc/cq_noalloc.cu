// Allocation-free variant of cq_fock_build.
//
// Some callers cannot let a library call cudaMalloc on their behalf: hosts
// that own every byte of device memory through their own allocator or a
// fixed budget reserved up front, and latency-critical loops where an
// allocation (and the device synchronisation cudaMalloc/cudaFree can imply)
// is not acceptable once the loop runs.  cq_fock_build grows its per-build
// scratch inside the basis handle on first use; this entry point instead
// takes its scratch from one file-scope device array of fixed size, so it
// never allocates.  The basis handle itself (created beforehand with
// cq_basis_create) is unchanged.
#include <cstring>
#include <mutex>

#include "cq_internal.h"
#include "cq_jk.cuh"

namespace cq {

// kernels of the ordinary build (cq_fock.cu), reused unchanged
__global__ void density_prep_kernel(int kind, int nmol, int ld, const int* __restrict__ mol_n,
                                    const int* __restrict__ mol_bfo, const double* __restrict__ P,
                                    const double* __restrict__ sc, double* __restrict__ Dp);
__global__ void dmax_kernel(int nmol, int ld, int lds, const int* __restrict__ mol_nsh, const int* __restrict__ mol_sho,
                            const int* __restrict__ mol_bfo, const int* __restrict__ bfo, int nk,
                            const double* __restrict__ Dp, const int* __restrict__ mol_mode,
                            float* __restrict__ Dmax);
__global__ void finalize_kernel(int kind, int nmol, int ld, const int* __restrict__ mol_n,
                                const int* __restrict__ mol_bfo, const double* __restrict__ sc,
                                const acc_t* __restrict__ Jp, const acc_t* __restrict__ Kp, double* __restrict__ J,
                                double* __restrict__ K, int want_j, int want_k);

// Scratch of the allocation-free build: 16 MiB on every device whose code
// module for this file is loaded, held until the library is unloaded.  With
// CUDA's lazy module loading the module is loaded (and the 16 MiB reserved)
// by the first cudaGetSymbolAddress below, i.e. by the first call on a
// device; eager loading reserves it when the library's code is loaded.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static void* g_scratch_addr[NOALLOC_MAX_DEVICES] = {nullptr};
static std::mutex g_scratch_mu;

static size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (looked up once
// per device; in host code the array's name is only a host-side stand-in).
static int scratch_address(void** out)
{
    int dev = 0;
    CQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("cq_fock_build_noalloc: device ordinal beyond the supported range");
        return CQ_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return CQ_OK;
}

}  // namespace cq

using namespace cq;

// Single-molecule bases only: a batched basis needs nmol slots of its
// largest molecule (noalloc_bytes below, which the call itself checks).
extern "C" size_t cq_fock_noalloc_scratch_bytes(int kind, int nbf, int nshell)
{
    const int nk = dens_nk(kind);
    const size_t nn = (size_t)nbf * nbf;
    return round256(nn * nk * sizeof(double)) + round256(2 * nn * nk * sizeof(acc_t)) +
           round256(2 * nn * sizeof(acc_t)) + round256((size_t)nshell * nshell * sizeof(float)) +
           round256(CNT_WORDS * sizeof(unsigned long long));
}

static size_t noalloc_bytes(const cq_basis* b, int kind)
{
    const int nk = dens_nk(kind);
    const size_t nn = b->mstride;
    return round256(nn * nk * sizeof(double)) + round256(2 * nn * nk * sizeof(acc_t)) +
           round256(2 * nn * sizeof(acc_t)) + round256((size_t)b->nmol * b->lds * b->lds * sizeof(float)) +
           round256(CNT_WORDS * sizeof(unsigned long long));
}

extern "C" int cq_fock_build_noalloc(cq_basis* b, int kind, const void* P, double* J, void* K,
                                     const cq_fock_opts* opts, void* stream)
{
    if (!b || !P) { set_error("cq_fock_build_noalloc: NULL basis or density"); return CQ_ERR_INVALID_ARG; }
    if (kind < CQ_DENS_REAL_SYM || kind > CQ_DENS_REAL_GENERAL) {
        set_error("cq_fock_build_noalloc: unknown density kind");
        return CQ_ERR_INVALID_ARG;
    }
    cq_fock_opts o{1e-14, 1e-5, CQ_PREC_FP64, 1, 1, 0.0};
    if (opts) o = *opts;
    if ((o.want_J && !J) || (o.want_K && !K)) {
        set_error("cq_fock_build_noalloc: requested output pointer is NULL");
        return CQ_ERR_INVALID_ARG;
    }
    if ((o.prec != CQ_PREC_FP64 && o.prec != CQ_PREC_MIXED) || !(o.schwarz_tol >= 0.0) ||
        !(o.mixed_tol >= 0.0) || !(o.fp64_tol >= 0.0)) {
        set_error("cq_fock_build_noalloc: bad options");
        return CQ_ERR_INVALID_ARG;
    }
    const size_t need = noalloc_bytes(b, kind);
    if (need > NOALLOC_SCRATCH_BYTES) {
        set_error("cq_fock_build_noalloc: basis too large for the fixed 16 MiB scratch (needs " +
                  std::to_string(need) + " bytes); use cq_fock_build");
        return CQ_ERR_INVALID_ARG;
    }
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    const int nk = dens_nk(kind);
    const int n = b->ld;
    const size_t nn = b->mstride;
    unsigned char* p = (unsigned char*)base;
    double* Dp = (double*)p;          p += round256(nn * nk * sizeof(double));
    acc_t* Kp = (acc_t*)p;            p += round256(2 * nn * nk * sizeof(acc_t));
    acc_t* Jp = (acc_t*)p;            p += round256(2 * nn * sizeof(acc_t));
    float* Dmax = (float*)p;          p += round256((size_t)b->nmol * b->lds * b->lds * sizeof(float));
    unsigned long long* cnt = (unsigned long long*)p;

    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((nn + 255) / 256);
    density_prep_kernel<<<nb, 256, 0, s>>>(kind, b->nmol, n, b->d_mol_n, b->d_mol_bfo, (const double*)P, b->d_scale, Dp);
    const size_t nsl = (size_t)b->nmol * b->lds * b->lds;
    dmax_kernel<<<(unsigned)((nsl + 127) / 128), 128, 0, s>>>(b->nmol, n, b->lds, b->d_mol_nsh, b->d_mol_sho,
                                                              b->d_mol_bfo, b->d_bfo, nk, Dp, nullptr, Dmax);
    // the array keeps the previous call's contents: clear the accumulators
    CQ_CUDA(cudaMemsetAsync(Jp, 0, 2 * nn * sizeof(acc_t), s));
    CQ_CUDA(cudaMemsetAsync(Kp, 0, 2 * nn * nk * sizeof(acc_t), s));
    CQ_CUDA(cudaMemsetAsync(cnt, 0, CNT_WORDS * sizeof(unsigned long long), s));
    JKArgs a;
    memset(&a, 0, sizeof a);
    a.pairs = b->d_pairs; a.prims = b->d_prims; a.primsf = b->d_primsf;
    a.Q = b->d_Qf; a.Dmax = Dmax; a.nsh = b->lds;
    a.mstride = (long long)nn;
    a.tau = (float)o.schwarz_tol;
    a.tau_mixed = (float)o.mixed_tol;
    a.D = Dp; a.nk = nk; a.nbf = n;
    a.want_j = o.want_J; a.want_k = o.want_K;
    a.J = Jp; a.K = Kp;
    a.boys_d = b->d_boys; a.boys_f = b->d_boysf;
    a.counters = cnt + 6;
    a.primsx = b->d_primsx;
    rc = classify_and_launch(b, a, o, false, s);
    if (rc) return rc;
    CQ_CUDA(cudaGetLastError());
    finalize_kernel<<<nb, 256, 0, s>>>(kind, b->nmol, n, b->d_mol_n, b->d_mol_bfo, b->d_scale, Jp, Kp, J, (double*)K,
                                       o.want_J, o.want_K);
    CQ_CUDA(cudaGetLastError());
    return CQ_OK;
}
