// Arithmetic-peak microbenchmark: independent dependent-FMA chains on every
// SM, timed with CUDA events.  Gives the FP64 / FP32 FMA throughput that the
// integral kernels (plain ALU work) are measured against.
#include "cq_internal.h"

namespace cq {

template <typename T>
__global__ void fma_chain_kernel(T* out, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == (T)12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keep the chains alive
}

}  // namespace cq

using namespace cq;

extern "C" int cq_peak_fma(int fp32, int iters, double* flops_per_s, void* stream)
{
    if (!flops_per_s || iters <= 0) { set_error("cq_peak_fma: bad argument"); return CQ_ERR_INVALID_ARG; }
    int dev = 0, nsm = 0;
    CQ_CUDA(cudaGetDevice(&dev));
    CQ_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256, blocks = nsm * 8;
    void* out = nullptr;
    CQ_CUDA(cudaMalloc(&out, (size_t)threads * blocks * sizeof(double)));
    cudaEvent_t e0, e1;
    CQ_CUDA(cudaEventCreate(&e0));
    CQ_CUDA(cudaEventCreate(&e1));
    for (int rep = 0; rep < 2; ++rep) {   // first launch warms up
        CQ_CUDA(cudaEventRecord(e0, s));
        if (fp32)
            fma_chain_kernel<float><<<blocks, threads, 0, s>>>((float*)out, iters, 0.999999f, 1e-7f);
        else
            fma_chain_kernel<double><<<blocks, threads, 0, s>>>((double*)out, iters, 0.999999, 1e-7);
        CQ_CUDA(cudaEventRecord(e1, s));
    }
    CQ_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    CQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *flops_per_s = 2.0 * 8.0 * iters * (double)threads * blocks / (ms * 1e-3);
    return CQ_OK;
}
