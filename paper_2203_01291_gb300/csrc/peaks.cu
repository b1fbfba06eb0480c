// Arithmetic throughput microbenchmark (instrumentation; no counterpart in the
// paper): FMA rate in FP32 or FP64 of this GPU, used as the ALU roofline of
// the FP64 path (on GB300 the FP64 rate is far below the FP32 one).
#include <cuda_runtime.h>

#include "internal.cuh"

namespace hol {
namespace {

template <typename R>
__global__ void __launch_bounds__(256) k_fma_peak(R* out, int iters, R a, R b)
{
    R x0 = (R)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    R x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    const R s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (R)-12345.678) out[threadIdx.x] = s;   // never true; keeps the work alive
}

}  // namespace
}  // namespace hol

using namespace hol;

extern "C" int hol_fma_peak(int prec, double* gflops, void* stream)
{
    HOL_TRACE("hol_fma_peak");
    if (!gflops || (prec != HOL_F64 && prec != HOL_F32))
        return set_error(HOL_EINVAL, "hol_fma_peak: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    HOL_CUDA(cudaGetDevice(&dev));
    HOL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;
    const int iters = prec == HOL_F64 ? 64 : 1024;
    cudaEvent_t e0, e1;
    HOL_CUDA(cudaEventCreate(&e0));
    HOL_CUDA(cudaEventCreate(&e1));
    float ms = 0.0f;
    for (int rep = 0; rep < 2; ++rep) {   // first pass warms up
        cudaEventRecord(e0, s);
        if (prec == HOL_F64)
            k_fma_peak<double><<<blocks, threads, 0, s>>>(nullptr, iters, 0.999999, 1e-7);
        else
            k_fma_peak<float><<<blocks, threads, 0, s>>>(nullptr, iters, 0.999999f, 1e-7f);
        count_launch();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_error(err, "k_fma_peak");
    const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
    *gflops = flops / (ms * 1e-3) / 1e9;
    return HOL_OK;
}
