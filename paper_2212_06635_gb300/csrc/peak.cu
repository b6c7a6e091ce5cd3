// Arithmetic-rate microbenchmark of the CUDA cores (FP64 or FP32 fused
// multiply-add), for the roofline denominators of the passes that arithmetic
// rather than memory bounds.  Every thread runs 8 independent FMA chains on
// registers; the grid fills every SM with resident blocks; the result is written
// so that no chain can be removed.
#include <cuda_runtime.h>

#include "../../include/tm.h"

namespace tmk {
tm_status tmk_failf(tm_status s, const char* fmt, ...);
}

namespace {

template <typename R>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, R a, R b, R* out) {
    R x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (R)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == (R)-1.2345) out[blockIdx.x] = s;   // never true for these inputs; keeps the chains live
}

template <typename R>
tm_status rate(int device, double* flops) {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return tmk::tmk_failf(TM_ERR_CUDA, "tm_fma_rate: %s", cudaGetErrorString(cudaGetLastError()));
    const int blocks = nsm * 8;          // 2048 resident threads per SM
    R* out = nullptr;
    cudaEvent_t e0, e1;
    if (cudaMalloc(&out, sizeof(R) * blocks) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaFree(out);
        return tmk::tmk_failf(TM_ERR_CUDA, "tm_fma_rate: %s", cudaGetErrorString(cudaGetLastError()));
    }
    const int iters = sizeof(R) == 8 ? 256 : 4096;
    k_fma_chains<R><<<blocks, 256>>>(iters, (R)0.999, (R)0.001, out);   // warm-up
    cudaEventRecord(e0);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) k_fma_chains<R><<<blocks, 256>>>(iters, (R)0.999, (R)0.001, out);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return tmk::tmk_failf(TM_ERR_CUDA, "tm_fma_rate: %s", cudaGetErrorString(e));
    const double fmas = (double)reps * blocks * 256.0 * iters * 16.0 * 8.0;
    *flops = 2.0 * fmas / (ms * 1e-3);
    return TM_OK;
}

}  // namespace

extern "C" tm_status tm_fma_rate(int device, tm_prec prec, double* flops_per_s) {
    if (!flops_per_s || (prec != TM_F64 && prec != TM_F32))
        return tmk::tmk_failf(TM_ERR_ARG, "tm_fma_rate: prec must be TM_F64 or TM_F32");
    if (cudaSetDevice(device) != cudaSuccess)
        return tmk::tmk_failf(TM_ERR_CUDA, "tm_fma_rate: %s", cudaGetErrorString(cudaGetLastError()));
    return prec == TM_F64 ? rate<double>(device, flops_per_s) : rate<float>(device, flops_per_s);
}
