// gp_fma_peak: the FP64 and FP32 fused multiply-add throughput of the device,
// the arithmetic ceiling the FP64 kernels are measured against (instrumentation;
// the paper has no counterpart).  Every thread of a full-occupancy grid runs
// eight independent FMA chains; an FMA counts as two flops.
#include <cstdio>

#include "gpmg_internal.cuh"

namespace gpmg {
namespace {

constexpr int PROBE_STEPS = 4096;

template <typename T> __global__ void __launch_bounds__(256) k_fma_chains(T *sink, T a, T c)
{
    T x[8];
#pragma unroll
    for (int q = 0; q < 8; q++) x[q] = (T)threadIdx.x * (T)1e-3 + (T)q;
    for (int s = 0; s < PROBE_STEPS; s++) {
#pragma unroll
        for (int q = 0; q < 8; q++) x[q] = fma(x[q], a, c);
    }
    T t = 0;
#pragma unroll
    for (int q = 0; q < 8; q++) t += x[q];
    if (t == (T)12345.678) sink[blockIdx.x] = t;  // keeps the chains live; never true for these inputs
}

template <typename T> int time_chains(int blocks, T *sink, cudaStream_t st, double *tflops)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GP_CUDA;
    k_fma_chains<T><<<blocks, 256, 0, st>>>(sink, (T)0.999999, (T)1e-9);
    cudaEventRecord(e0, st);
    const int reps = 5;
    for (int r = 0; r < reps; r++) k_fma_chains<T><<<blocks, 256, 0, st>>>(sink, (T)0.999999, (T)1e-9);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || !(ms > 0.0f)) return GP_CUDA;
    const double flops = (double)reps * blocks * 256.0 * 8.0 * PROBE_STEPS * 2.0;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return GP_OK;
}

}  // namespace
}  // namespace gpmg

extern "C" gp_status gp_fma_peak(void *sink, void *stream, double *fp64_tflops, double *fp32_tflops)
{
    if (!sink || !fp64_tflops || !fp32_tflops) return GP_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GP_CUDA;
    const int blocks = sms * 8;
    cudaStream_t st = (cudaStream_t)stream;
    int s = gpmg::time_chains<double>(blocks, (double *)sink, st, fp64_tflops);
    if (s == GP_OK) s = gpmg::time_chains<float>(blocks, (float *)sink, st, fp32_tflops);
    return (gp_status)s;
}
