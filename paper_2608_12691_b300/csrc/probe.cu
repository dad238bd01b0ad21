// probe.cu -- measured FP32 and FP64 arithmetic throughput of the device
// (FMA chains), the measured denominators beside the unit-count peaks that
// the pair kernel's ALU roofline is quoted against.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "lfe.h"

namespace {

// CHAINS independent FMA chains per thread, ITER rounds; the result is
// written only when it equals a value it never takes, so the chains stay
template <typename T, int CHAINS>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T b, T c, T* sink)
{
    T a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == (T)-12345.678) sink[threadIdx.x] = s;
}

template <typename T>
double measure(int nsm, int iters, T* sink)
{
    constexpr int CH = 8;
    const int blocks = nsm * 8, threads = 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // b slightly below 1 and c small keep the values finite and normal
    k_fma_chains<T, CH><<<blocks, threads>>>(iters / 4, (T)0.999999, (T)1e-6, sink);   // warm-up
    std::vector<float> ms(3);
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0);
        k_fma_chains<T, CH><<<blocks, threads>>>(iters, (T)0.999999, (T)1e-6, sink);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms[r], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double t = *std::min_element(ms.begin(), ms.end()) * 1e-3;
    const double flops = 2.0 * CH * (double)iters * blocks * threads;
    return flops / t / 1e12;
}

}  // namespace

extern "C" int lfe_alu_peak(double* fp32_tflops, double* fp64_tflops)
{
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LFE_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LFE_ERR_CUDA;
    void* sink = nullptr;
    if (cudaMalloc(&sink, 256 * sizeof(double)) != cudaSuccess) return LFE_ERR_CUDA;
    double f32 = 0, f64 = 0;
    if (fp32_tflops) f32 = measure<float>(nsm, 1 << 14, (float*)sink);
    if (fp64_tflops) f64 = measure<double>(nsm, 1 << 9, (double*)sink);
    const cudaError_t err = cudaGetLastError();
    cudaFree(sink);
    if (err != cudaSuccess) return LFE_ERR_CUDA;
    if (fp32_tflops) *fp32_tflops = f32;
    if (fp64_tflops) *fp64_tflops = f64;
    return LFE_OK;
}
