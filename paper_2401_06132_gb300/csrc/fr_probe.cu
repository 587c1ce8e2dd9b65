// fr_probe.cu -- CUDA-core FMA throughput probe (FP64 and FP32), used as the ALU roofline.
#include <cuda_runtime.h>

#include "fr_internal.h"

// Eight independent FMA chains per thread; the result is stored so nothing is optimised away.
template <typename T, int ITER>
__global__ void __launch_bounds__(256) k_fma(T *out, T a, T b)
{
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = T(threadIdx.x + k) * T(1e-3);
#pragma unroll 4
    for (int i = 0; i < ITER; i++)
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = x[k] * a + b;
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, int ITER>
static double probe(cudaStream_t s, int blocks)
{
    T *d = nullptr;
    if (cudaMalloc(&d, (size_t)blocks * 256 * sizeof(T)) != cudaSuccess) return -1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma<T, ITER><<<blocks, 256, 0, s>>>(d, T(0.999999), T(1e-7));  // warm-up
    cudaEventRecord(e0, s);
    const int reps = 3;
    for (int r = 0; r < reps; r++) k_fma<T, ITER><<<blocks, 256, 0, s>>>(d, T(0.999999), T(1e-7));
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    double flops = 2.0 * 8.0 * ITER * (double)blocks * 256 * reps;
    return flops / (ms * 1e-3) / 1e9;
}

extern "C" fr_status fr_probe_fma(double *out, void *stream)
{
    if (!out) return FR_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FR_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = (cudaStream_t)stream;
    out[0] = probe<double, 1024>(s, sms * 8);
    out[1] = probe<float, 16384>(s, sms * 8);
    if (cudaStreamSynchronize(s) != cudaSuccess) return FR_ECUDA;
    return (out[0] > 0 && out[1] > 0) ? FR_OK : FR_ECUDA;
}
