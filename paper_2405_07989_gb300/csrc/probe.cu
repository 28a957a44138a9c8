// Integer-throughput probe: the peak rate of the integer instructions the
// count walk is made of (32-bit add, three-input logic, multiply-add), for the
// roofline of the ALU-bound kernels.  Each thread runs 8 independent chains
// so that issue, not latency, bounds the loop.
#include <cuda_runtime.h>

#include "launch.h"

namespace fsi {

__device__ uint32_t g_probe_sink;

template <int KIND>
__global__ void __launch_bounds__(256) k_int_probe(uint32_t iters, uint32_t seed)
{
    uint32_t x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = seed + threadIdx.x * 8 + j;
    const uint32_t y = seed * 2654435761u + blockIdx.x;
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                if (KIND == 0) asm volatile("add.u32 %0, %0, %1;" : "+r"(x[j]) : "r"(y));
                if (KIND == 1) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[j]) : "r"(y), "r"(seed));
                if (KIND == 2) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[j]) : "r"(y), "r"(seed));
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) acc ^= x[j];
    if (acc == 0x12345678u) g_probe_sink = acc;  // keeps the chains alive
}

// ops/s of one kind, measured over `iters` loop trips on the whole GPU.
cudaError_t int_probe(int kind, uint32_t iters, double* ops_per_s, double* ms_out)
{
    int dev = 0, sms = 0, nb = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    void* k = kind == 0 ? (void*)k_int_probe<0> : kind == 1 ? (void*)k_int_probe<1> : (void*)k_int_probe<2>;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 256, 0);
    if (e != cudaSuccess) return e;
    const int blocks = sms * nb;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    uint32_t seed = 7;
    void* args[] = {&iters, &seed};
    e = cudaLaunchKernel(k, dim3(blocks), dim3(256), args, 0, 0);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(a, 0);
    if (e == cudaSuccess) e = cudaLaunchKernel(k, dim3(blocks), dim3(256), args, 0, 0);
    if (e == cudaSuccess) e = cudaEventRecord(b, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return e;
    const double ops = (double)blocks * 256.0 * (double)iters * 32.0;
    *ops_per_s = ops / (ms / 1000.0);
    if (ms_out) *ms_out = ms;
    return cudaSuccess;
}

}  // namespace fsi
