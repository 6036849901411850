// Throughput loops for the compositing kernels' ALU roofline: FP32 FMA, MUFU
// ex2 and MUFU rcp, each on 8 independent chains per thread over a grid of
// 8 CTAs x 256 threads per SM.  Prints one JSON line of operations per second.
#include <cstdio>
#include <cuda_runtime.h>

constexpr int kChains = 8;

__global__ void k_fma(float* out, int iters)
{
    float a[kChains];
    for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], 0.9999f, 1e-4f);
    float s = 0;
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ex2(float* out, int iters)
{
    float a[kChains];
    for (int k = 0; k < kChains; ++k) a[k] = -(threadIdx.x * 1e-4f + k * 1e-2f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            float r;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
            a[k] = -r;  // stays in [-1, 0): 2^a in (1/2, 1]
        }
    float s = 0;
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_rcp(float* out, int iters)
{
    float a[kChains];
    for (int k = 0; k < kChains; ++k) a[k] = 1.5f + threadIdx.x * 1e-4f + k * 1e-2f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            float r;
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
            a[k] = r + 1.0f;  // stays in [1, 2]
        }
    float s = 0;
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main()
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms <= 0) return 1;
    const int blocks = sms * 8, threads = 256, iters = 1 << 16;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return 1;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double rate[3] = {0, 0, 0};
    for (int which = 0; which < 3; ++which) {
        const int n = which == 0 ? iters : iters / 4;
        for (int rep = 0; rep < 4; ++rep) {  // the last of four runs (the first ones ramp the clocks)
            cudaEventRecord(a);
            if (which == 0) k_fma<<<blocks, threads>>>(out, n);
            else if (which == 1) k_ex2<<<blocks, threads>>>(out, n);
            else k_rcp<<<blocks, threads>>>(out, n);
            cudaEventRecord(b);
            cudaEventSynchronize(b);
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            rate[which] = (double)blocks * threads * kChains * n / (ms * 1e-3);
        }
    }
    const cudaError_t e = cudaGetLastError();
    printf("{\"sms\": %d, \"fma_per_s\": %.6e, \"ex2_per_s\": %.6e, \"rcp_per_s\": %.6e, \"status\": \"%s\"}\n", sms,
           rate[0], rate[1], rate[2], cudaGetErrorString(e));
    cudaFree(out);
    return e != cudaSuccess;
}
