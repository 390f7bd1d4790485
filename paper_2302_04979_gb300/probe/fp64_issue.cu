// FP64 FMA issue rate versus warps per SM and active lanes per warp.
//
// One CTA per SM with w warps; every thread runs 8 independent FMA chains
// (enough to cover the FMA latency) with only the first `active` lanes of
// each warp enabled.  Reports lane and warp-instruction throughput, which
// shows how many warps per SM the FP64 pipes need and whether inactive lanes
// cost issue slots.  out[] has exactly grid x block entries; every thread
// writes one value.
//
// Build and run:  nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_issue fp64_issue.cu && ./fp64_issue
#include <cstdio>
#include <cuda_runtime.h>
__global__ void k(double* out, int iters, int active, double a, double b) {
    double x[8];
    for (int q = 0; q < 8; ++q) x[q] = threadIdx.x * 1e-7 + q;
    if ((threadIdx.x & 31) < active) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
        }
    }
    double s = 0;
    for (int q = 0; q < 8; ++q) s += x[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
    int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    double* out; cudaMalloc(&out, (size_t)sms * 1024 * sizeof(double));
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    const int iters = 4096;
    for (int warps : {1, 2, 3, 4, 6, 8, 16}) for (int active : {32, 16, 8}) {
        const int block = 32 * warps;
        k<<<sms, block>>>(out, iters, active, 0.999, 1e-3);
        cudaEventRecord(e0);
        k<<<sms, block>>>(out, iters, active, 0.999, 1e-3);
        cudaEventRecord(e1); cudaEventSynchronize(e1);
        float ms; cudaEventElapsedTime(&ms, e0, e1);
        const double lane_ops = (double)sms * warps * active * iters * 8;
        printf("warps/SM %2d active lanes %2d: %.3f ms  %.1f G lane-DFMA/s  %.1f G warp-instr/s\n", warps, active, ms,
               lane_ops / ms / 1e6, (double)sms * warps * iters * 8 / ms / 1e6);
    }
    printf("%s\n", cudaGetErrorString(cudaDeviceSynchronize()));
    return 0;
}
