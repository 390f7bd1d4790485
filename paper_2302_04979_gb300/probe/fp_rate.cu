// Arithmetic-rate probe for the roofline of the FP64 leapfrog kernels.
//
// Measures, with CUDA events, the device-wide throughput of FP64 FMA, add and
// multiply, FP32 FMA, and the latency of a dependent FP64 FMA chain.  Every
// thread keeps its values in registers and writes one result to out[], whose
// size is exactly grid x block, so no access leaves the buffer.
//
// Build and run:  nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp_rate fp_rate.cu && ./fp_rate
#include <cuda_runtime.h>

#include <cstdio>

enum Op { kFma = 0, kAdd = 1, kMul = 2 };

template <class T, int OP>
__global__ void throughput(T* out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x * 1e-7 + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (OP == kFma) x[k] = fma(x[k], a, b);
            if (OP == kAdd) x[k] = x[k] + b;
            if (OP == kMul) x[k] = x[k] * a;
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void latency(double* out, long long* cycles, int iters, double a, double b) {
    double x = threadIdx.x * 1e-7;
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) x = fma(x, a, b);
    const long long t1 = clock64();
    out[blockIdx.x * blockDim.x + threadIdx.x] = x;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <class T, int OP>
static void run(const char* name, int blocks_per_sm, int threads, int iters, int nsm) {
    const int grid = nsm * blocks_per_sm;
    T* out = nullptr;
    cudaMalloc(&out, sizeof(T) * grid * threads);
    throughput<T, OP><<<grid, threads>>>(out, 64, (T)0.999999, (T)1e-7);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a);
    throughput<T, OP><<<grid, threads>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double ops = 8.0 * iters * (double)grid * threads;  // lane operations
    printf("%-10s grid=%5d x %3d: %8.3f ms  %8.2f G lane-ops/s  (%s)\n", name, grid, threads, ms, ops / ms / 1e6,
           cudaGetErrorString(cudaGetLastError()));
    cudaFree(out);
}

int main() {
    int nsm = 0, clk = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    printf("SMs %d, max SM clock %d kHz\n", nsm, clk);
    run<double, kFma>("dfma", 8, 256, 4000, nsm);
    run<double, kAdd>("dadd", 8, 256, 4000, nsm);
    run<double, kMul>("dmul", 8, 256, 4000, nsm);
    run<float, kFma>("ffma", 8, 256, 40000, nsm);
    double* out = nullptr;
    long long* cyc = nullptr;
    cudaMalloc(&out, sizeof(double) * 32);
    cudaMalloc(&cyc, sizeof(long long));
    latency<<<1, 32>>>(out, cyc, 1000, 0.999999, 1e-7);
    latency<<<1, 32>>>(out, cyc, 10000, 0.999999, 1e-7);
    long long h = 0;
    cudaMemcpy(&h, cyc, sizeof(long long), cudaMemcpyDeviceToHost);
    printf("dependent dfma chain (1 warp): %.1f cycles per fma (%s)\n", h / 10000.0,
           cudaGetErrorString(cudaGetLastError()));
    cudaFree(out);
    cudaFree(cyc);
    return 0;
}
