// Exhaustive-style check of the integer-pipe conversions in csrc/convert.cuh
// against the hardware conversions (__double2float_rn and float -> double).
//
// d2f_rn: 2^24 FP64 inputs per launch built from splitmix64 bits with the
// exponent drawn from [880, 1160] (every branch of d2f_rn: zero/subnormal,
// hardware fallback below and above the normal FP32 range, the integer path),
// a quarter of them forced onto exact rounding ties, plus a table of special
// values (+-0, FP64 subnormals, FP32 min normal and max, infinities, NaN).
// f2d_exact: all 2^32 FP32 bit patterns.  Each thread compares its values and
// counts mismatches (bitwise; NaN against NaN counts as equal); the buffers
// are exactly grid x block long.
//
// Build and run:  nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o convert_check convert_check.cu && ./convert_check
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdint>

#include "../paper_2302_04979_gb300/csrc/convert.cuh"

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ double make_input(unsigned long long idx) {
    const unsigned long long r = mix64(idx), r2 = mix64(idx ^ 0xD1B54A32D192ED03ULL);
    const unsigned long long sign = r & 0x8000000000000000ULL;
    const unsigned long long e = 880 + (r2 % 281);  // [880, 1160]
    unsigned long long m = r & 0xFFFFFFFFFFFFFULL;
    if ((r2 >> 40) % 4 == 0) m = (m & ~0x1FFFFFFFULL) | 0x10000000ULL;  // exact tie on the 29 dropped bits
    return __longlong_as_double(static_cast<long long>(sign | (e << 52) | m));
}

__device__ bool same_f(float a, float b) {
    if (isnan(a) && isnan(b)) return true;
    return __float_as_uint(a) == __float_as_uint(b);
}
__device__ bool same_d(double a, double b) {
    if (isnan(a) && isnan(b)) return true;
    return __double_as_longlong(a) == __double_as_longlong(b);
}

__global__ void check_d2f(unsigned long long base, int per_thread, unsigned long long* bad) {
    const unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    unsigned long long n = 0;
    for (int k = 0; k < per_thread; ++k) {
        const double x = make_input(base + t * per_thread + k);
        if (!same_f(smx::d2f_rn(x), __double2float_rn(x))) ++n;
    }
    bad[t] = n;
}

__global__ void check_d2f_special(const double* x, int n, unsigned long long* bad) {
    const int i = threadIdx.x;
    if (i < n) bad[i] = same_f(smx::d2f_rn(x[i]), __double2float_rn(x[i])) ? 0 : 1;
}

__global__ void check_f2d(unsigned long long base, int per_thread, unsigned long long* bad) {
    const unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    unsigned long long n = 0;
    for (int k = 0; k < per_thread; ++k) {
        const float v = __uint_as_float(static_cast<unsigned>(base + t * per_thread + k));
        if (!same_d(smx::f2d_exact(v), static_cast<double>(v))) ++n;
    }
    bad[t] = n;
}

static unsigned long long sum_bad(unsigned long long* d, int n) {
    unsigned long long* h = new unsigned long long[n];
    cudaMemcpy(h, d, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    unsigned long long s = 0;
    for (int i = 0; i < n; ++i) s += h[i];
    delete[] h;
    return s;
}

int main() {
    const int block = 256, grid = 1024, nt = block * grid;
    unsigned long long* bad = nullptr;
    if (cudaMalloc(&bad, nt * sizeof(unsigned long long)) != cudaSuccess) return 2;

    unsigned long long d2f_bad = 0;
    for (int launch = 0; launch < 4; ++launch) {  // 4 x 2^24 random inputs
        check_d2f<<<grid, block>>>((unsigned long long)launch << 24, 64, bad);
        d2f_bad += sum_bad(bad, nt);
    }
    const double special[] = {0.0, -0.0, 4.9e-324, -4.9e-324, 2.2250738585072014e-308, 1.1754943508222875e-38,
                              -1.1754943508222875e-38, 1.1754942106924411e-38, 1.401298464324817e-45,
                              7.006492321624085e-46, 3.4028234663852886e38, -3.4028234663852886e38,
                              3.4028235677973366e38, 1.0e39, 1.0, -1.0, 1.0 + 1.0 / (1 << 24), 1.0 + 3.0 / (1 << 24),
                              0.1, -0.3, INFINITY, -INFINITY, NAN};
    const int ns = sizeof(special) / sizeof(special[0]);
    double* dsp = nullptr;
    if (cudaMalloc(&dsp, sizeof(special)) != cudaSuccess) return 2;
    cudaMemcpy(dsp, special, sizeof(special), cudaMemcpyHostToDevice);
    check_d2f_special<<<1, block>>>(dsp, ns, bad);
    d2f_bad += sum_bad(bad, ns);

    unsigned long long f2d_bad = 0;
    for (int launch = 0; launch < 256; ++launch) {  // all 2^32 FP32 patterns, 2^24 per launch
        check_f2d<<<grid, block>>>((unsigned long long)launch << 24, 64, bad);
        f2d_bad += sum_bad(bad, nt);
    }
    const cudaError_t err = cudaDeviceSynchronize();
    printf("d2f_rn: %llu mismatches of %llu inputs; f2d_exact: %llu mismatches of %llu inputs; %s\n", d2f_bad,
           4ull * nt * 64 + ns, f2d_bad, 256ull * nt * 64, cudaGetErrorString(err));
    cudaFree(dsp);
    cudaFree(bad);
    return (err == cudaSuccess && d2f_bad == 0 && f2d_bad == 0) ? 0 : 1;
}
