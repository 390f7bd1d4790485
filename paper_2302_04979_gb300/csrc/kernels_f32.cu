// FP32 operator kernels of the mixed-precision leapfrog.
//
// The stepped state (d, b) stays FP64 and is updated with one FP64 FMA per
// coefficient; every operator (curl differences, Hodge mass, pairing sweeps)
// runs in FP32.  Operator coefficients are stored as FP32 pairs (hi, lo) with
// hi + lo equal to the FP64 value to about 2^-48, and every product is formed
// as hi*x + lo*x, so the operators themselves carry no FP32 rounding: only the
// data is rounded, and those roundings do not repeat systematically step
// after step.  FP32 FMA latency is a few cycles (FP64: about 64 on GB300), so
// the line recurrences here are no longer latency-bound.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace smx {

__device__ __forceinline__ float fma2(float2 c, float x, float acc) { return fmaf(c.x, x, fmaf(c.y, x, acc)); }

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8f(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all_f() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <class T>
__device__ __forceinline__ float to_f(T v) {
    return static_cast<float>(v);
}

// ------------------------------------------------------------------ curl (FP32 differences, FP64 state)
template <int A, bool DUAL>
__device__ __forceinline__ float incidence_f(const DevComp& u, const float* __restrict__ v, int i, int j, int k) {
    const int idx = i + u.n[0] * (j + u.n[1] * k);
    const int stride = A == 0 ? 1 : (A == 1 ? u.n[0] : u.n[0] * u.n[1]);
    const float* p = v + u.off + idx;
    if (DUAL) return __ldg(p + stride) - __ldg(p);
    const int m = A == 0 ? i : (A == 1 ? j : k);
    const float hi = (m < u.n[A]) ? __ldg(p) : 0.0f;
    const float lo = (m >= 1) ? __ldg(p - stride) : 0.0f;
    return hi - lo;
}

template <int C, bool DUAL>
__device__ __forceinline__ void curl_comp_f(const DevField& IN, const DevField& OUT, const float* __restrict__ in,
                                            double* __restrict__ out, double alpha, const double* __restrict__ jhat,
                                            const double* __restrict__ amp, int amp_index, double s_host, int i, int j,
                                            int k) {
    constexpr int a1 = (C + 1) % 3, a2 = (C + 2) % 3;
    const DevComp& O = OUT.c[C];
    if (i >= O.n[0] || j >= O.n[1] || k >= O.n[2]) return;
    const float vf = incidence_f<a1, DUAL>(IN.c[a2], in, i, j, k) - incidence_f<a2, DUAL>(IN.c[a1], in, i, j, k);
    double v = static_cast<double>(vf);
    const long long g = O.off + i + O.n[0] * (j + O.n[1] * k);
    if (DUAL && jhat != nullptr) {
        const double s = amp != nullptr ? __ldg(amp + amp_index) : s_host;
        v = fma(-s, __ldg(jhat + g), v);
    }
    out[g] = fma(alpha, v, out[g]);
}

template <bool DUAL>
__global__ void __launch_bounds__(128) curl_f32_kernel(DevField IN, DevField OUT, const float* __restrict__ in,
                                                       double* __restrict__ out, double alpha,
                                                       const double* __restrict__ jhat,
                                                       const double* __restrict__ amp, int amp_index, double s_host,
                                                       int nzmax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int c = blockIdx.z / nzmax;
    const int k = blockIdx.z - c * nzmax;
    if (c == 0)
        curl_comp_f<0, DUAL>(IN, OUT, in, out, alpha, jhat, amp, amp_index, s_host, i, j, k);
    else if (c == 1)
        curl_comp_f<1, DUAL>(IN, OUT, in, out, alpha, jhat, amp, amp_index, s_host, i, j, k);
    else
        curl_comp_f<2, DUAL>(IN, OUT, in, out, alpha, jhat, amp, amp_index, s_host, i, j, k);
}

cudaError_t launch_curl_f32(bool dual, const DevField& IN, const DevField& OUT, const float* in, double* out,
                            double alpha, const double* jhat, const double* amp, int amp_index, double s_host,
                            cudaStream_t s) {
    int nmax[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a) nmax[a] = std::max(nmax[a], OUT.c[c].n[a]);
    if (OUT.total == 0) return cudaSuccess;
    const dim3 grid((nmax[0] + 127) / 128, nmax[1], 3 * nmax[2]);
    if (dual)
        curl_f32_kernel<true><<<grid, 128, 0, s>>>(IN, OUT, in, out, alpha, jhat, amp, amp_index, s_host, nmax[2]);
    else
        curl_f32_kernel<false><<<grid, 128, 0, s>>>(IN, OUT, in, out, alpha, nullptr, nullptr, 0, 0.0, nmax[2]);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ casts
__global__ void cast_d2f_kernel(const double* __restrict__ x, float* __restrict__ y, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = static_cast<float>(x[i]);
}
__global__ void cast_f2d_kernel(const float* __restrict__ x, double* __restrict__ y, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = static_cast<double>(x[i]);
}
cudaError_t launch_cast_d2f(const double* x, float* y, long long n, cudaStream_t s) {
    if (n > 0) cast_d2f_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}
cudaError_t launch_cast_f2d(const float* x, double* y, long long n, cudaStream_t s) {
    if (n > 0) cast_f2d_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Hodge: block Kronecker, FP32
// Same algorithm as the FP64 block kernel (one CTA per tile and component,
// three banded passes in shared memory, atomics to scatter) with split FP32
// tile masses.  The input may be the FP64 state (converted on load).
template <class TIN>
__global__ void __launch_bounds__(256) hodge_block_f32_kernel(HodgeBlockF32Args A, const TIN* __restrict__ x,
                                                              float* __restrict__ y) {
    extern __shared__ float smf[];
    const int c = blockIdx.y;
    const int tile = blockIdx.x;
    const int tx = tile % A.ntile[0];
    const int tyz = tile / A.ntile[0];
    const int ty = tyz % A.ntile[1];
    const int tz = tyz / A.ntile[1];
    const int tpos[3] = {tx, ty, tz};
    int f0[3], L[3], dg[3];
    const float2* gmat[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int slot = A.kinds[c][a] * A.ntile[a] + tpos[a];
        f0[a] = A.tf0[a][slot];
        L[a] = A.tlen[a][slot];
        dg[a] = A.deg[c][a];
        gmat[a] = A.tmat[a] + (long long)slot * kLMax * kLMax;
    }
    const double gam = A.gamma[(tz * A.ntile[1] + ty) * A.ntile[0] + tx];
    float2* Mx = reinterpret_cast<float2*>(smf);
    float2* My = Mx + kLMax * kLMax;
    float2* Mz = My + kLMax * kLMax;
    float* s0 = reinterpret_cast<float*>(Mz + kLMax * kLMax);
    const int Lx = L[0], Ly = L[1], Lz = L[2];
    const int nloc = Lx * Ly * Lz;
    float* s1 = s0 + nloc;
    for (int t = threadIdx.x; t < kLMax * kLMax; t += blockDim.x) {
        Mx[t] = gmat[0][t];
        My[t] = gmat[1][t];
        // gamma folded into z in FP64, then split again
        const float2 z = gmat[2][t];
        const double v = gam * ((double)z.x + (double)z.y);
        const float hi = (float)v;
        Mz[t] = make_float2(hi, (float)(v - (double)hi));
    }
    const DevComp C = A.field.c[c];
    const long long nxy = (long long)C.n[0] * C.n[1];
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {
        const int ii = t % Lx, r = t / Lx, jj = r % Ly, kk = r / Ly;
        s0[t] = to_f(__ldg(x + C.off + (f0[0] + ii) + (long long)C.n[0] * (f0[1] + jj) + nxy * (f0[2] + kk)));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {
        const int ii = t % Lx, row = t - ii;
        const int lo = max(0, ii - dg[0]), hi = min(Lx - 1, ii + dg[0]);
        float acc = 0.0f;
        for (int m = lo; m <= hi; ++m) acc = fma2(Mx[ii * kLMax + m], s0[row + m], acc);
        s1[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {
        const int ii = t % Lx, r = t / Lx, jj = r % Ly, kk = r / Ly;
        const int lo = max(0, jj - dg[1]), hi = min(Ly - 1, jj + dg[1]);
        float acc = 0.0f;
        for (int m = lo; m <= hi; ++m) acc = fma2(My[jj * kLMax + m], s1[(kk * Ly + m) * Lx + ii], acc);
        s0[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {
        const int ii = t % Lx, r = t / Lx, jj = r % Ly, kk = r / Ly;
        const int lo = max(0, kk - dg[2]), hi = min(Lz - 1, kk + dg[2]);
        float acc = 0.0f;
        for (int m = lo; m <= hi; ++m) acc = fma2(Mz[kk * kLMax + m], s0[(m * Ly + jj) * Lx + ii], acc);
        atomicAdd(y + C.off + (f0[0] + ii) + (long long)C.n[0] * (f0[1] + jj) + nxy * (f0[2] + kk), acc);
    }
}

cudaError_t launch_hodge_block_f32(const HodgeBlockF32Args& a, const double* x64, const float* x32, float* y,
                                   cudaStream_t s) {
    const int ntiles = a.ntile[0] * a.ntile[1] * a.ntile[2];
    const size_t smem = 3 * kLMax * kLMax * sizeof(float2) + 2 * (size_t)a.max_nloc * sizeof(float);
    if (ntiles == 0) return cudaSuccess;
    if (x64)
        hodge_block_f32_kernel<double><<<dim3(ntiles, 3), 256, smem, s>>>(a, x64, y);
    else
        hodge_block_f32_kernel<float><<<dim3(ntiles, 3), 256, smem, s>>>(a, x32, y);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ pairing sweeps and fused separable star, FP32
template <int KL>
__device__ __forceinline__ void lu_forward_f(const float* __restrict__ y, float* __restrict__ z, int s, int n,
                                             const float2* __restrict__ fL) {
    float w[KL];
#pragma unroll
    for (int k = 0; k < KL; ++k) w[k] = 0.0f;
#pragma unroll 4
    for (int m = 0; m < n; ++m) {
        float u = y[m * s];
#pragma unroll
        for (int k = KL - 1; k >= 0; --k) {
            const float2 c = fL[m * KL + k];
            u = fmaf(-c.x, w[k], fmaf(-c.y, w[k], u));
        }
#pragma unroll
        for (int k = KL - 1; k > 0; --k) w[k] = w[k - 1];
        w[0] = u;
        z[m * s] = u;
    }
}

template <int KL>
__device__ __forceinline__ void lu_backward_f(const float* __restrict__ z, float* __restrict__ x, int s, int n,
                                              const float2* __restrict__ fU, const float2* __restrict__ fD) {
    float w[KL];
#pragma unroll
    for (int k = 0; k < KL; ++k) w[k] = 0.0f;
#pragma unroll 4
    for (int m = n - 1; m >= 0; --m) {
        const float2 d = fD[m];
        const float zm = z[m * s];
        float u = fmaf(d.x, zm, d.y * zm);
#pragma unroll
        for (int k = KL - 1; k >= 0; --k) {
            const float2 c = fU[m * KL + k];
            u = fmaf(-c.x, w[k], fmaf(-c.y, w[k], u));
        }
#pragma unroll
        for (int k = KL - 1; k > 0; --k) w[k] = w[k - 1];
        w[0] = u;
        x[m * s] = u;
    }
}

template <int D>
__device__ __forceinline__ void mass_line_f(const float* __restrict__ ypad, float* __restrict__ t, int s, int n,
                                            const float2* __restrict__ fM) {
    constexpr int W = 2 * D + 1;
#pragma unroll 4
    for (int m = 0; m < n; ++m) {
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < W; ++q) acc = fma2(fM[m * W + q], ypad[(m + q) * s], acc);
        t[m * s] = acc;
    }
}

// One CTA stages kSolveLines lines (FP64 input converted on load, or FP32),
// optionally applies the banded mass (MASS), then forward/backward LU.
template <int KL, int D, bool MASS, class TIN>
__device__ __forceinline__ void line_body_f(const LineF32Args& A, const TIN* __restrict__ in, float* __restrict__ out,
                                            float* sm) {
    const int c = blockIdx.y;
    const DevComp C = A.field.c[c];
    const int axis = A.axis;
    const int n = C.n[axis];
    const int nlines = C.n[0] * C.n[1] * C.n[2] / n;
    const int l0 = blockIdx.x * kSolveLines;
    if (l0 >= nlines) return;
    const int nl = min(kSolveLines, nlines - l0);
    constexpr int W = 2 * D + 1;
    const int Dp = MASS ? D : 0;
    float2* fL = reinterpret_cast<float2*>(sm);
    float2* fU = fL + n * KL;
    float2* fD = fU + n * KL;
    float2* fM = fD + n;
    float* Sin = reinterpret_cast<float*>(fM + (MASS ? n * W : 0));
    const int np = n + 2 * Dp;
    const int ldin = np | 1, ldout = n | 1;
    float* Sout = Sin + kSolveLines * ldin;
    const int tid = threadIdx.x, nt = blockDim.x;
    const float2* gL = A.L[c];
    const float2* gU = A.U[c];
    const float2* gD = A.dinv[c];
    for (int t = tid; t < n * KL; t += nt) {
        cp_async8f(fL + t, gL + t);
        cp_async8f(fU + t, gU + t);
    }
    for (int t = tid; t < n; t += nt) cp_async8f(fD + t, gD + t);
    if (MASS)
        for (int t = tid; t < n * W; t += nt) cp_async8f(fM + t, A.mass[c] + t);
    const int sL = axis == 0 ? ldin : 1;
    const int sM = axis == 0 ? 1 : kSolveLines;
    if (MASS) {
        for (int t = tid; t < kSolveLines * Dp; t += nt) {
            const int line = t / Dp, q = t - line * Dp;
            Sin[line * sL + q * sM] = 0.0f;
            Sin[line * sL + (n + Dp + q) * sM] = 0.0f;
        }
    }
    const int nx = C.n[0], nxy = C.n[0] * C.n[1];
    const TIN* src = in + C.off;
    if (axis == 0) {
        const TIN* chunk = src + (long long)l0 * n;
        for (int g = tid; g < nl * n; g += nt) {
            const int line = g / n, m = g - line * n;
            Sin[line * ldin + Dp + m] = to_f(__ldg(chunk + g));
        }
    } else if (tid < nl) {
        const int l = l0 + tid;
        const int base = axis == 1 ? (l % nx) + (l / nx) * nxy : l;
        const int stride = axis == 1 ? nx : nxy;
        for (int m = 0; m < n; ++m) Sin[(Dp + m) * kSolveLines + tid] = to_f(__ldg(src + base + m * stride));
    }
    cp_async_wait_all_f();
    __syncthreads();
    const int oL = axis == 0 ? ldout : 1;
    if (tid < nl) {
        if (MASS) {
            mass_line_f<D>(Sin + tid * sL, Sout + tid * oL, sM, n, fM);
            lu_forward_f<KL>(Sout + tid * oL, Sin + tid * sL, sM, n, fL);
        } else {
            lu_forward_f<KL>(Sin + tid * sL, Sout + tid * oL, sM, n, fL);
        }
        // the forward result sits in Sin (MASS) or Sout (no mass); backward into the other buffer
        if (MASS)
            lu_backward_f<KL>(Sin + tid * sL, Sout + tid * oL, sM, n, fU, fD);
        else
            lu_backward_f<KL>(Sout + tid * oL, Sin + tid * sL, sM, n, fU, fD);
    }
    __syncthreads();
    const float* res = MASS ? Sout : Sin;
    const int ldr = MASS ? ldout : ldin;
    float* dst = out + C.off;
    if (axis == 0) {
        float* chunk = dst + (long long)l0 * n;
        for (int g = tid; g < nl * n; g += nt) {
            const int line = g / n, m = g - line * n;
            chunk[g] = res[line * ldr + m];
        }
    } else if (tid < nl) {
        const int l = l0 + tid;
        const int base = axis == 1 ? (l % nx) + (l / nx) * nxy : l;
        const int stride = axis == 1 ? nx : nxy;
#pragma unroll 4
        for (int m = 0; m < n; ++m) dst[base + m * stride] = res[m * kSolveLines + tid];
    }
}

template <int KL, bool MASS, class TIN>
__global__ void __launch_bounds__(kSolveLines) line_f32_kernel(LineF32Args A, const TIN* __restrict__ in,
                                                               float* __restrict__ out) {
    extern __shared__ float smf[];
    if (!MASS) {
        line_body_f<KL, 0, false, TIN>(A, in, out, smf);
        return;
    }
    const int d = A.deg[blockIdx.y];
    if (d == KL - 1)
        line_body_f<KL, KL - 1, true, TIN>(A, in, out, smf);
    else if (d == KL)
        line_body_f<KL, KL, true, TIN>(A, in, out, smf);
    else
        line_body_f<KL, KL + 1, true, TIN>(A, in, out, smf);
}

template <int KL, bool MASS, class TIN>
static cudaError_t launch_line_t(const LineF32Args& a, const TIN* in, float* out, cudaStream_t s) {
    long long maxlines = 0;
    int maxn = 0;
    for (int c = 0; c < 3; ++c) {
        const long long nc = (long long)a.field.c[c].n[0] * a.field.c[c].n[1] * a.field.c[c].n[2];
        const int n = a.field.c[c].n[a.axis];
        if (n > 0) maxlines = std::max(maxlines, nc / n);
        maxn = std::max(maxn, n);
    }
    const int D = MASS ? KL + 1 : 0, W = MASS ? 2 * D + 1 : 0;
    const size_t smem = (size_t)(2 * KL + 1 + W) * maxn * sizeof(float2) +
                        ((size_t)((maxn + 2 * D) | 1) * kSolveLines + (size_t)(maxn | 1) * kSolveLines + 8) *
                            sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(line_f32_kernel<KL, MASS, TIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        attr = true;
    }
    const long long nb = (maxlines + kSolveLines - 1) / kSolveLines;
    if (nb > 0) line_f32_kernel<KL, MASS, TIN><<<dim3((unsigned)nb, 3), kSolveLines, smem, s>>>(a, in, out);
    return cudaGetLastError();
}

template <bool MASS, class TIN>
static cudaError_t launch_line_kl(const LineF32Args& a, int kl, const TIN* in, float* out, cudaStream_t s) {
    switch (kl) {
        case 1: return launch_line_t<1, MASS, TIN>(a, in, out, s);
        case 2: return launch_line_t<2, MASS, TIN>(a, in, out, s);
        case 3: return launch_line_t<3, MASS, TIN>(a, in, out, s);
        case 4: return launch_line_t<4, MASS, TIN>(a, in, out, s);
        case 5: return launch_line_t<5, MASS, TIN>(a, in, out, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_line_f32(const LineF32Args& a, int kl, bool mass, const double* in64, const float* in32, float* out,
                            cudaStream_t s) {
    if (mass) return in64 ? launch_line_kl<true, double>(a, kl, in64, out, s) : launch_line_kl<true, float>(a, kl, in32, out, s);
    return in64 ? launch_line_kl<false, double>(a, kl, in64, out, s) : launch_line_kl<false, float>(a, kl, in32, out, s);
}

}  // namespace smx
