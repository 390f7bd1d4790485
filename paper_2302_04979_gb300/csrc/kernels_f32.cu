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

#include "curl.cuh"
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

// ------------------------------------------------------------------ curl (FP32 differences, FP64 state; curl.cuh)
cudaError_t launch_curl_f32(bool dual, const DevField& IN, const DevField& OUT, const float* in, double* out,
                            double alpha, const double* jhat, const double* amp, int amp_index, double s_host,
                            cudaStream_t s) {
    if (dual) return launch_curl_t<true, float>(IN, OUT, in, out, alpha, jhat, amp, amp_index, s_host, s);
    return launch_curl_t<false, float>(IN, OUT, in, out, alpha, nullptr, nullptr, 0, 0.0, s);
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
// Threads (ii, jj) = (threadIdx.x, threadIdx.y) cover the tile's x-y face
// (L <= 16 per axis) and march along z, so no index is divided at run time.
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
    const int flat = threadIdx.y * 16 + threadIdx.x;
    for (int t = flat; t < kLMax * kLMax; t += 256) {
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
    const int ii = threadIdx.x, jj = threadIdx.y;
    const bool act = ii < Lx && jj < Ly;
    const TIN* xcol = x + C.off + (f0[0] + ii) + (long long)C.n[0] * (f0[1] + jj) + nxy * f0[2];
    if (act)
        for (int kk = 0; kk < Lz; ++kk) s0[(kk * Ly + jj) * Lx + ii] = to_f(__ldg(xcol + nxy * kk));
    __syncthreads();
    if (act) {  // x pass
        const int lo = max(0, ii - dg[0]), hi = min(Lx - 1, ii + dg[0]);
        for (int kk = 0; kk < Lz; ++kk) {
            const float* row = s0 + (kk * Ly + jj) * Lx;
            float acc = 0.0f;
            for (int m = lo; m <= hi; ++m) acc = fma2(Mx[ii * kLMax + m], row[m], acc);
            s1[(kk * Ly + jj) * Lx + ii] = acc;
        }
    }
    __syncthreads();
    if (act) {  // y pass
        const int lo = max(0, jj - dg[1]), hi = min(Ly - 1, jj + dg[1]);
        for (int kk = 0; kk < Lz; ++kk) {
            const float* col = s1 + kk * Ly * Lx + ii;
            float acc = 0.0f;
            for (int m = lo; m <= hi; ++m) acc = fma2(My[jj * kLMax + m], col[m * Lx], acc);
            s0[(kk * Ly + jj) * Lx + ii] = acc;
        }
    }
    __syncthreads();
    if (act) {  // z pass and scatter-add
        float* ycol = y + C.off + (f0[0] + ii) + (long long)C.n[0] * (f0[1] + jj) + nxy * f0[2];
        const float* col = s0 + jj * Lx + ii;
        for (int kk = 0; kk < Lz; ++kk) {
            const int lo = max(0, kk - dg[2]), hi = min(Lz - 1, kk + dg[2]);
            float acc = 0.0f;
            for (int m = lo; m <= hi; ++m) acc = fma2(Mz[kk * kLMax + m], col[m * Ly * Lx], acc);
            atomicAdd(ycol + nxy * kk, acc);
        }
    }
}

cudaError_t launch_hodge_block_f32(const HodgeBlockF32Args& a, const double* x64, const float* x32, float* y,
                                   cudaStream_t s) {
    const int ntiles = a.ntile[0] * a.ntile[1] * a.ntile[2];
    const size_t smem = 3 * kLMax * kLMax * sizeof(float2) + 2 * (size_t)a.max_nloc * sizeof(float);
    if (ntiles == 0) return cudaSuccess;
    if (x64)
        hodge_block_f32_kernel<double><<<dim3(ntiles, 3), dim3(16, 16), smem, s>>>(a, x64, y);
    else
        hodge_block_f32_kernel<float><<<dim3(ntiles, 3), dim3(16, 16), smem, s>>>(a, x32, y);
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

namespace smx {

// ------------------------------------------------------------------ dense mode products (mixed step)
// Along one axis, every line of a component is multiplied by a precomputed
// dense n x n operator B (FP64 values as FP32 (hi, lo) pairs): B = A^{-1}
// (pairing solve) or A^{-1} M (fused separable Hodge star).  Unlike the
// banded recurrence this has no dependency chain: each output is an
// independent dot product, so the pass runs at the FP32 throughput of the
// CUDA cores instead of the latency of a serial recurrence.
// CTA: kModeLines lines staged as T[j][line] in shared memory, B (transposed)
// in shared memory.
constexpr int kModeLines = 32;       // lines per CTA
constexpr int kModeLd = 36;          // tile row stride (floats): 16-byte aligned, spreads banks
constexpr int kModeLineGroups = 8;   // threads along lines: 4 lines each (one float4 of the tile)
constexpr int kModeOutGroups = 32;   // threads along outputs: outputs i = og + 32 r

// Register-blocked: thread (lg, og) accumulates 4 lines x NOUT outputs; per
// entry j it reads one float4 of the staged tile T[j][4 lg .. 4 lg + 3] and
// NOUT split coefficients Bt[j][og + 32 r] (shared by the 8 threads of a
// warp with the same og), then issues 8 NOUT FMAs.  Rows i >= n read zero
// padding and are not stored.
template <class TIN, int NOUT>
__global__ void __launch_bounds__(kModeLineGroups* kModeOutGroups) mode_f32_kernel(ModeF32Args A,
                                                                                   const TIN* __restrict__ in,
                                                                                   float* __restrict__ out) {
    extern __shared__ float smf[];
    const int c = blockIdx.y;
    const DevComp C = A.field.c[c];
    const int axis = A.axis;
    const int n = C.n[axis];
    const int nlines = C.n[0] * C.n[1] * C.n[2] / n;
    const int l0 = blockIdx.x * kModeLines;
    if (l0 >= nlines) return;
    const int nl = min(kModeLines, nlines - l0);
    constexpr int NPAD = kModeOutGroups * NOUT;                 // padded output count
    float2* Bt = reinterpret_cast<float2*>(smf);                // n x NPAD (transposed, zero padded)
    float* T = reinterpret_cast<float*>(Bt + n * NPAD);         // n x kModeLd (16-byte aligned rows)
    const int tid = threadIdx.x, nt = blockDim.x;
    const float2* Bg = A.B[c];
    for (int t = tid; t < n * NPAD; t += nt) {
        const int j = t / NPAD, i = t - j * NPAD;
        if (i < n)
            cp_async8f(Bt + t, Bg + i * n + j);
        else
            Bt[t] = make_float2(0.0f, 0.0f);
    }
    const int nx = C.n[0], nxy = C.n[0] * C.n[1];
    const TIN* src = in + C.off;
    if (axis == 0) {
        const TIN* chunk = src + (long long)l0 * n;
        for (int g = tid; g < nl * n; g += nt) {
            const int line = g / n, m = g - line * n;
            T[m * kModeLd + line] = to_f(__ldg(chunk + g));
        }
    } else {
        const int stride = axis == 1 ? nx : nxy;
        for (int g = tid; g < nl * n; g += nt) {
            const int m = g / nl, w = g - m * nl;
            const int l = l0 + w;
            const int base = axis == 1 ? (l % nx) + (l / nx) * nxy : l;
            T[m * kModeLd + w] = to_f(__ldg(src + base + m * stride));
        }
    }
    if (nl < kModeLines)  // keep the unused tile columns finite
        for (int g = tid; g < (kModeLines - nl) * n; g += nt) {
            const int m = g / (kModeLines - nl), w = nl + g - m * (kModeLines - nl);
            T[m * kModeLd + w] = 0.0f;
        }
    cp_async_wait_all_f();
    __syncthreads();
    const int lg = tid % kModeLineGroups, og = tid / kModeLineGroups;
    float acc[4][NOUT];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < NOUT; ++r) acc[q][r] = 0.0f;
#pragma unroll 2
    for (int j = 0; j < n; ++j) {
        const float4 t = *reinterpret_cast<const float4*>(T + j * kModeLd + 4 * lg);
        const float2* brow = Bt + j * NPAD + og;
#pragma unroll
        for (int r = 0; r < NOUT; ++r) {
            const float2 bb = brow[r * kModeOutGroups];
            acc[0][r] = fma2(bb, t.x, acc[0][r]);
            acc[1][r] = fma2(bb, t.y, acc[1][r]);
            acc[2][r] = fma2(bb, t.z, acc[2][r]);
            acc[3][r] = fma2(bb, t.w, acc[3][r]);
        }
    }
    __syncthreads();  // T is reused for the outputs
#pragma unroll
    for (int r = 0; r < NOUT; ++r) {
        const int i = og + r * kModeOutGroups;
        if (i < n)
            *reinterpret_cast<float4*>(T + i * kModeLd + 4 * lg) =
                make_float4(acc[0][r], acc[1][r], acc[2][r], acc[3][r]);
    }
    __syncthreads();
    float* dst = out + C.off;
    if (axis == 0) {
        float* chunk = dst + (long long)l0 * n;
        for (int g = tid; g < nl * n; g += nt) {
            const int line = g / n, m = g - line * n;
            chunk[g] = T[m * kModeLd + line];
        }
    } else {
        const int stride = axis == 1 ? nx : nxy;
        for (int g = tid; g < nl * n; g += nt) {
            const int m = g / nl, ww = g - m * nl;
            const int l = l0 + ww;
            const int base = axis == 1 ? (l % nx) + (l / nx) * nxy : l;
            dst[base + m * stride] = T[m * kModeLd + ww];
        }
    }
}

template <int NOUT>
static cudaError_t launch_mode_t(const ModeF32Args& a, const double* in64, const float* in32, float* out, int maxn,
                                 long long nb, cudaStream_t s) {
    const size_t smem = (size_t)maxn * kModeOutGroups * NOUT * sizeof(float2) + (size_t)maxn * kModeLd * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(mode_f32_kernel<double, NOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(mode_f32_kernel<float, NOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    const dim3 grid((unsigned)nb, 3);
    if (in64)
        mode_f32_kernel<double, NOUT><<<grid, kModeLineGroups * kModeOutGroups, smem, s>>>(a, in64, out);
    else
        mode_f32_kernel<float, NOUT><<<grid, kModeLineGroups * kModeOutGroups, smem, s>>>(a, in32, out);
    return cudaGetLastError();
}

cudaError_t launch_mode_f32(const ModeF32Args& a, const double* in64, const float* in32, float* out, cudaStream_t s) {
    long long maxlines = 0;
    int maxn = 0;
    for (int c = 0; c < 3; ++c) {
        const long long nc = (long long)a.field.c[c].n[0] * a.field.c[c].n[1] * a.field.c[c].n[2];
        const int n = a.field.c[c].n[a.axis];
        if (n > 0) maxlines = std::max(maxlines, nc / n);
        maxn = std::max(maxn, n);
    }
    if (maxn > kModeMaxN) return cudaErrorInvalidValue;
    const long long nb = (maxlines + kModeLines - 1) / kModeLines;
    if (nb == 0) return cudaSuccess;
    switch ((maxn + kModeOutGroups - 1) / kModeOutGroups) {
        case 1: return launch_mode_t<1>(a, in64, in32, out, maxn, nb, s);
        case 2: return launch_mode_t<2>(a, in64, in32, out, maxn, nb, s);
        case 3: return launch_mode_t<3>(a, in64, in32, out, maxn, nb, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace smx
