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

#include "batch.cuh"
#include "convert.cuh"
#include "curl.cuh"
#include "pdl.cuh"
#include "internal.h"

namespace smx {

__device__ __forceinline__ float fma2(float2 c, float x, float acc) { return fmaf(c.x, x, fmaf(c.y, x, acc)); }

// A compensated FP32 sum of products (a dot product in the manner of Ogita, Rump and Oishi's
// Dot2): s carries the running sum, e the rounding errors of every product (exact, by an FMA)
// and every addition (exact, by TwoSum) plus the small lo-coefficient terms, so the result
// s + e is as accurate as a sum computed in twice the precision, rounded once.  The _rn
// intrinsics keep the compiler from contracting a product and a sum into one FMA.
struct Acc2 {
    float s, e;
};
__device__ __forceinline__ void acc2_add(Acc2& a, float2 c, float x) {
    const float p = __fmul_rn(c.x, x);
    const float pe = __fmaf_rn(c.x, x, -p);  // the product's rounding error, exactly
    const float t = __fadd_rn(a.s, p);
    const float bb = __fsub_rn(t, a.s);
    const float se = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bb)), __fsub_rn(p, bb));  // the sum's, exactly
    a.e = __fadd_rn(a.e, __fadd_rn(se, __fmaf_rn(c.y, x, pe)));
    a.s = t;
}
__device__ __forceinline__ float acc2_value(const Acc2& a) { return __fadd_rn(a.s, a.e); }

// The block Hodge passes' accumulator: plain FMAs, or the compensated sum above (COMP).
template <bool COMP>
struct TileAcc;
template <>
struct TileAcc<false> {
    float v = 0.0f;
    __device__ __forceinline__ void add(float2 c, float x) { v = fma2(c, x, v); }
    __device__ __forceinline__ float value() const { return v; }
};
template <>
struct TileAcc<true> {
    Acc2 a{0.0f, 0.0f};
    __device__ __forceinline__ void add(float2 c, float x) { acc2_add(a, c, x); }
    __device__ __forceinline__ float value() const { return acc2_value(a); }
};

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8f(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16f(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all_f() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ float to_f(double v) { return d2f_rn(v); }  // integer pipe (convert.cuh)
__device__ __forceinline__ float to_f(float v) { return v; }

// ------------------------------------------------------------------ curl (FP32 differences, FP64 state; curl.cuh)
cudaError_t launch_curl_f32(bool dual, const DevField& IN, const DevField& OUT, const float* in, double* out,
                            double alpha, const double* jhat, const double* amp, int amp_index, double s_host,
                            cudaStream_t s, double* zero) {
    if (dual) return launch_curl_t<true, float>(IN, OUT, in, out, alpha, jhat, amp, amp_index, s_host, s, zero);
    return launch_curl_t<false, float>(IN, OUT, in, out, alpha, nullptr, nullptr, 0, 0.0, s, zero);
}

// ------------------------------------------------------------------ casts
__global__ void cast_d2f_kernel(const double* __restrict__ x, float* __restrict__ y, long long n) {
    pdl_wait();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = d2f_rn(x[i]);
}
__global__ void cast_f2d_kernel(const float* __restrict__ x, double* __restrict__ y, long long n) {
    pdl_wait();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = f2d_exact(x[i]);
}
cudaError_t launch_cast_d2f(const double* x, float* y, long long n, cudaStream_t s) {
    if (n > 0) return launch_k(cast_d2f_kernel, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, x, y, n);
    return cudaGetLastError();
}
cudaError_t launch_cast_f2d(const float* x, double* y, long long n, cudaStream_t s) {
    if (n > 0) return launch_k(cast_f2d_kernel, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, x, y, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ refinement residual, FP64
// One thread per entry: acc = sum_q A(m, m - kl + q) x(m - kl + q) along the
// entry's line (the FP64 pipe, 2 kl + 1 FMAs), out = acc or y - acc.  Reads
// along y and z are coalesced across threads (consecutive x); the input must
// not alias the output.
template <class TIN>
__device__ __forceinline__ void band_apply_entry(const BandApplyArgs& A, long long idx, const TIN* __restrict__ in,
                                                 const double* __restrict__ y, double* __restrict__ out) {
    if (idx < A.field.total) {
        int c = 0;
        while (c < 2 && idx >= A.field.c[c + 1].off) ++c;
        const DevComp C = A.field.c[c];
        const long long loc = idx - C.off;
        const int i = (int)(loc % C.n[0]);
        const long long r = loc / C.n[0];
        const int j = (int)(r % C.n[1]), k = (int)(r / C.n[1]);
        const int m = A.axis == 0 ? i : (A.axis == 1 ? j : k);
        const int n = C.n[A.axis];
        const long long st = A.axis == 0 ? 1 : (A.axis == 1 ? (long long)C.n[0] : (long long)C.n[0] * C.n[1]);
        const int W = 2 * A.kl + 1;
        const double* brow = A.band[c] + (long long)m * W;
        double acc = 0.0;
        for (int q = 0; q < W; ++q) {
            const int mm = m - A.kl + q;
            if (mm >= 0 && mm < n) acc = fma(__ldg(brow + q), widen(in[idx + (long long)(mm - m) * st]), acc);
        }
        out[idx] = y ? y[idx] - acc : acc;
    }
}

template <class TIN>
__global__ void __launch_bounds__(256) band_apply_kernel(BandApplyArgs A, const TIN* __restrict__ in,
                                                         const double* __restrict__ y, double* __restrict__ out) {
    pdl_wait();
    band_apply_entry<TIN>(A, blockIdx.x * 256ll + threadIdx.x, in, y, out);
    pdl_trigger();
}

cudaError_t launch_band_apply(const BandApplyArgs& a, const double* in64, const float* in32, const double* y,
                              double* out, cudaStream_t s) {
    const long long n = a.field.total;
    if (n <= 0) return cudaGetLastError();
    const dim3 grid((unsigned)((n + 255) / 256));
    if (in64) return launch_k(band_apply_kernel<double>, grid, dim3(256), 0, s, a, in64, y, out);
    return launch_k(band_apply_kernel<float>, grid, dim3(256), 0, s, a, in32, y, out);
}

__global__ void refine_sum_kernel(const float* __restrict__ x0, const float* __restrict__ c, double* __restrict__ out,
                                  long long n) {
    pdl_wait();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = f2d_exact(x0[i]) + f2d_exact(c[i]);
    pdl_trigger();
}

cudaError_t launch_refine_sum(const float* x0, const float* c, double* out, long long n, cudaStream_t s) {
    if (n > 0) return launch_k(refine_sum_kernel, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, x0, c, out, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Hodge: block Kronecker, FP32
// Same algorithm as the FP64 block kernel (one CTA per tile and component,
// three banded passes in shared memory, atomics to scatter) with split FP32
// tile masses.  The input may be the FP64 state (converted on load).
// Threads (ii, jj) = (threadIdx.x, threadIdx.y) cover the tile's x-y face
// (L <= 16 per axis) and march along z, so no index is divided at run time.
// One (component, tile): threads (ii, jj) of the tile face, flat index `flat` of `nthreads`.
template <class TIN, bool COMP>
__device__ __forceinline__ void hodge_block_f32_tile(const HodgeBlockF32Args& A, int c, int tile,
                                                     const TIN* __restrict__ x, double* __restrict__ y, float* smf,
                                                     int ii, int jj, int flat, int nthreads) {
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
    // tile masses with row stride kLd = kLMax + 1: the x pass reads rows ii of Mx at the
    // same column across a warp, which an unpadded 16-entry stride puts on one bank
    constexpr int kLd = kLMax + 1;
    float2* Mx = reinterpret_cast<float2*>(smf);
    float2* My = Mx + kLMax * kLd;
    float2* Mz = My + kLMax * kLd;
    float* s0 = reinterpret_cast<float*>(Mz + kLMax * kLd);
    const int Lx = L[0], Ly = L[1], Lz = L[2];
    const int nloc = Lx * Ly * Lz;
    float* s1 = s0 + nloc;
    for (int t = flat; t < kLMax * kLMax; t += nthreads) {
        const int d = (t / kLMax) * kLd + t % kLMax;
        Mx[d] = gmat[0][t];
        My[d] = gmat[1][t];
        // gamma folded into z in FP64, then split again
        const float2 z = gmat[2][t];
        const double v = gam * ((double)z.x + (double)z.y);
        const float hi = (float)v;
        Mz[d] = make_float2(hi, (float)(v - (double)hi));
    }
    const DevComp C = A.field.c[c];
    const long long nxy = (long long)C.n[0] * C.n[1];
    const bool act = ii < Lx && jj < Ly;
    const TIN* xcol = x + C.off + (f0[0] + ii) + (long long)C.n[0] * (f0[1] + jj) + nxy * f0[2];
    if (act)
        for (int kk = 0; kk < Lz; ++kk) s0[(kk * Ly + jj) * Lx + ii] = to_f(__ldg(xcol + nxy * kk));
    __syncthreads();
    // kU of a thread's Lz outputs are accumulated side by side (independent FMA chains)
    constexpr int kU = 4;
    const int plane = Ly * Lx;
    if (act) {  // x pass
        const int lo = max(0, ii - dg[0]), hi = min(Lx - 1, ii + dg[0]);
        for (int k0 = 0; k0 < Lz; k0 += kU) {
            TileAcc<COMP> acc[kU];
            for (int m = lo; m <= hi; ++m) {
                const float2 c = Mx[ii * kLd + m];
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (k0 + u < Lz) acc[u].add(c, s0[(k0 + u) * plane + jj * Lx + m]);
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (k0 + u < Lz) s1[(k0 + u) * plane + jj * Lx + ii] = acc[u].value();
        }
    }
    __syncthreads();
    if (act) {  // y pass
        const int lo = max(0, jj - dg[1]), hi = min(Ly - 1, jj + dg[1]);
        for (int k0 = 0; k0 < Lz; k0 += kU) {
            TileAcc<COMP> acc[kU];
            for (int m = lo; m <= hi; ++m) {
                const float2 c = My[jj * kLd + m];
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (k0 + u < Lz) acc[u].add(c, s1[(k0 + u) * plane + m * Lx + ii]);
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (k0 + u < Lz) s0[(k0 + u) * plane + jj * Lx + ii] = acc[u].value();
        }
    }
    __syncthreads();
    if (act) {  // z pass and scatter-add, over the union of the kU rows' bands (zeros outside a band)
        double* ycol = y + C.off + (f0[0] + ii) + (long long)C.n[0] * (f0[1] + jj) + nxy * f0[2];
        const float* col = s0 + jj * Lx + ii;
        for (int k0 = 0; k0 < Lz; k0 += kU) {
            TileAcc<COMP> acc[kU];
            const int lo = max(0, k0 - dg[2]), hi = min(Lz - 1, k0 + kU - 1 + dg[2]);
            for (int m = lo; m <= hi; ++m) {
                const float v = col[m * plane];
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (k0 + u < Lz) acc[u].add(Mz[(k0 + u) * kLd + m], v);
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (k0 + u < Lz) atomicAdd(ycol + nxy * (k0 + u), f2d_exact(acc[u].value()));
        }
    }
}

template <class TIN>
__global__ void __launch_bounds__(256) hodge_block_f32_kernel(HodgeBlockF32Args A, const TIN* __restrict__ x,
                                                              double* __restrict__ y) {
    extern __shared__ float smf[];
    pdl_wait();
    const int flat = threadIdx.y * blockDim.x + threadIdx.x, nthreads = blockDim.x * blockDim.y;
    if (A.compensated)
        hodge_block_f32_tile<TIN, true>(A, blockIdx.y, blockIdx.x, x, y, smf, threadIdx.x, threadIdx.y, flat, nthreads);
    else
        hodge_block_f32_tile<TIN, false>(A, blockIdx.y, blockIdx.x, x, y, smf, threadIdx.x, threadIdx.y, flat, nthreads);
}

cudaError_t launch_hodge_block_f32(const HodgeBlockF32Args& a, const double* x64, const float* x32, double* y,
                                   cudaStream_t s) {
    const int ntiles = a.ntile[0] * a.ntile[1] * a.ntile[2];
    const size_t smem = 3 * kLMax * (kLMax + 1) * sizeof(float2) + 2 * (size_t)a.max_nloc * sizeof(float);
    if (ntiles == 0) return cudaSuccess;
    // one thread per (x, y) position of the largest tile face: no idle rows or columns of a 16 x 16 block
    const dim3 block(a.max_len[0], a.max_len[1]);
    if (x64)
        return launch_k(hodge_block_f32_kernel<double>, dim3(ntiles, 3), block, smem, s, a, x64, y);
    return launch_k(hodge_block_f32_kernel<float>, dim3(ntiles, 3), block, smem, s, a, x32, y);
}

// ------------------------------------------------------------------ Hodge: quadrature, FP32
// Curved map or pointwise material (the FP64 kernel's algorithm): per element,
// interpolate the three components at the q^3 Gauss points by sum
// factorisation, apply the symmetric metric G (weight, material and 2-form
// pullback folded in), integrate back, scatter-add into the FP32 output with
// atomics.  One CTA per element.  The basis values and the metric are FP32
// (hi, lo) pairs, so the operator keeps FP64 accuracy and only the data is
// rounded to FP32, as in the block-Kronecker kernel.
constexpr int kQuadF32Threads = 128;

// One element, all `nt` threads of the CTA (tid = thread index).
__device__ __forceinline__ void hodge_quad_f32_element(const HodgeQuadF32Args& A, int e, const double* __restrict__ x,
                                                       double* __restrict__ y, float* smq, int tid, int nt) {
    const int ex = e % A.nel[0], exy = e / A.nel[0], ey = exy % A.nel[1], ez = exy / A.nel[1];
    const int el[3] = {ex, ey, ez};
    const int qx = A.q[0], qy = A.q[1], qz = A.q[2];
    const int Qe = qx * qy * qz;
    float2* Bv = reinterpret_cast<float2*>(smq);  // 3 axes x 8 points x kRMax (hi, lo)
    float* U = reinterpret_cast<float*>(Bv + 3 * 8 * kRMax);  // 3 * Qe values at the Gauss points
    float* T1 = U + 3 * Qe;                  // scratch, <= Qe * kRMax
    float* T2 = T1 + Qe * kRMax;             // scratch, <= Qe * kRMax
    float* X = T2 + Qe * kRMax;              // local coefficients, <= kRMax^3
    auto load_basis = [&](int c) {
        for (int t = tid; t < 3 * 8 * kRMax; t += nt) {
            const int a = t / (8 * kRMax), rem = t % (8 * kRMax), qp = rem / kRMax, r = rem % kRMax;
            if (qp < A.q[a])
                Bv[t] = __ldg(A.bval[a] + (((long long)A.kinds[c][a] * A.nel[a] + el[a]) * A.q[a] + qp) * kRMax + r);
        }
    };
    for (int c = 0; c < 3; ++c) {
        const DevComp C = A.field.c[c];
        const int rx = A.deg[c][0] + 1, ry = A.deg[c][1] + 1, rz = A.deg[c][2] + 1;
        load_basis(c);
        for (int t = tid; t < rx * ry * rz; t += nt) {
            const int r0 = t % rx, rr = t / rx, r1 = rr % ry, r2 = rr / ry;
            const int gi = el[0] + r0 + A.koff[c][0], gj = el[1] + r1 + A.koff[c][1], gk = el[2] + r2 + A.koff[c][2];
            float v = 0.0f;
            if (gi >= 0 && gi < C.n[0] && gj >= 0 && gj < C.n[1] && gk >= 0 && gk < C.n[2])
                v = to_f(__ldg(x + C.off + gi + (long long)C.n[0] * (gj + (long long)C.n[1] * gk)));
            X[t] = v;
        }
        __syncthreads();
        const float2* Bx = Bv;
        const float2* By = Bv + 8 * kRMax;
        const float2* Bz = Bv + 16 * kRMax;
        for (int t = tid; t < rz * ry * qx; t += nt) {  // T1[r2][r1][qx]
            const int a = t % qx, rr = t / qx;
            float acc = 0.0f;
            for (int r0 = 0; r0 < rx; ++r0) acc = fma2(Bx[a * kRMax + r0], X[rr * rx + r0], acc);
            T1[t] = acc;
        }
        __syncthreads();
        for (int t = tid; t < rz * qy * qx; t += nt) {  // T2[r2][qy][qx]
            const int a = t % qx, rr = t / qx, b = rr % qy, r2 = rr / qy;
            float acc = 0.0f;
            for (int r1 = 0; r1 < ry; ++r1) acc = fma2(By[b * kRMax + r1], T1[(r2 * ry + r1) * qx + a], acc);
            T2[t] = acc;
        }
        __syncthreads();
        for (int t = tid; t < Qe; t += nt) {  // U_c[qz][qy][qx]
            const int ab = t % (qx * qy), g = t / (qx * qy);
            float acc = 0.0f;
            for (int r2 = 0; r2 < rz; ++r2) acc = fma2(Bz[g * kRMax + r2], T2[r2 * qx * qy + ab], acc);
            U[c * Qe + t] = acc;
        }
        __syncthreads();
    }
    for (int t = tid; t < Qe; t += nt) {  // metric at each Gauss point
        const int a = t % qx, rr = t / qx, b = rr % qy, g = rr / qy;
        const long long qi = ((long long)(ez * qz + g) * A.Qn[1] + (ey * qy + b)) * A.Qn[0] + (ex * qx + a);
        const float2 g00 = __ldg(A.G + qi), g01 = __ldg(A.G + A.Qtot + qi), g02 = __ldg(A.G + 2 * A.Qtot + qi);
        const float2 g11 = __ldg(A.G + 3 * A.Qtot + qi), g12 = __ldg(A.G + 4 * A.Qtot + qi);
        const float2 g22 = __ldg(A.G + 5 * A.Qtot + qi);
        const float u0 = U[t], u1 = U[Qe + t], u2 = U[2 * Qe + t];
        U[t] = fma2(g00, u0, fma2(g01, u1, fma2(g02, u2, 0.0f)));
        U[Qe + t] = fma2(g01, u0, fma2(g11, u1, fma2(g12, u2, 0.0f)));
        U[2 * Qe + t] = fma2(g02, u0, fma2(g12, u1, fma2(g22, u2, 0.0f)));
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
        const DevComp C = A.field.c[c];
        const int rx = A.deg[c][0] + 1, ry = A.deg[c][1] + 1, rz = A.deg[c][2] + 1;
        load_basis(c);
        __syncthreads();
        const float2* Bx = Bv;
        const float2* By = Bv + 8 * kRMax;
        const float2* Bz = Bv + 16 * kRMax;
        for (int t = tid; t < rz * qy * qx; t += nt) {  // T2[r2][qy][qx] = sum_qz Bz[qz][r2] V[qz][qy][qx]
            const int ab = t % (qx * qy), r2 = t / (qx * qy);
            float acc = 0.0f;
            for (int g = 0; g < qz; ++g) acc = fma2(Bz[g * kRMax + r2], U[c * Qe + g * qx * qy + ab], acc);
            T2[t] = acc;
        }
        __syncthreads();
        for (int t = tid; t < rz * ry * qx; t += nt) {  // T1[r2][r1][qx] = sum_qy By[qy][r1] T2[r2][qy][qx]
            const int a = t % qx, rr = t / qx, r1 = rr % ry, r2 = rr / ry;
            float acc = 0.0f;
            for (int b = 0; b < qy; ++b) acc = fma2(By[b * kRMax + r1], T2[(r2 * qy + b) * qx + a], acc);
            T1[t] = acc;
        }
        __syncthreads();
        for (int t = tid; t < rx * ry * rz; t += nt) {  // sum_qx Bx[qx][r0] T1[r2][r1][qx], scatter-add
            const int r0 = t % rx, rr = t / rx, r1 = rr % ry, r2 = rr / ry;
            const int gi = el[0] + r0 + A.koff[c][0], gj = el[1] + r1 + A.koff[c][1], gk = el[2] + r2 + A.koff[c][2];
            if (gi >= 0 && gi < C.n[0] && gj >= 0 && gj < C.n[1] && gk >= 0 && gk < C.n[2]) {
                float acc = 0.0f;
                for (int a = 0; a < qx; ++a) acc = fma2(Bx[a * kRMax + r0], T1[rr * qx + a], acc);
                atomicAdd(y + C.off + gi + (long long)C.n[0] * (gj + (long long)C.n[1] * gk), f2d_exact(acc));
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kQuadF32Threads) hodge_quad_f32_kernel(HodgeQuadF32Args A,
                                                                        const double* __restrict__ x,
                                                                        double* __restrict__ y) {
    extern __shared__ float smq[];
    pdl_wait();
    hodge_quad_f32_element(A, blockIdx.x, x, y, smq, threadIdx.x, blockDim.x);
}

cudaError_t launch_hodge_quad_f32(const HodgeQuadF32Args& a, const double* x, double* y, cudaStream_t s) {
    const int nel = a.nel[0] * a.nel[1] * a.nel[2];
    const int Qe = a.q[0] * a.q[1] * a.q[2];
    const size_t smem =
        3 * 8 * kRMax * sizeof(float2) + (3 * Qe + 2 * Qe * kRMax + kRMax * kRMax * kRMax) * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(hodge_quad_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    if (nel > 0) return launch_k(hodge_quad_f32_kernel, dim3(nel), dim3(kQuadF32Threads), smem, s, a, x, y);
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

// One warp stages kSolveLines lines (line block lb of component c; FP64 input
// converted on load, or FP32), optionally applies the banded mass (MASS), then
// forward/backward LU.  tid is the lane.
template <int KL, int D, bool MASS, class TIN>
__device__ __forceinline__ void line_body_f(const LineF32Args& A, int c, int lb, const TIN* __restrict__ in,
                                            float* __restrict__ out, float* sm, int tid) {
    const DevComp C = A.field.c[c];
    const int axis = A.axis;
    const int n = C.n[axis];
    if (n <= 0) return;
    const int nlines = C.n[0] * C.n[1] * C.n[2] / n;
    const int l0 = lb * kSolveLines;
    if (l0 >= nlines) return;
    const int nl = min(kSolveLines, nlines - l0);
    constexpr int W = 2 * D + 1;
    constexpr int Dp = MASS ? D : 0;
    float2* fL = reinterpret_cast<float2*>(sm);
    float2* fU = fL + n * KL;
    float2* fD = fU + n * KL;
    float2* fM = fD + n;
    float* Sin = reinterpret_cast<float*>(fM + (MASS ? n * W : 0));
    const int np = n + 2 * Dp;
    const int ldin = np | 1, ldout = n | 1;
    float* Sout = Sin + kSolveLines * ldin;
    constexpr int nt = kSolveLines;
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
    if constexpr (Dp > 0) {  // zero pads (no pads, and no loop, without the mass)
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
        for (int line = 0; line < nl; ++line)  // no run-time division per entry
            for (int m = tid; m < n; m += nt) Sin[line * ldin + Dp + m] = to_f(__ldg(chunk + line * n + m));
    } else if (tid < nl) {
        const int l = l0 + tid;
        const int base = axis == 1 ? (l % nx) + (l / nx) * nxy : l;
        const int stride = axis == 1 ? nx : nxy;
        for (int m = 0; m < n; ++m) Sin[(Dp + m) * kSolveLines + tid] = to_f(__ldg(src + base + m * stride));
    }
    cp_async_wait_all_f();
    __syncwarp();
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
    __syncwarp();
    const float* res = MASS ? Sout : Sin;
    const int ldr = MASS ? ldout : ldin;
    float* dst = out + C.off;
    if (axis == 0) {
        float* chunk = dst + (long long)l0 * n;
        for (int line = 0; line < nl; ++line)
            for (int m = tid; m < n; m += nt) chunk[line * n + m] = res[line * ldr + m];
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
    pdl_wait();
    const int c = blockIdx.y, lb = blockIdx.x, tid = threadIdx.x;
    if (!MASS) {
        line_body_f<KL, 0, false, TIN>(A, c, lb, in, out, smf, tid);
        return;
    }
    const int d = A.deg[c];
    if (d == KL - 1)
        line_body_f<KL, KL - 1, true, TIN>(A, c, lb, in, out, smf, tid);
    else if (d == KL)
        line_body_f<KL, KL, true, TIN>(A, c, lb, in, out, smf, tid);
    else
        line_body_f<KL, KL + 1, true, TIN>(A, c, lb, in, out, smf, tid);
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
    if (nb > 0)
        return launch_k(line_f32_kernel<KL, MASS, TIN>, dim3((unsigned)nb, 3), dim3(kSolveLines), smem, s, a, in, out);
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
__global__ void __launch_bounds__(kModeLineGroups* kModeOutGroups) mode_f32_kernel(ModeF32Args A, const TIN* in,
                                                                                   float* out) {
    extern __shared__ float smf[];
    pdl_wait();
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
    // the table is already transposed and padded: one contiguous copy, 16 bytes per cp.async
    const float2* Bg = A.B[c];
    for (int t = tid; t < n * NPAD / 2; t += nt) cp_async16f(Bt + 2 * t, Bg + 2 * t);
    const int nx = C.n[0], nxy = C.n[0] * C.n[1];
    const TIN* src = in + C.off;
    // warps along lines (x sweep) or along entries (y, z), lanes the other way: no run-time
    // division per entry (kModeLines = 32 lines: one per lane)
    const int wq = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
    static_assert(kModeLines == 32, "one line per lane");
    if (axis == 0) {
        const TIN* chunk = src + (long long)l0 * n;
        for (int line = wq; line < nl; line += nwarps)
            for (int m = lane; m < n; m += 32) T[m * kModeLd + line] = to_f(chunk[line * n + m]);
    } else {
        const int stride = axis == 1 ? nx : nxy;
        const int l = l0 + lane;
        const int base = axis == 1 ? (l % nx) + (l / nx) * nxy : l;
        for (int m = wq; m < n; m += nwarps) T[m * kModeLd + lane] = lane < nl ? to_f(src[base + m * stride]) : 0.0f;
    }
    if (axis == 0 && nl < kModeLines)  // keep the unused tile columns finite
        for (int m = wq; m < n; m += nwarps)
            if (lane >= nl) T[m * kModeLd + lane] = 0.0f;
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
        for (int line = wq; line < nl; line += nwarps)
            for (int m = lane; m < n; m += 32) chunk[line * n + m] = T[m * kModeLd + line];
    } else if (lane < nl) {
        const int stride = axis == 1 ? nx : nxy;
        const int l = l0 + lane;
        const int base = axis == 1 ? (l % nx) + (l / nx) * nxy : l;
        for (int m = wq; m < n; m += nwarps) dst[base + m * stride] = T[m * kModeLd + lane];
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
        return launch_k(mode_f32_kernel<double, NOUT>, grid, dim3(kModeLineGroups * kModeOutGroups), smem, s, a, in64,
                        out);
    return launch_k(mode_f32_kernel<float, NOUT>, grid, dim3(kModeLineGroups * kModeOutGroups), smem, s, a, in32, out);
}

int mode_f32_npad(int maxn) { return kModeOutGroups * ((maxn + kModeOutGroups - 1) / kModeOutGroups); }

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
    if (a.npad != mode_f32_npad(maxn)) return cudaErrorInvalidValue;
    switch ((maxn + kModeOutGroups - 1) / kModeOutGroups) {
        case 1: return launch_mode_t<1>(a, in64, in32, out, maxn, nb, s);
        case 2: return launch_mode_t<2>(a, in64, in32, out, maxn, nb, s);
        case 3: return launch_mode_t<3>(a, in64, in32, out, maxn, nb, s);
        case 4: return launch_mode_t<4>(a, in64, in32, out, maxn, nb, s);
        case 5: return launch_mode_t<5>(a, in64, in32, out, maxn, nb, s);
        default: return cudaErrorInvalidValue;
    }
}


// ------------------------------------------------------------------ batched cavities, refined mixed step
// One persistent (cooperative) launch per step for many cavities in the refined
// mixed form (the phases are listed with BatchRefCavity).  Each phase walks a
// flat list of (cavity, unit) items: whole-CTA units (curl chunks, zeroing, FP32
// mass tiles or elements, chunks of 2048 entries for the residual and the sum)
// or line units (kSolveLines lines, one warp with its own shared-memory
// staging).  The work of a unit is the device function of the single-cavity
// kernel; the line sweeps are the banded FP32 recurrences.

template <bool DUAL>
__device__ __noinline__ void ref_curl(const BatchRefCavity& K, int unit, const double* in, double* out, double alpha,
                                      const double* jhat, const double* amp, int step) {
    const int c = (unit >> 28) & 3, zc = (unit >> 14) & 0x3FFF, pb = unit & 0x3FFF;
    const DevField& IN = DUAL ? K.fH : K.fE;
    const DevField& OUT = DUAL ? K.fD : K.fB;
    const int p = pb * kCurlThreads + threadIdx.x;
    if (c == 0)
        curl_plane_comp<0, DUAL, double>(IN, OUT, in, out, alpha, jhat, amp, step, 0.0, p, zc * kCurlKz, nullptr);
    else if (c == 1)
        curl_plane_comp<1, DUAL, double>(IN, OUT, in, out, alpha, jhat, amp, step, 0.0, p, zc * kCurlKz, nullptr);
    else
        curl_plane_comp<2, DUAL, double>(IN, OUT, in, out, alpha, jhat, amp, step, 0.0, p, zc * kCurlKz, nullptr);
}

__device__ __noinline__ void ref_mass_tile(const HodgeBlockF32Args& A, int c, int tile, const double* x, double* y,
                                           float* sm) {
    // the tile face on a 16 x 16 thread grid (tiles are at most kLMax = 16 functions per axis)
    if (A.compensated)
        hodge_block_f32_tile<double, true>(A, c, tile, x, y, sm, threadIdx.x & 15, threadIdx.x >> 4, threadIdx.x,
                                           kBatchThreads);
    else
        hodge_block_f32_tile<double, false>(A, c, tile, x, y, sm, threadIdx.x & 15, threadIdx.x >> 4, threadIdx.x,
                                            kBatchThreads);
}

__device__ __noinline__ void ref_mass_element(const HodgeQuadF32Args& A, int e, const double* x, double* y, float* sm) {
    hodge_quad_f32_element(A, e, x, y, sm, threadIdx.x, kBatchThreads);
}

// Each variant is its own (not inlined) function, so the persistent kernel does not carry
// the register pressure of all of them at once.
template <int KL, class TIN>
__device__ __noinline__ void ref_line_k(const LineF32Args& A, int c, int lb, const TIN* in, float* out, float* sm,
                                        int lane) {
    line_body_f<KL, 0, false, TIN>(A, c, lb, in, out, sm, lane);
}

template <class TIN>
__device__ __forceinline__ void ref_line(const LineF32Args& A, int kl, int c, int lb, const TIN* in, float* out,
                                         float* sm, int lane) {
    switch (kl) {
        case 1: ref_line_k<1, TIN>(A, c, lb, in, out, sm, lane); break;
        case 2: ref_line_k<2, TIN>(A, c, lb, in, out, sm, lane); break;
        case 3: ref_line_k<3, TIN>(A, c, lb, in, out, sm, lane); break;
        case 4: ref_line_k<4, TIN>(A, c, lb, in, out, sm, lane); break;
        default: ref_line_k<5, TIN>(A, c, lb, in, out, sm, lane); break;
    }
}

constexpr int kRefChunk = kBatchThreads * 8;  // entries of a residual, sum or zeroing unit

__global__ void __launch_bounds__(kBatchThreads, 1) batch_refined_kernel(BatchRefArgs B) {
    extern __shared__ float smr[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned nblocks = gridDim.x;
    // a barrier of an earlier launch gave up (its phases are incomplete and the
    // barrier words are stale until smx_batch_status resets them): do nothing
    if (*(volatile unsigned*)B.status & 2u) return;
    const int step = B.stepctr ? (int)*(volatile unsigned*)B.stepctr : B.step;
    for (int ph = 0; ph < kRefPhases; ++ph) {
        const int2* items = B.items[ph];
        const int n = B.nitems[ph];
        const int h = ph < 12 ? 0 : 1;          // star of B (phases 1..11), of D (13..23)
        const int r = ph < 12 ? ph : ph - 12;   // position within the half step
        const bool line_phase = ph != 24 && ((r >= 2 && r <= 4) || (r >= 8 && r <= 10));
        if (!line_phase) {
            for (int it = blockIdx.x; it < n; it += nblocks) {
                const int2 w = items[it];
                const BatchRefCavity& K = B.cav[w.x];
                if (r == 0 || ph == 24) {
                    if (w.y & (1 << 30)) {  // zero the mass accumulator of the star that follows
                        const long long z0 = (long long)(w.y & 0xFFFFFF) * kRefChunk;
                        const long long ntot = K.fS[h].total;
                        for (int q = 0; q < 8; ++q) {
                            const long long i = z0 + q * kBatchThreads + threadIdx.x;
                            if (i < ntot) K.y[i] = 0.0;
                        }
                    } else if (ph == 12) {
                        ref_curl<true>(K, w.y, K.h, K.d, K.dt, K.jhat, K.amp, step);
                    } else {
                        ref_curl<false>(K, w.y, K.e, K.b, -0.5 * K.dt, nullptr, nullptr, 0);
                    }
                } else if (r == 1) {  // mass apply into y
                    const double* x = h == 0 ? K.b : K.d;
                    if (K.mode[h] == 0)
                        ref_mass_tile(K.hb[h], w.y >> 24, w.y & 0xFFFFFF, x, K.y, smr);
                    else
                        ref_mass_element(K.hq[h], w.y, x, K.y, smr);
                    __syncthreads();  // the next unit reuses the shared memory
                } else if (r >= 5 && r <= 7) {  // residual t = y - K x0, one axis per phase
                    const long long i0 = (long long)w.y * kRefChunk;
                    for (int q = 0; q < 8; ++q) {
                        const long long i = i0 + q * kBatchThreads + threadIdx.x;
                        if (r == 5)
                            band_apply_entry<float>(K.band[h][0], i, K.x0[h], nullptr, K.t64);
                        else if (r == 6)
                            band_apply_entry<double>(K.band[h][1], i, K.t64, nullptr, K.s64);
                        else
                            band_apply_entry<double>(K.band[h][2], i, K.s64, K.y, K.t64);
                    }
                } else {  // r == 11: the star's output x0 + c in FP64
                    double* out = h == 0 ? K.h : K.e;
                    const long long i0 = (long long)w.y * kRefChunk;
                    const long long ntot = K.fS[h].total;
                    for (int q = 0; q < 8; ++q) {
                        const long long i = i0 + q * kBatchThreads + threadIdx.x;
                        if (i < ntot) out[i] = f2d_exact(K.x0[h][i]) + f2d_exact(K.c32[i]);
                    }
                }
            }
        } else if (warp < B.line_warps) {
            float* sm = smr + (size_t)warp * B.warp_floats;
            const int gw = blockIdx.x * B.line_warps + warp, nw = nblocks * B.line_warps;
            const bool second = r >= 8;  // the correction's sweeps
            const int a = second ? r - 8 : r - 2;
            for (int it = gw; it < n; it += nw) {
                const int2 w = items[it];
                const BatchRefCavity& K = B.cav[w.x];
                const int c = w.y >> 24, lb = w.y & 0xFFFFFF;
                float* out = second ? K.c32 : K.x0[h];
                if (a == 0)
                    ref_line<double>(K.ln[h][0], K.kl[0], c, lb, second ? K.t64 : K.y, out, sm, lane);
                else
                    ref_line<float>(K.ln[h][a], K.kl[a], c, lb, out, out, sm, lane);
                __syncwarp();  // the next unit reuses this warp's staging
            }
        }
        if (ph + 1 < kRefPhases && !batch_barrier(B.bar, B.status, nblocks, B.wait_ns)) return;
    }
    // every CTA read the step counter before the first barrier: advance it for the next replay
    if (B.stepctr && blockIdx.x == 0 && threadIdx.x == 0) *B.stepctr += 1u;
}

size_t batch_ref_line_warp_floats(int maxn, int kl) {
    // factors L, U (n x KL) and 1/diag (n) as (hi, lo) pairs, then input and output staging
    const size_t f = 2 * (size_t)(2 * kl + 1) * maxn + 2 * (size_t)kSolveLines * (maxn | 1) + 8;
    return (f + 1) & ~size_t(1);  // even: the next warp's pairs stay 8-byte aligned
}

size_t batch_ref_mass_floats(int max_nloc, int qx, int qy, int qz) {
    size_t m = 2 * (size_t)3 * kLMax * (kLMax + 1) + 2 * (size_t)max_nloc;
    if (qx > 0) {
        const size_t Qe = (size_t)qx * qy * qz;
        m = std::max(m, 2 * (size_t)3 * 8 * kRMax + 3 * Qe + 2 * Qe * kRMax + (size_t)kRMax * kRMax * kRMax);
    }
    return m;
}

int batch_refined_blocks_per_sm(size_t smem) {
    if (cudaFuncSetAttribute(batch_refined_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_refined_kernel, kBatchThreads, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_batch_refined_step(const BatchRefArgs& a, int grid, size_t smem, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_refined_kernel, a);
}

}  // namespace smx
