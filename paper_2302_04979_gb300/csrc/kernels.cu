// sm_103a kernels of the scheme-2 leapfrog (Kapidani & Vazquez, Sec. 3.4, Sec. 4).
//
// FP64 throughout.  On GB300 the FP64 pipe is the scarce resource (about
// 1/64 of the FP32 lane rate), so every kernel here is written to issue the
// fewest FP64 instructions per degree of freedom; index arithmetic is integer.
#include <cuda_runtime.h>

#include <algorithm>

#include "batch.cuh"
#include "curl.cuh"
#include "internal.h"
#include "pdl.cuh"

namespace smx {

// ------------------------------------------------------------------ curl (see curl.cuh)
cudaError_t launch_curl_primal(const DevField& E, const DevField& B, const double* e, double* b, double alpha,
                               cudaStream_t s, double* zero) {
    return launch_curl_t<false, double>(E, B, e, b, alpha, nullptr, nullptr, 0, 0.0, s, zero);
}

cudaError_t launch_curl_dual(const DevField& H, const DevField& D, const double* h, double* d, double alpha,
                             const double* jhat, const double* amp, int amp_index, double s_host,
                             cudaStream_t s, double* zero) {
    return launch_curl_t<true, double>(H, D, h, d, alpha, jhat, amp, amp_index, s_host, s, zero);
}

// ------------------------------------------------------------------ Hodge: block Kronecker
// Identity map, material constant on each tile of <= 8^3 elements: the tile's
// contribution to the mass matrix of one 2-form component is
//   gamma_t * (Mz_t (x) My_t (x) Mx_t)
// with M*_t the univariate mass restricted to the tile's elements (Sec. 3.4
// mass matrix; the Kronecker structure of the parametric integrals, Sec. 4.1).
// One CTA per (tile, component): gather the tile's coefficients into shared
// memory, three banded 1D passes, scatter-add (FP64 atomics) into y.
constexpr int kHodgeThreads = 256;

// The work of one (tile, component) by a CTA of kHodgeThreads threads.
__device__ __forceinline__ void hodge_block_tile(const HodgeBlockArgs& A, int c, int tile,
                                                 const double* __restrict__ x, double* __restrict__ y, double* sm) {
    const int tx = tile % A.ntile[0];
    const int tyz = tile / A.ntile[0];
    const int ty = tyz % A.ntile[1];
    const int tz = tyz / A.ntile[1];
    const int tpos[3] = {tx, ty, tz};
    int f0[3], L[3], dg[3];
    const double* gmat[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int slot = A.kinds[c][a] * A.ntile[a] + tpos[a];
        f0[a] = A.tf0[a][slot];
        L[a] = A.tlen[a][slot];
        dg[a] = A.deg[c][a];
        gmat[a] = A.tmat[a] + (long long)slot * kLMax * kLMax;
    }
    const double gam = A.gamma[(tz * A.ntile[1] + ty) * A.ntile[0] + tx];
    // tile masses with row stride kLd = kLMax + 1 (rows ii read at one column across a
    // warp fall on distinct banks)
    constexpr int kLd = kLMax + 1;
    double* Mx = sm;
    double* My = Mx + kLMax * kLd;
    double* Mz = My + kLMax * kLd;
    double* s0 = Mz + kLMax * kLd;
    const int Lx = L[0], Ly = L[1], Lz = L[2];
    const int nloc = Lx * Ly * Lz;
    double* s1 = s0 + nloc;
    // tile masses; gamma folded into Mz
    for (int t = threadIdx.x; t < kLMax * kLMax; t += blockDim.x) {
        const int d = (t / kLMax) * kLd + t % kLMax;
        Mx[d] = __ldg(gmat[0] + t);
        My[d] = __ldg(gmat[1] + t);
        Mz[d] = gam * __ldg(gmat[2] + t);
    }
    const DevComp C = A.field.c[c];
    const long long nxy = (long long)C.n[0] * C.n[1];
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {
        const int ii = t % Lx, r = t / Lx, jj = r % Ly, kk = r / Ly;
        s0[t] = __ldg(x + C.off + (f0[0] + ii) + (long long)C.n[0] * (f0[1] + jj) + nxy * (f0[2] + kk));
    }
    __syncthreads();
    // x pass
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {
        const int ii = t % Lx, row = t - ii;
        const int lo = max(0, ii - dg[0]), hi = min(Lx - 1, ii + dg[0]);
        double acc = 0.0;
        for (int m = lo; m <= hi; ++m) acc = fma(Mx[ii * kLd + m], s0[row + m], acc);
        s1[t] = acc;
    }
    __syncthreads();
    // y pass
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {
        const int ii = t % Lx, r = t / Lx, jj = r % Ly, kk = r / Ly;
        const int lo = max(0, jj - dg[1]), hi = min(Ly - 1, jj + dg[1]);
        double acc = 0.0;
        for (int m = lo; m <= hi; ++m) acc = fma(My[jj * kLd + m], s1[(kk * Ly + m) * Lx + ii], acc);
        s0[t] = acc;
    }
    __syncthreads();
    // z pass and scatter-add
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {
        const int ii = t % Lx, r = t / Lx, jj = r % Ly, kk = r / Ly;
        const int lo = max(0, kk - dg[2]), hi = min(Lz - 1, kk + dg[2]);
        double acc = 0.0;
        for (int m = lo; m <= hi; ++m) acc = fma(Mz[kk * kLd + m], s0[(m * Ly + jj) * Lx + ii], acc);
        atomicAdd(y + C.off + (f0[0] + ii) + (long long)C.n[0] * (f0[1] + jj) + nxy * (f0[2] + kk), acc);
    }
}

__global__ void __launch_bounds__(kHodgeThreads) hodge_block_kernel(HodgeBlockArgs A, const double* __restrict__ x,
                                                                    double* __restrict__ y) {
    extern __shared__ double sm[];
    pdl_wait();
    hodge_block_tile(A, blockIdx.y, blockIdx.x, x, y, sm);
    pdl_trigger();
}

cudaError_t launch_hodge_block(const HodgeBlockArgs& a, const double* x, double* y, cudaStream_t s) {
    const int ntiles = a.ntile[0] * a.ntile[1] * a.ntile[2];
    const size_t smem = (3 * kLMax * (kLMax + 1) + 2 * (size_t)a.max_nloc) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(hodge_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((3 * kLMax * (kLMax + 1) + 2 * kLMax * kLMax * kLMax) * sizeof(double)));
        attr = true;
    }
    if (ntiles > 0) return launch_k(hodge_block_kernel, dim3(ntiles, 3), dim3(kHodgeThreads), smem, s, a, x, y);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Hodge: quadrature
// General map / pointwise material: per element, interpolate the three
// components at the q^3 Gauss points (sum factorisation), apply the 3x3
// symmetric metric G = w gamma J^T J / det J (2-form pullback, Sec. 2.3),
// integrate back against the same basis, scatter-add.  One CTA per element.
constexpr int kQuadThreads = 128;

// The work of one element by the whole CTA (any block size); sm: hodge_quad_smem_doubles(q).
__device__ __forceinline__ void hodge_quad_element(const HodgeQuadArgs& A, int e, const double* __restrict__ x,
                                                   double* __restrict__ y, double* sm) {
    const int ex = e % A.nel[0], exy = e / A.nel[0], ey = exy % A.nel[1], ez = exy / A.nel[1];
    const int el[3] = {ex, ey, ez};
    const int qx = A.q[0], qy = A.q[1], qz = A.q[2];
    const int Qe = qx * qy * qz;
    double* U = sm;                 // 3 * Qe values at the Gauss points
    double* T1 = U + 3 * Qe;        // scratch, <= Qe * kRMax
    double* T2 = T1 + Qe * kRMax;   // scratch, <= Qe * kRMax
    double* X = T2 + Qe * kRMax;    // local coefficients, <= kRMax^3
    double* Bv = X + kRMax * kRMax * kRMax;  // 3 axes x q x kRMax
    const int tid = threadIdx.x, nt = blockDim.x;

    for (int c = 0; c < 3; ++c) {
        const DevComp C = A.field.c[c];
        const int rx = A.deg[c][0] + 1, ry = A.deg[c][1] + 1, rz = A.deg[c][2] + 1;
        // basis values of this component's kinds on this element
        for (int t = tid; t < 3 * 8 * kRMax; t += nt) {
            const int a = t / (8 * kRMax), rem = t % (8 * kRMax), qp = rem / kRMax, r = rem % kRMax;
            if (qp < A.q[a])
                Bv[t] = __ldg(A.bval[a] + (((long long)A.kinds[c][a] * A.nel[a] + el[a]) * A.q[a] + qp) * kRMax + r);
        }
        for (int t = tid; t < rx * ry * rz; t += nt) {
            const int r0 = t % rx, rr = t / rx, r1 = rr % ry, r2 = rr / ry;
            const int gi = el[0] + r0 + A.koff[c][0], gj = el[1] + r1 + A.koff[c][1], gk = el[2] + r2 + A.koff[c][2];
            double v = 0.0;
            if (gi >= 0 && gi < C.n[0] && gj >= 0 && gj < C.n[1] && gk >= 0 && gk < C.n[2])
                v = __ldg(x + C.off + gi + (long long)C.n[0] * (gj + (long long)C.n[1] * gk));
            X[t] = v;
        }
        __syncthreads();
        const double* Bx = Bv;
        const double* By = Bv + 8 * kRMax;
        const double* Bz = Bv + 16 * kRMax;
        // T1[r2][r1][qx] = sum_r0 Bx[qx][r0] X[r2][r1][r0]
        for (int t = tid; t < rz * ry * qx; t += nt) {
            const int a = t % qx, rr = t / qx;
            double acc = 0.0;
            for (int r0 = 0; r0 < rx; ++r0) acc = fma(Bx[a * kRMax + r0], X[rr * rx + r0], acc);
            T1[t] = acc;
        }
        __syncthreads();
        // T2[r2][qy][qx] = sum_r1 By[qy][r1] T1[r2][r1][qx]
        for (int t = tid; t < rz * qy * qx; t += nt) {
            const int a = t % qx, rr = t / qx, b = rr % qy, r2 = rr / qy;
            double acc = 0.0;
            for (int r1 = 0; r1 < ry; ++r1) acc = fma(By[b * kRMax + r1], T1[(r2 * ry + r1) * qx + a], acc);
            T2[t] = acc;
        }
        __syncthreads();
        // U_c[qz][qy][qx] = sum_r2 Bz[qz][r2] T2[r2][qy][qx]
        for (int t = tid; t < Qe; t += nt) {
            const int ab = t % (qx * qy), g = t / (qx * qy);
            double acc = 0.0;
            for (int r2 = 0; r2 < rz; ++r2) acc = fma(Bz[g * kRMax + r2], T2[r2 * qx * qy + ab], acc);
            U[c * Qe + t] = acc;
        }
        __syncthreads();
    }
    // metric at each Gauss point
    for (int t = tid; t < Qe; t += nt) {
        const int a = t % qx, rr = t / qx, b = rr % qy, g = rr / qy;
        const long long qi = ((long long)(ez * qz + g) * A.Qn[1] + (ey * qy + b)) * A.Qn[0] + (ex * qx + a);
        const double g00 = __ldg(A.G + qi), g01 = __ldg(A.G + A.Qtot + qi), g02 = __ldg(A.G + 2 * A.Qtot + qi);
        const double g11 = __ldg(A.G + 3 * A.Qtot + qi), g12 = __ldg(A.G + 4 * A.Qtot + qi);
        const double g22 = __ldg(A.G + 5 * A.Qtot + qi);
        const double u0 = U[t], u1 = U[Qe + t], u2 = U[2 * Qe + t];
        U[t] = g00 * u0 + g01 * u1 + g02 * u2;
        U[Qe + t] = g01 * u0 + g11 * u1 + g12 * u2;
        U[2 * Qe + t] = g02 * u0 + g12 * u1 + g22 * u2;
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
        const DevComp C = A.field.c[c];
        const int rx = A.deg[c][0] + 1, ry = A.deg[c][1] + 1, rz = A.deg[c][2] + 1;
        for (int t = tid; t < 3 * 8 * kRMax; t += nt) {
            const int a = t / (8 * kRMax), rem = t % (8 * kRMax), qp = rem / kRMax, r = rem % kRMax;
            if (qp < A.q[a])
                Bv[t] = __ldg(A.bval[a] + (((long long)A.kinds[c][a] * A.nel[a] + el[a]) * A.q[a] + qp) * kRMax + r);
        }
        __syncthreads();
        const double* Bx = Bv;
        const double* By = Bv + 8 * kRMax;
        const double* Bz = Bv + 16 * kRMax;
        // T2[r2][qy][qx] = sum_qz Bz[qz][r2] V[qz][qy][qx]
        for (int t = tid; t < rz * qy * qx; t += nt) {
            const int ab = t % (qx * qy), r2 = t / (qx * qy);
            double acc = 0.0;
            for (int g = 0; g < qz; ++g) acc = fma(Bz[g * kRMax + r2], U[c * Qe + g * qx * qy + ab], acc);
            T2[t] = acc;
        }
        __syncthreads();
        // T1[r2][r1][qx] = sum_qy By[qy][r1] T2[r2][qy][qx]
        for (int t = tid; t < rz * ry * qx; t += nt) {
            const int a = t % qx, rr = t / qx, r1 = rr % ry, r2 = rr / ry;
            double acc = 0.0;
            for (int b = 0; b < qy; ++b) acc = fma(By[b * kRMax + r1], T2[(r2 * qy + b) * qx + a], acc);
            T1[t] = acc;
        }
        __syncthreads();
        // Y[r2][r1][r0] = sum_qx Bx[qx][r0] T1[r2][r1][qx], scatter-add
        for (int t = tid; t < rx * ry * rz; t += nt) {
            const int r0 = t % rx, rr = t / rx, r1 = rr % ry, r2 = rr / ry;
            const int gi = el[0] + r0 + A.koff[c][0], gj = el[1] + r1 + A.koff[c][1], gk = el[2] + r2 + A.koff[c][2];
            if (gi >= 0 && gi < C.n[0] && gj >= 0 && gj < C.n[1] && gk >= 0 && gk < C.n[2]) {
                double acc = 0.0;
                for (int a = 0; a < qx; ++a) acc = fma(Bx[a * kRMax + r0], T1[rr * qx + a], acc);
                atomicAdd(y + C.off + gi + (long long)C.n[0] * (gj + (long long)C.n[1] * gk), acc);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kQuadThreads) hodge_quad_kernel(HodgeQuadArgs A, const double* __restrict__ x,
                                                                  double* __restrict__ y) {
    extern __shared__ double sm[];
    pdl_wait();
    hodge_quad_element(A, blockIdx.x, x, y, sm);
}

size_t hodge_quad_smem_doubles(int qx, int qy, int qz) {
    const size_t Qe = (size_t)qx * qy * qz;
    return 3 * Qe + 2 * Qe * kRMax + (size_t)kRMax * kRMax * kRMax + 3 * 8 * kRMax;
}

cudaError_t launch_hodge_quad(const HodgeQuadArgs& a, const double* x, double* y, cudaStream_t s) {
    const int nel = a.nel[0] * a.nel[1] * a.nel[2];
    const int Qe = a.q[0] * a.q[1] * a.q[2];
    const size_t smem = (3 * Qe + 2 * Qe * kRMax + kRMax * kRMax * kRMax + 3 * 8 * kRMax) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(hodge_quad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    if (nel > 0) return launch_k(hodge_quad_kernel, dim3(nel), dim3(kQuadThreads), smem, s, a, x, y);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ pairing solve sweeps
// x = A^{-1} y along every line of one axis (Sec. 4.2: Eq. kroninverse and
// the vec identity turn the Kronecker solve into independent 1D solves).
// A = L U without pivoting: forward z_m = y_m - sum_k L(m,m-k) z_{m-k},
// backward x_m = z_m / U(m,m) - sum_k U'(m,m+k) x_{m+k} with U' = U / diag.
// A CTA stages kSolveLines lines in shared memory with asynchronous copies
// (every load of the chunk in flight at once), each thread then solves one
// line with a register window of the last KL values, and the chunk is
// written back with coalesced stores.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Line recurrences.  The FP64 pipe of GB300 has a latency of about 64 cycles,
// so each recurrence keeps exactly one FMA per entry on its dependency chain
// (the one with the previous value), reads and writes distinct arrays so the
// compiler can hoist the next entries' loads above the current store, and is
// unrolled so off-chain FMAs of later entries overlap the chain.
template <int KL>
__device__ __forceinline__ void lu_forward(const double* __restrict__ y, double* __restrict__ z, int s, int n,
                                           const double* __restrict__ fL) {
    double w[KL];
#pragma unroll
    for (int k = 0; k < KL; ++k) w[k] = 0.0;
#pragma unroll 4
    for (int m = 0; m < n; ++m) {  // z_m = y_m - sum_k L(m, m-k) z_{m-k}
        double u = y[m * s];
#pragma unroll
        for (int k = KL - 1; k >= 1; --k) u = fma(-fL[m * KL + k], w[k], u);
        const double zm = fma(-fL[m * KL], w[0], u);
#pragma unroll
        for (int k = KL - 1; k > 0; --k) w[k] = w[k - 1];
        w[0] = zm;
        z[m * s] = zm;
    }
}

template <int KL>
__device__ __forceinline__ void lu_backward(const double* __restrict__ z, double* __restrict__ x, int s, int n,
                                            const double* __restrict__ fU, const double* __restrict__ fD) {
    double w[KL];
#pragma unroll
    for (int k = 0; k < KL; ++k) w[k] = 0.0;
#pragma unroll 4
    for (int m = n - 1; m >= 0; --m) {  // x_m = z_m / U(m,m) - sum_k U'(m, m+k) x_{m+k}
        double u = z[m * s] * fD[m];
#pragma unroll
        for (int k = KL - 1; k >= 1; --k) u = fma(-fU[m * KL + k], w[k], u);
        const double xm = fma(-fU[m * KL], w[0], u);
#pragma unroll
        for (int k = KL - 1; k > 0; --k) w[k] = w[k - 1];
        w[0] = xm;
        x[m * s] = xm;
    }
}

// One block of kSolveLines lines (index lb) of component c, by one warp (tid = lane).
template <int KL>
__device__ __forceinline__ void solve_lines(const SolveArgs& A, int c, int lb, const double* __restrict__ in,
                                            double* __restrict__ out, double* sm, int tid) {
    const DevComp C = A.field.c[c];
    const int axis = A.axis;
    const int n = C.n[axis];
    const int ncomp = C.n[0] * C.n[1] * C.n[2];
    const int nlines = ncomp / n;
    const int l0 = lb * kSolveLines;
    if (l0 >= nlines) return;
    const int nl = min(kSolveLines, nlines - l0);
    const DevFactor F = A.f[c];
    double* fL = sm;
    double* fU = fL + n * KL;
    double* fD = fU + n * KL;
    double* S = fD + n;
    const int nt = kSolveLines;
    for (int t = tid; t < n * KL; t += nt) {
        cp_async8(fL + t, F.L + t);
        cp_async8(fU + t, F.U + t);
    }
    for (int t = tid; t < n; t += nt) cp_async8(fD + t, F.dinv + t);
    // layout: x lines as [line][m] with odd leading dimension, y/z lines as [m][line]
    const int ldl = n | 1;
    const int nx = C.n[0], nxy = C.n[0] * C.n[1];
    const double* src = in + C.off;
    if (axis == 0) {
        const double* chunk = src + (long long)l0 * n;
        for (int line = 0; line < nl; ++line)  // no run-time division per entry
            for (int m = tid; m < n; m += nt) cp_async8(S + line * ldl + m, chunk + line * n + m);
    } else if (tid < nl) {
        const int l = l0 + tid;
        const int base = axis == 1 ? (l % nx) + (l / nx) * nxy : l;
        const int stride = axis == 1 ? nx : nxy;
        for (int m = 0; m < n; ++m) cp_async8(S + m * kSolveLines + tid, src + base + m * stride);
    }
    cp_async_wait_all();
    __syncwarp();
    if (tid < nl) {
        const int sL = axis == 0 ? ldl : 1;
        const int sM = axis == 0 ? 1 : kSolveLines;
        double* S2 = S + kSolveLines * ldl;
        lu_forward<KL>(S + tid * sL, S2 + tid * sL, sM, n, fL);
        lu_backward<KL>(S2 + tid * sL, S + tid * sL, sM, n, fU, fD);
    }
    __syncwarp();
    double* dst = out + C.off;
    if (axis == 0) {
        double* chunk = dst + (long long)l0 * n;
        for (int line = 0; line < nl; ++line)
            for (int m = tid; m < n; m += nt) chunk[line * n + m] = S[line * ldl + m];
    } else if (tid < nl) {
        const int l = l0 + tid;
        const int base = axis == 1 ? (l % nx) + (l / nx) * nxy : l;
        const int stride = axis == 1 ? nx : nxy;
#pragma unroll 4
        for (int m = 0; m < n; ++m) dst[base + m * stride] = S[m * kSolveLines + tid];
    }
}

template <int KL>
__global__ void __launch_bounds__(kSolveLines) solve_axis_kernel(SolveArgs A, const double* __restrict__ in,
                                                                 double* __restrict__ out) {
    extern __shared__ double sm[];
    pdl_wait();
    solve_lines<KL>(A, blockIdx.y, blockIdx.x, in, out, sm, threadIdx.x);
    pdl_trigger();
}

template <int KL>
static cudaError_t launch_solve_t(const SolveArgs& a, const double* in, double* out, cudaStream_t s) {
    long long maxlines = 0;
    int maxn = 0;
    for (int c = 0; c < 3; ++c) {
        const long long nc = (long long)a.field.c[c].n[0] * a.field.c[c].n[1] * a.field.c[c].n[2];
        const int n = a.field.c[c].n[a.axis];
        if (n > 0) maxlines = std::max(maxlines, nc / n);
        maxn = std::max(maxn, n);
    }
    const size_t smem = ((size_t)(2 * KL + 1) * maxn + 2 * (size_t)(maxn | 1) * kSolveLines + 8) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(solve_axis_kernel<KL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    const long long nb = (maxlines + kSolveLines - 1) / kSolveLines;
    if (nb > 0) return launch_k(solve_axis_kernel<KL>, dim3((unsigned)nb, 3), dim3(kSolveLines), smem, s, a, in, out);
    return cudaGetLastError();
}

cudaError_t launch_solve_axis(const SolveArgs& a, int kl, const double* in, double* out, cudaStream_t s) {
    switch (kl) {
        case 1: return launch_solve_t<1>(a, in, out, s);
        case 2: return launch_solve_t<2>(a, in, out, s);
        case 3: return launch_solve_t<3>(a, in, out, s);
        case 4: return launch_solve_t<4>(a, in, out, s);
        case 5: return launch_solve_t<5>(a, in, out, s);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ separable Hodge star
// Identity map and constant material: M = gamma (M_z (x) M_y (x) M_x) and the
// pairing block is C = A_z (x) A_y (x) A_x (Eq. tensor_K / tensor_Ktilde), so
// the Hodge star C^{-1} M = (A_z^{-1} M_z) (x) (A_y^{-1} M_y) (x) (A_x^{-1} M_x)
// (gamma folded into one axis' mass).  Each pass applies the banded mass and
// then the banded LU solve to every line of one axis, in shared memory.
// t_m = sum_q M(m, m-D+q) y_{m-D+q} on a line padded with D zeros at both ends.
template <int D>
__device__ __forceinline__ void mass_line(const double* __restrict__ ypad, double* __restrict__ t, int s, int n,
                                          const double* __restrict__ fM) {
    constexpr int W = 2 * D + 1;
    int m = 0;
    for (; m + 3 < n; m += 4) {  // four independent accumulations in flight
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            a0 = fma(fM[m * W + q], ypad[(m + q) * s], a0);
            a1 = fma(fM[(m + 1) * W + q], ypad[(m + 1 + q) * s], a1);
            a2 = fma(fM[(m + 2) * W + q], ypad[(m + 2 + q) * s], a2);
            a3 = fma(fM[(m + 3) * W + q], ypad[(m + 3 + q) * s], a3);
        }
        t[m * s] = a0;
        t[(m + 1) * s] = a1;
        t[(m + 2) * s] = a2;
        t[(m + 3) * s] = a3;
    }
    for (; m < n; ++m) {
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < W; ++q) acc = fma(fM[m * W + q], ypad[(m + q) * s], acc);
        t[m * s] = acc;
    }
}

template <int KL, int D>
__device__ __forceinline__ void mass_solve_body(const MassSolveArgs& A, int c, int lb, const double* __restrict__ in,
                                                double* __restrict__ out, double* sm, int tid) {
    const DevComp C = A.field.c[c];
    const int axis = A.axis;
    const int n = C.n[axis];
    const int nlines = C.n[0] * C.n[1] * C.n[2] / n;
    const int l0 = lb * kSolveLines;
    if (l0 >= nlines) return;
    const int nl = min(kSolveLines, nlines - l0);
    const DevFactor F = A.f[c];
    constexpr int W = 2 * D + 1;
    double* fL = sm;
    double* fU = fL + n * KL;
    double* fD = fU + n * KL;
    double* fM = fD + n;              // n x W mass band rows
    double* Sin = fM + n * W;         // input lines, padded with D zeros at both ends
    const int np = n + 2 * D;
    const int ldin = np | 1, ldout = n | 1;
    double* Sout = Sin + kSolveLines * ldin;
    const int nt = kSolveLines;
    const double* Mg = A.mass[c];
    for (int t = tid; t < n * KL; t += nt) {
        cp_async8(fL + t, F.L + t);
        cp_async8(fU + t, F.U + t);
    }
    for (int t = tid; t < n; t += nt) cp_async8(fD + t, F.dinv + t);
    for (int t = tid; t < n * W; t += nt) cp_async8(fM + t, Mg + t);
    // x lines: [line][m + D] (leading dimension ldin); y/z lines: [m + D][line]
    const int sL = axis == 0 ? ldin : 1;
    const int sM = axis == 0 ? 1 : kSolveLines;
    if constexpr (D > 0) {
        for (int t = tid; t < kSolveLines * D; t += nt) {  // zero pads
            const int line = t / D, q = t - line * D;
            Sin[line * sL + q * sM] = 0.0;
            Sin[line * sL + (n + D + q) * sM] = 0.0;
        }
    }
    const int nx = C.n[0], nxy = C.n[0] * C.n[1];
    const double* src = in + C.off;
    if (axis == 0) {
        const double* chunk = src + (long long)l0 * n;
        for (int line = 0; line < nl; ++line)  // no run-time division per entry
            for (int m = tid; m < n; m += nt) cp_async8(Sin + line * ldin + D + m, chunk + line * n + m);
    } else if (tid < nl) {
        const int l = l0 + tid;
        const int base = axis == 1 ? (l % nx) + (l / nx) * nxy : l;
        const int stride = axis == 1 ? nx : nxy;
        for (int m = 0; m < n; ++m) cp_async8(Sin + (D + m) * kSolveLines + tid, src + base + m * stride);
    }
    cp_async_wait_all();
    __syncwarp();
    const int oL = axis == 0 ? ldout : 1;
    if (tid < nl) {
        // t = M y: independent banded dot products, no recurrence
        mass_line<D>(Sin + tid * sL, Sout + tid * oL, sM, n, fM);
        // forward t -> z (z reuses the input line), backward z -> x
        lu_forward<KL>(Sout + tid * oL, Sin + tid * sL, sM, n, fL);
        lu_backward<KL>(Sin + tid * sL, Sout + tid * oL, sM, n, fU, fD);
    }
    __syncwarp();
    double* dst = out + C.off;
    if (axis == 0) {
        double* chunk = dst + (long long)l0 * n;
        for (int line = 0; line < nl; ++line)
            for (int m = tid; m < n; m += nt) chunk[line * n + m] = Sout[line * ldout + m];
    } else if (tid < nl) {
        const int l = l0 + tid;
        const int base = axis == 1 ? (l % nx) + (l / nx) * nxy : l;
        const int stride = axis == 1 ? nx : nxy;
#pragma unroll 4
        for (int m = 0; m < n; ++m) dst[base + m * stride] = Sout[m * kSolveLines + tid];
    }
}

// The fused pass for one block of lines, the mass half-bandwidth of the component chosen at run time.
template <int KL>
__device__ __forceinline__ void mass_solve_lines(const MassSolveArgs& A, int c, int lb, const double* __restrict__ in,
                                                 double* __restrict__ out, double* sm, int tid) {
    const int d = A.deg[c];
    if (d == KL - 1) {
        if constexpr (KL >= 1) mass_solve_body<KL, (KL >= 1 ? KL - 1 : 0)>(A, c, lb, in, out, sm, tid);
    } else if (d == KL) {
        mass_solve_body<KL, KL>(A, c, lb, in, out, sm, tid);
    } else {
        mass_solve_body<KL, KL + 1>(A, c, lb, in, out, sm, tid);
    }
}

template <int KL>
__global__ void __launch_bounds__(kSolveLines) mass_solve_axis_kernel(MassSolveArgs A, const double* __restrict__ in,
                                                                      double* __restrict__ out) {
    extern __shared__ double sm[];
    pdl_wait();
    mass_solve_lines<KL>(A, blockIdx.y, blockIdx.x, in, out, sm, threadIdx.x);
    pdl_trigger();
}

template <int KL>
static cudaError_t launch_mass_solve_t(const MassSolveArgs& a, const double* in, double* out, cudaStream_t s) {
    long long maxlines = 0;
    int maxn = 0;
    for (int c = 0; c < 3; ++c) {
        const long long nc = (long long)a.field.c[c].n[0] * a.field.c[c].n[1] * a.field.c[c].n[2];
        const int n = a.field.c[c].n[a.axis];
        if (n > 0) maxlines = std::max(maxlines, nc / n);
        maxn = std::max(maxn, n);
    }
    const int D = KL + 1, W = 2 * D + 1;
    const size_t smem = ((size_t)(2 * KL + 1 + W) * maxn + (size_t)((maxn + 2 * D) | 1) * kSolveLines +
                         (size_t)(maxn | 1) * kSolveLines + 8) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(mass_solve_axis_kernel<KL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    const long long nb = (maxlines + kSolveLines - 1) / kSolveLines;
    if (nb > 0)
        return launch_k(mass_solve_axis_kernel<KL>, dim3((unsigned)nb, 3), dim3(kSolveLines), smem, s, a, in, out);
    return cudaGetLastError();
}

cudaError_t launch_mass_solve_axis(const MassSolveArgs& a, int kl, const double* in, double* out, cudaStream_t s) {
    switch (kl) {
        case 1: return launch_mass_solve_t<1>(a, in, out, s);
        case 2: return launch_mass_solve_t<2>(a, in, out, s);
        case 3: return launch_mass_solve_t<3>(a, in, out, s);
        case 4: return launch_mass_solve_t<4>(a, in, out, s);
        case 5: return launch_mass_solve_t<5>(a, in, out, s);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ reductions
constexpr int kDotThreads = 256;

__global__ void __launch_bounds__(kDotThreads) dot_partial_kernel(const double* __restrict__ x,
                                                                  const double* __restrict__ y, long long n,
                                                                  double* __restrict__ partial) {
    __shared__ double red[kDotThreads];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc = fma(__ldg(x + i), __ldg(y + i), acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kDotThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kDotThreads) dot_final_kernel(const double* __restrict__ partial, int np,
                                                                double* __restrict__ out) {
    __shared__ double red[kDotThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kDotThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

cudaError_t launch_dot(const double* x, const double* y, long long n, double* partial, double* out,
                       cudaStream_t s) {
    dot_partial_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(x, y, n, partial);
    dot_final_kernel<<<1, kDotThreads, 0, s>>>(partial, kDotBlocks, out);
    return cudaGetLastError();
}

__global__ void scale_copy_kernel(const double* __restrict__ x, double* __restrict__ y, double a, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i];
}

cudaError_t launch_scale_copy(const double* x, double* y, double a, long long n, cudaStream_t s) {
    const long long nb = (n + 255) / 256;
    if (nb > 0) scale_copy_kernel<<<(unsigned)nb, 256, 0, s>>>(x, y, a, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ y = 0 (in the launch chain of a step)
__global__ void zero_kernel(double* __restrict__ y, long long n) {
    pdl_wait();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = 0.0;
    pdl_trigger();
}

cudaError_t launch_zero(double* y, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    return launch_k(zero_kernel, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, y, n);
}

// ------------------------------------------------------------------ conjugate gradients (scheme 1)
__global__ void cg_xr_kernel(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                             const double* __restrict__ Ap, const double* __restrict__ scal, long long n) {
    const double pap = scal[kCgPAp];
    const double alpha = pap > 0.0 ? scal[kCgRz] / pap : 0.0;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) {
        x[i] = fma(alpha, p[i], x[i]);
        r[i] = fma(-alpha, Ap[i], r[i]);
    }
}

__global__ void cg_p_kernel(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ scal,
                            long long n) {
    const double rz = scal[kCgRz];
    const double beta = rz > 0.0 ? scal[kCgRzNew] / rz : 0.0;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) p[i] = fma(beta, p[i], z[i]);
}

__global__ void cg_shift_kernel(double* scal) { scal[kCgRz] = scal[kCgRzNew]; }

__global__ void sub_from_kernel(const double* __restrict__ y, double* __restrict__ r, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) r[i] = y[i] - r[i];
}

__global__ void copy_kernel(const double* __restrict__ x, double* __restrict__ y, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i];
}

cudaError_t launch_cg_xr(double* x, double* r, const double* p, const double* Ap, const double* scal, long long n,
                         cudaStream_t s) {
    if (n > 0) cg_xr_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, r, p, Ap, scal, n);
    return cudaGetLastError();
}

cudaError_t launch_cg_p(double* p, const double* z, double* scal, long long n, cudaStream_t s) {
    if (n > 0) cg_p_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, z, scal, n);
    cg_shift_kernel<<<1, 1, 0, s>>>(scal);
    return cudaGetLastError();
}

cudaError_t launch_sub_from(const double* y, double* r, long long n, cudaStream_t s) {
    if (n > 0) sub_from_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, r, n);
    return cudaGetLastError();
}

cudaError_t launch_copy(const double* x, double* y, long long n, cudaStream_t s) {
    if (n > 0) copy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ batched cavities
// One persistent (cooperative) launch runs a whole leapfrog step of many
// independent cavities: eleven phases separated by grid barriers,
//   0 b -= dt/2 D^1 e; y = 0 (cavities whose star of B applies a mass)
//   1 y = M b (block tiles or quadrature elements)        2-4 h = star of B per axis
//   5 d += dt (D~^1 h - s jhat); y = 0 (star of D applies a mass)
//   6 y = M~ d                                            7-9 e = star of D per axis
//   10 b -= dt/2 D^1 e
// A star is either the fused mass + solve passes (identity map, constant
// material) or the pairing sweeps of y.  Each phase walks a flat list of
// (cavity, unit) items: whole-CTA units (curl chunks, Hodge tiles or elements,
// zeroing) or line units (kSolveLines lines, one warp, each line warp with its
// own shared-memory staging).  The work of a unit is the device function of the
// single-cavity kernel, so a batched step computes what the separate launches
// compute.

template <bool DUAL>
__device__ __noinline__ void batch_curl(const BatchCavity& K, int unit, const double* in, double* out,
                                           double alpha, const double* jhat, const double* amp, int step) {
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

// Each variant is its own (not inlined) function, so the persistent kernel
// does not carry the register pressure of all of them at once.
template <int KL>
__device__ __noinline__ void batch_mass_solve_k(const MassSolveArgs& A, int c, int lb, const double* in, double* out,
                                                double* sm, int lane) {
    mass_solve_lines<KL>(A, c, lb, in, out, sm, lane);
}
template <int KL>
__device__ __noinline__ void batch_solve_k(const SolveArgs& A, int c, int lb, const double* in, double* out,
                                           double* sm, int lane) {
    solve_lines<KL>(A, c, lb, in, out, sm, lane);
}
__device__ __noinline__ void batch_hodge_tile(const HodgeBlockArgs& A, int c, int tile, const double* x, double* y,
                                              double* sm) {
    hodge_block_tile(A, c, tile, x, y, sm);
}

__device__ __forceinline__ void batch_mass_solve(const MassSolveArgs& A, int kl, int c, int lb, const double* in,
                                                 double* out, double* sm, int lane) {
    switch (kl) {
        case 1: batch_mass_solve_k<1>(A, c, lb, in, out, sm, lane); break;
        case 2: batch_mass_solve_k<2>(A, c, lb, in, out, sm, lane); break;
        case 3: batch_mass_solve_k<3>(A, c, lb, in, out, sm, lane); break;
        case 4: batch_mass_solve_k<4>(A, c, lb, in, out, sm, lane); break;
        default: batch_mass_solve_k<5>(A, c, lb, in, out, sm, lane); break;
    }
}

__device__ __forceinline__ void batch_solve(const SolveArgs& A, int kl, int c, int lb, const double* in, double* out,
                                            double* sm, int lane) {
    switch (kl) {
        case 1: batch_solve_k<1>(A, c, lb, in, out, sm, lane); break;
        case 2: batch_solve_k<2>(A, c, lb, in, out, sm, lane); break;
        case 3: batch_solve_k<3>(A, c, lb, in, out, sm, lane); break;
        case 4: batch_solve_k<4>(A, c, lb, in, out, sm, lane); break;
        default: batch_solve_k<5>(A, c, lb, in, out, sm, lane); break;
    }
}

__device__ __noinline__ void batch_hodge_element(const HodgeQuadArgs& A, int e, const double* x, double* y, double* sm) {
    hodge_quad_element(A, e, x, y, sm);
}

// zero a chunk of y (unit z: kBatchThreads * 8 entries)
__device__ __forceinline__ void batch_zero(const BatchCavity& K, int unit, long long n) {
    const long long z0 = (long long)(unit & 0xFFFFFF) * (kBatchThreads * 8);
    for (int q = 0; q < 8; ++q) {
        const long long i = z0 + q * kBatchThreads + threadIdx.x;
        if (i < n) K.y[i] = 0.0;
    }
}

__global__ void __launch_bounds__(kBatchThreads, 1) batch_step_kernel(BatchArgs B) {
    extern __shared__ double smb[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned nblocks = gridDim.x;
    // a barrier of an earlier launch gave up (its phases are incomplete and the
    // barrier words are stale until smx_batch_status resets them): do nothing
    if (*(volatile unsigned*)B.status & 2u) return;
    // the step index (amplitude of the source): from the device counter when replayed from a graph
    const int step = B.stepctr ? (int)*(volatile unsigned*)B.stepctr : B.step;
    for (int ph = 0; ph < kBatchPhases; ++ph) {
        const int2* items = B.items[ph];
        const int n = B.nitems[ph];
        const bool line_phase = (ph >= 2 && ph <= 4) || (ph >= 7 && ph <= 9);
        if (!line_phase) {
            for (int it = blockIdx.x; it < n; it += nblocks) {
                const int2 w = items[it];
                const BatchCavity& K = B.cav[w.x];
                if (ph == 0 || ph == 10) {
                    if (w.y & (1 << 30))
                        batch_zero(K, w.y, K.fB.total);
                    else
                        batch_curl<false>(K, w.y, K.e, K.b, -0.5 * K.dt, nullptr, nullptr, 0);
                } else if (ph == 5) {
                    if (w.y & (1 << 30))
                        batch_zero(K, w.y, K.fD.total);
                    else
                        batch_curl<true>(K, w.y, K.h, K.d, K.dt, K.jhat, K.amp, step);
                } else {  // ph == 1 or 6: mass apply into y
                    const bool bside = ph == 1;
                    if ((bside ? K.modeB : K.modeD) == 0)
                        batch_hodge_tile(bside ? K.hbB : K.hbD, w.y >> 24, w.y & 0xFFFFFF, bside ? K.b : K.d, K.y, smb);
                    else
                        batch_hodge_element(bside ? K.hqB : K.hqD, w.y, bside ? K.b : K.d, K.y, smb);
                    __syncthreads();  // the next unit reuses the shared memory
                }
            }
        } else if (warp < B.line_warps) {
            double* sm = smb + (size_t)warp * B.warp_smem;
            const int gw = blockIdx.x * B.line_warps + warp, nw = nblocks * B.line_warps;
            for (int it = gw; it < n; it += nw) {
                const int2 w = items[it];
                const BatchCavity& K = B.cav[w.x];
                const int c = w.y >> 24, lb = w.y & 0xFFFFFF;
                if (ph <= 4) {
                    const int a = ph - 2;
                    if (K.sepB)
                        batch_mass_solve(K.msH[a], K.kl[a], c, lb, a == 0 ? K.b : K.h, K.h, sm, lane);
                    else
                        batch_solve(K.solveH[a], K.kl[a], c, lb, a == 0 ? K.y : K.h, K.h, sm, lane);
                } else {
                    const int a = ph - 7;
                    if (K.sepD)
                        batch_mass_solve(K.msD[a], K.kl[a], c, lb, a == 0 ? K.d : K.e, K.e, sm, lane);
                    else
                        batch_solve(K.solveE[a], K.kl[a], c, lb, a == 0 ? K.y : K.e, K.e, sm, lane);
                }
                __syncwarp();  // the next unit reuses this warp's staging
            }
        }
        if (ph + 1 < kBatchPhases && !batch_barrier(B.bar, B.status, nblocks, B.wait_ns)) return;
    }
    // every CTA read the step counter before the first barrier: advance it for the next replay
    if (B.stepctr && blockIdx.x == 0 && threadIdx.x == 0) *B.stepctr += 1u;
}

size_t batch_line_warp_doubles(int maxn, int kl) {
    const int D = kl + 1, W = 2 * D + 1;
    return (size_t)(2 * kl + 1 + W) * maxn + (size_t)((maxn + 2 * D) | 1) * kSolveLines +
           (size_t)(maxn | 1) * kSolveLines + 8;
}

int batch_blocks_per_sm(size_t smem) {
    // the dynamic shared memory the launch will request (the kernel's own static words come on top)
    if (cudaFuncSetAttribute(batch_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        (void)cudaGetLastError();  // clear: the shape does not fit
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_step_kernel, kBatchThreads, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_batch_step(const BatchArgs& a, int grid, size_t smem, cudaStream_t s) {
    // a cooperative launch through the extensible launch API, which a stream capture records
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
    return cudaLaunchKernelEx(&cfg, batch_step_kernel, a);
}

}  // namespace smx
