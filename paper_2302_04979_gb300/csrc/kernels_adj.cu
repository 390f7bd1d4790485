// Kernels of the reverse (adjoint) leapfrog step and of the receiver misfit.
//
// The reverse step itself reuses the forward kernels (the dual curl is the
// transpose of the primal curl, D~^1 = (D^1)^T, the pairing sweeps run with
// the transposed 1D factors, the masses are symmetric).  What is new:
//   * the per-block derivative of the electric mass, z^T (dM~/deps_c) d,
//     for the quadrature Hodge (curved map) and for the block-Kronecker Hodge
//     (identity map);
//   * the receiver evaluation R e and its transpose;
//   * rescaling the stored quadrature metric when the block permittivity
//     changes, and y += a x.
#include <cuda_runtime.h>

#include "internal.h"

namespace smx {

// ------------------------------------------------------------------ receivers
// Row r of R (3 per receiver point, one per E component): rec.ptr[r] .. rec.ptr[r+1]
// entries (index into e, basis value).  One warp per row.
__global__ void receivers_eval_kernel(RecArgs R, const double* __restrict__ e, double* __restrict__ out) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= R.nrows) return;
    double acc = 0.0;
    for (int k = R.ptr[row] + lane; k < R.ptr[row + 1]; k += 32) acc = fma(R.val[k], __ldg(e + R.idx[k]), acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[row] = acc;
}

__global__ void receivers_adjoint_kernel(RecArgs R, const double* __restrict__ w, double alpha,
                                         double* __restrict__ ebar) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= R.nrows) return;
    const double s = alpha * __ldg(w + row);
    for (int k = R.ptr[row] + lane; k < R.ptr[row + 1]; k += 32) atomicAdd(ebar + R.idx[k], s * R.val[k]);
}

cudaError_t launch_receivers_eval(const RecArgs& r, const double* e, double* out, cudaStream_t s) {
    if (r.nrows > 0) receivers_eval_kernel<<<(r.nrows + 7) / 8, 256, 0, s>>>(r, e, out);
    return cudaGetLastError();
}

cudaError_t launch_receivers_adjoint(const RecArgs& r, const double* w, double alpha, double* ebar, cudaStream_t s) {
    if (r.nrows > 0) receivers_adjoint_kernel<<<(r.nrows + 7) / 8, 256, 0, s>>>(r, w, alpha, ebar);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ y += a x
__global__ void axpy_kernel(const double* __restrict__ x, double* __restrict__ y, double a, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = fma(a, x[i], y[i]);
}

cudaError_t launch_axpy(const double* x, double* y, double a, long long n, cudaStream_t s) {
    if (n > 0) axpy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, y, a, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ metric rescale
// New block material: every quadrature point's metric (material folded in)
// is multiplied by ratio[block of its element] = gamma_new / gamma_old; the
// mixed form's (hi, lo) copy is rebuilt from the scaled FP64 value.
__global__ void rescale_metric_kernel(double* __restrict__ G, float2* __restrict__ G32, long long Qtot, int3 Qn, int3 q,
                                      int3 epb, int3 nb, const double* __restrict__ ratio) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= Qtot) return;
    const long long qx = i % Qn.x, r = i / Qn.x, qy = r % Qn.y, qz = r / Qn.y;
    const int bx = (int)(qx / q.x) / epb.x, by = (int)(qy / q.y) / epb.y, bz = (int)(qz / q.z) / epb.z;
    const double f = ratio[(bz * nb.y + by) * nb.x + bx];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double v = f * G[k * Qtot + i];
        G[k * Qtot + i] = v;
        if (G32) {
            const float hi = __double2float_rn(v);
            G32[k * Qtot + i] = make_float2(hi, __double2float_rn(v - (double)hi));
        }
    }
}

cudaError_t launch_rescale_metric(double* G64, float2* G32, const HodgeQuadArgs& a, const int epb[3], const int nb[3],
                                  const double* ratio, cudaStream_t s) {
    const int3 Qn = make_int3(a.Qn[0], a.Qn[1], a.Qn[2]), q = make_int3(a.q[0], a.q[1], a.q[2]);
    const int3 e = make_int3(epb[0], epb[1], epb[2]), b = make_int3(nb[0], nb[1], nb[2]);
    if (a.Qtot == 0) return cudaSuccess;
    rescale_metric_kernel<<<(unsigned)((a.Qtot + 255) / 256), 256, 0, s>>>(G64, G32, a.Qtot, Qn, q, e, b, ratio);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ per-block mass derivative, quadrature Hodge
// For every element: sum over its Gauss points of z(q)^T G(q) d(q) (z, d
// interpolated by sum factorisation exactly as in the Hodge apply), reduced
// over the CTA and added, times scale[block], into out[block of the element].
// With G = w gamma J^T J / det J and gamma = 1/eps_c on block c,
// dG/deps_c = -G / eps_c, so scale[c] = -1/eps_c gives z^T (dM~/deps_c) d.
constexpr int kPairThreads = 128;

__device__ void interp_component(const HodgeQuadArgs& A, const double* __restrict__ x, int c, const int el[3],
                                 double* U, double* T1, double* T2, double* X, const double* Bv) {
    const int qx = A.q[0], qy = A.q[1], qz = A.q[2], Qe = qx * qy * qz;
    const DevComp C = A.field.c[c];
    const int rx = A.deg[c][0] + 1, ry = A.deg[c][1] + 1, rz = A.deg[c][2] + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
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
    for (int t = tid; t < rz * ry * qx; t += nt) {
        const int a = t % qx, rr = t / qx;
        double acc = 0.0;
        for (int r0 = 0; r0 < rx; ++r0) acc = fma(Bx[a * kRMax + r0], X[rr * rx + r0], acc);
        T1[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < rz * qy * qx; t += nt) {
        const int a = t % qx, rr = t / qx, b = rr % qy, r2 = rr / qy;
        double acc = 0.0;
        for (int r1 = 0; r1 < ry; ++r1) acc = fma(By[b * kRMax + r1], T1[(r2 * ry + r1) * qx + a], acc);
        T2[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < Qe; t += nt) {
        const int ab = t % (qx * qy), g = t / (qx * qy);
        double acc = 0.0;
        for (int r2 = 0; r2 < rz; ++r2) acc = fma(Bz[g * kRMax + r2], T2[r2 * qx * qy + ab], acc);
        U[t] = acc;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kPairThreads) hodge_quad_pair_kernel(HodgeQuadArgs A, PairArgs P,
                                                                       const double* __restrict__ z,
                                                                       const double* __restrict__ d,
                                                                       double* __restrict__ out) {
    extern __shared__ double smp[];
    const int e = blockIdx.x;
    const int ex = e % A.nel[0], exy = e / A.nel[0], ey = exy % A.nel[1], ez = exy / A.nel[1];
    const int el[3] = {ex, ey, ez};
    const int qx = A.q[0], qy = A.q[1], qz = A.q[2], Qe = qx * qy * qz;
    double* Uz = smp;                  // 3 * Qe
    double* Ud = Uz + 3 * Qe;          // 3 * Qe
    double* T1 = Ud + 3 * Qe;          // Qe * kRMax
    double* T2 = T1 + Qe * kRMax;      // Qe * kRMax
    double* X = T2 + Qe * kRMax;       // kRMax^3
    double* Bv = X + kRMax * kRMax * kRMax;  // 3 x 8 x kRMax
    double* red = Bv + 3 * 8 * kRMax;  // kPairThreads / 32
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int c = 0; c < 3; ++c) {
        for (int t = tid; t < 3 * 8 * kRMax; t += nt) {
            const int a = t / (8 * kRMax), rem = t % (8 * kRMax), qp = rem / kRMax, r = rem % kRMax;
            if (qp < A.q[a])
                Bv[t] = __ldg(A.bval[a] + (((long long)A.kinds[c][a] * A.nel[a] + el[a]) * A.q[a] + qp) * kRMax + r);
        }
        __syncthreads();
        interp_component(A, z, c, el, Uz + c * Qe, T1, T2, X, Bv);
        interp_component(A, d, c, el, Ud + c * Qe, T1, T2, X, Bv);
    }
    double acc = 0.0;
    for (int t = tid; t < Qe; t += nt) {
        const int a = t % qx, rr = t / qx, b = rr % qy, g = rr / qy;
        const long long qi = ((long long)(ez * qz + g) * A.Qn[1] + (ey * qy + b)) * A.Qn[0] + (ex * qx + a);
        const double g00 = __ldg(A.G + qi), g01 = __ldg(A.G + A.Qtot + qi), g02 = __ldg(A.G + 2 * A.Qtot + qi);
        const double g11 = __ldg(A.G + 3 * A.Qtot + qi), g12 = __ldg(A.G + 4 * A.Qtot + qi);
        const double g22 = __ldg(A.G + 5 * A.Qtot + qi);
        const double d0 = Ud[t], d1 = Ud[Qe + t], d2 = Ud[2 * Qe + t];
        acc = fma(Uz[t], g00 * d0 + g01 * d1 + g02 * d2, acc);
        acc = fma(Uz[Qe + t], g01 * d0 + g11 * d1 + g12 * d2, acc);
        acc = fma(Uz[2 * Qe + t], g02 * d0 + g12 * d1 + g22 * d2, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) red[tid / 32] = acc;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < nt / 32; ++w) s += red[w];
        const int blk = ((ez / P.epb[2]) * P.nb[1] + ey / P.epb[1]) * P.nb[0] + ex / P.epb[0];
        atomicAdd(out + blk, P.scale[blk] * s);
    }
}

cudaError_t launch_hodge_quad_pair(const HodgeQuadArgs& a, const PairArgs& p, const double* z, const double* d,
                                   double* out, cudaStream_t s) {
    const int nel = a.nel[0] * a.nel[1] * a.nel[2];
    const int Qe = a.q[0] * a.q[1] * a.q[2];
    const size_t smem =
        (6 * Qe + 2 * Qe * kRMax + kRMax * kRMax * kRMax + 3 * 8 * kRMax + kPairThreads / 32) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(hodge_quad_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    if (nel > 0) hodge_quad_pair_kernel<<<nel, kPairThreads, smem, s>>>(a, p, z, d, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ per-block mass derivative, block Kronecker
// Identity map, material constant on tiles: per tile t (inside block c),
//   z_t^T gamma_t (Mz_t (x) My_t (x) Mx_t) d_t
// by the three banded passes of the block Hodge apply, then the dot with the
// tile's z, reduced and added, times scale[c], into out[c].  gamma_t = 1/eps_c,
// so scale[c] = -1/eps_c gives z^T (dM~/deps_c) d.
constexpr int kBlockPairThreads = 256;

__global__ void __launch_bounds__(kBlockPairThreads) hodge_block_pair_kernel(HodgeBlockArgs A, PairArgs P,
                                                                             const double* __restrict__ z,
                                                                             const double* __restrict__ x,
                                                                             double* __restrict__ out) {
    extern __shared__ double sb[];
    const int c = blockIdx.y;
    const int tile = blockIdx.x;
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
    constexpr int kLd = kLMax + 1;
    double* Mx = sb;
    double* My = Mx + kLMax * kLd;
    double* Mz = My + kLMax * kLd;
    double* red = Mz + kLMax * kLd;       // kBlockPairThreads / 32
    double* s0 = red + kBlockPairThreads / 32;
    const int Lx = L[0], Ly = L[1], Lz = L[2];
    const int nloc = Lx * Ly * Lz;
    double* s1 = s0 + nloc;
    for (int t = threadIdx.x; t < kLMax * kLMax; t += blockDim.x) {
        const int dd = (t / kLMax) * kLd + t % kLMax;
        Mx[dd] = __ldg(gmat[0] + t);
        My[dd] = __ldg(gmat[1] + t);
        Mz[dd] = gam * __ldg(gmat[2] + t);
    }
    const DevComp C = A.field.c[c];
    const long long nxy = (long long)C.n[0] * C.n[1];
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {
        const int ii = t % Lx, r = t / Lx, jj = r % Ly, kk = r / Ly;
        s0[t] = __ldg(x + C.off + (f0[0] + ii) + (long long)C.n[0] * (f0[1] + jj) + nxy * (f0[2] + kk));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {  // x pass
        const int ii = t % Lx, row = t - ii;
        const int lo = max(0, ii - dg[0]), hi = min(Lx - 1, ii + dg[0]);
        double acc = 0.0;
        for (int m = lo; m <= hi; ++m) acc = fma(Mx[ii * kLd + m], s0[row + m], acc);
        s1[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {  // y pass
        const int ii = t % Lx, r = t / Lx, jj = r % Ly, kk = r / Ly;
        const int lo = max(0, jj - dg[1]), hi = min(Ly - 1, jj + dg[1]);
        double acc = 0.0;
        for (int m = lo; m <= hi; ++m) acc = fma(My[jj * kLd + m], s1[(kk * Ly + m) * Lx + ii], acc);
        s0[t] = acc;
    }
    __syncthreads();
    double acc = 0.0;
    for (int t = threadIdx.x; t < nloc; t += blockDim.x) {  // z pass, dot with z
        const int ii = t % Lx, r = t / Lx, jj = r % Ly, kk = r / Ly;
        const int lo = max(0, kk - dg[2]), hi = min(Lz - 1, kk + dg[2]);
        double v = 0.0;
        for (int m = lo; m <= hi; ++m) v = fma(Mz[kk * kLd + m], s0[(m * Ly + jj) * Lx + ii], v);
        acc = fma(__ldg(z + C.off + (f0[0] + ii) + (long long)C.n[0] * (f0[1] + jj) + nxy * (f0[2] + kk)), v, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kBlockPairThreads / 32; ++w) s += red[w];
        const int blk = P.tile_block[tile];
        atomicAdd(out + blk, P.scale[blk] * s);
    }
}

cudaError_t launch_hodge_block_pair(const HodgeBlockArgs& a, const PairArgs& p, const double* z, const double* x,
                                    double* out, cudaStream_t s) {
    const int ntiles = a.ntile[0] * a.ntile[1] * a.ntile[2];
    const size_t smem =
        (3 * kLMax * (kLMax + 1) + kBlockPairThreads / 32 + 2 * (size_t)a.max_nloc) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(hodge_block_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((3 * kLMax * (kLMax + 1) + kBlockPairThreads / 32 + 2 * kLMax * kLMax * kLMax) *
                                   sizeof(double)));
        attr = true;
    }
    if (ntiles > 0) hodge_block_pair_kernel<<<dim3(ntiles, 3), kBlockPairThreads, smem, s>>>(a, p, z, x, out);
    return cudaGetLastError();
}

}  // namespace smx
