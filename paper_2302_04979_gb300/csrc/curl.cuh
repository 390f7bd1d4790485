// Discrete curl by incidence matrices (Eq. discrete2_faraday / discrete2_ampere;
// Remark on incidence matrices after Table 1), shared by the FP64 step (T =
// double) and the mixed step (T = float: FP32 differences, FP64 state update).
//
// Incidence along axis a:
//   primal (d u)_m = u_m - u_{m-1}, u_m = 0 outside [0, n_a) (removed BC functions);
//   dual   (d u)_m = u_{m+1} - u_m (the input has one more entry along a).
// (curl u)_c = d_{c+1} u_{c+2} - d_{c+2} u_{c+1}.
//
// Grid: x = blocks of kCurlThreads points of one component's (i, j) plane,
// y = chunks of kCurlKz planes along z, z = component.  Every thread marches
// through its chunk, so a CTA is always full and each thread has several
// independent outputs in flight.  The component is a template parameter, so
// every extent and stride is a compile-time field of the argument block.
#pragma once

#include <cuda_runtime.h>

#include "convert.cuh"
#include "internal.h"
#include "pdl.cuh"

namespace smx {


template <int A, bool DUAL, class T>
__device__ __forceinline__ T incidence_t(const DevComp& u, const T* __restrict__ v, int i, int j, int k) {
    const int idx = i + u.n[0] * (j + u.n[1] * k);
    const int stride = A == 0 ? 1 : (A == 1 ? u.n[0] : u.n[0] * u.n[1]);
    const T* p = v + u.off + idx;
    if (DUAL) return __ldg(p + stride) - __ldg(p);
    const int m = A == 0 ? i : (A == 1 ? j : k);
    const T hi = (m < u.n[A]) ? __ldg(p) : T(0);
    const T lo = (m >= 1) ? __ldg(p - stride) : T(0);
    return hi - lo;
}

__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return f2d_exact(v); }

template <int C, bool DUAL, class T>
__device__ __forceinline__ void curl_plane_comp(const DevField& IN, const DevField& OUT, const T* __restrict__ in,
                                                double* __restrict__ out, double alpha,
                                                const double* __restrict__ jhat, const double* __restrict__ amp,
                                                int amp_index, double s_host, int p, int k0,
                                                double* __restrict__ zero) {
    constexpr int a1 = (C + 1) % 3, a2 = (C + 2) % 3;
    const DevComp& O = OUT.c[C];
    const int nx = O.n[0], nxy = O.n[0] * O.n[1];
    if (p >= nxy) return;
    const int j = p / nx, i = p - j * nx;
    const int nk = min(kCurlKz, O.n[2] - k0);
    double s = 0.0;
    if (DUAL && jhat != nullptr) s = amp != nullptr ? __ldg(amp + amp_index) : s_host;
    // every load of the chunk first (the stores below cannot be hoisted over by the compiler), then the updates
    T d1[kCurlKz], d2[kCurlKz];
    double o[kCurlKz], jv[kCurlKz];
#pragma unroll
    for (int kk = 0; kk < kCurlKz; ++kk) {
        if (kk < nk) {
            const int k = k0 + kk;
            const long long g = O.off + p + (long long)nxy * k;
            d1[kk] = incidence_t<a1, DUAL, T>(IN.c[a2], in, i, j, k);
            d2[kk] = incidence_t<a2, DUAL, T>(IN.c[a1], in, i, j, k);
            o[kk] = out[g];
            jv[kk] = (DUAL && jhat != nullptr) ? __ldg(jhat + g) : 0.0;
        }
    }
#pragma unroll
    for (int kk = 0; kk < kCurlKz; ++kk) {
        if (kk < nk) {
            double v = widen(d1[kk] - d2[kk]);
            if (DUAL && jhat != nullptr) v = fma(-s, jv[kk], v);
            const long long g = O.off + p + (long long)nxy * (k0 + kk);
            out[g] = fma(alpha, v, o[kk]);
            if (zero) zero[g] = 0.0;  // the accumulation target of the next Hodge apply
        }
    }
}

template <bool DUAL, class T>
__global__ void __launch_bounds__(kCurlThreads) curl_plane_kernel(DevField IN, DevField OUT, const T* __restrict__ in,
                                                                  double* __restrict__ out, double alpha,
                                                                  const double* __restrict__ jhat,
                                                                  const double* __restrict__ amp, int amp_index,
                                                                  double s_host, double* __restrict__ zero) {
    pdl_wait();
    const int p = blockIdx.x * kCurlThreads + threadIdx.x;
    const int k0 = blockIdx.y * kCurlKz;
    if (blockIdx.z == 0)
        curl_plane_comp<0, DUAL, T>(IN, OUT, in, out, alpha, jhat, amp, amp_index, s_host, p, k0, zero);
    else if (blockIdx.z == 1)
        curl_plane_comp<1, DUAL, T>(IN, OUT, in, out, alpha, jhat, amp, amp_index, s_host, p, k0, zero);
    else
        curl_plane_comp<2, DUAL, T>(IN, OUT, in, out, alpha, jhat, amp, amp_index, s_host, p, k0, zero);
    pdl_trigger();
}

template <bool DUAL, class T>
static cudaError_t launch_curl_t(const DevField& IN, const DevField& OUT, const T* in, double* out, double alpha,
                                 const double* jhat, const double* amp, int amp_index, double s_host, cudaStream_t s,
                                 double* zero = nullptr) {
    if (OUT.total == 0) return cudaSuccess;
    int plane = 0, nz = 0;
    for (int c = 0; c < 3; ++c) {
        plane = max(plane, OUT.c[c].n[0] * OUT.c[c].n[1]);
        nz = max(nz, OUT.c[c].n[2]);
    }
    const dim3 grid((plane + kCurlThreads - 1) / kCurlThreads, (nz + kCurlKz - 1) / kCurlKz, 3);
    return launch_k(curl_plane_kernel<DUAL, T>, grid, dim3(kCurlThreads), 0, s, IN, OUT, in, out, alpha, jhat, amp,
                    amp_index, s_host, zero);
}

}  // namespace smx
