// Dense mode products of the mixed step on the 5th-generation tensor cores.
//
// Along one axis every line of a component is multiplied by a dense n x n
// line operator B -- A^{-1} (pairing sweep, Eq. kroninverse) or A^{-1} M (the
// fused separable Hodge star).  For the 128 lines of one tile that is a GEMM
//   D[line][i] = sum_k X[line][k] B[i][k],   M = 128 lines, N = K = n,
// with n padded to npad (a multiple of 16; padding is zero).
//
// Precision.  Each FP32 value v is split into three BF16 terms
// v0 = bf16(v), v1 = bf16(v - v0), v2 = bf16(v - v0 - v1) (each subtraction
// exact in FP32); the operator is split the same way on the host from its
// FP64 values.  Six products
//   X2 B0 + X1 B1 + X0 B2 + X1 B0 + X0 B1 + X0 B0
// keep every term down to about 2^-24 of the result (the three dropped terms
// are below 2^-25), accumulated in FP32 in tensor memory: the accuracy of an
// FP32 dot product at BF16 tensor-core rates.
//
// Shared-memory operands: no swizzle, K-major canonical layout.  Element
// (row r, k) of an R-row operand is at byte
//   (k / 8) * (16 R + 16) + 16 r + 2 (k % 8),
// i.e. 8-row x 16-byte core matrices, SBO (next 8 rows) = 128 B and LBO (next
// 8 k) = 16 R + 16 B; the extra 16 B puts consecutive k-chunks on different
// banks.  One tcgen05.mma (kind::f16, BF16 in, FP32 accumulate, M = 128,
// N = npad, K = 16) consumes two k-chunks.
//
// One CTA = one tile of kTcLines = 64 lines of one component, 256 threads.
// The MMA is M = 128; rows 64..127 are zero.  Half-filled tiles double the
// number of CTAs (about 200 at 64^3, against 152 SMs): the pass is bound by
// load latency, not by the tensor pipe, so more CTAs in flight is what counts.
//   1. warp 0 allocates tensor memory; B's three parts are copied to shared
//      memory with cp.async (the table already has the shared layout);
//   2. all threads issue every load of their items first, then split the
//      values and store the three BF16 parts (zero past the last line, zero
//      k past n);
//   3. one thread issues 6 x npad/16 MMAs and commits them to an mbarrier;
//   4. warps 0, 1, 4, 5 read TMEM lanes 0..63 (the lines), half the columns
//      each, and write the outputs: directly for the y and z sweeps
//      (consecutive lanes are consecutive addresses), through shared memory
//      for the x sweep (rows are contiguous there, so the tile is written as
//      one contiguous run).  Optionally the last sweep also writes the
//      result widened to FP64 (out64), which saves a separate cast kernel.
// The completion wait gives up after one second: it then sets bit 0 of the
// status word, skips the epilogue and still frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "convert.cuh"
#include "internal.h"
#include "pdl.cuh"
#include "tcgen05.cuh"

namespace smx {
namespace {

using namespace tc;

constexpr int kTcRows = 128;     // MMA M = TMEM lanes
constexpr int kTcLines = 64;     // lines per tile (rows kTcLines..127 are zero)
constexpr int kTcItems = (kTcLines * ((kModeMaxN + 15) / 16 * 2) + 255) / 256;  // (line, k-chunk) items per thread
constexpr int kTcThreads = 256;  // 8 warps: lane quarter = warp % 4, column half = warp / 4
constexpr int kTcHeader = 128;   // mbarrier + TMEM address holder
__device__ __forceinline__ float as_f32(double x) { return d2f_rn(x); }
__device__ __forceinline__ float as_f32(float x) { return x; }

// v = v0 + v1 + v2 in BF16 (the subtractions are exact in FP32).
__device__ __forceinline__ void split3(float v, uint32_t& h0, uint32_t& h1, uint32_t& h2) {
    const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(b0);
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b1);
    const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
    h0 = __bfloat16_as_ushort(b0);
    h1 = __bfloat16_as_ushort(b1);
    h2 = __bfloat16_as_ushort(b2);
}

__host__ __device__ inline int tc_tmem_cols(int npad) {
    int c = 32;
    while (c < npad) c *= 2;
    return c;
}

__host__ __device__ inline int tc_smem_bytes(int npad) {
    const int kc = npad / 8;
    return kTcHeader + 3 * kc * (16 * kTcRows + 16) + 3 * kc * (16 * npad + 16);
}

// Products (data part, operator part), smallest first.
__constant__ int kTcPairX[6] = {2, 1, 0, 1, 0, 0};
__constant__ int kTcPairB[6] = {0, 1, 2, 0, 1, 0};

template <class TIN>
__global__ void __launch_bounds__(kTcThreads) mode_tc_kernel(ModeTcArgs A, const TIN* in, float* out, double* out64) {
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_wait();
    const int c = blockIdx.y;
    const DevComp C = A.field.c[c];
    const int axis = A.axis;
    const int n = C.n[axis];
    if (n <= 0) return;
    const int nlines = C.n[0] * C.n[1] * C.n[2] / n;
    const int l0 = blockIdx.x * kTcLines;
    if (l0 >= nlines) return;  // whole CTA, before any allocation
    const int npad = A.npad[c], kc = npad / 8;
    const uint32_t lbA = 16 * kTcRows + 16, lbB = 16 * npad + 16;
    const int apart = kc * lbA, bpart = kc * lbB;
    unsigned char* sA = smem + kTcHeader;
    unsigned char* sB = sA + 3 * apart;
    const uint32_t mbar = smem_u32(smem);
    uint32_t* holder = reinterpret_cast<uint32_t*>(smem + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = (uint32_t)tc_tmem_cols(npad);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) mbar_init(mbar, 1);

    // operator parts: 3 * bpart bytes, already in the shared layout
    const unsigned char* Bg = static_cast<const unsigned char*>(A.B[c]);
    for (int t = tid; t < 3 * bpart / 16; t += kTcThreads) cp_async16(sB + 16 * t, Bg + 16 * t);

    // data tile: items (row r < kTcLines, k-chunk q) of 8 values each; every
    // load of a thread is issued before the first value is split
    const int nx = C.n[0], nxy = C.n[0] * C.n[1];
    const int stride = axis == 0 ? 1 : (axis == 1 ? nx : nxy);
    const TIN* src = in + C.off;
    const int nitems = kTcLines * kc;
    float val[kTcItems][8];
#pragma unroll
    for (int it = 0; it < kTcItems; ++it) {
        const int g = tid + it * kTcThreads;
        int r, q;
        if (axis == 0) {  // k-chunk fastest: a row's values are contiguous
            r = g / kc;
            q = g - r * kc;
        } else {  // row fastest: consecutive lines are consecutive addresses
            q = g / kTcLines;
            r = g - q * kTcLines;
        }
        const int L = l0 + r;
        const bool live = g < nitems && L < nlines;
        const long long base =
            axis == 0 ? (long long)L * n : (axis == 1 ? (long long)(L % nx) + (long long)(L / nx) * nxy : L);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int k = 8 * q + t;
            val[it][t] = (live && k < n) ? as_f32(src[base + (long long)k * stride]) : 0.0f;
        }
    }
#pragma unroll
    for (int it = 0; it < kTcItems; ++it) {
        const int g = tid + it * kTcThreads;
        if (g >= nitems) break;
        int r, q;
        if (axis == 0) {
            r = g / kc;
            q = g - r * kc;
        } else {
            q = g / kTcLines;
            r = g - q * kTcLines;
        }
        uint32_t w0[4] = {0, 0, 0, 0}, w1[4] = {0, 0, 0, 0}, w2[4] = {0, 0, 0, 0};
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            uint32_t h0, h1, h2;
            split3(val[it][t], h0, h1, h2);
            const int sh = 16 * (t & 1);
            w0[t >> 1] |= h0 << sh;
            w1[t >> 1] |= h1 << sh;
            w2[t >> 1] |= h2 << sh;
        }
        unsigned char* dst = sA + q * lbA + 16 * r;
        *reinterpret_cast<uint4*>(dst) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        *reinterpret_cast<uint4*>(dst + apart) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *reinterpret_cast<uint4*>(dst + 2 * apart) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
    }
    // rows kTcLines..127 of the MMA tile are zero
    for (int g = tid; g < (kTcRows - kTcLines) * kc; g += kTcThreads) {
        const int q = g / (kTcRows - kTcLines), r = kTcLines + g - q * (kTcRows - kTcLines);
        unsigned char* dst = sA + q * lbA + 16 * r;
        const uint4 z = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(dst) = z;
        *reinterpret_cast<uint4*>(dst + apart) = z;
        *reinterpret_cast<uint4*>(dst + 2 * apart) = z;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;

    if (tid == 0) {
        const uint32_t idesc = idesc_bf16_f32(kTcRows, npad);
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        uint32_t acc = 0;
        for (int pr = 0; pr < 6; ++pr) {
            const uint32_t pa = a0 + kTcPairX[pr] * apart, pb = b0 + kTcPairB[pr] * bpart;
            for (int ks = 0; ks < kc / 2; ++ks) {
                mma_bf16(tmem, smem_desc(pa + 2 * ks * lbA, lbA, 128), smem_desc(pb + 2 * ks * lbB, lbB, 128), idesc,
                         acc);
                acc = 1;
            }
        }
        mma_commit(mbar);
    }
    // every thread's wait is bounded, so all reach the barrier; the verdict is uniform
    const bool ok = __syncthreads_and(mbar_wait_bounded(mbar, 0)) != 0;
    tc_fence_after();
    if (!ok) {
        if (lane == 0) atomicOr(A.status, 1u);
    } else {
        // lanes 0..63 hold the lines: warps 0, 1 (quarters 0, 1) and 4, 5 (same quarters, other column half)
        const int quarter = warp & 3;
        const bool reader = quarter < kTcLines / 32;
        const int half = npad / 2, c0 = (warp >> 2) * half;
        const int r = 32 * quarter + lane, L = l0 + r;
        const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
        float* stage = reinterpret_cast<float*>(sA);  // x sweep: kTcLines x (n | 1) floats, the A parts are consumed
        const int S = n | 1;
        const long long base = axis == 0 ? 0 : (axis == 1 ? (long long)(L % nx) + (long long)(L / nx) * nxy : L);
        float* dst = out + C.off;
        double* dst64 = out64 ? out64 + C.off : nullptr;
        if (reader)
            for (int ch = 0; ch < half / 8; ++ch) {
                const int col = c0 + 8 * ch;
                float v[8];
                tmem_ld8(trow + (uint32_t)col, v);
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int i = col + t;
                    if (i >= n) continue;
                    if (axis == 0) {
                        stage[r * S + i] = v[t];
                    } else if (L < nlines) {
                        const long long o = base + (long long)i * stride;
                        dst[o] = v[t];
                        if (dst64) dst64[o] = f2d_exact(v[t]);
                    }
                }
            }
        if (axis == 0) {
            __syncthreads();
            const int nl = min(kTcLines, nlines - l0);
            const long long o0 = (long long)l0 * n;
            for (int g = tid; g < nl * n; g += kTcThreads) {
                const int rr = g / n;
                const float v = stage[rr * S + (g - rr * n)];
                dst[o0 + g] = v;
                if (dst64) dst64[o0 + g] = f2d_exact(v);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    pdl_trigger();  // after the tensor memory is released
}

}  // namespace

int mode_tc_npad(int n) { return (n + 15) / 16 * 16; }

cudaError_t launch_mode_tc(const ModeTcArgs& a, const double* in64, const float* in32, float* out, double* out64,
                           cudaStream_t s) {
    long long maxlines = 0;
    int maxpad = 0;
    for (int c = 0; c < 3; ++c) {
        const long long nc = (long long)a.field.c[c].n[0] * a.field.c[c].n[1] * a.field.c[c].n[2];
        const int n = a.field.c[c].n[a.axis];
        if (n <= 0) continue;
        if (n > kModeMaxN || a.npad[c] != mode_tc_npad(n)) return cudaErrorInvalidValue;
        maxlines = std::max(maxlines, nc / n);
        maxpad = std::max(maxpad, a.npad[c]);
    }
    if (maxlines == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        const int mx = tc_smem_bytes(mode_tc_npad(kModeMaxN));
        cudaFuncSetAttribute(mode_tc_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(mode_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        attr = true;
    }
    const dim3 grid((unsigned)((maxlines + kTcLines - 1) / kTcLines), 3);
    const size_t smem = (size_t)tc_smem_bytes(maxpad);
    if (in64)
        return launch_k(mode_tc_kernel<double>, grid, dim3(kTcThreads), smem, s, a, in64, out, out64);
    return launch_k(mode_tc_kernel<float>, grid, dim3(kTcThreads), smem, s, a, in32, out, out64);
}

}  // namespace smx
