// Mode products on the 5th-generation tensor cores by exact digit slicing: the
// FP64 step's line operators (seven digits) and the mixed step's tensor-core
// option (four digits).  The description below is for seven digits; the
// four-digit instantiation reads FP64 or FP32 lines, forms 31-bit fixed-point
// images (|X| < 2^31), accumulates levels 0..3 (10 digit products) and rounds
// the result once to FP32 (optionally also writing it widened to FP64).
//
// Along one axis every line x of a component becomes B x, with B the dense
// n x n line operator -- A^{-1} (pairing sweep, Eq. kroninverse) or A^{-1} M
// (the fused separable Hodge star).  The FP64 pipe of GB300 issues one warp
// DFMA per 64 cycles per SM sub-partition, so the FP64 line recurrences are
// bound by it; here the arithmetic runs on the BF16 tensor pipe instead, with
// results as accurate as an FP64 dot product.
//
// Digits.  Each line L is scaled by its own power of two sigma_L (from the
// largest exponent on the line) so that every entry becomes an integer
// X = round(x / sigma_L) with |X| < 2^55, written with seven balanced base-256
// digits, X = sum_t d_t 256^(6-t), d_t in [-128, 128] (exact in BF16).  Each
// operator row i is treated the same way on the host (scale tau_i, digits e_s).
// The digit products
//   P_ts[i][L] = sum_k e_s[i][k] d_t[L][k]
// are integers below 80 * 128^2 = 2^20.3; the products of one level
// l = s + t (at most seven of them) are accumulated in one FP32 tensor-memory
// accumulator, where every partial sum is an integer below 2^24 and hence exact.
// Levels 0..6 are formed.  The rounding of each entry to the line's fixed point
// (2^-55 of the line's largest entry, of the row's largest for the operator)
// and the dropped levels 7..12 keep the error within a few units of
// 2^-53 (max |x| sum |B_ik| + max |B_ik| sum |x|): comparable to the error
// bound of an FP64 dot product, and the same as FP64 wherever the entries of
// a line have similar size.  The levels are combined by Horner's rule in
// 64-bit integer arithmetic as they arrive,
//   acc = sum_{l<=5} P_l 256^(5-l) + floor(P_6 / 256)   (|acc| < 2^61),
// and acc * 2^56 * sigma_L * tau_i is rounded once to the nearest double
// (sigma_L = 2^(E_L - 1077), tau_i = 2^(F_i - 1077) for the largest exponent
// fields).  No FP64 instruction is issued on the normal path.
//
// Tile.  One CTA = NL lines of one component (NL = 96, or 128 where that
// still gives every SM a tile), 512 threads.  MMA (kind::f16,
// BF16 in, FP32 accumulate): M = 128 operator rows, N = NL lines, K = npad
// (n rounded up to 16); 28 digit pairs of npad / 16 instructions each.
// Tensor memory holds a ring of 512 / NL level accumulators of NL columns.
// Shared memory: the operator's seven digit planes and the tile's seven digit
// planes, both K-major in the 32-byte swizzle layout: per atom column of 16 K
// values, R rows of 32 bytes (8-row groups of 256 bytes, SBO 256), the two
// 16-byte halves of row r exchanged when bit 2 of r is set; atom columns
// follow each other (R x 32 bytes apart).  The operator planes store only its
// rows rounded up to 8 (R = r8): an MMA still reads 128 rows, and rows
// r8..127 are whatever follows in shared memory -- they only feed
// tensor-memory lanes r8..127, which are never used.
//   1. warp 0 allocates the ring's tensor memory; the operator digits are
//      copied with cp.async (one contiguous run: the table has this layout);
//   2. the tile's FP64 values are loaded as bit patterns, the largest
//      exponent of each line is found with shared-memory atomics, and every
//      value is cut into its digits: the offset C = 0x80808080808080 turns the
//      balanced digits of X into the bytes of X + C (d_t = byte - 128, the top
//      digit from 9 bits), and a biased digit b becomes BF16 through the FP32
//      value (2^23 + b) - (2^23 + 128);
//   3. one thread of warp 3 issues the MMAs level by level into the ring and
//      commits each level to that buffer's "full" mbarrier; before reusing a
//      buffer it waits on the buffer's "drained" mbarrier;
//   4. meanwhile the warps of the lane quarters that hold operator rows (at
//      most quarters 0..2; THREADS / 128 warps per quarter, each owning an
//      equal share of the NL columns) take each level as it
//      completes, fold it into their Horner accumulators and release the
//      buffer; after level 6 they round and write the outputs: directly for
//      the x sweep (consecutive rows are consecutive addresses), through
//      shared memory for the y and z sweeps (there consecutive lines are
//      consecutive addresses).
// Every mbarrier wait gives up after one second: the thread then sets bit 0
// of the status word and skips the rest of its work; the CTA still meets at
// its final barrier and frees its tensor memory.
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

constexpr int kDgRows = 128;       // MMA M: operator rows (TMEM lanes)
constexpr int kDgIssuer = 3;       // the warp (lane quarter 3: rows 96..127, never an output) issuing MMAs
constexpr int kDgKcMax = (kModeMaxN + 15) / 16 * 2;  // k-chunks of 8 at the largest npad
constexpr uint32_t kDgTmemCols = 512;
constexpr int kDgHeader = 2560;    // 8 full + 8 drained mbarriers, TMEM address, line exponents (<= 128),
                                   // row exponents (<= 80), line base offsets (<= 128)
constexpr int kDgSmemMax = 232448;  // opt-in shared memory per CTA

static_assert(kModeMaxN <= 96, "operator rows must stay in lane quarters 0..2");

__host__ __device__ inline int dg_op_bytes(int npad, int r8, int nd) { return nd * (npad / 16) * r8 * 32; }
__host__ __device__ inline int dg_x_bytes(int npad, int nl, int nd) { return nd * (npad / 16) * nl * 32; }
// after the last MMA the tile planes hold the final accumulators: r8 rows of nl + 1 64-bit words
__host__ __device__ inline int dg_acc_bytes(int nl, int r8) { return r8 * (nl + 1) * 8; }
// header, 256 bytes of slack to align the planes to the swizzle pattern, operator and tile planes
__host__ __device__ inline int dg_smem_bytes(int nl, int npad, int r8, int nd) {
    const int x = dg_x_bytes(npad, nl, nd), acc = dg_acc_bytes(nl, r8);
    return kDgHeader + 256 + dg_op_bytes(npad, r8, nd) + (x > acc ? x : acc);
}

// Bit-pattern layout of the two input formats.
template <class T>
struct Fmt;
template <>
struct Fmt<double> {
    using U = unsigned long long;
    static constexpr int kMant = 52, kBias = 1023;
    static constexpr unsigned kExpMask = 0x7FF;
    static __device__ __forceinline__ U bits(const double* p, long long i) {
        return reinterpret_cast<const unsigned long long*>(p)[i];
    }
};
template <>
struct Fmt<float> {
    using U = uint32_t;
    static constexpr int kMant = 23, kBias = 127;
    static constexpr unsigned kExpMask = 0xFF;
    static __device__ __forceinline__ U bits(const float* p, long long i) {
        return reinterpret_cast<const uint32_t*>(p)[i];
    }
};

// The integer image of a bit pattern relative to the exponent field E (the
// largest of the line, at least 1) for ND digits: X = round(v / sigma) with
// |X| < 2^(8 ND - 1), the line's largest significand shifted left by
// kTop = 8 ND - 1 - (kMant + 1) (negative: right), sigma = 2^(E - kBias - kMant -
// kTop).  Returned as X + C with C = 128 (256^ND - 1) / 255 (0x80...80):
// 0 < X + C < 2^(8 ND + 1).  With d_t the balanced base-256 digits of X (d_1..
// d_(ND-1) in [-128, 127], d_0 in [-128, 128]), bytes 0..ND-2 of X + C are
// d_(ND-1) + 128 .. d_1 + 128 and bits 8(ND-1)..8ND are d_0 + 128.
template <class TIN, int ND>
__device__ __forceinline__ unsigned long long digit_word(typename Fmt<TIN>::U bits, int E) {
    using F = Fmt<TIN>;
    constexpr int kTop = 8 * ND - 1 - (F::kMant + 1);
    const int e = (int)((bits >> F::kMant) & F::kExpMask);
    const unsigned long long frac = (unsigned long long)bits & ((1ull << F::kMant) - 1);
    const int eff = e ? e : 1;
    const unsigned long long M = e ? (frac | (1ull << F::kMant)) : frac;
    const int sh = E - eff - kTop;  // right shift of the significand (negative: left)
    unsigned long long mag;
    if (sh <= 0) {
        mag = M << (-sh);
    } else {
        mag = sh >= 60 ? 0ull : (M + (1ull << (sh - 1))) >> sh;
    }
    const bool neg = (bits >> (8 * sizeof(bits) - 1)) != 0;
    const unsigned long long x = neg ? (0ull - mag) : mag;
    return x + (0x8080808080808080ull >> (64 - 8 * ND));
}

// log2 of sigma for an exponent field E (see digit_word).
template <class TIN, int ND>
__device__ __forceinline__ int digit_scale(int E) {
    return E - Fmt<TIN>::kBias - Fmt<TIN>::kMant - (8 * ND - 1 - (Fmt<TIN>::kMant + 1));
}

// FP32 pattern of (byte j of w) - 128, exact: PRMT builds 0x4B0000bb = 2^23 + b,
// the subtraction of 2^23 + 128 is exact, and the BF16 pattern of the result
// is its top half (at most 8 significant bits).
__device__ __forceinline__ uint32_t digit_f32(uint32_t w, int j) {
    const uint32_t f = __byte_perm(w, 0x4B000000u, (uint32_t)j | 0x7540u);
    return __float_as_uint(__uint_as_float(f) - 8388736.0f);
}
// The same for the top digit, whose biased value (bits 8(ND-1)..8ND) may reach 256.
template <int ND>
__device__ __forceinline__ uint32_t top_digit_f32(unsigned long long u) {
    return __float_as_uint(__uint_as_float(0x4B000000u | (uint32_t)(u >> (8 * (ND - 1)))) - 8388736.0f);
}

// acc * 2^e2 rounded to the nearest double (ties to even), by integer
// instructions while the result is a normal number.  The significand m keeps its
// leading bit (2^52 <= m <= 2^53), so adding it to (biased exponent - 1) << 52
// lets a rounding carry (m = 2^53) step the exponent by itself.
__device__ __noinline__ double scaled_to_double_slow(long long acc, int e2) {
    const unsigned long long a = acc < 0 ? (unsigned long long)(-acc) : (unsigned long long)acc;
    int pb = 63 - __clzll((long long)a);
    unsigned long long m;
    if (pb <= 52) {
        m = a << (52 - pb);
    } else {
        const int sh = pb - 52;
        m = a >> sh;
        const unsigned long long rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (m & 1ull))) {
            m += 1;
            if (m >> 53) {
                m >>= 1;
                pb += 1;
            }
        }
    }
    // outside the normal range: exact m times 2^k in two power-of-two factors
    const int k = pb - 52 + e2;
    const int k1 = max(-1022, min(1023, k / 2)), k2 = max(-1022, min(1023, k - k1));
    const double f1 = __longlong_as_double((long long)(k1 + 1023) << 52);
    const double f2 = __longlong_as_double((long long)(k2 + 1023) << 52);
    const double v = (double)(long long)m * f1 * f2;
    return acc < 0 ? -v : v;
}

__device__ __forceinline__ double scaled_to_double(long long acc, int e2) {
    if (acc == 0) return 0.0;
    const unsigned long long a = acc < 0 ? 0ull - (unsigned long long)acc : (unsigned long long)acc;
    const int lz = __clzll((long long)a);
    unsigned long long m;
    if (lz >= 11) {
        m = a << (lz - 11);
    } else {
        const int sh = 11 - lz;  // round half to even: add half - 1, plus 1 when the kept part is odd
        m = (a + ((1ull << (sh - 1)) - 1) + ((a >> sh) & 1ull)) >> sh;
    }
    const int be = 63 - lz + e2 + 1023;  // biased exponent without a rounding carry
    if (be < 1 || be + (int)(m >> 53) > 2046) return scaled_to_double_slow(acc, e2);
    const unsigned long long bits = ((unsigned long long)(be - 1) << 52) + m;
    return __longlong_as_double((long long)(bits | ((unsigned long long)acc & (1ull << 63))));
}

// Outside the normal range: through the double routine (out of line, as above).
__device__ __noinline__ float scaled_to_float_slow(long long acc, int e2) {
    return (float)scaled_to_double(acc, e2);
}

// acc * 2^e2 rounded to the nearest float (ties to even), the same way (through the
// double routine outside the normal range).
__device__ __forceinline__ float scaled_to_float(long long acc, int e2) {
    if (acc == 0) return 0.0f;
    const unsigned long long a = acc < 0 ? 0ull - (unsigned long long)acc : (unsigned long long)acc;
    const int lz = __clzll((long long)a);
    unsigned long long m;
    if (lz >= 40) {
        m = a << (lz - 40);
    } else {
        const int sh = 40 - lz;
        m = (a + ((1ull << (sh - 1)) - 1) + ((a >> sh) & 1ull)) >> sh;
    }
    const int be = 63 - lz + e2 + 127;
    if (be < 1 || be + (int)(m >> 24) > 254) return scaled_to_float_slow(acc, e2);
    const uint32_t bits = ((uint32_t)(be - 1) << 23) + (uint32_t)m;
    return __uint_as_float(bits | (acc < 0 ? 0x80000000u : 0u));
}

// Output of a tile entry: FP64, or FP32 with an optional exact FP64 copy.
__device__ __forceinline__ double digit_out(long long acc, int e2, double*) { return scaled_to_double(acc, e2); }
__device__ __forceinline__ float digit_out(long long acc, int e2, float*) { return scaled_to_float(acc, e2); }


template <int NL, int ND, int THREADS, class TIN, class TOUT>
__global__ void __launch_bounds__(THREADS, THREADS == 256 ? 2 : 1)
    mode_digit_kernel(ModeDigitArgs A, const TIN* in, TOUT* out, double* out64) {
    using U = typename Fmt<TIN>::U;
    constexpr int kGroups = THREADS / 128;                     // reader warps per lane quarter
    constexpr int kBufs = ND < (int)kDgTmemCols / NL ? ND : (int)kDgTmemCols / NL;  // level buffers in the ring
    constexpr uint32_t kCols = kBufs * NL <= 128 ? 128u : (kBufs * NL <= 256 ? 256u : 512u);
    constexpr int kCpw = NL / kGroups;                         // columns (lines) per reader warp
    constexpr int kItems = (NL * kDgKcMax + THREADS - 1) / THREADS;
    constexpr int kTopOp = 8 * ND - 1 - 53;                    // operator rows: FP64 significands
    static_assert(kCpw % 8 == 0 && kBufs >= 1 && kBufs * NL <= (int)kDgTmemCols, "tile shape");
    extern __shared__ __align__(1024) unsigned char smem[];
    // nothing before pdl_wait reads what the previous kernel of the stream writes:
    // the operator table, tensor memory and the barriers are set up while it drains
    const int c = blockIdx.y;
    const DevComp C = A.field.c[c];
    const int axis = A.axis;
    const int n = C.n[axis];
    if (n <= 0) return;
    const int nlines = C.n[0] * C.n[1] * C.n[2] / n;
    const int l0 = blockIdx.x * NL;
    if (l0 >= nlines) return;  // whole CTA, before any allocation
    const int npad = A.npad[c], kc = npad / 8, r8 = (n + 7) & ~7;
    const int colA = 32 * r8, colX = 32 * NL;  // bytes per atom column (16 K values)
    const int opPlane = (npad / 16) * colA, xPlane = (npad / 16) * colX;
    const uint32_t full0 = smem_u32(smem), drained0 = full0 + 64;
    uint32_t* holder = reinterpret_cast<uint32_t*>(smem + 128);
    int* sExp = reinterpret_cast<int*>(smem + 256);
    int* sRowE = reinterpret_cast<int*>(smem + 1024);
    long long* sBase = reinterpret_cast<long long*>(smem + 1536);  // offset of each line's first entry
    unsigned char* sOp = smem + kDgHeader + ((256u - ((smem_u32(smem) + kDgHeader) & 255u)) & 255u);
    unsigned char* sX = sOp + dg_op_bytes(npad, r8, ND);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, group = warp >> 2;
    const int nquarters = (n + 31) / 32;          // lane quarters holding output rows (<= 3)
    const bool reader = quarter < nquarters;      // warp-uniform

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0)
        for (int b = 0; b < kBufs; ++b) {
            mbar_init(full0 + 8 * b, 1);
            mbar_init(drained0 + 8 * b, kGroups * nquarters);
        }
    if (tid < NL) sExp[tid] = 1;
    if (tid < n) sRowE[tid] = A.rowexp[c][tid];  // the table, not the previous kernel's output
    const int nx = C.n[0], nxy = C.n[0] * C.n[1];
    const int stride = axis == 0 ? 1 : (axis == 1 ? nx : nxy);
    // each line's base offset once (the only run-time integer divisions of the kernel: on GB300
    // they go through the conversion pipe, so none is left in the per-entry loops)
    if (tid < NL) {
        const int L = l0 + tid;
        sBase[tid] = axis == 0 ? (long long)L * n : (axis == 1 ? (long long)(L % nx) + (long long)(L / nx) * nxy : L);
    }
    // g / kc for the x sweep by a multiply: exact for g < 2^32 / kc^2 (here g < NL kc <= 1280)
    const unsigned kcMagic = 0xFFFFFFFFu / (unsigned)kc + 1u;
    __syncthreads();

    // operator digits: the table is the shared layout, one contiguous copy
    const unsigned char* Bg = static_cast<const unsigned char*>(A.B[c]);
    for (int t = tid; t < ND * opPlane / 16; t += THREADS) cp_async16(sOp + 16 * t, Bg + 16 * (size_t)t);
    pdl_wait();  // the input lines are the previous kernel's output

    // data tile as bit patterns: items (line r, k-chunk q) of 8 values
    const TIN* src = in + C.off;
    const int nitems = NL * kc;
    U val[kItems][8];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int g = tid + it * THREADS;
        int r, q;
        if (axis == 0) {  // k-chunk fastest: a line's values are contiguous
            r = (int)__umulhi((unsigned)g, kcMagic);
            q = g - r * kc;
        } else {  // line fastest: consecutive lines are consecutive addresses
            q = g / NL;
            r = g - q * NL;
        }
        const int L = l0 + r;
        const bool live = g < nitems && L < nlines;
        const long long base = live ? sBase[r] : 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int k = 8 * q + t;
            val[it][t] = (live && k < n) ? Fmt<TIN>::bits(src, base + (long long)k * stride) : (U)0;
        }
    }
    __syncthreads();  // sExp initialised
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int g = tid + it * THREADS;
        if (g >= nitems) break;
        const int r = axis == 0 ? g / kc : g % NL;
        int emax = 1;
#pragma unroll
        for (int t = 0; t < 8; ++t) emax = max(emax, (int)((val[it][t] >> Fmt<TIN>::kMant) & Fmt<TIN>::kExpMask));
        atomicMax(sExp + r, emax);
    }
    __syncthreads();
    // every item's line exponent before any digit-plane store (a load may not pass a store
    // that might alias it, which would serialise the items)
    int Ev[kItems];
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int g = tid + it * THREADS;
        const int r = axis == 0 ? (int)__umulhi((unsigned)g, kcMagic) : g % NL;
        Ev[it] = g < nitems ? sExp[r] : 1;
    }
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
        const int g = tid + it * THREADS;
        if (g >= nitems) break;
        int r, q;
        if (axis == 0) {
            r = (int)__umulhi((unsigned)g, kcMagic);
            q = g - r * kc;
        } else {
            q = g / NL;
            r = g - q * NL;
        }
        const int E = Ev[it];
        uint32_t w[ND][4];
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            const unsigned long long u0 = digit_word<TIN, ND>(val[it][t], E);
            const unsigned long long u1 = digit_word<TIN, ND>(val[it][t + 1], E);
            const uint32_t lo0 = (uint32_t)u0, hi0 = (uint32_t)(u0 >> 32);
            const uint32_t lo1 = (uint32_t)u1, hi1 = (uint32_t)(u1 >> 32);
#pragma unroll
            for (int j = 0; j < ND - 1; ++j) {  // byte j -> digit plane ND-1-j; two BF16 per word
                const uint32_t f0 = digit_f32(j < 4 ? lo0 : hi0, j & 3), f1 = digit_f32(j < 4 ? lo1 : hi1, j & 3);
                w[ND - 1 - j][t >> 1] = __byte_perm(f0, f1, 0x7632);
            }
            w[0][t >> 1] = __byte_perm(top_digit_f32<ND>(u0), top_digit_f32<ND>(u1), 0x7632);
        }
        // atom column q / 2, row r, 16-byte half (q & 1) exchanged by bit 2 of r
        unsigned char* dst = sX + (q >> 1) * colX + 32 * r + 16 * ((q & 1) ^ ((r >> 2) & 1));
#pragma unroll
        for (int s = 0; s < ND; ++s)
            *reinterpret_cast<uint4*>(dst + s * xPlane) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;
    bool ok = true;
    TOUT* dst = out + C.off;
    double* dst64 = out64 ? out64 + C.off : nullptr;
    long long* sAcc = reinterpret_cast<long long*>(sX);  // n x (NL + 1) final accumulators, after the last MMA

    if (warp == kDgIssuer) {
        // the whole warp runs the issue loop with warp-uniform values; one elected lane issues
        // each MMA and commit (level l into buffer l % kBufs, every digit pair t + s = l,
        // k-step by k-step; the first MMA of a level overwrites the buffer)
        constexpr uint32_t idesc = idesc_bf16_f32(kDgRows, NL);
        const uint64_t dA0 = smem_desc_sw32(smem_u32(sOp), 256), dB0 = smem_desc_sw32(smem_u32(sX), 256);
        const uint64_t stA = (uint64_t)(colA >> 4), stB = (uint64_t)(colX >> 4);
        const uint64_t plA = (uint64_t)(opPlane >> 4), plB = (uint64_t)(xPlane >> 4);
        const int nks = kc / 2;
        for (int lv = 0; lv < ND && ok; ++lv) {
            const int buf = lv % kBufs;
            if (lv >= kBufs) {
                ok = __all_sync(0xffffffffu, mbar_wait_bounded(drained0 + 8 * buf, ((lv - kBufs) / kBufs) & 1));
                tc_fence_after();
                if (!ok) break;
            }
            const uint32_t d = tmem + (uint32_t)(buf * NL);
            for (int t = 0; t <= lv; ++t) {
                uint64_t a = dA0 + (uint64_t)(lv - t) * plA, b = dB0 + (uint64_t)t * plB;
                mma_bf16_elect(d, a, b, idesc, t ? 1u : 0u);
                for (int ks = 1; ks < nks; ++ks) {
                    a += stA;
                    b += stB;
                    mma_bf16_elect(d, a, b, idesc, 1u);
                }
            }
            mma_commit_elect(full0 + 8 * buf);
        }
        if (!ok && lane == 0) atomicOr(A.status, 1u);
    } else if (reader) {
        const int i = 32 * quarter + lane;  // operator row = output entry along the line
        const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(group * kCpw);
        unsigned long long acc[kCpw];  // Horner accumulators, two's complement (wraps only on unused rows)
#pragma unroll
        for (int j = 0; j < kCpw; ++j) acc[j] = 0;
        for (int lv = 0; lv < ND; ++lv) {
            const int buf = lv % kBufs;
            ok = __all_sync(0xffffffffu, mbar_wait_bounded_sleep(full0 + 8 * buf, (lv / kBufs) & 1, 128));
            if (!ok) break;
            tc_fence_after();
            uint32_t v[kCpw / 8][8];
#pragma unroll
            for (int ch = 0; ch < kCpw / 8; ++ch) tmem_ld8_issue(trow + (uint32_t)(buf * NL + 8 * ch), v[ch]);
            tmem_wait_ld();
#pragma unroll
            for (int ch = 0; ch < kCpw / 8; ++ch) tmem_pin8(v[ch]);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(drained0 + 8 * buf);  // this warp is done with the buffer
#pragma unroll
            for (int ch = 0; ch < kCpw / 8; ++ch)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    // exact: the accumulators hold integers below 2^24
                    const long long p = __float2int_rn(__uint_as_float(v[ch][j]));
                    unsigned long long& a = acc[8 * ch + j];
                    a = lv < ND - 1 ? a * 256ull + (unsigned long long)p : a + (unsigned long long)(p >> 8);
                }
        }
        if (!ok) {
            if (lane == 0) atomicOr(A.status, 1u);
        } else if (i < n) {
            // every MMA has completed, so the tile planes are free: the accumulators go to
            // shared memory and all warps share the final rounding (the warps of the output
            // rows' lane quarters sit on only two or three of the four SM sub-partitions)
#pragma unroll
            for (int j = 0; j < kCpw; ++j) sAcc[i * (NL + 1) + group * kCpw + j] = (long long)acc[j];
        }
    }
    ok = __syncthreads_and(ok) != 0;
    pdl_trigger();  // the next kernel may be scheduled; its pdl_wait still waits for this grid
    if (ok) {
        // acc * 2^(8 ND) * sigma_L * tau_i rounded once; consecutive threads write consecutive
        // addresses: entries of one line along x, consecutive lines along y and z
        const int nl = min(NL, nlines - l0);
        // every shared-memory load of a batch before any global store: each rounding is a chain of
        // dependent integer instructions, and a load may not pass a store that might alias it
        if (axis == 0) {
            // one warp per line, lanes along the line's entries (contiguous in memory)
            constexpr int kR = (kModeMaxN + 31) / 32;
            for (int col = warp; col < nl; col += THREADS / 32) {
                const long long base = sBase[col];
                const int es = digit_scale<TIN, ND>(sExp[col]);
                long long av[kR];
                int e2v[kR];
#pragma unroll
                for (int j = 0; j < kR; ++j) {
                    const int ii = lane + 32 * j;
                    const int iis = ii < n ? ii : 0;
                    av[j] = sAcc[iis * (NL + 1) + col];
                    e2v[j] = 8 * ND + sRowE[iis] - 1075 - kTopOp + es;
                }
#pragma unroll
                for (int j = 0; j < kR; ++j) {
                    const int ii = lane + 32 * j;
                    const TOUT y = digit_out(av[j], e2v[j], (TOUT*)nullptr);
                    if (ii < n) {
                        dst[base + ii] = y;
                        if (dst64) dst64[base + ii] = f2d_exact(y);
                    }
                }
            }
        } else {
            // consecutive threads: consecutive lines (consecutive addresses)
            constexpr int kU = 4;
            const int total = n * NL;
            for (int g0 = tid; g0 < total; g0 += kU * THREADS) {
                long long av[kU], ov[kU];
                int e2v[kU];
                bool live[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int g = g0 + u * THREADS;
                    const int ii = g / NL, col = g - ii * NL;
                    live[u] = g < total && col < nl;
                    const int iis = live[u] ? ii : 0, cols = live[u] ? col : 0;
                    av[u] = sAcc[iis * (NL + 1) + cols];
                    e2v[u] = 8 * ND + sRowE[iis] - 1075 - kTopOp + digit_scale<TIN, ND>(sExp[cols]);
                    ov[u] = sBase[cols] + (long long)iis * stride;
                }
                TOUT yv[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) yv[u] = digit_out(av[u], e2v[u], (TOUT*)nullptr);
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (live[u]) {
                        dst[ov[u]] = yv[u];
                        if (dst64) dst64[ov[u]] = f2d_exact(yv[u]);
                    }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

}  // namespace

int mode_digit_npad(int n) { return (n + 15) / 16 * 16; }

// Lines per tile of an FP64 sweep.  An M = 128, K = 16 MMA with both operands in
// shared memory takes about 32 + N/4 cycles on GB300 (the operator's 4 KB and the
// tile's N x 32 bytes at 128 bytes per cycle) and N/2 at full rate, so a CTA's
// MMA time grows with its lines while the other phases (load, digit cut,
// rounding) are a fixed latency per CTA: 128-line tiles while they still fill
// all 152 SMs with one wave, else 96 (one wave of 135 CTAs at p = 3, 64^3).
static int digit_tile_lines(const ModeDigitArgs& a, long long maxlines) {
    const long long tiles128 = 3 * ((maxlines + 127) / 128);
    bool fits128 = true;
    for (int c = 0; c < 3; ++c) {
        const int n = a.field.c[c].n[a.axis];
        if (n > 0 && dg_smem_bytes(128, a.npad[c], (n + 7) & ~7, kDigits) > kDgSmemMax) fits128 = false;
    }
    return (fits128 && tiles128 >= 152) ? 128 : 96;
}

// Largest line count of the sweep (0: nothing to do; -1: invalid arguments).
static long long digit_lines(const ModeDigitArgs& a) {
    long long maxlines = 0;
    for (int c = 0; c < 3; ++c) {
        const long long nc = (long long)a.field.c[c].n[0] * a.field.c[c].n[1] * a.field.c[c].n[2];
        const int n = a.field.c[c].n[a.axis];
        if (n <= 0) continue;
        if (n > kModeMaxN || a.npad[c] != mode_digit_npad(n) || !a.B[c] || !a.rowexp[c]) return -1;
        maxlines = std::max(maxlines, nc / n);
    }
    return maxlines;
}

static int digit_smem(const ModeDigitArgs& a, int nl, int nd) {
    int smem = 0;
    for (int c = 0; c < 3; ++c) {
        const int n = a.field.c[c].n[a.axis];
        if (n > 0) smem = std::max(smem, dg_smem_bytes(nl, a.npad[c], (n + 7) & ~7, nd));
    }
    return smem;
}

template <int NL, int ND, int THREADS, class TIN, class TOUT>
static cudaError_t launch_digit_t(const ModeDigitArgs& a, const TIN* in, TOUT* out, double* out64,
                                  long long maxlines, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(mode_digit_kernel<NL, ND, THREADS, TIN, TOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kDgSmemMax);
        attr = true;
    }
    const int smem = digit_smem(a, NL, ND);
    if (smem > kDgSmemMax) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((maxlines + NL - 1) / NL), 3);
    return launch_k(mode_digit_kernel<NL, ND, THREADS, TIN, TOUT>, grid, dim3(THREADS), (size_t)smem, s, a, in, out,
                    out64);
}

cudaError_t launch_mode_digit(const ModeDigitArgs& a, const double* in, double* out, cudaStream_t s) {
    const long long maxlines = digit_lines(a);
    if (maxlines < 0) return cudaErrorInvalidValue;
    if (maxlines == 0) return cudaSuccess;
    return digit_tile_lines(a, maxlines) == 128
               ? launch_digit_t<128, kDigits, 512, double, double>(a, in, out, nullptr, maxlines, s)
               : launch_digit_t<96, kDigits, 512, double, double>(a, in, out, nullptr, maxlines, s);
}

// The mixed step's line operators: four digits, the FP64 kernel's tile shape.
cudaError_t launch_mode_digit_f32(const ModeDigitArgs& a, const double* in64, const float* in32, float* out,
                                  double* out64, cudaStream_t s) {
    const long long maxlines = digit_lines(a);
    if (maxlines < 0) return cudaErrorInvalidValue;
    if (maxlines == 0) return cudaSuccess;
    if (in64) return launch_digit_t<96, kDigitsF32, 512, double, float>(a, in64, out, out64, maxlines, s);
    return launch_digit_t<96, kDigitsF32, 512, float, float>(a, in32, out, out64, maxlines, s);
}

}  // namespace smx
