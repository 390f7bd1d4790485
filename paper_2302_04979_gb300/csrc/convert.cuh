// FP64 <-> FP32 conversions on the integer pipe.
//
// On GB300 the hardware conversion instructions issue on the FP64 pipe, which
// runs at 1/63 of the FP32 rate, so a kernel that converts every value it
// touches spends most of its issue slots there.  These helpers do the IEEE 754
// conversions with integer operations for the values that occur in practice
// (normal numbers and zeros) and hand the rare rest (float subnormals,
// infinities, NaN) to the hardware conversion, so every input converts exactly
// as the hardware would.
#pragma once

#include <cuda_runtime.h>

namespace smx {

// The hardware conversions of the rare inputs.  Out of line, so that the compiler
// cannot turn the branches below into selects that run the slow conversion for
// every input.
static __device__ __noinline__ float d2f_hw(double x) { return static_cast<float>(x); }
static __device__ __noinline__ double f2d_hw(float v) { return static_cast<double>(v); }

// double -> float, round to nearest even (IEEE 754 default rounding).
__device__ __forceinline__ float d2f_rn(double x) {
    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned sign = static_cast<unsigned>(u >> 32) & 0x80000000u;
    const int e = static_cast<int>((u >> 52) & 0x7FF);  // biased FP64 exponent
    if (e == 0) return __uint_as_float(sign);           // +-0 and FP64 subnormals (< 2^-1022) round to +-0
    // normal FP32 result: FP32 exponent e - 1023 + 127 in [1, 253] (253 leaves room for the rounding carry)
    if (e < 897 || e > 1149) return d2f_hw(x);
    const unsigned long long m = u & 0xFFFFFFFFFFFFFull;  // 52 stored mantissa bits
    unsigned f = (static_cast<unsigned>(e - 896) << 23) | static_cast<unsigned>(m >> 29);
    const unsigned rest = static_cast<unsigned>(m & 0x1FFFFFFFull);  // the 29 dropped bits
    const unsigned half = 0x10000000u;
    f += (rest > half || (rest == half && (f & 1u))) ? 1u : 0u;  // a mantissa carry moves into the exponent
    return __uint_as_float(f | sign);
}

// float -> double (exact).
__device__ __forceinline__ double f2d_exact(float v) {
    const unsigned u = __float_as_uint(v);
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned long long sign = static_cast<unsigned long long>(u & 0x80000000u) << 32;
    if ((u & 0x7FFFFFFFu) == 0) return __longlong_as_double(static_cast<long long>(sign));
    if (e == 0 || e == 255) return f2d_hw(v);  // subnormal, inf, nan
    const unsigned long long d =
        sign | (static_cast<unsigned long long>(e + 896) << 52) | (static_cast<unsigned long long>(u & 0x7FFFFFu) << 29);
    return __longlong_as_double(static_cast<long long>(d));
}

}  // namespace smx
