// Fixed-point slicing of FP64 values into seven 7-bit digits that BF16 holds exactly, for the
// FP64-accurate products on the tensor cores (T update of the UDT chain, trailing updates of the
// blocked QR). A row or column with largest magnitude in [2^e, 2^(e+1)) is written as
//   v = 2^(e - 6) sum_{s=0..6} d_s 2^(-7 s) + r,   |d_0| <= 128, |d_s| <= 64 (s >= 1), |r| <= 2^(e - 49),
// with integer arithmetic only (the FP64 pipe is the scarce unit). Products of two such operands
// summed per level a + b are exact in FP32 accumulators while the level's sum of absolute terms
// stays below 2^24 (after Ozaki, Ogita, Oishi, Rump 2012).
#pragma once

#include <cuda_bf16.h>

namespace slmc {
namespace s7 {

constexpr int kS = 7;  // slices per operand

__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// |v| as an ordered integer (the bit pattern without the sign), and its warp maximum.
__device__ __forceinline__ long long abs_bits(double v) { return __double_as_longlong(v) & 0x7fffffffffffffffll; }

__device__ __forceinline__ long long warp_max_bits(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Power of two of the largest |v| from its bit pattern (0 for a zero row or column).
__device__ __forceinline__ int exponent_of_bits(long long m) {
    return m == 0 ? 0 : (int)((m >> 52) & 0x7ff) - 1023;
}

// The seven slices of v in units of 2^(e - 6 - 42), with integer arithmetic only (the FP64 pipe
// is the scarce unit): v is rounded once to n = round(v 2^(48 - e)) (|n| <= 2^49, half away from
// zero) and n is written in balanced base-128 digits d_6..d_1 in [-64, 63] and d_0 = the rest,
// |d_0| <= 128, so v ~ 2^(e - 6) sum_s d_s 2^(-7 s). Each digit is exact in BF16.
__device__ __forceinline__ void slice7(double v, int e, __nv_bfloat16 (&q)[kS]) {
    const long long bits = __double_as_longlong(v);
    const int ex = (int)((bits >> 52) & 0x7ff);
    long long n = 0;
    const int r = 1027 + e - ex;  // right shift of the 53-bit significand; >= 4 whenever |v| < 2^(e + 1)
    if (ex != 0 && r < 63) {
        const long long m = (bits & 0xfffffffffffffll) | 0x10000000000000ll;
        n = r > 0 ? (m + (1ll << (r - 1))) >> r : m;
        if (bits < 0) n = -n;
    }
#pragma unroll
    for (int s = kS - 1; s >= 1; --s) {
        const int d = (int)((n + 64) & 127) - 64;
        n = (n - d) >> 7;
        q[s] = __ushort_as_bfloat16((unsigned short)(__float_as_uint((float)d) >> 16));
    }
    q[0] = __ushort_as_bfloat16((unsigned short)(__float_as_uint((float)n) >> 16));
}

}  // namespace s7
}  // namespace slmc
