// FP32 -> scaled FP64 conversion on the integer pipe.
//
// GB300 executes FP64 arithmetic at a small fraction of its FP32 and INT32 rates (about
// 1.25 TFLOP/s on the whole chip). The tensor-core GEMM epilogue widens every FP32 accumulator to
// FP64; as a hardware conversion per element that was a visible part of the GEMM time of the
// n = 16 line workload. This routine works on the IEEE-754 encodings with integer operations:
//   binary32: sign (1 bit), exponent (8 bits, bias 127), fraction (23 bits);
//   binary64: sign (1 bit), exponent (11 bits, bias 1023), fraction (52 bits).
// Only normal numbers take the integer path; zero is handled inline; subnormal, infinite and NaN
// values (none occur in a contraction of unitaries and Kraus operators, but the routine stays
// total) take the hardware conversion and multiply.
#pragma once

#include <cstdint>

namespace ajf {

// Fixed-point unit of the scale correction of f32_to_f64_scaled: scale = 1 + q * 2^-46.
constexpr int kScaleFracBits = 46;

// x (binary32) -> x * (1 + q * 2^-46) (binary64), for |q| < 2^36 (|scale - 1| < 2^-10).
// The 24-bit significand s of a normal x is widened to s * 2^29 (the binary64 significand of x
// exactly) and the correction s * q * 2^-17 is added in 64-bit integer arithmetic (floor), then
// renormalised by at most one bit. The result is within 2 units in the last place (binary64) of
// x * (1 + q * 2^-46); `scale` (that same factor as a double) serves the rare operands.
__device__ __forceinline__ double f32_to_f64_scaled(float x, int64_t q, double scale) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t e = (b >> 23) & 0xFFu;
  const uint64_t sign = static_cast<uint64_t>(b & 0x80000000u) << 32;
  if (e == 0u || e == 0xFFu) {
    if ((b & 0x7FFFFFFFu) == 0u) return __longlong_as_double(static_cast<long long>(sign));  // +-0
    return static_cast<double>(x) * scale;                                                   // rare
  }
  const int64_t s = static_cast<int64_t>((b & 0x7FFFFFu) | 0x800000u);
  int64_t r = (s << 29) + ((s * q) >> (kScaleFracBits - 29));
  uint64_t ex = e + (1023u - 127u);
  if (r >= (int64_t(1) << 53)) {
    r >>= 1;
    ++ex;
  } else if (r < (int64_t(1) << 52)) {
    r <<= 1;
    --ex;
  }
  return __longlong_as_double(
      static_cast<long long>(sign | (ex << 52) | (static_cast<uint64_t>(r) & 0xFFFFFFFFFFFFFull)));
}

}  // namespace ajf
