// Correct rounding of exact integer sums to FP64 with integer operations
// (shared by the product epilogue and the selector's label kernel).
#pragma once
#include <cstdint>

namespace emul {

// Correctly rounded double of T * 2^sh (round to nearest even), computed with
// integer operations on the IEEE-754 fields (overflow gives +-inf, results
// below the normal range are rounded as subnormals).
__device__ __noinline__ static double rn_scaled(__int128 T, int sh) {
  if (T == 0) return 0.0;
  const bool neg = T < 0;
  const unsigned __int128 mag = neg ? (unsigned __int128)(-(T + 1)) + 1u : (unsigned __int128)T;
  const uint64_t hi = (uint64_t)(mag >> 64), lo = (uint64_t)mag;
  const int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  const int E = msb + sh;
  const uint64_t sign = neg ? 0x8000000000000000ull : 0ull;
  if (E > 1023) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  const int keep = (E >= -1022) ? msb - 52 : -1074 - sh;   // bit of mag kept as the last mantissa bit
  uint64_t q;
  if (keep <= 0) {
    q = (uint64_t)(mag << (-keep));
  } else {
    if (keep > msb + 1) return __longlong_as_double((long long)sign);   // below half the smallest subnormal
    q = (uint64_t)(mag >> keep);
    const unsigned __int128 rem = mag - ((unsigned __int128)q << keep);
    const unsigned __int128 half = (unsigned __int128)1 << (keep - 1);
    if (rem > half || (rem == half && (q & 1ull))) q += 1;
  }
  const uint64_t bits = (E >= -1022) ? ((uint64_t)(E + 1022) << 52) + q : q;
  return __longlong_as_double((long long)(sign | bits));
}

}  // namespace emul
