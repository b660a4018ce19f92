// Exact arithmetic shared by host and device code: correctly rounded
// conversion of a 128-bit integer to double.  The local-moving phase's
// tolerance test compares (double)(2 * gain) / (double)(2m)^2 with tau;
// when the test runs on the device it must take the same decision as the
// host, whose compiler converts 128-bit integers with round-to-nearest-even,
// so the device does the same, written from the IEEE 754 definition: keep
// the 53 most significant bits, round half to even on the bits below.
#pragma once
#include <cstdint>

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#define __device__
#endif
#endif

namespace lv {

// Number of leading zero bits of a non-zero 64-bit value.
__host__ __device__ inline int clz64(uint64_t v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}

// v * 2^e for an integer-valued v < 2^54 and 0 <= e < 128 (exact: a power of
// two times a double with at most 54 significant bits stays representable).
__host__ __device__ inline double scale2(double v, int e) {
  while (e >= 60) {
    v *= 1152921504606846976.0;  // 2^60
    e -= 60;
  }
  return v * (double)(1ull << e);
}

// Round-to-nearest-even conversion of an unsigned 128-bit value (hi, lo).
__host__ __device__ inline double u128_to_double(uint64_t hi, uint64_t lo) {
  if (hi == 0) {
    if (lo < (1ull << 53)) return (double)lo;  // exact
  }
  // top bit position p (>= 53): value = hi * 2^64 + lo
  const int p = hi ? 127 - clz64(hi) : 63 - clz64(lo);
  const int shift = p - 52;  // bits below the 53 kept ones
  uint64_t mant, rest_hi = 0, rest_lo;  // kept bits; dropped bits as a 128-bit value
  if (shift >= 64) {
    mant = hi >> (shift - 64);
    rest_hi = shift > 64 ? hi & ((1ull << (shift - 64)) - 1) : 0;
    rest_lo = lo;
  } else {
    mant = (hi << (64 - shift)) | (lo >> shift);
    if (shift == 0) mant = lo;
    rest_lo = shift ? lo & ((1ull << shift) - 1) : 0;
  }
  // compare the dropped bits with half of the last kept bit: 2^(shift - 1)
  int cmp;  // -1 below half, 0 exactly half, 1 above
  if (shift == 0) {
    cmp = -1;
  } else if (shift - 1 >= 64) {
    const uint64_t half_hi = 1ull << (shift - 1 - 64);
    cmp = rest_hi > half_hi || (rest_hi == half_hi && rest_lo > 0) ? 1 : (rest_hi == half_hi && rest_lo == 0) ? 0 : -1;
  } else {
    const uint64_t half_lo = 1ull << (shift - 1);
    cmp = rest_hi > 0 || rest_lo > half_lo ? 1 : rest_lo == half_lo ? 0 : -1;
  }
  if (cmp > 0 || (cmp == 0 && (mant & 1ull))) ++mant;  // may reach 2^53: still exact after scaling
  return scale2((double)mant, shift);
}

// Signed 128-bit value given as (hi, lo) two's complement halves.
__host__ __device__ inline double i128_to_double(int64_t hi, uint64_t lo) {
  if (hi < 0) {
    const uint64_t nlo = ~lo + 1ull;
    const uint64_t nhi = ~(uint64_t)hi + (nlo == 0 ? 1ull : 0ull);
    return -u128_to_double(nhi, nlo);
  }
  return u128_to_double((uint64_t)hi, lo);
}

}  // namespace lv
