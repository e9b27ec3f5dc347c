// Integer arithmetic of the fixed-point patch apply (k_patch_fixed.cu), for
// the device and, so that it can be checked against exact rational
// arithmetic, for the host: exact scaling and round-to-nearest-even of a
// double to an integer, the binary exponent of a double, the split of a
// 57/58-bit integer into two 29-bit limbs, and the correctly rounded double
// of an exact 128-bit limb sum.  No FP64 arithmetic instruction is used
// (the library's ldexp only outside the normal range).
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define FX_HD __host__ __device__ __forceinline__
#else
#define FX_HD inline
#endif

namespace irkmg {

FX_HD uint64_t fx_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

FX_HD double fx_from_bits(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}

FX_HD int fx_clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// round(x · 2^k) to the nearest integer, ties to even, for |x · 2^k| ≤ 2^62,
// from the bits of x (|x| = m 2^e with a 53-bit integer m): a shift of m,
// with round-half-even on the bits shifted out.
FX_HD int64_t fx_scale_round(double x, int k) {
  const uint64_t b = fx_bits(x);
  const int ef = (int)((b >> 52) & 0x7ff);
  uint64_t m = b & 0xfffffffffffffull;
  int e = -1074;
  if (ef != 0) {
    m |= 1ull << 52;
    e = ef - 1075;
  }
  const int sh = e + k;
  uint64_t v;
  if (sh >= 0) {
    v = m << sh;
  } else if (sh <= -64) {
    v = 0;  // m < 2^53: below one half
  } else {
    const int r = -sh;
    const uint64_t q = m >> r, rem = m & ((1ull << r) - 1), half = 1ull << (r - 1);
    v = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
  }
  return (b >> 63) ? -(int64_t)v : (int64_t)v;
}

// F with |y| < 2^F ≤ 2|y| for y > 0 (the exponent frexp returns), from the bits.
FX_HD int fx_exponent(double y) {
  const uint64_t b = fx_bits(y);
  const int ef = (int)((b >> 52) & 0x7ff);
  if (ef != 0) return ef - 1022;
  return -1010 - fx_clz64(b & 0xfffffffffffffull);  // subnormal
}

// q = hi 2^29 + lo with lo in [−2^28, 2^28) (lo: the low 29 bits of q read as
// a signed number); |q| ≤ 2^58 gives |hi| ≤ 2^29.
FX_HD void fx_split29(int64_t q, int32_t* hi, int32_t* lo) {
  const int32_t l = (int32_t)((int64_t)((uint64_t)q << 35) >> 35);
  *lo = l;
  *hi = (int32_t)((q - l) >> 29);
}

// The double nearest to t · 2^e (ties to even) for the exact sum
// t = a[0] 2^58 + (a[1] + a[2]) 2^29 + a[3], |t| < 2^127: the top 64 bits of
// |t| (the rest folded into a sticky bit), rounded to 53 bits and packed with
// the exponent by integer operations.  A result below the normal range is
// rounded once, from the same 64 bits and sticky bit, to a multiple of
// 2^−1074 (the subnormal spacing); an overflow goes through the library's
// ldexp (an exact m 2^X, or infinity).
FX_HD double fx_round(const int64_t* a, int e) {
  const __int128 t = (__int128)a[0] * ((__int128)1 << 58) +
                     ((__int128)a[1] + (__int128)a[2]) * ((__int128)1 << 29) + (__int128)a[3];
  if (t == 0) return 0.0;
  const bool neg = t < 0;
  const unsigned __int128 u = neg ? (unsigned __int128)0 - (unsigned __int128)t : (unsigned __int128)t;
  const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
  uint64_t w;  // |t| ~ w 2^x, top bit of w at 63
  int x;
  if (hi == 0) {
    const int lz = fx_clz64(lo);
    w = lo << lz;
    x = -lz;
  } else {
    const int sh = 64 - fx_clz64(hi);  // 1 .. 63
    w = (uint64_t)(u >> sh) | (uint64_t)((lo << (64 - sh)) != 0);
    x = sh;
  }
  uint64_t m = w >> 11;
  const uint64_t rem = w & 0x7ff;
  if (rem > 0x400 || (rem == 0x400 && (m & 1))) ++m;
  int X = x + e + 11;  // |t 2^e| rounds to m 2^X, m in [2^52, 2^53]
  if (m >> 53) {
    m >>= 1;
    ++X;
  }
  const int be = X + 52 + 1023;
  if (be <= 0) {
    // |t 2^e| = w 2^(x+e) rounds to k 2^−1074: shift w right by sh >= 11
    const int sh = -(x + e + 1074);
    uint64_t k;
    if (sh >= 65) {
      k = 0;  // below a quarter of the spacing
    } else if (sh == 64) {
      k = w > (1ull << 63) ? 1 : 0;  // w 2^−64 in [1/2, 1): an exact half goes to 0 (even)
    } else {
      const uint64_t q = w >> sh, rem = w & ((1ull << sh) - 1), half = 1ull << (sh - 1);
      k = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
    }
    return fx_from_bits(((uint64_t)neg << 63) | k);  // k = 2^52 packs the least normal
  }
  if (be >= 2047) {
    const double d = ldexp((double)m, X);
    return neg ? -d : d;
  }
  return fx_from_bits(((uint64_t)neg << 63) | ((uint64_t)be << 52) | (m & 0xfffffffffffffull));
}

}  // namespace irkmg
