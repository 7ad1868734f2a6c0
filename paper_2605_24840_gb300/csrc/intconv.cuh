// intconv.cuh -- FP64 <-> FP32 / FP16 conversions by integer operations.
//
// GB300 executes FP64 arithmetic and FP64 conversions at about two per clock
// per SM, while a kernel that streams FP64 data at HBM speed needs about 2.7
// elements per clock per SM: any FP64 instruction per element makes such a
// kernel FP64-bound.  These helpers take the bit patterns apart on the
// integer pipe (and the int -> float conversion) instead.  They compile for
// the host as well, where the tests compare them with the C casts.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define RS_HD __host__ __device__ __forceinline__
#else
#define RS_HD inline
#endif

namespace rsign {

RS_HD uint64_t ic_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  memcpy(&b, &x, 8);
  return b;
#endif
}
RS_HD double ic_double(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}
RS_HD uint32_t ic_fbits(float x) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(x);
#else
  uint32_t b;
  memcpy(&b, &x, 4);
  return b;
#endif
}
RS_HD float ic_float(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  memcpy(&x, &b, 4);
  return x;
#endif
}
// int -> float, round to nearest even
RS_HD float ic_i2f(int v) {
#ifdef __CUDA_ARCH__
  return __int2float_rn(v);
#else
  return (float)v;
#endif
}
RS_HD int ic_msb64(uint64_t v) {  // index of the highest set bit, v != 0
#ifdef __CUDA_ARCH__
  return 63 - __clzll((long long)v);
#else
  return 63 - __builtin_clzll(v);
#endif
}

// floor(log2 |x|) of a normal, finite, nonzero double; -1023 for zero and
// subnormals
RS_HD int ic_exponent(double x) { return (int)((ic_bits(x) >> 52) & 0x7FF) - 1023; }

// x 2^k split into hi + lo: hi the float nearest to x 2^k (ties to even), lo
// the exact remainder x 2^k - hi rounded to the nearest float, so that
// hi + lo = x 2^k to 2^-47 relative.  Values with |x 2^k| < 2^-126 (and
// subnormal x) give hi = lo = 0; a remainder below the normal float range
// gives lo = 0 (an absolute error below 2^-126); |x 2^k| >= 2^128, infinities
// and NaNs give hi = +-inf, lo = 0.
RS_HD void ic_split_f32(double x, int k, float* hi, float* lo) {
  const uint64_t b = ic_bits(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t a = b & 0x7FFFFFFFFFFFFFFFull;
  const int ex = (int)(a >> 52);
  const int e = ex - 1023 + k;  // x 2^k = m 2^(e - 52), m in [2^52, 2^53)
  if (ex == 0 || e < -126) {
    *hi = ic_float(sign);
    *lo = ic_float(sign);
    return;
  }
  if (ex == 2047 || e > 127) {
    *hi = ic_float(sign | 0x7F800000u);
    *lo = ic_float(sign);
    return;
  }
  const uint64_t m = (a & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  uint64_t q = m >> 29;  // 24 significant bits
  const uint64_t rem = m & 0x1FFFFFFFull;
  if (rem > 0x10000000ull || (rem == 0x10000000ull && (q & 1ull))) ++q;
  const int64_t r = (int64_t)m - (int64_t)(q << 29);  // |r| <= 2^28, units of 2^(e - 52)
  int eh = e;
  if (q == (1ull << 24)) {
    q >>= 1;
    ++eh;
  }
  if (eh > 127) {
    *hi = ic_float(sign | 0x7F800000u);
    *lo = ic_float(sign);
    return;
  }
  *hi = ic_float(sign | ((uint32_t)(eh + 127) << 23) | ((uint32_t)q & 0x7FFFFFu));
  if (r == 0) {
    *lo = ic_float(sign);
    return;
  }
  const uint32_t rb = ic_fbits(ic_i2f((int)r));  // rounded to 24 bits
  const int er = (int)((rb >> 23) & 0xFF) + (e - 52);
  if (er <= 0) {
    *lo = ic_float(sign);
    return;
  }
  *lo = ic_float(((rb & 0x807FFFFFu) | ((uint32_t)er << 23)) ^ sign);
}

// The value of an FP16 bit pattern in units of 2^-24 (exact; |v| < 2^40).
RS_HD int64_t ic_f16_units(uint16_t h) {
  const int ex = (h >> 10) & 0x1F;
  const int64_t mant = h & 0x3FF;
  const int64_t v = ex == 0 ? mant : ((mant | 0x400) << (ex - 1));
  return (h & 0x8000) ? -v : v;
}

// v 2^k as a double, exact for |v| < 2^53 (and a normal result)
RS_HD double ic_i64_scaled(int64_t v, int k) {
  if (v == 0) return 0.0;
  const uint64_t sign = v < 0 ? (1ull << 63) : 0ull;
  const uint64_t a = v < 0 ? (uint64_t)(-v) : (uint64_t)v;
  const int msb = ic_msb64(a);
  const uint64_t mant = a << (52 - msb);
  const int e = msb + k;
  return ic_double(sign | ((uint64_t)(e + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull));
}

// a float as a double, exactly (subnormal floats included)
RS_HD double ic_f2d(float f) {
  const uint32_t b = ic_fbits(f);
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  const int ex = (int)((b >> 23) & 0xFF);
  const uint64_t mant = b & 0x7FFFFFu;
  if (ex == 0) {
    if (mant == 0) return ic_double(sign);
    const double v = ic_i64_scaled((int64_t)mant, -149);
    return ic_double(ic_bits(v) | sign);
  }
  const uint64_t e64 = ex == 255 ? 2047 : (uint64_t)(ex - 127 + 1023);
  return ic_double(sign | (e64 << 52) | (mant << 29));
}

}  // namespace rsign
