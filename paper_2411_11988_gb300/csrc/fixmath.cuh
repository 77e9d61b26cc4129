// fixmath.cuh -- exact 128-bit integer helpers of the FP64 pair sweep.
//
// On this part the FP64 unit runs two lanes per clock per SM, so the pair
// sweep keeps its FP64 instructions for the potential itself and does the
// rest in integer arithmetic, which is exact:
//  * squared distances from the 2^-48 A fixed-point displacements, as 128-bit
//    integers in units of 2^-96 A^2 (the cut-off test is then exact);
//  * the binary64 of r^2 rounded once from the integer, whose top bits give
//    the interval key of the DSF table (the offset x = s - s0 inside the
//    interval is then an exact subtraction);
//  * force components f d rounded once to the fixed point of the
//    accumulators from the 53-bit mantissa of f times the integer d.
// The functions compile for the host as well, so that a CPU test can check
// them against exact big-integer arithmetic.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define FM_HD __host__ __device__ __forceinline__
#else
#define FM_HD inline
#endif

namespace fm {

struct u128 {
  unsigned long long hi, lo;
};

FM_HD unsigned long long dbl_bits(double v) {
#if defined(__CUDA_ARCH__)
  return (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long b;
  memcpy(&b, &v, 8);
  return b;
#endif
}

FM_HD double bits_dbl(unsigned long long b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double v;
  memcpy(&v, &b, 8);
  return v;
#endif
}

FM_HD int clz64(unsigned long long a) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)a);
#else
  return a ? __builtin_clzll(a) : 64;
#endif
}

FM_HD u128 mul64(unsigned long long a, unsigned long long b) {
#if defined(__CUDA_ARCH__)
  return u128{__umul64hi(a, b), a * b};
#else
  const unsigned __int128 p = (unsigned __int128)a * b;
  return u128{(unsigned long long)(p >> 64), (unsigned long long)p};
#endif
}

FM_HD u128 add128(u128 a, u128 b) {
  u128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}

FM_HD bool lt128(u128 a, u128 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// bit index of the most significant set bit, -1 for zero
FM_HD int msb128(u128 a) { return a.hi ? 127 - clz64(a.hi) : (a.lo ? 63 - clz64(a.lo) : -1); }

// a >> s for 0 <= s < 128
FM_HD u128 shr128(u128 a, int s) {
  if (s == 0) return a;
  if (s >= 64) return u128{0ull, a.hi >> (s - 64)};
  return u128{a.hi >> s, (a.lo >> s) | (a.hi << (64 - s))};
}

// squared length of an integer vector, |d| < 2^62 per axis
FM_HD u128 norm2(long long dx, long long dy, long long dz) {
  const unsigned long long ax = dx < 0 ? (unsigned long long)(-dx) : (unsigned long long)dx;
  const unsigned long long ay = dy < 0 ? (unsigned long long)(-dy) : (unsigned long long)dy;
  const unsigned long long az = dz < 0 ? (unsigned long long)(-dz) : (unsigned long long)dz;
  return add128(add128(mul64(ax, ax), mul64(ay, ay)), mul64(az, az));
}

// binary64 value of a * 2^-scale for a != 0 with msb p; the bits below the
// 53 kept are dropped with round half up
FM_HD double u128_to_dbl(u128 a, int p, int scale) {
  unsigned long long m;
  if (p <= 52) {
    m = a.lo << (52 - p);
  } else {
    const u128 t = shr128(a, p - 53);  // 54 bits: the kept 53 and the rounding bit
    m = (t.lo + 1ull) >> 1;
    if (m >> 53) {  // rounding carried into a new leading bit
      m >>= 1;
      ++p;
    }
  }
  const unsigned long long e = (unsigned long long)(p - scale + 1023);
  return bits_dbl((e << 52) | (m & 0xFFFFFFFFFFFFFull));
}

// The DSF interval of a positive normal binary64 s (in A^2; 64 sub-intervals
// per octave): returns key = (biased exponent of s << 6) | (its top 6
// mantissa bits), i.e. the top 18 bits of s, and x = s - s0, s0 the interval
// start. s0 <= s < 2 s0 share the exponent, so the subtraction is exact.
FM_HD int dsf_key(double s, double* x) {
  const int key = (int)(dbl_bits(s) >> 46);
  const double s0 = bits_dbl((unsigned long long)key << 46);
#if defined(__CUDA_ARCH__)
  *x = __dsub_rn(s, s0);
#else
  *x = s - s0;
#endif
  return key;
}

// round(f * d * 2^-k) for a normal or zero binary64 f and |d| < 2^62, with
// one rounding (half away from zero); *bad is set when the result would
// reach 2^62 in magnitude, or f is not finite
FM_HD long long mulfix(double f, long long d, int k, int* bad) {
  const unsigned long long b = dbl_bits(f);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0 || d == 0) return 0;
  if (e == 0x7FF) {
    *bad = 1;
    return 0;
  }
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const unsigned long long ad = d < 0 ? (unsigned long long)(-d) : (unsigned long long)d;
  const u128 pr = mul64(m, ad);  // |f d| = pr * 2^(e - 1075)
  const int s = 1075 + k - e;    // result = pr >> s
  unsigned long long r;
  if (s <= 0) {
    *bad = 1;
    return 0;
  } else if (s >= 128) {
    r = 0ull;
  } else {
    const u128 half = s >= 65 ? u128{1ull << (s - 65), 0ull} : u128{0ull, 1ull << (s - 1)};
    const u128 t = shr128(add128(pr, half), s);
    if (t.hi || (t.lo >> 62)) {
      *bad = 1;
      return 0;
    }
    r = t.lo;
  }
  const bool neg = ((b >> 63) != 0) != (d < 0);
  return neg ? -(long long)r : (long long)r;
}

// round(f * 2^scale) for a binary32 f (halves away from zero; subnormal f
// gives 0), by 32-bit integer instructions: f = m 2^(ex - 150) with a 24-bit
// m. *bad is set when the result would reach 2^62 in magnitude, or f is not
// finite. Equal to rounding the exact binary64 of f the same way.
FM_HD long long fixf(float f, int scale, int* bad) {
  unsigned u;
#if defined(__CUDA_ARCH__)
  u = __float_as_uint(f);
#else
  memcpy(&u, &f, 4);
#endif
  const int ex = (int)((u >> 23) & 0xFFu);
  const int sh = ex - 150 + scale;
  const unsigned m = (u & 0x7FFFFFu) | 0x800000u;
  long long r;
  if (ex == 0) {
    r = 0;
  } else if (sh > 38) {  // m 2^sh >= 2^62 (and inf, NaN)
    *bad = 1;
    r = 0;
  } else if (sh >= 0) {
    r = (long long)m << sh;
  } else if (sh >= -24) {
    r = (long long)((m + (1u << (-sh - 1))) >> (-sh));
  } else {
    r = 0;  // below one half
  }
  return (u >> 31) ? -r : r;
}

}  // namespace fm
