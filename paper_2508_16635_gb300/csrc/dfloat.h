// Double-float arithmetic: FP64 values carried as unevaluated sums hi + lo of two FP32
// numbers (48 significant bits), for the FP64 stages of the mixed path and the Krylov
// basis.  GB300 issues FP32 at 64 times its FP64 rate, and the error-free transformations
// below need no FP64 instruction:
//   * TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b), e = (a + b) - s exactly;
//   * TwoProd with a fused multiply-add: p = fl(a b), e = fma(a, b, -p) = a b - p exactly;
//   * Dot2 (Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26 (2005), Algorithm 5.3): a sum of
//     products accumulated as (s, c), s the FP32 sum and c the sum of the errors, as if the
//     sum were evaluated in twice the working precision.
// The operations use the _rn intrinsics so that the compiler never contracts a product and
// a sum into one multiply-add (which would break the error-free transformations).
//
// Everything but the warp shuffle is host/device code, checked on the host by
// tests/test_dfloat_split.py; split48 cuts a double into hi + lo with integer operations
// only (conversions between double and float would run on the FP64 pipe).
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define RSC_HD __host__ __device__ __forceinline__
#else
#define RSC_HD inline
#endif

namespace rsc {

// d = hi + lo + err with |err| <= 2^-48 |d| for 2^-74 <= |d| < 2^128.  hi is d truncated to
// 24 significant bits, lo the remaining 29 mantissa bits rounded to 24.  For
// 2^-126 <= |d| < 2^-74 lo is 0 (absolute error below 2^-97); below 2^-126 both are 0;
// from 2^128 on (or for an infinity or NaN) hi is an infinity or NaN of d's sign.
RSC_HD void split48(double d, float& hi, float& lo) {
  uint64_t u;
  memcpy(&u, &d, sizeof u);
  const uint32_t h32 = (uint32_t)(u >> 32), l32 = (uint32_t)u;
  const uint32_t e = (h32 >> 20) & 0x7FFu;
  const uint32_t sgn = h32 & 0x80000000u;
  uint32_t hb = 0;
  float lf = 0.0f;
  if (e >= 897u) {
    if (e <= 1150u) {
      // rebias the exponent (1023 -> 127) and keep the top 23 of the 52 mantissa bits
      hb = sgn | ((e - 896u) << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29);
      if (e >= 949u) {
        // the low 29 bits weigh 2^(e - 1075); that power of two is a normal float here
        const uint32_t sb = (e - 948u) << 23;
        float sc;
        memcpy(&sc, &sb, sizeof sc);
        lf = (float)(l32 & 0x1FFFFFFFu) * sc;
        if (sgn) lf = -lf;
      }
    } else {
      hb = sgn | 0x7F800000u | ((((h32 & 0xFFFFFu) | l32) != 0u && e == 0x7FFu) ? 0x400000u : 0u);
    }
  }
  memcpy(&hi, &hb, sizeof hi);
  lo = lf;
}

// Correctly rounded FP32 operations that the compiler may not contract: the _rn intrinsics
// on the device; on the host (tests) volatile stores, with an ISO C++ mode (no contraction
// across statements) and IEEE single precision.
#if defined(__CUDA_ARCH__)
__device__ __forceinline__ float df_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float df_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float df_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
inline float df_add(float a, float b) { volatile float r = a + b; return r; }
inline float df_mul(float a, float b) { volatile float r = a * b; return r; }
inline float df_fma(float a, float b, float c) { volatile float r = __builtin_fmaf(a, b, c); return r; }
#endif

// A double-float accumulator: the value is s + c.
struct dfl {
  float s, c;
};

RSC_HD dfl dfl_zero() { return dfl{0.0f, 0.0f}; }

// a += (xh + xl)(yh + yl), the xl yl term (2^-48 relative) dropped.
RSC_HD void dfl_fma(dfl& a, float xh, float xl, float yh, float yl) {
  const float p = df_mul(xh, yh);
  const float e = df_fma(xh, yh, -p);
  const float t = df_add(a.s, p);
  const float z = df_add(t, -a.s);
  const float err = df_add(df_add(a.s, -df_add(t, -z)), df_add(p, -z));
  const float cross = df_fma(xh, yl, df_mul(xl, yh));
  a.c = df_add(a.c, df_add(err, df_add(e, cross)));
  a.s = t;
}

// a + b
RSC_HD dfl dfl_add(dfl a, dfl b) {
  const float t = df_add(a.s, b.s);
  const float z = df_add(t, -a.s);
  const float err = df_add(df_add(a.s, -df_add(t, -z)), df_add(b.s, -z));
  return dfl{t, df_add(df_add(a.c, b.c), err)};
}

RSC_HD dfl dfl_neg(dfl a) { return dfl{-a.s, -a.c}; }

// (s, c) -> (s', c') with s' = fl(s + c) and s' + c' = s + c exactly (TwoSum: after a
// cancellation |c| may exceed |s|, where the cheaper Fast2Sum would not be exact).  The
// pair then satisfies |c'| <= ulp(s') / 2, which the products of dfl_fma rely on when they
// drop the lo * lo term and round the cross terms.
RSC_HD dfl dfl_norm(dfl a) {
  const float t = df_add(a.s, a.c);
  const float z = df_add(t, -a.s);
  return dfl{t, df_add(df_add(a.s, -df_add(t, -z)), df_add(a.c, -z))};
}

RSC_HD double dfl_to_double(dfl a) { return (double)a.s + (double)a.c; }

RSC_HD dfl dfl_from_double(double d) {
  dfl a;
  split48(d, a.s, a.c);
  return a;
}

#if defined(__CUDACC__)
__device__ __forceinline__ dfl dfl_shfl_xor(dfl a, int o) {
  return dfl{__shfl_xor_sync(0xffffffffu, a.s, o), __shfl_xor_sync(0xffffffffu, a.c, o)};
}
#endif

}  // namespace rsc
