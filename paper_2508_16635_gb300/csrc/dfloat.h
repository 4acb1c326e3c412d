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
// split48 is host/device code (a host test checks it): it cuts a double into hi + lo with
// integer operations only (conversions between double and float would run on the FP64
// pipe).
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

#if defined(__CUDACC__)

// A double-float accumulator: the value is s + c.
struct dfl {
  float s, c;
};

__device__ __forceinline__ dfl dfl_zero() { return dfl{0.0f, 0.0f}; }

// a += (xh + xl)(yh + yl), the xl yl term (2^-48 relative) dropped.
__device__ __forceinline__ void dfl_fma(dfl& a, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  const float e = __fmaf_rn(xh, yh, -p);
  const float t = __fadd_rn(a.s, p);
  const float z = __fadd_rn(t, -a.s);
  const float err = __fadd_rn(__fadd_rn(a.s, -__fadd_rn(t, -z)), __fadd_rn(p, -z));
  const float cross = __fmaf_rn(xh, yl, __fmul_rn(xl, yh));
  a.c = __fadd_rn(a.c, __fadd_rn(err, __fadd_rn(e, cross)));
  a.s = t;
}

// a + b
__device__ __forceinline__ dfl dfl_add(dfl a, dfl b) {
  const float t = __fadd_rn(a.s, b.s);
  const float z = __fadd_rn(t, -a.s);
  const float err = __fadd_rn(__fadd_rn(a.s, -__fadd_rn(t, -z)), __fadd_rn(b.s, -z));
  return dfl{t, __fadd_rn(__fadd_rn(a.c, b.c), err)};
}

__device__ __forceinline__ dfl dfl_neg(dfl a) { return dfl{-a.s, -a.c}; }

// (s, c) -> (s', c') with s' = fl(s + c) and s' + c' = s + c exactly (TwoSum: after a
// cancellation |c| may exceed |s|, where the cheaper Fast2Sum would not be exact).  The
// pair then satisfies |c'| <= ulp(s') / 2, which the products of dfl_fma rely on when they
// drop the lo * lo term and round the cross terms.
__device__ __forceinline__ dfl dfl_norm(dfl a) {
  const float t = __fadd_rn(a.s, a.c);
  const float z = __fadd_rn(t, -a.s);
  return dfl{t, __fadd_rn(__fadd_rn(a.s, -__fadd_rn(t, -z)), __fadd_rn(a.c, -z))};
}

__device__ __forceinline__ dfl dfl_shfl_xor(dfl a, int o) {
  return dfl{__shfl_xor_sync(0xffffffffu, a.s, o), __shfl_xor_sync(0xffffffffu, a.c, o)};
}

__device__ __forceinline__ double dfl_to_double(dfl a) { return (double)a.s + (double)a.c; }

__device__ __forceinline__ dfl dfl_from_double(double d) {
  dfl a;
  split48(d, a.s, a.c);
  return a;
}

#endif

}  // namespace rsc
