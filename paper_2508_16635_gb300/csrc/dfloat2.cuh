// Packed double-float arithmetic for the device: two double-float values (s = the FP32
// sums, c = their errors) carried in float2 pairs and updated with GB300's FP32x2
// instructions (__fadd2_rn, __fmul2_rn, __ffma2_rn: two correctly rounded FP32 operations
// per lane per instruction).  Every routine is the scalar routine of dfloat.h applied to
// both components, step for step, so the results are those of the scalar code bit for bit
// in half the instructions.  Used for the (re, im) parts of complex row sums (chain_df.cuh)
// and for pairs of Krylov inner products and updates (krylov_split.cuh).
#pragma once

#include <cuda_runtime.h>

#include "dfloat.h"

namespace rsc {

// Two double-float accumulators: s = (s_0, s_1), c = (c_0, c_1).
struct cdfl {
  float2 s, c;
};

__device__ __forceinline__ float2 f2neg(float2 v) { return make_float2(-v.x, -v.y); }

__device__ __forceinline__ cdfl cdfl_zero() {
  return cdfl{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
}

// a += (xh + xl)(yh + yl) per component (dfl_fma)
__device__ __forceinline__ void cdfl_fma(cdfl& a, float2 xh, float2 xl, float2 yh, float2 yl) {
  const float2 p = __fmul2_rn(xh, yh);
  const float2 e = __ffma2_rn(xh, yh, f2neg(p));
  const float2 t = __fadd2_rn(a.s, p);
  const float2 z = __fadd2_rn(t, f2neg(a.s));
  const float2 err = __fadd2_rn(__fadd2_rn(a.s, f2neg(__fadd2_rn(t, f2neg(z)))), __fadd2_rn(p, f2neg(z)));
  const float2 cross = __ffma2_rn(xh, yl, __fmul2_rn(xl, yh));
  a.c = __fadd2_rn(a.c, __fadd2_rn(err, __fadd2_rn(e, cross)));
  a.s = t;
}

// a + b per component (dfl_add)
__device__ __forceinline__ cdfl cdfl_add(cdfl a, cdfl b) {
  const float2 t = __fadd2_rn(a.s, b.s);
  const float2 z = __fadd2_rn(t, f2neg(a.s));
  const float2 err = __fadd2_rn(__fadd2_rn(a.s, f2neg(__fadd2_rn(t, f2neg(z)))), __fadd2_rn(b.s, f2neg(z)));
  return cdfl{t, __fadd2_rn(__fadd2_rn(a.c, b.c), err)};
}

// normalisation per component (dfl_norm)
__device__ __forceinline__ cdfl cdfl_norm(cdfl a) {
  const float2 t = __fadd2_rn(a.s, a.c);
  const float2 z = __fadd2_rn(t, f2neg(a.s));
  return cdfl{t, __fadd2_rn(__fadd2_rn(a.s, f2neg(__fadd2_rn(t, f2neg(z)))), __fadd2_rn(a.c, f2neg(z)))};
}

__device__ __forceinline__ cdfl cdfl_shfl_xor(cdfl a, int o) {
  return cdfl{make_float2(__shfl_xor_sync(0xffffffffu, a.s.x, o), __shfl_xor_sync(0xffffffffu, a.s.y, o)),
              make_float2(__shfl_xor_sync(0xffffffffu, a.c.x, o), __shfl_xor_sync(0xffffffffu, a.c.y, o))};
}

__device__ __forceinline__ double cdfl_to_double_x(cdfl a) { return (double)a.s.x + (double)a.c.x; }
__device__ __forceinline__ double cdfl_to_double_y(cdfl a) { return (double)a.s.y + (double)a.c.y; }

}  // namespace rsc
