// Orthogonalisation against a Krylov basis held in double-float form: beside the FP64
// basis V (the Jacobian actions read and write FP64 vectors), Vs_j[i] = (hi, lo) of V_j[i]
// (split48, 48 significant bits) with the same column stride, and the one-reduction MGS
// passes and the final update run Dot2 sums in FP32 (dfloat.h).  Per basis element they
// issue about a dozen FP32 instructions instead of one or two FP64 multiply-adds, which
// GB300 issues at 1/64 of its FP32 rate; the loads stay 8 bytes per element, so the passes
// become bound by HBM instead of by the FP64 pipe.  Every FP64 instruction left is per
// vector element (the final subtraction, |w|^2), not per basis element.
//
// Accuracy: each product carries a relative error of about 2^-48 (the dropped lo*lo term
// and the split), and Dot2 sums as if in twice FP32 precision, so the inner products and
// updates agree with FP64 to about 1e-14 of the magnitudes involved -- far below the
// 1e-10 GMRES and Newton tolerances.
//
// Alignment: columns padded to ld (a multiple of 1024 elements), n even, so every element
// pair is one float4 / double2.
#pragma once

#include "dfloat.h"

namespace rsc {

// Warm L2 with the line of p (a hint: no register, no wait; p must lie inside the basis).
__device__ __forceinline__ void ks_prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// out = s * in and outs = split48(out).  With part given, |in|^2 = the sum of part[0, np)
// (the blocks' shares of k_axpy_norm_s), summed by every block in the same order (threads
// strided, then the warp and block trees), written to nrm2_out[0] by block 0, and
// s = 1 / sqrt(|in|^2) (1 when |in|^2 <= 0, a breakdown the host detects); else s is the
// argument.  One thread per block evaluates the FP64 square root and division.  in may
// equal out.  block = 256.
__global__ void __launch_bounds__(256) k_scale_split(const double* in, double* out,
                                                     float2* __restrict__ outs, long n,
                                                     const double* __restrict__ part, int np,
                                                     double* __restrict__ nrm2_out, double s) {
  if (part) {
    __shared__ double red[8];
    __shared__ double sc;
    double t = 0.0;
    for (int b = threadIdx.x; b < np; b += blockDim.x) t += part[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
      t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (threadIdx.x == 0) {
        sc = (t > 0.0) ? 1.0 / sqrt(t) : 1.0;
        if (blockIdx.x == 0) nrm2_out[0] = t;
      }
    }
    __syncthreads();
    s = sc;
  }
  const long n2 = n >> 1;
  const double2* in2 = reinterpret_cast<const double2*>(in);
  double2* out2 = reinterpret_cast<double2*>(out);
  float4* outs4 = reinterpret_cast<float4*>(outs);
  for (long i2 = (long)blockIdx.x * blockDim.x + threadIdx.x; i2 < n2;
       i2 += (long)gridDim.x * blockDim.x) {
    double2 v = in2[i2];
    v.x *= s;
    v.y *= s;
    out2[i2] = v;
    float4 q;
    split48(v.x, q.x, q.y);
    split48(v.y, q.z, q.w);
    outs4[i2] = q;
  }
}

// First MGS pass on the split basis: partial[j * nchunk + c] = Vs_j . w and
// partial[(nv + j) * nchunk + c] = Vs_j . q over chunk c (1024 elements).  w is FP64 (the
// fresh Jacobian action, split while staging), q = Vs_k already split.
// grid = (ld / 1024, ceil(nv / 16)), block = 512: warp u streams vector 16 g + u over the
// chunk, its 16 float4 loads per lane issued together (one vector per warp, so no warp waits
// out the load latency twice).
__global__ void __launch_bounds__(512) k_dots_pair_s(const float2* __restrict__ Vs, long ld,
                                                     int nv, const double* __restrict__ w,
                                                     const float2* __restrict__ qs,
                                                     double* __restrict__ partial) {
  constexpr int E2 = 512, PER = E2 / 32;
  __shared__ float4 ws[E2], qsh[E2];
  const long b2 = (long)blockIdx.x * E2;
  const double2* w2 = reinterpret_cast<const double2*>(w) + b2;
  const float4* q4 = reinterpret_cast<const float4*>(qs) + b2;
  for (int i = threadIdx.x; i < E2; i += blockDim.x) {
    const double2 x = w2[i];
    float4 a;
    split48(x.x, a.x, a.y);
    split48(x.y, a.z, a.w);
    ws[i] = a;
    qsh[i] = q4[i];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunk = gridDim.x;
  const int j = blockIdx.y * 16 + warp;
  if (j >= nv) return;
  const float4* v4 = reinterpret_cast<const float4*>(Vs + (long)j * ld) + b2 + lane;
  float4 vv[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) vv[u] = __ldcs(v4 + u * 32);
  dfl a0 = dfl_zero(), a1 = dfl_zero(), b0 = dfl_zero(), b1 = dfl_zero();
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const float4 x = ws[u * 32 + lane], y = qsh[u * 32 + lane];
    dfl_fma(a0, vv[u].x, vv[u].y, x.x, x.y);
    dfl_fma(a1, vv[u].z, vv[u].w, x.z, x.w);
    dfl_fma(b0, vv[u].x, vv[u].y, y.x, y.y);
    dfl_fma(b1, vv[u].z, vv[u].w, y.z, y.w);
  }
  dfl a = dfl_add(a0, a1), b = dfl_add(b0, b1);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = dfl_add(a, dfl_shfl_xor(a, o));
    b = dfl_add(b, dfl_shfl_xor(b, o));
  }
  if (lane == 0) {
    partial[(long)j * nchunk + blockIdx.x] = dfl_to_double(a);
    partial[(long)(nv + j) * nchunk + blockIdx.x] = dfl_to_double(b);
  }
}

// Second MGS pass on the split basis: w <- w - sum_j h[j] Vs_j (h split into shared memory,
// dynamic size nv float2), partial[b] = block b's share of |w_new|^2 (FP64).
// grid = nb (grid-stride over element pairs), block = 256.
__global__ void __launch_bounds__(256) k_axpy_norm_s(const float2* __restrict__ Vs, long ld,
                                                     int nv, const double* __restrict__ h,
                                                     double* __restrict__ w, long n,
                                                     double* __restrict__ partial) {
  extern __shared__ float2 hs[];
  __shared__ double red[8];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    float a, b;
    split48(h[j], a, b);
    hs[j] = make_float2(a, b);
  }
  __syncthreads();
  const long n2 = n >> 1;
  double2* w2 = reinterpret_cast<double2*>(w);
  double ss = 0.0;
  for (long i2 = (long)blockIdx.x * blockDim.x + threadIdx.x; i2 < n2;
       i2 += (long)gridDim.x * blockDim.x) {
    dfl sx = dfl_zero(), sy = dfl_zero(), tx = dfl_zero(), ty = dfl_zero();
    int j = 0;
    for (; j + 8 <= nv; j += 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = reinterpret_cast<const float4*>(Vs + (long)(j + u) * ld)[i2];
      // the next group's lines, while this group is summed
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j + 8 + u < nv) ks_prefetch_l2(reinterpret_cast<const float4*>(Vs + (long)(j + 8 + u) * ld) + i2);
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        const float2 c0 = hs[j + u], c1 = hs[j + u + 1];
        dfl_fma(sx, c0.x, c0.y, v[u].x, v[u].y);
        dfl_fma(sy, c0.x, c0.y, v[u].z, v[u].w);
        dfl_fma(tx, c1.x, c1.y, v[u + 1].x, v[u + 1].y);
        dfl_fma(ty, c1.x, c1.y, v[u + 1].z, v[u + 1].w);
      }
    }
    for (; j < nv; ++j) {
      const float4 v = reinterpret_cast<const float4*>(Vs + (long)j * ld)[i2];
      const float2 c = hs[j];
      dfl_fma(sx, c.x, c.y, v.x, v.y);
      dfl_fma(sy, c.x, c.y, v.z, v.w);
    }
    double2 o = w2[i2];
    o.x -= dfl_to_double(dfl_add(sx, tx));
    o.y -= dfl_to_double(dfl_add(sy, ty));
    w2[i2] = o;
    ss = fma(o.x, o.x, fma(o.y, o.y, ss));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int r = 0; r < (int)(blockDim.x >> 5); ++r) a += red[r];
    partial[blockIdx.x] = a;
  }
}

// x += sum_j coef[j] Vs_j (the GMRES update), coef split into shared memory (dynamic, nv
// float2).  grid-stride over element pairs, block = 256.
__global__ void __launch_bounds__(256) k_multi_axpy_s(const float2* __restrict__ Vs, long ld,
                                                      int nv, const double* __restrict__ coef,
                                                      double* __restrict__ x, long n) {
  extern __shared__ float2 cs[];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    float a, b;
    split48(coef[j], a, b);
    cs[j] = make_float2(a, b);
  }
  __syncthreads();
  const long n2 = n >> 1;
  double2* x2 = reinterpret_cast<double2*>(x);
  for (long i2 = (long)blockIdx.x * blockDim.x + threadIdx.x; i2 < n2;
       i2 += (long)gridDim.x * blockDim.x) {
    dfl sx = dfl_zero(), sy = dfl_zero(), tx = dfl_zero(), ty = dfl_zero();
    int j = 0;
    for (; j + 8 <= nv; j += 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = reinterpret_cast<const float4*>(Vs + (long)(j + u) * ld)[i2];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        const float2 c0 = cs[j + u], c1 = cs[j + u + 1];
        dfl_fma(sx, c0.x, c0.y, v[u].x, v[u].y);
        dfl_fma(sy, c0.x, c0.y, v[u].z, v[u].w);
        dfl_fma(tx, c1.x, c1.y, v[u + 1].x, v[u + 1].y);
        dfl_fma(ty, c1.x, c1.y, v[u + 1].z, v[u + 1].w);
      }
    }
    for (; j < nv; ++j) {
      const float4 v = reinterpret_cast<const float4*>(Vs + (long)j * ld)[i2];
      const float2 c = cs[j];
      dfl_fma(sx, c.x, c.y, v.x, v.y);
      dfl_fma(sy, c.x, c.y, v.z, v.w);
    }
    double2 o = x2[i2];
    o.x += dfl_to_double(dfl_add(sx, tx));
    o.y += dfl_to_double(dfl_add(sy, ty));
    x2[i2] = o;
  }
}

}  // namespace rsc
