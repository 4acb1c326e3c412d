// The e/f chain solve of the mixed path after one level of odd-even (cyclic) reduction of
// every Coriolis chain (Sec. 3.2, Fig. blocks; HostFactorCR in rsc_internal.h): with D_i the
// diagonal block of block row i and A_i, C_i its couplings to blocks i - 1 and i + 1,
//   odd blocks:   u_i = D_i^-1 b_i,
//   even blocks:  b'_j = b_j - A_j u_{j-1} - C_j u_{j+1},
//   the reduced chain on the even blocks: twisted block Thomas (the sweeps of chain_df.cuh
//   over every second block),
//   odd blocks:   x_i = D_i^-1 (b_i - A_i x_{i-1} - C_i x_{i+1}).
// The couplings are never stored: on the rows between the boundary rows
//   A_i v = (2 a_l / r^2) ((l / r) E0 v - E1 v),   C_i v = (2 c_l / r^2) (-((l + 1) / r) E0 v - E1 v)
// (Eqs. impcor_e_final / impcor_f_final; l the degree of block i, a_l and c_l the
// normalised l -+ 1 coefficients), so a coupling costs two products with the Chebyshev
// tables E0, E1 (d^o T_k / dr^o at the collocation radii, shared by every block and held in
// L2) instead of a factor block read from HBM.  The solve reads the factor blocks D_i^-1
// once for the odd blocks in each direction and G', H', W' once each for the even blocks:
// 2.5 blocks per block pair against 3 for the unreduced chains, and the sequential sweeps
// run over half as many blocks.
//
// Arithmetic as chain_df.cuh: factor blocks and the tables as double-float pairs
// {hi, lo} (float4 per complex entry), row sums as Dot2 sums in FP32, vectors FP64 in
// global memory.  Grid of each kernel: 2 CTAs (e and f block) per pair (m, l) of the given
// parity of l - m, 256 threads, 8 lanes per row (as k_block_gemv_df).
#pragma once

#include "chain_df.cuh"

namespace rsc {

// Coupling factors in double-float pairs, prepared on the host from the collocation radii
// and the normalised coefficients (Eqs. impcor_e_final / impcor_f_final):
//   rowf[j]     = {s ir hi, s ir lo, s hi, s lo},  s = 2 / r_j^2, ir = 1 / r_j;
//   pairf[2 p]  = {a l hi, a l lo, a hi, a lo},    a = a_l of pair p (coupling to l - 1);
//   pairf[2p+1] = {c (l+1) hi, lo, c hi, c lo},     c = c_l (coupling to l + 1),
// so that on the coupled rows
//   A v = (s ir a l) E0 v - (s a) E1 v,   C v = -(s ir c (l + 1)) E0 v - (s c) E1 v.
// Nothing here needs an FP64 instruction (GB300 issues FP64 at 1/64 of the FP32 rate).

// Rows of field fld (0 = e, 1 = f) that carry the coupling (the others are boundary rows).
__device__ __forceinline__ bool cr_coupled_row(int fld, int j, int Nr) {
  return fld == 1 ? (j >= 2 && j <= Nr - 3) : (j >= 1 && j <= Nr - 2);
}

// The block of CTA blockIdx.x: pair p from the parity list, field fld, its index i = l - m
// in its chain c and the chain length nb.
struct CrBlock {
  int p, fld, m, l, i, c, nb;
  long row0;
};

__device__ __forceinline__ CrBlock cr_block(const DevGeom& g, const int* __restrict__ pairs) {
  CrBlock b;
  b.p = pairs[blockIdx.x >> 1];
  b.fld = blockIdx.x & 1;
  b.m = g.pair_m[b.p];
  b.l = g.pair_l[b.p];
  b.i = b.l - b.m;
  const int cls = (b.fld == 0) ? (b.i & 1) : 1 - (b.i & 1);
  b.c = 2 * (b.m / g.Ms) + cls;
  b.nb = g.L - b.m + 1;
  b.row0 = ((long)b.fld * g.P + b.p) * g.Nr;
  return b;
}

// Normalised complex double-float (re, im) as a float4 {re_hi, im_hi, re_lo, im_lo}.
__device__ __forceinline__ float4 cd_pack(dfl re, dfl im) {
  const dfl a = dfl_norm(re), b = dfl_norm(im);
  return make_float4(a.s, b.s, a.c, b.c);
}

// The product of two real double-float factors {hi, lo}, normalised.
__device__ __forceinline__ dfl cr_mul(float ah, float al, float bh, float bl) {
  dfl p = dfl_zero();
  dfl_fma(p, ah, al, bh, bl);
  return dfl_norm(p);
}

// (re, im) += k v for a real double-float factor k and a complex double-float v.
__device__ __forceinline__ void cr_axpy(dfl& re, dfl& im, dfl k, float4 v) {
  dfl_fma(re, k.s, k.c, v.x, v.z);
  dfl_fma(im, k.s, k.c, v.y, v.w);
}

// y = M v for one Nr x Nr double-float block M (row-major), v in shared memory; row r of y
// goes to y[r] (shared memory, packed).  All 256 threads take part; the caller syncs.
template <int Q>
__device__ __forceinline__ void cr_gemv(const float4* __restrict__ M, const float4* v, int Nr,
                                        bool real_op, float4* y) {
  const int s8 = threadIdx.x & 7;
  const int rows_per_pass = blockDim.x >> 3;
  for (int r = threadIdx.x >> 3; r < Nr + ((rows_per_pass - Nr % rows_per_pass) % rows_per_pass);
       r += rows_per_pass) {
    float4 a[Q];
    cd_load<Q>(M, r, s8, 0, Nr, r < Nr, a);
    dfl re0 = dfl_zero(), im0 = dfl_zero(), re1 = dfl_zero(), im1 = dfl_zero();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k = s8 + 8 * q;
      if (k < Nr) {
        if (q & 1)
          cd_cmac(re1, im1, a[q], v[k], real_op);
        else
          cd_cmac(re0, im0, a[q], v[k], real_op);
      }
    }
    dfl re = dfl_add(re0, re1), im = dfl_add(im0, im1);
    cd_reduce8(re, im);
    if (r < Nr && s8 == 0) y[r] = cd_pack(re, im);
  }
}

// (E0 v0)_j and (E1 v1)_j for every row j (E01[j][k] = {E0 hi, E0 lo, E1 hi, E1 lo}, real),
// v0, v1 complex double-float in shared memory, packed into e0[j], e1[j] (shared or global).
template <int Q>
__device__ __forceinline__ void cr_e01(const float4* __restrict__ E01, const float4* v0,
                                       const float4* v1, int Nr, float4* e0, float4* e1) {
  const int s8 = threadIdx.x & 7;
  const int rows_per_pass = blockDim.x >> 3;
  for (int j = threadIdx.x >> 3; j < Nr + ((rows_per_pass - Nr % rows_per_pass) % rows_per_pass);
       j += rows_per_pass) {
    float4 e[Q];
    cd_load<Q>(E01, j, s8, 0, Nr, j < Nr, e);
    dfl a = dfl_zero(), b = dfl_zero(), c = dfl_zero(), d = dfl_zero();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k = s8 + 8 * q;
      if (k < Nr) {
        const float4 x = v0[k], y = v1[k];
        dfl_fma(a, e[q].x, e[q].y, x.x, x.z);
        dfl_fma(b, e[q].x, e[q].y, x.y, x.w);
        dfl_fma(c, e[q].z, e[q].w, y.x, y.z);
        dfl_fma(d, e[q].z, e[q].w, y.y, y.w);
      }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      a = dfl_add(a, dfl_shfl_xor(a, o));
      b = dfl_add(b, dfl_shfl_xor(b, o));
      c = dfl_add(c, dfl_shfl_xor(c, o));
      d = dfl_add(d, dfl_shfl_xor(d, o));
    }
    if (j < Nr && s8 == 0) {
      e0[j] = cd_pack(a, b);
      e1[j] = cd_pack(c, d);
    }
  }
}

// out[row0 + k] = y[k] joined to FP64, one row per thread (full warps: each FP64 warp
// instruction costs the same whatever the number of active lanes).
__device__ __forceinline__ void cr_store(const float4* y, double2* __restrict__ out, long row0,
                                         int Nr) {
  for (int k = threadIdx.x; k < Nr; k += blockDim.x) out[row0 + k] = cd_join(y[k]);
}

// Odd blocks, first pass: u = D^-1 b, then w0 = E0 u and w1 = E1 u at the block's own rows
// (w: [2][2 P Nr] float4), for the even neighbours' right-hand sides.
// Dynamic shared memory: 2 Nr float4.
template <int Q>
__global__ void __launch_bounds__(256) k_cr_odd_df(DevGeom g, const int* __restrict__ odd_pairs,
                                                   const long* __restrict__ odd_off,
                                                   const float4* __restrict__ Dinv,
                                                   const float4* __restrict__ E01,
                                                   const double2* __restrict__ rhs,
                                                   float4* __restrict__ w) {
  extern __shared__ float4 cr_sh[];
  const int Nr = g.Nr;
  const CrBlock b = cr_block(g, odd_pairs);
  float4* sb = cr_sh;
  float4* su = cr_sh + Nr;
  for (int k = threadIdx.x; k < Nr; k += blockDim.x) sb[k] = cd_split(rhs[b.row0 + k]);
  __syncthreads();
  const float4* Di = Dinv + (odd_off[b.c] + (b.i >> 1)) * (long)Nr * Nr;
  cr_gemv<Q>(Di, sb, Nr, b.m == 0, su);
  __syncthreads();
  cr_e01<Q>(E01, su, su, Nr, w + b.row0, w + 2L * g.P * Nr + b.row0);
}

// Even blocks: b' = b - A u_{i-1} - C u_{i+1} from the neighbours' w, then g' = G' b' into
// out.  Dynamic shared memory: 2 Nr float4.
template <int Q>
__global__ void __launch_bounds__(256) k_cr_even_df(DevGeom g, const int* __restrict__ even_pairs,
                                                    const long* __restrict__ red_off,
                                                    const float4* __restrict__ Gr,
                                                    const float4* __restrict__ rowf,
                                                    const float4* __restrict__ pairf,
                                                    const double2* __restrict__ rhs,
                                                    const float4* __restrict__ w,
                                                    double2* __restrict__ out) {
  extern __shared__ float4 cr_sh[];
  const int Nr = g.Nr;
  const CrBlock b = cr_block(g, even_pairs);
  float4* sb = cr_sh;
  float4* sy = cr_sh + Nr;
  const long half = 2L * g.P * Nr;
  const bool left = b.i >= 1, right = b.i + 1 <= b.nb - 1;
  const long rowL = ((long)(1 - b.fld) * g.P + b.p - 1) * Nr;
  const long rowR = ((long)(1 - b.fld) * g.P + b.p + 1) * Nr;
  const float4 pa = pairf[2 * b.p], pc = pairf[2 * b.p + 1];
  for (int j = threadIdx.x; j < Nr; j += blockDim.x) {
    const double2 bv = rhs[b.row0 + j];
    dfl re = dfl_from_double(bv.x), im = dfl_from_double(bv.y);
    if (cr_coupled_row(b.fld, j, Nr) && b.l > 0) {
      const float4 rf = rowf[j];
      if (left) {   // - A u_{i-1} = -(s ir a l) E0 u + (s a) E1 u
        const dfl k0 = cr_mul(rf.x, rf.y, pa.x, pa.y), k1 = cr_mul(rf.z, rf.w, pa.z, pa.w);
        cr_axpy(re, im, dfl_neg(k0), w[rowL + j]);
        cr_axpy(re, im, k1, w[half + rowL + j]);
      }
      if (right) {  // - C u_{i+1} = (s ir c (l+1)) E0 u + (s c) E1 u
        const dfl k0 = cr_mul(rf.x, rf.y, pc.x, pc.y), k1 = cr_mul(rf.z, rf.w, pc.z, pc.w);
        cr_axpy(re, im, k0, w[rowR + j]);
        cr_axpy(re, im, k1, w[half + rowR + j]);
      }
    }
    sb[j] = cd_pack(re, im);
  }
  __syncthreads();
  const float4* Gt = Gr + (red_off[b.c] + (b.i >> 1)) * (long)Nr * Nr;
  cr_gemv<Q>(Gt, sb, Nr, b.m == 0, sy);
  __syncthreads();
  cr_store(sy, out, b.row0, Nr);
}

// Odd blocks, last pass: x_i = D^-1 (b - A x_{i-1} - C x_{i+1}) with the even neighbours'
// solution in out.  The two couplings share the row factor s = 2 / r^2, so
//   A x_{i-1} + C x_{i+1} = s ir E0 y0 - s E1 y1,
//   y0 = a l x_{i-1} - c (l + 1) x_{i+1},   y1 = a x_{i-1} + c x_{i+1}:
// two table products per block.  Dynamic shared memory: 5 Nr float4.
template <int Q>
__global__ void __launch_bounds__(256) k_cr_back_df(DevGeom g, const int* __restrict__ odd_pairs,
                                                    const long* __restrict__ odd_off,
                                                    const float4* __restrict__ Dinv,
                                                    const float4* __restrict__ E01,
                                                    const float4* __restrict__ rowf,
                                                    const float4* __restrict__ pairf,
                                                    const double2* __restrict__ rhs,
                                                    double2* __restrict__ out) {
  extern __shared__ float4 cr_sh[];
  const int Nr = g.Nr;
  const CrBlock b = cr_block(g, odd_pairs);
  float4* y0 = cr_sh;
  float4* y1 = cr_sh + Nr;
  float4* e0 = cr_sh + 2 * Nr;
  float4* e1 = cr_sh + 3 * Nr;
  float4* sr = cr_sh + 4 * Nr;
  const bool right = b.i + 1 <= b.nb - 1;
  const long rowL = ((long)(1 - b.fld) * g.P + b.p - 1) * Nr;
  const long rowR = ((long)(1 - b.fld) * g.P + b.p + 1) * Nr;
  const float4 pa = pairf[2 * b.p], pc = pairf[2 * b.p + 1];
  for (int k = threadIdx.x; k < Nr; k += blockDim.x) {
    const float4 xl = cd_split(out[rowL + k]);
    dfl r0 = dfl_zero(), i0 = dfl_zero(), r1 = dfl_zero(), i1 = dfl_zero();
    cr_axpy(r0, i0, dfl{pa.x, pa.y}, xl);
    cr_axpy(r1, i1, dfl{pa.z, pa.w}, xl);
    if (right) {
      const float4 xr = cd_split(out[rowR + k]);
      cr_axpy(r0, i0, dfl{-pc.x, -pc.y}, xr);
      cr_axpy(r1, i1, dfl{pc.z, pc.w}, xr);
    }
    y0[k] = cd_pack(r0, i0);
    y1[k] = cd_pack(r1, i1);
  }
  __syncthreads();
  cr_e01<Q>(E01, y0, y1, Nr, e0, e1);
  __syncthreads();
  for (int j = threadIdx.x; j < Nr; j += blockDim.x) {
    const double2 bv = rhs[b.row0 + j];
    dfl re = dfl_from_double(bv.x), im = dfl_from_double(bv.y);
    if (cr_coupled_row(b.fld, j, Nr)) {   // - s ir E0 y0 + s E1 y1
      const float4 rf = rowf[j];
      cr_axpy(re, im, dfl{-rf.x, -rf.y}, e0[j]);
      cr_axpy(re, im, dfl{rf.z, rf.w}, e1[j]);
    }
    sr[j] = cd_pack(re, im);
  }
  __syncthreads();
  const float4* Di = Dinv + (odd_off[b.c] + (b.i >> 1)) * (long)Nr * Nr;
  cr_gemv<Q>(Di, sr, Nr, b.m == 0, y0);
  __syncthreads();
  cr_store(y0, out, b.row0, Nr);
}

}  // namespace rsc
