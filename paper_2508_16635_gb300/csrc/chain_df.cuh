// The chain solve of the implicit Coriolis operator (Sec. 3.2) in double-float arithmetic,
// for the Jacobian actions and steps of the mixed path: g = G b per block, then the
// twisted block-Thomas sweeps y_i = g_i - H_i y_(i-+1) and x_i = y_i - W_i x_(i+-1), exactly as
// the FP64 kernels (k_block_gemv, chain_async.cuh) but with the factor blocks stored as
// float4 {re_hi, im_hi, re_lo, im_lo} (each FP64 entry rounded to hi, the remainder rounded
// to lo; prepared on the host with the factorisation) and every row sum a Dot2 sum in FP32
// (dfloat.h).  Vectors stay FP64 in global memory between kernels (split on load with
// integer operations, joined on store), and travel between the CTAs of a cluster as
// float4 in the same format.
//
// Why: these sweeps are sequential in l, and on GB300 their FP64 multiply-adds run at 1/64
// of the FP32 rate with a 66-cycle dependent latency.  Double-float needs about 12 FP32
// instructions per real product (4-cycle latency) and no FP64 instruction per block entry.
// Accuracy: on the L = 127, N_r = 64, Ek = 1e-5 chains at dt = 200 (block norms up to
// 4e4) an exact float32 emulation of these sweeps stays within 1e-11 of FP64 sweeps over
// the same tables; the solve amplifies the 2^-48 perturbation of the tables by its
// conditioning, and a Jacobian action moves by about 1e-7 of its e/f part -- below the
// FP32 transform error of a mixed Jacobian action (about 2e-5).  A plain FP32 solve is not
// enough: it errs by 1e-4 to 5e-2 on the same chains.
//
// Bounded waits and the closing cluster barrier follow chain_async.cuh.
#pragma once

#include "dfloat.h"

namespace rsc {

__device__ __forceinline__ float4 cd_split(double2 v) {
  float4 q;
  split48(v.x, q.x, q.z);
  split48(v.y, q.y, q.w);
  return q;
}

__device__ __forceinline__ double2 cd_join(float4 q) {
  return make_double2((double)q.x + (double)q.z, (double)q.y + (double)q.w);
}

// acc (re, im) += a b for complex double-float a, b (a real when real_op: im parts of the
// table are zero at m = 0 and skipped).
__device__ __forceinline__ void cd_cmac(dfl& re, dfl& im, float4 a, float4 b, bool real_op) {
  dfl_fma(re, a.x, a.z, b.x, b.z);
  dfl_fma(im, a.x, a.z, b.y, b.w);
  if (!real_op) {
    dfl_fma(re, -a.y, -a.w, b.y, b.w);
    dfl_fma(im, a.y, a.w, b.x, b.z);
  }
}

// Reduction of a row sum over the 8 lanes that share the row.
__device__ __forceinline__ void cd_reduce8(dfl& re, dfl& im) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    re = dfl_add(re, dfl_shfl_xor(re, o));
    im = dfl_add(im, dfl_shfl_xor(im, o));
  }
}

__device__ __forceinline__ void cd_send(uint32_t raddr, uint32_t rbar, float4 v) {
  asm volatile(
      "st.async.weak.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::
          "r"(raddr),
      "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
      "r"(__float_as_uint(v.w)), "r"(rbar)
      : "memory");
}

// One lane's share of a row sum over the columns s + 8 q, q in [q0, q0 + QH), reduced over
// the 8 lanes of the row.
template <int QH>
__device__ __forceinline__ void cd_dot(const float4 (&reg)[QH], const float4* v, int s, int q0,
                                       int Nr, bool real_op, dfl& re, dfl& im) {
  dfl r0 = dfl_zero(), i0 = dfl_zero(), r1 = dfl_zero(), i1 = dfl_zero();
#pragma unroll
  for (int q = 0; q < QH; ++q) {
    const int k = s + 8 * (q0 + q);
    if (k < Nr) {
      if (q & 1)
        cd_cmac(r1, i1, reg[q], v[k], real_op);
      else
        cd_cmac(r0, i0, reg[q], v[k], real_op);
    }
  }
  re = dfl_add(r0, r1);
  im = dfl_add(i0, i1);
  cd_reduce8(re, im);
}

template <int QH>
__device__ __forceinline__ void cd_load(const float4* __restrict__ M, int r, int s, int q0, int Nr,
                                        bool active, float4 (&reg)[QH]) {
#pragma unroll
  for (int q = 0; q < QH; ++q) {
    const int k = s + 8 * (q0 + q);
    reg[q] = (active && k < Nr) ? M[(long)r * Nr + k] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// g = G b per diagonal block; the layout and grid of k_block_gemv (grid = 2 P,
// block = 256, 8 lanes per row, Q >= ceil(Nr / 8) columns per lane, all loaded before the
// Dot2 steps).  Dynamic shared memory: Nr float4.
template <int Q>
__global__ void __launch_bounds__(256) k_block_gemv_df(DevGeom g, const long* __restrict__ chain_off,
                                                       const float4* __restrict__ G,
                                                       const double2* __restrict__ rhs,
                                                       double2* __restrict__ out) {
  extern __shared__ float4 svf[];
  const int Nr = g.Nr, P = g.P;
  const int p = blockIdx.x >> 1, fld = blockIdx.x & 1;
  const int m = g.pair_m[p], a = m / g.Ms, i = g.pair_l[p] - m;
  const int cls = (fld == 0) ? (i & 1) : 1 - (i & 1);
  const float4* Gi = G + (chain_off[2 * a + cls] + i) * (long)Nr * Nr;
  const long row0 = ((long)fld * P + p) * Nr;
  for (int k = threadIdx.x; k < Nr; k += blockDim.x) svf[k] = cd_split(rhs[row0 + k]);
  __syncthreads();
  const int s8 = threadIdx.x & 7;
  const int rows_per_pass = blockDim.x >> 3;
  const bool real_op = (m == 0);
  for (int r = threadIdx.x >> 3; r < Nr + ((rows_per_pass - Nr % rows_per_pass) % rows_per_pass);
       r += rows_per_pass) {
    float4 a[Q];
    cd_load<Q>(Gi, r, s8, 0, Nr, r < Nr, a);
    dfl re0 = dfl_zero(), im0 = dfl_zero(), re1 = dfl_zero(), im1 = dfl_zero();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k = s8 + 8 * q;
      if (k < Nr) {
        if (q & 1)
          cd_cmac(re1, im1, a[q], svf[k], real_op);
        else
          cd_cmac(re0, im0, a[q], svf[k], real_op);
      }
    }
    dfl re = dfl_add(re0, re1), im = dfl_add(im0, im1);
    cd_reduce8(re, im);
    if (r < Nr && s8 == 0) out[row0 + r] = make_double2(dfl_to_double(re), dfl_to_double(im));
  }
}

// Row sum of this lane's row over all NS column parts (the h = 0 warp gathers the others'
// partial sums from shared memory).
template <int NS>
__device__ __forceinline__ void cd_gather(const float4* part, int RPC, int lr, dfl& re, dfl& im) {
#pragma unroll
  for (int q = 1; q < NS; ++q) {
    const float4 p = part[(q - 1) * RPC + lr];
    re = dfl_add(re, dfl{p.x, p.z});
    im = dfl_add(im, dfl{p.y, p.w});
  }
}

// v - (re, im) as a normalised complex double-float
__device__ __forceinline__ float4 cd_sub(double2 v, dfl re, dfl im) {
  const dfl a = dfl_norm(dfl_add(dfl_from_double(v.x), dfl_neg(re)));
  const dfl b = dfl_norm(dfl_add(dfl_from_double(v.y), dfl_neg(im)));
  return make_float4(a.s, b.s, a.c, b.c);
}

// Geometry of part c of a partitioned chain (cluster pair blockIdx.x / CS / 2), from the
// part table [p0, cls, nb, boff, m, chain] per part: the sweeps treat a part as a chain.
__device__ __forceinline__ ChainInfo chain_info_part(const DevGeom& g, const long* __restrict__ parts,
                                                     int CS) {
  ChainInfo ci;
  const int cl = blockIdx.x / CS;
  ci.c = cl >> 1;
  ci.dir = cl & 1;
  const long* q = parts + (long)ci.c * 6;
  ci.p0 = (int)q[0];
  ci.cls = (int)q[1];
  ci.nb = (int)q[2];
  ci.boff = q[3];
  ci.m = (int)q[4];
  ci.bs = 1;
  ci.km = (ci.nb - 1) / 2;
  ci.P = g.P;
  ci.Nr = g.Nr;
  ci.blk = (long)g.Nr * g.Nr;
  return ci;
}

// Blocks prefetched ahead of the one being swept (a shift register of PD x QH float4 per
// lane).  One is enough: deeper prefetch (4 blocks) measured slower on GB300 (28.9 -> 30.8
// ms per Newton iteration at L = 127, N_r = 64, and fewer co-resident CTAs), so a block
// step is bound by the cluster exchange, not by the HBM round trip of its rows.
template <int QH>
struct CdDepth {
  static constexpr int PD = 1;
};

// Shared memory: v[2][Nr], part[NS-1][RPC], hist[steps][RPC] (float4), two mbarriers: the
// byte layout of k_chain_half_async.  grid = 2 * 2 * nm * CS (clusters of CS),
// block = 32 NS ceil(RPC / 4).  bs = 2 sweeps the reduced chains of chain_cr.cuh (chain_off
// their first blocks in H), 1 the full chains.
template <int QH, int NS>
__global__ void k_chain_half_df(DevGeom g, const long* __restrict__ chain_off,
                                const float4* __restrict__ H, double2* __restrict__ out,
                                double2* __restrict__ mid, int CS, int steps_cap,
                                int* __restrict__ status, const long* __restrict__ parts,
                                int bs) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ float4 cd_sh[];
  const ChainInfo ci = parts ? chain_info_part(g, parts, CS) : chain_info(g, chain_off, CS, bs);
  const int Nr = ci.Nr;
  const CaLane c = ca_lane<QH, NS>(Nr, CS, (int)cluster.block_rank());
  float4* v = cd_sh;                        // [2][Nr]
  float4* part = v + 2 * Nr;                // [NS - 1][RPC]
  float4* hist = part + (NS - 1) * c.RPC;   // [steps_cap][RPC]
  uint64_t* bar = reinterpret_cast<uint64_t*>(hist + (long)steps_cap * c.RPC);
  const uint32_t bar0 = ca_smem(&bar[0]);
  const bool has = ci.dir == 0 ? (ci.km >= 1) : (ci.km <= ci.nb - 2);
  const int first = ci.dir == 0 ? 0 : ci.nb - 1;
  const int step = ci.dir == 0 ? 1 : -1;
  const int count = ci.dir == 0 ? ci.km - 1 : ci.nb - 2 - ci.km;
  const bool real_op = ci.m == 0;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = threadIdx.x; k < Nr; k += blockDim.x)
    v[k] = has ? cd_split(out[ci.row(first) + k]) : make_float4(0.f, 0.f, 0.f, 0.f);
  constexpr int PD = CdDepth<QH>::PD;
  float4 mc[QH], mb[PD][QH];   // mb[q]: rows of block t + q (t the next step)
  double2 gb[PD];
#pragma unroll
  for (int q = 0; q < PD; ++q) {
    gb[q] = make_double2(0, 0);
    if (q + 1 <= count) {
      cd_load<QH>(H + (ci.boff + first + (q + 1) * step) * ci.blk, c.r, c.s, c.q0, Nr, c.active, mb[q]);
      if (c.active) gb[q] = out[ci.row(first + (q + 1) * step) + c.r];
    }
  }
  cluster.sync();   // barriers initialised and v[0] loaded everywhere before any st.async
  bool ok = true;
  for (int t = 1; t <= count; ++t) {
    const int b = t & 1;
    if (threadIdx.x == 0) ca_expect(bar0 + 8 * b, (uint32_t)Nr * 16u);
#pragma unroll
    for (int q = 0; q < QH; ++q) mc[q] = mb[0][q];
    const double2 gc = gb[0];
#pragma unroll
    for (int d = 0; d + 1 < PD; ++d) {
#pragma unroll
      for (int q = 0; q < QH; ++q) mb[d][q] = mb[d + 1][q];
      gb[d] = gb[d + 1];
    }
    if (t + PD <= count) {
      const int ip = first + (t + PD) * step;
      cd_load<QH>(H + (ci.boff + ip) * ci.blk, c.r, c.s, c.q0, Nr, c.active, mb[PD - 1]);
      if (c.active) gb[PD - 1] = out[ci.row(ip) + c.r];
    }
    dfl re, im;
    cd_dot<QH>(mc, v + (b ^ 1) * Nr, c.s, c.q0, Nr, real_op, re, im);
    if (c.h > 0 && c.s == 0 && c.active)
      part[(c.h - 1) * c.RPC + c.lr] = make_float4(re.s, im.s, re.c, im.c);
    __syncthreads();
    if (c.h == 0 && c.active) {
      cd_gather<NS>(part, c.RPC, c.lr, re, im);
      const float4 y = cd_sub(gc, re, im);
      if (c.s == 0) hist[(t - 1) * c.RPC + c.lr] = y;
      const uint32_t la = ca_smem(v + b * Nr + c.r);
      for (int dst = c.s; dst < CS; dst += 8)
        cd_send(ca_mapa(la, (uint32_t)dst), ca_mapa(bar0 + 8 * b, (uint32_t)dst), y);
    }
    if (!ca_wait(bar0 + 8 * b, (uint32_t)(((t - 1) >> 1) & 1))) ok = false;
  }
  if (!ok && status) atomicExch(status, 7);
  for (int idx = threadIdx.x; idx < count * c.RPC; idx += blockDim.x) {
    const int t = idx / c.RPC + 1, r = c.rank * c.RPC + idx % c.RPC;
    if (r < Nr) out[ci.row(first + t * step) + r] = cd_join(hist[idx]);
  }
  if (c.rank == 0) {
    const float4* last = v + ((count > 0 ? count : 0) & 1) * Nr;
    double2* dst = mid + ((long)ci.c * 3 + ci.dir) * Nr;
    for (int k = threadIdx.x; k < Nr; k += blockDim.x)
      dst[k] = has ? cd_join(last[k]) : make_double2(0, 0);
    if (ci.dir == 0) {
      double2* gm = mid + ((long)ci.c * 3 + 2) * Nr;
      for (int k = threadIdx.x; k < Nr; k += blockDim.x) gm[k] = out[ci.row(ci.km) + k];
    }
  }
  cluster.sync();   // no CTA leaves while a peer may still write into its shared memory
}

// Shared memory: v[2][Nr], yup[Nr], zdn[Nr], part[NS-1][RPC], hist[steps][RPC] (float4),
// two mbarriers: the byte layout of k_chain_out_async.
template <int QH, int NS>
__global__ void k_chain_out_df(DevGeom g, const long* __restrict__ chain_off,
                               const float4* __restrict__ H, const float4* __restrict__ W,
                               double2* __restrict__ out, const double2* __restrict__ mid,
                               int CS, int steps_cap, int* __restrict__ status,
                               const long* __restrict__ parts, int bs) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ float4 cd_sh[];
  const ChainInfo ci = parts ? chain_info_part(g, parts, CS) : chain_info(g, chain_off, CS, bs);
  const int Nr = ci.Nr;
  const CaLane c = ca_lane<QH, NS>(Nr, CS, (int)cluster.block_rank());
  float4* v = cd_sh;
  float4* yup = v + 2 * Nr;    // y_{k-1}
  float4* zdn = yup + Nr;      // z_{k+1}
  float4* part = zdn + Nr;     // [NS - 1][RPC]
  float4* hist = part + (NS - 1) * c.RPC;
  uint64_t* bar = reinterpret_cast<uint64_t*>(hist + (long)steps_cap * c.RPC);
  const uint32_t bar0 = ca_smem(&bar[0]);
  const int km = ci.km, nb = ci.nb;
  const bool real_op = ci.m == 0;
  const double2* mc0 = mid + (long)ci.c * 3 * Nr;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = threadIdx.x; k < Nr; k += blockDim.x) {
    yup[k] = cd_split(mc0[k]);
    zdn[k] = cd_split(mc0[Nr + k]);
  }
  __syncthreads();
  constexpr int PD = CdDepth<QH>::PD;
  float4 mc[QH], mb[PD][QH];   // mb[q]: rows of block km + (t + q) step (t the next step)
  double2 yb[PD];
  // middle block: x_k = g_k - H_k y_{k-1} - W_k z_{k+1}
  dfl are = dfl_zero(), aim = dfl_zero();
  if (km > 0) {
    cd_load<QH>(H + (ci.boff + km) * ci.blk, c.r, c.s, c.q0, Nr, c.active, mc);
    dfl re, im;
    cd_dot<QH>(mc, yup, c.s, c.q0, Nr, real_op, re, im);
    are = dfl_add(are, re);
    aim = dfl_add(aim, im);
  }
  if (km < nb - 1) {
    cd_load<QH>(W + (ci.boff + km) * ci.blk, c.r, c.s, c.q0, Nr, c.active, mc);
    dfl re, im;
    cd_dot<QH>(mc, zdn, c.s, c.q0, Nr, real_op, re, im);
    are = dfl_add(are, re);
    aim = dfl_add(aim, im);
  }
  const int step = ci.dir == 0 ? -1 : 1;
  const int count = ci.dir == 0 ? km : nb - 1 - km;
#pragma unroll
  for (int q = 0; q < PD; ++q) {
    yb[q] = make_double2(0, 0);
    if (q + 1 <= count) {
      cd_load<QH>(W + (ci.boff + km + (q + 1) * step) * ci.blk, c.r, c.s, c.q0, Nr, c.active, mb[q]);
      if (c.active) yb[q] = out[ci.row(km + (q + 1) * step) + c.r];
    }
  }
  if (c.h > 0 && c.s == 0 && c.active)
    part[(c.h - 1) * c.RPC + c.lr] = make_float4(are.s, aim.s, are.c, aim.c);
  cluster.sync();   // barriers initialised everywhere, part written
  bool ok = true;
  if (threadIdx.x == 0) ca_expect(bar0, (uint32_t)Nr * 16u);
  if (c.h == 0 && c.active) {
    cd_gather<NS>(part, c.RPC, c.lr, are, aim);
    const float4 xk = cd_sub(mc0[2 * Nr + c.r], are, aim);
    if (c.s == 0 && ci.dir == 0) out[ci.row(km) + c.r] = cd_join(xk);
    const uint32_t la = ca_smem(v + c.r);
    for (int dst = c.s; dst < CS; dst += 8)
      cd_send(ca_mapa(la, (uint32_t)dst), ca_mapa(bar0, (uint32_t)dst), xk);
  }
  if (!ca_wait(bar0, 0u)) ok = false;
  // outward: top i = km-1 .. 0 with W_i x_{i+1}; bottom i = km+1 .. nb-1 with W_i x_{i-1}
  for (int t = 1; t <= count; ++t) {
    const int b = t & 1;
    if (threadIdx.x == 0) ca_expect(bar0 + 8 * b, (uint32_t)Nr * 16u);
#pragma unroll
    for (int q = 0; q < QH; ++q) mc[q] = mb[0][q];
    const double2 yc = yb[0];
#pragma unroll
    for (int d = 0; d + 1 < PD; ++d) {
#pragma unroll
      for (int q = 0; q < QH; ++q) mb[d][q] = mb[d + 1][q];
      yb[d] = yb[d + 1];
    }
    if (t + PD <= count) {
      const int ip = km + (t + PD) * step;
      cd_load<QH>(W + (ci.boff + ip) * ci.blk, c.r, c.s, c.q0, Nr, c.active, mb[PD - 1]);
      if (c.active) yb[PD - 1] = out[ci.row(ip) + c.r];
    }
    dfl re, im;
    cd_dot<QH>(mc, v + (b ^ 1) * Nr, c.s, c.q0, Nr, real_op, re, im);
    if (c.h > 0 && c.s == 0 && c.active)
      part[(c.h - 1) * c.RPC + c.lr] = make_float4(re.s, im.s, re.c, im.c);
    __syncthreads();
    if (c.h == 0 && c.active) {
      cd_gather<NS>(part, c.RPC, c.lr, re, im);
      const float4 x = cd_sub(yc, re, im);
      if (c.s == 0) hist[(t - 1) * c.RPC + c.lr] = x;
      const uint32_t la = ca_smem(v + b * Nr + c.r);
      for (int dst = c.s; dst < CS; dst += 8)
        cd_send(ca_mapa(la, (uint32_t)dst), ca_mapa(bar0 + 8 * b, (uint32_t)dst), x);
    }
    if (!ca_wait(bar0 + 8 * b, (uint32_t)((t >> 1) & 1))) ok = false;
  }
  if (!ok && status) atomicExch(status, 7);
  for (int idx = threadIdx.x; idx < count * c.RPC; idx += blockDim.x) {
    const int t = idx / c.RPC + 1, r = c.rank * c.RPC + idx % c.RPC;
    if (r < Nr) out[ci.row(km + t * step) + r] = cd_join(hist[idx]);
  }
  cluster.sync();
}

// Reduced system of partitioned chains: z = (I + K)^-1 xl_z per chain, xl_z the part-local
// solutions at the blocks that couple parts (unk_row: their element offsets in a state).
// grid = (ceil(nu_max Nr / 32), chains), block = 256 (8 lanes per row of the inverse),
// dynamic shared memory nu_max Nr float4.
__global__ void __launch_bounds__(256) k_spike_reduce_df(const long* __restrict__ unk_row,
                                                         const int* __restrict__ zoff,
                                                         const int* __restrict__ red_nu,
                                                         const long* __restrict__ red_off,
                                                         const float4* __restrict__ red,
                                                         const double2* __restrict__ out,
                                                         double2* __restrict__ zbuf, int Nr) {
  extern __shared__ float4 rv[];
  const int c = blockIdx.y;
  const int n = red_nu[c] * Nr;
  if (blockIdx.x * 32 >= n) return;   // the whole block: no unknown rows here
  const int z0 = zoff[c];
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x)
    rv[idx] = cd_split(out[unk_row[z0 + idx / Nr] + idx % Nr]);
  __syncthreads();
  const int s8 = threadIdx.x & 7;
  const int r = blockIdx.x * 32 + (threadIdx.x >> 3);
  dfl re0 = dfl_zero(), im0 = dfl_zero(), re1 = dfl_zero(), im1 = dfl_zero();
  if (r < n) {
    const float4* Mr = red + red_off[c] + (long)r * n;
    int k = s8;
    for (; k + 8 < n; k += 16) {
      cd_cmac(re0, im0, Mr[k], rv[k], false);
      cd_cmac(re1, im1, Mr[k + 8], rv[k + 8], false);
    }
    if (k < n) cd_cmac(re0, im0, Mr[k], rv[k], false);
  }
  dfl re = dfl_add(re0, re1), im = dfl_add(im0, im1);
  cd_reduce8(re, im);
  if (r < n && s8 == 0)
    zbuf[(long)(z0 + r / Nr) * Nr + r % Nr] = make_double2(dfl_to_double(re), dfl_to_double(im));
}

// Correction of partitioned chains: x_i = xl_i - V_i z(T) - Wsp_i z(B) in place, for the
// blocks of the parts that have a next (T) or a previous (B) part (blk_z: their z blocks,
// -1 for none).  The layout and grid of k_block_gemv_df (grid = 2 P, block = 256, Q >=
// ceil(Nr / 8) columns per lane); dynamic shared memory 2 Nr float4.
template <int Q>
__global__ void __launch_bounds__(256) k_spike_correct_df(DevGeom g, const long* __restrict__ chain_off,
                                                          const int* __restrict__ blk_z,
                                                          const float4* __restrict__ V,
                                                          const float4* __restrict__ Wsp,
                                                          const double2* __restrict__ zbuf,
                                                          double2* __restrict__ out) {
  extern __shared__ float4 zs[];
  const int Nr = g.Nr, P = g.P;
  const int p = blockIdx.x >> 1, fld = blockIdx.x & 1;
  const int m = g.pair_m[p], a = m / g.Ms, i = g.pair_l[p] - m;
  const int cls = (fld == 0) ? (i & 1) : 1 - (i & 1);
  const long gb = chain_off[2 * a + cls] + i;
  const int zT = blk_z[2 * gb], zB = blk_z[2 * gb + 1];
  if (zT < 0 && zB < 0) return;   // the whole block: a chain without parts
  const long row0 = ((long)fld * P + p) * Nr;
  for (int k = threadIdx.x; k < Nr; k += blockDim.x) {
    zs[k] = zT >= 0 ? cd_split(zbuf[(long)zT * Nr + k]) : make_float4(0.f, 0.f, 0.f, 0.f);
    zs[Nr + k] = zB >= 0 ? cd_split(zbuf[(long)zB * Nr + k]) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  const int s8 = threadIdx.x & 7;
  const int rows_per_pass = blockDim.x >> 3;
  const bool real_op = (m == 0);
  const float4* Vi = V + gb * (long)Nr * Nr;
  const float4* Wi = Wsp + gb * (long)Nr * Nr;
  for (int r = threadIdx.x >> 3; r < Nr + ((rows_per_pass - Nr % rows_per_pass) % rows_per_pass);
       r += rows_per_pass) {
    float4 av[Q], aw[Q];
    cd_load<Q>(Vi, r, s8, 0, Nr, r < Nr && zT >= 0, av);
    cd_load<Q>(Wi, r, s8, 0, Nr, r < Nr && zB >= 0, aw);
    dfl re0 = dfl_zero(), im0 = dfl_zero(), re1 = dfl_zero(), im1 = dfl_zero();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k = s8 + 8 * q;
      if (k < Nr) {
        cd_cmac(re0, im0, av[q], zs[k], real_op);
        cd_cmac(re1, im1, aw[q], zs[Nr + k], real_op);
      }
    }
    dfl re = dfl_add(re0, re1), im = dfl_add(im0, im1);
    cd_reduce8(re, im);
    if (r < Nr && s8 == 0) out[row0 + r] = cd_join(cd_sub(out[row0 + r], re, im));
  }
}

}  // namespace rsc
