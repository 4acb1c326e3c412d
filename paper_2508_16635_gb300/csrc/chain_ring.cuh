// Double-float chain sweeps with a shared-memory ring of prefetched blocks (chain_ring = D):
// the sweeps of chain_df.cuh (y_i = g_i - H_i y_(i-+1), x_i = y_i - W_i x_(i+-1), twisted
// block Thomas of Sec. 3.2), with each CTA's rows of the next D blocks (and their g / y
// values) brought into shared memory by bulk copies (cp.async.bulk, completing on one
// mbarrier per ring stage) up to D block steps ahead, instead of one block ahead in
// registers.  The rows of one CTA in one block are contiguous (RPC rows of N_r float4), so
// a stage is one copy of RPC N_r 16 bytes plus one of RPC 16 bytes.
//
// One block step: wait for the stage, the lane's row sums from shared memory (Dot2 in
// FP32 pairs), the column-part reduction, the new rows sent to every CTA of the cluster
// with st.async (complete_tx on the receivers' exchange mbarrier), the stage refilled with
// the block D steps ahead (after the CTA barrier that ends every read of it), and the
// wait for the cluster's new vector.  Every wait is bounded (status RSC_ETIMEOUT); a final
// cluster barrier keeps each CTA resident until its peers stop writing into it.
#pragma once

#include "dfloat.h"

namespace rsc {

__device__ __forceinline__ void cr_bulk(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void cr_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Byte layout of the ring sweeps' dynamic shared memory (all offsets multiples of 16):
//   v[2][Nr], (outward: yup[Nr], zdn[Nr]), part[NS-1][RPC], hist[steps][RPC]  (float4)
//   ring[D][RPC * Nr] (float4), gring[D][RPC] (double2)
//   bars: exchange[2], full[D] (uint64)
struct CrLayout {
  size_t ring, gring, bars, total;
};

__host__ __device__ inline CrLayout cr_layout(int Nr, int RPC, int NS, int steps_cap, int D,
                                              bool outward) {
  CrLayout l;
  size_t o = ((outward ? 4 : 2) * (size_t)Nr + (size_t)RPC * (NS - 1 + steps_cap)) * 16;
  l.ring = o;
  o += (size_t)D * RPC * Nr * 16;
  l.gring = o;
  o += (size_t)D * RPC * 16;
  l.bars = o;
  o += (2 + (size_t)D) * 8;
  l.total = (o + 15) / 16 * 16;
  return l;
}

// The stage of step t (t = 1..count): the rows [r0, r0 + nrows) of block `blkp` and the
// nrows values vec[row(i) + r0 ..].
__device__ __forceinline__ void cr_issue(uint32_t ring_s, uint32_t gring_s, uint32_t bar,
                                         const float4* blkp, const double2* vrow, int r0,
                                         int nrows, int Nr) {
  if (nrows <= 0) {
    cr_arrive(bar);
    return;
  }
  const uint32_t bh = (uint32_t)nrows * Nr * 16u, bg = (uint32_t)nrows * 16u;
  ca_expect(bar, bh + bg);
  cr_bulk(ring_s, blkp + (long)r0 * Nr, bh, bar);
  cr_bulk(gring_s, vrow + r0, bg, bar);
}

template <int QH>
__device__ __forceinline__ void cr_load(const float4* __restrict__ rows, int lr, int s, int q0, int Nr,
                                        bool active, float4 (&reg)[QH]) {
#pragma unroll
  for (int q = 0; q < QH; ++q) {
    const int k = s + 8 * (q0 + q);
    reg[q] = (active && k < Nr) ? rows[(long)lr * Nr + k] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Forward half sweeps (as k_chain_half_df).  grid = 2 * 2 * nm * CS, block = 32 NS ceil(RPC / 4).
template <int QH, int NS>
__global__ void k_chain_half_ring(DevGeom g, const long* __restrict__ chain_off,
                                  const float4* __restrict__ H, double2* __restrict__ out,
                                  double2* __restrict__ mid, int CS, int steps_cap, int D,
                                  int* __restrict__ status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char cr_raw[];
  const ChainInfo ci = chain_info(g, chain_off, CS);
  const int Nr = ci.Nr;
  const CaLane c = ca_lane<QH, NS>(Nr, CS, (int)cluster.block_rank());
  const CrLayout lay = cr_layout(Nr, c.RPC, NS, steps_cap, D, false);
  float4* v = reinterpret_cast<float4*>(cr_raw);   // [2][Nr]
  float4* part = v + 2 * Nr;                        // [NS - 1][RPC]
  float4* hist = part + (NS - 1) * c.RPC;           // [steps_cap][RPC]
  float4* ring = reinterpret_cast<float4*>(cr_raw + lay.ring);
  double2* gring = reinterpret_cast<double2*>(cr_raw + lay.gring);
  uint64_t* bars = reinterpret_cast<uint64_t*>(cr_raw + lay.bars);
  const uint32_t bar0 = ca_smem(&bars[0]);         // exchange barriers [2]
  const uint32_t full0 = ca_smem(&bars[2]);        // ring barriers [D]
  const bool has = ci.dir == 0 ? (ci.km >= 1) : (ci.km <= ci.nb - 2);
  const int first = ci.dir == 0 ? 0 : ci.nb - 1;
  const int step = ci.dir == 0 ? 1 : -1;
  const int count = ci.dir == 0 ? ci.km - 1 : ci.nb - 2 - ci.km;
  const bool real_op = ci.m == 0;
  const int r0 = c.rank * c.RPC;
  const int nrows = min(c.RPC, Nr - r0);
  auto issue = [&](int t) {
    const int st = (t - 1) % D;
    const int i = first + t * step;
    cr_issue(ca_smem(ring + (size_t)st * c.RPC * Nr), ca_smem(gring + (size_t)st * c.RPC),
             full0 + 8 * st, H + (ci.boff + i) * ci.blk, out + ci.row(i), r0, nrows, Nr);
  };
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    for (int q = 0; q < D; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * q) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int t = 1; t <= min(D, count); ++t) issue(t);
  for (int k = threadIdx.x; k < Nr; k += blockDim.x)
    v[k] = has ? cd_split(out[ci.row(first) + k]) : make_float4(0.f, 0.f, 0.f, 0.f);
  cluster.sync();   // barriers initialised and v[0] loaded everywhere before any st.async
  bool ok = true;
  for (int t = 1; t <= count; ++t) {
    const int b = t & 1;
    const int st = (t - 1) % D;
    if (threadIdx.x == 0) ca_expect(bar0 + 8 * b, (uint32_t)Nr * 16u);
    if (!ca_wait(full0 + 8 * st, (uint32_t)(((t - 1) / D) & 1))) ok = false;
    float4 mc[QH];
    cr_load<QH>(ring + (size_t)st * c.RPC * Nr, c.lr, c.s, c.q0, Nr, c.active, mc);
    const double2 gc = c.active ? gring[(size_t)st * c.RPC + c.lr] : make_double2(0, 0);
    dfl re, im;
    cd_dot<QH>(mc, v + (b ^ 1) * Nr, c.s, c.q0, Nr, real_op, re, im);
    if (c.h > 0 && c.s == 0 && c.active)
      part[(c.h - 1) * c.RPC + c.lr] = make_float4(re.s, im.s, re.c, im.c);
    __syncthreads();   // every read of stage st done; parts written
    if (threadIdx.x == 0 && t + D <= count) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + D);
    }
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

// Middle block and outward sweeps (as k_chain_out_df).
template <int QH, int NS>
__global__ void k_chain_out_ring(DevGeom g, const long* __restrict__ chain_off,
                                 const float4* __restrict__ H, const float4* __restrict__ W,
                                 double2* __restrict__ out, const double2* __restrict__ mid,
                                 int CS, int steps_cap, int D, int* __restrict__ status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char cr_raw[];
  const ChainInfo ci = chain_info(g, chain_off, CS);
  const int Nr = ci.Nr;
  const CaLane c = ca_lane<QH, NS>(Nr, CS, (int)cluster.block_rank());
  const CrLayout lay = cr_layout(Nr, c.RPC, NS, steps_cap, D, true);
  float4* v = reinterpret_cast<float4*>(cr_raw);
  float4* yup = v + 2 * Nr;    // y_{k-1}
  float4* zdn = yup + Nr;      // z_{k+1}
  float4* part = zdn + Nr;     // [NS - 1][RPC]
  float4* hist = part + (NS - 1) * c.RPC;
  float4* ring = reinterpret_cast<float4*>(cr_raw + lay.ring);
  double2* gring = reinterpret_cast<double2*>(cr_raw + lay.gring);
  uint64_t* bars = reinterpret_cast<uint64_t*>(cr_raw + lay.bars);
  const uint32_t bar0 = ca_smem(&bars[0]);
  const uint32_t full0 = ca_smem(&bars[2]);
  const int km = ci.km, nb = ci.nb;
  const bool real_op = ci.m == 0;
  const double2* mc0 = mid + (long)ci.c * 3 * Nr;
  const int step = ci.dir == 0 ? -1 : 1;
  const int count = ci.dir == 0 ? km : nb - 1 - km;
  const int r0 = c.rank * c.RPC;
  const int nrows = min(c.RPC, Nr - r0);
  auto issue = [&](int t) {
    const int st = (t - 1) % D;
    const int i = km + t * step;
    cr_issue(ca_smem(ring + (size_t)st * c.RPC * Nr), ca_smem(gring + (size_t)st * c.RPC),
             full0 + 8 * st, W + (ci.boff + i) * ci.blk, out + ci.row(i), r0, nrows, Nr);
  };
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    for (int q = 0; q < D; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * q) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = threadIdx.x; k < Nr; k += blockDim.x) {
    yup[k] = cd_split(mc0[k]);
    zdn[k] = cd_split(mc0[Nr + k]);
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int t = 1; t <= min(D, count); ++t) issue(t);
  // middle block: x_k = g_k - H_k y_{k-1} - W_k z_{k+1}
  float4 mc[QH];
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
  for (int t = 1; t <= count; ++t) {
    const int b = t & 1;
    const int st = (t - 1) % D;
    if (threadIdx.x == 0) ca_expect(bar0 + 8 * b, (uint32_t)Nr * 16u);
    if (!ca_wait(full0 + 8 * st, (uint32_t)(((t - 1) / D) & 1))) ok = false;
    cr_load<QH>(ring + (size_t)st * c.RPC * Nr, c.lr, c.s, c.q0, Nr, c.active, mc);
    const double2 yc = c.active ? gring[(size_t)st * c.RPC + c.lr] : make_double2(0, 0);
    dfl re, im;
    cd_dot<QH>(mc, v + (b ^ 1) * Nr, c.s, c.q0, Nr, real_op, re, im);
    if (c.h > 0 && c.s == 0 && c.active)
      part[(c.h - 1) * c.RPC + c.lr] = make_float4(re.s, im.s, re.c, im.c);
    __syncthreads();
    if (threadIdx.x == 0 && t + D <= count) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + D);
    }
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

}  // namespace rsc
