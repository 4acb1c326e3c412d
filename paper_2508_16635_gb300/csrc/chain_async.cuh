// Chain sweeps of the implicit-Coriolis solve (Sec. 3.2) with asynchronous cluster
// exchange: the same twisted block-Thomas sweeps as k_chain_half / k_chain_out, laid out for
// GB300's FP64 units (one per SM sub-partition, 64 cycles per warp instruction):
//   * each row group of 4 rows (8 lanes per row) is split over NS = 2 or 4 warps by
//     columns, so one block step issues 1/NS as many FP64 multiply-adds per warp;
//   * a block's new rows travel to every CTA of the cluster as st.async stores that
//     complete on the receiver's mbarrier (expect_tx of Nr x 16 bytes per step), instead of
//     a cluster-wide barrier per block.
// Every wait on an mbarrier is bounded; a timeout sets *status = RSC_ETIMEOUT (7) and the
// sweep runs on (with meaningless values) so that no peer waits forever; the kernel ends
// with a hardware cluster barrier so no CTA leaves while peers may still write into it.
#pragma once

namespace rsc {

__device__ __forceinline__ uint32_t ca_smem(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t ca_mapa(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void ca_send(uint32_t raddr, uint32_t rbar, double2 v) {
  asm volatile(
      "st.async.weak.shared::cluster.mbarrier::complete_tx::bytes.v2.b64 [%0], {%1, %2}, [%3];" ::"r"(
          raddr),
      "l"(__double_as_longlong(v.x)), "l"(__double_as_longlong(v.y)), "r"(rbar)
      : "memory");
}

__device__ __forceinline__ void ca_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool ca_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 18) && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 q, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// One lane's share of a row dot product over the columns s + 8 q, q in [q0, q0 + QH).
template <int QH>
__device__ __forceinline__ double2 ca_dot(const double2 (&reg)[QH], const double2* v, int s, int q0,
                                          int Nr, bool real_op) {
  double2 a0 = {0, 0}, a1 = {0, 0};
  if (real_op) {
#pragma unroll
    for (int q = 0; q < QH; q += 2) {
      const int k0 = s + 8 * (q0 + q), k1 = k0 + 8;
      if (k0 < Nr) { a0.x = fma(reg[q].x, v[k0].x, a0.x); a0.y = fma(reg[q].x, v[k0].y, a0.y); }
      if (q + 1 < QH && k1 < Nr) {
        a1.x = fma(reg[q + 1].x, v[k1].x, a1.x);
        a1.y = fma(reg[q + 1].x, v[k1].y, a1.y);
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < QH; q += 2) {
      const int k0 = s + 8 * (q0 + q), k1 = k0 + 8;
      if (k0 < Nr) a0 = cmac(a0, reg[q], v[k0]);
      if (q + 1 < QH && k1 < Nr) a1 = cmac(a1, reg[q + 1], v[k1]);
    }
  }
  double2 acc = make_double2(a0.x + a1.x, a0.y + a1.y);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  return acc;
}

template <int QH>
__device__ __forceinline__ void ca_load(const double2* __restrict__ M, int r, int s, int q0, int Nr,
                                        bool active, double2 (&reg)[QH]) {
#pragma unroll
  for (int q = 0; q < QH; ++q) {
    const int k = s + 8 * (q0 + q);
    reg[q] = (active && k < Nr) ? M[(long)r * Nr + k] : make_double2(0, 0);
  }
}

// Per-CTA layout shared by both kernels.
struct CaLane {
  int rank, RPC, lr, r, s, h, q0;
  bool active;
};

template <int QH, int NS>
__device__ __forceinline__ CaLane ca_lane(int Nr, int CS, int rank) {
  CaLane c;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  c.rank = rank;
  c.RPC = (Nr + CS - 1) / CS;
  c.h = warp % NS;                        // column part
  c.lr = (warp / NS) * 4 + (lane >> 3);   // row within the CTA
  c.r = rank * c.RPC + c.lr;
  c.s = lane & 7;
  c.q0 = c.h * QH;
  c.active = c.lr < c.RPC && c.r < Nr;
  return c;
}

// Shared memory: v[2][Nr] (double2), part[NS-1][RPC], hist[steps][RPC], then two
// mbarriers (8-byte aligned: every region is a multiple of 16 bytes).
// grid = 2 * 2 * nm * CS (clusters of CS), block = 32 NS ceil(RPC / 4).
template <int QH, int NS>
__global__ void k_chain_half_async(DevGeom g, const long* __restrict__ chain_off,
                                   const double2* __restrict__ H, double2* __restrict__ out,
                                   double2* __restrict__ mid, int CS, int steps_cap,
                                   int* __restrict__ status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double2 ca_sh[];
  const ChainInfo ci = chain_info(g, chain_off, CS);
  const int Nr = ci.Nr;
  const CaLane c = ca_lane<QH, NS>(Nr, CS, (int)cluster.block_rank());
  double2* v = ca_sh;                       // [2][Nr]
  double2* part = v + 2 * Nr;               // [NS - 1][RPC]
  double2* hist = part + (NS - 1) * c.RPC;  // [steps_cap][RPC]
  uint64_t* bar = reinterpret_cast<uint64_t*>(hist + (long)steps_cap * c.RPC);
  const uint32_t bar0 = ca_smem(&bar[0]);
  const bool has = ci.dir == 0 ? (ci.km >= 1) : (ci.km <= ci.nb - 2);
  const int first = ci.dir == 0 ? 0 : ci.nb - 1;
  const int step = ci.dir == 0 ? 1 : -1;
  const int count = ci.dir == 0 ? ci.km - 1 : ci.nb - 2 - ci.km;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = threadIdx.x; k < Nr; k += blockDim.x)
    v[k] = has ? out[ci.row(first) + k] : make_double2(0, 0);
  double2 mc[QH], mn[QH];
  double2 gn = {0, 0};
  if (count > 0) {
    ca_load<QH>(H + (ci.boff + first + step) * ci.blk, c.r, c.s, c.q0, Nr, c.active, mn);
    if (c.active) gn = out[ci.row(first + step) + c.r];
  }
  cluster.sync();   // barriers initialised and v[0] loaded everywhere before any st.async
  bool ok = true;
  for (int t = 1; t <= count; ++t) {
    const int i = first + t * step;
    const int b = t & 1;
    if (threadIdx.x == 0) ca_expect(bar0 + 8 * b, (uint32_t)Nr * 16u);
#pragma unroll
    for (int q = 0; q < QH; ++q) mc[q] = mn[q];
    const double2 gc = gn;
    if (t < count) {
      ca_load<QH>(H + (ci.boff + i + step) * ci.blk, c.r, c.s, c.q0, Nr, c.active, mn);
      if (c.active) gn = out[ci.row(i + step) + c.r];
    }
    const double2 acc = ca_dot<QH>(mc, v + (b ^ 1) * Nr, c.s, c.q0, Nr, ci.m == 0);
    if (c.h > 0 && c.s == 0 && c.active) part[(c.h - 1) * c.RPC + c.lr] = acc;
    __syncthreads();
    if (c.h == 0 && c.active) {
      double2 p = acc;
#pragma unroll
      for (int q = 1; q < NS; ++q) {
        p.x += part[(q - 1) * c.RPC + c.lr].x;
        p.y += part[(q - 1) * c.RPC + c.lr].y;
      }
      const double2 y = make_double2(gc.x - p.x, gc.y - p.y);
      if (c.s == 0) hist[(t - 1) * c.RPC + c.lr] = y;
      const uint32_t la = ca_smem(v + b * Nr + c.r);
      for (int dst = c.s; dst < CS; dst += 8)
        ca_send(ca_mapa(la, (uint32_t)dst), ca_mapa(bar0 + 8 * b, (uint32_t)dst), y);
    }
    if (!ca_wait(bar0 + 8 * b, (uint32_t)(((t - 1) >> 1) & 1))) ok = false;
  }
  if (!ok && status) atomicExch(status, 7);
  for (int idx = threadIdx.x; idx < count * c.RPC; idx += blockDim.x) {
    const int t = idx / c.RPC + 1, r = c.rank * c.RPC + idx % c.RPC;
    if (r < Nr) out[ci.row(first + t * step) + r] = hist[idx];
  }
  if (c.rank == 0) {
    const double2* last = v + ((count > 0 ? count : 0) & 1) * Nr;
    double2* dst = mid + ((long)ci.c * 3 + ci.dir) * Nr;
    for (int k = threadIdx.x; k < Nr; k += blockDim.x) dst[k] = has ? last[k] : make_double2(0, 0);
    if (ci.dir == 0) {
      double2* gm = mid + ((long)ci.c * 3 + 2) * Nr;
      for (int k = threadIdx.x; k < Nr; k += blockDim.x) gm[k] = out[ci.row(ci.km) + k];
    }
  }
  cluster.sync();   // no CTA leaves while a peer may still write into its shared memory
}

// Shared memory: v[2][Nr], yup[Nr], zdn[Nr], part[NS-1][RPC], hist[steps][RPC], two mbarriers.
template <int QH, int NS>
__global__ void k_chain_out_async(DevGeom g, const long* __restrict__ chain_off,
                                  const double2* __restrict__ H, const double2* __restrict__ W,
                                  double2* __restrict__ out, const double2* __restrict__ mid,
                                  int CS, int steps_cap, int* __restrict__ status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double2 ca_sh[];
  const ChainInfo ci = chain_info(g, chain_off, CS);
  const int Nr = ci.Nr;
  const CaLane c = ca_lane<QH, NS>(Nr, CS, (int)cluster.block_rank());
  double2* v = ca_sh;
  double2* yup = v + 2 * Nr;    // y_{k-1}
  double2* zdn = yup + Nr;      // z_{k+1}
  double2* part = zdn + Nr;                 // [NS - 1][RPC]
  double2* hist = part + (NS - 1) * c.RPC;
  uint64_t* bar = reinterpret_cast<uint64_t*>(hist + (long)steps_cap * c.RPC);
  const uint32_t bar0 = ca_smem(&bar[0]);
  const int km = ci.km, nb = ci.nb;
  const double2* mc0 = mid + (long)ci.c * 3 * Nr;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = threadIdx.x; k < Nr; k += blockDim.x) {
    yup[k] = mc0[k];
    zdn[k] = mc0[Nr + k];
  }
  __syncthreads();
  double2 mc[QH], mn[QH];
  // middle block: x_k = g_k - H_k y_{k-1} - W_k z_{k+1}
  double2 acc = {0, 0};
  if (km > 0) {
    ca_load<QH>(H + (ci.boff + km) * ci.blk, c.r, c.s, c.q0, Nr, c.active, mc);
    const double2 a1 = ca_dot<QH>(mc, yup, c.s, c.q0, Nr, ci.m == 0);
    acc.x += a1.x; acc.y += a1.y;
  }
  if (km < nb - 1) {
    ca_load<QH>(W + (ci.boff + km) * ci.blk, c.r, c.s, c.q0, Nr, c.active, mc);
    const double2 a2 = ca_dot<QH>(mc, zdn, c.s, c.q0, Nr, ci.m == 0);
    acc.x += a2.x; acc.y += a2.y;
  }
  const int step = ci.dir == 0 ? -1 : 1;
  const int count = ci.dir == 0 ? km : nb - 1 - km;
  double2 yn = {0, 0};
  if (count > 0) {
    ca_load<QH>(W + (ci.boff + km + step) * ci.blk, c.r, c.s, c.q0, Nr, c.active, mn);
    if (c.active) yn = out[ci.row(km + step) + c.r];
  }
  if (c.h > 0 && c.s == 0 && c.active) part[(c.h - 1) * c.RPC + c.lr] = acc;
  cluster.sync();   // barriers initialised everywhere, part written
  bool ok = true;
  if (threadIdx.x == 0) ca_expect(bar0, (uint32_t)Nr * 16u);
  if (c.h == 0 && c.active) {
    const double2 gk = mc0[2 * Nr + c.r];
    double2 p = acc;
#pragma unroll
    for (int q = 1; q < NS; ++q) {
      p.x += part[(q - 1) * c.RPC + c.lr].x;
      p.y += part[(q - 1) * c.RPC + c.lr].y;
    }
    const double2 xk = make_double2(gk.x - p.x, gk.y - p.y);
    if (c.s == 0 && ci.dir == 0) out[ci.row(km) + c.r] = xk;
    const uint32_t la = ca_smem(v + c.r);
    for (int dst = c.s; dst < CS; dst += 8)
      ca_send(ca_mapa(la, (uint32_t)dst), ca_mapa(bar0, (uint32_t)dst), xk);
  }
  if (!ca_wait(bar0, 0u)) ok = false;
  // outward: top i = km-1 .. 0 with W_i x_{i+1}; bottom i = km+1 .. nb-1 with W_i x_{i-1}
  for (int t = 1; t <= count; ++t) {
    const int i = km + t * step;
    const int b = t & 1;
    if (threadIdx.x == 0) ca_expect(bar0 + 8 * b, (uint32_t)Nr * 16u);
#pragma unroll
    for (int q = 0; q < QH; ++q) mc[q] = mn[q];
    const double2 yc = yn;
    if (t < count) {
      ca_load<QH>(W + (ci.boff + i + step) * ci.blk, c.r, c.s, c.q0, Nr, c.active, mn);
      if (c.active) yn = out[ci.row(i + step) + c.r];
    }
    const double2 a3 = ca_dot<QH>(mc, v + (b ^ 1) * Nr, c.s, c.q0, Nr, ci.m == 0);
    if (c.h > 0 && c.s == 0 && c.active) part[(c.h - 1) * c.RPC + c.lr] = a3;
    __syncthreads();
    if (c.h == 0 && c.active) {
      double2 p = a3;
#pragma unroll
      for (int q = 1; q < NS; ++q) {
        p.x += part[(q - 1) * c.RPC + c.lr].x;
        p.y += part[(q - 1) * c.RPC + c.lr].y;
      }
      const double2 x = make_double2(yc.x - p.x, yc.y - p.y);
      if (c.s == 0) hist[(t - 1) * c.RPC + c.lr] = x;
      const uint32_t la = ca_smem(v + b * Nr + c.r);
      for (int dst = c.s; dst < CS; dst += 8)
        ca_send(ca_mapa(la, (uint32_t)dst), ca_mapa(bar0 + 8 * b, (uint32_t)dst), x);
    }
    if (!ca_wait(bar0 + 8 * b, (uint32_t)((t >> 1) & 1))) ok = false;
  }
  if (!ok && status) atomicExch(status, 7);
  for (int idx = threadIdx.x; idx < count * c.RPC; idx += blockDim.x) {
    const int t = idx / c.RPC + 1, r = c.rank * c.RPC + idx % c.RPC;
    if (r < Nr) out[ci.row(km + t * step) + r] = hist[idx];
  }
  cluster.sync();
}

}  // namespace rsc
