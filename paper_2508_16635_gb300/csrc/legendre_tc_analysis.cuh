// Legendre analysis on the 5th-generation tensor cores (tcgen05), FP32 path.
//
// For one m and one parity class s of l - m, the Gauss-weighted projections of the
// analysis (Sec. 3.1 transforms) are GEMMs over the north latitudes t:
//     D[k, col] = sum_t W_w[l = m + s + 2k, t] B[col, t]
// with rows k the degrees of the class (M = 128, zero-padded), K = latitudes (staged in
// chunks of kTaKc), and the columns of B the equatorially symmetric or antisymmetric
// parts F(t) +- F(pi - t) of the products of 8 radii.  Three table types w: P (with F_r
// and U.grad T), P/sin (with F_theta, F_phi) and dP/dtheta (with F_theta, F_phi of the
// other symmetry); every GEMM has N = 32 columns (8 radii x 2 fields x re/im).  The
// symmetric and antisymmetric B blocks are staged once per chunk and serve both parity
// classes.  Accuracy as in the synthesis: 3xTF32 (hi hi + hi lo + lo hi) in FP32 tensor
// memory.  The epilogue reads tensor memory (tcgen05.ld) and forms Q, S, T, N of the
// CUDA-core analysis (k_analysis) for its degree (one TMEM lane per degree).
//
// One CTA = (m, 8 radii); kTaThreads = 256 threads.  All waits are bounded; a timeout sets
// *status and the CTA still frees its tensor memory.
#pragma once

namespace rsc {

constexpr int kTaRadii = 8;     // radii per CTA
constexpr int kTaKc = 48;       // latitudes per staged chunk (multiple of 8)
constexpr int kTaN = 32;        // columns of each GEMM
constexpr int kTaAlloc = 256;   // tensor-memory columns: 2 parities x 3 tables x 32
constexpr int kTaThreads = 256; // two warpgroups: both gather B; in the epilogue warpgroup g
                                // reads parity class g from its warp quadrant's lanes

struct TaTables {
  const float* tiles;   // A tiles, hi then lo, K-major core-matrix layout
  const long* off;      // [a][s][w][chunk] float offset of the hi part
  int nchunk;           // latitude chunks of kTaKc
  int* status;
};

template <int NX>
__device__ __forceinline__ void ta_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// Shared memory: A[3] (hi | lo, 128 x kTaKc each), B[2] (sym, ant; hi | lo, 64 x kTaKc
// each), then two mbarriers and the TMEM slot.
inline size_t ta_smem() {
  return (3 * 2 * 128 * (size_t)kTaKc + 2 * 2 * 64 * (size_t)kTaKc) * sizeof(float) + 64;
}

// grid = (nm, ceil(Nd / 8)); block = kTaThreads.
__global__ void __launch_bounds__(kTaThreads) k_analysis_tc(DevGeom g, TaTables tt,
                                                     const float2* __restrict__ FA,
                                                     float2* __restrict__ AR) {
  extern __shared__ __align__(1024) unsigned char ta_raw[];
  const int a = blockIdx.x;
  const int i0 = blockIdx.y * kTaRadii;
  const int m = g.m_of[a];
  const int p0 = g.pstart[a];
  const int nl = g.L - m + 1;
  const int Nd = g.Nd, K1 = g.K + 1, nlat = g.nlat, n2 = g.nlat2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int AT = 128 * kTaKc;   // floats per A half-tile
  constexpr int BT = 64 * kTaKc;    // floats per B half-block
  float* sA = reinterpret_cast<float*>(ta_raw);   // [w][hi | lo]
  float* sB = sA + 3 * 2 * AT;                    // [sym | ant][hi | lo]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB + 2 * 2 * BT);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const uint32_t bar_copy = tc_smem(&bar[0]), bar_mma = tc_smem(&bar[1]);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(tslot)),
                 "r"(kTaAlloc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_copy), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_mma), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  bool ok = true;
  uint32_t ph = 0;
  const uint32_t sboA = (uint32_t)(kTaKc / 4) * 128u;   // row-group stride of both operands
  const int qmap[4] = {1, 2, 0, 3};                        // B fields: theta, phi, r, U.grad T
  for (int c = 0; c < tt.nchunk && ok; ++c) {
    // (1) B: sym / ant of the 4 fields of 8 radii at latitudes c kTaKc + k; column
    // n = f * 16 + rr * 2 + re/im, K-major core-matrix layout; eight pairs of gathers in flight
    const int total = 4 * kTaRadii * kTaKc;
    for (int base = tid; base < total; base += kTaThreads * 8) {
      float2 nv[8], sv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + kTaThreads * u;
        const int f = idx / (kTaRadii * kTaKc);
        const int rem = idx - f * kTaRadii * kTaKc;
        const int rr = rem / kTaKc, k = rem - rr * kTaKc;
        const int t = c * kTaKc + k, i = i0 + rr;
        nv[u] = make_float2(0.f, 0.f);
        sv[u] = make_float2(0.f, 0.f);
        if (idx < total && t < n2 && i < Nd) {
          const float2* src = FA + (((long)qmap[f] * Nd + i) * K1 + a) * nlat;
          nv[u] = __ldg(src + t);
          sv[u] = __ldg(src + (nlat - 1 - t));
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + kTaThreads * u;
        if (idx >= total) continue;
        const int f = idx / (kTaRadii * kTaKc);
        const int rem = idx - f * kTaRadii * kTaKc;
        const int rr = rem / kTaKc, k = rem - rr * kTaKc;
        const float val[4] = {nv[u].x + sv[u].x, nv[u].y + sv[u].y, nv[u].x - sv[u].x,
                              nv[u].y - sv[u].y};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int blk = q >> 1, n = f * 16 + rr * 2 + (q & 1);
          const int off = (n >> 3) * (kTaKc / 4) * 32 + (k >> 2) * 32 + (n & 7) * 4 + (k & 3);
          const float h = tf32_hi(val[q]);
          sB[(blk * 2 + 0) * BT + off] = h;
          sB[(blk * 2 + 1) * BT + off] = val[q] - h;
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    for (int s = 0; s < 2 && ok; ++s) {
      // (2) tables P, P/sin, dP/dtheta of this parity and chunk: six bulk copies
      if (tid == 0) {
        const uint32_t bytes = (uint32_t)(AT * 4);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_copy),
                     "r"(6 * bytes)
                     : "memory");
        for (int w = 0; w < 3; ++w) {
          const float* src = tt.tiles + tt.off[((a * 2 + s) * 3 + w) * tt.nchunk + c];
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  tc_smem(sA + w * 2 * AT)),
              "l"(src), "r"(bytes), "r"(bar_copy)
              : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  tc_smem(sA + w * 2 * AT + AT)),
              "l"(src + AT), "r"(bytes), "r"(bar_copy)
              : "memory");
        }
      }
      ok = tc_wait(bar_copy, ph);
      // (3) MMAs: P with (r, U.grad T) of CP; P/sin with (theta, phi) of CP; dP with
      // (theta, phi) of CD; CP = sym for s = 0 (P even about the equator), ant for s = 1
      if (tid == 0 && ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int cp = s, cd = 1 - s;
        const uint32_t idesc = tc_idesc(kTaN);
        const uint32_t col_half = 4u * sboA;   // B columns 32.. (four 8-row groups)
        for (int w = 0; w < 3; ++w) {
          const uint32_t dcol = (uint32_t)(s * 96 + w * 32);
          const float* Ah = sA + w * 2 * AT;
          const float* Bh = sB + ((w == 2 ? cd : cp) * 2) * BT;
          const uint32_t boff = (w == 0) ? col_half : 0u;
          for (int t = 0; t < kTaKc / 8; ++t) {
            const uint32_t ko = (uint32_t)t * 256u;
            const uint64_t ah = tc_desc(tc_smem(Ah) + ko, 128, sboA);
            const uint64_t al = tc_desc(tc_smem(Ah + AT) + ko, 128, sboA);
            const uint64_t bh = tc_desc(tc_smem(Bh) + boff + ko, 128, sboA);
            const uint64_t bl = tc_desc(tc_smem(Bh + BT) + boff + ko, 128, sboA);
            tc_mma(tmem + dcol, ah, bh, idesc, (c > 0 || t > 0) ? 1u : 0u);
            tc_mma(tmem + dcol, ah, bl, idesc, 1u);
            tc_mma(tmem + dcol, al, bh, idesc, 1u);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         bar_mma)
                     : "memory");
      }
      // the tables and (after the last parity) the B blocks are reused: wait for the MMAs
      const bool mma_ok = ok ? tc_wait(bar_mma, ph) : false;
      ok = ok && mma_ok;
      ph ^= 1u;
      __syncthreads();
    }
  }
  if (!ok && tid == 0) atomicExch(tt.status, 7);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // (4) epilogue: TMEM lane = degree index k of the class; warp w owns lanes 32 (w % 4) ..
  // 32 (w % 4) + 31 (its quadrant), for the parity class w / 4
  const int quad = warp & 3;
  const int row = quad * 32 + lane;
  const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
  const float mm = (float)m;
  for (int s = warp >> 2; s < 2; s += kTaThreads / 128) {
    float Pv[32], Xv[32], Yv[32];
    {
      float v[16];
      ta_ld16<16>(tl + s * 96 + 0, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) Pv[q] = v[q];
      ta_ld16<16>(tl + s * 96 + 16, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) Pv[16 + q] = v[q];
      ta_ld16<16>(tl + s * 96 + 32, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) Xv[q] = v[q];
      ta_ld16<16>(tl + s * 96 + 48, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) Xv[16 + q] = v[q];
      ta_ld16<16>(tl + s * 96 + 64, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) Yv[q] = v[q];
      ta_ld16<16>(tl + s * 96 + 80, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) Yv[16 + q] = v[q];
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int qd = s + 2 * row;   // l - m
    if (!ok || qd >= nl) continue;
    const int l = m + qd;
    const float il = (l > 0) ? 1.0f / ((float)l * (float)(l + 1)) : 0.0f;
    for (int rr = 0; rr < kTaRadii; ++rr) {
      const int i = i0 + rr;
      if (i >= Nd) break;
      // P region columns: r (rr*2 + re/im), U.grad T (16 + ...); P/sin and dP regions:
      // theta (rr*2 + re/im), phi (16 + ...)
      const float Qr = Pv[rr * 2], Qi = Pv[rr * 2 + 1];
      const float Nr = Pv[16 + rr * 2], Ni = Pv[16 + rr * 2 + 1];
      const float Xtr = Xv[rr * 2], Xti = Xv[rr * 2 + 1];
      const float Xpr = Xv[16 + rr * 2], Xpi = Xv[16 + rr * 2 + 1];
      const float Ytr = Yv[rr * 2], Yti = Yv[rr * 2 + 1];
      const float Ypr = Yv[16 + rr * 2], Ypi = Yv[16 + rr * 2 + 1];
      // S = dP F_th - i m P/s F_ph ;  T = -i m P/s F_th - dP F_ph
      const float Sr = Ytr + mm * Xpi, Si = Yti - mm * Xpr;
      const float Tr = mm * Xti - Ypr, Ti = -mm * Xtr - Ypi;
      float2* o = AR + ((long)(p0 + qd) * Nd + i) * 4;
      o[0] = make_float2(Qr, Qi);
      o[1] = make_float2(Sr * il, Si * il);
      o[2] = make_float2(Tr * il, Ti * il);
      o[3] = make_float2(Nr, Ni);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTaAlloc)
                 : "memory");
  }
}

}  // namespace rsc
