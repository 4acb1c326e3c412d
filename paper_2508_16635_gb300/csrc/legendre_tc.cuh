// Legendre synthesis on the 5th-generation tensor cores (tcgen05), FP32 path.
//
// For one m, one parity class s of l - m (Sec. 3.1 transforms, split by the
// equatorial symmetry of P_l^m) and one table type w (P, dP/dtheta, P/sin),
// the sums over l are a GEMM
//     C[theta, col] = sum_k T_w[theta, l = m + s + 2k] X_w[k, col]
// with theta the north latitudes (M, padded to 128), k the degrees of the
// class (K) and col = (radius, component, re/im) (N).  Accuracy: each FP32
// operand x is split into hi = x with the low 13 mantissa bits cleared and
// lo = x - hi; three TF32 MMAs (hi hi + hi lo + lo hi) accumulate in FP32 in
// tensor memory, about 21 significant bits.  A tiles (tables) are prepared on
// the host in the canonical K-major core-matrix layout (8 rows x 16 bytes,
// K-direction stride 128 B, row-group stride Kpad/4 * 128 B) with hi and lo
// parts, and staged with bulk copies (cp.async.bulk) completing on an
// mbarrier; B tiles are transposed from the radial values by the CTA.  The
// epilogue reads tensor memory (tcgen05.ld) and forms the nine grid fields
// exactly as the CUDA-core synthesis does.
//
// One CTA = (m, RT = 8 radii, one 128-latitude tile); 128 threads (4 warps).
// All waits are bounded; a timeout sets *status and the CTA still frees its
// tensor memory before returning.
#pragma once

#include <stdint.h>

namespace rsc {

constexpr int kTcRadii = 8;               // radii per CTA
constexpr int kTcNP = 48;                 // 6 columns per radius (3 fields x re/im)
constexpr int kTcNV = 80;                 // 10 columns per radius (5 fields x re/im)
constexpr int kTcCols = 2 * kTcNP + 4 * kTcNV;   // 416 accumulator columns
constexpr int kTcAlloc = 512;             // tensor-memory columns allocated

struct TcTables {
  const float* tiles;        // all A tiles
  const long* off;           // [a][s][w][mt] float offset of the hi part (lo follows)
  const int* kpad;           // [a] padded K (multiple of 8) of m index a
  int nmt;                   // latitude tiles (of 128)
  int* status;               // set to RSC_ETIMEOUT (7) when a wait gives up
};

__device__ __forceinline__ uint32_t tc_smem(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05 (bits 46-48 = 0b001)
  return d;                // base offset 0, no swizzle
}

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128.
__device__ __forceinline__ uint32_t tc_idesc(int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
  }
  return done != 0;
}

__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

template <int NX>
__device__ __forceinline__ void tc_ld(uint32_t taddr, float (&v)[NX]);
template <>
__device__ __forceinline__ void tc_ld<2>(uint32_t taddr, float (&v)[2]) {
  uint32_t r0, r1;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
               : "=r"(r0), "=r"(r1) : "r"(taddr) : "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
}

// grid = (nm, ceil(Nd / 8), nmt); block = 128; dynamic smem from tc_synth_smem().
__global__ void __launch_bounds__(128) k_synth_tc(DevGeom g, TcTables tt, const float2* __restrict__ SR,
                                                  float2* __restrict__ FC) {
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  const int a = blockIdx.x;
  const int i0 = blockIdx.y * kTcRadii;
  const int mt = blockIdx.z;
  const int m = g.m_of[a];
  const int p0 = g.pstart[a];
  const int nl = g.L - m + 1;
  const int Kp = tt.kpad[a];
  const int Nd = g.Nd;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // shared memory: A hi | A lo (128 x Kp each), B hi | B lo (kTcNV x Kp each), barriers
  float* sAh = reinterpret_cast<float*>(tc_raw);
  float* sAl = sAh + 128 * Kp;
  float* sBh = sAl + 128 * Kp;
  float* sBl = sBh + kTcNV * Kp;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sBl + kTcNV * Kp);   // [0] copies, [1] MMAs
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const uint32_t bar_copy = tc_smem(&bar[0]), bar_mma = tc_smem(&bar[1]);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(tslot)),
                 "r"(kTcAlloc)
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
  const uint32_t sbo = (uint32_t)(Kp / 4) * 128u;
  const int nks = Kp / 8;
  uint32_t ph = 0;
  // phases (s, w): parity class outer, table type inner, so that the B operand of
  // w = 2 (P/sin) is the one already staged for w = 1 (dP/dtheta): the same columns
  for (int s = 0; s < 2 && ok; ++s) {
    for (int w = 0; w < 3 && ok; ++w) {
    const int NC = (w == 0) ? 3 : 5;          // components of this table type
    const int NW = (w == 0) ? kTcNP : kTcNV;  // N of the GEMM (padded)
    {
      // (1) tables: bulk copy of the hi and lo tiles
      if (tid == 0) {
        const float* src = tt.tiles + tt.off[((a * 2 + s) * 3 + w) * tt.nmt + mt];
        const uint32_t bytes = (uint32_t)(128 * Kp * 4);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_copy),
                     "r"(2 * bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                tc_smem(sAh)),
            "l"(src), "r"(bytes), "r"(bar_copy)
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                tc_smem(sAl)),
            "l"(src + 128 * Kp), "r"(bytes), "r"(bar_copy)
            : "memory");
      }
      // (2) B: columns n = (radius, component, re/im), K-major core-matrix layout; eight
      // independent gathers per thread are in flight before the first store
      const int vi[5] = {1, 2, 4, 5, 7};
      const int total = (w == 2) ? 0 : NW * Kp;   // w = 2 reuses the operand of w = 1
      for (int base = tid; base < total; base += 128 * 8) {
        float vals[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base + 128 * u;
          const int k = idx / NW;
          const int n = idx - k * NW;
          const int q = s + 2 * k;
          const int rr = n / (2 * NC);
          const int rem = n - rr * 2 * NC;
          const int c = rem >> 1, ri = rem & 1;
          const int i = i0 + rr;
          float v = 0.f;
          if (idx < total && q < nl && rr < kTcRadii && i < Nd) {
            const int comp = (w == 0) ? (c == 0 ? 0 : (c == 1 ? 3 : 6)) : vi[c];
            const float* z = reinterpret_cast<const float*>(SR + ((long)(p0 + q) * Nd + i) * 8 + comp);
            v = __ldg(z + ri);
          }
          vals[u] = v;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base + 128 * u;
          if (idx < total) {
            const int k = idx / NW;
            const int n = idx - k * NW;
            const float v = vals[u];
            const float h = tf32_hi(v);
            const int off = (n >> 3) * (Kp / 4) * 32 + (k >> 2) * 32 + (n & 7) * 4 + (k & 3);
            sBh[off] = h;
            sBl[off] = v - h;
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      ok = tc_wait(bar_copy, ph);
      // (3) the MMAs, issued by one thread
      if (tid == 0 && ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t col = (w == 0) ? s * kTcNP : 2 * kTcNP + ((w - 1) * 2 + s) * kTcNV;
        const uint32_t idesc = tc_idesc(NW);
        for (int t = 0; t < nks; ++t) {
          const uint32_t ko = (uint32_t)t * 256u;   // two core matrices of 128 B per k-step
          const uint64_t ah = tc_desc(tc_smem(sAh) + ko, 128, sbo);
          const uint64_t al = tc_desc(tc_smem(sAl) + ko, 128, sbo);
          const uint64_t bh = tc_desc(tc_smem(sBh) + ko, 128, sbo);
          const uint64_t bl = tc_desc(tc_smem(sBl) + ko, 128, sbo);
          tc_mma(tmem + col, ah, bh, idesc, t > 0 ? 1u : 0u);
          tc_mma(tmem + col, ah, bl, idesc, 1u);
          tc_mma(tmem + col, al, bh, idesc, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         bar_mma)
                     : "memory");
      }
      // shared operands are reused by the next phase: wait for the MMAs
      const bool mma_ok = ok ? tc_wait(bar_mma, ph) : false;
      ok = ok && mma_ok;
      ph ^= 1u;
      __syncthreads();
    }
    }
  }
  if (!ok && tid == 0) atomicExch(tt.status, 7);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // (4) epilogue: warp w owns latitudes (TMEM lanes) 32 w .. 32 w + 31 of this tile
  const int t = mt * 128 + warp * 32 + lane;
  const bool live = ok && t < g.nlat2;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
  const float mm = (float)m;
  const int K1 = g.K + 1, nlat = g.nlat;
  for (int rr = 0; rr < kTcRadii; ++rr) {
    const int i = i0 + rr;
    float Pe[6], Po[6], De[10], Do[10], Se[10], So[10];
    // the loads are warp-collective: every lane takes part
    for (int c = 0; c < 6; c += 2) {
      float v[2];
      tc_ld<2>(tl + rr * 6 + c, v); Pe[c] = v[0]; Pe[c + 1] = v[1];
      tc_ld<2>(tl + kTcNP + rr * 6 + c, v); Po[c] = v[0]; Po[c + 1] = v[1];
    }
    for (int c = 0; c < 10; c += 2) {
      float v[2];
      tc_ld<2>(tl + 2 * kTcNP + 0 * kTcNV + rr * 10 + c, v); De[c] = v[0]; De[c + 1] = v[1];
      tc_ld<2>(tl + 2 * kTcNP + 1 * kTcNV + rr * 10 + c, v); Do[c] = v[0]; Do[c + 1] = v[1];
      tc_ld<2>(tl + 2 * kTcNP + 2 * kTcNV + rr * 10 + c, v); Se[c] = v[0]; Se[c + 1] = v[1];
      tc_ld<2>(tl + 2 * kTcNP + 3 * kTcNV + rr * 10 + c, v); So[c] = v[0]; So[c + 1] = v[1];
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (!live || i >= Nd) continue;
#pragma unroll
    for (int hemi = 0; hemi < 2; ++hemi) {
      // north: E + O (P-type and dP-type); south: E - O (P-type), -E + O (dP-type)
      const float sg = hemi ? -1.f : 1.f;
      const int th = hemi ? (nlat - 1 - t) : t;
      float Pr[3], Pi[3], Dr[5], Di[5], Sr[5], Si[5];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Pr[c] = Pe[2 * c] + sg * Po[2 * c];
        Pi[c] = Pe[2 * c + 1] + sg * Po[2 * c + 1];
      }
#pragma unroll
      for (int u = 0; u < 5; ++u) {
        Dr[u] = sg * De[2 * u] + Do[2 * u];
        Di[u] = sg * De[2 * u + 1] + Do[2 * u + 1];
        Sr[u] = Se[2 * u] + sg * So[2 * u];
        Si[u] = Se[2 * u + 1] + sg * So[2 * u + 1];
      }
      float2 out[9];
      out[0] = make_float2(Pr[0], Pi[0]);                                    // u_r
      out[1] = make_float2(Dr[0] - mm * Si[1], Di[0] + mm * Sr[1]);           // u_th
      out[2] = make_float2(-mm * Si[0] - Dr[1], mm * Sr[0] - Di[1]);          // u_ph
      out[3] = make_float2(Pr[1], Pi[1]);                                    // omega_r
      out[4] = make_float2(Dr[2] - mm * Si[3], Di[2] + mm * Sr[3]);           // omega_th
      out[5] = make_float2(-mm * Si[2] - Dr[3], mm * Sr[2] - Di[3]);          // omega_ph
      out[6] = make_float2(Pr[2], Pi[2]);                                    // d_r T
      out[7] = make_float2(Dr[4], Di[4]);                                    // (1/r) d_th T
      out[8] = make_float2(-mm * Si[4], mm * Sr[4]);                          // (1/(r s)) d_ph T
#pragma unroll
      for (int fld = 0; fld < 9; ++fld)
        FC[(((long)fld * Nd + i) * K1 + a) * nlat + th] = out[fld];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcAlloc)
                 : "memory");
  }
}

}  // namespace rsc
