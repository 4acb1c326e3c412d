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
// One CTA = (m, RT = 8 radii, one 128-latitude tile); kTcThreads = 256 threads (8 warps).
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
constexpr int kTcThreads = 256;           // two warpgroups: both gather the B operands; in
                                          // the epilogue each reads its warp quadrant's
                                          // tensor-memory lanes for half of the radii

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

// B operand of phase (s, w): columns n = (radius, component, re/im), K-major core-matrix
// layout; eight independent gathers per thread are in flight before the first store.
// (Consecutive threads take consecutive columns of one degree, whose sources lie in one
// 512-byte span of the radial values; a lane-per-core-matrix-entry mapping measured 17 %
// slower.)
__device__ __forceinline__ void tc_gather_b(const float2* __restrict__ SR, int p0, int nl, int i0,
                                            int Nd, int Kp, int s, int w, float* sBh, float* sBl,
                                            int tid) {
  const int NC = (w == 0) ? 3 : 5;          // components of this table type
  const int NW = (w == 0) ? kTcNP : kTcNV;  // N of the GEMM (padded)
  const int total = NW * Kp;
  for (int base = tid; base < total; base += kTcThreads * 8) {
    float vals[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + kTcThreads * u;
      const int k = idx / NW;
      const int n = idx - k * NW;
      const int q = s + 2 * k;
      const int rr = n / (2 * NC);
      const int rem = n - rr * 2 * NC;
      const int c = rem >> 1, ri = rem & 1;
      const int i = i0 + rr;
      float v = 0.f;
      if (idx < total && q < nl && rr < kTcRadii && i < Nd) {
        const int comp = (w == 0) ? (c == 0 ? 0 : (c == 1 ? 3 : 6))
                                  : (c < 2 ? c + 1 : (c < 4 ? c + 2 : 7));   // 1, 2, 4, 5, 7
        const float* z = reinterpret_cast<const float*>(SR + ((long)(p0 + q) * Nd + i) * 8 + comp);
        v = __ldg(z + ri);
      }
      vals[u] = v;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + kTcThreads * u;
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
}

// Bulk copy of the hi and lo A tiles of one phase (one thread), completing on `bar`.
__device__ __forceinline__ void tc_copy_a(uint32_t bar, float* sAh, float* sAl, const float* src,
                                          int Kp) {
  const uint32_t bytes = (uint32_t)(128 * Kp * 4);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(2 * bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc_smem(sAh)),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc_smem(sAl)),
      "l"(src + 128 * Kp), "r"(bytes), "r"(bar)
      : "memory");
}

// The 3xTF32 MMAs of one phase into accumulator columns `col` (one thread), committed to `bar`.
__device__ __forceinline__ void tc_mma_phase(uint32_t tmem, uint32_t col, const float* sAh,
                                             const float* sAl, const float* sBh, const float* sBl,
                                             int NW, int Kp, uint32_t bar) {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t sbo = (uint32_t)(Kp / 4) * 128u;
  const uint32_t idesc = tc_idesc(NW);
  for (int t = 0; t < Kp / 8; ++t) {
    const uint32_t ko = (uint32_t)t * 256u;   // two core matrices of 128 B per k-step
    const uint64_t ah = tc_desc(tc_smem(sAh) + ko, 128, sbo);
    const uint64_t al = tc_desc(tc_smem(sAl) + ko, 128, sbo);
    const uint64_t bh = tc_desc(tc_smem(sBh) + ko, 128, sbo);
    const uint64_t bl = tc_desc(tc_smem(sBl) + ko, 128, sbo);
    tc_mma(tmem + col, ah, bh, idesc, t > 0 ? 1u : 0u);
    tc_mma(tmem + col, ah, bl, idesc, 1u);
    tc_mma(tmem + col, al, bh, idesc, 1u);
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// Shared memory of the synthesis for padded K `kmax`: one A stage and one B buffer (PIPE =
// false), or two A stages and separate B buffers for the P-type and the vector-type phases
// (PIPE = true), plus four mbarriers and the tensor-memory slot.
__host__ __device__ constexpr size_t tc_synth_smem(int kmax, bool pipe) {
  return pipe ? (4 * 128 * (size_t)kmax + 2 * (size_t)(kTcNP + kTcNV) * kmax) * sizeof(float) + 64
              : (2 * 128 * (size_t)kmax + 2 * (size_t)kTcNV * kmax) * sizeof(float) + 64;
}

// Six phases (s, w): parity class outer, table type inner, so that the B operand of w = 2
// (P/sin) is the one already staged for w = 1 (dP/dtheta): the same columns.
// PIPE = false: each phase copies its A tile, gathers its B operand, runs its MMAs and
// waits for them before the next phase starts.  PIPE = true: the A tile and B operand of
// phase p + 1 are staged (second A stage, the other B buffer) while the MMAs of phase p run;
// a buffer is refilled only after the MMAs that read it have completed.
// grid = (nm, ceil(Nd / 8), nmt); block = kTcThreads; dynamic smem tc_synth_smem(kmax, PIPE).
template <bool PIPE>
__global__ void __launch_bounds__(kTcThreads) k_synth_tc(DevGeom g, TcTables tt, const float2* __restrict__ SR,
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
  // shared memory: A (hi | lo, 128 x Kp each; two stages when PIPE), B (hi | lo; one buffer
  // of kTcNV columns, or kTcNP- and kTcNV-column buffers when PIPE), barriers
  // (pointers chosen with selects, not arrays, so that nothing lands in local memory)
  float *sA0, *sA1, *sBh0, *sBl0, *sBh1, *sBl1;
  uint64_t* bar;
  if constexpr (PIPE) {
    sA0 = reinterpret_cast<float*>(tc_raw);
    sA1 = sA0 + 2 * 128 * Kp;
    sBh0 = sA1 + 2 * 128 * Kp;
    sBl0 = sBh0 + kTcNP * Kp;
    sBh1 = sBl0 + kTcNP * Kp;
    sBl1 = sBh1 + kTcNV * Kp;
    bar = reinterpret_cast<uint64_t*>(sBl1 + kTcNV * Kp);   // copy[2], mma[2]
  } else {
    sA0 = sA1 = reinterpret_cast<float*>(tc_raw);
    sBh0 = sBh1 = sA0 + 2 * 128 * Kp;
    sBl0 = sBl1 = sBh0 + kTcNV * Kp;
    bar = reinterpret_cast<uint64_t*>(sBl0 + kTcNV * Kp);
  }
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 4);
  const uint32_t bc0 = tc_smem(&bar[0]), bc1 = tc_smem(&bar[1]);
  const uint32_t bm0 = tc_smem(&bar[2]), bm1 = tc_smem(&bar[3]);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(tslot)),
                 "r"(kTcAlloc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (uint32_t b : {bc0, bc1, bm0, bm1})
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  bool ok = true;
  auto tile = [&](int p) {
    return tt.tiles + tt.off[((a * 2 + p / 3) * 3 + p % 3) * tt.nmt + mt];
  };
  auto col_of = [&](int p) -> uint32_t {
    const int s = p / 3, w = p % 3;
    return (w == 0) ? s * kTcNP : 2 * kTcNP + ((w - 1) * 2 + s) * kTcNV;
  };
  if constexpr (!PIPE) {
    uint32_t ph = 0;
    for (int p = 0; p < 6 && ok; ++p) {
      const int s = p / 3, w = p % 3;
      // (1) tables: bulk copy of the hi and lo tiles; (2) B (w = 2 reuses the operand of w = 1)
      if (tid == 0) tc_copy_a(bc0, sA0, sA0 + 128 * Kp, tile(p), Kp);
      if (w != 2) tc_gather_b(SR, p0, nl, i0, Nd, Kp, s, w, sBh0, sBl0, tid);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      ok = tc_wait(bc0, ph);
      // (3) the MMAs, issued by one thread
      if (tid == 0 && ok)
        tc_mma_phase(tmem, col_of(p), sA0, sA0 + 128 * Kp, sBh0, sBl0, (w == 0) ? kTcNP : kTcNV,
                     Kp, bm0);
      // shared operands are reused by the next phase: wait for the MMAs
      const bool mma_ok = ok ? tc_wait(bm0, ph) : false;
      ok = ok && mma_ok;
      ph ^= 1u;
      __syncthreads();
    }
  } else {
    // bit b of `ph`: parity of the next wait on barrier b (copy 0, copy 1, MMA 0, MMA 1);
    // bit b of `pend`: an operation completing on barrier b not yet waited for (every exit
    // path waits for it)
    uint32_t ph = 0u, pend = 0u;
    auto bar_of = [&](int b) { return b == 0 ? bc0 : b == 1 ? bc1 : b == 2 ? bm0 : bm1; };
    auto wait_bar = [&](int b) {
      const bool done = tc_wait(bar_of(b), (ph >> b) & 1u);
      if (done) {
        ph ^= 1u << b;
        pend &= ~(1u << b);
      }
      return done;
    };
    if (tid == 0) tc_copy_a(bc0, sA0, sA0 + 128 * Kp, tile(0), Kp);
    pend |= 1u;
    tc_gather_b(SR, p0, nl, i0, Nd, Kp, 0, 0, sBh0, sBl0, tid);
    for (int p = 0; p < 6; ++p) {
      const int st = p & 1, w = p % 3;
      float* A = st ? sA1 : sA0;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();   // B of phase p stored by every thread
      const bool got = wait_bar(st);
      ok = __syncthreads_and(got ? 1 : 0) != 0;   // one decision for the whole CTA
      if (!ok) break;
      if (tid == 0)
        tc_mma_phase(tmem, col_of(p), A, A + 128 * Kp, w == 0 ? sBh0 : sBh1, w == 0 ? sBl0 : sBl1,
                     (w == 0) ? kTcNP : kTcNV, Kp, st ? bm1 : bm0);
      pend |= 1u << (2 + st);
      if (p + 1 < 6) {
        const int nst = st ^ 1;
        // phase p + 1 refills A stage nst, last read by the MMAs of phase p - 1, and (when
        // it gathers) the B buffer of its table type, last read by phase p - 1 or earlier
        if (pend & (1u << (2 + nst))) {
          const bool done = wait_bar(2 + nst);
          ok = __syncthreads_and(done ? 1 : 0) != 0;
          if (!ok) break;
        }
        float* An = nst ? sA1 : sA0;
        if (tid == 0) tc_copy_a(nst ? bc1 : bc0, An, An + 128 * Kp, tile(p + 1), Kp);
        pend |= 1u << nst;
        const int w1 = (p + 1) % 3;
        if (w1 != 2)
          tc_gather_b(SR, p0, nl, i0, Nd, Kp, (p + 1) / 3, w1, w1 == 0 ? sBh0 : sBh1,
                      w1 == 0 ? sBl0 : sBl1, tid);
      }
    }
    // the last MMAs (and, after a timeout, every copy and MMA still in flight: a wait that
    // gave up is retried once more, bounded, before the tensor memory is released)
    for (int b = 3; b >= 0; --b)
      if (pend & (1u << b)) {
        const bool done = wait_bar(b);
        ok = ok && done;
      }
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
  }
  if (!ok && tid == 0) atomicExch(tt.status, 7);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // (4) epilogue: warp w owns latitudes (TMEM lanes) 32 (w % 4) .. 32 (w % 4) + 31 of this
  // tile (its quadrant) for the radii of its warpgroup w / 4
  const int quad = warp & 3, grp = warp >> 2;
  const int t = mt * 128 + quad * 32 + lane;
  const bool live = ok && t < g.nlat2;
  const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
  const float mm = (float)m;
  const int K1 = g.K + 1, nlat = g.nlat;
  constexpr int kRadGrp = kTcRadii / (kTcThreads / 128);
  for (int rr = grp * kRadGrp; rr < (grp + 1) * kRadGrp; ++rr) {
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
