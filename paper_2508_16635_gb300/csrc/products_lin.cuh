// a3-a5 for the Jacobian actions of the mixed path: the inverse DFT in phi of the
// perturbation's nine fields, the linearised products with the base state's cached grid
// values, and the forward DFT of the four products (Sec. 3.1, Eqs. advec / curl terms,
// linearised about the wave as in Sec. 3.3), in FP32.  The same arithmetic as
// k_products<float, true> with the base state read from UG (k_base_grid), arranged for
// the small transforms of the wave workloads (K + 1 <= KM <= 16 wavenumbers, nphi <= 32
// longitudes):
//  - a warp per latitude, lane j = longitude j for the inverse DFT: its twiddles
//    cos / sin(2 pi a j / nphi) sit in registers for every latitude the warp takes, and
//    the coefficients of one wavenumber reach all lanes as 128-bit shared-memory
//    broadcasts (two fields each), so the inner step is one load for four FMAs;
//  - forward DFT: lane 2a (2a + 1) sums the real (imaginary) part of wavenumber a over the
//    longitudes: per longitude one 128-bit broadcast of its four products and one
//    conflict-free twiddle load for four FMAs;
//  - the coefficient gathers of the warp's next latitude are issued before the current
//    one is summed.
// grid = (Nd, ceil(nlat / (WPB LPW))), block = 32 WPB (WPB <= 8): warp w takes the
// latitudes th0 + w + WPB r, r < LPW (as k_products).
#pragma once

#include "kernels.cuh"

namespace rsc {

constexpr int kPlMaxWarps = 8;

template <int KM>
__global__ void __launch_bounds__(256) k_products_lin(DevGeom g, DevLegendre<float> T, float Ek,
                                                      const float2* __restrict__ FC,
                                                      float2* __restrict__ FA, int LPW,
                                                      const float* __restrict__ UG) {
  static_assert(2 * KM <= 32, "a lane per real / imaginary part of each wavenumber");
  constexpr int NG = (9 * KM + 31) / 32;          // coefficient gathers per lane
  __shared__ float4 cs[kPlMaxWarps][KM][5];         // [a][field pair]: (f 2u, f 2u + 1)
  __shared__ float4 ps[kPlMaxWarps][32];            // [j]: (F_r, F_th, F_ph, N)
  __shared__ float wt[32][32];                      // forward twiddles [j][2a + part]
  const int K1 = g.K + 1, nphi = g.nphi, nlat = g.nlat, Nd = g.Nd;
  const int WPB = blockDim.x >> 5;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x;
  const float inv = 1.0f / (float)nphi;
  // inverse twiddles of longitude j = lane
  float ci[KM], si[KM];
#pragma unroll
  for (int a = 0; a < KM; ++a) {
    const bool on = a < K1 && lane < nphi;
    ci[a] = on ? T.twc[a * nphi + lane] : 0.f;
    si[a] = on ? -T.tws[a * nphi + lane] : 0.f;
  }
  // forward twiddle columns, staged once per block: wt[j][2a + part] = cos / nphi (part 0)
  // or -sin / nphi (part 1) of wavenumber a at longitude j
  const int fa = lane >> 1, fpart = lane & 1;
  const bool fwd = fa < K1;
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int j = e >> 5, c = e & 31, a = c >> 1;
    float v = 0.f;
    if (a < K1 && j < nphi) v = (c & 1) ? -T.tws[a * nphi + j] * inv : T.twc[a * nphi + j] * inv;
    wt[j][c] = v;
  }
  // this lane's coefficient gathers: element e = lane + 32 u -> (field f, wavenumber a);
  // gslot = float2 slot in cs[w] (+ 1, negative for a = 0, 0 for none)
  int goff[NG], gslot[NG];
#pragma unroll
  for (int u = 0; u < NG; ++u) {
    const int e = lane + 32 * u;
    const int f = e / K1, a = e - f * K1;
    const bool on = f < 9;
    goff[u] = on ? ((f * Nd + i) * K1 + a) * nlat : 0;
    gslot[u] = on ? (a ? 1 : -1) * (a * 10 + f + 1) : 0;
  }
  float2* cw = reinterpret_cast<float2*>(&cs[w][0][0]);
  // the unused field slot 9 of every wavenumber (and wavenumbers K1..KM-1) stay zero
  for (int s = lane; s < KM * 10; s += 32) cw[s] = make_float2(0.f, 0.f);
  const int th0 = blockIdx.y * WPB * LPW;
  float2 pre[NG];
  {
    const int th = th0 + w;
#pragma unroll
    for (int u = 0; u < NG; ++u)
      pre[u] = (gslot[u] != 0 && th < nlat) ? FC[goff[u] + th] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int rep = 0; rep < LPW; ++rep) {
    const int th = th0 + w + WPB * rep;
    if (th >= nlat) break;
    __syncwarp();
#pragma unroll
    for (int u = 0; u < NG; ++u) {
      if (gslot[u] > 0) {
        cw[gslot[u] - 1] = make_float2(2.f * pre[u].x, 2.f * pre[u].y);
      } else if (gslot[u] < 0) {
        cw[-gslot[u] - 1] = make_float2(pre[u].x, 0.f);   // a = 0 enters with its real part
      }
    }
    __syncwarp();
    // the next latitude's gathers, in flight while this one is summed
    const int thn = th + WPB;
    if (rep + 1 < LPW) {
#pragma unroll
      for (int u = 0; u < NG; ++u)
        pre[u] = (gslot[u] != 0 && thn < nlat) ? FC[goff[u] + thn] : make_float2(0.f, 0.f);
    }
    // base state at (th, j)
    float U[9];
#pragma unroll
    for (int f = 0; f < 9; ++f)
      U[f] = lane < nphi ? UG[(((long)f * Nd + i) * nlat + th) * nphi + lane] : 0.f;
    // inverse DFT: u_f(phi_j) = sum_a Re(c_fa e^{i a phi_j}) (factor 2 for a > 0 folded in)
    float u[10];
#pragma unroll
    for (int f = 0; f < 10; ++f) u[f] = 0.f;
#pragma unroll
    for (int a = 0; a < KM; ++a) {
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const float4 c = cs[w][a][q];
        u[2 * q] = fmaf(c.x, ci[a], u[2 * q]);
        u[2 * q] = fmaf(c.y, si[a], u[2 * q]);
        u[2 * q + 1] = fmaf(c.z, ci[a], u[2 * q + 1]);
        u[2 * q + 1] = fmaf(c.w, si[a], u[2 * q + 1]);
      }
    }
    // linearised products (fields: 0 u_r, 1 u_th, 2 u_ph, 3-5 omega, 6-8 grad T)
    const float Fr = Ek * ((U[1] * u[5] - U[2] * u[4]) + (u[1] * U[5] - u[2] * U[4]));
    const float Ft = Ek * ((U[2] * u[3] - U[0] * u[5]) + (u[2] * U[3] - u[0] * U[5]));
    const float Fp = Ek * ((U[0] * u[4] - U[1] * u[3]) + (u[0] * U[4] - u[1] * U[3]));
    const float N = U[0] * u[6] + U[1] * u[7] + U[2] * u[8] + u[0] * U[6] + u[1] * U[7] + u[2] * U[8];
    ps[w][lane] = make_float4(Fr, Ft, Fp, N);
    __syncwarp();
    // forward DFT of the four products
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j < nphi) {
        const float4 p = ps[w][j];
        const float c = wt[j][lane];
        acc[0] = fmaf(p.x, c, acc[0]);
        acc[1] = fmaf(p.y, c, acc[1]);
        acc[2] = fmaf(p.z, c, acc[2]);
        acc[3] = fmaf(p.w, c, acc[3]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float im = __shfl_down_sync(0xffffffffu, acc[q], 1);
      if (fwd && fpart == 0) FA[(((long)q * Nd + i) * K1 + fa) * nlat + th] = make_float2(acc[q], im);
    }
  }
}

}  // namespace rsc
