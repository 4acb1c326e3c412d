// The radial stages of the mixed path in FP32, as persistent kernels that hold their
// Chebyshev tables in shared memory:
//  - k_radial_f32 (a1, steps and Jacobian actions): the eight radial fields of each pair at
//    the de-aliased radii (Sec. 3.1, the poloidal / toroidal representation), as
//    k_radial<float>;
//  - k_rhs_lin (a7, Jacobian actions): per pair the radial projection of the analysed
//    products, the curl / double-curl rows, the mass products of the direction and (with
//    the drift unknown, Sec. 3.4) of the base state, and the boundary rows (Sec. 3.1;
//    Eqs. impcor_e_final / impcor_f_final without the implicit Coriolis blocks, which the
//    chain solve applies), as k_rhs<float> in mode 1, the result stored in FP64.
// Every pair applies the same tables (N_r x N_d and N_r x N_r, 80-100 KB at N_r = 64), so a
// grid of one or two blocks per SM stages them in shared memory once and loops over the
// pairs p = blockIdx.x, blockIdx.x + gridDim.x, ...; the next pair's inputs are loaded into
// registers while the current one is summed.  Four lanes share each output radius: lane s
// sums the table rows k = s, s + 4, ... and two butterfly steps combine the partial sums.
// Table rows are padded to a stride of 8 (mod 32) floats, so the four row offsets of a warp
// fall in distinct banks; the tables arrive by cp.async, all copies in flight together.
#pragma once

#include "kernels.cuh"

namespace rsc {

// Row stride (floats) of a staged table with n columns: >= n, 8 (mod 32).
__host__ __device__ __forceinline__ int rr_stride(int n) { return ((n + 23) / 32) * 32 + 8; }

__device__ __forceinline__ float rl_sum4(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

// Stage a rows x cols row-major table (contiguous in global memory) into shared memory with
// row stride ds: 16-byte cp.async copies, all in flight together, when rows, stride and
// source allow it, else plain loads.  The caller waits with rr_stage_wait().
__device__ __forceinline__ void rr_stage(float* dst, int ds, const float* __restrict__ src,
                                         int rows, int cols) {
  if ((cols & 3) == 0 && (ds & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const int q = cols >> 2;
    for (int c = threadIdx.x; c < rows * q; c += blockDim.x) {
      const int r = c / q, u = c - r * q;
      const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + r * ds + 4 * u);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src + (long)r * cols + 4 * u)
                   : "memory");
    }
  } else {
    for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
      const int r = idx / cols, c = idx - r * cols;
      dst[r * ds + c] = src[idx];
    }
  }
}
__device__ __forceinline__ void rr_stage_wait() {
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
}

// Shared memory (bytes) of the two kernels.
__host__ __forceinline__ size_t radial_f32_smem(int Nr, int Nd) {
  return (3 * (size_t)Nr * rr_stride(Nd)) * sizeof(float) + 3 * (size_t)Nr * sizeof(float2);
}
__host__ __forceinline__ size_t rhs_lin_smem(int Nr, int Nd) {
  return (2 * (size_t)Nd + 2 * (size_t)Nr) * rr_stride(Nr) * sizeof(float) +
         (4 * (size_t)Nd + 6 * (size_t)Nr) * sizeof(float2);
}

// grid <= P blocks, block = 4 * round8(Nd) threads (>= 3 Nr), dynamic shared memory
// radial_f32_smem.  SR[(p * Nd + i) * 8 + q], q = u_r, S_u, T_u, omega_r, S_w, T_w, d_r T, S_T.
// NR_, ND_ > 0 fix N_r, N_d at compile time (both multiples of 4: the four-lane loops unroll
// fully); 0, 0 reads them from g.
template <int NR_, int ND_>
__global__ void __launch_bounds__(1024) k_radial_f32(DevGeom g, const double2* __restrict__ x,
                                                     float2* __restrict__ SR) {
  extern __shared__ __align__(16) float rr_sh[];
  constexpr bool FIX = NR_ > 0;
  static_assert(!FIX || (NR_ % 4 == 0 && ND_ % 4 == 0), "fixed sizes are multiples of 4");
  const int Nr = FIX ? NR_ : g.Nr, Nd = FIX ? ND_ : g.Nd, P = g.P;
  const int SI = rr_stride(Nd);
  float* E0 = rr_sh;                 // [k][i], stride SI
  float* E1 = E0 + Nr * SI;
  float* E2 = E1 + Nr * SI;
  float2* xs = reinterpret_cast<float2*>(E2 + Nr * SI);   // [3][Nr]
  rr_stage(E0, SI, g.EdT0f, Nr, Nd);
  rr_stage(E1, SI, g.EdT1f, Nr, Nd);
  rr_stage(E2, SI, g.EdT2f, Nr, Nd);
  const int s = threadIdx.x & 3;
  const int ir_ = threadIdx.x >> 2;
  const int i = ir_ < Nd ? ir_ : Nd - 1;   // lanes past the last radius repeat it, store nothing
  const float ir = 1.0f / g.rdf[i], ir2 = ir * ir;
  // this thread's share of the next pair's coefficients
  const int t = threadIdx.x;
  const bool ld = t < 3 * Nr;
  const int tf = ld ? t / Nr : 0, tk = ld ? t - tf * Nr : 0;
  double2 nx = make_double2(0, 0);
  if (ld && blockIdx.x < P) nx = x[((long)tf * P + blockIdx.x) * Nr + tk];
  rr_stage_wait();
  for (int p = blockIdx.x; p < P; p += gridDim.x) {
    __syncthreads();   // the previous pair's coefficients are read
    if (ld) xs[t] = make_float2((float)nx.x, (float)nx.y);
    __syncthreads();
    if (ld && p + gridDim.x < P) nx = x[((long)tf * P + p + gridDim.x) * Nr + tk];
    float fvx = 0, fvy = 0, f1x = 0, f1y = 0, f2x = 0, f2y = 0, evx = 0, evy = 0, e1x = 0, e1y = 0;
    float Tvx = 0, Tvy = 0, T1x = 0, T1y = 0;
    auto step = [&](int k) {
      const float a0 = E0[k * SI + i], a1 = E1[k * SI + i], a2 = E2[k * SI + i];
      const float2 e = xs[k], f = xs[Nr + k], T = xs[2 * Nr + k];
      fvx += a0 * f.x; fvy += a0 * f.y;
      f1x += a1 * f.x; f1y += a1 * f.y;
      f2x += a2 * f.x; f2y += a2 * f.y;
      evx += a0 * e.x; evy += a0 * e.y;
      e1x += a1 * e.x; e1y += a1 * e.y;
      Tvx += a0 * T.x; Tvy += a0 * T.y;
      T1x += a1 * T.x; T1y += a1 * T.y;
    };
    if constexpr (FIX) {
#pragma unroll
      for (int u = 0; u < NR_ / 4; ++u) step(4 * u + s);
    } else {
      for (int k = s; k < Nr; k += 4) step(k);
    }
    fvx = rl_sum4(fvx); fvy = rl_sum4(fvy); f1x = rl_sum4(f1x); f1y = rl_sum4(f1y);
    f2x = rl_sum4(f2x); f2y = rl_sum4(f2y); evx = rl_sum4(evx); evy = rl_sum4(evy);
    e1x = rl_sum4(e1x); e1y = rl_sum4(e1y); Tvx = rl_sum4(Tvx); Tvy = rl_sum4(Tvy);
    T1x = rl_sum4(T1x); T1y = rl_sum4(T1y);
    if (ir_ < Nd) {
      const int l = g.pair_l[p];
      const float lam = (float)(l * (l + 1));
      float2* o = SR + ((long)p * Nd + i) * 8 + 2 * s;
      if (s == 0) {
        o[0] = make_float2(lam * fvx * ir2, lam * fvy * ir2);                             // u_r
        o[1] = make_float2(f1x * ir, f1y * ir);                                           // S_u
      } else if (s == 1) {
        o[0] = make_float2(evx * ir, evy * ir);                                           // T_u
        o[1] = make_float2(lam * evx * ir2, lam * evy * ir2);                             // omega_r
      } else if (s == 2) {
        o[0] = make_float2(e1x * ir, e1y * ir);                                           // S_w
        o[1] = make_float2(-(f2x - lam * fvx * ir2) * ir, -(f2y - lam * fvy * ir2) * ir); // T_w
      } else {
        o[0] = make_float2(T1x, T1y);                                                     // d_r T
        o[1] = make_float2(Tvx * ir, Tvy * ir);                                           // S_T
      }
    }
  }
}

// grid <= P blocks, block = 4 * round8(Nr) threads (>= 3 Nr, >= 2 Nd, <= 512), dynamic shared memory
// rhs_lin_smem.  rhs[(f * P + p) * Nr + j], f = e, f, T.
// NR_, ND_ as for k_radial_f32.
template <int NR_, int ND_>
__global__ void __launch_bounds__(512) k_rhs_lin(DevGeom g, RhsParams rp,
                                                  const float2* __restrict__ AR,
                                                  const double2* __restrict__ x,
                                                  const double2* __restrict__ U,
                                                  const double* __restrict__ u_orig,
                                                  double2* __restrict__ rhs) {
  extern __shared__ __align__(16) float rl_sh[];
  constexpr bool FIX = NR_ > 0;
  static_assert(!FIX || (NR_ % 4 == 0 && ND_ % 4 == 0), "fixed sizes are multiples of 4");
  const int Nr = FIX ? NR_ : g.Nr, Nd = FIX ? ND_ : g.Nd, P = g.P;
  const int SJ = rr_stride(Nr);
  const bool has_c = rp.J >= 0;
  float* W0 = rl_sh;                 // [i][j] projection onto T_j's row j
  float* W1 = W0 + Nd * SJ;          // [i][j] the same with the radial derivative, times r_i
  float* C0 = W1 + Nd * SJ;          // [k][j] T_k(r_j)
  float* C2 = C0 + Nr * SJ;          // [k][j] T_k''(r_j)
  float2* ar = reinterpret_cast<float2*>(C2 + Nr * SJ);   // [Nd][4]: q, s, t, n
  float2* xf = ar + 4 * Nd;          // [3][Nr]: e, f, T of the direction
  float2* uf = xf + 3 * Nr;          // [3][Nr]: of the base state (drift term)
  rr_stage(W0, SJ, g.R0Tf, Nd, Nr);
  rr_stage(W1, SJ, g.R1Tf, Nd, Nr);
  rr_stage(C0, SJ, g.EcT0f, Nr, Nr);
  rr_stage(C2, SJ, g.EcT2f, Nr, Nr);
  const int s = threadIdx.x & 3;
  const int jr = threadIdx.x >> 2;
  const int j = jr < Nr ? jr : Nr - 1;   // lanes past the last row repeat it and store nothing
  const float ir = 1.0f / (float)g.rc[j], ir2 = ir * ir;
  const float Ek = (float)rp.Ek, Ra = (float)rp.Ra, ro = (float)rp.r_out;
  const float fr = (float)rp.inv_dt;
  const float cdrift = has_c ? (float)u_orig[rp.J] : 0.f;
  // this thread's share of the next pair's inputs: AR elements t and t + blockDim.x, the
  // coefficients of x and U at t
  const int t = threadIdx.x, nt = blockDim.x;
  const bool la0 = t < 4 * Nd, la1 = t + nt < 4 * Nd, lx = t < 3 * Nr;
  const int tf = lx ? t / Nr : 0, tk = lx ? t - tf * Nr : 0;
  float2 na0 = make_float2(0, 0), na1 = make_float2(0, 0);
  double2 nx = make_double2(0, 0), nu = make_double2(0, 0);
  auto fetch = [&](int q) {
    if (la0) na0 = AR[(long)q * Nd * 4 + t];
    if (la1) na1 = AR[(long)q * Nd * 4 + t + nt];
    if (lx) {
      const long off = ((long)tf * P + q) * Nr + tk;
      nx = x[off];
      if (has_c) nu = U[off];
    }
  };
  if (blockIdx.x < P) fetch(blockIdx.x);
  rr_stage_wait();
  for (int idx = threadIdx.x; idx < Nd * Nr; idx += blockDim.x) {
    const int i = idx / Nr, j = idx - i * Nr;
    W1[i * SJ + j] *= g.rdf[i];
  }
  for (int p = blockIdx.x; p < P; p += gridDim.x) {
    __syncthreads();   // the previous pair's inputs are read; W1 is scaled
    if (la0) ar[t] = na0;
    if (la1) ar[t + nt] = na1;
    if (lx) {
      xf[t] = make_float2((float)nx.x, (float)nx.y);
      uf[t] = make_float2((float)nu.x, (float)nu.y);
    }
    __syncthreads();
    if (p + gridDim.x < P) fetch(p + gridDim.x);
    // radial projection of the analysed products
    float Qx = 0, Qy = 0, Tx = 0, Ty = 0, Nx = 0, Ny = 0, Sx = 0, Sy = 0;
    auto pstep = [&](int i) {
      const float w0 = W0[i * SJ + j], w1 = W1[i * SJ + j];
      const float2 q = ar[i * 4 + 0], sv = ar[i * 4 + 1], tt = ar[i * 4 + 2], n = ar[i * 4 + 3];
      Qx += w0 * q.x; Qy += w0 * q.y;
      Tx += w0 * tt.x; Ty += w0 * tt.y;
      Nx += w0 * n.x; Ny += w0 * n.y;
      Sx += w1 * sv.x; Sy += w1 * sv.y;
    };
    if constexpr (FIX) {
#pragma unroll
      for (int u = 0; u < ND_ / 4; ++u) pstep(4 * u + s);
    } else {
      for (int i = s; i < Nd; i += 4) pstep(i);
    }
    // mass products: e0 = sum_k T_k(r_j) e_k, f0, f2 = sum_k T_k''(r_j) f_k, t0
    auto mass = [&](const float2* vf, float* o) {
      float e0x = 0, e0y = 0, f0x = 0, f0y = 0, f2x = 0, f2y = 0, t0x = 0, t0y = 0;
      auto mstep = [&](int k) {
        const float c0 = C0[k * SJ + j], c2 = C2[k * SJ + j];
        const float2 e = vf[k], f = vf[Nr + k], T = vf[2 * Nr + k];
        e0x += c0 * e.x; e0y += c0 * e.y;
        f0x += c0 * f.x; f0y += c0 * f.y;
        f2x += c2 * f.x; f2y += c2 * f.y;
        t0x += c0 * T.x; t0y += c0 * T.y;
      };
      if constexpr (FIX) {
#pragma unroll
        for (int u = 0; u < NR_ / 4; ++u) mstep(4 * u + s);
      } else {
        for (int k = s; k < Nr; k += 4) mstep(k);
      }
      o[0] = rl_sum4(e0x); o[1] = rl_sum4(e0y); o[2] = rl_sum4(f0x); o[3] = rl_sum4(f0y);
      o[4] = rl_sum4(f2x); o[5] = rl_sum4(f2y); o[6] = rl_sum4(t0x); o[7] = rl_sum4(t0y);
    };
    float mx[8], mu[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    mass(xf, mx);
    if (has_c) mass(uf, mu);
    Qx = rl_sum4(Qx); Qy = rl_sum4(Qy); Tx = rl_sum4(Tx); Ty = rl_sum4(Ty);
    Nx = rl_sum4(Nx); Ny = rl_sum4(Ny); Sx = rl_sum4(Sx); Sy = rl_sum4(Sy);
    if (jr >= Nr || s >= 3) continue;
    // lane s of the row forms and stores field s (0 e, 1 f, 2 T)
    const int l = g.pair_l[p], m = g.pair_m[p];
    const float lam = (float)(l * (l + 1));
    const float ce = lam * Ek * ir2, cl = lam * ir2;
    const float fi = (float)(rp.C * m);            // (1/dt + i C m)
    const float cmv = cdrift * (float)m;           // c i m M U
    float2 M, Nt, Mu;
    if (s == 0) {
      M = make_float2(ce * mx[0], ce * mx[1]);
      Mu = make_float2(ce * mu[0], ce * mu[1]);
      Nt = make_float2(lam * ir * Tx, lam * ir * Ty);
    } else if (s == 1) {
      M = make_float2(-ce * (mx[4] - cl * mx[2]), -ce * (mx[5] - cl * mx[3]));
      Mu = make_float2(-ce * (mu[4] - cl * mu[2]), -ce * (mu[5] - cl * mu[3]));
      const float cb = lam * Ra * ir / ro;
      Nt = make_float2(cl * (Qx - Sx) + cb * mx[6], cl * (Qy - Sy) + cb * mx[7]);
    } else {
      M = make_float2(mx[6], mx[7]);
      Mu = make_float2(mu[6], mu[7]);
      Nt = make_float2(-Nx, -Ny);
    }
    float2 o = make_float2(fr * M.x - fi * M.y + Nt.x, fr * M.y + fi * M.x + Nt.y);
    o.x -= cmv * Mu.y;
    o.y += cmv * Mu.x;
    // boundary rows (Sec. 3.1) and the identity rows of e_00, f_00
    const bool wall = j == 0 || j == Nr - 1;
    if (s != 1 && wall) o = make_float2(0, 0);
    if (s == 1 && (wall || j == 1 || j == Nr - 2)) o = make_float2(0, 0);
    if (s != 2 && l == 0) o = make_float2(0, 0);
    if (m == 0) o.y = 0;
    rhs[((long)s * P + p) * Nr + j] = make_double2(o.x, o.y);
  }
}

}  // namespace rsc
