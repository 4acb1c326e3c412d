// Device kernels of one IMEX step / Jacobian action (Sec. 3.1-3.4).
//
// Data flow of a step (rows of the hot path):
//   k_radial    Chebyshev coefficients -> spectral values on the de-aliased
//               radii (u_r, S_u, T_u, omega_r, S_w, T_w, d_r T, T/r)   [a1]
//   k_synth     per (m, r): Legendre sums over l, parity split     [a2]
//   k_products  per (r, theta tile): inverse DFT in phi, U x omega and
//               U.grad T (or their linearisation), forward DFT     [a3-a5]
//   k_analysis  per (m, r): Gauss-weighted Legendre projection      [a6]
//   k_rhs       per (l, m): radial projection, curl / double curl,
//               mass, drift and boundary rows (FP64)               [a7]
//   k_block_gemv, k_chain_half, k_chain_out, k_temp_solve: block-tridiagonal
//               Coriolis chains and per-l temperature solves (FP64) [a8]
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <climits>

namespace rsc {

template <typename R> struct C2;
template <> struct C2<double> { using T = double2; };
template <> struct C2<float> { using T = float2; };

template <typename R>
__device__ __forceinline__ typename C2<R>::T mk(R x, R y) {
  typename C2<R>::T v;
  v.x = x;
  v.y = y;
  return v;
}

// Device view of the tables.
template <typename R>
struct DevLegendre {
  const R* P;      // synthesis layout [off_m + q * nlat2 + t]
  const R* dP;
  const R* Ps;
  const R* Pw;     // analysis layout [off_m + t * nl + q]
  const R* dPw;
  const R* Psw;
  const R* twc;    // cos(2 pi a j / nphi) [a][j]
  const R* tws;    // sin(2 pi a j / nphi) [a][j]
};

struct DevGeom {
  int L, Ms, Nr, Nd, nlat, nlat2, nphi, nm, K, P;
  double r_in, r_out;
  const int* m_of;      // [nm]
  const int* pstart;    // [nm + 1]
  const long* leg_off;  // [nm + 1]
  const int* pair_l;    // [P]
  const int* pair_m;    // [P]
  const double* rc;     // [Nr]
  const double* rd;     // [Nd]
  const double* EcT0;   // [k][j] T_k(r_j)
  const double* EcT2;   // [k][j] d2 T_k / dr2 (r_j)
  const double* EcT1;   // [k][j] d T_k / dr (r_j)
  const double* EdT0;   // [k][i] at the de-aliased radii
  const double* EdT1;
  const double* EdT2;
  const double* R0T;    // [i][j]
  const double* R1T;    // [i][j]
  // FP32 copies for the transforms of the mixed path
  const float* EdT0f;
  const float* EdT1f;
  const float* EdT2f;
  const float* R0Tf;
  const float* R1Tf;
  const float* rdf;
  const float* EcT0f;
  const float* EcT2f;
};

template <typename R> struct Tab;
template <> struct Tab<double> {
  static __device__ __forceinline__ const double* Ed0(const DevGeom& g) { return g.EdT0; }
  static __device__ __forceinline__ const double* Ed1(const DevGeom& g) { return g.EdT1; }
  static __device__ __forceinline__ const double* Ed2(const DevGeom& g) { return g.EdT2; }
  static __device__ __forceinline__ const double* R0(const DevGeom& g) { return g.R0T; }
  static __device__ __forceinline__ const double* R1(const DevGeom& g) { return g.R1T; }
  static __device__ __forceinline__ const double* rd(const DevGeom& g) { return g.rd; }
};
template <> struct Tab<float> {
  static __device__ __forceinline__ const float* Ed0(const DevGeom& g) { return g.EdT0f; }
  static __device__ __forceinline__ const float* Ed1(const DevGeom& g) { return g.EdT1f; }
  static __device__ __forceinline__ const float* Ed2(const DevGeom& g) { return g.EdT2f; }
  static __device__ __forceinline__ const float* R0(const DevGeom& g) { return g.R0Tf; }
  static __device__ __forceinline__ const float* R1(const DevGeom& g) { return g.R1Tf; }
  static __device__ __forceinline__ const float* rd(const DevGeom& g) { return g.rdf; }
};

// ---------------------------------------------------------------------------
// a1: radial evaluation.  grid = P, block >= Nd.
// SR[(p * Nd + i) * 8 + q], q = ur, Su, Tu, wr, Sw, Tw, dT, ST.
template <typename R>
__global__ void k_radial(DevGeom g, const double2* __restrict__ x,
                         typename C2<R>::T* __restrict__ SR) {
  using V = typename C2<R>::T;
  extern __shared__ unsigned char sh_raw[];
  V* sc = reinterpret_cast<V*>(sh_raw);  // [3][Nr] coefficients in precision R
  const int p = blockIdx.x;
  const int Nr = g.Nr, Nd = g.Nd;
  for (int idx = threadIdx.x; idx < 3 * Nr; idx += blockDim.x) {
    const int f = idx / Nr, k = idx % Nr;
    const double2 v = x[((long)f * g.P + p) * Nr + k];
    sc[idx] = mk<R>((R)v.x, (R)v.y);
  }
  __syncthreads();
  const int i = threadIdx.x;
  if (i >= Nd) return;
  const R* E0 = Tab<R>::Ed0(g);
  const R* E1 = Tab<R>::Ed1(g);
  const R* E2 = Tab<R>::Ed2(g);
  R fvx = 0, fvy = 0, f1x = 0, f1y = 0, f2x = 0, f2y = 0, evx = 0, evy = 0, e1x = 0, e1y = 0;
  R Tvx = 0, Tvy = 0, T1x = 0, T1y = 0;
  for (int k = 0; k < Nr; ++k) {
    const R a0 = E0[k * Nd + i], a1 = E1[k * Nd + i], a2 = E2[k * Nd + i];
    const V e = sc[k], f = sc[Nr + k], T = sc[2 * Nr + k];
    fvx += a0 * f.x; fvy += a0 * f.y;
    f1x += a1 * f.x; f1y += a1 * f.y;
    f2x += a2 * f.x; f2y += a2 * f.y;
    evx += a0 * e.x; evy += a0 * e.y;
    e1x += a1 * e.x; e1y += a1 * e.y;
    Tvx += a0 * T.x; Tvy += a0 * T.y;
    T1x += a1 * T.x; T1y += a1 * T.y;
  }
  const int l = g.pair_l[p];
  const R lam = (R)(l * (l + 1.0));
  const R ir = (R)1 / Tab<R>::rd(g)[i], ir2 = ir * ir;
  V* o = SR + ((long)p * Nd + i) * 8;
  o[0] = mk<R>(lam * fvx * ir2, lam * fvy * ir2);                                // u_r
  o[1] = mk<R>(f1x * ir, f1y * ir);                                              // S_u
  o[2] = mk<R>(evx * ir, evy * ir);                                              // T_u
  o[3] = mk<R>(lam * evx * ir2, lam * evy * ir2);                                // omega_r
  o[4] = mk<R>(e1x * ir, e1y * ir);                                              // S_w
  o[5] = mk<R>(-(f2x - lam * fvx * ir2) * ir, -(f2y - lam * fvy * ir2) * ir);    // T_w
  o[6] = mk<R>(T1x, T1y);                                                        // d_r T
  o[7] = mk<R>(Tvx * ir, Tvy * ir);                                              // S_T
}

// ---------------------------------------------------------------------------
// a2: Legendre synthesis.  grid = (nm, ceil(Nd / blockDim.y)), block =
// (>= nlat2, multiple of 32) x RT radii; the RT threads of one latitude read
// the same table entries, so the table traffic is served from L1.
// FC[((fld * Nd + i) * (K+1) + a) * nlat + th], fld = ur, ut, up, wr, wt, wp, Tr, Tt, Tp.
template <typename R>
__global__ void k_synth(DevGeom g, DevLegendre<R> T, const typename C2<R>::T* __restrict__ SR,
                        typename C2<R>::T* __restrict__ FC) {
  using V = typename C2<R>::T;
  extern __shared__ unsigned char sh_raw[];
  const int RT = blockDim.y;
  V* sh = reinterpret_cast<V*>(sh_raw);  // [RT][nl][8]
  const int a = blockIdx.x;
  const int m = g.m_of[a];
  const int p0 = g.pstart[a];
  const int nl = g.L - m + 1;
  const int Nd = g.Nd;
  const int i0 = blockIdx.y * RT;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int idx = tid; idx < RT * nl * 8; idx += blockDim.x * RT) {
    const int rr = idx / (nl * 8);
    const int rem = idx - rr * nl * 8;
    const int q = rem >> 3, c = rem & 7;
    const int i = i0 + rr;
    sh[idx] = (i < Nd) ? SR[((long)(p0 + q) * Nd + i) * 8 + c] : mk<R>(0, 0);
  }
  const int t = threadIdx.x;
  const int i = i0 + threadIdx.y;
  const bool live = t < g.nlat2 && i < Nd;
  const V* shr = sh + threadIdx.y * nl * 8;
  const long off = g.leg_off[a];
  const int n2 = g.nlat2;
  // table chunks of QC degrees staged in shared memory by the whole block
  constexpr int QC = 16;
  R* tab = reinterpret_cast<R*>(sh + RT * nl * 8);   // [QC][3][n2]
  R sPr[2][3], sPi[2][3];   // P-sums of ur, wr, dT
  R dRr[2][5], dRi[2][5];   // dP-sums of Su, Tu, Sw, Tw, ST
  R qRr[2][5], qRi[2][5];   // Ps-sums of Su, Tu, Sw, Tw, ST
#pragma unroll
  for (int s = 0; s < 2; ++s) {
#pragma unroll
    for (int c = 0; c < 3; ++c) sPr[s][c] = sPi[s][c] = 0;
#pragma unroll
    for (int c = 0; c < 5; ++c) dRr[s][c] = dRi[s][c] = qRr[s][c] = qRi[s][c] = 0;
  }
  const int nthr = blockDim.x * RT;
  for (int qc = 0; qc < nl; qc += QC) {
    const int nq = min(QC, nl - qc);
    __syncthreads();
    for (int idx = tid; idx < nq * 3 * n2; idx += nthr) {
      const int q = idx / (3 * n2);
      const int rem = idx - q * 3 * n2;
      const int w = rem / n2, tt = rem - w * n2;
      const R* src = (w == 0) ? T.P : (w == 1) ? T.dP : T.Ps;
      tab[idx] = src[off + (long)(qc + q) * n2 + tt];
    }
    __syncthreads();
    if (live) {
      for (int q0 = 0; q0 < nq; q0 += 2) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int q = q0 + s;   // qc is even, so the parity of q is that of l - m
          if (q < nq) {
            const R pv = tab[(q * 3 + 0) * n2 + t];
            const R dv = tab[(q * 3 + 1) * n2 + t];
            const R sv = tab[(q * 3 + 2) * n2 + t];
            const V* c = shr + (qc + q) * 8;
            sPr[s][0] += pv * c[0].x; sPi[s][0] += pv * c[0].y;
            sPr[s][1] += pv * c[3].x; sPi[s][1] += pv * c[3].y;
            sPr[s][2] += pv * c[6].x; sPi[s][2] += pv * c[6].y;
            const int vi[5] = {1, 2, 4, 5, 7};
#pragma unroll
            for (int u = 0; u < 5; ++u) {
              dRr[s][u] += dv * c[vi[u]].x; dRi[s][u] += dv * c[vi[u]].y;
              qRr[s][u] += sv * c[vi[u]].x; qRi[s][u] += sv * c[vi[u]].y;
            }
          }
        }
      }
    }
  }
  if (!live) return;
  const R mm = (R)m;
  const int K1 = g.K + 1, nlat = g.nlat;
#pragma unroll
  for (int hemi = 0; hemi < 2; ++hemi) {
    // north: E + O for P-type and dP-type; south: E - O (P-type), -E + O (dP-type)
    const R sP = hemi ? (R)-1 : (R)1;
    const R sD = hemi ? (R)-1 : (R)1;
    const int th = hemi ? (nlat - 1 - t) : t;
    R Pr[3], Pi[3], Dr[5], Di[5], Sr[5], Si[5];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Pr[c] = sPr[0][c] + sP * sPr[1][c];
      Pi[c] = sPi[0][c] + sP * sPi[1][c];
    }
#pragma unroll
    for (int u = 0; u < 5; ++u) {
      Dr[u] = sD * dRr[0][u] + dRr[1][u];
      Di[u] = sD * dRi[0][u] + dRi[1][u];
      Sr[u] = qRr[0][u] + sP * qRr[1][u];
      Si[u] = qRi[0][u] + sP * qRi[1][u];
    }
    // i m X = (-m X.y, m X.x)
    V out[9];
    out[0] = mk<R>(Pr[0], Pi[0]);                                        // u_r
    out[1] = mk<R>(Dr[0] - mm * Si[1], Di[0] + mm * Sr[1]);               // u_th = dS_u + i m T_u/s
    out[2] = mk<R>(-mm * Si[0] - Dr[1], mm * Sr[0] - Di[1]);              // u_ph = i m S_u/s - dT_u
    out[3] = mk<R>(Pr[1], Pi[1]);                                        // omega_r
    out[4] = mk<R>(Dr[2] - mm * Si[3], Di[2] + mm * Sr[3]);               // omega_th
    out[5] = mk<R>(-mm * Si[2] - Dr[3], mm * Sr[2] - Di[3]);              // omega_ph
    out[6] = mk<R>(Pr[2], Pi[2]);                                        // d_r T
    out[7] = mk<R>(Dr[4], Di[4]);                                        // (1/r) d_th T
    out[8] = mk<R>(-mm * Si[4], mm * Sr[4]);                              // (1/(r s)) d_ph T
#pragma unroll
    for (int fld = 0; fld < 9; ++fld)
      FC[(((long)fld * Nd + i) * K1 + a) * nlat + th] = out[fld];
  }
}

// ---------------------------------------------------------------------------
// a3-a5: inverse DFT, products, forward DFT.  grid = (Nd, ceil(nlat / (WPB LPW))),
// block = 32 x WPB: warp w handles latitudes th0 + w + WPB r, r < LPW.  Inverse DFT: lane j
// sums the (K+1) coefficients of each field at its longitudes (coefficients
// are warp broadcasts, twiddles [a][j] are bank-conflict free).  Forward DFT:
// lane a sums its wavenumber over the nphi longitudes (twiddles stored [j][a]).
// LIN = false: F = Ek U x omega, N = U.grad T from FC.
// LIN = true : F = Ek (U x omega_u + u x omega_U), N = U.grad tau + u.grad T
//              with U from FCU and u from FC; when UG is given, U's grid values are read
//              from it (k_base_grid, once per base state) instead of transformed again.
template <typename R, bool LIN>
__global__ void k_products(DevGeom g, DevLegendre<R> T, R Ek,
                           const typename C2<R>::T* __restrict__ FC,
                           const typename C2<R>::T* __restrict__ FCU,
                           typename C2<R>::T* __restrict__ FA, int LPW,
                           const R* __restrict__ UG) {
  using V = typename C2<R>::T;
  constexpr int NF = LIN ? 18 : 9;
  extern __shared__ unsigned char sh_raw[];
  const int K1 = g.K + 1, nphi = g.nphi, nlat = g.nlat, Nd = g.Nd;
  const int WPB = blockDim.x >> 5;
  V* coef = reinterpret_cast<V*>(sh_raw);                 // [WPB][NF][K1]
  R* twc = reinterpret_cast<R*>(coef + WPB * NF * K1);    // [K1][nphi] (x2 for a > 0)
  R* tws = twc + K1 * nphi;
  R* twcT = tws + K1 * nphi;                              // [nphi][K1] / nphi
  R* twsT = twcT + K1 * nphi;
  R* prod = twsT + K1 * nphi;                             // [WPB][4][nphi + 1]
  const int i = blockIdx.x;
  const R inv = (R)1 / (R)nphi;
  for (int idx = threadIdx.x; idx < K1 * nphi; idx += blockDim.x) {
    const int a = idx / nphi, j = idx - a * nphi;
    const R f = a ? (R)2 : (R)1;
    const R c = T.twc[idx], sn = T.tws[idx];
    twc[idx] = f * c;
    tws[idx] = f * sn;
    twcT[j * K1 + a] = c * inv;
    twsT[j * K1 + a] = sn * inv;
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  V* cw = coef + w * NF * K1;
  const int pst = nphi + 1;   // padded row: the four products of one j sit in four banks
  R* pw = prod + w * 4 * pst;
  // warp w takes latitudes th0 + w, th0 + w + WPB, ... (LPW of them): the twiddles staged
  // above serve all of them
  const int th0 = blockIdx.y * WPB * LPW;
  for (int rep = 0; rep < LPW; ++rep) {
    const int th = th0 + w + WPB * rep;
    if (th >= nlat) break;
    const bool cached = LIN && UG != nullptr;
    const int nfl = cached ? 9 : NF;   // fields transformed here
    __syncwarp();
    for (int idx = lane; idx < nfl * K1; idx += 32) {
      const int a = idx % K1;
      const int f = idx / K1;
      const V* src = (f < 9) ? FC : FCU;
      const int ff = (f < 9) ? f : f - 9;
      V v = src[(((long)ff * Nd + i) * K1 + a) * nlat + th];
      if (a == 0) v.y = 0;                // the m = 0 coefficient enters with its real part
      cw[f * K1 + a] = v;
    }
    __syncwarp();
    for (int j = lane; j < nphi; j += 32) {
      R val[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) val[f] = 0;
      for (int a = 0; a < K1; ++a) {
        const R c = twc[a * nphi + j], sn = tws[a * nphi + j];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if (f < 9 || !cached) {
            const V cf = cw[f * K1 + a];
            val[f] += cf.x * c - cf.y * sn;
          }
        }
      }
      if (cached) {
#pragma unroll
        for (int f = 0; f < 9; ++f) val[(f + 9) % NF] = UG[(((long)f * Nd + i) * nlat + th) * nphi + j];
      }
      R Fr, Ft, Fp, N;
      if (!LIN) {
        // val: 0 ur 1 ut 2 up 3 wr 4 wt 5 wp 6 Tr 7 Tt 8 Tp
        Fr = Ek * (val[1] * val[5] - val[2] * val[4]);
        Ft = Ek * (val[2] * val[3] - val[0] * val[5]);
        Fp = Ek * (val[0] * val[4] - val[1] * val[3]);
        N = val[0] * val[6] + val[1] * val[7] + val[2] * val[8];
      } else {
        const R* u = val;      // perturbation
        const R* U = val + 9;  // base state
        Fr = Ek * ((U[1] * u[5] - U[2] * u[4]) + (u[1] * U[5] - u[2] * U[4]));
        Ft = Ek * ((U[2] * u[3] - U[0] * u[5]) + (u[2] * U[3] - u[0] * U[5]));
        Fp = Ek * ((U[0] * u[4] - U[1] * u[3]) + (u[0] * U[4] - u[1] * U[3]));
        N = U[0] * u[6] + U[1] * u[7] + U[2] * u[8] + u[0] * U[6] + u[1] * U[7] + u[2] * U[8];
      }
      pw[0 * pst + j] = Fr;
      pw[1 * pst + j] = Ft;
      pw[2 * pst + j] = Fp;
      pw[3 * pst + j] = N;
    }
    __syncwarp();
    // forward DFT: one (product q, wavenumber a) output per lane, 4 (K + 1) outputs per
    // latitude (a lane per wavenumber left 32 - (K + 1) lanes idle)
    for (int t = lane; t < 4 * K1; t += 32) {
      const int q = t / K1, a = t - q * K1;
      const R* pq = pw + q * pst;
      R sr = 0, si = 0;
      for (int j = 0; j < nphi; ++j) {
        const R v = pq[j];
        sr += v * twcT[j * K1 + a];
        si -= v * twsT[j * K1 + a];
      }
      FA[(((long)q * Nd + i) * K1 + a) * nlat + th] = mk<R>(sr, si);
    }
  }
}

// The base state's nine grid fields UG[f][i][th][j] (f: u_r, u_th, u_ph, w_r, w_th, w_ph,
// T_r, T_th, T_ph) from its Fourier coefficients FCU, with the inverse DFT of k_products;
// computed once per base state so that every Jacobian action transforms only the
// perturbation.  grid = (Nd, ceil(nlat / WPB)), block = 32 WPB (a warp per latitude),
// dynamic shared memory WPB 9 (K+1) complex.
template <typename R>
__global__ void k_base_grid(DevGeom g, DevLegendre<R> T, const typename C2<R>::T* __restrict__ FCU,
                            R* __restrict__ UG) {
  using V = typename C2<R>::T;
  extern __shared__ unsigned char sh_raw[];
  const int K1 = g.K + 1, nphi = g.nphi, nlat = g.nlat, Nd = g.Nd;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  V* cw = reinterpret_cast<V*>(sh_raw) + w * 9 * K1;
  const int i = blockIdx.x;
  const int th = blockIdx.y * (blockDim.x >> 5) + w;
  if (th >= nlat) return;
  for (int idx = lane; idx < 9 * K1; idx += 32) {
    const int a = idx % K1, f = idx / K1;
    V v = FCU[(((long)f * Nd + i) * K1 + a) * nlat + th];
    if (a == 0) v.y = 0;
    cw[f * K1 + a] = v;
  }
  __syncwarp();
  for (int j = lane; j < nphi; j += 32) {
    R val[9];
#pragma unroll
    for (int f = 0; f < 9; ++f) val[f] = 0;
    for (int a = 0; a < K1; ++a) {
      const R fa = a ? (R)2 : (R)1;
      const R c = fa * T.twc[a * nphi + j], sn = fa * T.tws[a * nphi + j];
#pragma unroll
      for (int f = 0; f < 9; ++f) {
        const V cf = cw[f * K1 + a];
        val[f] += cf.x * c - cf.y * sn;
      }
    }
#pragma unroll
    for (int f = 0; f < 9; ++f) UG[(((long)f * Nd + i) * nlat + th) * nphi + j] = val[f];
  }
}

// ---------------------------------------------------------------------------
// a6: Legendre analysis.  grid = (nm, ceil(Nd / blockDim.y)), block =
// (>= L + 1, multiple of 32) x RT radii; the Legendre tables are staged TC latitudes at a
// time (dynamic shared memory RT 8 nlat/2 sizeof(V) + TC 3 (L + 1) sizeof(R)).
// AR[((p * Nd) + i) * 4 + c], c = Q (F_r), S_F, T_F, (U.grad T).
template <typename R>
__global__ void k_analysis(DevGeom g, DevLegendre<R> T, const typename C2<R>::T* __restrict__ FA,
                           typename C2<R>::T* __restrict__ AR, int TC) {
  using V = typename C2<R>::T;
  extern __shared__ unsigned char sh_raw[];
  const int n2 = g.nlat2, nlat = g.nlat, K1 = g.K + 1, Nd = g.Nd;
  const int RT = blockDim.y;
  V* sym = reinterpret_cast<V*>(sh_raw);   // [RT][4][n2]
  V* ant = sym + RT * 4 * n2;              // [RT][4][n2]
  const int a = blockIdx.x;
  const int i0 = blockIdx.y * RT;
  const int m = g.m_of[a];
  const int nl = g.L - m + 1;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int idx = tid; idx < RT * 4 * n2; idx += blockDim.x * RT) {
    const int rr = idx / (4 * n2);
    const int rem = idx - rr * 4 * n2;
    const int q = rem / n2, t = rem % n2;
    const int i = i0 + rr;
    V sv = mk<R>(0, 0), av = mk<R>(0, 0);
    if (i < Nd) {
      const V* base = FA + (((long)q * Nd + i) * K1 + a) * nlat;
      const V n = base[t], s = base[nlat - 1 - t];
      sv = mk<R>(n.x + s.x, n.y + s.y);
      av = mk<R>(n.x - s.x, n.y - s.y);
    }
    sym[idx] = sv;
    ant[idx] = av;
  }
  const int ql = threadIdx.x;
  const int i = i0 + threadIdx.y;
  const bool live = ql < nl && i < Nd;
  const bool even = (ql & 1) == 0;
  const V* CP = (even ? sym : ant) + threadIdx.y * 4 * n2;   // parity of P and P/sin
  const V* CD = (even ? ant : sym) + threadIdx.y * 4 * n2;   // parity of dP/dtheta
  const long off = g.leg_off[a];
  R Qr = 0, Qi = 0, Nr_ = 0, Ni = 0, Sr = 0, Si = 0, Tr = 0, Ti = 0;
  const R mm = (R)m;
  R* tab = reinterpret_cast<R*>(ant + RT * 4 * n2);   // [TC][3][nl]: TC latitudes per stage
  const int nthr = blockDim.x * RT;
  for (int tc = 0; tc < n2; tc += TC) {
    const int nt = min(TC, n2 - tc);
    __syncthreads();
    for (int idx = tid; idx < nt * 3 * nl; idx += nthr) {
      const int tt = idx / (3 * nl);
      const int rem = idx - tt * 3 * nl;
      const int w = rem / nl, q = rem - w * nl;
      const R* src = (w == 0) ? T.Pw : (w == 1) ? T.dPw : T.Psw;
      tab[idx] = src[off + (long)(tc + tt) * nl + q];
    }
    __syncthreads();
    if (live) {
      for (int tt = 0; tt < nt; ++tt) {
        const int t = tc + tt;
        const R pw = tab[(tt * 3 + 0) * nl + ql];
        const R dw = tab[(tt * 3 + 1) * nl + ql];
        const R sw = tab[(tt * 3 + 2) * nl + ql];
        const V fr = CP[0 * n2 + t], nt4 = CP[3 * n2 + t];
        const V ftD = CD[1 * n2 + t], fpD = CD[2 * n2 + t];
        const V ftP = CP[1 * n2 + t], fpP = CP[2 * n2 + t];
        Qr += pw * fr.x; Qi += pw * fr.y;
        Nr_ += pw * nt4.x; Ni += pw * nt4.y;
        // S = dP F_th - i m P/s F_ph ;  -i m (x + i y) = (m y, -m x)
        Sr += dw * ftD.x + mm * sw * fpP.y;
        Si += dw * ftD.y - mm * sw * fpP.x;
        // T = -i m P/s F_th - dP F_ph
        Tr += mm * sw * ftP.y - dw * fpD.x;
        Ti += -mm * sw * ftP.x - dw * fpD.y;
      }
    }
  }
  if (!live) return;
  const int l = m + ql;
  const R il = (l > 0) ? (R)1 / ((R)l * (R)(l + 1)) : (R)0;
  V* o = AR + ((long)(g.pstart[a] + ql) * Nd + i) * 4;
  o[0] = mk<R>(Qr, Qi);
  o[1] = mk<R>(Sr * il, Si * il);
  o[2] = mk<R>(Tr * il, Ti * il);
  o[3] = mk<R>(Nr_, Ni);
}

// ---------------------------------------------------------------------------
// a7: right-hand side at the collocation radii.  grid = ceil(P / PPB), block = (>= Nr) x PPB.
// mode 0: time step (inhomogeneous T_00 wall values)
// mode 1: Jacobian action (homogeneous rows), c * i m M U added when has_c
// mode 2: explicit terms only (no mass, drift or boundary rows)
struct RhsParams {
  double inv_dt, C, Ek, Ra, r_out;
  long J;        // drift slot (Sec. 3.4), < 0 for none; c is read from u_orig[J]
  int mode;      // 0 step, 1 Jacobian action, 2 explicit terms only, 3 half step of the
                 // second-order scheme (boundary rows (bc + B x)/2, linear explicit terms at xe)
  int explicit_coriolis;  // subtract the Coriolis rows of x (Eqs. expcor_e/f) in modes 0, 1
};

template <typename R>
__global__ void k_rhs(DevGeom g, RhsParams rp, const typename C2<R>::T* __restrict__ AR,
                      const double2* __restrict__ x, const double2* __restrict__ U,
                      const double* __restrict__ u_orig, const double2* __restrict__ xe,
                      double2* __restrict__ rhs) {
  const int has_c = rp.J >= 0;
  using V = typename C2<R>::T;
  extern __shared__ double2 sh2[];
  const int Nr = g.Nr, Nd = g.Nd, P = g.P;
  const bool low = sizeof(R) == 4 && rp.mode == 1;
  // blockDim.y pairs per block, one per thread row; per pair: xs, us (double2),
  // xf, uf (float2 copies for the low-precision mass), ar ([Nd][4] in precision R)
  const size_t per = 10 * (size_t)Nr * sizeof(double2) + 6 * (size_t)Nr * sizeof(float2) +
                     4 * (size_t)Nd * sizeof(V);
  unsigned char* base = reinterpret_cast<unsigned char*>(sh2) + threadIdx.y * per;
  double2* xs = reinterpret_cast<double2*>(base);          // [3][Nr]
  double2* us = xs + 3 * Nr;                                // [3][Nr]
  float2* xf = reinterpret_cast<float2*>(us + 3 * Nr);      // [3][Nr]
  float2* uf = xf + 3 * Nr;                                 // [3][Nr]
  V* ar = reinterpret_cast<V*>(uf + 3 * Nr);                // [Nd][4]
  double2* nb = reinterpret_cast<double2*>(ar + 4 * Nd);    // [4][Nr]: f_{l-1}, f_{l+1}, e_{l-1}, e_{l+1}
  const int p = blockIdx.x * blockDim.y + threadIdx.y;
  const bool coriolis_rhs = rp.explicit_coriolis && rp.mode != 2;
  // mode 3: buoyancy and explicit Coriolis of the state xe (held in `us`)
  const bool sep = rp.mode == 3 && xe != x;
  const double2* xc = sep ? xe : x;     // source of the Coriolis neighbours
  if (p < P) {
    for (int idx = threadIdx.x; idx < 4 * Nd; idx += blockDim.x) ar[idx] = AR[(long)p * Nd * 4 + idx];
    for (int idx = threadIdx.x; idx < 3 * Nr; idx += blockDim.x) {
      const int f = idx / Nr, k = idx % Nr;
      const double2 xv = x[((long)f * P + p) * Nr + k];
      xs[idx] = xv;
      if (low) xf[idx] = make_float2((float)xv.x, (float)xv.y);
      if (has_c) {
        const double2 uv = U[((long)f * P + p) * Nr + k];
        us[idx] = uv;
        if (low) uf[idx] = make_float2((float)uv.x, (float)uv.y);
      }
      if (sep) us[idx] = xe[((long)f * P + p) * Nr + k];
    }
    if (coriolis_rhs) {
      const int lp = g.pair_l[p], mp = g.pair_m[p];
      for (int idx = threadIdx.x; idx < 4 * Nr; idx += blockDim.x) {
        const int w = idx / Nr, k = idx % Nr;
        const int fld = (w < 2) ? 1 : 0;         // f neighbours for the e rows and vice versa
        const int side = (w & 1) ? 1 : -1;
        const int l2 = lp + side;
        double2 v = make_double2(0, 0);
        if (lp > 0 && l2 >= mp && l2 <= g.L) v = xc[((long)fld * P + p + side) * Nr + k];
        nb[idx] = v;
      }
    }
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j >= Nr || p >= P) return;
  const int l = g.pair_l[p], m = g.pair_m[p];
  const double lam = l * (l + 1.0);
  const double r = g.rc[j], ir = 1.0 / r, ir2 = ir * ir;
  // radial projection of the analysed products (precision of the transforms)
  R Tcx = 0, Tcy = 0, Qcx = 0, Qcy = 0, dSx = 0, dSy = 0, Ncx = 0, Ncy = 0;
  {
    const R* R0 = Tab<R>::R0(g);
    const R* R1 = Tab<R>::R1(g);
    const R* rdv = Tab<R>::rd(g);
    for (int i = 0; i < Nd; ++i) {
      const R w0 = R0[i * Nr + j], w1 = R1[i * Nr + j] * rdv[i];
      const V q = ar[i * 4 + 0], s = ar[i * 4 + 1], t = ar[i * 4 + 2], n = ar[i * 4 + 3];
      Qcx += w0 * q.x; Qcy += w0 * q.y;
      Tcx += w0 * t.x; Tcy += w0 * t.y;
      Ncx += w0 * n.x; Ncy += w0 * n.y;
      dSx += w1 * s.x; dSy += w1 * s.y;
    }
  }
  if constexpr (sizeof(R) == 4) {
    if (low && !coriolis_rhs) {
      // Jacobian action of the mixed path: every term is FP32-accurate (FP32 transforms and
      // mass products), so the combination runs in FP32 too (the FP64 pipe of GB300 issues
      // at 1/64 of the FP32 rate); only the stores widen to FP64.
      const float lamf = (float)(l * (l + 1));
      const float irf = 1.0f / (float)g.rc[j], ir2f = irf * irf;
      const float Ekf = (float)rp.Ek, Raf = (float)rp.Ra, rof = (float)rp.r_out;
      auto mass_f = [&](const float2* vf, float2& me, float2& mf, float2& mt) {
        float e0x = 0, e0y = 0, f0x = 0, f0y = 0, f2x = 0, f2y = 0, t0x = 0, t0y = 0;
        for (int k = 0; k < Nr; ++k) {
          const float c0 = g.EcT0f[k * Nr + j], c2 = g.EcT2f[k * Nr + j];
          const float2 e = vf[k], f = vf[Nr + k], t = vf[2 * Nr + k];
          e0x += c0 * e.x; e0y += c0 * e.y;
          f0x += c0 * f.x; f0y += c0 * f.y;
          f2x += c2 * f.x; f2y += c2 * f.y;
          t0x += c0 * t.x; t0y += c0 * t.y;
        }
        const float ce = lamf * Ekf * ir2f, cl = lamf * ir2f;
        me = make_float2(ce * e0x, ce * e0y);
        mf = make_float2(-ce * (f2x - cl * f0x), -ce * (f2y - cl * f0y));
        mt = make_float2(t0x, t0y);
      };
      float2 Me, Mf, MT;
      mass_f(xf, Me, Mf, MT);
      const float cb = lamf * Raf * irf / rof;
      const float2 Ne = make_float2(lamf * irf * Tcx, lamf * irf * Tcy);
      const float2 Nf = make_float2(lamf * ir2f * (Qcx - dSx) + cb * MT.x, lamf * ir2f * (Qcy - dSy) + cb * MT.y);
      const float2 NT = make_float2(-Ncx, -Ncy);
      const float fr = (float)rp.inv_dt, fi = (float)(rp.C * m);  // (1/dt + i C m)
      auto cm = [&](float2 v, float2 n) {
        return make_float2(fr * v.x - fi * v.y + n.x, fr * v.y + fi * v.x + n.y);
      };
      float2 o[3] = {cm(Me, Ne), cm(Mf, Nf), cm(MT, NT)};
      if (has_c) {
        float2 ue, uf_, ut;
        mass_f(uf, ue, uf_, ut);
        const float cmv = (float)u_orig[rp.J] * (float)m;  // c * i m * v = (-cm v.y, cm v.x)
        o[0].x -= cmv * ue.y; o[0].y += cmv * ue.x;
        o[1].x -= cmv * uf_.y; o[1].y += cmv * uf_.x;
        o[2].x -= cmv * ut.y; o[2].y += cmv * ut.x;
      }
      // boundary rows (Sec. 3.1) and identity rows of e_00, f_00
      if (j == 0 || j == Nr - 1) { o[0] = make_float2(0, 0); o[2] = make_float2(0, 0); }
      if (j == 0 || j == 1 || j == Nr - 2 || j == Nr - 1) o[1] = make_float2(0, 0);
      if (l == 0) { o[0] = make_float2(0, 0); o[1] = make_float2(0, 0); }
      if (m == 0) { o[0].y = 0; o[1].y = 0; o[2].y = 0; }
#pragma unroll
      for (int f = 0; f < 3; ++f) rhs[((long)f * P + p) * Nr + j] = make_double2(o[f].x, o[f].y);
      return;
    }
  }
  const double2 Tc = make_double2(Tcx, Tcy), Qc = make_double2(Qcx, Qcy);
  const double2 dS = make_double2(dSx, dSy), Nc = make_double2(Ncx, Ncy);
  // M x at the collocation radius r_j.  FP64 except in Jacobian actions of the
  // mixed path (mode 1, R = float), whose other terms are FP32-accurate anyway;
  // the time step keeps M x^n / dt in FP64 because it dominates small-dt steps.
  double2 e0v = {0, 0}, f0v = {0, 0}, f2v = {0, 0};   // raw e, f, d2f of the last mass() call
  auto mass = [&](const double2* v, const float2* vf, double2& me, double2& mf, double2& mt) {
    double2 e0 = {0, 0}, f0 = {0, 0}, f2 = {0, 0}, t0 = {0, 0};
    if (low) {
      float e0x = 0, e0y = 0, f0x = 0, f0y = 0, f2x = 0, f2y = 0, t0x = 0, t0y = 0;
      for (int k = 0; k < Nr; ++k) {
        const float c0 = g.EcT0f[k * Nr + j], c2 = g.EcT2f[k * Nr + j];
        const float2 e = vf[k], f = vf[Nr + k], t = vf[2 * Nr + k];
        e0x += c0 * e.x; e0y += c0 * e.y;
        f0x += c0 * f.x; f0y += c0 * f.y;
        f2x += c2 * f.x; f2y += c2 * f.y;
        t0x += c0 * t.x; t0y += c0 * t.y;
      }
      e0 = make_double2(e0x, e0y); f0 = make_double2(f0x, f0y);
      f2 = make_double2(f2x, f2y); t0 = make_double2(t0x, t0y);
    } else {
      for (int k = 0; k < Nr; ++k) {
        const double c0 = g.EcT0[k * Nr + j], c2 = g.EcT2[k * Nr + j];
        const double2 e = v[k], f = v[Nr + k], t = v[2 * Nr + k];
        e0.x += c0 * e.x; e0.y += c0 * e.y;
        f0.x += c0 * f.x; f0.y += c0 * f.y;
        f2.x += c2 * f.x; f2.y += c2 * f.y;
        t0.x += c0 * t.x; t0.y += c0 * t.y;
      }
    }
    e0v = e0;
    f0v = f0;
    f2v = f2;
    const double ce = lam * rp.Ek * ir2;
    me = make_double2(ce * e0.x, ce * e0.y);
    mf = make_double2(-ce * (f2.x - lam * ir2 * f0.x), -ce * (f2.y - lam * ir2 * f0.y));
    mt = t0;
  };
  double2 Me, Mf, MT;
  mass(xs, xf, Me, Mf, MT);
  // boundary values of x for the half step of the second-order scheme
  const double2 bxe = e0v, bxf = f0v, bxT = MT;
  double2 MTe = MT;   // temperature of the state whose buoyancy enters (xe in mode 3)
  if (sep) {
    double2 t0_, t1_;
    mass(us, uf, t0_, t1_, MTe);   // also leaves e0v, f0v, f2v of xe for the Coriolis rows
  }
  // explicit Coriolis rows (Eqs. impcor_e_final / impcor_f_final applied to x)
  double2 Ce = {0, 0}, Cf = {0, 0};
  if (coriolis_rhs && l > 0) {
    double2 v0[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}}, v1[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int k = 0; k < Nr; ++k) {
      const double c0 = g.EcT0[k * Nr + j], c1 = g.EcT1[k * Nr + j];
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const double2 a = nb[w * Nr + k];
        v0[w].x += c0 * a.x; v0[w].y += c0 * a.y;
        v1[w].x += c1 * a.x; v1[w].y += c1 * a.y;
      }
    }
    const double lm1 = (double)l * l - 1.0;
    const double alpha = (l - 1 >= m) ? lm1 * sqrt(((double)l * l - (double)m * m) / (4.0 * l * l - 1.0)) : 0.0;
    const double l1 = l + 1.0;
    const double beta = (l + 1 <= g.L) ? l * (l + 2.0) * sqrt((l1 * l1 - (double)m * m) / (4.0 * l1 * l1 - 1.0)) : 0.0;
    const double ca = 2.0 * ir2 * alpha, cb2 = 2.0 * ir2 * beta;
    const double am = (double)l * ir, bp = -(l + 1.0) * ir;
    // -2 i m / r^2 e  and  +2 i m / r^2 (f'' - l(l+1)/r^2 f)
    const double dm = 2.0 * m * ir2;
    const double2 Lf = make_double2(f2v.x - lam * ir2 * f0v.x, f2v.y - lam * ir2 * f0v.y);
    Ce.x = dm * e0v.y + ca * (am * v0[0].x - v1[0].x) + cb2 * (bp * v0[1].x - v1[1].x);
    Ce.y = -dm * e0v.x + ca * (am * v0[0].y - v1[0].y) + cb2 * (bp * v0[1].y - v1[1].y);
    Cf.x = -dm * Lf.y + ca * (am * v0[2].x - v1[2].x) + cb2 * (bp * v0[3].x - v1[3].x);
    Cf.y = dm * Lf.x + ca * (am * v0[2].y - v1[2].y) + cb2 * (bp * v0[3].y - v1[3].y);
  }
  // explicit terms (curl projections and buoyancy)
  double2 Ne = make_double2(lam * ir * Tc.x, lam * ir * Tc.y);
  const double cb = lam * rp.Ra * ir / rp.r_out;
  double2 Nf = make_double2(lam * ir2 * (Qc.x - dS.x) + cb * MTe.x, lam * ir2 * (Qc.y - dS.y) + cb * MTe.y);
  double2 NT = make_double2(-Nc.x, -Nc.y);
  double2 out[3];
  if (rp.mode == 2) {
    out[0] = Ne; out[1] = Nf; out[2] = NT;
  } else {
    const double fr = rp.inv_dt, fi = rp.C * m;  // (1/dt + i C m)
    auto cm = [&](double2 v, double2 n) {
      return make_double2(fr * v.x - fi * v.y + n.x, fr * v.y + fi * v.x + n.y);
    };
    out[0] = cm(Me, Ne);
    out[1] = cm(Mf, Nf);
    out[2] = cm(MT, NT);
    out[0].x -= Ce.x; out[0].y -= Ce.y;
    out[1].x -= Cf.x; out[1].y -= Cf.y;
    if (has_c) {
      double2 ue, uf_, ut;
      mass(us, uf, ue, uf_, ut);
      const double cmv = u_orig[rp.J] * m;  // c * i m * v = (-cm v.y, cm v.x)
      out[0].x -= cmv * ue.y; out[0].y += cmv * ue.x;
      out[1].x -= cmv * uf_.y; out[1].y += cmv * uf_.x;
      out[2].x -= cmv * ut.y; out[2].y += cmv * ut.x;
    }
    // boundary rows (Sec. 3.1) and identity rows of e_00, f_00
    if (j == 0 || j == Nr - 1) { out[0] = make_double2(0, 0); out[2] = make_double2(0, 0); }
    if (j == 0 || j == 1 || j == Nr - 2 || j == Nr - 1) out[1] = make_double2(0, 0);
    if ((rp.mode == 0 || rp.mode == 3) && l == 0 && j == Nr - 1)
      out[2] = make_double2(1.0, 0.0);  // T(r_in) = 1
    if (l == 0) { out[0] = make_double2(0, 0); out[1] = make_double2(0, 0); }
    if (rp.mode == 3) {
      // the half step solves for y = (x^{n+1} + x)/2: boundary rows (bc + B x)/2 so that
      // x^{n+1} = 2 y - x meets the boundary conditions exactly
      auto half = [](double2 a, double2 b) { return make_double2(0.5 * (a.x + b.x), 0.5 * (a.y + b.y)); };
      if (j == 0 || j == Nr - 1) {
        out[0] = half(out[0], bxe);
        out[2] = half(out[2], bxT);
        out[1] = half(out[1], bxf);
      }
      if (j == 1 || j == Nr - 2) {
        const int jj = (j == 1) ? 0 : Nr - 1;     // d_r f at the wall next to row j
        double2 d1 = {0, 0};
        for (int k = 0; k < Nr; ++k) {
          const double c1 = g.EcT1[k * Nr + jj];
          d1.x += c1 * xs[Nr + k].x;
          d1.y += c1 * xs[Nr + k].y;
        }
        out[1] = half(out[1], d1);
      }
      if (l == 0) {   // identity rows of e_00, f_00: y = x / 2 keeps them at zero
        out[0] = make_double2(0.5 * xs[j].x, 0.5 * xs[j].y);
        out[1] = make_double2(0.5 * xs[Nr + j].x, 0.5 * xs[Nr + j].y);
      }
    }
    if (m == 0) { out[0].y = 0; out[1].y = 0; out[2].y = 0; }
  }
#pragma unroll
  for (int f = 0; f < 3; ++f) rhs[((long)f * P + p) * Nr + j] = out[f];
}

// a <- (a + b) / 2 over n complex values in precision R (the Heun average of the analysed
// products of the second-order scheme).
template <typename R>
__global__ void k_average(typename C2<R>::T* __restrict__ a, const typename C2<R>::T* __restrict__ b,
                          long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    typename C2<R>::T v = a[i];
    const typename C2<R>::T w = b[i];
    v.x = (R)0.5 * (v.x + w.x);
    v.y = (R)0.5 * (v.y + w.y);
    a[i] = v;
  }
}

// ---------------------------------------------------------------------------
// a8: block-tridiagonal chain solve (block Thomas with stored
// G = D'^{-1}, H = D'^{-1} A, W = D'^{-1} C from the factorisation).
__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

__device__ __forceinline__ double2 cmac(double2 acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
  return acc;
}

// a8, parallel part: g = G b for every diagonal block of every chain (the
// part of the forward sweep that does not depend on earlier blocks).
// grid = 2 P (blockIdx.x = 2 p + field), block = 256.  g is written to out.
__global__ void k_block_gemv(DevGeom g, const long* __restrict__ chain_off,
                             const double2* __restrict__ G, const double2* __restrict__ rhs,
                             double2* __restrict__ out) {
  extern __shared__ double2 sv[];
  const int Nr = g.Nr, P = g.P;
  const int p = blockIdx.x >> 1, fld = blockIdx.x & 1;
  const int m = g.pair_m[p], a = m / g.Ms, i = g.pair_l[p] - m;
  const int cls = (fld == 0) ? (i & 1) : 1 - (i & 1);
  const double2* Gi = G + (chain_off[2 * a + cls] + i) * (long)Nr * Nr;
  const long row0 = ((long)fld * P + p) * Nr;
  for (int k = threadIdx.x; k < Nr; k += blockDim.x) sv[k] = rhs[row0 + k];
  __syncthreads();
  // 8 lanes per row (lane s takes columns s, s+8, ...): few FP64 adds in the reduction
  const int s8 = threadIdx.x & 7;
  const int rows_per_pass = blockDim.x >> 3;
  for (int r = threadIdx.x >> 3; r < Nr + ((rows_per_pass - Nr % rows_per_pass) % rows_per_pass);
       r += rows_per_pass) {
    double2 acc = {0, 0};
    if (r < Nr) {
      if (m == 0) {   // real factors at m = 0
        for (int k = s8; k < Nr; k += 8) {
          const double gr = Gi[(long)r * Nr + k].x;
          acc.x = fma(gr, sv[k].x, acc.x);
          acc.y = fma(gr, sv[k].y, acc.y);
        }
      } else {
        for (int k = s8; k < Nr; k += 8) acc = cmac(acc, Gi[(long)r * Nr + k], sv[k]);
      }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (r < Nr && s8 == 0) out[row0 + r] = acc;
  }
}

// a8, sequential part: the twisted sweeps of each chain, on thread-block
// clusters.  Cluster (c, dir) handles chain c from the top (dir 0: blocks
// 1..k-1, y_i = g_i - H_i y_{i-1}) or from the bottom (dir 1: blocks
// n-2..k+1, z_i = g_i - H_i z_{i+1}), k = (n-1)/2, concurrently.  In
// k_chain_out both clusters of a chain form the middle block
// x_k = g_k - H_k y_{k-1} - W_k z_{k+1} and then run outward:
// x_i = y_i - W_i x_{i+1} (top) and x_i = z_i - W_i x_{i-1} (bottom).
//
// CTA `rank` of a cluster of CS CTAs owns rows [rank*RPC, rank*RPC + RPC);
// 8 lanes share one row (lane s takes columns s, s+8, ...), 4 rows per warp.
// The vector of the previous block is held in every CTA's shared memory; each
// new slice is broadcast through distributed shared memory, then one cluster
// barrier (hardware, no spin loop; every CTA runs the same iterations).  The
// next block's matrix rows and g value are loaded before the current product.
template <int MAXQ>
struct ChainLane {
  int r, s;        // row and column phase of this lane
  bool active;
  __device__ __forceinline__ void load(const double2* __restrict__ M, int Nr, double2 (&reg)[MAXQ]) const {
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int k = s + 8 * q;
      reg[q] = (active && k < Nr) ? M[(long)r * Nr + k] : make_double2(0, 0);
    }
  }
  // real_op: the m = 0 chains, whose factors are real (no 2im/r^2 terms): 2 FMA per entry
  __device__ __forceinline__ double2 dot(const double2 (&reg)[MAXQ], const double2* v, int Nr,
                                         bool real_op) const {
    // two independent accumulators halve the dependent FP64 chain
    double2 a0 = {0, 0}, a1 = {0, 0};
    if (real_op) {
#pragma unroll
      for (int q = 0; q < MAXQ; q += 2) {
        const int k0 = s + 8 * q, k1 = k0 + 8;
        if (k0 < Nr) { a0.x = fma(reg[q].x, v[k0].x, a0.x); a0.y = fma(reg[q].x, v[k0].y, a0.y); }
        if (q + 1 < MAXQ && k1 < Nr) {
          a1.x = fma(reg[q + 1].x, v[k1].x, a1.x);
          a1.y = fma(reg[q + 1].x, v[k1].y, a1.y);
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < MAXQ; q += 2) {
        const int k0 = s + 8 * q, k1 = k0 + 8;
        if (k0 < Nr) a0 = cmac(a0, reg[q], v[k0]);
        if (q + 1 < MAXQ && k1 < Nr) a1 = cmac(a1, reg[q + 1], v[k1]);
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
};

// bs = 2: the chain of every second block (the reduced chains of chain_cr.cuh), block i of
// it being block bs i of the full chain.
struct ChainInfo {
  int c, dir, cls, p0, nb, km, P, Nr, m, bs;
  long boff, blk;
  __device__ __forceinline__ long row(int i) const {
    const int ib = i * bs;
    const int fld = ((ib + cls) & 1) ? 1 : 0;
    return ((long)fld * P + p0 + ib) * Nr;
  }
};

__device__ __forceinline__ ChainInfo chain_info(const DevGeom& g, const long* chain_off, int CS,
                                                int bs = 1) {
  ChainInfo ci;
  const int cl = blockIdx.x / CS;
  ci.c = cl >> 1;
  ci.dir = cl & 1;
  const int a = ci.c >> 1;
  ci.cls = ci.c & 1;
  const int m = g.m_of[a];
  ci.m = m;
  ci.p0 = g.pstart[a];
  ci.bs = bs;
  ci.nb = (g.L - m + bs) / bs;
  ci.km = (ci.nb - 1) / 2;
  ci.P = g.P;
  ci.Nr = g.Nr;
  ci.boff = chain_off[ci.c];
  ci.blk = (long)g.Nr * g.Nr;
  return ci;
}

// mid[(c * 3 + q) * Nr + k]: q = 0 the last top vector y_{k-1}, q = 1 the
// last bottom vector z_{k+1}, q = 2 the middle g_k.  Staging them lets the
// two clusters of a chain run their outward sweeps without touching anything
// the other cluster reads.
template <int MAXQ>
__global__ void k_chain_half(DevGeom g, const long* __restrict__ chain_off,
                             const double2* __restrict__ H, double2* __restrict__ out,
                             double2* __restrict__ mid, int CS) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double2 sv[];  // [2][Nr] ping-pong, then hist[steps][RPC]
  const ChainInfo ci = chain_info(g, chain_off, CS);
  const int Nr = ci.Nr;
  const int rank = (int)cluster.block_rank();
  const int RPC = (Nr + CS - 1) / CS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lr = warp * 4 + (lane >> 3);   // row within this CTA
  double2* hist = sv + 2 * Nr;              // this CTA's rows of every swept block
  ChainLane<MAXQ> ln;
  ln.r = rank * RPC + lr;
  ln.s = lane & 7;
  ln.active = lr < RPC && ln.r < Nr;
  // top: start at block 0, sweep 1 .. km-1; bottom: start at nb-1, sweep nb-2 .. km+1
  const bool has = ci.dir == 0 ? (ci.km >= 1) : (ci.km <= ci.nb - 2);
  const int first = ci.dir == 0 ? 0 : ci.nb - 1;
  const int step = ci.dir == 0 ? 1 : -1;
  const int count = ci.dir == 0 ? ci.km - 1 : ci.nb - 2 - ci.km;
  for (int k = threadIdx.x; k < Nr; k += blockDim.x)
    sv[k] = has ? out[ci.row(first) + k] : make_double2(0, 0);
  double2 mc[MAXQ], mn[MAXQ];
  double2 gn = {0, 0};
  if (count > 0) {
    ln.load(H + (ci.boff + first + step) * ci.blk, Nr, mn);
    if (ln.active) gn = out[ci.row(first + step) + ln.r];
  }
  cluster.sync();  // every CTA of the cluster has started before any DSMEM store
  for (int t = 1; t <= count; ++t) {
    const int i = first + t * step;
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) mc[q] = mn[q];
    const double2 gc = gn;
    if (t < count) {
      ln.load(H + (ci.boff + i + step) * ci.blk, Nr, mn);
      if (ln.active) gn = out[ci.row(i + step) + ln.r];
    }
    const double2 acc = ln.dot(mc, sv + ((t - 1) & 1) * Nr, Nr, ci.m == 0);
    const double2 v = make_double2(gc.x - acc.x, gc.y - acc.y);
    if (ln.active) {
      // the global store waits until after the sweep: the barrier's release fence would
      // otherwise wait for it at every block
      if (ln.s == 0) hist[(t - 1) * RPC + lr] = v;
      for (int dst = ln.s; dst < CS; dst += 8)
        cluster.map_shared_rank(sv + (t & 1) * Nr, dst)[ln.r] = v;
    }
    cluster.sync();
  }
  for (int idx = threadIdx.x; idx < count * RPC; idx += blockDim.x) {
    const int t = idx / RPC + 1, r = rank * RPC + idx % RPC;
    if (r < Nr) out[ci.row(first + t * step) + r] = hist[idx];
  }
  if (rank == 0) {
    const double2* last = sv + ((count > 0 ? count : 0) & 1) * Nr;
    double2* dst = mid + ((long)ci.c * 3 + ci.dir) * Nr;
    for (int k = threadIdx.x; k < Nr; k += blockDim.x) dst[k] = has ? last[k] : make_double2(0, 0);
    if (ci.dir == 0) {
      double2* gm = mid + ((long)ci.c * 3 + 2) * Nr;
      for (int k = threadIdx.x; k < Nr; k += blockDim.x) gm[k] = out[ci.row(ci.km) + k];
    }
  }
}

template <int MAXQ>
__global__ void k_chain_out(DevGeom g, const long* __restrict__ chain_off,
                            const double2* __restrict__ H, const double2* __restrict__ W,
                            double2* __restrict__ out, const double2* __restrict__ mid, int CS) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double2 sv[];  // [2][Nr] ping-pong, [2][Nr] middle inputs, hist[steps][RPC]
  const ChainInfo ci = chain_info(g, chain_off, CS);
  const int Nr = ci.Nr;
  const int rank = (int)cluster.block_rank();
  const int RPC = (Nr + CS - 1) / CS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lr = warp * 4 + (lane >> 3);
  double2* hist = sv + 4 * Nr;
  ChainLane<MAXQ> ln;
  ln.r = rank * RPC + lr;
  ln.s = lane & 7;
  ln.active = lr < RPC && ln.r < Nr;
  const int km = ci.km, nb = ci.nb;
  double2* yup = sv + 2 * Nr;   // y_{k-1}
  double2* zdn = sv + 3 * Nr;   // z_{k+1}
  const double2* mc0 = mid + (long)ci.c * 3 * Nr;
  for (int k = threadIdx.x; k < Nr; k += blockDim.x) {
    yup[k] = mc0[k];
    zdn[k] = mc0[Nr + k];
  }
  __syncthreads();
  double2 mc[MAXQ], mn[MAXQ];
  // middle block: x_k = g_k - H_k y_{k-1} - W_k z_{k+1} (both clusters, same arithmetic)
  double2 acc = {0, 0};
  if (km > 0) {
    ln.load(H + (ci.boff + km) * ci.blk, Nr, mc);
    const double2 a1 = ln.dot(mc, yup, Nr, ci.m == 0);
    acc.x += a1.x; acc.y += a1.y;
  }
  if (km < nb - 1) {
    ln.load(W + (ci.boff + km) * ci.blk, Nr, mc);
    const double2 a2 = ln.dot(mc, zdn, Nr, ci.m == 0);
    acc.x += a2.x; acc.y += a2.y;
  }
  const double2 gk = ln.active ? mc0[2 * Nr + ln.r] : make_double2(0, 0);
  const double2 xk = make_double2(gk.x - acc.x, gk.y - acc.y);
  const int step = ci.dir == 0 ? -1 : 1;
  const int count = ci.dir == 0 ? km : nb - 1 - km;
  double2 yn = {0, 0};
  if (count > 0) {
    ln.load(W + (ci.boff + km + step) * ci.blk, Nr, mn);
    if (ln.active) yn = out[ci.row(km + step) + ln.r];
  }
  cluster.sync();  // every CTA of the cluster has started before any DSMEM store
  if (ln.active) {
    if (ln.s == 0 && ci.dir == 0) out[ci.row(km) + ln.r] = xk;
    for (int dst = ln.s; dst < CS; dst += 8) cluster.map_shared_rank(sv, dst)[ln.r] = xk;
  }
  cluster.sync();
  // outward: top i = km-1 .. 0 with W_i x_{i+1}; bottom i = km+1 .. nb-1 with W_i x_{i-1}
  for (int t = 1; t <= count; ++t) {
    const int i = km + t * step;
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) mc[q] = mn[q];
    const double2 yc = yn;
    if (t < count) {
      ln.load(W + (ci.boff + i + step) * ci.blk, Nr, mn);
      if (ln.active) yn = out[ci.row(i + step) + ln.r];
    }
    const double2 a3 = ln.dot(mc, sv + ((t - 1) & 1) * Nr, Nr, ci.m == 0);
    const double2 v = make_double2(yc.x - a3.x, yc.y - a3.y);
    if (ln.active) {
      if (ln.s == 0) hist[(t - 1) * RPC + lr] = v;   // stored after the sweep
      for (int dst = ln.s; dst < CS; dst += 8)
        cluster.map_shared_rank(sv + (t & 1) * Nr, dst)[ln.r] = v;
    }
    cluster.sync();
  }
  for (int idx = threadIdx.x; idx < count * RPC; idx += blockDim.x) {
    const int t = idx / RPC + 1, r = rank * RPC + idx % RPC;
    if (r < Nr) out[ci.row(km + t * step) + r] = hist[idx];
  }
}

// Temperature: y = Tinv_l rhs per pair.  grid = P, block >= Nr.
__global__ void k_temp_solve(DevGeom g, const double* __restrict__ Tinv,
                             const double2* __restrict__ rhs, double2* __restrict__ out) {
  extern __shared__ double2 sv[];
  const int Nr = g.Nr, P = g.P;
  const int p = blockIdx.x;
  const long row0 = ((long)2 * P + p) * Nr;
  for (int k = threadIdx.x; k < Nr; k += blockDim.x) sv[k] = rhs[row0 + k];
  __syncthreads();
  const int j = threadIdx.x;
  if (j >= Nr) return;
  const double* Ti = Tinv + (long)g.pair_l[p] * Nr * Nr + (long)j * Nr;
  double2 acc = {0, 0};
  for (int k = 0; k < Nr; ++k) {
    acc.x = fma(Ti[k], sv[k].x, acc.x);
    acc.y = fma(Ti[k], sv[k].y, acc.y);
  }
  out[row0 + j] = acc;
}

// ---------------------------------------------------------------------------
// GMRES / Newton BLAS-1 (FP64).
// Tiled V^T w: block b owns elements [b * 2048, (b+1) * 2048) (8 per thread),
// keeps its slice of w in registers and streams every V_j over it; per-warp
// sums go to shared memory, one cross-warp pass writes partial[j * nblk + b].
// grid = ceil(n / 2048), block = 256, smem = 8 * nv doubles.
__global__ void __launch_bounds__(256) k_dots_tiled(const double* __restrict__ V, long ld, int nv,
                                                    const double* __restrict__ w, long n,
                                                    double* __restrict__ partial) {
  extern __shared__ double red2[];   // [8 warps][nv]
  const long base = (long)blockIdx.x * 2048;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double wv[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const long i = base + threadIdx.x + 256 * e;
    wv[e] = (i < n) ? w[i] : 0.0;
  }
  int j = 0;
  for (; j + 4 <= nv; j += 4) {
    double acc[4] = {0, 0, 0, 0};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const long i = base + threadIdx.x + 256 * e;
      if (i < n) {
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fma(V[(long)(j + u) * ld + i], wv[e], acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      double a = acc[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) red2[warp * nv + j + u] = a;
    }
  }
  for (; j < nv; ++j) {
    double a = 0.0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const long i = base + threadIdx.x + 256 * e;
      if (i < n) a = fma(V[(long)j * ld + i], wv[e], a);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red2[warp * nv + j] = a;
  }
  __syncthreads();
  for (int jj = threadIdx.x; jj < nv; jj += blockDim.x) {
    double a = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) a += red2[q * nv + jj];
    partial[(long)jj * gridDim.x + blockIdx.x] = a;
  }
}

// V^T w split over (element chunk, group of 8 basis vectors): block (c, gidx)
// reads elements [c * 4096, (c+1) * 4096) of w and of V_j, j in [8 gidx, 8 gidx + 8),
// as double2 (8 per thread), every load issued before the first FMA; one block
// reduction of 8 values writes partial[j * nchunk + c].  grid = (nchunk, ceil(nv / 8)),
// block = 256.  Requires n even and V, w 16-byte aligned (ld even).
__global__ void __launch_bounds__(256) k_dots_split(const double* __restrict__ V, long ld, int nv,
                                                    const double* __restrict__ w, long n,
                                                    double* __restrict__ partial) {
  __shared__ double red[8][8];
  const long base = (long)blockIdx.x * 4096;
  const int j0 = blockIdx.y * 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long n2 = n >> 1;
  const double2* w2 = reinterpret_cast<const double2*>(w);
  double2 wv[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const long i2 = (base >> 1) + threadIdx.x + 256 * e;
    wv[e] = (i2 < n2) ? w2[i2] : make_double2(0, 0);
  }
  double acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    acc[u] = 0.0;
    const int j = j0 + u;
    if (j < nv) {
      const double2* v2 = reinterpret_cast<const double2*>(V + (long)j * ld);
      double2 vv[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const long i2 = (base >> 1) + threadIdx.x + 256 * e;
        vv[e] = (i2 < n2) ? v2[i2] : make_double2(0, 0);
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[u] = fma(vv[e].x, wv[e].x, fma(vv[e].y, wv[e].y, acc[u]));
    }
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    double a = acc[u];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[warp][u] = a;
  }
  __syncthreads();
  if (threadIdx.x < 8 && j0 + threadIdx.x < nv) {
    double a = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) a += red[q][threadIdx.x];
    partial[(long)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = a;
  }
}

// First pass of the one-reduction modified Gram-Schmidt step (the low-synchronisation
// MGS of Swirydowicz, Langou, Ananthan, Yang, Thomas, Numer. Linear Algebra Appl. 2021):
// one read of the basis gives both V^T w and V^T q (q = the newest basis vector, whose
// products with the older vectors form the new row of the strictly lower Gram matrix).
// Block (c, g) stages elements [c * 1024, (c+1) * 1024) of w and q in shared memory;
// warp u then streams basis vectors j = 16 g + u and 16 g + 8 + u over that chunk
// (16 double2 loads per lane issued together) and writes
//   partial[j * nchunk + c] = V_j . w,   partial[(nv + j) * nchunk + c] = V_j . q.
// grid = (ld / 1024, ceil(nv / 16)), block = 256.  The basis columns (and w, q) are
// padded to ld, a multiple of 1024, with zeros beyond the vector length, so no
// element needs a bounds check.  On GB300 this pass is bound by the FP64 FMA rate
// (two FMAs per basis element), not by HBM.
__global__ void __launch_bounds__(256) k_dots_pair(const double* __restrict__ V, long ld, int nv,
                                                   const double* __restrict__ w,
                                                   const double* __restrict__ q,
                                                   double* __restrict__ partial) {
  constexpr int E2 = 512, PER = E2 / 32;
  __shared__ double2 ws[E2], qs[E2];
  const long b2 = (long)blockIdx.x * E2;
  const double2* w2 = reinterpret_cast<const double2*>(w) + b2;
  const double2* q2 = reinterpret_cast<const double2*>(q) + b2;
  for (int i = threadIdx.x; i < E2; i += blockDim.x) {
    ws[i] = w2[i];
    qs[i] = q2[i];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunk = gridDim.x;
#pragma unroll 1
  for (int r = 0; r < 2; ++r) {
    const int j = blockIdx.y * 16 + warp + 8 * r;
    if (j >= nv) break;
    const double2* v2 = reinterpret_cast<const double2*>(V + (long)j * ld) + b2 + lane;
    double2 vv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) vv[u] = __ldcs(v2 + u * 32);
    double a = 0.0, b = 0.0;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const double2 x = ws[u * 32 + lane], y = qs[u * 32 + lane];
      a = fma(vv[u].x, x.x, fma(vv[u].y, x.y, a));
      b = fma(vv[u].x, y.x, fma(vv[u].y, y.y, b));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      partial[(long)j * nchunk + blockIdx.x] = a;
      partial[(long)(nv + j) * nchunk + blockIdx.x] = b;
    }
  }
}

// Second pass of the one-reduction MGS step: w <- w - sum_j h[j] V_j with double2 loads
// (eight basis vectors per iteration), and partial[b] = block b's share of |w_new|^2.
// grid = nb (grid-stride over double2 elements), block = 256.  Same alignment rule.
__global__ void __launch_bounds__(256) k_axpy_norm(const double* __restrict__ V, long ld, int nv,
                                                   const double* __restrict__ h,
                                                   double* __restrict__ w, long n,
                                                   double* __restrict__ partial) {
  __shared__ double red[8];
  const long n2 = n >> 1;
  double2* w2 = reinterpret_cast<double2*>(w);
  double ss = 0.0;
  for (long i2 = (long)blockIdx.x * blockDim.x + threadIdx.x; i2 < n2;
       i2 += (long)gridDim.x * blockDim.x) {
    double sx = 0.0, sy = 0.0, tx = 0.0, ty = 0.0;
    int j = 0;
    for (; j + 8 <= nv; j += 8) {
      double2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = reinterpret_cast<const double2*>(V + (long)(j + u) * ld)[i2];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        const double c0 = h[j + u], c1 = h[j + u + 1];
        sx = fma(c0, v[u].x, sx); sy = fma(c0, v[u].y, sy);
        tx = fma(c1, v[u + 1].x, tx); ty = fma(c1, v[u + 1].y, ty);
      }
    }
    for (; j < nv; ++j) {
      const double2 v = reinterpret_cast<const double2*>(V + (long)j * ld)[i2];
      sx = fma(h[j], v.x, sx);
      sy = fma(h[j], v.y, sy);
    }
    double2 o = w2[i2];
    o.x -= sx + tx;
    o.y -= sy + ty;
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

// w <- w / sqrt(nrm2[0]) (left unchanged when nrm2[0] is zero: a breakdown the host sees).
__global__ void k_scale_inv_sqrt(double* __restrict__ w, long n, const double* __restrict__ nrm2) {
  // one FP64 square root and division per block (the FP64 pipe is narrow)
  __shared__ double sinv;
  const double s2 = nrm2[0];
  if (!(s2 > 0.0)) return;
  if (threadIdx.x == 0) sinv = 1.0 / sqrt(s2);
  __syncthreads();
  const double inv = sinv;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x)
    w[idx] *= inv;
}

// w += sign * sum_j coef[j] V_j with double2 loads, eight vectors per iteration.
// Requires n even and 16-byte aligned V, w (ld even).
__global__ void k_multi_axpy2(const double* __restrict__ V, long ld, int nv,
                              const double* __restrict__ coef, double sign, double* __restrict__ w,
                              long n) {
  const long n2 = n >> 1;
  double2* w2 = reinterpret_cast<double2*>(w);
  for (long i2 = (long)blockIdx.x * blockDim.x + threadIdx.x; i2 < n2;
       i2 += (long)gridDim.x * blockDim.x) {
    double sx = 0.0, sy = 0.0, tx = 0.0, ty = 0.0;
    int j = 0;
    for (; j + 8 <= nv; j += 8) {
      double2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = reinterpret_cast<const double2*>(V + (long)(j + u) * ld)[i2];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        const double c0 = coef[j + u], c1 = coef[j + u + 1];
        sx = fma(c0, v[u].x, sx); sy = fma(c0, v[u].y, sy);
        tx = fma(c1, v[u + 1].x, tx); ty = fma(c1, v[u + 1].y, ty);
      }
    }
    for (; j < nv; ++j) {
      const double2 v = reinterpret_cast<const double2*>(V + (long)j * ld)[i2];
      sx = fma(coef[j], v.x, sx);
      sy = fma(coef[j], v.y, sy);
    }
    double2 o = w2[i2];
    o.x = fma(sign, sx + tx, o.x);
    o.y = fma(sign, sy + ty, o.y);
    w2[i2] = o;
  }
}

// out[j] = sum_b partial[j * nblk + b].  grid = nv, block = 256.
__global__ void k_reduce_rows(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(long)j * nblk + b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[j] = s;
  }
}

// y = a * x + b * y
__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y,
                        long n) {
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x)
    y[idx] = a * x[idx] + b * y[idx];
}

// Graph-replayed Jacobian action: the input and output vectors are reached
// through pointers held in device memory (set by k_set_ptrs before each replay).
__global__ void k_set_ptrs(const double** slots, const double* u, double* out) {
  slots[0] = u;
  slots[1] = out;
}

// x = u with u_J zeroed; c = u_J stored in cslot[0] (Sec. 3.4)
__global__ void k_copy_zero_slot_ind(const double* const* slots, long J, double* __restrict__ x,
                                     double* __restrict__ cslot, long n) {
  const double* u = slots[0];
  if (J >= 0 && blockIdx.x == 0 && threadIdx.x == 0) cslot[0] = u[J];
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x)
    x[idx] = (idx == J) ? 0.0 : u[idx];
}

// out = y - x through the output pointer slot
__global__ void k_finish_ind(const double* const* slots, const double* __restrict__ y,
                             const double* __restrict__ x, long n) {
  double* out = const_cast<double*>(slots[1]);
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x)
    out[idx] = y[idx] - x[idx];
}

// copy with u_J zeroed (x holds the canonical layout)
__global__ void k_copy_zero_slot(const double* __restrict__ u, long J, double* __restrict__ x,
                                 long n) {
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x)
    x[idx] = (idx == J) ? 0.0 : u[idx];
}


// ---------------------------------------------------------------------------
// Diagnostics (kinetic energy and Nusselt numbers).
// Kinetic energy of one pair by Parseval's identity for the potentials of
// Sec. 2.1: int |U|^2 dOmega = w_m [l(l+1)|e|^2/r^2 + (l(l+1))^2 |f|^2/r^4
// + l(l+1)|d_r f|^2/r^2], w_m = 4 pi (m = 0) or 16 pi (m > 0, the real field
// a Y + conj(a Y)), integrated against r^2 dr with the Gauss-Legendre rule
// (rq, wq; wq includes dr/dx).  Tq[q][k] = T_k(x_q), dTq[q][k] = d T_k/dr.
// grid = P, block = 128, dynamic smem = 2 Nr double2.
__global__ void k_ke_pairs(const double* __restrict__ U, int P, int Nr, int nq,
                           const double* __restrict__ Tq, const double* __restrict__ dTq,
                           const double* __restrict__ rq, const double* __restrict__ wq,
                           const int* __restrict__ pair_l, const int* __restrict__ pair_m,
                           double* __restrict__ partial) {
  extern __shared__ double2 kes[];
  __shared__ double red[32];
  const int p = blockIdx.x;
  const double2* U2 = reinterpret_cast<const double2*>(U);
  for (int k = threadIdx.x; k < Nr; k += blockDim.x) {
    kes[k] = U2[(long)p * Nr + k];                 // e
    kes[Nr + k] = U2[((long)P + p) * Nr + k];      // f
  }
  __syncthreads();
  const double lam = pair_l[p] * (pair_l[p] + 1.0);
  double s = 0.0;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    double er = 0, ei = 0, fr = 0, fi = 0, gr = 0, gi = 0;
    for (int k = 0; k < Nr; ++k) {
      const double t = Tq[(long)q * Nr + k], dt = dTq[(long)q * Nr + k];
      const double2 e = kes[k], f = kes[Nr + k];
      er = fma(t, e.x, er); ei = fma(t, e.y, ei);
      fr = fma(t, f.x, fr); fi = fma(t, f.y, fi);
      gr = fma(dt, f.x, gr); gi = fma(dt, f.y, gi);
    }
    const double r = rq[q], ir2 = 1.0 / (r * r);
    const double dens = lam * (er * er + ei * ei) * ir2 +
                        lam * lam * (fr * fr + fi * fi) * ir2 * ir2 +
                        lam * (gr * gr + gi * gi) * ir2;
    s = fma(wq[q] * r * r, dens, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
    const double pi = 3.141592653589793238;
    partial[p] = (pair_m[p] == 0 ? 4.0 * pi : 16.0 * pi) * a;
  }
}

// out[0] = KE = (1/2) sum_p partial[p] / V; out[1], out[2] = Nu at r_in, r_out:
// d_r of the mean temperature T_00 at each wall (T'_k(+-1) = (+-1)^(k+1) k^2)
// over the conductive gradient g_in, g_out.  One block of 256 threads.
__global__ void k_diag_finish(const double* __restrict__ partial, int P,
                              const double* __restrict__ U, int Nr, double inv_2V,
                              double dxdr, double g_in, double g_out, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int p = threadIdx.x; p < P; p += blockDim.x) s += partial[p];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
    out[0] = a * inv_2V;
    // T_00: field 2, pair 0 (m = 0, l = 0), real parts
    const double* T00 = U + 2L * P * Nr * 2;
    double din = 0.0, dout = 0.0;
    for (int k = 0; k < Nr; ++k) {
      const double k2 = (double)k * k;
      dout = fma(k2, T00[2 * k], dout);
      din = fma((k & 1) ? k2 : -k2, T00[2 * k], din);
    }
    out[1] = din * dxdr / g_in;
    out[2] = dout * dxdr / g_out;
  }
}

// ---------------------------------------------------------------------------
// Continuation helpers.
// out = a x0 + b x1 + c x2 (the Lagrange extrapolation of Sec. 4.3); x1 / x2 may be null
// when their weight is unused.
__global__ void k_lincomb3(double* __restrict__ out, double a, const double* __restrict__ x0,
                           double b, const double* __restrict__ x1, double c,
                           const double* __restrict__ x2, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double v = a * x0[i];
    if (x1) v = fma(b, x1[i], v);
    if (x2) v = fma(c, x2[i], v);
    out[i] = v;
  }
}

// Index of the largest |x - y| (lowest index on ties): per-block (value, index) pairs,
// then one block reduces them.  grid = nb <= 1024, block = 256.
__device__ __forceinline__ void argmax_merge(double& v, long& i, double v2, long i2) {
  if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

__global__ void k_argmax_absdiff(const double* __restrict__ x, const double* __restrict__ y, long n,
                                 double* __restrict__ pv, long* __restrict__ pi) {
  __shared__ double sv[256];
  __shared__ long si[256];
  double v = -1.0;
  long idx = n;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    argmax_merge(v, idx, fabs(x[i] - y[i]), i);
  sv[threadIdx.x] = v;
  si[threadIdx.x] = idx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      double a = sv[threadIdx.x];
      long ia = si[threadIdx.x];
      argmax_merge(a, ia, sv[threadIdx.x + o], si[threadIdx.x + o]);
      sv[threadIdx.x] = a;
      si[threadIdx.x] = ia;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = sv[0];
    pi[blockIdx.x] = si[0];
  }
}

__global__ void k_argmax_finish(const double* __restrict__ pv, const long* __restrict__ pi, int nb,
                                long* __restrict__ out) {
  __shared__ double sv[256];
  __shared__ long si[256];
  double v = -1.0;
  long idx = LONG_MAX;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) argmax_merge(v, idx, pv[b], pi[b]);
  sv[threadIdx.x] = v;
  si[threadIdx.x] = idx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      double a = sv[threadIdx.x];
      long ia = si[threadIdx.x];
      argmax_merge(a, ia, sv[threadIdx.x + o], si[threadIdx.x + o]);
      sv[threadIdx.x] = a;
      si[threadIdx.x] = ia;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = si[0];
}

// Spectral tail of a state (the under-resolution test of Sec. 4.4): out[0] = the largest
// |coefficient| of U - Uc, out[1] = the largest at the last Chebyshev degree k = Nr - 1,
// out[2] = the largest at the last spherical-harmonic degree l = L, as the bit patterns
// of non-negative doubles (whose unsigned order is their numeric order).
__global__ void k_spectral_tail(const double2* __restrict__ U, const double2* __restrict__ Uc,
                                int P, int Nr, int L, const int* __restrict__ pair_l,
                                unsigned long long* __restrict__ out) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  const long n = 3L * P * Nr;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x) {
    const double2 z = U[idx], c = Uc[idx];
    const double a = hypot(z.x - c.x, z.y - c.y);
    const int k = (int)(idx % Nr);
    const int p = (int)((idx / Nr) % P);
    a0 = fmax(a0, a);
    if (k == Nr - 1) a1 = fmax(a1, a);
    if (pair_l[p] == L) a2 = fmax(a2, a);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 = fmax(a0, __shfl_xor_sync(0xffffffffu, a0, o));
    a1 = fmax(a1, __shfl_xor_sync(0xffffffffu, a1, o));
    a2 = fmax(a2, __shfl_xor_sync(0xffffffffu, a2, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out + 0, (unsigned long long)__double_as_longlong(a0));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(a1));
    atomicMax(out + 2, (unsigned long long)__double_as_longlong(a2));
  }
}

// Spectral interpolation between truncations of the same M_s (Sec. 4.4, refinement by
// zero-filling the new modes): dst coefficient (field, m, l, k) = src coefficient when
// l <= Ls, m <= Ls and k < Nrs, else zero.  One thread per complex dst coefficient.
// The src pair of (m = a M_s, l) is a (Ls + 1) - M_s a (a - 1) / 2 + (l - m).
__global__ void k_regrid(const double2* __restrict__ src, int Ls, int Nrs, int Ps,
                         double2* __restrict__ dst, int Nrd, int Pd,
                         const int* __restrict__ dpair_l, const int* __restrict__ dpair_m, int Ms) {
  const long n = 3L * Pd * Nrd;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x) {
    const int k = (int)(idx % Nrd);
    const int p = (int)((idx / Nrd) % Pd);
    const int f = (int)(idx / ((long)Nrd * Pd));
    const int l = dpair_l[p], m = dpair_m[p];
    double2 v = make_double2(0.0, 0.0);
    if (l <= Ls && k < Nrs) {
      const int a = m / Ms;
      const long ps = (long)a * (Ls + 1) - (long)Ms * a * (a - 1) / 2 + (l - m);
      v = src[((long)f * Ps + ps) * Nrs + k];
    }
    dst[idx] = v;
  }
}

}  // namespace rsc
