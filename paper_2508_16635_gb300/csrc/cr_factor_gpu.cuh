// GPU factorisation of the odd-even reduced chains (HostFactorCR in rsc_internal.h; the
// solve is chain_cr.cuh), FP64, with the block LU of factor_gpu.cuh (row equilibration and
// partial pivoting inside each block):
//   k_cr_fac_odd:    per odd block i, D_i^-1, P_i = D_i^-1 A_i and Q_i = D_i^-1 C_i
//                    (all odd blocks at once);
//   k_cr_fac_reduce: per even block j, the reduced chain's blocks
//                    D'_j = D_j - A_j Q_{j-1} - C_j P_{j+1},  A'_j = -A_j P_{j-1},
//                    C'_j = -C_j Q_{j+1}  (all even blocks at once; the couplings A_j, C_j
//                    applied from the Chebyshev tables: (A X)(r, k) = a2_r (al_r (E0 X) - (E1 X)));
//   k_cr_fac_half, k_cr_fac_mid: the twisted block factors G', H', W' of every reduced
//                    chain, with the same conventions as k_factor_half / k_factor_mid but
//                    dense couplings A', C' read from global memory.
// The same factors as build_factor_cr to rounding.  Shared memory: fac_smem_bytes(Nr).
#pragma once

#include "factor_gpu.cuh"

namespace rsc {

struct CrFacGeom {
  const int* pairs;       // pair list of the parity the kernel runs over
  const int* pair_l;
  const int* pair_m;
  int Ms;
  const long* odd_off;    // per chain: first odd block
  const long* red_off;    // per chain: first reduced block
};

__device__ __forceinline__ void cr_fac_block_of(const FacGeom& g, const CrFacGeom& cg, int& c,
                                                int& i, int& fld, int& l, int& m, int& nb) {
  const int p = cg.pairs[blockIdx.x >> 1];
  fld = blockIdx.x & 1;
  m = cg.pair_m[p];
  l = cg.pair_l[p];
  i = l - m;
  const int cls = (fld == 0) ? (i & 1) : 1 - (i & 1);
  c = 2 * (m / cg.Ms) + cls;
  nb = g.L - m + 1;
}

// Coupling row factors of block (fld, l, m) into shared memory; sides absent from the chain
// (i = 0, i = nb - 1) get a2 = 0.
__device__ __forceinline__ void cr_fac_rows(const FacGeom& g, const FacShared& sh, int fld, int l,
                                            int m, bool left, bool right) {
  for (int j = threadIdx.x; j < g.Nr; j += kFacThreads) {
    double a2, al;
    fac_coupling_row(g, fld, l, m, -1, j, a2, al);
    sh.a2[0][j] = left ? a2 : 0.0;
    sh.al[0][j] = al;
    fac_coupling_row(g, fld, l, m, +1, j, a2, al);
    sh.a2[1][j] = right ? a2 : 0.0;
    sh.al[1][j] = al;
  }
}

// Odd blocks.  grid = 2 x (pairs with odd l - m).  status[c] = 1 on a singular block.
__global__ void __launch_bounds__(kFacThreads) k_cr_fac_odd(FacGeom g, CrFacGeom cg, double2* Dinv,
                                                            double2* Pm, double2* Qm, int* status) {
  extern __shared__ __align__(16) unsigned char fac_smem[];
  const FacShared sh = fac_shared(fac_smem, g.Nr);
  const int Nr = g.Nr, tid = threadIdx.x;
  int c, i, fld, l, m, nb;
  cr_fac_block_of(g, cg, c, i, fld, l, m, nb);
  const bool right = i + 1 < nb;
  cr_fac_rows(g, sh, fld, l, m, true, right);
  for (int j = tid; j < Nr; j += kFacThreads) {   // row scales of D alone
    double mx = 0.0;
    for (int k = 0; k < Nr; ++k) mx = fmax(mx, fx_abs(fac_diag(g, fld, l, m, j, k)));
    sh.S[j] = 1.0 / mx;
  }
  __syncthreads();
  for (int e = tid; e < Nr * Nr; e += kFacThreads) {
    const double2 d = fac_diag(g, fld, l, m, e / Nr, e % Nr);
    const double sj = sh.S[e / Nr];
    sh.Mx[e] = make_double2(d.x * sj, d.y * sj);
  }
  __syncthreads();
  if (!fac_lu(sh, Nr)) {
    if (tid == 0) status[c] = 1;
    return;
  }
  const size_t blk = (size_t)Nr * Nr;
  const long slot = cg.odd_off[c] + (i >> 1);
  const double* S = sh.S;
  fac_solve(sh, Nr, [&](int j, int k) { return make_double2(j == k ? S[j] : 0.0, 0.0); },
            Dinv + slot * blk);
  for (int q = 0; q < 2; ++q) {
    if (q == 1 && !right) break;
    fac_solve(sh, Nr, [&](int j, int k) {
      const double a2 = sh.a2[q][j];
      if (a2 == 0.0) return make_double2(0.0, 0.0);
      return make_double2(S[j] * a2 * (sh.al[q][j] * g.E0[(size_t)j * Nr + k] - g.E1[(size_t)j * Nr + k]), 0.0);
    }, (q == 0 ? Pm : Qm) + slot * blk);
  }
}

// Even blocks.  grid = 2 x (pairs with even l - m).  Dr, Ar, Cr: [reduced block][Nr][Nr].
__global__ void __launch_bounds__(kFacThreads) k_cr_fac_reduce(FacGeom g, CrFacGeom cg,
                                                               const double2* __restrict__ Pm,
                                                               const double2* __restrict__ Qm,
                                                               double2* Dr, double2* Ar, double2* Cr) {
  extern __shared__ __align__(16) unsigned char fac_smem[];
  const FacShared sh = fac_shared(fac_smem, g.Nr);
  const int Nr = g.Nr, tid = threadIdx.x;
  int c, i, fld, l, m, nb;
  cr_fac_block_of(g, cg, c, i, fld, l, m, nb);
  const bool left = i >= 1, right = i + 1 < nb;
  cr_fac_rows(g, sh, fld, l, m, left, right);
  __syncthreads();
  const size_t blk = (size_t)Nr * Nr;
  const long o0 = cg.odd_off[c];
  const double2* QL = left ? Qm + (o0 + ((i - 1) >> 1)) * blk : nullptr;
  const double2* PL = i >= 2 ? Pm + (o0 + ((i - 1) >> 1)) * blk : nullptr;
  const double2* PR = right ? Pm + (o0 + ((i + 1) >> 1)) * blk : nullptr;
  const double2* QR = i + 2 < nb ? Qm + (o0 + ((i + 1) >> 1)) * blk : nullptr;
  const long slot = cg.red_off[c] + (i >> 1);
  // (A X)(j, k) or (C X)(j, k) for side q
  auto apply = [&](int q, const double2* X, int j, int k) {
    double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
    const double* e0r = g.E0 + (size_t)j * Nr;
    const double* e1r = g.E1 + (size_t)j * Nr;
    for (int t = 0; t < Nr; ++t) {
      const double2 x = X[(size_t)t * Nr + k];
      s0.x = fma(e0r[t], x.x, s0.x);
      s0.y = fma(e0r[t], x.y, s0.y);
      s1.x = fma(e1r[t], x.x, s1.x);
      s1.y = fma(e1r[t], x.y, s1.y);
    }
    const double a2 = sh.a2[q][j], al = sh.al[q][j];
    return make_double2(a2 * (al * s0.x - s1.x), a2 * (al * s0.y - s1.y));
  };
  for (int e = tid; e < Nr * Nr; e += kFacThreads) {
    const int j = e / Nr, k = e % Nr;
    double2 d = fac_diag(g, fld, l, m, j, k);
    double2 a = make_double2(0.0, 0.0), cc = make_double2(0.0, 0.0);
    if (sh.a2[0][j] != 0.0) {
      const double2 t = apply(0, QL, j, k);
      d.x -= t.x;
      d.y -= t.y;
      if (PL) {
        const double2 u = apply(0, PL, j, k);
        a = make_double2(-u.x, -u.y);
      }
    }
    if (sh.a2[1][j] != 0.0) {
      const double2 t = apply(1, PR, j, k);
      d.x -= t.x;
      d.y -= t.y;
      if (QR) {
        const double2 u = apply(1, QR, j, k);
        cc = make_double2(-u.x, -u.y);
      }
    }
    Dr[slot * blk + e] = d;
    Ar[slot * blk + e] = a;
    Cr[slot * blk + e] = cc;
  }
}

// One block t of a reduced chain: D'' = D' - A' W_lo - C' W_hi (either term absent), rows
// scaled by the largest entry over D', A' (t > 0) and C' (t < nr - 1), LU, then G = D''^-1,
// H = D''^-1 hsrc, W = D''^-1 wsrc (hsrc / wsrc null: not formed).
__device__ bool cr_fac_dense(const FacShared& sh, int Nr, const double2* __restrict__ Dm,
                             const double2* __restrict__ Am, const double2* __restrict__ Cm,
                             const double2* Wlo, const double2* Whi, const double2* hsrc,
                             const double2* wsrc, double2* G, double2* H, double2* W) {
  const int tid = threadIdx.x;
  for (int j = tid; j < Nr; j += kFacThreads) {
    double mx = 0.0;
    for (int k = 0; k < Nr; ++k) {
      const size_t jk = (size_t)j * Nr + k;
      mx = fmax(mx, fx_abs(Dm[jk]));
      if (Am) mx = fmax(mx, fx_abs(Am[jk]));
      if (Cm) mx = fmax(mx, fx_abs(Cm[jk]));
    }
    sh.S[j] = 1.0 / mx;
  }
  __syncthreads();
  for (int e = tid; e < Nr * Nr; e += kFacThreads) {
    const int j = e / Nr, k = e % Nr;
    double2 d = Dm[e];
    for (int side = 0; side < 2; ++side) {
      const double2* X = side == 0 ? Am : Cm;
      const double2* Wp = side == 0 ? Wlo : Whi;
      if (!Wp) continue;
      const double2* xr = X + (size_t)j * Nr;
      for (int t = 0; t < Nr; ++t) d = fx_sub_mul(d, xr[t], Wp[(size_t)t * Nr + k]);
    }
    const double sj = sh.S[j];
    sh.Mx[e] = make_double2(d.x * sj, d.y * sj);
  }
  __syncthreads();
  if (!fac_lu(sh, Nr)) return false;
  const double* S = sh.S;
  fac_solve(sh, Nr, [&](int j, int k) { return make_double2(j == k ? S[j] : 0.0, 0.0); }, G);
  const double2* srcs[2] = {hsrc, wsrc};
  double2* dsts[2] = {H, W};
  for (int q = 0; q < 2; ++q) {
    const double2* X = srcs[q];
    if (!X) continue;
    fac_solve(sh, Nr, [&](int j, int k) {
      const double2 x = X[(size_t)j * Nr + k];
      return make_double2(S[j] * x.x, S[j] * x.y);
    }, dsts[q]);
  }
  return true;
}

// Half sweeps of the reduced chains: blockIdx.x = 2 c + half (half 0 top-down over
// t = 0..km-1, half 1 bottom-up over t = nr-1..km+1).
__global__ void __launch_bounds__(kFacThreads) k_cr_fac_half(FacGeom g, const long* red_off,
                                                             const double2* Dr, const double2* Ar,
                                                             const double2* Cr, double2* G,
                                                             double2* H, double2* W, int* status) {
  extern __shared__ __align__(16) unsigned char fac_smem[];
  const FacShared sh = fac_shared(fac_smem, g.Nr);
  const int c = blockIdx.x >> 1, half = blockIdx.x & 1;
  const int m = g.m_of[c >> 1];
  const int nb = g.L - m + 1, nr = (nb + 1) / 2, km = (nr - 1) / 2;
  const size_t blk = (size_t)g.Nr * g.Nr;
  const long off = red_off[c];
  auto at = [&](const double2* v, int t) { return v + (off + t) * blk; };
  auto atw = [&](double2* v, int t) { return v + (off + t) * blk; };
  if (half == 0) {
    for (int t = 0; t < km; ++t)
      if (!cr_fac_dense(sh, g.Nr, at(Dr, t), t > 0 ? at(Ar, t) : nullptr, at(Cr, t),
                        t > 0 ? at(W, t - 1) : nullptr, nullptr, t > 0 ? at(Ar, t) : nullptr,
                        at(Cr, t), atw(G, t), atw(H, t), atw(W, t))) {
        if (threadIdx.x == 0) status[c] = 1;
        return;
      }
  } else {
    for (int t = nr - 1; t > km; --t)
      if (!cr_fac_dense(sh, g.Nr, at(Dr, t), at(Ar, t), t < nr - 1 ? at(Cr, t) : nullptr,
                        nullptr, t < nr - 1 ? at(W, t + 1) : nullptr,
                        t < nr - 1 ? at(Cr, t) : nullptr, at(Ar, t), atw(G, t), atw(H, t),
                        atw(W, t))) {
        if (threadIdx.x == 0) status[c] = 1;
        return;
      }
  }
}

// Middle blocks of the reduced chains, one CTA per chain (after k_cr_fac_half).
__global__ void __launch_bounds__(kFacThreads) k_cr_fac_mid(FacGeom g, const long* red_off,
                                                            const double2* Dr, const double2* Ar,
                                                            const double2* Cr, double2* G,
                                                            double2* H, double2* W, int* status) {
  extern __shared__ __align__(16) unsigned char fac_smem[];
  const FacShared sh = fac_shared(fac_smem, g.Nr);
  const int c = blockIdx.x;
  const int m = g.m_of[c >> 1];
  const int nb = g.L - m + 1, nr = (nb + 1) / 2, km = (nr - 1) / 2;
  const size_t blk = (size_t)g.Nr * g.Nr;
  const long o = (red_off[c] + km) * blk;
  const bool lo = km > 0, hi = km < nr - 1;
  if (!cr_fac_dense(sh, g.Nr, Dr + o, lo ? Ar + o : nullptr, hi ? Cr + o : nullptr,
                    lo ? W + o - blk : nullptr, hi ? W + o + blk : nullptr, lo ? Ar + o : nullptr,
                    hi ? Cr + o : nullptr, G + o, H + o, W + o))
    if (threadIdx.x == 0) status[c] = 1;
}

}  // namespace rsc
