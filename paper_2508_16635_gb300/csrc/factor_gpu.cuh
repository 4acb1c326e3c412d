// GPU factorisation of the implicit operator (Sec. 3.2, Fig. blocks; Sec. 4.4 refactorises
// at every new Ek): the twisted block Thomas factors of every Coriolis chain and the
// per-l temperature inverses, in FP64, with row equilibration and partial pivoting inside
// each block.  The same factors as the host routine build_factor (tables.cpp), built on
// the device from the Chebyshev tables:
//
//   chain c = 2 * (m index) + class, block i = degree l = m + i (fields e / f alternate),
//   km = (nb - 1) / 2 the middle block;
//   top    i < km : D' = D_i - A_i W_{i-1};   G = D'^-1, H = D'^-1 A_i, W = D'^-1 C_i
//   bottom i > km : D' = D_i - C_i W_{i+1};   G = D'^-1, H = D'^-1 C_i, W = D'^-1 A_i
//   middle i = km : D' = D_i - A_i W_{km-1} - C_i W_{km+1};  G, H = D'^-1 A_i, W = D'^-1 C_i
//
// with D_i the diagonal block (M/dt + K with boundary rows, Eqs. impcor_e_final /
// impcor_f_final), A_i / C_i the Coriolis couplings to blocks i - 1 / i + 1.  Every row
// of block row i is divided by its largest entry over D_i, A_i and C_i (S_i) before the
// LU, and the inverse absorbs the scaling: D'^-1 = (S D')^-1 S.
//
// Layout: one CTA per (chain, half) sweeps its half of the chain block by block; a
// second kernel closes the middle blocks.  Each CTA keeps the block being factorised in
// shared memory (N_r^2 complex) and a chunk of right-hand-side columns (N_r x kFacCols),
// reads W of the previous block back from global memory (just written by the same CTA,
// an L2 hit), and builds D, A and C entry by entry from the Chebyshev tables (the
// couplings are a2_j (alpha_j E0 - E1), so A W needs only E0 W and E1 W).
// Shared memory: 16 (N_r^2 + N_r kFacCols) + 16 N_r bytes, 193 KB at N_r = 96; larger N_r
// use the host routine.
#pragma once

#include <cuda_runtime.h>

namespace rsc {

constexpr int kFacThreads = 256;
constexpr int kFacCols = 32;    // right-hand-side columns per chunk of the triangular solves
constexpr int kFacMaxNr = 96;

struct FacGeom {
  int Nr, L, nm;
  const int* m_of;          // [nm]
  const long* chain_off;    // [2 nm + 1] first block of each chain
  const double* rc;         // [Nr] collocation radii
  const double* E0;         // [Nr][Nr] row-major: d^o T_k / dr^o at r_j
  const double* E1;
  const double* E2;
  const double* E4;
  double Ek, Pr, inv_dt;
  int explicit_coriolis;
};

__device__ __forceinline__ double2 fx_mul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 fx_sub_mul(double2 acc, double2 a, double2 b) {  // acc - a b
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 fx_inv(double2 z) {
  const double d = 1.0 / fma(z.x, z.x, z.y * z.y);
  return make_double2(z.x * d, -z.y * d);
}
__device__ __forceinline__ double fx_abs(double2 z) { return hypot(z.x, z.y); }

// Diagonal block entry (j, k) of field fld (0 = e, 1 = f) at degree l, order m: M/dt + K
// with the boundary rows (e: f = ... rows 0 and Nr-1 hold T_k(+-1); f also rows 1 and
// Nr-2 hold dT_k/dr at +-1); the l = 0 blocks of e and f are identities.
__device__ double2 fac_diag(const FacGeom& g, int fld, int l, int m, int j, int k) {
  const int Nr = g.Nr;
  if (l == 0) return make_double2(j == k ? 1.0 : 0.0, 0.0);
  if (j == 0) return make_double2(g.E0[k], 0.0);
  if (j == Nr - 1) return make_double2(g.E0[(size_t)(Nr - 1) * Nr + k], 0.0);
  if (fld == 1 && j == 1) return make_double2(g.E1[k], 0.0);
  if (fld == 1 && j == Nr - 2) return make_double2(g.E1[(size_t)(Nr - 1) * Nr + k], 0.0);
  const size_t jk = (size_t)j * Nr + k;
  const double r = g.rc[j], r2 = r * r;
  const double lam = l * (l + 1.0);
  const double e0 = g.E0[jk], e2 = g.E2[jk];
  const double Ll = e2 - lam / r2 * e0;
  const double mk = lam * g.Ek / r2;
  if (fld == 0)
    return make_double2(mk * g.inv_dt * e0 - mk * Ll,
                        g.explicit_coriolis ? 0.0 : -2.0 * m / r2 * e0);
  const double LL = g.E4[jk] - 2.0 * lam / r2 * e2 + 4.0 * lam / (r2 * r) * g.E1[jk] +
                    (lam * lam - 6.0 * lam) / (r2 * r2) * e0;
  return make_double2(-mk * g.inv_dt * Ll + mk * LL, g.explicit_coriolis ? 0.0 : 2.0 * m / r2 * Ll);
}

// Coupling of the fld equation at l to the other potential at l + side: row factor a2_j and
// radial factor alpha_j, so that the entry is a2_j (alpha_j E0[j][k] - E1[j][k]); a2_j = 0
// on the boundary rows and when there is no coupling (l = 0, explicit Coriolis).
__device__ void fac_coupling_row(const FacGeom& g, int fld, int l, int m, int side, int j,
                                 double& a2, double& alpha) {
  a2 = 0.0;
  alpha = 0.0;
  const int Nr = g.Nr;
  if (l == 0 || g.explicit_coriolis) return;
  const int j0 = (fld == 1) ? 2 : 1, j1 = (fld == 1) ? Nr - 3 : Nr - 2;
  if (j < j0 || j > j1) return;
  double coef;
  if (side < 0) {
    coef = ((double)l * l - 1.0) * sqrt(((double)l * l - (double)m * m) / (4.0 * l * l - 1.0));
  } else {
    const double l1 = l + 1.0;
    coef = l * (l + 2.0) * sqrt((l1 * l1 - (double)m * m) / (4.0 * l1 * l1 - 1.0));
  }
  const double r = g.rc[j];
  a2 = 2.0 / (r * r) * coef;
  alpha = (side < 0) ? (double)l / r : -(l + 1.0) / r;
}

struct FacShared {
  double2* Mx;     // [Nr][Nr] block being factorised (LU in place)
  double2* X;      // [Nr][kFacCols] right-hand-side chunk
  double* S;       // [Nr] row scales
  double* a2[2];   // [Nr] coupling row factors, side -1 / +1
  double* al[2];   // [Nr] coupling radial factors
  int* piv;        // [Nr]
  double* red;     // [kFacThreads / 32] reduction scratch
  int* redi;       // [kFacThreads / 32]
};

__device__ FacShared fac_shared(void* base, int Nr) {
  FacShared s;
  char* p = static_cast<char*>(base);
  s.Mx = reinterpret_cast<double2*>(p);
  p += (size_t)Nr * Nr * sizeof(double2);
  s.X = reinterpret_cast<double2*>(p);
  p += (size_t)Nr * kFacCols * sizeof(double2);
  s.S = reinterpret_cast<double*>(p);
  p += Nr * sizeof(double);
  for (int q = 0; q < 2; ++q) {
    s.a2[q] = reinterpret_cast<double*>(p);
    p += Nr * sizeof(double);
    s.al[q] = reinterpret_cast<double*>(p);
    p += Nr * sizeof(double);
  }
  s.red = reinterpret_cast<double*>(p);
  p += (kFacThreads / 32) * sizeof(double);
  s.piv = reinterpret_cast<int*>(p);
  p += Nr * sizeof(int);
  s.redi = reinterpret_cast<int*>(p);
  return s;
}

inline size_t fac_smem_bytes(int Nr) {
  return (size_t)Nr * Nr * 16 + (size_t)Nr * kFacCols * 16 + 5 * (size_t)Nr * 8 +
         (kFacThreads / 32) * 8 + (size_t)Nr * 4 + (kFacThreads / 32) * 4 + 64;
}

// LU with partial pivoting of sh.Mx in place (the pivot of column q is the first row of
// largest modulus at or below q); returns false for a zero or non-finite pivot.
__device__ bool fac_lu(const FacShared& sh, int Nr) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int q = 0; q < Nr; ++q) {
    // pivot search over rows q..Nr-1 of column q
    double best = -1.0;
    int bi = Nr;
    for (int r = q + tid; r < Nr; r += kFacThreads) {
      const double v = fx_abs(sh.Mx[(size_t)r * Nr + q]);
      if (v > best) {
        best = v;
        bi = r;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      sh.red[warp] = best;
      sh.redi[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double b = -1.0;
      int p = Nr;
      for (int w = 0; w < kFacThreads / 32; ++w)
        if (sh.red[w] > b || (sh.red[w] == b && sh.redi[w] < p)) {
          b = sh.red[w];
          p = sh.redi[w];
        }
      sh.piv[q] = (b > 0.0 && isfinite(b)) ? p : -1;
    }
    __syncthreads();
    const int p = sh.piv[q];
    if (p < 0) return false;
    if (p != q)
      for (int k = tid; k < Nr; k += kFacThreads) {
        const double2 t = sh.Mx[(size_t)q * Nr + k];
        sh.Mx[(size_t)q * Nr + k] = sh.Mx[(size_t)p * Nr + k];
        sh.Mx[(size_t)p * Nr + k] = t;
      }
    __syncthreads();
    const double2 inv = fx_inv(sh.Mx[(size_t)q * Nr + q]);
    for (int r = q + 1 + tid; r < Nr; r += kFacThreads)
      sh.Mx[(size_t)r * Nr + q] = fx_mul(sh.Mx[(size_t)r * Nr + q], inv);
    __syncthreads();
    const int w = Nr - q - 1;
    for (int e = tid; e < w * w; e += kFacThreads) {
      const int r = q + 1 + e / w, k = q + 1 + e % w;
      sh.Mx[(size_t)r * Nr + k] =
          fx_sub_mul(sh.Mx[(size_t)r * Nr + k], sh.Mx[(size_t)r * Nr + q], sh.Mx[(size_t)q * Nr + k]);
    }
    __syncthreads();
  }
  return true;
}

// out = (LU)^-1 R with R given column chunk by column chunk by rhs(j, k) (complex), written
// row-major [Nr][Nr] to global memory.  Rows are permuted as the LU's pivots, then forward
// and back substitution run column-oriented on the chunk in shared memory.
template <typename Rhs>
__device__ void fac_solve(const FacShared& sh, int Nr, Rhs rhs, double2* __restrict__ out) {
  const int tid = threadIdx.x;
  for (int k0 = 0; k0 < Nr; k0 += kFacCols) {
    const int nc = min(kFacCols, Nr - k0);
    for (int e = tid; e < Nr * kFacCols; e += kFacThreads) {
      const int j = e / kFacCols, c = e % kFacCols;
      sh.X[e] = (c < nc) ? rhs(j, k0 + c) : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int q = 0; q < Nr; ++q) {   // the LU's row interchanges, in order
      const int p = sh.piv[q];
      if (p != q && tid < kFacCols) {
        const double2 t = sh.X[q * kFacCols + tid];
        sh.X[q * kFacCols + tid] = sh.X[p * kFacCols + tid];
        sh.X[p * kFacCols + tid] = t;
      }
      __syncthreads();
    }
    for (int q = 0; q < Nr - 1; ++q) {   // L y = P r (unit diagonal)
      const int w = Nr - q - 1;
      for (int e = tid; e < w * kFacCols; e += kFacThreads) {
        const int r = q + 1 + e / kFacCols, c = e % kFacCols;
        sh.X[r * kFacCols + c] =
            fx_sub_mul(sh.X[r * kFacCols + c], sh.Mx[(size_t)r * Nr + q], sh.X[q * kFacCols + c]);
      }
      __syncthreads();
    }
    for (int q = Nr - 1; q >= 0; --q) {  // U x = y
      if (tid < kFacCols)
        sh.X[q * kFacCols + tid] = fx_mul(sh.X[q * kFacCols + tid], fx_inv(sh.Mx[(size_t)q * Nr + q]));
      __syncthreads();
      for (int e = tid; e < q * kFacCols; e += kFacThreads) {
        const int r = e / kFacCols, c = e % kFacCols;
        sh.X[r * kFacCols + c] =
            fx_sub_mul(sh.X[r * kFacCols + c], sh.Mx[(size_t)r * Nr + q], sh.X[q * kFacCols + c]);
      }
      __syncthreads();
    }
    for (int e = tid; e < Nr * nc; e += kFacThreads) {
      const int j = e / nc, c = e % nc;
      out[(size_t)j * Nr + k0 + c] = sh.X[j * kFacCols + c];
    }
    __syncthreads();
  }
}

// One block of chain c: build D' (minus the couplings times W of the neighbouring blocks
// given), equilibrate, factorise, and write G, H, W.  prevLo / prevHi: W of block i - 1 /
// i + 1 to subtract (nullptr: none); hSide: the coupling whose solve goes to H (0: none),
// wSide: the coupling whose solve goes to W (0: none).
__device__ bool fac_block(const FacGeom& g, const FacShared& sh, int c, int i,
                          const double2* prevLo, const double2* prevHi, int hSide, int wSide,
                          double2* G, double2* H, double2* W) {
  const int Nr = g.Nr, tid = threadIdx.x;
  const int a = c >> 1, cls = c & 1;
  const int m = g.m_of[a];
  const int l = m + i;
  const int nb = g.L - m + 1;
  const int fld = ((i + cls) & 1) ? 1 : 0;
  // coupling row factors, and row scales over D and both couplings present in the chain
  for (int j = tid; j < Nr; j += kFacThreads) {
    double a2, al;
    fac_coupling_row(g, fld, l, m, -1, j, a2, al);
    if (i == 0) a2 = 0.0;
    sh.a2[0][j] = a2;
    sh.al[0][j] = al;
    fac_coupling_row(g, fld, l, m, +1, j, a2, al);
    if (i == nb - 1) a2 = 0.0;
    sh.a2[1][j] = a2;
    sh.al[1][j] = al;
  }
  __syncthreads();
  for (int j = tid; j < Nr; j += kFacThreads) {
    double mx = 0.0;
    for (int k = 0; k < Nr; ++k) {
      mx = fmax(mx, fx_abs(fac_diag(g, fld, l, m, j, k)));
      const double e0 = g.E0[(size_t)j * Nr + k], e1 = g.E1[(size_t)j * Nr + k];
      mx = fmax(mx, fabs(sh.a2[0][j] * (sh.al[0][j] * e0 - e1)));
      mx = fmax(mx, fabs(sh.a2[1][j] * (sh.al[1][j] * e0 - e1)));
    }
    sh.S[j] = 1.0 / mx;
  }
  __syncthreads();
  // D' = D - A W_{i-1} - C W_{i+1}, rows scaled: (A W)(j, k) = a2_j (al_j (E0 W) - (E1 W))
  for (int e = tid; e < Nr * Nr; e += kFacThreads) {
    const int j = e / Nr, k = e % Nr;
    double2 d = fac_diag(g, fld, l, m, j, k);
    for (int side = 0; side < 2; ++side) {
      const double2* Wp = side == 0 ? prevLo : prevHi;
      const double a2 = sh.a2[side][j];
      if (!Wp || a2 == 0.0) continue;
      double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
      const double* e0r = g.E0 + (size_t)j * Nr;
      const double* e1r = g.E1 + (size_t)j * Nr;
      for (int q = 0; q < Nr; ++q) {
        const double2 w = Wp[(size_t)q * Nr + k];
        s0.x = fma(e0r[q], w.x, s0.x);
        s0.y = fma(e0r[q], w.y, s0.y);
        s1.x = fma(e1r[q], w.x, s1.x);
        s1.y = fma(e1r[q], w.y, s1.y);
      }
      const double al = sh.al[side][j];
      d.x -= a2 * (al * s0.x - s1.x);
      d.y -= a2 * (al * s0.y - s1.y);
    }
    const double sj = sh.S[j];
    sh.Mx[e] = make_double2(d.x * sj, d.y * sj);
  }
  __syncthreads();
  if (!fac_lu(sh, Nr)) return false;
  const double* S = sh.S;
  fac_solve(sh, Nr, [&](int j, int k) { return make_double2(j == k ? S[j] : 0.0, 0.0); }, G);
  auto coupling_rhs = [&](int side) {
    const int q = side < 0 ? 0 : 1;
    return [&, q](int j, int k) {
      const double a2 = sh.a2[q][j];
      if (a2 == 0.0) return make_double2(0.0, 0.0);
      return make_double2(S[j] * a2 * (sh.al[q][j] * g.E0[(size_t)j * Nr + k] - g.E1[(size_t)j * Nr + k]),
                          0.0);
    };
  };
  if (hSide) fac_solve(sh, Nr, coupling_rhs(hSide), H);
  if (wSide) fac_solve(sh, Nr, coupling_rhs(wSide), W);
  return true;
}

// Half sweeps: blockIdx.x = 2 c + half; half 0 factorises blocks 0..km-1 top-down, half 1
// blocks nb-1..km+1 bottom-up.  status[c] is set to 1 on a singular block.
__global__ void __launch_bounds__(kFacThreads) k_factor_half(FacGeom g, double2* G, double2* H,
                                                             double2* W, int* status) {
  extern __shared__ __align__(16) unsigned char fac_smem[];
  const FacShared sh = fac_shared(fac_smem, g.Nr);
  const int c = blockIdx.x >> 1, half = blockIdx.x & 1;
  const int m = g.m_of[c >> 1];
  const int nb = g.L - m + 1, km = (nb - 1) / 2;
  const size_t blk = (size_t)g.Nr * g.Nr;
  const long off = g.chain_off[c];
  if (half == 0) {
    for (int i = 0; i < km; ++i) {
      const double2* prev = i > 0 ? W + (off + i - 1) * blk : nullptr;
      if (!fac_block(g, sh, c, i, prev, nullptr, i > 0 ? -1 : 0, +1, G + (off + i) * blk,
                     H + (off + i) * blk, W + (off + i) * blk)) {
        if (threadIdx.x == 0) status[c] = 1;
        return;
      }
    }
  } else {
    for (int i = nb - 1; i > km; --i) {
      const double2* prev = i < nb - 1 ? W + (off + i + 1) * blk : nullptr;
      if (!fac_block(g, sh, c, i, nullptr, prev, i < nb - 1 ? +1 : 0, -1, G + (off + i) * blk,
                     H + (off + i) * blk, W + (off + i) * blk)) {
        if (threadIdx.x == 0) status[c] = 1;
        return;
      }
    }
  }
}

// Middle blocks, one CTA per chain (after k_factor_half).
__global__ void __launch_bounds__(kFacThreads) k_factor_mid(FacGeom g, double2* G, double2* H,
                                                            double2* W, int* status) {
  extern __shared__ __align__(16) unsigned char fac_smem[];
  const FacShared sh = fac_shared(fac_smem, g.Nr);
  const int c = blockIdx.x;
  const int m = g.m_of[c >> 1];
  const int nb = g.L - m + 1, km = (nb - 1) / 2;
  const size_t blk = (size_t)g.Nr * g.Nr;
  const long off = g.chain_off[c];
  const double2* lo = km > 0 ? W + (off + km - 1) * blk : nullptr;
  const double2* hi = km < nb - 1 ? W + (off + km + 1) * blk : nullptr;
  if (!fac_block(g, sh, c, km, lo, hi, km > 0 ? -1 : 0, km < nb - 1 ? +1 : 0, G + (off + km) * blk,
                 H + (off + km) * blk, W + (off + km) * blk))
    if (threadIdx.x == 0) status[c] = 1;
}

// Temperature: Tinv_l = (S T_l)^-1 S per degree l (real), one CTA per l; the block is the
// real part of the shared-memory matrix (imaginary parts zero).
__global__ void __launch_bounds__(kFacThreads) k_factor_temp(FacGeom g, double* Tinv, int* status) {
  extern __shared__ __align__(16) unsigned char fac_smem[];
  const FacShared sh = fac_shared(fac_smem, g.Nr);
  const int Nr = g.Nr, l = blockIdx.x, tid = threadIdx.x;
  const double lam = l * (l + 1.0);
  auto entry = [&](int j, int k) {
    if (j == 0) return g.E0[k];
    if (j == Nr - 1) return g.E0[(size_t)(Nr - 1) * Nr + k];
    const size_t jk = (size_t)j * Nr + k;
    const double r = g.rc[j];
    return g.inv_dt * g.E0[jk] - (1.0 / g.Pr) * (g.E2[jk] + 2.0 / r * g.E1[jk] - lam / (r * r) * g.E0[jk]);
  };
  for (int j = tid; j < Nr; j += kFacThreads) {
    double mx = 0.0;
    for (int k = 0; k < Nr; ++k) mx = fmax(mx, fabs(entry(j, k)));
    sh.S[j] = 1.0 / mx;
  }
  __syncthreads();
  for (int e = tid; e < Nr * Nr; e += kFacThreads)
    sh.Mx[e] = make_double2(entry(e / Nr, e % Nr) * sh.S[e / Nr], 0.0);
  __syncthreads();
  if (!fac_lu(sh, Nr)) {
    if (tid == 0) status[0] = 1;
    return;
  }
  // solve into a complex scratch chunk, keep the real parts
  for (int k0 = 0; k0 < Nr; k0 += kFacCols) {
    const int nc = min(kFacCols, Nr - k0);
    for (int e = tid; e < Nr * kFacCols; e += kFacThreads) {
      const int j = e / kFacCols, cc = e % kFacCols;
      sh.X[e] = make_double2((cc < nc && j == k0 + cc) ? sh.S[j] : 0.0, 0.0);
    }
    __syncthreads();
    for (int q = 0; q < Nr; ++q) {
      const int p = sh.piv[q];
      if (p != q && tid < kFacCols) {
        const double2 t = sh.X[q * kFacCols + tid];
        sh.X[q * kFacCols + tid] = sh.X[p * kFacCols + tid];
        sh.X[p * kFacCols + tid] = t;
      }
      __syncthreads();
    }
    for (int q = 0; q < Nr - 1; ++q) {
      const int w = Nr - q - 1;
      for (int e = tid; e < w * kFacCols; e += kFacThreads) {
        const int r = q + 1 + e / kFacCols, cc = e % kFacCols;
        sh.X[r * kFacCols + cc].x =
            fma(-sh.Mx[(size_t)r * Nr + q].x, sh.X[q * kFacCols + cc].x, sh.X[r * kFacCols + cc].x);
      }
      __syncthreads();
    }
    for (int q = Nr - 1; q >= 0; --q) {
      if (tid < kFacCols) sh.X[q * kFacCols + tid].x /= sh.Mx[(size_t)q * Nr + q].x;
      __syncthreads();
      for (int e = tid; e < q * kFacCols; e += kFacThreads) {
        const int r = e / kFacCols, cc = e % kFacCols;
        sh.X[r * kFacCols + cc].x =
            fma(-sh.Mx[(size_t)r * Nr + q].x, sh.X[q * kFacCols + cc].x, sh.X[r * kFacCols + cc].x);
      }
      __syncthreads();
    }
    for (int e = tid; e < Nr * nc; e += kFacThreads) {
      const int j = e / nc, cc = e % nc;
      Tinv[(size_t)l * Nr * Nr + (size_t)j * Nr + k0 + cc] = sh.X[j * kFacCols + cc].x;
    }
    __syncthreads();
  }
}

// Residual of the e/f chains, for iterative refinement of the FP64 chain solve:
// r = b - (M/dt + K) x on the e and f rows (the operator of fac_diag / fac_coupling_row
// applied to x through the Chebyshev tables: D x needs E0 x, E1 x, E2 x, E4 x of the
// pair's own coefficients, the couplings E0 x and E1 x of the other potential at l - 1 and
// l + 1), in place over rb (b on entry, r on exit); the temperature rows are set to 0.
// The block Thomas sweeps multiply by explicit block inverses, which is not backward
// stable: at Ek = 1e-5 the small poloidal field f of the m = 0 chains can carry relative
// errors of 1e-8.  One refinement step x += solve(r) with this FP64 residual brings the
// solution to the accuracy of a pivoted banded LU (1e-15 on the same chains).
// grid = P (one CTA per pair), block = (round32(Nr), 2): threadIdx.y = field e / f.
__global__ void k_chain_residual(FacGeom g, const int* __restrict__ pair_l,
                                 const int* __restrict__ pair_m, int P,
                                 const double2* __restrict__ x, double2* __restrict__ rb) {
  extern __shared__ double2 xs_[];   // [fld][pair offset -1, 0, +1][Nr]
  const int Nr = g.Nr, p = blockIdx.x;
  const int l = pair_l[p], m = pair_m[p];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  for (int idx = tid; idx < 6 * Nr; idx += nt) {
    const int fld = idx / (3 * Nr), o = (idx / Nr) % 3 - 1, k = idx % Nr;
    const int l2 = l + o;
    double2 v = make_double2(0.0, 0.0);
    if (l2 >= m && l2 <= g.L) v = x[((long)fld * P + p + o) * Nr + k];
    xs_[idx] = v;
  }
  __syncthreads();
  const int j = threadIdx.x, fld = threadIdx.y;
  if (j >= Nr) return;
  const long row = ((long)fld * P + p) * Nr + j;
  if (fld == 0) rb[((long)2 * P + p) * Nr + j] = make_double2(0.0, 0.0);
  const double2* xo = xs_ + (fld * 3 + 1) * Nr;   // own coefficients at l
  double2 Ax;
  if (l == 0) {
    Ax = xo[j];
  } else {
    double2 e0 = {0, 0}, e1 = {0, 0}, e2 = {0, 0}, e4 = {0, 0};
    // rows of the tables: interior rows use row j; the boundary rows their wall rows
    const bool bc = (j == 0 || j == Nr - 1) || (fld == 1 && (j == 1 || j == Nr - 2));
    const int jr = (j <= 1) ? 0 : (j >= Nr - 2 ? Nr - 1 : j);
    const int rr = bc ? jr : j;
    for (int k = 0; k < Nr; ++k) {
      const size_t rk = (size_t)rr * Nr + k;
      const double2 v = xo[k];
      const double c0 = g.E0[rk], c1 = g.E1[rk];
      e0.x = fma(c0, v.x, e0.x); e0.y = fma(c0, v.y, e0.y);
      e1.x = fma(c1, v.x, e1.x); e1.y = fma(c1, v.y, e1.y);
      if (!bc) {
        const double c2 = g.E2[rk], c4 = g.E4[rk];
        e2.x = fma(c2, v.x, e2.x); e2.y = fma(c2, v.y, e2.y);
        e4.x = fma(c4, v.x, e4.x); e4.y = fma(c4, v.y, e4.y);
      }
    }
    if (bc) {
      Ax = (j == 0 || j == Nr - 1) ? e0 : e1;   // f: rows 1, Nr - 2 hold d_r f at the walls
    } else {
      const double r = g.rc[j], r2 = r * r, lam = l * (l + 1.0), mk = lam * g.Ek / r2;
      const double2 Ll = make_double2(e2.x - lam / r2 * e0.x, e2.y - lam / r2 * e0.y);
      if (fld == 0) {
        const double cm = g.explicit_coriolis ? 0.0 : -2.0 * m / r2;   // times i e
        Ax = make_double2(mk * g.inv_dt * e0.x - mk * Ll.x - cm * e0.y,
                          mk * g.inv_dt * e0.y - mk * Ll.y + cm * e0.x);
      } else {
        const double c2 = -2.0 * lam / r2, c1 = 4.0 * lam / (r2 * r), c0 = (lam * lam - 6.0 * lam) / (r2 * r2);
        const double2 LL = make_double2(e4.x + c2 * e2.x + c1 * e1.x + c0 * e0.x,
                                        e4.y + c2 * e2.y + c1 * e1.y + c0 * e0.y);
        const double cm = g.explicit_coriolis ? 0.0 : 2.0 * m / r2;     // times i Ll f
        Ax = make_double2(-mk * g.inv_dt * Ll.x + mk * LL.x - cm * Ll.y,
                          -mk * g.inv_dt * Ll.y + mk * LL.y + cm * Ll.x);
      }
      // Coriolis couplings to the other potential at l - 1 and l + 1
      for (int side = -1; side <= 1; side += 2) {
        if ((side < 0 && l - 1 < m) || (side > 0 && l + 1 > g.L)) continue;
        double a2, al;
        fac_coupling_row(g, fld, l, m, side, j, a2, al);
        if (a2 == 0.0) continue;
        const double2* xn = xs_ + ((1 - fld) * 3 + 1 + side) * Nr;
        double2 n0 = {0, 0}, n1 = {0, 0};
        for (int k = 0; k < Nr; ++k) {
          const size_t jk = (size_t)j * Nr + k;
          const double c0 = g.E0[jk], c1 = g.E1[jk];
          n0.x = fma(c0, xn[k].x, n0.x); n0.y = fma(c0, xn[k].y, n0.y);
          n1.x = fma(c1, xn[k].x, n1.x); n1.y = fma(c1, xn[k].y, n1.y);
        }
        Ax.x += a2 * (al * n0.x - n1.x);
        Ax.y += a2 * (al * n0.y - n1.y);
      }
    }
  }
  const double2 b = rb[row];
  rb[row] = make_double2(b.x - Ax.x, b.y - Ax.y);
}

// Double-float copies of the factors for the mixed path: hi = the entry rounded to FP32,
// lo = the remainder rounded to FP32 (as the host split).
__global__ void k_split_factor(const double2* __restrict__ src, float4* __restrict__ dst, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    const float rh = (float)v.x, ih = (float)v.y;
    dst[i] = make_float4(rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih));
  }
}

}  // namespace rsc
