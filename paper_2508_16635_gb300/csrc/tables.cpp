// Host-side FP64 construction of the tables and of the block-tridiagonal
// factorisation of the implicit operator.
//
// Radial: Chebyshev polynomials of x = 2r - r_in - r_out on Gauss-Lobatto
// points (Sec. 3.1, Eq. expansion; 3/2-rule de-aliasing).  Derivatives are
// taken exactly in coefficient space and evaluated with cos(k theta_j).
// Angular: Gauss-Legendre nodes by Newton's method on P_n; normalised
// associated Legendre functions of Eq. Ylm_norm by the three-term recursion in
// l, with d/dtheta from the recursion Eq. recu1.
// Implicit operator: Eqs. impcor_e_final and impcor_f_final (diffusion and
// Coriolis on the left-hand side), the temperature equation Eq. temp, with
// boundary rows replacing the rows at the walls (Sec. 3.1).
#include <algorithm>
#include <climits>
#include <cmath>
#include <stdexcept>
#include <thread>

#include "rsc_internal.h"

namespace rsc {

static const double kPi = 3.14159265358979323846;

static int nlat_for(int L) { return 2 * ((3 * (L + 1) + 3) / 4); }

static int nphi_for(int L, int Ms) {
  const long need = 3L * (L / Ms) + 1;
  long best = LONG_MAX;
  for (long a = 1; a < 4 * need; a *= 2)
    for (long b = a; b < 4 * need; b *= 3)
      if (b >= need && b < best) best = b;
  return (int)best;
}

void build_dims(const rsc_params& p, Dims& d) {
  d.L = p.L;
  d.Ms = p.Ms;
  d.Nr = p.Nr;
  d.Nd = (3 * p.Nr + 1) / 2;
  d.nlat = nlat_for(p.L);
  d.nlat2 = d.nlat / 2;
  d.nphi = nphi_for(p.L, p.Ms);
  d.nm = p.L / p.Ms + 1;
  d.K = d.nm - 1;
  d.P = 0;
  for (int a = 0; a < d.nm; ++a) d.P += p.L - a * p.Ms + 1;
  d.r_out = 1.0 / (1.0 - p.eta);
  d.r_in = p.eta / (1.0 - p.eta);
}

// Coefficients of d/dx of a Chebyshev series a[0..n-1].
static void cheb_derivative(const std::vector<double>& a, std::vector<double>& b) {
  const int n = (int)a.size();
  b.assign(n, 0.0);
  if (n < 2) return;
  std::vector<double> c(n + 1, 0.0);
  for (int k = n - 1; k >= 1; --k) c[k - 1] = c[k + 1] + 2.0 * k * a[k];
  for (int k = 0; k < n; ++k) b[k] = c[k];
  b[0] *= 0.5;
}

// out[j][k] = d^order T_k / dr^order at x_j = cos(pi j / (npts - 1)), k < nk.
static void cheb_table(int npts, int nk, int order, double r_in, double r_out,
                       std::vector<double>& out) {
  out.assign((size_t)npts * nk, 0.0);
  const double scale = std::pow(2.0 / (r_out - r_in), order);
  std::vector<double> a(nk), b;
  for (int k = 0; k < nk; ++k) {
    std::fill(a.begin(), a.end(), 0.0);
    a[k] = 1.0;
    for (int o = 0; o < order; ++o) {
      cheb_derivative(a, b);
      a = b;
    }
    for (int j = 0; j < npts; ++j) {
      const double th = kPi * j / (npts - 1);
      double s = 0.0;
      for (int q = 0; q < nk; ++q)
        if (a[q] != 0.0) s += a[q] * std::cos(q * th);
      out[(size_t)j * nk + k] = s * scale;
    }
  }
}

// Gauss-Legendre rule, north (x ~ +1) first.  Newton's method on P_n runs in
// long double (64- or 113-bit significand) and the node and weight are rounded
// to double at the end: in double arithmetic, P_n' is so large near the poles
// that the rounding of x alone puts 1e-10 relative errors into those weights
// at n = 384.  Weight w = 2 (1 - x^2) / (n P_{n-1}(x))^2, valid at a root.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  auto bonnet = [n](long double z, long double& pn, long double& pm) {
    long double p0 = 1.0L, p1 = z;
    for (int k = 1; k < n; ++k) {
      const long double p2 = ((2.0L * k + 1.0L) * z * p1 - (long double)k * p0) / (k + 1.0L);
      p0 = p1;
      p1 = p2;
    }
    pn = p1;
    pm = p0;
  };
  for (int i = 0; i < (n + 1) / 2; ++i) {
    long double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    long double pn = 0.0L, pm = 0.0L;
    for (int it = 0; it < 100; ++it) {
      bonnet(z, pn, pm);
      const long double dp = n * (pm - z * pn) / ((1.0L - z) * (1.0L + z));
      const long double dz = pn / dp;
      z -= dz;
      if (std::fabs((double)dz) < 1e-30) break;
    }
    bonnet(z, pn, pm);
    const long double wi = 2.0L * (1.0L - z) * (1.0L + z) / ((n * pm) * (n * pm));
    x[i] = (double)z;
    w[i] = (double)wi;
    x[n - 1 - i] = -x[i];
    w[n - 1 - i] = w[i];
  }
  if (n % 2) x[n / 2] = 0.0;
}

// Normalised P_l^m (Eq. Ylm_norm, no Condon-Shortley phase) for l = m..lmax at
// one node x with s = sqrt(1 - x^2).  The start s^m prod sqrt((2k+1)/2k) leaves
// the double range near the poles for large m, so the recursion carries an
// extra exponent: values are rescaled by exact powers 2^+-500 and put back
// with ldexp, which gives 0 where the true value is below the double range
// and full precision elsewhere.
static void legendre_column(int lmax, int m, double x, double s, std::vector<double>& out) {
  out.assign(lmax - m + 1, 0.0);
  const double norm = (m > 0) ? std::sqrt(2.0) : 1.0;
  long E = 0;  // true value = stored * 2^E
  double v1 = 1.0;
  for (int k = 1; k <= m; ++k) {
    v1 *= s * std::sqrt((2.0 * k + 1.0) / (2.0 * k));
    if (v1 != 0.0 && std::fabs(v1) < 0x1p-500) {
      v1 = std::ldexp(v1, 500);
      E -= 500;
    }
  }
  auto put = [&](int q, double v) {
    out[q] = (E < -2200) ? 0.0 : norm * std::ldexp(v, (int)E);
  };
  put(0, v1);
  if (lmax == m) return;
  double v0 = v1;
  v1 = x * std::sqrt(2.0 * m + 3.0) * v0;
  put(1, v1);
  for (int l = m + 2; l <= lmax; ++l) {
    const double a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
    const double b = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) /
                               (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
    const double v2 = a * (x * v1 - b * v0);
    v0 = v1;
    v1 = v2;
    if (E < 0 && std::fabs(v1) > 0x1p500) {
      v0 = std::ldexp(v0, -500);
      v1 = std::ldexp(v1, -500);
      E += 500;
    }
    put(l - m, v1);
  }
}

void build_tables(const rsc_params& p, const Dims& d, HostTables& t) {
  const int Nr = d.Nr, Nd = d.Nd;
  t.rc.resize(Nr);
  t.rd.resize(Nd);
  for (int j = 0; j < Nr; ++j)
    t.rc[j] = d.r_in + 0.5 * (std::cos(kPi * j / (Nr - 1)) + 1.0) * (d.r_out - d.r_in);
  for (int i = 0; i < Nd; ++i)
    t.rd[i] = d.r_in + 0.5 * (std::cos(kPi * i / (Nd - 1)) + 1.0) * (d.r_out - d.r_in);
  for (int o = 0; o < 5; ++o) cheb_table(Nr, Nr, o, d.r_in, d.r_out, t.Ec[o]);
  for (int o = 0; o < 3; ++o) cheb_table(Nd, Nr, o, d.r_in, d.r_out, t.Ed[o]);
  // Interpolation on the N_d Gauss-Lobatto radii (DCT-I), truncated to k < Nr.
  const int N = Nd - 1;
  std::vector<double> Cm((size_t)Nr * Nd);
  for (int k = 0; k < Nr; ++k) {
    const double gk = (k == 0 || k == N) ? 2.0 : 1.0;
    for (int i = 0; i < Nd; ++i) {
      const double gi = (i == 0 || i == N) ? 2.0 : 1.0;
      Cm[(size_t)k * Nd + i] = 2.0 / (N * gk * gi) * std::cos(kPi * (double)k * i / N);
    }
  }
  t.R0.assign((size_t)Nr * Nd, 0.0);
  t.R1.assign((size_t)Nr * Nd, 0.0);
  for (int j = 0; j < Nr; ++j)
    for (int i = 0; i < Nd; ++i) {
      double s0 = 0.0, s1 = 0.0;
      for (int k = 0; k < Nr; ++k) {
        s0 += t.Ec[0][(size_t)j * Nr + k] * Cm[(size_t)k * Nd + i];
        s1 += t.Ec[1][(size_t)j * Nr + k] * Cm[(size_t)k * Nd + i];
      }
      t.R0[(size_t)j * Nd + i] = s0;
      t.R1[(size_t)j * Nd + i] = s1;
    }
  // Angular tables.
  gauss_legendre(d.nlat, t.xlat, t.wlat);
  t.m_of.resize(d.nm);
  t.pstart.resize(d.nm + 1);
  t.pair_l.clear();
  t.pair_m.clear();
  t.leg_off.resize(d.nm + 1);
  long off = 0;
  for (int a = 0; a < d.nm; ++a) {
    const int m = a * d.Ms;
    t.m_of[a] = m;
    t.pstart[a] = (int)t.pair_l.size();
    for (int l = m; l <= d.L; ++l) {
      t.pair_l.push_back(l);
      t.pair_m.push_back(m);
    }
    t.leg_off[a] = off;
    off += (long)(d.L - m + 1) * d.nlat2;
  }
  t.pstart[d.nm] = d.P;
  t.leg_off[d.nm] = off;
  t.P.assign(off, 0.0);
  t.dP.assign(off, 0.0);
  t.Ps.assign(off, 0.0);
  t.Pw.assign(off, 0.0);
  t.dPw.assign(off, 0.0);
  t.Psw.assign(off, 0.0);
  std::vector<double> col;
  for (int a = 0; a < d.nm; ++a) {
    const int m = t.m_of[a];
    const int nl = d.L - m + 1;
    const double nrm = 2.0 * (m > 0 ? 2.0 : 1.0);  // int P^2 dx with Eq. Ylm_norm
    for (int tt = 0; tt < d.nlat2; ++tt) {
      const double x = t.xlat[tt];
      const double s = std::sqrt((1.0 - x) * (1.0 + x));
      legendre_column(d.L + 1, m, x, s, col);  // rows l = m..L+1
      for (int q = 0; q < nl; ++q) {
        const int l = m + q;
        const double cl = std::sqrt(((double)l * l - (double)m * m) / (4.0 * l * l - 1.0));
        const double cl1 = std::sqrt(((l + 1.0) * (l + 1.0) - (double)m * m) /
                                     (4.0 * (l + 1.0) * (l + 1.0) - 1.0));
        const double pm1 = (q > 0) ? col[q - 1] : 0.0;
        // Eq. recu1 in normalised form: sin th dP_l = l c_{l+1} P_{l+1} - (l+1) c_l P_{l-1}
        const double dpv = (l * cl1 * col[q + 1] - (l + 1.0) * cl * pm1) / s;
        const double pv = col[q];
        const size_t is = t.leg_off[a] + (size_t)q * d.nlat2 + tt;
        t.P[is] = pv;
        t.dP[is] = dpv;
        t.Ps[is] = pv / s;
        const size_t ia = t.leg_off[a] + (size_t)tt * nl + q;
        const double wn = t.wlat[tt] / nrm;
        t.Pw[ia] = wn * pv;
        t.dPw[ia] = wn * dpv;
        t.Psw[ia] = wn * pv / s;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Implicit operator blocks (rows at the collocation radii).
namespace {

struct Ops {
  const Dims& d;
  const HostTables& t;
  double Ek, Pr, inv_dt;
  int Nr;
  bool explicit_coriolis;  // Coriolis kept out of the implicit operator (Eqs. expcor_e/f)
  double E(int o, int j, int k) const { return t.Ec[o][(size_t)j * Nr + k]; }

  // field 0 = e, 1 = f
  void diag(int field, int l, int m, std::vector<cplx>& D) const {
    D.assign((size_t)Nr * Nr, cplx(0.0));
    if (l == 0) {
      for (int j = 0; j < Nr; ++j) D[(size_t)j * Nr + j] = 1.0;
      return;
    }
    const double lam = l * (l + 1.0);
    for (int j = 0; j < Nr; ++j) {
      const double r = t.rc[j];
      const double r2 = r * r;
      for (int k = 0; k < Nr; ++k) {
        const double e0 = E(0, j, k), e1 = E(1, j, k), e2 = E(2, j, k), e4 = E(4, j, k);
        cplx v;
        if (field == 0) {
          const double Ll = e2 - lam / r2 * e0;
          v = cplx(lam * Ek / r2 * inv_dt * e0 - lam * Ek / r2 * Ll,
                   explicit_coriolis ? 0.0 : -2.0 * m / r2 * e0);
        } else {
          const double Ll = e2 - lam / r2 * e0;
          const double LL = e4 - 2.0 * lam / r2 * e2 + 4.0 * lam / (r2 * r) * e1 +
                            (lam * lam - 6.0 * lam) / (r2 * r2) * e0;
          v = cplx(-lam * Ek / r2 * inv_dt * Ll + lam * Ek / r2 * LL,
                   explicit_coriolis ? 0.0 : 2.0 * m / r2 * Ll);
        }
        D[(size_t)j * Nr + k] = v;
      }
    }
    bc_rows(field, D);
  }

  void bc_rows(int field, std::vector<cplx>& D) const {
    auto setrow = [&](int j, int o, int src) {
      for (int k = 0; k < Nr; ++k) D[(size_t)j * Nr + k] = E(o, src, k);
    };
    setrow(0, 0, 0);
    setrow(Nr - 1, 0, Nr - 1);
    if (field == 1) {
      setrow(1, 1, 0);
      setrow(Nr - 2, 1, Nr - 1);
    }
  }

  // Coupling of the equation at l to the other potential at l + side (Coriolis).
  void coupling(int field, int l, int m, int side, std::vector<cplx>& B) const {
    B.assign((size_t)Nr * Nr, cplx(0.0));
    if (l == 0 || explicit_coriolis) return;
    double coef;
    if (side < 0) {
      coef = ((double)l * l - 1.0) * std::sqrt(((double)l * l - (double)m * m) / (4.0 * l * l - 1.0));
    } else {
      const double l1 = l + 1.0;
      coef = l * (l + 2.0) * std::sqrt((l1 * l1 - (double)m * m) / (4.0 * l1 * l1 - 1.0));
    }
    const int j0 = (field == 1) ? 2 : 1;
    const int j1 = (field == 1) ? Nr - 3 : Nr - 2;
    for (int j = j0; j <= j1; ++j) {
      const double r = t.rc[j];
      const double a = (side < 0) ? (double)l / r : -(l + 1.0) / r;
      for (int k = 0; k < Nr; ++k)
        B[(size_t)j * Nr + k] = 2.0 / (r * r) * coef * (a * E(0, j, k) - E(1, j, k));
    }
  }

  void temp(int l, std::vector<double>& D) const {
    D.assign((size_t)Nr * Nr, 0.0);
    const double lam = l * (l + 1.0);
    for (int j = 0; j < Nr; ++j) {
      const double r = t.rc[j];
      for (int k = 0; k < Nr; ++k)
        D[(size_t)j * Nr + k] = inv_dt * E(0, j, k) -
                                (1.0 / Pr) * (E(2, j, k) + 2.0 / r * E(1, j, k) - lam / (r * r) * E(0, j, k));
    }
    for (int k = 0; k < Nr; ++k) {
      D[k] = E(0, 0, k);
      D[(size_t)(Nr - 1) * Nr + k] = E(0, Nr - 1, k);
    }
  }
};

// LU with partial pivoting, in place (row-major n x n).  Returns false if singular.
template <typename T>
bool lu_factor(int n, std::vector<T>& A, std::vector<int>& piv) {
  piv.resize(n);
  for (int c = 0; c < n; ++c) {
    int best = c;
    double bv = std::abs(A[(size_t)c * n + c]);
    for (int r = c + 1; r < n; ++r) {
      const double v = std::abs(A[(size_t)r * n + c]);
      if (v > bv) {
        bv = v;
        best = r;
      }
    }
    if (bv == 0.0 || !std::isfinite(bv)) return false;
    piv[c] = best;
    if (best != c)
      for (int k = 0; k < n; ++k) std::swap(A[(size_t)c * n + k], A[(size_t)best * n + k]);
    const T inv = T(1.0) / A[(size_t)c * n + c];
    for (int r = c + 1; r < n; ++r) {
      const T f = A[(size_t)r * n + c] * inv;
      A[(size_t)r * n + c] = f;
      if (f != T(0.0))
        for (int k = c + 1; k < n; ++k) A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
    }
  }
  return true;
}

// Solve LU X = B for nrhs columns of B (row-major n x nrhs), in place.
template <typename T>
void lu_solve(int n, const std::vector<T>& LU, const std::vector<int>& piv, int nrhs,
              std::vector<T>& B) {
  for (int c = 0; c < n; ++c)
    if (piv[c] != c)
      for (int q = 0; q < nrhs; ++q)
        std::swap(B[(size_t)c * nrhs + q], B[(size_t)piv[c] * nrhs + q]);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < r; ++c) {
      const T f = LU[(size_t)r * n + c];
      if (f != T(0.0))
        for (int q = 0; q < nrhs; ++q) B[(size_t)r * nrhs + q] -= f * B[(size_t)c * nrhs + q];
    }
  for (int r = n - 1; r >= 0; --r) {
    for (int c = r + 1; c < n; ++c) {
      const T f = LU[(size_t)r * n + c];
      if (f != T(0.0))
        for (int q = 0; q < nrhs; ++q) B[(size_t)r * nrhs + q] -= f * B[(size_t)c * nrhs + q];
    }
    const T inv = T(1.0) / LU[(size_t)r * n + r];
    for (int q = 0; q < nrhs; ++q) B[(size_t)r * nrhs + q] *= inv;
  }
}

}  // namespace

// Spikes, reduced systems and index tables of partitioned chains (a SPIKE-type solve,
// HostFactor).  Part q of a chain has blocks s_q..e_q-1; its part-local factors are in
// G, H, W.  V_q = A_q^-1 [0; ...; C] is its response to the coupling of its last block to
// the next part's first block, Wsp_q = A_q^-1 [A; 0; ...] to the coupling of its first block
// to the previous part's last block.  With xl the part-local solution, every block obeys
//   x_i = xl_i - V_i x(s_{q+1}) - Wsp_i x(e_{q-1} - 1),
// and these relations at the blocks that couple parts (B_q = x(e_q - 1), T_{q+1} = x(s_{q+1}))
// form (I + K) z = xl_z, whose inverse is stored per chain.
static bool partition_extras(const Dims& d, const HostTables& t, const Ops& ops,
                             const std::vector<std::vector<int>>& cuts, HostFactor& f) {
  const int Nr = d.Nr;
  const size_t blk = (size_t)Nr * Nr;
  const int nchains = 2 * d.nm;
  const long nblk = f.chain_off[nchains];
  f.V.assign(nblk * blk, cplx(0.0));
  f.Wsp.assign(nblk * blk, cplx(0.0));
  f.blk_z.assign(nblk * 2, -1);
  f.parts.clear();
  f.red_off.assign(nchains, 0);
  f.red_nu.assign(nchains, 0);
  f.zoff.assign(nchains, 0);
  f.unk_row.clear();
  f.unk_chain.clear();
  long roff = 0;
  int z = 0;
  for (int c = 0; c < nchains; ++c) {
    const int a = c / 2, cls = c % 2, m = t.m_of[a];
    const int Pc = (int)cuts[c].size() - 1;
    for (int q = 0; q < Pc; ++q) {
      const int s = cuts[c][q], e = cuts[c][q + 1];
      f.parts.insert(f.parts.end(), {(long)(t.pstart[a] + s), (long)((cls + s) & 1), (long)(e - s),
                                     f.chain_off[c] + s, (long)m, (long)c});
    }
    const int nu = 2 * (Pc - 1);
    f.red_nu[c] = nu;
    f.zoff[c] = z;
    f.red_off[c] = roff;
    for (int u = 0; u < nu; ++u) {   // B_q (u = 2q): last block of part q; T_{q+1} (u = 2q+1)
      const int i = (u % 2 == 0) ? cuts[c][u / 2 + 1] - 1 : cuts[c][u / 2 + 1];
      const int fld = (i + cls) & 1;
      f.unk_row.push_back(((long)fld * d.P + t.pstart[a] + i) * Nr);
      f.unk_chain.push_back(c);
    }
    for (int q = 0; q < Pc; ++q)
      for (int i = cuts[c][q]; i < cuts[c][q + 1]; ++i) {
        const long g = f.chain_off[c] + i;
        f.blk_z[g * 2 + 0] = (q < Pc - 1) ? z + 2 * q + 1 : -1;
        f.blk_z[g * 2 + 1] = (q > 0) ? z + 2 * (q - 1) : -1;
      }
    z += nu;
    roff += (long)nu * Nr * nu * Nr;
  }
  f.red.assign(roff, cplx(0.0));

  auto mm_sub = [&](const cplx* A, const std::vector<cplx>& X, std::vector<cplx>& Y) {
    for (int r = 0; r < Nr; ++r)
      for (int k = 0; k < Nr; ++k) {
        const cplx x = A[(size_t)r * Nr + k];
        if (x == cplx(0.0)) continue;
        for (int q = 0; q < Nr; ++q) Y[(size_t)r * Nr + q] -= x * X[(size_t)k * Nr + q];
      }
  };
  auto mm = [&](const cplx* A, std::vector<cplx>& X) {   // X <- A X
    std::vector<cplx> Y(blk, cplx(0.0));
    for (int r = 0; r < Nr; ++r)
      for (int k = 0; k < Nr; ++k) {
        const cplx x = A[(size_t)r * Nr + k];
        if (x == cplx(0.0)) continue;
        for (int q = 0; q < Nr; ++q) Y[(size_t)r * Nr + q] += x * X[(size_t)k * Nr + q];
      }
    X.swap(Y);
  };
  // X[i - s] <- (part-local operator)^-1 X[i - s] with the part's twisted factors (the
  // order of the GPU sweeps: g = G b, half sweeps from both ends, middle, outward sweeps)
  auto part_solve = [&](int c, int s, int e, std::vector<std::vector<cplx>>& X) {
    const int km = s + (e - s - 1) / 2;
    auto at = [&](const std::vector<cplx>& v, int i) { return &v[(f.chain_off[c] + i) * blk]; };
    for (int i = s; i < e; ++i) mm(at(f.G, i), X[i - s]);
    for (int i = s + 1; i < km; ++i) mm_sub(at(f.H, i), X[i - 1 - s], X[i - s]);
    for (int i = e - 2; i > km; --i) mm_sub(at(f.H, i), X[i + 1 - s], X[i - s]);
    if (km > s) mm_sub(at(f.H, km), X[km - 1 - s], X[km - s]);
    if (km < e - 1) mm_sub(at(f.W, km), X[km + 1 - s], X[km - s]);
    for (int i = km - 1; i >= s; --i) mm_sub(at(f.W, i), X[i + 1 - s], X[i - s]);
    for (int i = km + 1; i < e; ++i) mm_sub(at(f.W, i), X[i - 1 - s], X[i - s]);
  };
  std::vector<int> bad(nchains, 0);
  auto work = [&](int c) {
    const int a = c / 2, cls = c % 2, m = t.m_of[a];
    const int Pc = (int)cuts[c].size() - 1;
    if (Pc < 2) return;
    auto field_of = [&](int i) { return ((i + cls) % 2 == 0) ? 0 : 1; };
    std::vector<cplx> B;
    for (int q = 0; q < Pc; ++q) {
      const int s = cuts[c][q], e = cuts[c][q + 1];
      for (int side = 0; side < 2; ++side) {
        if ((side == 0 && q == Pc - 1) || (side == 1 && q == 0)) continue;
        std::vector<std::vector<cplx>> X(e - s, std::vector<cplx>(blk, cplx(0.0)));
        if (side == 0) {   // coupling of block e-1 to block e (the next part's first)
          ops.coupling(field_of(e - 1), m + e - 1, m, +1, B);
          X[e - 1 - s] = B;
        } else {           // coupling of block s to block s-1 (the previous part's last)
          ops.coupling(field_of(s), m + s, m, -1, B);
          X[0] = B;
        }
        part_solve(c, s, e, X);
        std::vector<cplx>& dst = side == 0 ? f.V : f.Wsp;
        for (int i = s; i < e; ++i)
          std::copy(X[i - s].begin(), X[i - s].end(), &dst[(f.chain_off[c] + i) * blk]);
      }
    }
    // (I + K) z = xl_z over the nu unknown blocks, inverted
    const int nu = f.red_nu[c], n = nu * Nr;
    std::vector<cplx> M((size_t)n * n, cplx(0.0)), I((size_t)n * n, cplx(0.0));
    for (int r = 0; r < n; ++r) M[(size_t)r * n + r] = I[(size_t)r * n + r] = 1.0;
    for (int u = 0; u < nu; ++u) {
      const int q = (u % 2 == 0) ? u / 2 : u / 2 + 1;     // the part of unknown u
      const int i = (u % 2 == 0) ? cuts[c][u / 2 + 1] - 1 : cuts[c][u / 2 + 1];
      const long g = f.chain_off[c] + i;
      for (int side = 0; side < 2; ++side) {
        const int uc = side == 0 ? (q < Pc - 1 ? 2 * q + 1 : -1) : (q > 0 ? 2 * (q - 1) : -1);
        if (uc < 0) continue;
        const cplx* S = &(side == 0 ? f.V : f.Wsp)[g * blk];
        for (int r = 0; r < Nr; ++r)
          for (int k = 0; k < Nr; ++k) M[(size_t)(u * Nr + r) * n + uc * Nr + k] += S[(size_t)r * Nr + k];
      }
    }
    std::vector<int> piv;
    if (!lu_factor(n, M, piv)) {
      bad[c] = 1;
      return;
    }
    lu_solve(n, M, piv, n, I);
    std::copy(I.begin(), I.end(), f.red.begin() + f.red_off[c]);
  };
  const int nth = std::max(1, std::min<int>(nchains, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int w = 0; w < nth; ++w)
    pool.emplace_back([&, w]() {
      for (int c = w; c < nchains; c += nth) work(c);
    });
  for (auto& th : pool) th.join();
  for (int c = 0; c < nchains; ++c)
    if (bad[c]) return false;
  return true;
}

int build_factor(const rsc_params& p, const Dims& d, const HostTables& t, double dt,
                 HostFactor& f, int nparts) {
  const int Nr = d.Nr;
  const size_t blk = (size_t)Nr * Nr;
  Ops ops{d, t, p.Ek, p.Pr, std::isfinite(dt) ? 1.0 / dt : 0.0, Nr, p.explicit_coriolis != 0};
  f.dt = dt;
  const int nchains = 2 * d.nm;
  f.chain_off.resize(nchains + 1);
  long off = 0;
  for (int c = 0; c < nchains; ++c) {
    f.chain_off[c] = off;
    off += d.L - t.m_of[c / 2] + 1;
  }
  f.chain_off[nchains] = off;
  f.G.assign(off * blk, cplx(0.0));
  f.H.assign(off * blk, cplx(0.0));
  f.W.assign(off * blk, cplx(0.0));
  std::vector<int> bad(nchains, 0);
  // part boundaries of each chain: Pc parts of at least 8 blocks (one part: the whole chain)
  std::vector<std::vector<int>> cuts(nchains);
  for (int c = 0; c < nchains; ++c) {
    const int nb = d.L - t.m_of[c / 2] + 1;
    const int Pc = std::max(1, std::min(std::max(1, nparts), nb / 8));
    for (int q = 0; q <= Pc; ++q) cuts[c].push_back((int)((long)q * nb / Pc));
  }

  // Twisted block factorisation of the blocks s..e-1 of a chain (the whole chain, or one
  // part of it): blocks s..k-1 are eliminated top-down (block Thomas), blocks k+1..e-1
  // bottom-up, and the middle block k = s + (e-s-1)/2 closes the system, so the forward
  // sweeps run from both ends at once and meet in the middle.  Per block three matrices
  // are stored:
  //   top    i < k : G = D'^-1, H = D'^-1 A, W = D'^-1 C
  //   bottom i > k : G = E'^-1, H = E'^-1 C, W = E'^-1 A
  //   middle i = k : G = Z, H = Z A, W = Z C,  Z = (D - A W_{k-1} - C W_{k+1})^-1
  // with A (C) the Coriolis coupling to block i-1 (i+1) inside the range.
  auto sub_prod = [&](std::vector<cplx>& Dm, const std::vector<cplx>& X, const cplx* Y) {
    for (int r = 0; r < Nr; ++r)
      for (int q = 0; q < Nr; ++q) {
        const cplx x = X[(size_t)r * Nr + q];
        if (x == cplx(0.0)) continue;
        for (int k = 0; k < Nr; ++k) Dm[(size_t)r * Nr + k] -= x * Y[(size_t)q * Nr + k];
      }
  };
  // Row equilibration: every row of a block row is divided by its largest entry over the
  // diagonal block and both Coriolis couplings before the block is factorised, and the
  // factors absorb the scaling (G = (S D')^-1 S, H = (S D')^-1 S A, W = (S D')^-1 S C are
  // the same matrices as without it).  The rows of one block span thirteen orders of
  // magnitude (boundary rows ~1, fourth-order rows ~1e13 at N_r = 64); pivoting on the
  // unscaled rows costs the boundary rows up to 1e-9 of their accuracy.
  auto row_scale = [&](int fld, int l, int m, int i, int nb, const std::vector<cplx>& Dm,
                       std::vector<double>& S) {
    std::vector<cplx> B;
    S.assign(Nr, 0.0);
    for (int r = 0; r < Nr; ++r)
      for (int k = 0; k < Nr; ++k) S[r] = std::max(S[r], std::abs(Dm[(size_t)r * Nr + k]));
    for (int side = -1; side <= 1; side += 2) {
      if ((side < 0 && i == 0) || (side > 0 && i == nb - 1)) continue;
      ops.coupling(fld, l, m, side, B);
      for (int r = 0; r < Nr; ++r)
        for (int k = 0; k < Nr; ++k) S[r] = std::max(S[r], std::abs(B[(size_t)r * Nr + k]));
    }
    for (int r = 0; r < Nr; ++r) S[r] = 1.0 / S[r];
  };
  auto scale_rows = [&](std::vector<cplx>& Mx, const std::vector<double>& S) {
    for (int r = 0; r < Nr; ++r)
      for (int k = 0; k < Nr; ++k) Mx[(size_t)r * Nr + k] *= S[r];
  };
  auto factor_range = [&](int c, int s, int e) -> bool {
    const int a = c / 2, cls = c % 2;
    const int m = t.m_of[a];
    const int nb = d.L - m + 1;
    const int km = s + (e - s - 1) / 2;
    auto field_of = [&](int i) { return ((i + cls) % 2 == 0) ? 0 : 1; };
    auto slot = [&](std::vector<cplx>& v, int i) { return &v[(f.chain_off[c] + i) * blk]; };
    std::vector<cplx> D, A, C, tmp;
    std::vector<double> S;
    std::vector<int> piv;
    auto invert_into = [&](int i) {
      tmp.assign(blk, cplx(0.0));
      for (int r = 0; r < Nr; ++r) tmp[(size_t)r * Nr + r] = S[r];
      lu_solve(Nr, D, piv, Nr, tmp);
      std::copy(tmp.begin(), tmp.end(), slot(f.G, i));
    };
    for (int i = s; i < km; ++i) {  // top-down
      const int l = m + i, fld = field_of(i);
      ops.diag(fld, l, m, D);
      row_scale(fld, l, m, i, nb, D, S);
      if (i > s) {
        ops.coupling(fld, l, m, -1, A);
        sub_prod(D, A, slot(f.W, i - 1));
      }
      scale_rows(D, S);
      if (!lu_factor(Nr, D, piv)) return false;
      invert_into(i);
      if (i > s) {
        scale_rows(A, S);
        lu_solve(Nr, D, piv, Nr, A);
        std::copy(A.begin(), A.end(), slot(f.H, i));
      }
      ops.coupling(fld, l, m, +1, C);
      scale_rows(C, S);
      lu_solve(Nr, D, piv, Nr, C);
      std::copy(C.begin(), C.end(), slot(f.W, i));
    }
    for (int i = e - 1; i > km; --i) {  // bottom-up
      const int l = m + i, fld = field_of(i);
      ops.diag(fld, l, m, D);
      row_scale(fld, l, m, i, nb, D, S);
      if (i < e - 1) {
        ops.coupling(fld, l, m, +1, C);
        sub_prod(D, C, slot(f.W, i + 1));
      }
      scale_rows(D, S);
      if (!lu_factor(Nr, D, piv)) return false;
      invert_into(i);
      if (i < e - 1) {
        scale_rows(C, S);
        lu_solve(Nr, D, piv, Nr, C);
        std::copy(C.begin(), C.end(), slot(f.H, i));
      }
      ops.coupling(fld, l, m, -1, A);
      scale_rows(A, S);
      lu_solve(Nr, D, piv, Nr, A);
      std::copy(A.begin(), A.end(), slot(f.W, i));
    }
    {  // middle
      const int i = km, l = m + i, fld = field_of(i);
      ops.diag(fld, l, m, D);
      row_scale(fld, l, m, i, nb, D, S);
      if (i > s) {
        ops.coupling(fld, l, m, -1, A);
        sub_prod(D, A, slot(f.W, i - 1));
      }
      if (i < e - 1) {
        ops.coupling(fld, l, m, +1, C);
        sub_prod(D, C, slot(f.W, i + 1));
      }
      scale_rows(D, S);
      if (!lu_factor(Nr, D, piv)) return false;
      invert_into(i);
      if (i > s) {
        scale_rows(A, S);
        lu_solve(Nr, D, piv, Nr, A);
        std::copy(A.begin(), A.end(), slot(f.H, i));
      }
      if (i < e - 1) {
        scale_rows(C, S);
        lu_solve(Nr, D, piv, Nr, C);
        std::copy(C.begin(), C.end(), slot(f.W, i));
      }
    }
    return true;
  };
  auto work = [&](int c) {
    for (size_t q = 0; q + 1 < cuts[c].size(); ++q)
      if (!factor_range(c, cuts[c][q], cuts[c][q + 1])) {
        bad[c] = 1;
        return;
      }
  };
  const int nth = std::max(1, std::min<int>(nchains, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int w = 0; w < nth; ++w)
    pool.emplace_back([&, w]() {
      for (int c = w; c < nchains; c += nth) work(c);
    });
  for (auto& th : pool) th.join();
  for (int c = 0; c < nchains; ++c)
    if (bad[c]) return 1 + c;
  if (nparts > 1 && !partition_extras(d, t, ops, cuts, f)) return 1 + nchains;
  // Temperature: real inverse per l.
  f.Tinv.assign((size_t)(d.L + 1) * blk, 0.0);
  std::vector<double> D, I;
  std::vector<int> piv;
  std::vector<double> St(Nr);
  for (int l = 0; l <= d.L; ++l) {
    ops.temp(l, D);
    for (int r = 0; r < Nr; ++r) {  // row equilibration, as for the chains
      double mx = 0.0;
      for (int k = 0; k < Nr; ++k) mx = std::max(mx, std::fabs(D[(size_t)r * Nr + k]));
      St[r] = 1.0 / mx;
      for (int k = 0; k < Nr; ++k) D[(size_t)r * Nr + k] *= St[r];
    }
    if (!lu_factor(Nr, D, piv)) return 1 + nchains;
    I.assign(blk, 0.0);
    for (int r = 0; r < Nr; ++r) I[(size_t)r * Nr + r] = St[r];
    lu_solve(Nr, D, piv, Nr, I);
    std::copy(I.begin(), I.end(), f.Tinv.begin() + (size_t)l * blk);
  }
  return 0;
}

// One level of odd-even reduction of every e/f chain (HostFactorCR): the inverses of the
// odd diagonal blocks, the reduced chains on the even blocks, and the twisted block factors
// of the reduced chains (the conventions of build_factor on a range 0..nr-1, with row
// equilibration over the reduced block row).
int build_factor_cr(const rsc_params& p, const Dims& d, const HostTables& t, double dt,
                    HostFactorCR& f) {
  const int Nr = d.Nr;
  const size_t blk = (size_t)Nr * Nr;
  Ops ops{d, t, p.Ek, p.Pr, std::isfinite(dt) ? 1.0 / dt : 0.0, Nr, p.explicit_coriolis != 0};
  f.dt = dt;
  const int nchains = 2 * d.nm;
  f.odd_off.resize(nchains + 1);
  f.red_off.resize(nchains + 1);
  long no = 0, nr = 0;
  for (int c = 0; c < nchains; ++c) {
    const int nb = d.L - t.m_of[c / 2] + 1;
    f.odd_off[c] = no;
    f.red_off[c] = nr;
    no += nb / 2;
    nr += (nb + 1) / 2;
  }
  f.odd_off[nchains] = no;
  f.red_off[nchains] = nr;
  f.Dinv.assign(no * blk, cplx(0.0));
  f.G.assign(nr * blk, cplx(0.0));
  f.H.assign(nr * blk, cplx(0.0));
  f.W.assign(nr * blk, cplx(0.0));
  // Cm -= Am Bm (row-major Nr x Nr)
  auto sub_prod = [&](cplx* Cm, const cplx* Am, const cplx* Bm) {
    for (int r = 0; r < Nr; ++r)
      for (int q = 0; q < Nr; ++q) {
        const cplx a = Am[(size_t)r * Nr + q];
        if (a == cplx(0.0)) continue;
        const cplx* br = Bm + (size_t)q * Nr;
        cplx* cr = Cm + (size_t)r * Nr;
        for (int k = 0; k < Nr; ++k) cr[k] -= a * br[k];
      }
  };
  auto row_max = [&](const cplx* Mx, std::vector<double>& S) {
    for (int r = 0; r < Nr; ++r)
      for (int k = 0; k < Nr; ++k) S[r] = std::max(S[r], std::abs(Mx[(size_t)r * Nr + k]));
  };
  auto scale_rows = [&](cplx* Mx, const std::vector<double>& S) {
    for (int r = 0; r < Nr; ++r)
      for (int k = 0; k < Nr; ++k) Mx[(size_t)r * Nr + k] *= S[r];
  };
  std::vector<int> bad(nchains, 0);
  auto work = [&](int c) -> bool {
    const int a = c / 2, cls = c % 2, m = t.m_of[a];
    const int nb = d.L - m + 1, nodd = nb / 2, nred = (nb + 1) / 2;
    auto field_of = [&](int i) { return ((i + cls) % 2 == 0) ? 0 : 1; };
    std::vector<cplx> D, A, C, tmp;
    std::vector<double> S(Nr);
    std::vector<int> piv;
    // odd blocks i = 2q + 1: D_i^-1, Pq = D_i^-1 A_i, Qq = D_i^-1 C_i
    std::vector<cplx> Pm((size_t)nodd * blk, cplx(0.0)), Qm((size_t)nodd * blk, cplx(0.0));
    for (int q = 0; q < nodd; ++q) {
      const int i = 2 * q + 1, l = m + i, fld = field_of(i);
      ops.diag(fld, l, m, D);
      std::fill(S.begin(), S.end(), 0.0);
      row_max(D.data(), S);
      for (int r = 0; r < Nr; ++r) S[r] = 1.0 / S[r];
      scale_rows(D.data(), S);
      if (!lu_factor(Nr, D, piv)) return false;
      tmp.assign(blk, cplx(0.0));
      for (int r = 0; r < Nr; ++r) tmp[(size_t)r * Nr + r] = S[r];
      lu_solve(Nr, D, piv, Nr, tmp);
      std::copy(tmp.begin(), tmp.end(), &f.Dinv[(f.odd_off[c] + q) * blk]);
      ops.coupling(fld, l, m, -1, A);
      scale_rows(A.data(), S);
      lu_solve(Nr, D, piv, Nr, A);
      std::copy(A.begin(), A.end(), &Pm[(size_t)q * blk]);
      if (i + 1 < nb) {
        ops.coupling(fld, l, m, +1, C);
        scale_rows(C.data(), S);
        lu_solve(Nr, D, piv, Nr, C);
        std::copy(C.begin(), C.end(), &Qm[(size_t)q * blk]);
      }
    }
    // reduced chain on the even blocks j = 2 tt
    std::vector<cplx> Dr((size_t)nred * blk, cplx(0.0)), Ar((size_t)nred * blk, cplx(0.0)),
        Cr((size_t)nred * blk, cplx(0.0));
    for (int tt = 0; tt < nred; ++tt) {
      const int j = 2 * tt, l = m + j, fld = field_of(j);
      ops.diag(fld, l, m, D);
      cplx* dr = &Dr[(size_t)tt * blk];
      std::copy(D.begin(), D.end(), dr);
      if (j >= 1) {
        ops.coupling(fld, l, m, -1, A);
        sub_prod(dr, A.data(), &Qm[(size_t)(tt - 1) * blk]);
        if (j >= 2) sub_prod(&Ar[(size_t)tt * blk], A.data(), &Pm[(size_t)(tt - 1) * blk]);
      }
      if (j + 1 < nb) {
        ops.coupling(fld, l, m, +1, C);
        sub_prod(dr, C.data(), &Pm[(size_t)tt * blk]);
        if (j + 2 < nb) sub_prod(&Cr[(size_t)tt * blk], C.data(), &Qm[(size_t)tt * blk]);
      }
    }
    // twisted block factors of the reduced chain
    const int km = (nred - 1) / 2;
    auto slot = [&](std::vector<cplx>& v, int tt) { return &v[(f.red_off[c] + tt) * blk]; };
    auto factor_block = [&](int tt, bool up, bool down) -> bool {
      // up: subtract A' W_{tt-1}; down: subtract C' W_{tt+1}
      const bool hasA = tt > 0, hasC = tt < nred - 1;
      std::fill(S.begin(), S.end(), 0.0);
      row_max(&Dr[(size_t)tt * blk], S);
      if (hasA) row_max(&Ar[(size_t)tt * blk], S);
      if (hasC) row_max(&Cr[(size_t)tt * blk], S);
      for (int r = 0; r < Nr; ++r) S[r] = 1.0 / S[r];
      D.assign(Dr.begin() + (size_t)tt * blk, Dr.begin() + (size_t)(tt + 1) * blk);
      if (up) sub_prod(D.data(), &Ar[(size_t)tt * blk], slot(f.W, tt - 1));
      if (down) sub_prod(D.data(), &Cr[(size_t)tt * blk], slot(f.W, tt + 1));
      scale_rows(D.data(), S);
      if (!lu_factor(Nr, D, piv)) return false;
      tmp.assign(blk, cplx(0.0));
      for (int r = 0; r < Nr; ++r) tmp[(size_t)r * Nr + r] = S[r];
      lu_solve(Nr, D, piv, Nr, tmp);
      std::copy(tmp.begin(), tmp.end(), slot(f.G, tt));
      // top / middle: H = D'^-1 A', W = D'^-1 C';  bottom: H = E'^-1 C', W = E'^-1 A'
      const bool bottom = tt > km;
      const std::vector<cplx>& Hsrc = bottom ? Cr : Ar;
      const std::vector<cplx>& Wsrc = bottom ? Ar : Cr;
      const bool hasH = bottom ? hasC : hasA, hasW = bottom ? hasA : hasC;
      if (hasH) {
        A.assign(Hsrc.begin() + (size_t)tt * blk, Hsrc.begin() + (size_t)(tt + 1) * blk);
        scale_rows(A.data(), S);
        lu_solve(Nr, D, piv, Nr, A);
        std::copy(A.begin(), A.end(), slot(f.H, tt));
      }
      if (hasW) {
        C.assign(Wsrc.begin() + (size_t)tt * blk, Wsrc.begin() + (size_t)(tt + 1) * blk);
        scale_rows(C.data(), S);
        lu_solve(Nr, D, piv, Nr, C);
        std::copy(C.begin(), C.end(), slot(f.W, tt));
      }
      return true;
    };
    for (int tt = 0; tt < km; ++tt)
      if (!factor_block(tt, tt > 0, false)) return false;
    for (int tt = nred - 1; tt > km; --tt)
      if (!factor_block(tt, false, tt < nred - 1)) return false;
    return factor_block(km, km > 0, km < nred - 1);
  };
  const int nth = std::max(1, std::min<int>(nchains, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int w = 0; w < nth; ++w)
    pool.emplace_back([&, w]() {
      for (int c = w; c < nchains; c += nth)
        if (!work(c)) bad[c] = 1;
    });
  for (auto& th : pool) th.join();
  for (int c = 0; c < nchains; ++c)
    if (bad[c]) return 1 + c;
  return 0;
}

void conductive_T00(const rsc_params& p, const Dims& d, const HostTables& t,
                    std::vector<double>& coef) {
  const int Nr = d.Nr;
  Ops ops{d, t, p.Ek, p.Pr, 0.0, Nr, false};
  std::vector<double> D;
  ops.temp(0, D);
  std::vector<int> piv;
  lu_factor(Nr, D, piv);
  coef.assign(Nr, 0.0);
  coef[Nr - 1] = 1.0;  // row Nr-1 is x = -1, r = r_in, where T = 1 (Eq. BCtemp)
  lu_solve(Nr, D, piv, 1, coef);
}

}  // namespace rsc
