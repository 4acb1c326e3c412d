// Internal declarations of the rotating-shell GB300 library.
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <string>
#include <vector>

#include "rsc.h"

namespace rsc {

using cplx = std::complex<double>;

// Problem sizes (Sec. 3.1).  Pairs (m, l) are ordered by m then l, as in the
// canonical state layout.
struct Dims {
  int L = 0, Ms = 0, Nr = 0;
  int Nd = 0;        // de-aliased radial points, ceil(3 Nr / 2)
  int nlat = 0;      // Gauss-Legendre latitudes (even)
  int nlat2 = 0;     // nlat / 2 (one hemisphere)
  int nphi = 0;      // longitudes per sector
  int nm = 0;        // active m values
  int K = 0;         // nm - 1
  int P = 0;         // (l, m) pairs
  double r_in = 0, r_out = 0;
  long n() const { return 6L * P * Nr; }
};

// Host-side tables, all FP64.
struct HostTables {
  std::vector<double> rc, rd;          // collocation radii (Nr), de-aliased radii (Nd)
  std::vector<double> Ec[5];           // [j][k] d^o T_k / dr^o at rc, o = 0..4
  std::vector<double> Ed[3];           // [i][k] d^o T_k / dr^o at rd, o = 0..2
  std::vector<double> R0, R1;          // [j][i]: N_d values -> value / d_r at rc of
                                       // the N_r-truncated interpolant
  std::vector<double> xlat, wlat;      // Gauss-Legendre nodes (north first), weights
  std::vector<int> m_of, pstart;       // per m index: m, first pair
  std::vector<int> pair_l, pair_m;     // per pair
  std::vector<long> leg_off;           // per m index: offset into Legendre tables
  // synthesis layout [m block][l - m][t], t < nlat2 (north hemisphere)
  std::vector<double> P, dP, Ps;
  // analysis layout [m block][t][l - m], weighted by w_t / (2 (2 - delta_m0))
  std::vector<double> Pw, dPw, Psw;
};

// Factorisation of the implicit operator for one dt (Sec. 3.2, block Thomas).
// Chain c = 2 * m_index + class; block i of a chain is l = m + i.
struct HostFactor {
  double dt = 0;
  std::vector<long> chain_off;        // first block of each chain
  std::vector<cplx> G, H, W;          // per block Nr x Nr, row-major
  std::vector<double> Tinv;           // per l: Nr x Nr inverse of the T operator
  // Partitioned chains (nparts > 1): every chain is cut into parts, each factorised on its
  // own (G, H, W above, same slots); the parts are coupled through spikes and a reduced
  // system for the first and last blocks of the parts (a SPIKE-type solve):
  //   x_i = xl_i - V_i x(first block of the next part) - Wsp_i x(last block of the previous),
  // xl the part-local solution.
  std::vector<long> parts;            // per part: p0, cls, nb, boff, m, chain
  std::vector<cplx> V, Wsp;           // spikes per block, Nr x Nr (zero where absent)
  std::vector<long> red_off;          // per chain: offset of its reduced inverse in red
  std::vector<int> red_nu, zoff;      // per chain: unknown blocks, first z block
  std::vector<cplx> red;              // per chain: (nu Nr)^2 inverse of I + K, row-major
  std::vector<long> unk_row;          // per z block: element offset of that block in a state
  std::vector<int> unk_chain;         // per z block: its chain
  std::vector<int> blk_z;             // per block: z block of the next part's first block
                                      // and of the previous part's last block (-1: none)
};

// One level of odd-even (cyclic) reduction of every e/f chain, for the double-float solve
// of the mixed path.  With D_i, A_i, C_i the diagonal block of block row i and its
// couplings to blocks i - 1 and i + 1, the odd blocks are eliminated:
//   x_i = D_i^-1 (b_i - A_i x_{i-1} - C_i x_{i+1}),   i odd,
// which leaves a block-tridiagonal chain of half the length on the even blocks j = 2t:
//   D'_t = D_j - A_j D_{j-1}^-1 C_{j-1} - C_j D_{j+1}^-1 A_{j+1},
//   A'_t = -A_j D_{j-1}^-1 A_{j-1},   C'_t = -C_j D_{j+1}^-1 C_{j+1},
//   b'_t = b_j - A_j D_{j-1}^-1 b_{j-1} - C_j D_{j+1}^-1 b_{j+1}.
// The reduced chains carry the twisted block factors of HostFactor (G, H, W; middle block
// t = (nr - 1) / 2 of nr = (nb + 1) / 2), so the solve is: u_i = D_i^-1 b_i (odd), b'
// (even), the twisted sweeps over the reduced chains, then the odd blocks from their
// neighbours.  Terms that reach past a chain end are absent.
struct HostFactorCR {
  double dt = 0;
  std::vector<long> odd_off;   // per chain (+1 total): first odd block in Dinv
  std::vector<long> red_off;   // per chain (+1 total): first reduced block in G, H, W
  std::vector<cplx> Dinv;      // per odd block i = 1, 3, ...: D_i^-1, Nr x Nr row-major
  std::vector<cplx> G, H, W;   // twisted factors of the reduced chains, as HostFactor
};

void build_dims(const rsc_params& p, Dims& d);
void build_tables(const rsc_params& p, const Dims& d, HostTables& t);
// Returns 0 on success, or 1 + chain index of a singular block.
// nparts > 1: partitioned chains (parts of at least 8 blocks, at most nparts per chain).
int build_factor(const rsc_params& p, const Dims& d, const HostTables& t, double dt,
                 HostFactor& f, int nparts = 1);
// Returns 0 on success, or 1 + chain index of a singular block (implicit Coriolis only).
int build_factor_cr(const rsc_params& p, const Dims& d, const HostTables& t, double dt,
                    HostFactorCR& f);
// Gauss-Legendre nodes (descending from +1) and weights on [-1, 1].
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
void conductive_T00(const rsc_params& p, const Dims& d, const HostTables& t,
                    std::vector<double>& coef);

// ---------------------------------------------------------------------------
// Device kernels (launch wrappers).  Real = double (FP64 path) or float
// (transforms of the mixed path).
struct DevTables;

template <typename Real>
struct Work {
  // SR: spectral values on the de-aliased radii [P][Nd][8]
  // FC: Fourier coefficients of 9 grid fields [9][Nd][K+1][nlat]
  // FCU: the same for the base state of a Jacobian action
  // FA: Fourier coefficients of the 4 products [4][Nd][K+1][nlat]
  // AR: analysed products on the de-aliased radii [P][Nd][4]
  void* SR = nullptr;
  void* FC = nullptr;
  void* FCU = nullptr;
  void* FA = nullptr;
  void* AR = nullptr;
};

}  // namespace rsc
