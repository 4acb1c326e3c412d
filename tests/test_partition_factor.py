"""Host check of the partitioned chain factorisation (csrc/tables.cpp, build_factor with
nparts > 1, the SPIKE-type option of the double-float solve): random right-hand sides on
every chain are solved with the unpartitioned twisted factors and with the partitioned ones
(part-local solves, reduced system, correction: the data flow of the GPU kernels), in FP64 on
the host.  On a well-conditioned case the two agree to rounding; at Delta t = 200 the chains'
conditioning separates any two FP64 solves (a numpy check puts the direct FP64 solve itself
2e-8 to 4e-7 from the exact solution of the RW12 chains), so the bound there is that level.
"""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2508_16635_gb300", "csrc")

HARNESS = r"""
// CPU check of the partitioned chain factorisation: solve random right-hand sides on every
// chain with the unpartitioned twisted factors and with the partitioned ones (part solves,
// reduced system, correction; the data flow of the GPU kernels) and compare.
#include <cstdio>
#include <cstdlib>
#include <random>
#include "rsc_internal.h"
using namespace rsc;

static void twisted(const HostFactor& f, int Nr, long boff, int nb, std::vector<cplx>& x) {
  // x: nb blocks of Nr (vector), in: b, out: solution of the range's local system
  const size_t blk = (size_t)Nr * Nr;
  auto mv = [&](const cplx* A, const cplx* v, cplx* out, double sgn) {
    std::vector<cplx> t(Nr, cplx(0));
    for (int r = 0; r < Nr; ++r) for (int k = 0; k < Nr; ++k) t[r] += A[(size_t)r * Nr + k] * v[k];
    for (int r = 0; r < Nr; ++r) out[r] = (sgn == 0 ? cplx(0) : out[r]) + (sgn == 0 ? t[r] : sgn * t[r]);
  };
  const int km = (nb - 1) / 2;
  auto X = [&](int i) { return &x[(size_t)i * Nr]; };
  for (int i = 0; i < nb; ++i) { std::vector<cplx> b(X(i), X(i) + Nr); mv(&f.G[(boff + i) * blk], b.data(), X(i), 0); }
  for (int i = 1; i < km; ++i) mv(&f.H[(boff + i) * blk], X(i - 1), X(i), -1);
  for (int i = nb - 2; i > km; --i) mv(&f.H[(boff + i) * blk], X(i + 1), X(i), -1);
  if (km > 0) mv(&f.H[(boff + km) * blk], X(km - 1), X(km), -1);
  if (km < nb - 1) mv(&f.W[(boff + km) * blk], X(km + 1), X(km), -1);
  for (int i = km - 1; i >= 0; --i) mv(&f.W[(boff + i) * blk], X(i + 1), X(i), -1);
  for (int i = km + 1; i < nb; ++i) mv(&f.W[(boff + i) * blk], X(i - 1), X(i), -1);
}

int main(int argc, char** argv) {
  rsc_params p{};
  p.L = atoi(argv[1]); p.Ms = atoi(argv[2]); p.Nr = atoi(argv[3]); p.Ek = atof(argv[4]);
  const double dt = atof(argv[5]); const int P = atoi(argv[6]);
  p.Ra = 100; p.Pr = 1; p.eta = 0.35; p.precision = 0; p.explicit_coriolis = 0;
  Dims d; build_dims(p, d); HostTables t; build_tables(p, d, t);
  HostFactor f1, fP;
  if (build_factor(p, d, t, dt, f1, 1) || build_factor(p, d, t, dt, fP, P)) { printf("factor failed\n"); return 1; }
  const int Nr = d.Nr; const size_t blk = (size_t)Nr * Nr;
  const int nchains = 2 * d.nm;
  // right-hand side in the state layout [fld][pair][k]
  std::mt19937_64 rng(1); std::normal_distribution<double> N(0, 1);
  std::vector<cplx> b((size_t)2 * d.P * Nr);
  for (auto& v : b) v = cplx(N(rng), N(rng));
  for (int a = 0; a < d.nm; ++a) if (t.m_of[a] == 0) for (int l = 0; l <= d.L; ++l) for (int f2 = 0; f2 < 2; ++f2)
    for (int k = 0; k < Nr; ++k) b[((size_t)f2 * d.P + t.pstart[a] + l) * Nr + k] = b[((size_t)f2 * d.P + t.pstart[a] + l) * Nr + k].real();
  auto gather = [&](int c, std::vector<cplx>& v) {   // chain c's blocks from a state
    const int a = c / 2, cls = c % 2, nb = d.L - t.m_of[a] + 1;
    v.resize((size_t)nb * Nr);
    for (int i = 0; i < nb; ++i) { const int fld = (i + cls) & 1;
      for (int k = 0; k < Nr; ++k) v[(size_t)i * Nr + k] = b[((size_t)fld * d.P + t.pstart[a] + i) * Nr + k]; }
  };
  double num = 0, den = 0, worst = 0;
  // partitioned: part solves into a state-shaped xl, then z = Minv xl_z, then the correction
  std::vector<cplx> xl(b.size(), cplx(0));
  const int npart = (int)fP.parts.size() / 6;
  for (int q = 0; q < npart; ++q) {
    const long* pr = &fP.parts[(size_t)q * 6];
    const long p0 = pr[0]; const int cls = (int)pr[1], nb = (int)pr[2]; const long boff = pr[3];
    std::vector<cplx> v((size_t)nb * Nr);
    for (int i = 0; i < nb; ++i) { const int fld = (i + cls) & 1;
      for (int k = 0; k < Nr; ++k) v[(size_t)i * Nr + k] = b[((size_t)fld * d.P + p0 + i) * Nr + k]; }
    twisted(fP, Nr, boff, nb, v);
    for (int i = 0; i < nb; ++i) { const int fld = (i + cls) & 1;
      for (int k = 0; k < Nr; ++k) xl[((size_t)fld * d.P + p0 + i) * Nr + k] = v[(size_t)i * Nr + k]; }
  }
  const int nz = (int)fP.unk_row.size();
  std::vector<cplx> zb((size_t)nz * Nr, cplx(0));
  for (int c = 0; c < nchains; ++c) {
    const int nu = fP.red_nu[c], n = nu * Nr; if (!nu) continue;
    const cplx* Mi = &fP.red[fP.red_off[c]];
    for (int r = 0; r < n; ++r) { cplx s = 0;
      for (int col = 0; col < n; ++col) s += Mi[(size_t)r * n + col] * xl[fP.unk_row[fP.zoff[c] + col / Nr] + col % Nr];
      zb[(size_t)(fP.zoff[c] + r / Nr) * Nr + r % Nr] = s; }
  }
  std::vector<cplx> x = xl;
  for (int a = 0; a < d.nm; ++a) for (int cls = 0; cls < 2; ++cls) {
    const int c = 2 * a + cls, nb = d.L - t.m_of[a] + 1;
    for (int i = 0; i < nb; ++i) { const long g = fP.chain_off[c] + i; const int fld = (i + cls) & 1;
      cplx* xi = &x[((size_t)fld * d.P + t.pstart[a] + i) * Nr];
      for (int side = 0; side < 2; ++side) { const int zi = fP.blk_z[g * 2 + side]; if (zi < 0) continue;
        const cplx* S = &(side == 0 ? fP.V : fP.Wsp)[g * blk];
        for (int r = 0; r < Nr; ++r) { cplx s = 0; for (int k = 0; k < Nr; ++k) s += S[(size_t)r * Nr + k] * zb[(size_t)zi * Nr + k]; xi[r] -= s; } } }
  }
  for (int c = 0; c < nchains; ++c) {
    std::vector<cplx> v; gather(c, v);
    const int a = c / 2, cls = c % 2, nb = d.L - t.m_of[a] + 1;
    twisted(f1, Nr, f1.chain_off[c], nb, v);
    double n1 = 0, e1 = 0;
    for (int i = 0; i < nb; ++i) { const int fld = (i + cls) & 1;
      for (int k = 0; k < Nr; ++k) { const cplx u = v[(size_t)i * Nr + k], w = x[((size_t)fld * d.P + t.pstart[a] + i) * Nr + k];
        n1 += std::norm(u); e1 += std::norm(u - w); } }
    num += e1; den += n1; worst = std::max(worst, std::sqrt(e1 / n1));
  }
  printf("L=%d Ms=%d Nr=%d Ek=%g dt=%g P=%d: parts %d, z blocks %d; partitioned vs direct: overall %.2e, worst chain %.2e\n",
         p.L, p.Ms, p.Nr, p.Ek, dt, P, npart, nz, std::sqrt(num / den), worst);
  return 0;
}
"""


def _cuda_include():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            return os.path.join(cand, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


@pytest.fixture(scope="module")
def check_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("no host C++ compiler or CUDA headers")
    d = tmp_path_factory.mktemp("partition")
    src = d / "check.cpp"
    src.write_text(HARNESS)
    exe = d / "check"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", inc, str(src), os.path.join(CSRC, "tables.cpp"), "-o", str(exe),
                    "-lpthread"], check=True)
    return exe


def run_check(exe, L, Ms, Nr, Ek, dt, P):
    out = subprocess.run([str(exe), str(L), str(Ms), str(Nr), repr(Ek), repr(dt), str(P)],
                         capture_output=True, text=True, check=True, timeout=600).stdout
    m = re.search(r"parts (\d+), z blocks (\d+); partitioned vs direct: overall ([0-9.e+-]+), "
                  r"worst chain ([0-9.e+-]+)", out)
    return int(m.group(1)), int(m.group(2)), float(m.group(3)), float(m.group(4))


# Bounds: rounding for N_r = 12; from N_r = 24 on, the FP64 sensitivity of the e/f solve (the
# oracle's own step moves by 3e-10 to 5e-10 at L = 31, N_r = 24 under 1e-16 noise on its
# tables, and by up to 4e-9 at L = 63, N_r = 48 and dt = 200), which any two FP64 solve
# orders may differ by.
@pytest.mark.parametrize("L,Ms,Nr,Ek,dt,P,bound", [
    (15, 4, 12, 1e-3, 1e-3, 2, 1e-13),
    (31, 4, 24, 1e-3, 1e-3, 4, 1e-10),
    (31, 4, 24, 1e-3, 200.0, 4, 1e-9),
    (63, 8, 48, 1e-4, 200.0, 3, 1e-7),
])
def test_partitioned_factorisation_solves_the_same_chains(check_exe, L, Ms, Nr, Ek, dt, P, bound):
    nparts, nz, overall, worst = run_check(check_exe, L, Ms, Nr, Ek, dt, P)
    nm = L // Ms + 1
    assert nparts > 2 * nm          # some chains were cut
    assert nz > 0
    assert worst < bound, (overall, worst)
