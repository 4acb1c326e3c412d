"""The library's host block factorisation (csrc/tables.cpp, build_factor: the twisted block
Thomas factors G, H, W with row equilibration) against the oracle's chain operator, on the
CPU.  Random right-hand sides on every chain are solved with the factors in the order of the
GPU sweeps (G b, half sweeps from both ends, middle block, outward sweeps) and checked
  * by the row-scaled backward error of the oracle's assembled chain system (Sec. 3.2, the
    block-tridiagonal chains of Fig. blocks): max_i |A x - b|_i / (||A_i||_1 ||x||_inf + |b_i|)
    must stay below 64 u, the level of a backward-stable LU-type solve (u = 2^-53);
  * element by element against the oracle's own solve (row-equilibrated banded LU): the
    largest difference over the largest entry of the chain's solution.
Without the row equilibration the same solves had backward errors of 100 u to 2e4 u and
differed from the oracle by up to 1e-9 at L = 127, N_r = 64, dt = 200.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.shell import Shell

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2508_16635_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "rsc_internal.h"
using namespace rsc;
// usage: L Ms Nr Ek dt rhs.bin out.bin ; rhs/out are complex [2][P][Nr] (e,f)
int main(int argc, char** argv) {
  rsc_params p{};
  p.L = atoi(argv[1]); p.Ms = atoi(argv[2]); p.Nr = atoi(argv[3]); p.Ek = atof(argv[4]);
  const double dt = atof(argv[5]);
  p.Ra = 100; p.Pr = 1; p.eta = 0.35; p.precision = 0; p.explicit_coriolis = 0;
  Dims d; build_dims(p, d); HostTables t; build_tables(p, d, t);
  HostFactor f;
  if (build_factor(p, d, t, dt, f, 1)) { printf("factor failed\n"); return 1; }
  const int Nr = d.Nr; const size_t blk = (size_t)Nr * Nr;
  std::vector<cplx> b((size_t)2 * d.P * Nr);
  FILE* fi = fopen(argv[6], "rb");
  if (!fi || fread(b.data(), sizeof(cplx), b.size(), fi) != b.size()) return 2;
  fclose(fi);
  std::vector<cplx> out(b.size());
  for (int a = 0; a < d.nm; ++a) for (int cls = 0; cls < 2; ++cls) {
    const int c = 2 * a + cls, nb = d.L - t.m_of[a] + 1; const long boff = f.chain_off[c];
    std::vector<cplx> x((size_t)nb * Nr);
    for (int i = 0; i < nb; ++i) { const int fld = (i + cls) & 1;
      for (int k = 0; k < Nr; ++k) x[(size_t)i * Nr + k] = b[((size_t)fld * d.P + t.pstart[a] + i) * Nr + k]; }
    auto mv = [&](const cplx* A, const cplx* v, cplx* o, int mode) {
      std::vector<cplx> tt(Nr, cplx(0));
      for (int r = 0; r < Nr; ++r) for (int k = 0; k < Nr; ++k) tt[r] += A[(size_t)r * Nr + k] * v[k];
      for (int r = 0; r < Nr; ++r) o[r] = mode == 0 ? tt[r] : o[r] - tt[r]; };
    const int km = (nb - 1) / 2;
    auto X = [&](int i) { return &x[(size_t)i * Nr]; };
    for (int i = 0; i < nb; ++i) { std::vector<cplx> bb(X(i), X(i) + Nr); mv(&f.G[(boff + i) * blk], bb.data(), X(i), 0); }
    for (int i = 1; i < km; ++i) mv(&f.H[(boff + i) * blk], X(i - 1), X(i), 1);
    for (int i = nb - 2; i > km; --i) mv(&f.H[(boff + i) * blk], X(i + 1), X(i), 1);
    if (km > 0) mv(&f.H[(boff + km) * blk], X(km - 1), X(km), 1);
    if (km < nb - 1) mv(&f.W[(boff + km) * blk], X(km + 1), X(km), 1);
    for (int i = km - 1; i >= 0; --i) mv(&f.W[(boff + i) * blk], X(i + 1), X(i), 1);
    for (int i = km + 1; i < nb; ++i) mv(&f.W[(boff + i) * blk], X(i - 1), X(i), 1);
    for (int i = 0; i < nb; ++i) { const int fld = (i + cls) & 1;
      for (int k = 0; k < Nr; ++k) out[((size_t)fld * d.P + t.pstart[a] + i) * Nr + k] = x[(size_t)i * Nr + k]; }
  }
  FILE* fo = fopen(argv[7], "wb"); fwrite(out.data(), sizeof(cplx), out.size(), fo); fclose(fo);
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
def solve_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("no host C++ compiler or CUDA headers")
    d = tmp_path_factory.mktemp("hostfactor")
    src = d / "solve.cpp"
    src.write_text(HARNESS)
    exe = d / "solve"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", inc, str(src), os.path.join(CSRC, "tables.cpp"), "-o", str(exe),
                    "-lpthread"], check=True)
    return exe, d


def chain_residuals(s, dt, b, x):
    """Worst row-scaled backward error (in units of u) and worst max-abs difference against
    the oracle's solve, over every chain, for e/f right-hand sides b and solutions x [2, P, N_r]."""
    full = np.zeros((3, s.P, s.Nr), complex)
    full[:2] = b
    xo = s.solve(full, dt)[:2]
    u = 2.0 ** -53
    worst_eta = worst_fwd = 0.0
    for a, m in enumerate(s.ms):
        p0 = s.starts[a]
        for cls in (0, 1):
            flds, D, A, C = s.chain_system(m, cls, dt)
            fi = [0 if f == "e" else 1 for f in flds]
            xs = [x[fi[i], p0 + i] for i in range(len(D))]
            bs = [b[fi[i], p0 + i] for i in range(len(D))]
            xn = max(np.abs(v).max() for v in xs)
            for i in range(len(D)):
                r = D[i] @ xs[i] - bs[i]
                rown = np.abs(D[i]).sum(axis=1)
                if A[i] is not None:
                    r = r + A[i] @ xs[i - 1]
                    rown = rown + np.abs(A[i]).sum(axis=1)
                if C[i] is not None:
                    r = r + C[i] @ xs[i + 1]
                    rown = rown + np.abs(C[i]).sum(axis=1)
                worst_eta = max(worst_eta, float((np.abs(r) / (rown * xn + np.abs(bs[i]))).max()) / u)
            xo_c = np.concatenate([xo[fi[i], p0 + i] for i in range(len(D))])
            worst_fwd = max(worst_fwd, float(np.abs(xo_c - np.concatenate(xs)).max() / np.abs(xo_c).max()))
    return worst_eta, worst_fwd


@pytest.mark.parametrize("L,Ms,Nr,Ek,dt,fwd", [
    (15, 4, 12, 1e-3, 1e-3, 1e-13),
    (31, 4, 24, 1e-3, 200.0, 1e-12),
    (63, 8, 48, 1e-4, 200.0, 1e-12),
    (127, 12, 64, 1e-5, 200.0, 1e-11),
    (127, 12, 64, 1e-5, 5e-6, 1e-11),
])
def test_host_factors_solve_the_oracle_chains(solve_exe, L, Ms, Nr, Ek, dt, fwd):
    exe, d = solve_exe
    s = Shell(L, Ms, Nr, Ek, 100.0)
    rng = np.random.default_rng(L + Nr)
    b = rng.standard_normal((2, s.P, Nr)) + 1j * rng.standard_normal((2, s.P, Nr))
    rhs, out = d / f"rhs_{L}_{Nr}.bin", d / f"out_{L}_{Nr}.bin"
    b.astype(np.complex128).tofile(rhs)
    subprocess.run([str(exe), str(L), str(Ms), str(Nr), repr(Ek), repr(dt), str(rhs), str(out)],
                   check=True, timeout=600)
    x = np.fromfile(out, dtype=np.complex128).reshape(2, s.P, Nr)
    eta, diff = chain_residuals(s, dt, b, x)
    assert eta < 64.0, eta
    assert diff < fwd, diff
