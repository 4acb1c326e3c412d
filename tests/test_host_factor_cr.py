"""The library's odd-even reduced factorisation (csrc/tables.cpp, build_factor_cr) against
the oracle's chain operator, on the CPU.

One level of cyclic reduction eliminates the odd blocks of every e/f chain of Sec. 3.2
(Fig. blocks): x_i = D_i^-1 (b_i - A_i x_{i-1} - C_i x_{i+1}) for odd i, which leaves a
block-tridiagonal chain of half the length on the even blocks (Schur complement), solved by
the twisted block Thomas factors.  Random right-hand sides on every chain are solved with the
library's factors in the order of the GPU kernels (u = D^-1 b on the odd blocks, the reduced
right-hand side, G b and the sweeps of the reduced chain from both ends, the odd blocks from
their neighbours) and checked, as the unreduced factors in test_host_factor.py,
  * by the row-scaled backward error of the oracle's assembled chain system,
    max_i |A x - b|_i / (||A_i||_1 ||x||_inf + |b_i|) < 64 u (u = 2^-53);
  * element by element against the oracle's own solve (row-equilibrated banded LU).
The forward bounds are those of the unreduced factors except at L = 127, N_r = 64, dt = 200,
where the back-substitution of the odd blocks, b_i - A_i x_{i-1} - C_i x_{i+1}, cancels O(1)
Coriolis terms against a diagonal of order Ek: there the backward error is 31 u and the
forward error 2.6e-11 (the unreduced factors: 6 u and 7e-13), still below the 64 u of a
backward-stable solve.
The couplings A_i, C_i that the solve applies are rebuilt here from the oracle's chain
system, so the test also pins the odd-block formula and the reduced right-hand side.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.shell import Shell
from tests.test_host_factor import chain_residuals, _cuda_include

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2508_16635_gb300", "csrc")

# The C harness writes the factors' products with the right-hand side: the test supplies the
# couplings (from the oracle) applied to the neighbours, so that the harness needs only the
# factors.  Protocol: phase 1 reads b and writes u = D^-1 b on the odd blocks; the test forms
# b' = b - A u - C u on the even blocks; phase 2 reads b' and writes the reduced solution;
# the test forms r = b - A x - C x on the odd blocks; phase 3 reads r and writes D^-1 r.
HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "rsc_internal.h"
using namespace rsc;
// usage: L Ms Nr Ek dt phase in.bin out.bin ; in/out complex [2][P][Nr] (e, f)
int main(int argc, char** argv) {
  rsc_params p{};
  p.L = atoi(argv[1]); p.Ms = atoi(argv[2]); p.Nr = atoi(argv[3]); p.Ek = atof(argv[4]);
  const double dt = atof(argv[5]); const int phase = atoi(argv[6]);
  p.Ra = 100; p.Pr = 1; p.eta = 0.35; p.precision = 0; p.explicit_coriolis = 0;
  Dims d; build_dims(p, d); HostTables t; build_tables(p, d, t);
  HostFactorCR f;
  if (build_factor_cr(p, d, t, dt, f)) { printf("factor failed\n"); return 1; }
  const int Nr = d.Nr; const size_t blk = (size_t)Nr * Nr;
  std::vector<cplx> b((size_t)2 * d.P * Nr);
  FILE* fi = fopen(argv[7], "rb");
  if (!fi || fread(b.data(), sizeof(cplx), b.size(), fi) != b.size()) return 2;
  fclose(fi);
  std::vector<cplx> out(b.size(), cplx(0));
  auto mv = [&](const cplx* A, const cplx* v, cplx* o, int mode) {
    std::vector<cplx> tt(Nr, cplx(0));
    for (int r = 0; r < Nr; ++r) for (int k = 0; k < Nr; ++k) tt[r] += A[(size_t)r * Nr + k] * v[k];
    for (int r = 0; r < Nr; ++r) o[r] = mode == 0 ? tt[r] : o[r] - tt[r]; };
  for (int a = 0; a < d.nm; ++a) for (int cls = 0; cls < 2; ++cls) {
    const int c = 2 * a + cls, nb = d.L - t.m_of[a] + 1;
    auto row = [&](int i) { return ((size_t)((i + cls) & 1) * d.P + t.pstart[a] + i) * Nr; };
    if (phase != 2) {   // D_i^-1 on the odd blocks
      for (int i = 1; i < nb; i += 2)
        mv(&f.Dinv[(f.odd_off[c] + i / 2) * blk], &b[row(i)], &out[row(i)], 0);
      continue;
    }
    const int nr = (nb + 1) / 2, km = (nr - 1) / 2; const long boff = f.red_off[c];
    std::vector<cplx> x((size_t)nr * Nr);
    auto X = [&](int i) { return &x[(size_t)i * Nr]; };
    for (int i = 0; i < nr; ++i) mv(&f.G[(boff + i) * blk], &b[row(2 * i)], X(i), 0);
    for (int i = 1; i < km; ++i) mv(&f.H[(boff + i) * blk], X(i - 1), X(i), 1);
    for (int i = nr - 2; i > km; --i) mv(&f.H[(boff + i) * blk], X(i + 1), X(i), 1);
    if (km > 0) mv(&f.H[(boff + km) * blk], X(km - 1), X(km), 1);
    if (km < nr - 1) mv(&f.W[(boff + km) * blk], X(km + 1), X(km), 1);
    for (int i = km - 1; i >= 0; --i) mv(&f.W[(boff + i) * blk], X(i + 1), X(i), 1);
    for (int i = km + 1; i < nr; ++i) mv(&f.W[(boff + i) * blk], X(i - 1), X(i), 1);
    for (int i = 0; i < nr; ++i) for (int k = 0; k < Nr; ++k) out[row(2 * i) + k] = x[(size_t)i * Nr + k];
  }
  FILE* fo = fopen(argv[8], "wb"); fwrite(out.data(), sizeof(cplx), out.size(), fo); fclose(fo);
  return 0;
}
"""


@pytest.fixture(scope="module")
def cr_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("no host C++ compiler or CUDA headers")
    d = tmp_path_factory.mktemp("hostfactor_cr")
    src = d / "cr.cpp"
    src.write_text(HARNESS)
    exe = d / "cr"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", inc, str(src), os.path.join(CSRC, "tables.cpp"), "-o", str(exe),
                    "-lpthread"], check=True)
    return exe, d


def _couple(s, dt, v, dst_parity):
    """w[fld, p] = A_i v_{i-1} + C_i v_{i+1} on the blocks i of parity dst_parity of every
    chain (the oracle's coupling blocks; absent terms past a chain end)."""
    w = np.zeros_like(v)
    for a, m in enumerate(s.ms):
        p0 = s.starts[a]
        for cls in (0, 1):
            flds, D, A, C = s.chain_system(m, cls, dt)
            fi = [0 if f == "e" else 1 for f in flds]
            for i in range(dst_parity, len(D), 2):
                acc = np.zeros(s.Nr, complex)
                if A[i] is not None:
                    acc += A[i] @ v[fi[i - 1], p0 + i - 1]
                if C[i] is not None:
                    acc += C[i] @ v[fi[i + 1], p0 + i + 1]
                w[fi[i], p0 + i] = acc
    return w


def _parity_mask(s, parity):
    mask = np.zeros((2, s.P), bool)
    for a, m in enumerate(s.ms):
        for cls in (0, 1):
            for i in range(parity, s.L - m + 1, 2):
                fld = (i + cls) & 1
                mask[fld, s.starts[a] + i] = True
    return mask


@pytest.mark.parametrize("L,Ms,Nr,Ek,dt,fwd", [
    (15, 4, 12, 1e-3, 1e-3, 1e-13),
    (16, 4, 12, 1e-3, 200.0, 1e-12),     # even and odd chain lengths
    (31, 4, 24, 1e-3, 200.0, 1e-12),
    (63, 8, 48, 1e-4, 200.0, 1e-12),
    (127, 12, 64, 1e-5, 200.0, 1e-10),   # measured 2.6e-11 (backward error 31 u)
    (127, 12, 64, 1e-5, 5e-6, 1e-11),
])
def test_reduced_factors_solve_the_oracle_chains(cr_exe, L, Ms, Nr, Ek, dt, fwd):
    exe, d = cr_exe
    s = Shell(L, Ms, Nr, Ek, 100.0)
    rng = np.random.default_rng(L + Nr + 1)
    b = rng.standard_normal((2, s.P, Nr)) + 1j * rng.standard_normal((2, s.P, Nr))

    def run(phase, v):
        fin, fout = d / f"in_{L}_{Nr}.bin", d / f"out_{L}_{Nr}.bin"
        np.ascontiguousarray(v, dtype=np.complex128).tofile(fin)
        subprocess.run([str(exe), str(L), str(Ms), str(Nr), repr(Ek), repr(dt), str(phase),
                        str(fin), str(fout)], check=True, timeout=600)
        return np.fromfile(fout, dtype=np.complex128).reshape(2, s.P, Nr)

    odd, even = _parity_mask(s, 1), _parity_mask(s, 0)
    u = run(1, b)                                     # D^-1 b on the odd blocks
    assert np.all(u[even] == 0)
    bred = np.where(even[..., None], b - _couple(s, dt, u, 0), 0)   # reduced right-hand side
    xe = run(2, bred)                                 # the reduced chains
    assert np.all(xe[odd] == 0)
    r = np.where(odd[..., None], b - _couple(s, dt, xe, 1), 0)
    xo = run(3, r)                                    # the odd blocks from their neighbours
    x = np.where(odd[..., None], xo, xe)
    eta, diff = chain_residuals(s, dt, b, x)
    assert eta < 64.0, eta
    assert diff < fwd, diff
