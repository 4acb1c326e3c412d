"""Host checks of the double-float arithmetic of csrc/dfloat.h (split48, TwoSum, the Dot2
multiply-add, normalisation), the same source the chain-solve and Krylov kernels compile,
built here with the host C++ compiler and compared with exact rational arithmetic.

split48: hi keeps 24 significant bits, lo the next 29 bits rounded to 24, so
|d - hi - lo| <= 2^-48 |d| wherever both are normal floats.

Dot2 (Ogita, Rump and Oishi 2005): a sum of n products accumulated with error-free TwoSum
and TwoProd steps has error at most gamma_n^2 sum|x_i y_i| (gamma_n = n u / (1 - n u),
u = 2^-24) before the final rounding, which the (s, c) pair avoids; splitting each operand
into hi + lo adds the dropped lo*lo term and the rounding of the cross terms, each below
2^-45 |x_i y_i|.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2508_16635_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "dfloat.h"
int main(int argc, char** argv) {
  FILE* f = std::fopen(argv[1], "rb");
  std::vector<double> d;
  double x;
  while (std::fread(&x, sizeof x, 1, f) == 1) d.push_back(x);
  std::fclose(f);
  FILE* o = std::fopen(argv[2], "wb");
  for (double v : d) {
    float hi, lo;
    rsc::split48(v, hi, lo);
    std::fwrite(&hi, sizeof hi, 1, o);
    std::fwrite(&lo, sizeof lo, 1, o);
  }
  std::fclose(o);
  return 0;
}
"""


@pytest.fixture(scope="module")
def split_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("split48")
    src = d / "drv.cpp"
    src.write_text(HARNESS)
    exe = d / "drv"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return d, exe


def run_split(split_exe, vals):
    d, exe = split_exe
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    vals.tofile(d / "in.bin")
    subprocess.run([str(exe), str(d / "in.bin"), str(d / "out.bin")], check=True)
    out = np.fromfile(d / "out.bin", dtype=np.float32).reshape(-1, 2)
    return out[:, 0].astype(np.float64), out[:, 1].astype(np.float64)


def test_split48_error_bound_over_the_normal_range(split_exe):
    rng = np.random.default_rng(5)
    n = 200_000
    mant = rng.uniform(1.0, 2.0, n)
    mant[:1000] = np.nextafter(2.0, 0.0)          # all mantissa bits set (lo rounds up)
    mant[1000:2000] = 1.0                          # powers of two
    expo = rng.integers(-74, 128, n)
    vals = np.ldexp(mant, expo) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    hi, lo = run_split(split_exe, vals)
    err = np.abs(vals - (hi + lo))                 # hi + lo is exact in double
    assert np.all(err <= 2.0 ** -48 * np.abs(vals))
    # hi is the truncation: same sign, |hi| <= |d|, and lo shares the sign (or is zero)
    assert np.all(np.sign(hi) == np.sign(vals))
    assert np.all(np.abs(hi) <= np.abs(vals))
    assert np.all((lo == 0) | (np.sign(lo) == np.sign(vals)))


def test_split48_small_and_special_values(split_exe):
    tiny = np.ldexp(1.5, np.arange(-126, -74))     # lo dropped: absolute error < 2^-97
    hi, lo = run_split(split_exe, tiny)
    assert np.all(lo == 0)
    assert np.all(np.abs(tiny - hi) < 2.0 ** -97)
    below = np.array([0.0, -0.0, 5e-324, np.ldexp(1.0, -127), -np.ldexp(1.9, -1000)])
    hi, lo = run_split(split_exe, below)
    assert np.all(hi == 0) and np.all(lo == 0)
    big = np.array([np.ldexp(1.0, 128), -np.ldexp(1.7, 500), np.inf, -np.inf, np.nan])
    hi, lo = run_split(split_exe, big)
    assert np.isposinf(hi[0]) and np.isneginf(hi[1]) and np.isposinf(hi[2])
    assert np.isneginf(hi[3]) and np.isnan(hi[4])
    edge = np.array([np.nextafter(np.ldexp(1.0, 128), 0.0), np.ldexp(1.0, -74)])
    hi, lo = run_split(split_exe, edge)
    assert np.all(np.isfinite(hi))
    assert np.all(np.abs(edge - (hi + lo)) <= 2.0 ** -48 * np.abs(edge))


ARITH = r"""
#include <cstdio>
#include <cstring>
#include <vector>
#include "dfloat.h"
// stdin: mode n then 2n doubles.  mode 0: TwoSum of float pairs (x_i, y_i) -> (s, c) each;
// mode 1: normalisation of (s, c) = (x_i, y_i) as floats -> (s', c') each;
// mode 2: Dot2 of the split vectors x, y -> (s, c) once, then the FP32 naive dot.
int main() {
  int mode, n;
  while (std::scanf("%d %d", &mode, &n) == 2) {
    std::vector<double> x(n), y(n);
    for (int i = 0; i < n; ++i) std::scanf("%lf %lf", &x[i], &y[i]);
    if (mode == 0 || mode == 1) {
      for (int i = 0; i < n; ++i) {
        const rsc::dfl a{(float)x[i], 0.0f}, b{(float)y[i], 0.0f};
        const rsc::dfl r = mode == 0 ? rsc::dfl_add(a, b) : rsc::dfl_norm(rsc::dfl{(float)x[i], (float)y[i]});
        std::printf("%a %a\n", (double)r.s, (double)r.c);
      }
    } else {
      rsc::dfl acc = rsc::dfl_zero();
      float naive = 0.0f;
      for (int i = 0; i < n; ++i) {
        float xh, xl, yh, yl;
        rsc::split48(x[i], xh, xl);
        rsc::split48(y[i], yh, yl);
        rsc::dfl_fma(acc, xh, xl, yh, yl);
        volatile float t = naive + (float)x[i] * (float)y[i];
        naive = t;
      }
      std::printf("%a %a %a\n", (double)acc.s, (double)acc.c, (double)naive);
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def arith_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("dfarith")
    src = d / "arith.cpp"
    src.write_text(ARITH)
    exe = d / "arith"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o",
                    str(exe)], check=True)
    return exe


def run_arith(exe, mode, x, y):
    inp = f"{mode} {len(x)}\n" + "\n".join(f"{float(a).hex()} {float(b).hex()}"
                                              for a, b in zip(x, y)) + "\n"
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout
    return [[float.fromhex(t) for t in line.split()] for line in out.strip().splitlines()]


def test_two_sum_and_normalisation_are_exact(arith_exe):
    from fractions import Fraction as F
    rng = np.random.default_rng(9)
    n = 400
    a = (rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))).astype(np.float32)
    b = (rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))).astype(np.float32)
    b[:50] = -a[:50] * (1 + 2.0 ** -20)           # heavy cancellation
    for mode in (0, 1):
        res = run_arith(arith_exe, mode, a.astype(float), b.astype(float))
        for (s, c), x, y in zip(res, a, b):
            assert F(s) + F(c) == F(float(x)) + F(float(y))   # error-free
            assert s == float(np.float32(float(x) + float(y)))  # s is the rounded sum
            if mode == 1 and s != 0.0:
                assert abs(c) <= np.spacing(np.float32(abs(s))) / 2


def _exact_split_dot(x, y):
    from fractions import Fraction as F
    hx = run_split_pairs(x)
    hy = run_split_pairs(y)
    return sum((F(a) + F(b)) * (F(c) + F(d)) for (a, b), (c, d) in zip(hx, hy))


def run_split_pairs(v):
    out = []
    for d in v:
        # split48 truncates hi to 24 significant bits: reproduce it exactly
        m, e = np.frexp(d)                        # d = m 2^e, 0.5 <= |m| < 1
        hi = float(np.trunc(m * 2.0 ** 24) * 2.0 ** (e - 24))
        lo = float(np.float32(d - hi))
        out.append((hi, lo))
    return out


@pytest.mark.parametrize("n,cond", [(8, 1.0), (64, 1.0), (64, 1e6), (256, 1e9), (1000, 1.0)])
def test_dot2_meets_its_error_bound(arith_exe, n, cond):
    """Dot2 of split operands against the exact rational dot product of the same split
    values: within gamma_n^2 + 2^-44 of sum|x_i y_i|, also when the sum cancels (cond =
    sum|x_i y_i| / |x . y| up to 1e9), where the plain FP32 sum is off by orders of
    magnitude."""
    from fractions import Fraction as F
    rng = np.random.default_rng(n + int(np.log10(cond)))
    x = rng.standard_normal(n) * np.exp2(rng.integers(-8, 8, n))
    y = rng.standard_normal(n) * np.exp2(rng.integers(-8, 8, n))
    if cond > 1:
        # make the last product cancel the others up to 1/cond of their magnitude
        partial = float(np.dot(x[:-1], y[:-1]))
        scale = float(np.sum(np.abs(x * y)))
        y[-1] = (-partial + scale / cond * rng.standard_normal()) / x[-1]
    (s, c, naive), = run_arith(arith_exe, 2, x, y)
    exact = _exact_split_dot(x, y)
    pairs_x, pairs_y = run_split_pairs(x), run_split_pairs(y)
    sabs = sum(abs((F(a) + F(b)) * (F(c2) + F(d))) for (a, b), (c2, d) in zip(pairs_x, pairs_y))
    u = 2.0 ** -24
    gam = n * u / (1 - n * u)
    bound = (gam * gam + 2.0 ** -44) * float(sabs)
    err = abs(float(F(s) + F(c) - exact))
    assert err <= bound, (err, bound)
    if cond >= 1e6:
        assert abs(float(F(naive) - exact)) > 100 * bound    # FP32 alone fails here
