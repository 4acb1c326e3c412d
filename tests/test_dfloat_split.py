"""Host check of split48 (csrc/dfloat.h), the integer-only cut of a double into two floats
used by the double-float kernels (compiled here with the host C++ compiler).

The bound follows from the construction: hi keeps 24 significant bits, lo the next 29 bits
rounded to 24, so |d - hi - lo| <= 2^-48 |d| wherever both are normal floats.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2508_16635_gb300", "csrc")

DRIVER = r"""
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
    src.write_text(DRIVER)
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
