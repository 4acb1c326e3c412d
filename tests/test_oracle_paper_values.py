"""The oracle's rotating wave against the drift speed printed in Table 1 of the paper."""
import os

import numpy as np
import pytest

from oracle import krylov
from oracle.shell import Shell

HERE = os.path.dirname(os.path.abspath(__file__))


def table1():
    rows = []
    for line in open(os.path.join(HERE, "golden", "table1_drift.txt")):
        if line.strip() and not line.startswith("#"):
            ek, ra, M, nr, nth, nph, C = line.split()
            rows.append(dict(Ek=float(ek), Ra=float(ra), M=int(M), Nr=int(nr), Nth=int(nth), C=float(C)))
    return rows


def solve_rw_settled(L, Nr, Ek, Ra, M, dt, max_steps=20000):
    """Oracle time stepping from the m = M seed of seeded_inputs.mode_seed until the m = M
    temperature amplitude changes by less than 1e-4 per 100 steps, then Newton-GMRES."""
    import seeded_inputs as si
    s = Shell(L, M, Nr, Ek, Ra)
    U = s.conductive_state() + si.mode_seed(L, M, Nr, M, seed=4000, amp=1e-2)
    pM = s.pair_index(M, M)
    prev, steps = None, 0
    while steps < max_steps:
        U = s.step(U, 0.0, dt, nsteps=100)
        steps += 100
        amp = float(np.linalg.norm(s.to_complex(U)[2, pM]))
        if prev is not None and amp > 1e-3 and abs(amp - prev) < 1e-4 * amp:
            break
        prev = amp
    U1 = s.step(U, 0.0, dt, nsteps=10)
    C0 = krylov.drift_estimate(s, U, U1, 10 * dt, M)
    J = krylov.phase_index(s, U, M)
    Us, C, hist = krylov.newton(s, U, C0, J, dt=200.0, tol=1e-10, max_newton=10, kmax=400)
    return s, Us, C, hist


def solve_rw(L, Nr, Ek, Ra, M, nsteps, dt=2e-3):
    s = Shell(L, M, Nr, Ek, Ra)
    x = s.to_complex(s.conductive_state())
    prof = 1e-2 * np.sin(np.pi * (s.rc - s.r_in))
    x[2, s.pair_index(M, M)] += np.linalg.solve(s.E[0], prof)
    U = s.step(s.to_real(x), 0.0, dt, nsteps=nsteps)
    U1 = s.step(U, 0.0, dt, nsteps=5)
    C0 = krylov.drift_estimate(s, U, U1, 5 * dt, M)
    J = krylov.phase_index(s, U, M)
    Us, C, hist = krylov.newton(s, U, C0, J, dt=200.0, tol=1e-10, max_newton=12, kmax=120)
    return s, Us, C, hist


def test_rw4_drift_at_reduced_resolution():
    """Table 1 row 1 (Ek = 1e-3, Ra = 120, M = 4) at L = 31, N_r = 24: drift within 1e-3."""
    row = table1()[0]
    s, U, C, hist = solve_rw(31, 24, row["Ek"], row["Ra"], row["M"], nsteps=400)
    assert hist[-1]["residual"] < 1e-10
    assert abs(C - row["C"]) < 1e-3 * abs(row["C"])
    nu_in, nu_out = s.nusselt(U)
    assert abs(nu_in - nu_out) < 1e-4 * nu_in      # heat-flux balance of a steady wave


@pytest.mark.slow
def test_rw4_drift_at_paper_resolution():
    """Same wave at N_r = 46, N_theta = 72 (L = 47): every printed digit of C_exact."""
    row = table1()[0]
    L = 2 * row["Nth"] // 3 - 1
    s, U, C, hist = solve_rw(L, row["Nr"], row["Ek"], row["Ra"], row["M"], nsteps=600)
    assert hist[-1]["residual"] < 1e-10
    assert abs(C - row["C"]) < 5e-5            # the table prints 4 decimals


@pytest.mark.slow
def test_rw8_drift_at_paper_resolution():
    """Table 1 row 2 (Ek = 1e-4, Ra = 130, M = 8) at N_r = 60, N_theta = 80 (L = 52): the
    printed C_exact = 3.9998 to its last digit (about ten minutes on 8 cores)."""
    row = table1()[1]
    L = 2 * row["Nth"] // 3 - 1
    s, U, C, hist = solve_rw_settled(L, row["Nr"], row["Ek"], row["Ra"], row["M"], dt=5e-4)
    assert hist[-1]["residual"] < 1e-10
    assert abs(C - row["C"]) < 5e-5


def _golden(name):
    vals = {}
    for line in open(os.path.join(HERE, "golden", name)):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_rw12_drift_of_the_stored_oracle_wave():
    """Table 1 row 3 (Ek = 1e-5, Ra = 140, M = 12): the oracle's wave at the benchmark
    truncation L = 127, N_r = 64 (tests/golden/rw12_c3_oracle.txt, written by
    make_rw12_c3.py) against the printed C_exact = 51.2817.  The resolution study of the
    same wave (FP64 GPU path, L 89..191, N_r 64..96) converges to C = 51.24432 at L >= 127,
    N_r >= 96, and moves by at most 5e-4 between any of those grids; the printed value sits
    7.3e-4 above the converged one, so the pin is 1e-3 relative.  The heat flux through
    the two walls balances (Nu_in = Nu_out) to the truncation's accuracy."""
    row = table1()[2]
    g = _golden("rw12_c3_oracle.txt")
    assert g["residual"] < 1e-10
    assert abs(g["C"] - row["C"]) < 1e-3 * row["C"]
    assert abs(g["Nu_in"] - g["Nu_out"]) < 1e-6 * g["Nu_in"]


@pytest.mark.slow
def test_rw12_stored_oracle_wave_is_reproduced():
    """Recompute the stored RW12 wave with the script that wrote it (about 45 minutes)."""
    import subprocess
    import sys
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        env = dict(os.environ, RSC_GOLDEN_OUT=os.path.join(d, "rw12.txt"))
        subprocess.run([sys.executable, os.path.join(HERE, "golden", "make_rw12_c3.py")],
                       check=True, env=env)
        new = _golden_path_values(env["RSC_GOLDEN_OUT"])
    old = _golden("rw12_c3_oracle.txt")
    for k in ("C", "KE", "Nu_in", "Nu_out"):
        assert abs(new[k] - old[k]) < 1e-12 * abs(old[k]), k


def _golden_path_values(path):
    vals = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals
