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
