"""Pins of the oracle's second-order time step (Crank-Nicolson + Heun, the time-stepping
scheme of Sec. 5): closed-form decay, fixed points, and the order of accuracy."""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import basis
from oracle.shell import Shell


@pytest.mark.parametrize("Pr", [1.0, 0.3])
def test_crank_nicolson_factor_for_temperature_modes(Pr):
    """At Ra = 0 the l = 0 mode sin(n pi (r - r_in))/r decays at (n pi)^2/Pr; one step of the
    scheme multiplies it by the Crank-Nicolson factor (1 - z/2)/(1 + z/2), z = dt (n pi)^2/Pr."""
    s = Shell(15, 4, 32, 1e-3, 0.0, Pr=Pr)
    U = s.to_complex(s.conductive_state())
    p00 = s.pair_index(0, 0)
    A = basis.cheb_matrix(s.xc, s.Nr, 0, s.r_in, s.r_out)
    dt = 3e-3
    for n in (1, 2, 3):
        prof = 1e-2 * np.sin(n * np.pi * (s.rc - s.r_in)) / s.rc
        x = U.copy()
        x[2, p00] += np.linalg.solve(A, prof)
        y = s.to_complex(s.step2(s.to_real(x), dt))
        got = A @ (y[2, p00] - U[2, p00]).real
        z = dt * (n * np.pi) ** 2 / Pr
        ref = prof * (1.0 - 0.5 * z) / (1.0 + 0.5 * z)
        assert np.abs(got - ref).max() < 1e-10 * np.abs(prof).max()


def test_conductive_state_is_a_fixed_point():
    s = Shell(15, 4, 24, 1e-3, 150.0)
    c = s.conductive_state()
    assert np.abs(s.step2(c, 1e-3) - c).max() < 1e-12


@pytest.mark.parametrize("coriolis", ["implicit", "explicit"])
def test_second_order_in_time(coriolis):
    """Self-convergence over a fixed interval: the error ratio between dt and dt/2 is 4
    (second order) for the scheme, 2 for the IMEX Euler step of Eq. discrete."""
    L, Ms, Nr = 7, 4, 10
    s = Shell(L, Ms, Nr, 1e-2, 120.0, coriolis=coriolis)
    x0 = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=5, amp=5e-2)
    x0 = s.step(x0, 0.0, 1e-4)          # a state that satisfies the boundary conditions
    T = 4e-3
    runs2 = {k: s.step2(x0, T / k, nsteps=k) for k in (4, 8, 16, 64)}
    e1 = np.linalg.norm(runs2[4] - runs2[64])
    e2 = np.linalg.norm(runs2[8] - runs2[64])
    e3 = np.linalg.norm(runs2[16] - runs2[64])
    r2 = [e1 / e2, e2 / e3]
    runs1 = {k: s.step(x0, 0.0, T / k, nsteps=k) for k in (4, 8, 64)}
    r1 = np.linalg.norm(runs1[4] - runs1[64]) / np.linalg.norm(runs1[8] - runs1[64])
    assert 3.3 < r2[0] < 5.0 and 3.3 < r2[1] < 5.5, r2
    assert 1.6 < r1 < 2.6, r1
