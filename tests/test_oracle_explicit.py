"""Pins of the explicit-Coriolis variant (Eqs. expcor_e/f), the comparison scheme of Sec. 5.

Moving the Coriolis term between the implicit and the explicit part changes the
time step by O(dt^2) per step, and leaves the roots of B - I unchanged
(Eq. finalrhs: B - I = P(dt) A with the same A = N + L), so both schemes
converge to the same rotating wave; only the cost of the linear solves differs.
"""
import numpy as np

import seeded_inputs as si
from oracle import krylov
from oracle.shell import Shell


def test_explicit_and_implicit_steps_differ_at_second_order():
    L, Ms, Nr = 15, 4, 16
    x = None
    diffs = []
    for dt in (4e-5, 2e-5, 1e-5):
        si_ = Shell(L, Ms, Nr, 1e-3, 100.0)
        se = Shell(L, Ms, Nr, 1e-3, 100.0, coriolis="explicit")
        if x is None:
            x = si_.conductive_state() + si.perturbation(L, Ms, Nr, 5, amp=1e-2)
            x = si_.step(x, 0.0, 1e-4, nsteps=2)   # meet the boundary conditions first
        diffs.append(np.linalg.norm(si_.step(x, 0.0, dt) - se.step(x, 0.0, dt)))
    # the splitting error of one step scales like dt^2
    assert 3.5 < diffs[0] / diffs[1] < 4.5
    assert 3.5 < diffs[1] / diffs[2] < 4.5


def test_explicit_coriolis_terms_match_grid_force():
    """coriolis_terms is the same operator as the implicit rows (checked against 2 e_z x U on
    the grid in test_oracle_shell); here: it vanishes at m = 0 only for the diagonal part."""
    s = Shell(8, 1, 12, 1.0, 0.0)
    x = s.to_complex(si.perturbation(8, 1, 12, 6, amp=1.0))
    Kx = s.coriolis_terms(x)
    # rows of l = 0 are empty; the temperature rows are untouched
    assert np.all(Kx[:, s.pair_l == 0] == 0) and np.all(Kx[2] == 0)
    assert np.linalg.norm(Kx) > 0


def test_same_rotating_wave_with_either_scheme():
    L, Ms, Nr, Ek, Ra = 23, 4, 20, 1e-3, 120.0
    si_ = Shell(L, Ms, Nr, Ek, Ra)
    se = Shell(L, Ms, Nr, Ek, Ra, coriolis="explicit")
    x = si_.to_complex(si_.conductive_state())
    prof = 1e-2 * np.sin(np.pi * (si_.rc - si_.r_in))
    x[2, si_.pair_index(4, 4)] += np.linalg.solve(si_.E[0], prof)
    U0 = si_.step(si_.to_real(x), 0.0, 2e-3, nsteps=400)
    U1 = si_.step(U0, 0.0, 2e-3, nsteps=5)
    C0 = krylov.drift_estimate(si_, U0, U1, 1e-2, 4)
    J = krylov.phase_index(si_, U0, 4)
    Ui, Ci, hi = krylov.newton(si_, U0, C0, J, tol=1e-11, max_newton=12, kmax=150)
    Ue, Ce, he = krylov.newton(se, U0, C0, J, tol=1e-11, max_newton=12, kmax=400)
    assert hi[-1]["residual"] < 1e-11 and he[-1]["residual"] < 1e-11
    assert np.linalg.norm(Ui - Ue) < 1e-8 * np.linalg.norm(Ui)
    assert abs(Ci - Ce) < 1e-8 * abs(Ci)
    # Sec. 5: the implicit treatment needs fewer Jacobian actions per Newton step
    gi = sum(h.get("gmres_iterations", 0) for h in hi)
    ge = sum(h.get("gmres_iterations", 0) for h in he)
    assert ge > gi
