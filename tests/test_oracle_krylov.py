"""Pins of the oracle's GMRES and Newton iteration (Secs. 3.3-3.4).

* GMRES (Saad-Schultz, modified Gram-Schmidt) on the Jacobian action with the drift
  unknown against a dense LU solve of the same operator, assembled column by column.
* The rotating wave does not depend on the Newton pseudo-timestep: B(U) - U = P(dt) A(U)
  with P(dt) invertible (Eq. finalrhs), so the roots at dt = 200 and dt = 20 coincide.
* Newton converges quadratically once close to the wave (Eq. precond, Eq. twNewton).
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import krylov
from oracle.shell import Shell


def test_gmres_matches_dense_lu_solve():
    L, Ms, Nr = 7, 4, 10
    s = Shell(L, Ms, Nr, 1e-3, 80.0)
    U = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=3, amp=3e-2)
    J = s.real_index("T", 4, 4, 1, 1)
    C, dt = 0.3, 200.0
    gU = s.grid_fields(s.to_complex(U))
    n = s.n
    A = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = s.jvp(U, C, J, e, dt, gU)
    b = np.random.default_rng(1).standard_normal(n)
    x_lu = np.linalg.solve(A, b)
    x, its, rel = krylov.gmres(lambda v: s.jvp(U, C, J, v, dt, gU), b, tol=1e-13, kmax=n)
    assert rel <= 1e-13 and its < n
    # cond(A) is about 2e5 here: 1e-13 relative residual bounds the error by ~2e-8; the
    # two solutions agree far better (1e-13) because GMRES converged well past the bound
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-11
    # and the Krylov solution solves the assembled system itself
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-12


def _rw4_guess(L, Ms, Nr):
    s = Shell(L, Ms, Nr, 1e-3, 120.0)
    M = 4
    x = s.to_complex(s.conductive_state())
    prof = 1e-2 * np.sin(np.pi * (s.rc - s.r_in))
    x[2, s.pair_index(M, M)] += np.linalg.solve(s.E[0], prof)
    U = s.step(s.to_real(x), 0.0, 2e-3, nsteps=400)
    U1 = s.step(U, 0.0, 2e-3, nsteps=5)
    return s, U, krylov.drift_estimate(s, U, U1, 5 * 2e-3, M), krylov.phase_index(s, U, M)


@pytest.fixture(scope="module")
def rw4():
    s, U0, C0, J = _rw4_guess(15, 4, 16)
    sols = {}
    for dt in (200.0, 20.0):
        U, C, hist = krylov.newton(s, U0, C0, J, dt=dt, tol=1e-12, max_newton=12, kmax=300)
        sols[dt] = (U, C, hist)
    return s, sols


def test_rotating_wave_does_not_depend_on_the_newton_timestep(rw4):
    s, sols = rw4
    (U1, C1, h1), (U2, C2, h2) = sols[200.0], sols[20.0]
    assert h1[-1]["residual"] < 1e-12 and h2[-1]["residual"] < 1e-12
    assert np.linalg.norm(U1 - U2) / np.linalg.norm(U1) < 1e-12
    assert abs(C1 - C2) < 1e-12 * abs(C1)
    # a drifting wave, not the conductive state
    assert abs(C1) > 1.0 and s.kinetic_energy(U1) > 1.0


def test_newton_converges_quadratically(rw4):
    _, sols = rw4
    r = [h["residual"] for h in sols[200.0][2]]
    assert all(b < a for a, b in zip(r, r[1:]))
    # the last step taken from a residual below 1e-4 at least squares it (up to a constant)
    k = next(i for i, v in enumerate(r) if v < 1e-4)
    assert k + 1 < len(r)
    assert np.log10(r[k + 1]) < 1.8 * np.log10(r[k])
