"""Pins of the oracle's GMRES and Newton iteration (Secs. 3.3-3.4).

* GMRES (Saad-Schultz, modified Gram-Schmidt) on the Jacobian action with the drift
  unknown against a dense LU solve of the same operator, assembled column by column.
* The rotating wave does not depend on the Newton pseudo-timestep: B(U) - U = P(dt) A(U)
  with P(dt) invertible (Eq. finalrhs), so the roots at dt = 200 and dt = 20 coincide.
* Newton converges quadratically once close to the wave (Eq. precond, Eq. twNewton).
* The converged wave is steady in its drifting frame, so two balances of the continuous
  equations hold on it to spectral accuracy (and fail on a state that is still evolving):
  the heat flux through the inner and outer walls is the same (Nu_in = Nu_out), and the
  buoyancy work equals the viscous dissipation.  With the momentum equation of the model,
  Ek dU/dt = Ek lap U - 2 e_z x U + Ek U x omega + Ra T r / r_out - grad p (Sec. 2), and
  no-slip walls, Coriolis and U x omega do no work and int U . lap U dV = -int |omega|^2 dV,
  so on the wave Ek int |omega|^2 dV = (Ra / r_out) int T r u_r dV.  The integrals are
  computed here by synthesis at Gauss-Legendre radii, independently of the time step.
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import basis, krylov
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


def _dissipation_and_work(s, vec):
    """(Ek int |omega|^2 dV, (Ra / r_out) int T r u_r dV) of a state: omega = curl U has
    poloidal potential e and toroidal potential -L_l f (Sec. 2.1); the fields are synthesised
    on the transform grid at 2 N_r + 16 Gauss-Legendre radii and integrated with the
    latitude weights, over the sector, and in r."""
    x = s.to_complex(vec)
    xq, wq = np.polynomial.legendre.leggauss(2 * s.Nr + 16)
    rq = basis.x_to_r(xq, s.r_in, s.r_out)
    E0, E1, E2 = (basis.cheb_matrix(xq, s.Nr, o, s.r_in, s.r_out) for o in range(3))
    e, f, T = x[0], x[1], x[2]
    r = rq[None, :]
    lam = s.lam[:, None]
    fv, f2, ev = f @ E0.T, f @ E2.T, e @ E0.T
    sp = s.sph

    def scalar(a):
        return sp.fourier_to_grid(sp.synth_scalar(s.split_m(a)))

    w_r = scalar(lam * ev / r ** 2)
    w_t, w_p = sp.synth_vector(s.split_m((e @ E1.T) / r), s.split_m(-(f2 - lam * fv / r ** 2) / r))
    w_t, w_p = sp.fourier_to_grid(w_t), sp.fourier_to_grid(w_p)
    u_r = scalar(lam * fv / r ** 2)
    Tg = scalar(T @ E0.T)
    wlat = sp.w[None, :, None]
    dphi = 2.0 * np.pi / sp.nphi
    rad = 0.5 * (s.r_out - s.r_in) * wq * rq ** 2

    def integral(g):
        return float((rad * (g * wlat).sum(axis=(0, 1)) * dphi).sum())

    D = integral(w_r ** 2 + w_t ** 2 + w_p ** 2)
    W = integral(Tg * u_r * rq[None, None, :])
    return s.Ek * D, s.Ra / s.r_out * W


@pytest.fixture(scope="module")
def rw4_fine():
    """The RW4 wave at L = 23, N_r = 20 (resolved to about 1e-4 in the balances below)."""
    s, U0, C0, J = _rw4_guess(23, 4, 20)
    U, C, hist = krylov.newton(s, U0, C0, J, dt=200.0, tol=1e-12, max_newton=12, kmax=300)
    assert hist[-1]["residual"] < 1e-12
    return s, U0, U


def _power_imbalance(s, vec):
    D, W = _dissipation_and_work(s, vec)
    return abs(D - W) / D


def _heat_imbalance(s, vec):
    nin, nout = s.nusselt(vec)
    return abs(nin - nout) / abs(nin - 1.0)


def test_rotating_wave_balances_heat_flux_and_power(rw4_fine):
    s, U0, U = rw4_fine
    assert _heat_imbalance(s, U) < 2e-3          # measured 2.4e-4
    assert _power_imbalance(s, U) < 5e-4         # measured 4.1e-5
    # the time-stepped guess is still evolving: neither balance holds
    assert _heat_imbalance(s, U0) > 0.1          # measured 0.34
    assert _power_imbalance(s, U0) > 1e-2        # measured 0.040


def test_balance_defects_are_truncation_errors(rw4, rw4_fine):
    """The imbalance of the converged wave falls by orders of magnitude from L = 15, N_r = 16
    to L = 23, N_r = 20 (a wrong factor in the model would leave an O(1) defect)."""
    s_c, sols = rw4
    s_f, _, U_f = rw4_fine
    coarse = _power_imbalance(s_c, sols[200.0][0])   # measured 1.4e-2
    fine = _power_imbalance(s_f, U_f)
    assert fine < coarse / 30.0
