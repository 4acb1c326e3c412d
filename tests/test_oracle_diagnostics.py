"""Pins of the oracle's diagnostics: kinetic energy and Nusselt numbers.

The oracle integrates |U|^2 on the transform grid (synthesis, Gauss-Legendre
and sector quadrature, Chebyshev interpolation in r).  The pin below reaches
the same number by a different route, Parseval's identity for the potentials
of Sec. 2.1 (U = curl(e r_hat) + curl curl(f r_hat)):

    int |U|^2 dOmega = ||Y_l^m||^2 [ l(l+1)|e|^2/r^2 + (l(l+1))^2 |f|^2/r^4
                                     + l(l+1) |d_r f|^2/r^2 ]

with ||Y_l^m||^2 = 4 pi (2 - delta_m0) for the normalisation of Eq. Ylm_norm,
and a factor 2 for m > 0 from the real field a Y + conj(a Y).
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle.shell import Shell


def parseval_ke(s, vec, nq=200):
    """KE density from the spectral coefficients (numpy Chebyshev evaluation)."""
    x = s.to_complex(vec)
    xq, wq = np.polynomial.legendre.leggauss(nq)
    r = 0.5 * (s.r_out - s.r_in) * xq + 0.5 * (s.r_out + s.r_in)
    dxdr = 2.0 / (s.r_out - s.r_in)
    total = 0.0
    pl, pm = si.layout(s.L, s.Ms, s.Nr)
    for p, (l, m) in enumerate(zip(pl, pm)):
        if l == 0:
            continue
        e = np.polynomial.chebyshev.chebval(xq, x[0, p])
        f = np.polynomial.chebyshev.chebval(xq, x[1, p])
        df = np.polynomial.chebyshev.chebval(xq, np.polynomial.chebyshev.chebder(x[1, p])) * dxdr
        ll = l * (l + 1.0)
        dens = (ll * np.abs(e) ** 2 / r ** 2 + ll ** 2 * np.abs(f) ** 2 / r ** 4
                + ll * np.abs(df) ** 2 / r ** 2)
        wm = 4.0 * np.pi if m == 0 else 16.0 * np.pi
        total += wm * 0.5 * (s.r_out - s.r_in) * np.sum(wq * r ** 2 * dens)
    V = 4.0 * np.pi * (s.r_out ** 3 - s.r_in ** 3) / 3.0
    return 0.5 * total / V


@pytest.mark.parametrize("L,Ms,Nr", [(7, 4, 10), (15, 2, 12), (12, 3, 9)])
def test_kinetic_energy_grid_quadrature_equals_parseval(L, Ms, Nr):
    s = Shell(L, Ms, Nr, 1e-3, 100.0)
    vec = si.perturbation(L, Ms, Nr, seed=L * 7 + Ms, amp=1.0)
    ke_grid = s.kinetic_energy(vec)
    ke_spec = parseval_ke(s, vec)
    assert ke_grid > 0
    assert abs(ke_grid - ke_spec) < 1e-12 * ke_spec


def test_kinetic_energy_single_toroidal_mode_closed_form():
    """e = T_0 (constant radial profile) at (l, m) = (1, 0): |U|^2 integrates to
    2 * 4 pi * int r^2 (1/r^2) dr = 8 pi (r_out - r_in), so KE = 4 pi (r_out - r_in) / V."""
    s = Shell(7, 1, 8, 1e-3, 100.0)
    x = np.zeros((3, s.P, s.Nr), complex)
    x[0, s.pair_index(1, 0), 0] = 1.0
    ke = s.kinetic_energy(s.to_real(x))
    V = 4.0 * np.pi * (s.r_out ** 3 - s.r_in ** 3) / 3.0
    assert abs(ke - 4.0 * np.pi * (s.r_out - s.r_in) / V) < 1e-13 * ke


def test_kinetic_energy_quadratic_scaling_and_zero_temperature_dependence():
    s = Shell(7, 4, 10, 1e-3, 100.0)
    vec = si.perturbation(7, 4, 10, seed=3, amp=1.0)
    ke = s.kinetic_energy(vec)
    assert abs(s.kinetic_energy(3.0 * vec) - 9.0 * ke) < 1e-12 * ke
    x = s.to_complex(vec)
    x[2] = 0.0
    assert abs(s.kinetic_energy(s.to_real(x)) - ke) < 1e-13 * ke


def test_nusselt_of_the_conductive_state_is_one():
    """Sec. 2.1: the conductive profile carries exactly the conductive heat flux."""
    s = Shell(15, 4, 24, 1e-3, 100.0)
    nu_in, nu_out = s.nusselt(s.conductive_state())
    assert abs(nu_in - 1.0) < 1e-11 and abs(nu_out - 1.0) < 1e-11


def test_nusselt_of_a_pure_l0_temperature_mode():
    """T_00 = 1/r (a harmonic profile) has d_r T = -1/r^2: Nu = 1/(r_out r_in) at both walls."""
    s = Shell(7, 4, 30, 1e-3, 100.0)
    x = np.zeros((3, s.P, s.Nr), complex)
    prof = 1.0 / s.rc
    x[2, s.pair_index(0, 0)] = np.linalg.solve(s.E[0], prof)
    nu_in, nu_out = s.nusselt(s.to_real(x))
    ref = 1.0 / (s.r_out * s.r_in)
    assert abs(nu_in - ref) < 1e-10 and abs(nu_out - ref) < 1e-10
