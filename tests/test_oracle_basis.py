"""Pins of the oracle's radial and angular tables against closed forms and libraries."""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import basis

R_IN, R_OUT = basis.shell_radii(0.35)


def test_radii_match_paper():
    # Sec. 2.1: r_out = 20/13, r_in = 7/13 for eta = 0.35 and unit gap.
    assert abs(R_OUT - 20.0 / 13.0) < 1e-15
    assert abs(R_IN - 7.0 / 13.0) < 1e-15


def test_chebyshev_values_are_cos_k_arccos():
    x = np.random.default_rng(1).uniform(-1, 1, 50)
    M = basis.cheb_matrix(x, 30, 0, R_IN, R_OUT)
    ref = np.cos(np.arange(30)[None, :] * np.arccos(x)[:, None])
    assert np.abs(M - ref).max() < 1e-13


def test_chebyshev_endpoint_derivatives_closed_form():
    k = np.arange(25.0)
    d1 = basis.cheb_matrix(np.array([1.0, -1.0]), 25, 1, R_IN, R_OUT) / 2.0  # d/dx = (1/2) d/dr
    d2 = basis.cheb_matrix(np.array([1.0, -1.0]), 25, 2, R_IN, R_OUT) / 4.0
    assert np.allclose(d1[0], k ** 2, rtol=1e-13, atol=1e-12)
    assert np.allclose(d1[1], (-1.0) ** (k + 1) * k ** 2, rtol=1e-13, atol=1e-12)
    assert np.allclose(d2[0], k ** 2 * (k ** 2 - 1) / 3.0, rtol=1e-12, atol=1e-10)
    assert np.allclose(d2[1], (-1.0) ** k * k ** 2 * (k ** 2 - 1) / 3.0, rtol=1e-12, atol=1e-10)


def test_chebyshev_differentiates_polynomials_exactly():
    rng = np.random.default_rng(2)
    n = 14
    a = rng.standard_normal(n)            # p(r) = sum a_j (r - 1)^j
    xs = basis.lobatto_x(n)
    rs = basis.x_to_r(xs, R_IN, R_OUT)
    vals = np.polynomial.polynomial.polyval(rs - 1.0, a)
    coef = np.linalg.solve(basis.cheb_matrix(xs, n, 0, R_IN, R_OUT), vals)
    rq = np.linspace(R_IN, R_OUT, 17)
    xq = 2 * rq - R_IN - R_OUT
    for order in range(5):
        got = basis.cheb_matrix(xq, n, order, R_IN, R_OUT) @ coef
        ref = np.polynomial.polynomial.polyval(rq - 1.0, np.polynomial.polynomial.polyder(a, order) if order else a)
        assert np.abs(got - ref).max() < 1e-9 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("n", [4, 12, 48, 96])
def test_gauss_legendre_exact_on_monomials(n):
    x, w = basis.gauss_legendre(n)
    assert np.all(np.diff(x) < 0)            # north first
    for k in range(2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs((w * x ** k).sum() - exact) < 1e-13


@pytest.mark.parametrize("n", [192, 384])
def test_gauss_legendre_weights_at_large_n(n):
    """Sum_j w_j P_k(x_j) = 2 delta_k0 for every k < 2n, with P_k from scipy.

    Double-precision Newton (as in numpy's leggauss) misses this by 2-4e-14
    because the weights near the poles carry 1e-10 relative errors; the
    oracle's nodes and weights meet it at the rounding level.
    """
    x, w = basis.gauss_legendre(n)
    s = basis.gauss_legendre_sin(n)
    assert np.abs(s * s + x * x - 1.0).max() < 4e-16
    for k in range(2 * n):
        v = (w * sp.eval_legendre(k, x)).sum() - (2.0 if k == 0 else 0.0)
        assert abs(v) < 3e-15, k


def _n_lm(l, m):
    return math.sqrt((2.0 - (m == 0)) * (2 * l + 1)
                     * math.exp(math.lgamma(l - m + 1) - math.lgamma(l + m + 1)))


def test_plm_against_scipy_lpmv():
    x = np.linspace(-0.95, 0.95, 11)
    for m in range(0, 9):
        tab = basis.ylm_norm_factor(m) * basis.plm_bar(20, m, x)
        for l in range(m, 21):
            # scipy includes the Condon-Shortley phase (-1)^m; Eq. Ylm_norm has none.
            ref = _n_lm(l, m) * (-1.0) ** m * sp.lpmv(m, l, x)
            assert np.allclose(tab[l - m], ref, rtol=1e-11, atol=1e-12), (l, m)


def test_discrete_orthogonality():
    L = 31
    x, w = basis.gauss_legendre(basis.nlat_for(L))
    for m in (0, 4, 17, 31):
        p = basis.ylm_norm_factor(m) * basis.plm_bar(L, m, x)
        G = (p * w) @ p.T
        assert np.abs(G - 2.0 * (2.0 - (m == 0)) * np.eye(L - m + 1)).max() < 5e-13


@pytest.mark.parametrize("L,Ms", [(127, 12), (255, 8)])
def test_discrete_orthogonality_large_truncations(L, Ms):
    n = basis.nlat_for(L)
    x, w = basis.gauss_legendre(n)
    s = basis.gauss_legendre_sin(n)
    for m in range(0, L + 1, Ms):
        p = basis.ylm_norm_factor(m) * basis.plm_bar(L, m, x, s)
        G = (p * w) @ p.T / (2.0 * (2.0 - (m == 0)))
        assert np.abs(G - np.eye(L - m + 1)).max() < 5e-14, m


def test_unsold_sum_rule_at_L255():
    """Unsold's theorem: sum_m |Y_l^m|^2 = (2l+1)/(4 pi), i.e.
    sum_{m=0..l} (2 - delta_m0) pbar_l^m(x)^2 = 2l + 1 at every x."""
    L = 255
    n = basis.nlat_for(L)
    x = basis.gauss_legendre(n)[0]
    s = basis.gauss_legendre_sin(n)
    acc = np.zeros((L + 1, n))
    for m in range(L + 1):
        acc[m:] += (2.0 - (m == 0)) * basis.plm_bar(L, m, x, s) ** 2
    ref = (2.0 * np.arange(L + 1) + 1.0)[:, None]
    assert np.abs(acc / ref - 1.0).max() < 2e-13


def _pbar_rodrigues(l, m, t):
    """pbar_l^m at s = 2t/(1+t^2), x = (1-t^2)/(1+t^2) (t rational), from
    P_l^m = (1-x^2)^{m/2} d^m/dx^m P_l(x) with the explicit coefficients of P_l,
    all in exact rational arithmetic; only the normalisation's square root is
    taken in 60-digit decimal arithmetic.  Returns a Decimal."""
    import decimal
    from fractions import Fraction
    x = (1 - t * t) / (1 + t * t)
    s = 2 * t / (1 + t * t)
    # P_l(x) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k, l) x^(l-2k)
    total = Fraction(0)
    for k in range(l // 2 + 1):
        deg = l - 2 * k
        if deg < m:
            continue
        c = Fraction((-1) ** k * math.comb(l, k) * math.comb(2 * l - 2 * k, l), 2 ** l)
        c *= math.perm(deg, m)            # d^m/dx^m x^deg = deg!/(deg-m)! x^(deg-m)
        total += c * x ** (deg - m)
    val = total * s ** m
    with decimal.localcontext() as ctx:
        ctx.prec = 60
        ctx.Emin, ctx.Emax = -999999, 999999
        norm = (decimal.Decimal((2 * l + 1) * math.factorial(l - m))
                / decimal.Decimal(math.factorial(l + m))).sqrt()
        return norm * decimal.Decimal(val.numerator) / decimal.Decimal(val.denominator)


def test_plm_scaled_start_against_rodrigues():
    """Near the pole the start pbar_m^m ~ s^m is far below the double range, but
    pbar_l^m grows back into it for large l: the scaled start must reproduce
    the exact values there, and entries that stay below the range must be 0."""
    from fractions import Fraction
    import decimal
    t = Fraction(1, 2000)                      # s ~ 1e-3
    m, lmax = 120, 420
    s = float(2 * t / (1 + t * t))
    x = float((1 - t * t) / (1 + t * t))
    tab = basis.plm_bar(lmax, m, np.array([x]), np.array([s]))[:, 0]
    assert tab[0] == 0.0                       # s^120 ~ 1e-360: below the range
    for l in (346, 360, 400, 420):
        ref = _pbar_rodrigues(l, m, t)
        assert abs(decimal.Decimal(tab[l - m]) / ref - 1) < decimal.Decimal("1e-13"), l
    # mid-latitude: every row against the closed form
    t2 = Fraction(1, 3)
    s2, x2 = float(2 * t2 / (1 + t2 * t2)), float((1 - t2 * t2) / (1 + t2 * t2))
    tab2 = basis.plm_bar(60, 17, np.array([x2]), np.array([s2]))[:, 0]
    for l in (17, 18, 30, 60):
        ref = _pbar_rodrigues(l, 17, t2)
        assert abs(decimal.Decimal(tab2[l - 17]) - ref) < decimal.Decimal("1e-13") * (1 + abs(ref))


def test_recursions_of_the_paper_hold_on_the_grid():
    """Eq. recu1 and Eq. recu2, written with the N_l^m ratios of Eq. recu1_b / recu2_b."""
    L = 24
    x, _ = basis.gauss_legendre(basis.nlat_for(L))
    s = np.sqrt(1 - x * x)
    for m in (0, 1, 3, 8):
        f = basis.ylm_norm_factor(m)
        Y = f * basis.plm_bar(L, m, x)
        dY = f * basis.dplm_bar_dtheta(L, m, x)
        for l in range(m, L):
            up = l * (l - m + 1) / (2 * l + 1) * _n_lm(l, m) / _n_lm(l + 1, m) * Y[l + 1 - m]
            cu = (l - m + 1) / (2 * l + 1) * _n_lm(l, m) / _n_lm(l + 1, m) * Y[l + 1 - m]
            dn = cd = 0.0
            if l - 1 >= m:
                dn = (l + m) * (l + 1) / (2 * l + 1) * _n_lm(l, m) / _n_lm(l - 1, m) * Y[l - 1 - m]
                cd = (l + m) / (2 * l + 1) * _n_lm(l, m) / _n_lm(l - 1, m) * Y[l - 1 - m]
            assert np.allclose(s * dY[l - m], up - dn, atol=1e-12), (l, m)
            assert np.allclose(x * Y[l - m], cu + cd, atol=1e-12), (l, m)


def test_dtheta_against_finite_differences():
    th = np.linspace(0.2, 2.9, 9)
    h = 1e-5
    for m in (0, 2, 5):
        d = basis.dplm_bar_dtheta(15, m, np.cos(th))
        fd = (basis.plm_bar(15, m, np.cos(th + h)) - basis.plm_bar(15, m, np.cos(th - h))) / (2 * h)
        assert np.abs(d - fd).max() < 1e-7 * max(1.0, np.abs(d).max())


def test_grid_sizes():
    assert basis.nlat_for(31) == 48 and basis.nlat_for(63) == 96 and basis.nlat_for(127) == 192
    assert basis.nlat_for(47) == 72          # the paper's N_theta at (46, 72, 32x4)
    assert basis.nphi_for(31, 4) == 24 and basis.nphi_for(63, 8) == 24
    assert basis.nphi_for(127, 12) == 32 and basis.nphi_for(255, 8) == 96
    assert basis.dealias_nr(24) == 36 and basis.dealias_nr(64) == 96
