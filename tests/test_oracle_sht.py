"""Pins of the oracle's spherical-harmonic transforms: round trips and closed forms."""
import numpy as np
import pytest

from oracle import sht


def _random_coeffs(g, rng, lmin=0, extra=()):
    out = []
    for m in g.ms:
        a = rng.standard_normal((g.L - m + 1,) + extra) + 1j * rng.standard_normal((g.L - m + 1,) + extra)
        if m == 0:
            a = a.real + 0j
        a[: max(0, lmin - m)] = 0.0
        out.append(a)
    return out


@pytest.mark.parametrize("L,Ms", [(31, 4), (15, 1), (24, 3), (63, 8), (127, 12), (255, 8)])
def test_scalar_round_trip(L, Ms):
    g = sht.SphereGrid(L, Ms)
    a = _random_coeffs(g, np.random.default_rng(L), extra=(3,))
    grid = g.fourier_to_grid(g.synth_scalar(a))
    b = g.analyse_scalar(g.grid_to_fourier(grid))
    num = np.sqrt(sum((np.abs(x - y) ** 2).sum() for x, y in zip(a, b)))
    den = np.sqrt(sum((np.abs(x) ** 2).sum() for x in a))
    assert num / den < 1e-13      # relative 2-norm over all coefficients


@pytest.mark.parametrize("L,Ms", [(31, 4), (15, 1), (63, 8), (127, 12), (255, 8)])
def test_vector_round_trip(L, Ms):
    g = sht.SphereGrid(L, Ms)
    rng = np.random.default_rng(100 + L)
    S = _random_coeffs(g, rng, lmin=1, extra=(2,))
    T = _random_coeffs(g, rng, lmin=1, extra=(2,))
    vt, vp = g.synth_vector(S, T)
    gt, gp = g.fourier_to_grid(vt), g.fourier_to_grid(vp)
    S2, T2 = g.analyse_vector(g.grid_to_fourier(gt), g.grid_to_fourier(gp))
    num = np.sqrt(sum((np.abs(x - y) ** 2).sum() for x, y in zip(S + T, S2 + T2)))
    den = np.sqrt(sum((np.abs(x) ** 2).sum() for x in S + T))
    assert num / den < 1e-13      # relative 2-norm over all coefficients


def _single(g, l, m, val=1.0):
    a = [np.zeros(g.L - mm + 1, dtype=complex) for mm in g.ms]
    a[g.ms.index(m)][l - m] = val
    return a


def test_single_harmonics_closed_forms():
    g = sht.SphereGrid(6, 1)
    th, ph = np.meshgrid(g.theta, g.phi)  # [nphi, nlat]
    c, s = np.cos(th), np.sin(th)
    cases = [
        ((0, 0, 1.0), np.ones_like(th)),
        ((1, 0, 1.0), np.sqrt(3.0) * c),
        ((1, 1, 1.0), 2 * np.sqrt(3.0) * s * np.cos(ph)),                  # 2 Re(Y_1^1)
        ((1, 1, 1j), -2 * np.sqrt(3.0) * s * np.sin(ph)),
        ((2, 0, 1.0), np.sqrt(5.0) * 0.5 * (3 * c ** 2 - 1)),
        ((2, 2, 1.0), 2 * 3 * np.sqrt(10.0 / 24.0) * s ** 2 * np.cos(2 * ph)),
        ((3, 1, 1.0), 2 * np.sqrt(2 * 7 / 12.0) * 1.5 * (5 * c ** 2 - 1) * s * np.cos(ph)),
    ]
    for (l, m, v), ref in cases:
        grid = g.fourier_to_grid(g.synth_scalar(_single(g, l, m, v)))
        assert np.abs(grid - ref).max() < 1e-13, (l, m, v)


def test_vector_closed_forms():
    g = sht.SphereGrid(4, 1)
    th, ph = np.meshgrid(g.theta, g.phi)
    c, s = np.cos(th), np.sin(th)
    z = [np.zeros(g.L - m + 1, dtype=complex) for m in g.ms]
    # S = Y_1^0: v = grad_H (sqrt3 cos th) = (-sqrt3 sin th, 0)
    vt, vp = g.synth_vector(_single(g, 1, 0), z)
    assert np.abs(g.fourier_to_grid(vt) + np.sqrt(3) * s).max() < 1e-13
    assert np.abs(g.fourier_to_grid(vp)).max() < 1e-13
    # T = Y_1^0: v = (0, -d_th T) = (0, sqrt3 sin th)
    vt, vp = g.synth_vector(z, _single(g, 1, 0))
    assert np.abs(g.fourier_to_grid(vt)).max() < 1e-13
    assert np.abs(g.fourier_to_grid(vp) - np.sqrt(3) * s).max() < 1e-13
    # S = Y_1^1 (real field 2 sqrt3 sin th cos ph): v_th = 2 sqrt3 cos th cos ph, v_ph = -2 sqrt3 sin ph
    vt, vp = g.synth_vector(_single(g, 1, 1), z)
    assert np.abs(g.fourier_to_grid(vt) - 2 * np.sqrt(3) * c * np.cos(ph)).max() < 1e-13
    assert np.abs(g.fourier_to_grid(vp) + 2 * np.sqrt(3) * np.sin(ph)).max() < 1e-13


def test_dft_conventions():
    g = sht.SphereGrid(12, 4)
    rng = np.random.default_rng(5)
    G = rng.standard_normal((g.K + 1, 3)) + 1j * rng.standard_normal((g.K + 1, 3))
    G[0] = G[0].real
    vals = g.fourier_to_grid(G)
    # direct definition: real field = Re G_0 + 2 Re sum_{k>0} G_k exp(i k Ms phi)
    ref = np.zeros_like(vals)
    for k in range(g.K + 1):
        ref += (1 if k == 0 else 2) * (G[k][None, :] * np.exp(1j * k * g.Ms * g.phi)[:, None]).real
    assert np.abs(vals - ref).max() < 1e-13
    assert np.abs(g.grid_to_fourier(vals) - G).max() < 1e-13
