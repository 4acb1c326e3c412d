"""Pins of the Ra continuation logic (Sec. 4.3, Eqs. new_Ra, alpha_cont, lagrange,
tp_detection_Ra, quad_extra_Ra) on closed-form branches."""
import numpy as np
import pytest

from oracle import continuation as ct


def test_lagrange_weights_reproduce_quadratics():
    xs = [1.3, 0.7, -0.4]
    for x in (2.0, 0.1, -1.0):
        w = ct.lagrange_coefficients(x, xs)
        assert abs(w.sum() - 1.0) < 1e-14
        for f in (lambda t: 3.0 - 2.0 * t + 0.5 * t * t, lambda t: t):
            assert abs(np.dot(w, [f(t) for t in xs]) - f(x)) < 1e-13
    w2 = ct.lagrange_coefficients(2.0, [1.0, 0.0])
    assert np.allclose(w2, [2.0, -1.0, 0.0])


def test_step_size_rule():
    """alpha = (N_opt + 1)/(N + 1): the increment is kept at N = N_opt, halved at 2 N_opt + 1."""
    Ra, s = [110.0, 100.0], [1.0, 0.999]
    assert ct.predict(Ra, s, 4, 4, 20.0)[1] == pytest.approx(120.0)
    assert ct.predict(Ra, s, 9, 4, 20.0)[1] == pytest.approx(115.0)
    assert ct.predict(Ra, s, 1, 4, 20.0)[1] == pytest.approx(135.0)


def _fold_solver(its=3):
    """Exact branches of a saddle-node at Ra = 10: 0 = (Ra - 10) - (x - 1)^2; a 'Newton solve'
    at Ra converges to the root on the side of the guess (x >= 1 upper, x < 1 lower)."""
    def solve(U, C, Ra):
        if Ra < 10.0:
            return U, C, its, False
        side = 1.0 if U[0] >= 1.0 else -1.0
        return np.array([1.0 + side * np.sqrt(Ra - 10.0)]), C, its, True
    return solve


def test_continuation_goes_around_a_turning_point():
    """From the upper branch towards smaller Ra the loop must switch to U_J as the
    independent variable near the fold, pass it and come back up along the lower branch."""
    pts = ct.follow(_fold_solver(), [1.0 + np.sqrt(2.0)], 0.0, 12.0, 11.6, 0.0, np.zeros(1),
                    n_opt=3, gamma=5.0, max_points=25)
    x = np.array([p["U"][0] for p in pts])
    Ra = np.array([p["Ra"] for p in pts])
    modes = [p["mode"] for p in pts]
    assert 1 in modes                                    # switched to U_J near the fold
    assert x.min() < 1.0 - 0.3                           # reached the lower branch
    k = int(np.argmin(Ra))
    assert Ra[k] < 10.2 and Ra[-1] > Ra[k] + 0.3         # Ra turned around
    assert np.all(np.abs(Ra - 10.0 - (x - 1.0) ** 2) < 1e-12)   # every point on the branch


def test_without_switching_the_fold_is_not_passed():
    """gamma so large that Ra stays the independent variable: the continuation stops at the
    fold (no solution beyond it) instead of turning."""
    pts = ct.follow(_fold_solver(), [1.0 + np.sqrt(2.0)], 0.0, 12.0, 11.6, 0.0, np.zeros(1),
                    n_opt=3, gamma=1e9, max_points=25)
    x = np.array([p["U"][0] for p in pts])
    assert x.min() > 1.0 - 1e-9 and all(p["mode"] == 0 for p in pts)   # never below the fold
