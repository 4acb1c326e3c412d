"""Natural-parameter continuation in Ra (Sec. 4.3 of the paper), plain Python over the oracle.

Test infrastructure: imported only by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg.

The paper's continuation adds no equation to Newton's method; it only chooses the next
parameter value and the initial estimate:
  * Eq. new_Ra: Ra^(i+1) = Ra^(i) + alpha (Ra^(i) - Ra^(i-1));
  * Eq. alpha_cont: alpha = (N_opt + 1) / (N^(i) + 1), N^(i) the Newton iterations of the
    last point;
  * Eq. lagrange: quadratic Lagrange extrapolation through the last three points,
    Ra^(i+1) = a Ra^(i) + b Ra^(i-1) + c Ra^(i-2) fixes (a, b, c), and
    U^(i+1) = a U^(i) + b U^(i-1) + c U^(i-2) is the estimate (the drift C likewise);
  * Eqs. tp_detection_Ra / quad_extra_Ra (turning points): when
    |Delta U_J / U_J| > gamma |Delta Ra / Ra|, U_J becomes the independent variable:
    U_J^(i+1) = U_J^(i) + alpha (U_J^(i) - U_J^(i-1)) fixes (a, b, c) and
    Ra^(i+1) = a Ra^(i) + b Ra^(i-1) + c Ra^(i-2).
Readings (the passage is partly garbled):
  * J is the element of largest magnitude of U - U_cond (the deviation from the
    conductive state; the total temperature's conductive profile would otherwise always
    be the largest element and never change);
  * the comparison chooses the independent variable at every step: U_J while
    |Delta U_J / U_J| > gamma |Delta Ra / Ra|, Ra otherwise;
  * with two points the extrapolation is linear, with one it is the last point;
  * a Newton failure retries the step with alpha halved, at most `retries` times.
"""
import numpy as np

from . import krylov


def lagrange_coefficients(x, xs):
    """Weights (a, b, c) of the values at nodes xs = (x_i, x_{i-1}, x_{i-2}) (or fewer) that
    interpolate at x (Lagrange basis polynomials evaluated at x)."""
    k = len(xs)
    w = np.zeros(3)
    for p in range(k):
        v = 1.0
        for q in range(k):
            if q != p:
                v *= (x - xs[q]) / (xs[p] - xs[q])
        w[p] = v
    return w


def predict(Ra, s, n_its, n_opt, gamma, alpha_scale=1.0):
    """Next parameter value and extrapolation weights.

    Ra, s: values at the last points, most recent first (1 to 3 entries), s = U_J at the
    most recent point's J.  Returns (mode, Ra_new, (a, b, c)), mode 0 = Ra independent,
    1 = U_J independent.  Needs at least two points."""
    k = min(len(Ra), 3)
    if k < 2:
        raise ValueError("prediction needs two converged points")
    alpha = alpha_scale * (n_opt + 1.0) / (n_its + 1.0)
    dRa = (Ra[0] - Ra[1]) / Ra[0]
    ds = (s[0] - s[1]) / s[0] if s[0] != 0.0 else 0.0
    mode = 1 if abs(ds) > gamma * abs(dRa) else 0
    if mode == 0:
        Ra_new = Ra[0] + alpha * (Ra[0] - Ra[1])
        w = lagrange_coefficients(Ra_new, list(Ra[:k]))
    else:
        s_new = s[0] + alpha * (s[0] - s[1])
        w = lagrange_coefficients(s_new, list(s[:k]))
        Ra_new = float(np.dot(w[:k], Ra[:k]))
    return mode, Ra_new, w


def follow(solve, U0, C0, Ra0, Ra1, Ra_end, ucond, n_opt=4, gamma=20.0, max_points=8,
           retries=3):
    """The continuation loop over a Newton solver `solve(U, C, Ra) -> (U, C, its, ok)`.
    Returns the converged points, each dict(Ra, C, its, mode, U)."""
    pts = []
    U, C, its, ok = solve(np.array(U0, dtype=float), C0, Ra0)
    if not ok:
        return pts
    pts.append(dict(Ra=Ra0, C=C, its=its, mode=0, U=U))
    U, C, its, ok = solve(np.array(U, dtype=float), C, Ra1)
    if not ok:
        return pts
    pts.append(dict(Ra=Ra1, C=C, its=its, mode=0, U=U))
    direction = np.sign(Ra1 - Ra0)
    while len(pts) < max_points:
        last = pts[-3:][::-1]
        dev = last[0]["U"] - ucond
        jmax = int(np.argmax(np.abs(dev)))
        Ra = [p["Ra"] for p in last]
        s = [p["U"][jmax] - ucond[jmax] for p in last]
        done = False
        for attempt in range(retries + 1):
            mode, Ra_new, w = predict(Ra, s, last[0]["its"], n_opt, gamma, 0.5 ** attempt)
            Ug = sum(w[q] * last[q]["U"] for q in range(len(last)))
            Cg = float(sum(w[q] * last[q]["C"] for q in range(len(last))))
            Un, Cn, its, ok = solve(Ug, Cg, Ra_new)
            if ok:
                pts.append(dict(Ra=Ra_new, C=Cn, its=its, mode=mode, U=Un))
                done = True
                break
        if not done:
            break
        if direction * (pts[-1]["Ra"] - Ra_end) >= 0:
            break
    return pts


def continue_ra(shell, U0, C0, J, Ra0, Ra1, Ra_end, n_opt=4, gamma=20.0, max_points=8,
                tol=1e-10, max_newton=12, kmax=200, gmres_tol=1e-10, dt_newton=200.0,
                retries=3):
    """Follow a rotating-wave branch of `shell` from Ra0 towards Ra_end with the oracle's
    Newton-GMRES (J: the frozen phase slot of Sec. 3.4)."""

    def solve(U, C, Ra):
        shell.Ra = Ra     # Ra enters only the explicit part: the factorisations stay valid
        Us, Cs, hist = krylov.newton(shell, U, C, J, dt=dt_newton, tol=tol, max_newton=max_newton,
                                     kmax=kmax, gmres_tol=gmres_tol)
        return Us, Cs, len(hist) - 1, hist[-1]["residual"] < tol

    return follow(solve, U0, C0, Ra0, Ra1, Ra_end, shell.conductive_state(), n_opt, gamma,
                  max_points, retries)


def continue_ek(shell, U0, C0, J, Ek0, Ek1, Ek_end, ra_coef=0.0, n_opt=3, gamma=400.0,
                max_points=8, tol=1e-10, max_newton=12, kmax=200, gmres_tol=1e-10,
                dt_newton=200.0, retries=3):
    """Continuation in the Ekman number (Sec. 4.4, Eq. new_EK): the loop of `follow` with
    log10 Ek as the parameter; every new Ek refactorises, and with ra_coef > 0 the
    Rayleigh number follows Ra = ra_coef Ek^(-1/3).  Returns points whose "Ra" entry holds
    log10 Ek (as in `follow`)."""

    def solve(U, C, x):
        shell.Ek = 10.0 ** x
        if ra_coef > 0:
            shell.Ra = ra_coef * shell.Ek ** (-1.0 / 3.0)
        shell._fact = {}          # Ek enters the implicit operator: refactorise
        Us, Cs, hist = krylov.newton(shell, U, C, J, dt=dt_newton, tol=tol, max_newton=max_newton,
                                     kmax=kmax, gmres_tol=gmres_tol)
        return Us, Cs, len(hist) - 1, hist[-1]["residual"] < tol

    return follow(solve, U0, C0, np.log10(Ek0), np.log10(Ek1), np.log10(Ek_end),
                  shell.conductive_state(), n_opt, gamma, max_points, retries)


def regrid(vec, L0, Ms, Nr0, L1, Nr1):
    """Zero-fill (or truncate) the coefficients of a state between truncations of the same
    M_s (Sec. 4.4: the new modes of a refined grid start at zero)."""
    def pairs(L):
        return [(m, l) for m in range(0, L + 1, Ms) for l in range(m, L + 1)]
    p0 = {pl: i for i, pl in enumerate(pairs(L0))}
    x0 = np.asarray(vec, dtype=float).reshape(3, len(p0), Nr0, 2)
    P1 = pairs(L1)
    x1 = np.zeros((3, len(P1), Nr1, 2))
    k = min(Nr0, Nr1)
    for i, pl in enumerate(P1):
        if pl in p0:
            x1[:, i, :k] = x0[:, p0[pl], :k]
    return x1.reshape(-1)
