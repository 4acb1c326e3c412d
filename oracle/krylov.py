"""GMRES and the Newton iteration for steady states and rotating waves (Secs. 3.3-3.4).

Newton solves (B_U - I) u = (B - I) U (Eq. precond) with B the IMEX Euler step
at a large pseudo-timestep (dt = 200, Sec. 3.3), then sets U <- U - u.  For a
rotating wave the drift C is an extra unknown; its decrement c is carried in
slot J of u (the imaginary part of one coefficient, whose value is thereby
frozen: the phase condition of Sec. 3.4).

GMRES is the Saad-Schultz method with modified Gram-Schmidt, zero initial
guess, no restart, stopped when the least-squares residual falls below
tol * ||b|| (Sec. 3.3 accepts at relative 1e-10).

Pins: tests/test_oracle_krylov.py (GMRES against a dense LU solve of the
assembled Jacobian with the drift unknown; the converged rotating wave is the
same at pseudo-timesteps 200 and 20 (Eq. finalrhs); quadratic convergence of
Newton onto the wave; the converged wave balances the heat flux through the two
walls and the buoyancy work against the viscous dissipation, as a steady state
of the continuous equations does) and tests/test_oracle_paper_values.py (the
drift speeds of Table 1).
"""
import numpy as np


def gmres(apply, b, tol=1e-10, kmax=40):
    """Solve A x = b.  Returns (x, iterations, relative residual estimate)."""
    n = b.size
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return np.zeros(n), 0, 0.0
    V = np.zeros((kmax + 1, n))
    H = np.zeros((kmax + 1, kmax))
    V[0] = b / beta
    y = np.zeros(0)
    k = 0
    rel = 1.0
    for k in range(kmax):
        w = apply(V[k])
        for i in range(k + 1):                    # modified Gram-Schmidt
            H[i, k] = V[i] @ w
            w = w - H[i, k] * V[i]
        H[k + 1, k] = np.linalg.norm(w)
        rhs = np.zeros(k + 2)
        rhs[0] = beta
        y, *_ = np.linalg.lstsq(H[: k + 2, : k + 1], rhs, rcond=None)
        rel = np.linalg.norm(H[: k + 2, : k + 1] @ y - rhs) / beta
        if rel <= tol or H[k + 1, k] == 0.0:
            break
        V[k + 1] = w / H[k + 1, k]
    x = V[: k + 1].T @ y
    return x, k + 1, rel


def newton(shell, U, C=0.0, J=None, dt=200.0, tol=1e-10, max_newton=10, kmax=40,
           gmres_tol=1e-10, verbose=False):
    """Newton-GMRES with Stokes preconditioning (Eq. precond, Eq. twNewton).

    Returns (U, C, history) with history a list of dicts (residual norm, GMRES
    iterations) per Newton iteration.  J = None solves for a steady state.
    The residual norm is the Euclidean norm of the whole real vector B(U) - U.
    """
    U = np.array(U, dtype=np.float64, copy=True)
    hist = []
    for it in range(max_newton + 1):
        r = shell.step(U, C, dt) - U
        rn = float(np.linalg.norm(r))
        hist.append({"residual": rn})
        if verbose:
            print(f"newton {it}: |B(U)-U| = {rn:.3e}  C = {C:.12g}", flush=True)
        if rn < tol or it == max_newton:
            break
        gU = shell.grid_fields(shell.to_complex(U))
        x, its, rel = gmres(lambda v: shell.jvp(U, C, J, v, dt, gU), r, gmres_tol, kmax)
        hist[-1].update(gmres_iterations=its, gmres_relres=rel)
        c = 0.0
        if J is not None:
            c = x[J]
            x[J] = 0.0
        U = U - x
        C = C - c
    return U, C, hist


def phase_index(shell, U, M):
    """Phase slot J: Im of the T coefficient at (l = m = M, k*), k* = argmax_k |Re T_k,M,M|.

    (Sec. 3.4 leaves the choice of the single frozen component open.)
    """
    x = shell.to_complex(U)
    p = shell.pair_index(M, M)
    k = int(np.argmax(np.abs(x[2, p].real)))
    return shell.real_index("T", M, M, k, 1)


def drift_estimate(shell, U_a, U_b, t_ab, M):
    """C from the phase advance of the (l = m = M) T coefficients between two states t_ab apart.

    A rotating wave U(phi - C t) has coefficients a_m(t) = a_m(0) exp(-i m C t).
    """
    xa = shell.to_complex(U_a)[2, shell.pair_index(M, M)]
    xb = shell.to_complex(U_b)[2, shell.pair_index(M, M)]
    k = int(np.argmax(np.abs(xa)))
    dphase = np.angle(xb[k] / xa[k])
    return -dphase / (M * t_ab)
