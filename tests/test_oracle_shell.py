"""Pins of the oracle's model against physics and mathematics (not against itself).

Each test names the property it checks; a dropped term, a wrong sign, index
or coefficient anywhere in the step fails at least one of them.
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import basis
from oracle.shell import BC_ROWS, FIELDS, Shell


def _low_degree_state(s, rng, kmax=8, bc=True, fields=(0, 1, 2), amp=1.0):
    """Random smooth state (Chebyshev degree < kmax) that meets no-slip / zero-T walls."""
    x = np.zeros((3, s.P, s.Nr), dtype=complex)
    for fi in fields:
        z = (rng.standard_normal((s.P, kmax)) + 1j * rng.standard_normal((s.P, kmax))) * amp
        x[fi, :, :kmax] = z
    x[:, s.pair_m == 0] = x[:, s.pair_m == 0].real
    x[0:2, s.pair_l == 0] = 0.0
    if bc:
        # project each radial profile onto the null space of its wall conditions
        E0, E1 = s.E[0], s.E[1]
        for fi, fl in enumerate(FIELDS):
            rows = [E0[0], E0[-1]] if fl in ("e", "T") else [E0[0], E0[-1], E1[0], E1[-1]]
            B = np.array(rows)[:, :kmax]
            Q, _ = np.linalg.qr(B.T, mode="complete")
            N = Q[:, len(rows):]                   # orthonormal basis of the null space
            x[fi, :, :kmax] = (x[fi, :, :kmax] @ N) @ N.T
    return x


def _interior(field, Nr):
    rows = np.ones(Nr, dtype=bool)
    for j in BC_ROWS[field]:
        rows[j] = False
    return rows


def _radial_quadrature(s, n=120):
    xq, wq = np.polynomial.legendre.leggauss(n)
    rq = basis.x_to_r(xq, s.r_in, s.r_out)
    E = [basis.cheb_matrix(xq, s.Nr, o, s.r_in, s.r_out) for o in range(5)]
    return rq[:, None], 0.5 * (s.r_out - s.r_in) * wq, E


# ---------------------------------------------------------------------------
def test_conductive_state_matches_closed_form_and_is_fixed_point():
    s = Shell(31, 4, 24, 1e-3, 120.0)
    U = s.conductive_state()
    T00 = s.to_complex(U)[2, s.pair_index(0, 0)]
    r = np.linspace(s.r_in, s.r_out, 31)
    vals = basis.cheb_matrix(2 * r - s.r_in - s.r_out, s.Nr, 0, s.r_in, s.r_out) @ T00.real
    assert np.abs(vals - (s.r_out * s.r_in / r - s.r_in)).max() < 1e-12   # Sec. 2.1
    for dt in (1e-4, 200.0):
        assert np.abs(s.step(U, 0.0, dt) - U).max() < 1e-13


@pytest.mark.parametrize("Pr", [1.0, 2.5])
def test_ra0_decay_of_spherical_temperature_modes(Pr):
    """Mode sin(n pi (r - r_in))/r of the l = 0 Laplacian decays at (n pi)^2 / Pr per unit time.

    One implicit Euler step multiplies it by 1 / (1 + dt (n pi)^2 / Pr) (Eq. discrete).
    """
    s = Shell(15, 4, 32, 1e-3, 0.0, Pr=Pr)
    U = s.to_complex(s.conductive_state())
    p00 = s.pair_index(0, 0)
    A = basis.cheb_matrix(s.xc, s.Nr, 0, s.r_in, s.r_out)
    dt = 3e-3
    for n in (1, 2, 3):
        prof = 1e-2 * np.sin(n * np.pi * (s.rc - s.r_in)) / s.rc
        x = U.copy()
        x[2, p00] += np.linalg.solve(A, prof)
        y = s.to_complex(s.step(s.to_real(x), 0.0, dt))
        got = A @ (y[2, p00] - U[2, p00]).real
        ref = prof / (1.0 + dt * (n * np.pi) ** 2 / Pr)
        assert np.abs(got - ref).max() < 1e-11 * np.abs(prof).max() * 10


def test_coriolis_does_no_work():
    """int U.(2 e_z x U) dV = 0 (Sec. 3.2): the l +- 1 couplings of e and f are mutually adjoint.

    Integrating by parts, int U.G dV = sum_lm w_m int r^2 Re[e conj(e_r.curl G)
    + f conj(e_r.curl curl G)] dr for f = 0 at the walls, with w_0 = 4 pi,
    w_{m>0} = 16 pi for the normalisation of Eq. Ylm_norm.  The e_r.curl and
    e_r.curl curl of 2 e_z x U are the Coriolis rows of Eqs. impcor_e_final /
    impcor_f_final.
    """
    s = Shell(10, 1, 20, 1.0, 0.0)
    rng = np.random.default_rng(3)
    x = _low_degree_state(s, rng, kmax=12)
    rq, wq, E = _radial_quadrature(s)
    vals = {}
    for fi, fl in enumerate(("e", "f")):
        vals[fl] = np.stack([E[0] @ x[fi, p] for p in range(s.P)])
    total, scale = 0.0, 0.0
    for p in range(s.P):
        l, m = int(s.pair_l[p]), int(s.pair_m[p])
        w = 4 * np.pi if m == 0 else 16 * np.pi
        for fi, fl in enumerate(("e", "f")):
            other = 1 - fi
            G = s.coriolis_diag_rows(fl, l, m, E, rq) @ x[fi, p]
            if l - 1 >= m:
                G = G + s.coupling_rows(l, m, -1, E, rq) @ x[other, p - 1]
            if l + 1 <= s.L:
                G = G + s.coupling_rows(l, m, +1, E, rq) @ x[other, p + 1]
            term = w * np.sum(wq * rq[:, 0] ** 2 * np.real(vals[fl][p] * np.conj(G)))
            total += term
            scale += abs(term)
    assert scale > 1.0
    assert abs(total) < 1e-12 * scale


def _coriolis_force_grid(s, x):
    """2 e_z x U on the grid: e_z = cos th r_hat - sin th th_hat."""
    g = s.grid_fields(x)
    c = np.cos(s.sph.theta)[None, :, None]
    sn = np.sin(s.sph.theta)[None, :, None]
    Gr = 2 * (-sn * g["up"])
    Gt = 2 * (-c * g["up"])
    Gp = 2 * (c * g["ut"] + sn * g["ur"])
    return Gr, Gt, Gp


def test_grid_coriolis_equals_spectral_l_pm1_formula():
    """The curl projections of 2 e_z x U computed on the grid equal the Coriolis rows of Eqs.
    impcor_e_final / impcor_f_final (diagonal -2im/r^2 e, +2im/r^2 L_l f and l +- 1 couplings)."""
    s = Shell(8, 1, 40, 1.0, 0.0)
    rng = np.random.default_rng(4)
    x = _low_degree_state(s, rng, kmax=8, bc=False, fields=(0, 1))
    Gr, Gt, Gp = _coriolis_force_grid(s, x)
    Ne, Nf, _ = s.curl_terms(*s.analyse(Gr, Gt, Gp, np.zeros_like(Gr)))
    got = {"e": Ne, "f": Nf}
    r = s.rc[:, None]
    worst = 0.0
    for p in range(s.P):
        l, m = int(s.pair_l[p]), int(s.pair_m[p])
        if l == 0:
            continue
        for fi, fl in enumerate(("e", "f")):
            other = 1 - fi
            ref = s.coriolis_diag_rows(fl, l, m, s.E, r) @ x[fi, p]
            if l - 1 >= m:
                ref = ref + s.coupling_rows(l, m, -1, s.E, r) @ x[other, p - 1]
            if l + 1 <= s.L:
                ref = ref + s.coupling_rows(l, m, +1, s.E, r) @ x[other, p + 1]
            rows = _interior(fl, s.Nr)
            err = np.abs(got[fl][p][rows] - ref[rows]).max() / max(1.0, np.abs(ref[rows]).max())
            worst = max(worst, err)
    assert worst < 1e-10


def test_curl_of_a_gradient_vanishes():
    s = Shell(12, 2, 30, 1.0, 0.0)
    rng = np.random.default_rng(5)
    phi = _low_degree_state(s, rng, kmax=8, bc=False, fields=(2,))[2]
    q = s.split_m(phi @ s.Ed[1].T)         # d_r phi
    S = s.split_m((phi @ s.Ed[0].T) / s.rd[None, :])
    zero = [np.zeros_like(a) for a in S]
    sp = s.sph
    Fr = sp.fourier_to_grid(sp.synth_scalar(q))
    Ft, Fp = (sp.fourier_to_grid(v) for v in sp.synth_vector(S, zero))
    Ne, Nf, _ = s.curl_terms(*s.analyse(Fr, Ft, Fp, np.zeros_like(Fr)))
    scale = np.abs(phi).max() * 100
    assert np.abs(Ne).max() < 1e-10 * scale
    assert np.abs(Nf[:, 1:-1]).max() < 1e-10 * scale


def _solid_body(s, Omega):
    """U = Omega e_z x r: toroidal e = Omega r^2 cos th = (Omega r^2/sqrt3) Y_1^0."""
    x = np.zeros((3, s.P, s.Nr), dtype=complex)
    A = basis.cheb_matrix(s.xc, s.Nr, 0, s.r_in, s.r_out)
    x[0, s.pair_index(1, 0)] = np.linalg.solve(A, Omega * s.rc ** 2 / np.sqrt(3.0))
    return x


def test_temperature_advection_by_solid_body_rotation():
    """U.grad T = Omega d_phi T for U = Omega e_z x r, so N_T = -i m Omega T (Eq. temp)."""
    s = Shell(10, 2, 24, 1e-2, 0.0)
    Om = 0.7
    x = _solid_body(s, Om)
    x[2] = _low_degree_state(s, np.random.default_rng(6), kmax=8, bc=False, fields=(2,))[2]
    NT = s.explicit_terms(x)[2]
    ref = -1j * s.pair_m[:, None] * Om * (x[2] @ s.E[0].T)
    assert np.abs(NT - ref).max() < 1e-11 * np.abs(ref).max()


def test_momentum_advection_linearised_about_solid_body_rotation():
    """For U = Omega e_z x r: (U.grad)u + (u.grad)U = Omega [d_phi u]_sph + 2 Omega e_z x u.

    So the linearised explicit term is -Ek Omega times (i m e_r.curl u + Coriolis rows) for e
    and (i m e_r.curl curl u + Coriolis rows) for f, with e_r.curl u = l(l+1) e/r^2 and
    e_r.curl curl u = -l(l+1) L_l f / r^2 (Eq. Navier-Stokes, Eqs. impcor_e/f_final).
    """
    Ek, Om = 0.3, 0.9
    s = Shell(8, 1, 40, Ek, 0.0)
    U = _solid_body(s, Om)
    u = _low_degree_state(s, np.random.default_rng(7), kmax=8, bc=False, fields=(0, 1))
    N = s.explicit_terms_linear(U, u)
    r = s.rc[:, None]
    worst = 0.0
    for p in range(s.P):
        l, m = int(s.pair_l[p]), int(s.pair_m[p])
        if l == 0:
            continue
        lam = l * (l + 1.0)
        for fi, fl in enumerate(("e", "f")):
            other = 1 - fi
            cor = s.coriolis_diag_rows(fl, l, m, s.E, r) @ u[fi, p]
            if l - 1 >= m:
                cor = cor + s.coupling_rows(l, m, -1, s.E, r) @ u[other, p - 1]
            if l + 1 <= s.L:
                cor = cor + s.coupling_rows(l, m, +1, s.E, r) @ u[other, p + 1]
            if fl == "e":
                curl = lam / r[:, 0] ** 2 * (s.E[0] @ u[0, p])
            else:
                curl = -lam / r[:, 0] ** 2 * ((s.E[2] - lam / r ** 2 * s.E[0]) @ u[1, p])
            ref = -Ek * Om * (1j * m * curl + cor)
            rows = _interior(fl, s.Nr)
            err = np.abs(N[fi, p][rows] - ref[rows]).max() / max(1.0, np.abs(ref[rows]).max())
            worst = max(worst, err)
    assert worst < 1e-9


def _cc_integral(s, vals_on_nd):
    """Integral over r of the Chebyshev interpolant of values on the N_d radii."""
    Td = basis.cheb_matrix(s.xd, s.Nd, 0, s.r_in, s.r_out)
    coef = np.linalg.solve(Td, vals_on_nd)
    xq, wq = np.polynomial.legendre.leggauss(2 * s.Nd)
    v = basis.cheb_matrix(xq, s.Nd, 0, s.r_in, s.r_out) @ coef
    return 0.5 * (s.r_out - s.r_in) * (wq * v).sum()


def test_advection_conserves_heat():
    """int U.grad T dV = 0 for no-slip U (div U = 0): the l = 0 projection integrates to zero."""
    s = Shell(12, 2, 20, 1.0, 0.0)
    x = _low_degree_state(s, np.random.default_rng(8), kmax=7)
    g = s.grid_fields(x)
    _, _, _, NT = s.analyse(*s.products(g))
    val = _cc_integral(s, s.rd ** 2 * NT[s.pair_index(0, 0)].real)
    scale = _cc_integral(s, s.rd ** 2 * np.abs(NT).sum(axis=0))
    assert abs(val) < 1e-12 * scale


def test_advection_does_no_work():
    """int U.(U x omega) dV = 0, through the curl projections (integration by parts as above)."""
    s = Shell(10, 2, 20, 1.0, 0.0)
    x = _low_degree_state(s, np.random.default_rng(9), kmax=7)
    g = s.grid_fields(x)
    Q, S, T, _ = s.analyse(*s.products(g))
    Td = basis.cheb_matrix(s.xd, s.Nd, 0, s.r_in, s.r_out)
    D1 = basis.cheb_matrix(s.xd, s.Nd, 1, s.r_in, s.r_out) @ np.linalg.inv(Td)
    rd = s.rd
    total, scale = 0.0, 0.0
    for p in range(s.P):
        l, m = int(s.pair_l[p]), int(s.pair_m[p])
        if l == 0:
            continue
        lam = l * (l + 1.0)
        w = 4 * np.pi if m == 0 else 16 * np.pi
        ev = s.Ed[0] @ x[0, p]
        fv = s.Ed[0] @ x[1, p]
        ce = lam * T[p] / rd
        cf = lam / rd ** 2 * (Q[p] - D1 @ (rd * S[p]))
        for a, b in ((ev, ce), (fv, cf)):
            term = w * _cc_integral(s, rd ** 2 * np.real(a * np.conj(b)))
            total += term
            scale += w * _cc_integral(s, rd ** 2 * np.abs(a * b))
    assert abs(total) < 1e-10 * scale


def _rotate(s, vec, phi0):
    x = s.to_complex(vec)
    return s.to_real(x * np.exp(-1j * s.pair_m * phi0)[None, :, None])


def test_step_commutes_with_rotation():
    c = si.config("C1")
    s = Shell(15, 4, 16, c["Ek"], c["Ra"])
    x = s.conductive_state() + si.perturbation(15, 4, 16, 11, amp=1e-2)
    a = s.step(_rotate(s, x, 0.37), 1.3, 1e-3)
    b = _rotate(s, s.step(x, 1.3, 1e-3), 0.37)
    # exact in exact arithmetic; the bound is the measured round-off spread of the
    # e/f chain solve (about 1e-10 relative for this truncation)
    assert np.abs(a - b).max() < 1e-10 * np.abs(b).max()


def test_jacobian_action_matches_finite_differences():
    c = si.config("C1")
    s = Shell(15, 4, 16, c["Ek"], c["Ra"])
    U = s.conductive_state() + si.perturbation(15, 4, 16, 12, amp=3e-2)
    u = si.random_vector(15, 4, 16, 13)
    C, dt, eps = 0.8, 1e-2, 1e-5
    fd = (s.step(U + eps * u, C, dt) - s.step(U - eps * u, C, dt)) / (2 * eps) - u
    got = s.jvp(U, C, None, u, dt)
    assert np.linalg.norm(got - fd) < 1e-7 * np.linalg.norm(fd)
    # with the drift unknown c stored in slot J (Sec. 3.4)
    J = s.real_index("T", 4, 4, 2, 1)
    cval = 0.37
    u2 = u.copy()
    u2[J] = cval
    uz = u.copy()
    uz[J] = 0.0
    fd2 = ((s.step(U + eps * uz, C + eps * cval, dt) - s.step(U - eps * uz, C - eps * cval, dt))
           / (2 * eps) - uz)
    got2 = s.jvp(U, C, J, u2, dt)
    assert np.linalg.norm(got2 - fd2) < 1e-7 * np.linalg.norm(fd2)


def test_linearised_step_spectrum_at_rest():
    """Dense B_U from Jacobian actions at U = 0, Ra = 0 on a tiny truncation.

    Its eigenvalues are 1/(1 - dt sigma) with sigma the generalised eigenvalues of
    -K v = sigma M v (Eq. discrete); the l = 0 temperature modes have
    sigma = -(n pi)^2 / Pr (Eq. temp)."""
    s = Shell(7, 4, 16, 1e-2, 0.0)
    dt = 2e-3
    U = np.zeros(s.n)
    n = s.n
    B = np.empty((n, n))
    for j in range(n):
        ej = np.zeros(n)
        ej[j] = 1.0
        B[:, j] = s.jvp(U, 0.0, None, ej, dt) + ej
    mu = np.linalg.eigvals(B)
    # l = 0 temperature decay rates
    for k in (1, 2, 3):
        target = 1.0 / (1.0 + dt * (k * np.pi) ** 2 / s.Pr)
        assert np.min(np.abs(mu - target)) < 1e-7
    # Coriolis-coupled spectrum of one m = 4 chain against the generalised problem
    sig = []
    r = s.rc[:, None]
    for cls in (0, 1):
        flds = s.chain_fields(4, cls)
        nb = len(flds)
        K = np.zeros((nb * s.Nr, nb * s.Nr), dtype=complex)
        M = np.zeros_like(K)
        for i, fl in enumerate(flds):
            l = 4 + i
            rows = _interior(fl, s.Nr)
            blk = slice(i * s.Nr, (i + 1) * s.Nr)
            Kd = s.diffusion_rows(fl, l, s.E, r) + s.coriolis_diag_rows(fl, l, 4, s.E, r)
            Md = s.mass_rows(fl, l, s.E, r)
            s._bc_rows(Kd, fl)
            Md[~rows] = 0.0
            K[blk, blk] = Kd
            M[blk, blk] = Md
            for side in (-1, 1):
                if 0 <= i + side < nb:
                    Cp = np.array(s.coupling_rows(l, 4, side, s.E, r), dtype=complex)
                    Cp[~rows] = 0.0
                    K[blk, slice((i + side) * s.Nr, (i + side + 1) * s.Nr)] = Cp
        import scipy.linalg as sla
        w = sla.eigvals(-K, M)
        sig.extend(w[np.isfinite(w)])
    for sg in sig:
        target = 1.0 / (1.0 - dt * sg)
        assert np.min(np.abs(mu - target)) < 1e-6 * max(1.0, abs(target))
