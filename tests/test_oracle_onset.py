"""Pins of the oracle's linear onset (oracle/onset.py).

* An independent plane-layer solver (Chebyshev collocation written here) gives the
  rigid-rigid Rayleigh-Benard onset, 1707.762 at wavenumber 3.117 (Chandrasekhar 1961,
  cited by the paper in Sec. 1); the oracle's non-rotating shell onset tends to it as
  r_in/r_out -> 1 (Richardson extrapolation over four radius ratios).  This pins the
  diffusion, mass and boundary rows, the buoyancy Ra T r / r_out and the advection of the
  conductive profile through the oracle's transforms.
* Without rotation the onset of degree l is the same for every m.
* At (Ra_c, C_c) the oracle's linearised step B_U (Secs. 3.3-3.4, columns from
  Shell.jvp) fixes the pencil's eigenvector and has the eigenvalue 1: the pencil and the
  time stepper are one discretisation.
* The Arnoldi eigenvalues near a shift equal the dense QZ ones; the columnar onset
  mode at Ek = 1e-3, m = 4 is equatorially symmetric (the antisymmetric class is stable).
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as sopt
from numpy.polynomial import chebyshev as C

from oracle import onset as on
from oracle.shell import Shell


def _plane_layer_ra(a, n=28):
    """Smallest positive Ra of (D^2 - a^2)^2 W = Ra a^2 Theta, (D^2 - a^2) Theta = -W on
    z in [-1/2, 1/2] with W = DW = Theta = 0 at both walls; unknowns are Chebyshev
    coefficients, equations collocated at Gauss-Lobatto points, walls replacing the end rows."""
    z = np.cos(np.pi * np.arange(n) / (n - 1))   # in [-1, 1], z_phys = z / 2
    V = [np.empty((n, n)) for _ in range(5)]
    for k in range(n):
        c = np.zeros(n)
        c[k] = 1.0
        for o in range(5):
            V[o][:, k] = C.chebval(z, C.chebder(c, o) if o else c) * 2.0 ** o
    I0, D2, D4 = V[0], V[2], V[4]
    L2 = D2 - a * a * I0
    L4 = D4 - 2 * a * a * D2 + a ** 4 * I0
    A = np.zeros((2 * n, 2 * n))
    B = np.zeros((2 * n, 2 * n))
    A[:n, :n] = L4
    B[:n, n:] = a * a * I0
    A[n:, n:] = L2
    A[n:, :n] = I0
    for row, blk in [(0, V[0][0]), (1, V[1][0]), (n - 2, V[1][-1]), (n - 1, V[0][-1])]:
        A[row] = 0.0
        B[row] = 0.0
        A[row, :n] = blk
    for row, blk in [(n, V[0][0]), (2 * n - 1, V[0][-1])]:
        A[row] = 0.0
        B[row] = 0.0
        A[row, n:] = blk
    w = sla.eigvals(A, B)
    w = w[np.isfinite(w)]
    w = w[(np.abs(w.imag) < 1e-6 * np.abs(w)) & (w.real > 0)]
    return float(np.min(w.real))


def _plane_layer_onset():
    r = sopt.minimize_scalar(_plane_layer_ra, bounds=(2.6, 3.6), method="bounded",
                             options={"xatol": 1e-7})
    return r.fun, r.x


def test_plane_layer_solver_reproduces_the_textbook_onset():
    Ra, a = _plane_layer_onset()
    assert abs(Ra - 1707.762) < 0.005
    assert abs(a - 3.117) < 0.002


def _thin_shell_onset(eta, Nr=20):
    """Continuous minimum over the degree of the non-rotating onset (m = 0, Ek = Pr = 1, so
    Ra is the thermal Rayleigh number): a parabola in a = sqrt(l(l+1))/r_mid through the
    three degrees around the discrete minimum."""
    r_in, r_out = eta / (1 - eta), 1 / (1 - eta)
    r_mid = 0.5 * (r_in + r_out)
    lc = int(round(3.117 * r_mid))
    sh = Shell(lc + 3, lc + 4, Nr, 1.0, 1.0, Pr=1.0, eta=eta)
    blocks = on.conductive_blocks(sh)
    pts = []
    for l in range(lc - 2, lc + 3):
        pen = on.Pencil(sh, 0, (l + 1) % 2, blocks, rotation=False, l_only=l)
        pts.append((np.sqrt(l * (l + 1.0)) / r_mid, on.critical_rayleigh(pen, (1000, 3000))["Ra"]))
    pts = np.array(pts)
    j = int(np.clip(np.argmin(pts[:, 1]), 1, len(pts) - 2))
    c = np.polyfit(pts[j - 1:j + 2, 0], pts[j - 1:j + 2, 1], 2)
    amin = -c[1] / (2 * c[0])
    return np.polyval(c, amin), amin


def test_non_rotating_thin_shell_onset_tends_to_the_plane_layer():
    Ra_plane, a_plane = _plane_layer_onset()
    eps, R, A = [], [], []
    for eta in (0.9, 0.95, 0.975, 0.9875):
        Ra, a = _thin_shell_onset(eta)
        eps.append(1 - eta)
        R.append(Ra)
        A.append(a)
    # curvature raises the onset by about 5 % at eta = 0.9 and the excess halves with 1 - eta
    assert 1.04 < R[0] / Ra_plane < 1.07
    assert 1.005 < R[-1] / Ra_plane < 1.008
    ext = np.polyfit(eps, R, 3)[-1]
    assert abs(ext - Ra_plane) < 0.02, (ext, Ra_plane)
    assert abs(A[-1] - a_plane) < 2e-3


def test_non_rotating_onset_does_not_depend_on_m():
    sh = Shell(12, 4, 14, 1.0, 1.0)
    blocks = on.conductive_blocks(sh)
    assert blocks[2] == 0.0   # no linear momentum advection at rest
    vals = []
    for m in (0, 4, 8):
        i = 8 - m
        pen = on.Pencil(sh, m, (i + 1) % 2, blocks, rotation=False, l_only=8)
        vals.append(on.critical_rayleigh(pen, (500, 20000))["Ra"])
    assert max(vals) - min(vals) < 1e-9 * vals[0], vals


@pytest.fixture(scope="module")
def tiny_onset():
    """m = 4, Ek = 1e-3 on L = 9, N_r = 10 (4-fold symmetry)."""
    sh = Shell(9, 4, 10, 1e-3, 1.0)
    pen = on.Pencil(sh, 4, 1)
    return on.critical_rayleigh(pen, (20.0, 200.0)), pen


def test_onset_mode_is_fixed_by_the_linearised_step(tiny_onset):
    res, pen = tiny_onset
    s = Shell(9, 4, 10, 1e-3, res["Ra"])
    U = s.conductive_state()
    u = res["state"]
    assert abs(res["sigma"].real) < 1e-8 * abs(res["sigma"])
    for dt in (1e-3, 200.0):
        r = s.jvp(U, res["C"], None, u, dt)
        assert np.linalg.norm(r) < 1e-9 * np.linalg.norm(u), dt
    # the rotated mode i v as well (the two real directions of the neutral pair)
    r = s.jvp(U, res["C"], None, pen.state(1j * res["v"]), 200.0)
    assert np.linalg.norm(r) < 1e-9 * np.linalg.norm(u)
    # brute force: the dense linearised step has the eigenvalue 1, and not without the drift
    n = s.n
    for C, near in ((res["C"], True), (0.0, False)):
        B = np.empty((n, n))
        for j in range(n):
            ej = np.zeros(n)
            ej[j] = 1.0
            B[:, j] = s.jvp(U, C, None, ej, 200.0) + ej
        d = np.min(np.abs(np.linalg.eigvals(B) - 1.0))
        assert (d < 1e-8) if near else (d > 1e-3), (C, d)


def test_onset_drift_sign_and_class(tiny_onset):
    """The mode drifts prograde at onset (C > 0; the paper's drift decreases with Ra from
    prograde to retrograde, Sec. 2.2) and equatorially symmetric columns go first."""
    sh = Shell(23, 4, 16, 1e-3, 1.0)
    blocks = on.conductive_blocks(sh)
    s1 = on.rightmost(on.Pencil(sh, 4, 1, blocks), 60.0)[0]
    s0 = on.rightmost(on.Pencil(sh, 4, 0, blocks), 60.0)[0]
    assert s1.real > 0 > s0.real
    assert -s1.imag / 4 > 0
    assert tiny_onset[0]["C"] > 0


def test_arnoldi_eigenvalues_match_qz():
    sh = Shell(15, 4, 12, 1e-3, 1.0)
    pen = on.Pencil(sh, 4, 1)
    w = on.eig_dense(pen, 70.0)[0]
    s = w[np.argmax(w.real)] + (0.3 + 0.2j)
    near = on.eig_near(pen, 70.0, s, k=6)[0]
    ref = w[np.argsort(np.abs(w - s))[:6]]
    for z in near:
        assert np.min(np.abs(ref - z)) < 1e-9 * max(1.0, abs(z))


def _golden():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "onset_workloads.txt")
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows[f[0]] = dict(Ek=float(f[1]), m=int(f[2]), L=int(f[3]), Nr=int(f[4]),
                              Ra=float(f[5]), omega=float(f[6]), C=float(f[7]))
    return rows


def test_stored_onset_of_the_first_workload_reproduces():
    """onset_workloads.txt (make_onset.py) against a fresh computation at L = 31, N_r = 24."""
    g = _golden()["C1"]
    pen = on.Pencil(Shell(g["L"], g["m"], g["Nr"], g["Ek"], 1.0), g["m"], 1)
    sig = on.eig_near(pen, g["Ra"], 1j * g["omega"], k=4)[0]
    j = np.argmin(np.abs(sig - 1j * g["omega"]))
    assert abs(sig[j].real) < 1e-8 * abs(sig[j])
    assert abs(sig[j].imag - g["omega"]) < 1e-8 * abs(g["omega"])


@pytest.mark.slow
def test_rotating_wave_branch_ends_at_the_linear_onset():
    """The oracle's nonlinear RW4 branch (Newton-GMRES, Secs. 3.3-3.4, pinned by Table 1 row
    1) followed down from Ra = 120 to 1.01 Ra_c: its kinetic energy vanishes linearly and its
    drift tends to the onset drift, at the pencil's Ra_c and C_c (linear extrapolation from
    1.01 and 1.02 Ra_c: within 5e-4 and 2e-4; about 45 s)."""
    from oracle import krylov
    L, Ms, Nr, Ek, M = 23, 4, 16, 1e-3, 4
    lin = on.critical_rayleigh(on.Pencil(Shell(L, M, Nr, Ek, 1.0), M, 1), (40.0, 80.0),
                               shift="auto")
    s = Shell(L, Ms, Nr, Ek, 120.0)
    x = s.to_complex(s.conductive_state())
    x[2, s.pair_index(M, M)] += np.linalg.solve(s.E[0], 1e-2 * np.sin(np.pi * (s.rc - s.r_in)))
    U = s.step(s.to_real(x), 0.0, 2e-3, nsteps=400)
    U1 = s.step(U, 0.0, 2e-3, nsteps=5)
    C = krylov.drift_estimate(s, U, U1, 1e-2, M)
    J = krylov.phase_index(s, U, M)
    U, C, _ = krylov.newton(s, U, C, J, dt=200.0, tol=1e-11, max_newton=14, kmax=150)
    Uc = s.conductive_state()
    Ra_prev, pts = 120.0, []
    for f in (1.6, 1.3, 1.15, 1.07, 1.04, 1.02, 1.01):
        Ra = f * lin["Ra"]
        U = Uc + (U - Uc) * np.sqrt((Ra - lin["Ra"]) / (Ra_prev - lin["Ra"]))
        s = Shell(L, Ms, Nr, Ek, Ra)
        U, C, hist = krylov.newton(s, U, C, J, dt=200.0, tol=1e-11, max_newton=20, kmax=200)
        assert hist[-1]["residual"] < 1e-11
        pts.append((Ra, s.kinetic_energy(U), C))
        Ra_prev = Ra
    (Ra2, k2, c2), (Ra1, k1, c1) = pts[-2], pts[-1]
    Ra_ext = Ra1 - k1 * (Ra2 - Ra1) / (k2 - k1)
    C_ext = c1 + (c2 - c1) * (Ra_ext - Ra1) / (Ra2 - Ra1)
    assert abs(Ra_ext - lin["Ra"]) < 5e-4 * lin["Ra"]
    assert abs(C_ext - lin["C"]) < 2e-4 * abs(lin["C"])


def test_workload_onset_table_matches_the_stored_values():
    """seeded_inputs.ONSET_RA (used to set the workloads' Ra) holds make_onset.py's values."""
    import seeded_inputs as si
    g = _golden()
    for name, ra in si.ONSET_RA.items():
        assert name in g and abs(g[name]["Ra"] - ra) <= 1e-9 * ra, name
