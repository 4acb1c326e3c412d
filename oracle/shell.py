"""The discretised rotating-shell Boussinesq model, written out plainly (FP64).

Unknowns (Sec. 3.1): toroidal potential e, poloidal potential f and total
temperature T, with U = curl(e r_hat) + curl curl(f r_hat), each expanded as
sum_k sum_lm c_klm T_k(x) Y_l^m.  The state is the real vector of Chebyshev
coefficients in the canonical order [field e,f,T][pair (m, l)][k][re, im],
pairs ordered by m = 0, Ms, 2Ms, ... <= L and, inside each m, by l = m..L.

Time step (Sec. 3.3, Eq. discrete, with the drift of Sec. 3.4):
    (M/dt + K) x^{n+1} = (1/dt + i C m) M x^n + N(x^n)
where, collocated at the N_r Gauss-Lobatto radii r_j,
    M_e = l(l+1) Ek / r^2                      (Eq. impcor_e_final)
    M_f = -l(l+1) Ek / r^2 L_l,  L_l = d_r^2 - l(l+1)/r^2   (Eq. impcor_f_final)
    M_T = 1                                    (Eq. temp)
K holds diffusion and the Coriolis terms of Eqs. impcor_e_final /
impcor_f_final (diagonal -2im/r^2 and the l +- 1 couplings of e with f), and
N holds the curl / double-curl projections of
    F = Ek U x omega + Ra T r / r_out
(the gradient part of the advection drops out under the curl; the sign of
the advective term follows Eq. Navier-Stokes) and -U.grad T for T.
Boundary conditions replace rows (Sec. 3.1): e, T at r_j = r_out, r_in;
f and df/dr at the two end points and their neighbours.

Readings of the paper taken here (where it is silent or ambiguous):
  * collocation at Gauss-Lobatto radii, BC rows replacing the rows at the
    walls (and, for f, their neighbours);
  * radial de-aliasing: products on N_d = ceil(3 N_r/2) Gauss-Lobatto radii,
    projected to N_r Chebyshev coefficients by exact interpolation and
    truncation, then evaluated at the collocation radii;
  * d_r(r S_F) is the derivative of the truncated interpolant of r S_F;
  * rows of e_00, f_00 (l = 0) are identity rows with zero right-hand side;
    imaginary parts of m = 0 coefficients are set to zero;
  * in the Jacobian action c = u_J is read, u_J zeroed, and c i m M U added
    to the explicit part (Sec. 3.4).

Pins: tests/test_oracle_shell.py (conductive state, Ra = 0 decay of the
l = 0 temperature mode, Coriolis zero power, grid-space Coriolis against the
spectral l +- 1 formula, curl of a gradient, advection by solid-body
rotation, heat-flux identity, finite-difference Jacobian, eigenvalues of the
linearised step against those of the continuous operator).
"""
import math

import numpy as np
import scipy.linalg as sla
from scipy.linalg import lapack

from . import basis, sht

FIELDS = ("e", "f", "T")
BC_ROWS = {"e": (0, -1), "T": (0, -1), "f": (0, 1, -2, -1)}


def ylm_log_n(l, m):
    """log N_l^m of Eq. Ylm_norm: N = sqrt((2 - delta_m0)(2l+1)(l-m)!/(l+m)!) (log avoids underflow)."""
    return 0.5 * (math.log(2.0 - (m == 0)) + math.log(2 * l + 1)
                  + math.lgamma(l - m + 1) - math.lgamma(l + m + 1))


def coriolis_coefficients(l, m):
    """(alpha_l, beta_l) of Eq. impcor_e_final / impcor_f_final.

    alpha multiplies (2/r^2)[l/r - d_r] acting on the other potential at l-1,
    beta multiplies (2/r^2)[-(l+1)/r - d_r] acting on it at l+1.
    """
    alpha = 0.0
    if l - 1 >= m and l >= 1:
        alpha = ((l - 1) * (l + 1) * (l - m) / (2 * l - 1)
                 * math.exp(ylm_log_n(l - 1, m) - ylm_log_n(l, m)))
    beta = (l * (l + 2) * (l + 1 + m) / (2 * l + 3)
            * math.exp(ylm_log_n(l + 1, m) - ylm_log_n(l, m)))
    return alpha, beta


class Shell:
    """One rotating-shell problem at fixed truncation and parameters."""

    def __init__(self, L, Ms, Nr, Ek, Ra, Pr=1.0, eta=0.35, coriolis="implicit"):
        """coriolis = "implicit" (Sec. 3.2, the method) or "explicit" (Eqs. expcor_e/f:
        Coriolis in F, block-diagonal implicit operator), the comparison of Sec. 5."""
        if coriolis not in ("implicit", "explicit"):
            raise ValueError(coriolis)
        self.coriolis = coriolis
        self.L, self.Ms, self.Nr = int(L), int(Ms), int(Nr)
        self.Ek, self.Ra, self.Pr, self.eta = float(Ek), float(Ra), float(Pr), float(eta)
        self.r_in, self.r_out = basis.shell_radii(eta)
        self.sph = sht.SphereGrid(self.L, self.Ms)
        self.ms = self.sph.ms
        pl, pm, starts = [], [], []
        for m in self.ms:
            starts.append(len(pl))
            for l in range(m, self.L + 1):
                pl.append(l)
                pm.append(m)
        starts.append(len(pl))
        self.pair_l = np.array(pl)
        self.pair_m = np.array(pm)
        self.starts = starts
        self.P = len(pl)
        self.lam = self.pair_l * (self.pair_l + 1.0)
        self.n = 3 * self.P * self.Nr * 2
        # Radial tables.
        self.Nd = basis.dealias_nr(self.Nr)
        self.xc = basis.lobatto_x(self.Nr)
        self.rc = basis.x_to_r(self.xc, self.r_in, self.r_out)
        self.xd = basis.lobatto_x(self.Nd)
        self.rd = basis.x_to_r(self.xd, self.r_in, self.r_out)
        self.E = [basis.cheb_matrix(self.xc, self.Nr, o, self.r_in, self.r_out) for o in range(5)]
        self.Ed = [basis.cheb_matrix(self.xd, self.Nr, o, self.r_in, self.r_out) for o in range(3)]
        Td = basis.cheb_matrix(self.xd, self.Nd, 0, self.r_in, self.r_out)
        fine_to_coef = np.linalg.solve(Td, np.eye(self.Nd))[: self.Nr]
        self.R0 = self.E[0] @ fine_to_coef   # values on N_d radii -> values at r_j
        self.R1 = self.E[1] @ fine_to_coef   # values on N_d radii -> d_r at r_j
        self._fact = {}

    # ---- layout helpers --------------------------------------------------
    def to_complex(self, v):
        v = np.asarray(v, dtype=np.float64).reshape(3, self.P, self.Nr, 2)
        return v[..., 0] + 1j * v[..., 1]

    def to_real(self, x):
        out = np.empty((3, self.P, self.Nr, 2))
        out[..., 0] = x.real
        out[..., 1] = x.imag
        return out.reshape(-1)

    def split_m(self, a):
        return [a[self.starts[i]:self.starts[i + 1]] for i in range(len(self.ms))]

    def pair_index(self, l, m):
        i = self.ms.index(m)
        return self.starts[i] + (l - m)

    def real_index(self, field, l, m, k, part):
        """Index into the canonical real vector (part 0 = Re, 1 = Im)."""
        return (((FIELDS.index(field) * self.P + self.pair_index(l, m)) * self.Nr + k) * 2
                + part)

    # ---- a1-a3: radial evaluation, Legendre synthesis, inverse DFT ---------
    def radial_fields(self, x):
        """Spectral quantities on the de-aliased radii [P, N_d] (Sec. 3.1)."""
        e, f, T = x[0], x[1], x[2]
        E0, E1, E2 = self.Ed
        rd = self.rd[None, :]
        lam = self.lam[:, None]
        fv, f1, f2 = f @ E0.T, f @ E1.T, f @ E2.T
        ev, e1 = e @ E0.T, e @ E1.T
        Tv, T1 = T @ E0.T, T @ E1.T
        return {
            "ur": lam * fv / rd ** 2,          # u_r = l(l+1) f / r^2
            "Su": f1 / rd,                     # spheroidal potential of u_H: d_r f / r
            "Tu": ev / rd,                     # toroidal potential of u_H: e / r
            "wr": lam * ev / rd ** 2,          # omega_r = l(l+1) e / r^2
            "Sw": e1 / rd,                     # omega = curl U has poloidal potential e
            "Tw": -(f2 - lam * fv / rd ** 2) / rd,   # and toroidal potential -L_l f
            "dT": T1,                          # d_r T
            "ST": Tv / rd,                     # grad_H T / r
        }

    def grid_fields(self, x):
        """The nine grid fields U, omega, grad T on [nphi, nlat, N_d]."""
        q = {k: self.split_m(v) for k, v in self.radial_fields(x).items()}
        s = self.sph
        zero = [np.zeros_like(a) for a in q["ST"]]
        ut, up = s.synth_vector(q["Su"], q["Tu"])
        wt, wp = s.synth_vector(q["Sw"], q["Tw"])
        tt, tp = s.synth_vector(q["ST"], zero)
        G = {
            "ur": s.synth_scalar(q["ur"]), "ut": ut, "up": up,
            "wr": s.synth_scalar(q["wr"]), "wt": wt, "wp": wp,
            "Tr": s.synth_scalar(q["dT"]), "Tt": tt, "Tp": tp,
        }
        return {k: s.fourier_to_grid(v) for k, v in G.items()}

    # ---- a4: products on the grid ------------------------------------------
    def products(self, g):
        """F = Ek U x omega and U.grad T on the grid."""
        Ek = self.Ek
        Fr = Ek * (g["ut"] * g["wp"] - g["up"] * g["wt"])
        Ft = Ek * (g["up"] * g["wr"] - g["ur"] * g["wp"])
        Fp = Ek * (g["ur"] * g["wt"] - g["ut"] * g["wr"])
        NT = g["ur"] * g["Tr"] + g["ut"] * g["Tt"] + g["up"] * g["Tp"]
        return Fr, Ft, Fp, NT

    def products_linear(self, gU, gu):
        """Linearised products (Sec. 3.3): U x omega_u + u x omega_U and U.grad tau + u.grad T."""
        Ek = self.Ek

        def cross(a, b):
            return (a["ut"] * b["wp"] - a["up"] * b["wt"],
                    a["up"] * b["wr"] - a["ur"] * b["wp"],
                    a["ur"] * b["wt"] - a["ut"] * b["wr"])

        c1 = cross(gU, gu)
        c2 = cross(gu, gU)
        Fr, Ft, Fp = (Ek * (c1[i] + c2[i]) for i in range(3))
        NT = (gU["ur"] * gu["Tr"] + gU["ut"] * gu["Tt"] + gU["up"] * gu["Tp"]
              + gu["ur"] * gU["Tr"] + gu["ut"] * gU["Tt"] + gu["up"] * gU["Tp"])
        return Fr, Ft, Fp, NT

    # ---- a5-a6: forward DFT and Legendre analysis ----------------------------
    def analyse(self, Fr, Ft, Fp, NT):
        """Grid products -> (Q_F, S_F, T_F, (U.grad T)_lm) on the de-aliased radii [P, N_d]."""
        s = self.sph
        GFr, GFt, GFp, GNT = (s.grid_to_fourier(a) for a in (Fr, Ft, Fp, NT))
        Q = np.concatenate(s.analyse_scalar(GFr))
        S, T = s.analyse_vector(GFt, GFp)
        N = np.concatenate(s.analyse_scalar(GNT))
        return Q, np.concatenate(S), np.concatenate(T), N

    # ---- a7: curl projections at the collocation radii ------------------------
    def curl_terms(self, Q, S, T, NT):
        """e_r.curl F = l(l+1) T_F / r; e_r.curl curl F = l(l+1)/r^2 [Q_F - d_r(r S_F)]."""
        lam = self.lam[:, None]
        rc = self.rc[None, :]
        Tc = T @ self.R0.T
        Qc = Q @ self.R0.T
        dS = (S * self.rd[None, :]) @ self.R1.T
        Nc = NT @ self.R0.T
        return lam * Tc / rc, lam / rc ** 2 * (Qc - dS), -Nc

    def buoyancy(self, T):
        """e_r.curl curl of Ra T r / r_out: l(l+1) Ra T / (r r_out) at the collocation radii."""
        lam = self.lam[:, None]
        rc = self.rc[None, :]
        return lam * self.Ra * (T @ self.E[0].T) / (rc * self.r_out)

    def explicit_terms(self, x):
        """N(x) at the collocation radii: (N_e, N_f, N_T), each [P, N_r] complex."""
        g = self.grid_fields(x)
        Ne, Nf, NT = self.curl_terms(*self.analyse(*self.products(g)))
        return np.stack([Ne, Nf + self.buoyancy(x[2]), NT])

    def explicit_terms_linear(self, X, x, gX=None):
        """N_X x: the linearisation of N about X applied to x."""
        if gX is None:
            gX = self.grid_fields(X)
        g = self.grid_fields(x)
        Ne, Nf, NT = self.curl_terms(*self.analyse(*self.products_linear(gX, g)))
        return np.stack([Ne, Nf + self.buoyancy(x[2]), NT])

    def mass(self, x):
        """M x at the collocation radii (the operators under d/dt), [3, P, N_r]."""
        out = np.zeros_like(x)
        r = self._rows()
        for p in range(self.P):
            l = int(self.pair_l[p])
            for fi, fl in enumerate(FIELDS):
                out[fi, p] = self.mass_rows(fl, l, self.E, r) @ x[fi, p]
        return out

    # ---- implicit operator (Sec. 3.2) -------------------------------------------
    # The *_rows functions evaluate the operators at any radii r (column vector)
    # given the Chebyshev tables E[o][j, k] = d^o T_k / dr^o at those radii.
    def mass_rows(self, field, l, E, r):
        """Rows of M for one (l, field): the operator under d/dt."""
        lam = l * (l + 1.0)
        if field == "e":
            return (lam * self.Ek / r ** 2) * E[0]
        if field == "f":
            return -(lam * self.Ek / r ** 2) * (E[2] - lam / r ** 2 * E[0])
        return E[0]

    def diffusion_rows(self, field, l, E, r):
        """Rows of the diffusive part of K (Eqs. impcor_e_final, impcor_f_final, temp)."""
        lam = l * (l + 1.0)
        if field == "e":
            return -(lam * self.Ek / r ** 2) * (E[2] - lam / r ** 2 * E[0])
        if field == "f":
            L2 = (E[4] - 2.0 * lam / r ** 2 * E[2] + 4.0 * lam / r ** 3 * E[1]
                  + (lam * lam - 6.0 * lam) / r ** 4 * E[0])   # L_l L_l
            return (lam * self.Ek / r ** 2) * L2
        return -(1.0 / self.Pr) * (E[2] + (2.0 / r) * E[1] - lam / r ** 2 * E[0])

    def coriolis_diag_rows(self, field, l, m, E, r):
        """-2im/r^2 e (e equation) and +2im/r^2 L_l f (f equation)."""
        lam = l * (l + 1.0)
        if field == "e":
            return -(2j * m / r ** 2) * E[0]
        return (2j * m / r ** 2) * (E[2] - lam / r ** 2 * E[0])

    def coupling_rows(self, l, m, side, E, r):
        """Coriolis coupling of the equation at l to the other potential at l + side."""
        alpha, beta = coriolis_coefficients(l, m)
        if l == 0:
            return np.zeros((r.shape[0], E[0].shape[1]))
        if side < 0:
            return (2.0 / r ** 2) * alpha * ((l / r) * E[0] - E[1])
        return (2.0 / r ** 2) * beta * (-((l + 1.0) / r) * E[0] - E[1])

    def _rows(self):
        return self.rc[:, None]

    def diag_block(self, field, l, m, dt):
        """Diagonal block M/dt + K at the collocation radii with BC rows replaced."""
        r = self._rows()
        if field != "T" and l == 0:
            return np.eye(self.Nr, dtype=np.complex128)
        D = ((1.0 / dt) * self.mass_rows(field, l, self.E, r)
             + self.diffusion_rows(field, l, self.E, r)).astype(np.complex128)
        if field != "T" and self.coriolis == "implicit":
            D = D + self.coriolis_diag_rows(field, l, m, self.E, r)
        self._bc_rows(D, field)
        return D

    def _bc_rows(self, D, field):
        E0, E1 = self.E[0], self.E[1]
        if field in ("e", "T"):
            D[0], D[-1] = E0[0], E0[-1]
        else:
            D[0], D[1], D[-2], D[-1] = E0[0], E1[0], E1[-1], E0[-1]

    def coupling_block(self, field, l, m, side):
        """Off-diagonal block of the `field` equation at l (BC rows zero; zero when explicit)."""
        if self.coriolis == "explicit":
            return np.zeros((self.Nr, self.Nr), dtype=np.complex128)
        B = np.array(self.coupling_rows(l, m, side, self.E, self._rows()), dtype=np.complex128)
        for j in BC_ROWS[field]:
            B[j] = 0.0
        return B

    def chain_fields(self, m, cls):
        """Fields of the blocks of chain `cls` for this m, l = m..L (Sec. 3.2 parity classes)."""
        return ["e" if (i + cls) % 2 == 0 else "f" for i in range(self.L - m + 1)]

    # ---- a8: factorisation and solve -------------------------------------------
    def factor(self, dt):
        """Whole-chain banded LU with partial pivoting (LAPACK gbtrf) per (m, class); real LU per l for T.

        Every row of a chain is first divided by its largest entry (row
        equilibration; the solution is unchanged in exact arithmetic).  The
        rows of one chain span thirteen orders of magnitude (boundary rows of
        Chebyshev values ~1 next to fourth-order rows ~1e13 at N_r = 64), and
        without the scaling, pivoting on the large rows costs the boundary rows
        up to 1e-8 of their accuracy.
        """
        key = float(dt)
        if key in self._fact:
            return self._fact[key]
        Nr = self.Nr
        kl = ku = 2 * Nr - 1
        chains = {}
        for a, m in enumerate(self.ms):
            for cls in (0, 1):
                flds = self.chain_fields(m, cls)
                nb = len(flds)
                N = nb * Nr
                ab = np.zeros((2 * kl + ku + 1, N), dtype=np.complex128)
                scale = np.empty(N)

                def put(B, bi, bj):
                    rows = np.arange(Nr)[:, None] + bi * Nr
                    cols = np.arange(Nr)[None, :] + bj * Nr
                    ab[kl + ku + rows - cols, np.broadcast_to(cols, B.shape)] = B

                for i, fld in enumerate(flds):
                    l = m + i
                    blocks = [(self.diag_block(fld, l, m, dt), i)]
                    if i > 0:
                        blocks.append((self.coupling_block(fld, l, m, -1), i - 1))
                    if i < nb - 1:
                        blocks.append((self.coupling_block(fld, l, m, +1), i + 1))
                    rmax = np.max([np.abs(B).max(axis=1) for B, _ in blocks], axis=0)
                    sc = 1.0 / rmax
                    scale[i * Nr:(i + 1) * Nr] = sc
                    for B, j in blocks:
                        put(sc[:, None] * B, i, j)
                lu, piv, info = lapack.zgbtrf(ab, kl, ku)
                if info != 0:
                    raise np.linalg.LinAlgError(f"singular chain m={m} class={cls}")
                chains[(a, cls)] = (lu, piv, flds, scale)
        temp = {}
        for l in range(self.L + 1):
            D = self.diag_block("T", l, 0, dt).real
            sc = 1.0 / np.abs(D).max(axis=1)
            temp[l] = (sla.lu_factor(sc[:, None] * D), sc)
        self._fact[key] = (chains, temp)
        return self._fact[key]

    def solve(self, rhs, dt):
        """Solve (M/dt + K) y = rhs, rhs [3, P, N_r] complex with BC rows set."""
        chains, temp = self.factor(dt)
        Nr = self.Nr
        kl = ku = 2 * Nr - 1
        y = np.zeros_like(rhs)
        for a, m in enumerate(self.ms):
            p0 = self.starts[a]
            for cls in (0, 1):
                lu, piv, flds, scale = chains[(a, cls)]
                b = np.concatenate([rhs[FIELDS.index(fl), p0 + i] for i, fl in enumerate(flds)])
                xs, info = lapack.zgbtrs(lu, kl, ku, scale * b, piv)
                for i, fl in enumerate(flds):
                    y[FIELDS.index(fl), p0 + i] = xs[i * Nr:(i + 1) * Nr]
        for p in range(self.P):
            lu, sc = temp[int(self.pair_l[p])]
            y[2, p] = (sla.lu_solve(lu, sc * rhs[2, p].real)
                       + 1j * sla.lu_solve(lu, sc * rhs[2, p].imag))
        return y

    def chain_system(self, m, cls, dt):
        """The blocks of chain (m, cls) of M/dt + K, unscaled, as (fields, D, A, C): D[i] the
        diagonal block of block row i, A[i] its coupling to block i-1 (None for i = 0), C[i]
        to block i+1 (None for the last).  For residual checks of a solve."""
        flds = self.chain_fields(m, cls)
        D, A, C = [], [], []
        for i, fld in enumerate(flds):
            l = m + i
            D.append(self.diag_block(fld, l, m, dt))
            A.append(self.coupling_block(fld, l, m, -1) if i > 0 else None)
            C.append(self.coupling_block(fld, l, m, +1) if i < len(flds) - 1 else None)
        return flds, D, A, C

    def step_rhs(self, vec, C=0.0, dt=1e-4):
        """The right-hand side of one IMEX Euler step from vec, [3, P, N_r] complex, with the
        boundary rows set (the system that step() solves is (M/dt + K) x = step_rhs)."""
        x = self.to_complex(vec)
        rhs = (1.0 / dt + self.drift(C)) * self.mass(x) + self.explicit_terms(x)
        if self.coriolis == "explicit":
            rhs = rhs - self.coriolis_terms(x)
        return self.apply_rows(rhs, homogeneous=False)

    def jvp_rhs(self, Uvec, C, J, uvec, dt, gU=None):
        """The right-hand side of the solve inside jvp(), [3, P, N_r] complex (gU: the
        grid fields of U, if already computed)."""
        u = np.array(uvec, dtype=np.float64, copy=True)
        c = 0.0
        if J is not None:
            c = u[J]
            u[J] = 0.0
        U = self.to_complex(Uvec)
        x = self.to_complex(u)
        rhs = ((1.0 / dt + self.drift(C)) * self.mass(x)
               + self.explicit_terms_linear(U, x, gU)
               + c * (1j * self.pair_m)[None, :, None] * self.mass(U))
        if self.coriolis == "explicit":
            rhs = rhs - self.coriolis_terms(x)
        return self.apply_rows(rhs, homogeneous=True)

    def apply_rows(self, rhs, homogeneous):
        """Boundary rows, l = 0 identity rows and real m = 0 rows of the right-hand side."""
        for fi, fl in enumerate(FIELDS):
            for j in BC_ROWS[fl]:
                rhs[fi, :, j] = 0.0
        if not homogeneous:
            p00 = self.pair_index(0, 0)
            rhs[2, p00, 0] = 0.0     # T(r_out) = 0   (Eq. BCtemp; x = +1 is r_out)
            rhs[2, p00, -1] = 1.0    # T(r_in) = 1
        l0 = self.pair_l == 0
        rhs[0, l0] = 0.0
        rhs[1, l0] = 0.0
        m0 = self.pair_m == 0
        rhs[:, m0] = rhs[:, m0].real
        return rhs

    def drift(self, C):
        return (1j * C * self.pair_m)[None, :, None]

    def coriolis_terms(self, x):
        """Coriolis rows of Eqs. impcor_e_final / impcor_f_final applied to x at the
        collocation radii: e_r.curl(2 e_z x U) and e_r.curl curl(2 e_z x U), [3, P, N_r]."""
        out = np.zeros_like(x)
        r = self._rows()
        for p in range(self.P):
            l, m = int(self.pair_l[p]), int(self.pair_m[p])
            if l == 0:
                continue
            for fi, fl in enumerate(("e", "f")):
                other = 1 - fi
                v = self.coriolis_diag_rows(fl, l, m, self.E, r) @ x[fi, p]
                if l - 1 >= m:
                    v = v + self.coupling_rows(l, m, -1, self.E, r) @ x[other, p - 1]
                if l + 1 <= self.L:
                    v = v + self.coupling_rows(l, m, +1, self.E, r) @ x[other, p + 1]
                out[fi, p] = v
        return out

    # ---- the step and the Jacobian action ---------------------------------------
    def step(self, vec, C=0.0, dt=1e-4, nsteps=1):
        """B(U): IMEX Euler steps with the drift C d_phi in the explicit part (Eq. discrete)."""
        x = np.asarray(vec, dtype=np.float64)
        for _ in range(nsteps):
            x = self.to_real(self.solve(self.step_rhs(x, C, dt), dt))
        return x

    def diffusion(self, x):
        """The diffusive part of K applied to x at the collocation radii, [3, P, N_r]."""
        out = np.zeros_like(x)
        r = self._rows()
        for p in range(self.P):
            l = int(self.pair_l[p])
            for fi, fl in enumerate(FIELDS):
                out[fi, p] = self.diffusion_rows(fl, l, self.E, r) @ x[fi, p]
        return out

    def step2(self, vec, dt=1e-4, nsteps=1):
        """Second-order time step in the laboratory frame (the scheme of the time-stepping
        runs of Sec. 5, which combines a Runge-Kutta predictor-corrector with the implicit
        treatment of the linear operator).  Reading: Crank-Nicolson for the implicit
        operator K (diffusion, plus Coriolis when implicit) and Heun's predictor-corrector
        for the explicit terms N (products, buoyancy, plus Coriolis when explicit):
            (M/dt + K/2) x*      = (M/dt - K/2) x^n + N(x^n)
            (M/dt + K/2) x^{n+1} = (M/dt - K/2) x^n + (N(x^n) + N(x*)) / 2
        with the boundary rows of Eq. BCs.  M/dt + K/2 = (M (2/dt) + K)/2 is solved with
        the factorisation at dt/2 and a doubled right-hand side."""
        x = self.to_complex(vec)

        def explicit(z):
            n = self.explicit_terms(z)
            if self.coriolis == "explicit":
                n = n - self.coriolis_terms(z)
            return n

        for _ in range(nsteps):
            Kx = self.diffusion(x)
            if self.coriolis == "implicit":
                Kx = Kx + self.coriolis_terms(x)
            base = self.mass(x) / dt - 0.5 * Kx
            Nx = explicit(x)
            xs = self.solve(self.apply_rows(2.0 * (base + Nx), homogeneous=False), 0.5 * dt)
            Ns = explicit(xs)
            x = self.solve(self.apply_rows(2.0 * (base + 0.5 * (Nx + Ns)), homogeneous=False),
                           0.5 * dt)
        return self.to_real(x)

    def jvp(self, Uvec, C, J, uvec, dt, gU=None):
        """(B_U - I) applied to (u, c) with c stored in slot J (Secs. 3.3-3.4).

        J = None gives the plain steady-state action without the drift unknown.
        """
        u = np.array(uvec, dtype=np.float64, copy=True)
        if J is not None:
            u[J] = 0.0
        y = self.solve(self.jvp_rhs(Uvec, C, J, uvec, dt, gU), dt)
        return self.to_real(y) - u

    def conductive_state(self):
        """Steady conductive solution of the discrete T_00 equation with U = 0 (Sec. 2.1)."""
        x = np.zeros((3, self.P, self.Nr), dtype=np.complex128)
        D = self.diag_block("T", 0, 0, np.inf).real
        b = np.zeros(self.Nr)
        b[-1] = 1.0
        x[2, self.pair_index(0, 0)] = np.linalg.solve(D, b)
        return self.to_real(x)

    # ---- physical diagnostics (the paper plots them without defining them) ------------
    def kinetic_energy(self, vec, nquad=None):
        """KE density (1/V) int |U|^2/2 dV (the kinetic energy of the bifurcation diagrams,
        Secs. 4-5; V = 4 pi (r_out^3 - r_in^3)/3).  The velocity of Sec. 2.1 is synthesised on
        the transform grid at nquad Gauss-Legendre radii (default 2 N_r + 16, exact for the
        polynomial part of r^2 |U|^2), summed with the latitude weights and over the sector,
        then integrated in r by the Gauss-Legendre rule."""
        x = self.to_complex(vec)
        nq = nquad or 2 * self.Nr + 16
        xq, wq = np.polynomial.legendre.leggauss(nq)
        rq = basis.x_to_r(xq, self.r_in, self.r_out)
        E0 = basis.cheb_matrix(xq, self.Nr, 0, self.r_in, self.r_out)
        E1 = basis.cheb_matrix(xq, self.Nr, 1, self.r_in, self.r_out)
        e, f = x[0], x[1]
        r = rq[None, :]
        lam = self.lam[:, None]
        ur = lam * (f @ E0.T) / r ** 2
        Su = (f @ E1.T) / r
        Tu = (e @ E0.T) / r
        s = self.sph
        g_ur = s.fourier_to_grid(s.synth_scalar(self.split_m(ur)))
        ut, up = s.synth_vector(self.split_m(Su), self.split_m(Tu))
        g_ut, g_up = s.fourier_to_grid(ut), s.fourier_to_grid(up)
        w = self.sph.w[None, :, None]
        dphi = 2.0 * np.pi / self.sph.nphi  # sector mean times 2 pi
        ang = ((g_ur ** 2 + g_ut ** 2 + g_up ** 2) * w).sum(axis=(0, 1)) * dphi  # [nq]
        integral = 0.5 * (self.r_out - self.r_in) * (wq * rq ** 2 * ang).sum()
        V = 4.0 * np.pi * (self.r_out ** 3 - self.r_in ** 3) / 3.0
        return 0.5 * integral / V

    def nusselt(self, vec):
        """(Nu_in, Nu_out): d_r of the mean temperature at each wall over the conductive value."""
        x = self.to_complex(vec)
        T00 = x[2, self.pair_index(0, 0)].real
        d_in = (self.E[1][-1] @ T00)
        d_out = (self.E[1][0] @ T00)
        g_in = -self.r_out * self.r_in / self.r_in ** 2
        g_out = -self.r_out * self.r_in / self.r_out ** 2
        return d_in / g_in, d_out / g_out
