"""Spherical-harmonic transforms of the oracle, by direct sums (Sec. 3.1).

Real fields on the sphere are represented by complex coefficients a_lm for
m >= 0 (Y_l^{-m} = conj(Y_l^m)):
    a(theta, phi) = sum_l a_l0 Y_l^0 + 2 Re sum_{m>0} sum_l a_lm Y_l^m.
Only m in Ms*Z are carried (azimuthal symmetry restriction, Sec. 3.1), and
the grid covers one sector 0 <= phi < 2 pi / Ms with nphi points.

Tangent vector fields use a spheroidal potential S and a toroidal potential T:
    v_theta = dS/dth + (1/sin th) dT/dphi,   v_phi = (1/sin th) dS/dphi - dT/dth.
The analysis of v into (S, T) follows from the orthogonality of grad_H Y and
r x grad_H Y, whose squared norms are l(l+1) times that of Y.

Pins (tests/test_oracle_sht.py): analysis(synthesis(a)) = a for band-limited
scalar and vector fields; synthesis of single harmonics against closed forms.
"""
import numpy as np

from . import basis


class SphereGrid:
    """Tables for the sector grid (nlat Gauss-Legendre latitudes x nphi longitudes)."""

    def __init__(self, L, Ms):
        self.L, self.Ms = L, Ms
        self.ms = [k * Ms for k in range(L // Ms + 1)]
        self.K = len(self.ms) - 1
        self.nlat = basis.nlat_for(L)
        self.nphi = basis.nphi_for(L, Ms)
        self.x, self.w = basis.gauss_legendre(self.nlat)
        self.sin = basis.gauss_legendre_sin(self.nlat)
        # Per m: P = N P_l^m, dP = d/dtheta of it, Ps = P / sin(theta); rows l = m..L.
        self.P, self.dP, self.Ps = [], [], []
        for m in self.ms:
            f = basis.ylm_norm_factor(m)
            p = f * basis.plm_bar(L, m, self.x, self.sin)
            self.P.append(p)
            self.dP.append(f * basis.dplm_bar_dtheta(L, m, self.x, self.sin))
            self.Ps.append(p / self.sin[None, :])
        # Azimuthal DFT matrices over the sector: phi_j = 2 pi j / (Ms nphi),
        # so m phi_j = 2 pi k j / nphi for m = k Ms.
        j = np.arange(self.nphi)
        k = np.arange(self.K + 1)
        ang = 2.0 * np.pi * np.outer(j, k) / self.nphi
        self.inv_dft = np.exp(1j * ang) * np.where(k == 0, 1.0, 2.0)[None, :]
        self.fwd_dft = np.exp(-1j * ang.T) / self.nphi
        self.phi = 2.0 * np.pi * j / (Ms * self.nphi)
        self.theta = np.arccos(self.x)

    # ---- Fourier <-> grid (Sec. 3.1: FFT in phi) -------------------------
    def fourier_to_grid(self, G):
        """G[k, ...] complex Fourier coefficients (k = m/Ms) -> real values [nphi, ...].

        The m = 0 coefficient contributes its real part only.
        """
        G = np.array(G, dtype=np.complex128, copy=True)
        G[0] = G[0].real
        out = np.tensordot(self.inv_dft, G, axes=(1, 0))
        return out.real

    def grid_to_fourier(self, g):
        """g[nphi, ...] real -> G[k, ...] = (1/nphi) sum_j g_j exp(-i m phi_j)."""
        return np.tensordot(self.fwd_dft, g, axes=(1, 0))

    # ---- Legendre sums ----------------------------------------------------
    def norm(self, m):
        """Integral of P_lm^2 over x in [-1, 1] with the paper's N_l^m: 2(2 - delta_m0)."""
        return 2.0 * (2.0 if m > 0 else 1.0)

    def synth_scalar(self, a):
        """a: list over m of [nl, ...] coefficients -> Fourier coeffs [K+1, nlat, ...]."""
        return np.stack([np.tensordot(self.P[i].T, a[i], axes=(1, 0))
                         for i in range(self.K + 1)])

    def synth_vector(self, S, T):
        """Spheroidal S, toroidal T (lists over m) -> Fourier coeffs of (v_theta, v_phi)."""
        vt, vp = [], []
        for i, m in enumerate(self.ms):
            dS = np.tensordot(self.dP[i].T, S[i], axes=(1, 0))
            dT = np.tensordot(self.dP[i].T, T[i], axes=(1, 0))
            sS = np.tensordot(self.Ps[i].T, S[i], axes=(1, 0))
            sT = np.tensordot(self.Ps[i].T, T[i], axes=(1, 0))
            vt.append(dS + 1j * m * sT)
            vp.append(1j * m * sS - dT)
        return np.stack(vt), np.stack(vp)

    def analyse_scalar(self, G):
        """Fourier coeffs [K+1, nlat, ...] -> list over m of [nl, ...] coefficients."""
        out = []
        for i, m in enumerate(self.ms):
            wp = self.P[i] * self.w[None, :] / self.norm(m)
            out.append(np.tensordot(wp, G[i], axes=(1, 0)))
        return out

    def analyse_vector(self, Gt, Gp):
        """Fourier coeffs of (v_theta, v_phi) -> lists over m of (S, T) coefficients."""
        S, T = [], []
        for i, m in enumerate(self.ms):
            ls = np.arange(m, self.L + 1)
            lam = ls * (ls + 1.0)
            inv = np.where(lam > 0, 1.0 / np.where(lam > 0, lam, 1.0), 0.0)
            wd = self.dP[i] * self.w[None, :] / self.norm(m)
            ws = self.Ps[i] * self.w[None, :] / self.norm(m)
            s = (np.tensordot(wd, Gt[i], axes=(1, 0))
                 - 1j * m * np.tensordot(ws, Gp[i], axes=(1, 0)))
            t = (-1j * m * np.tensordot(ws, Gt[i], axes=(1, 0))
                 - np.tensordot(wd, Gp[i], axes=(1, 0)))
            shape = (-1,) + (1,) * (s.ndim - 1)
            S.append(s * inv.reshape(shape))
            T.append(t * inv.reshape(shape))
        return S, T
