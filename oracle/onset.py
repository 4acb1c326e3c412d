"""Linear onset of convection about the conductive state (oracle, plain FP64).

TEST INFRASTRUCTURE: imported only by the tests, smoke() and the CPU legs of bench.py.

The paper's rotating waves RW_M bifurcate from the conductive state (Sec. 2.2), at a
Rayleigh number that grows like Ek^(-1/3) (Sec. 4.4); it prints no onset values.  This
module computes them for the discretisation of the time stepper.

About U_cond (U = 0, T = T_cond(r)) the linearised equations decouple in the azimuthal
wavenumber m and in the two equatorial symmetry classes of the chains of Sec. 3.2.  For
one (m, class) they are the pencil

    A(Ra) x = sigma M x,   A(Ra) = -K + N_cond(Ra),

with M and K the operators of the implicit step (Eq. discrete; M the operators under
d/dt, K diffusion plus the Coriolis terms of Eqs. impcor_e_final / impcor_f_final
including the l +- 1 couplings), boundary conditions as rows of A with zero rows of M,
and N_cond the linearisation of the explicit terms: the buoyancy Ra T r / r_out in the f
equation (linear in Ra) and the advection -u_r dT_cond/dr in the T equation.  Both are
taken from the oracle's own explicit terms (Shell.buoyancy, Shell.explicit_terms_linear)
by probing with unit Chebyshev coefficients: at the conductive state they are block
diagonal in the (l, m) pairs, so N_r probes give every block.

The rotating wave condition of Sec. 3.4 at the conductive state, (B_U - I) u = 0 with
the drift C in the explicit part, is (A + i C m M) u = 0 for every dt.  So the onset of
mode m is the smallest Ra at which the rightmost eigenvalue sigma of the pencil reaches
the imaginary axis, sigma = i omega, and the wave drifts there with
C = -omega / m (a mode e^{i m phi + sigma t} = e^{i m (phi - C t)}, the convention
U(phi - C t) of the Newton solver).

Eigenvalues: dense QZ (scipy.linalg.eig) on small pencils; on large ones the eigenvalues
nearest a shift s, from Arnoldi (ARPACK) on (A - s M)^{-1} M with a sparse LU (the
standard-form operator, since M is neither symmetric nor definite).  Ra_c is the root of
max Re sigma(Ra) by Brent's method.

Pins (tests/test_oracle_onset.py): without rotation and with eta -> 1 the onset tends to
the rigid-rigid Rayleigh-Benard value (1707.76, computed there by an independent
plane-layer solver); without rotation the onset of degree l does not depend on m; at
(Ra_c, C_c) the dense linearised step of the oracle (columns from Shell.jvp) has the
eigenvalue 1 with the pencil's eigenvector; the probed blocks leave the e and f equations
untouched at rest; the sparse and the dense eigenvalues agree.
"""
import numpy as np
import scipy.linalg as sla
import scipy.optimize as sopt
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .shell import BC_ROWS, Shell


def conductive_blocks(shell):
    """Per-pair blocks of N_cond: (adv, buo, leak).

    adv[p] (N_r x N_r): the T-equation rows of the linearised explicit terms at U_cond
    applied to f of pair p (coefficients -> values at the collocation radii);
    buo[p]: the f-equation rows of the buoyancy per unit Ra applied to T of pair p;
    leak: the largest e/f-equation entry of the advection probes (zero at rest)."""
    Nr, P = shell.Nr, shell.P
    X = shell.to_complex(shell.conductive_state())
    gX = shell.grid_fields(X)
    adv = np.zeros((P, Nr, Nr), dtype=np.complex128)
    buo = np.zeros((P, Nr, Nr), dtype=np.complex128)
    leak = 0.0
    for k in range(Nr):
        x = np.zeros((3, P, Nr), dtype=np.complex128)
        x[1, :, k] = 1.0
        N = shell.explicit_terms_linear(X, x, gX)
        adv[:, :, k] = N[2]
        leak = max(leak, float(np.abs(N[0]).max()), float(np.abs(N[1]).max()))
        T = np.zeros((P, Nr), dtype=np.complex128)
        T[:, k] = 1.0
        buo[:, :, k] = shell.buoyancy(T) / shell.Ra
    return adv, buo, leak


class Pencil:
    """A(Ra) = A0 + Ra A1 and M for one (m, class), with the unknowns' layout.

    Unknowns: for block i of chain_fields(m, cls) (l = m + i) the N_r Chebyshev
    coefficients of that potential (e or f), followed, for an f block, by those of T at
    the same l (T shares the equatorial symmetry of f)."""

    def __init__(self, shell, m, cls, blocks=None, rotation=True, l_only=None):
        """l_only: without rotation the degrees decouple; keep only the blocks of degree
        l_only (its class must hold f at that degree)."""
        self.shell, self.m, self.cls, self.rotation = shell, int(m), int(cls), bool(rotation)
        s = shell
        Nr = s.Nr
        adv, buo, _ = blocks if blocks is not None else conductive_blocks(s)
        flds = s.chain_fields(self.m, self.cls)
        if l_only is not None:
            if rotation or flds[l_only - self.m] != "f":
                raise ValueError("l_only needs rotation=False and an f block at that degree")
        layout = []   # (field, l, offset)
        off = 0
        for i, fl in enumerate(flds):
            if l_only is not None and self.m + i != l_only:
                continue
            layout.append((fl, self.m + i, off))
            off += Nr
            if fl == "f":
                layout.append(("T", self.m + i, off))
                off += Nr
        self.layout, self.n = layout, off
        where = {(fl, l): o for fl, l, o in layout}
        r = s._rows()
        E = s.E
        # block lists (row offset, column offset, N_r x N_r block) of A0, A1 and M, assembled
        # as sparse matrices (the pencil is block-tridiagonal in l)
        blk = {"A0": [], "A1": [], "M": []}
        m = self.m
        for fl, l, o in layout:
            p = s.pair_index(l, m)
            if fl != "T" and l == 0:
                blk["A0"].append((o, o, np.eye(Nr)))   # e_00, f_00 vanish (identity rows)
                continue
            K = s.diffusion_rows(fl, l, E, r).astype(np.complex128)
            if fl != "T" and self.rotation:
                K = K + s.coriolis_diag_rows(fl, l, m, E, r)
            D = -K
            Mb = s.mass_rows(fl, l, E, r).astype(np.complex128)
            s._bc_rows(D, fl)            # boundary functionals replace the wall rows
            for j in BC_ROWS[fl]:
                Mb[j] = 0.0
            blk["A0"].append((o, o, D))
            blk["M"].append((o, o, Mb))
            if fl in ("e", "f") and self.rotation:
                other = "f" if fl == "e" else "e"
                for side in (-1, 1):
                    key = (other, l + side)
                    if key in where and l + side >= m:
                        Cp = -np.array(s.coupling_rows(l, m, side, E, r), dtype=np.complex128)
                        for j in BC_ROWS[fl]:
                            Cp[j] = 0.0
                        blk["A0"].append((o, where[key], Cp))
            if fl == "f":
                B = buo[p].copy()
                for j in BC_ROWS["f"]:
                    B[j] = 0.0
                blk["A1"].append((o, where[("T", l)], B))
            if fl == "T":
                Ad = adv[p].copy()
                for j in BC_ROWS["T"]:
                    Ad[j] = 0.0
                blk["A0"].append((o, where[("f", l)], Ad))

        def assemble(blocks):
            rows, cols, vals = [], [], []
            ii, jj = np.meshgrid(np.arange(Nr), np.arange(Nr), indexing="ij")
            for r0, c0, b in blocks:
                rows.append((r0 + ii).ravel())
                cols.append((c0 + jj).ravel())
                vals.append(np.asarray(b, dtype=np.complex128).ravel())
            if not blocks:
                return sp.csr_matrix((off, off), dtype=np.complex128)
            return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                 shape=(off, off))

        self.A0, self.A1, self.M = assemble(blk["A0"]), assemble(blk["A1"]), assemble(blk["M"])

    def matrix(self, Ra):
        """A(Ra) as a sparse matrix."""
        return self.A0 + Ra * self.A1

    def state(self, v):
        """The canonical real state vector (shell layout) holding eigenvector v."""
        s = self.shell
        x = np.zeros((3, s.P, s.Nr), dtype=np.complex128)
        fi = {"e": 0, "f": 1, "T": 2}
        for fl, l, o in self.layout:
            x[fi[fl], s.pair_index(l, self.m)] = v[o:o + s.Nr]
        return s.to_real(x)


def _finite(w, V=None):
    ok = np.isfinite(w) & (np.abs(w) < 1e12)
    return (w[ok], V[:, ok]) if V is not None else w[ok]


def eig_dense(pen, Ra, vectors=True):
    """All finite eigenvalues (and eigenvectors) of A(Ra) x = sigma M x (QZ)."""
    A, M = pen.matrix(Ra).toarray(), pen.M.toarray()
    if not vectors:
        return _finite(sla.eigvals(A, M)), None
    w, V = sla.eig(A, M)
    return _finite(w, V)


def eig_near(pen, Ra, shift, k=8, seed=0):
    """The k eigenvalues nearest `shift` (and eigenvectors): Arnoldi on (A - s M)^{-1} M."""
    A = sp.csc_matrix(pen.matrix(Ra) - shift * pen.M)
    Ms = pen.M
    lu = spla.splu(A)
    op = spla.LinearOperator(A.shape, matvec=lambda x: lu.solve(Ms @ x), dtype=np.complex128)
    v0 = np.random.default_rng(seed).standard_normal(A.shape[0]) + 0j
    nu, V = spla.eigs(op, k=k, which="LM", v0=v0, ncv=max(2 * k + 1, 40), tol=1e-13)
    return shift + 1.0 / nu, V


def rightmost(pen, Ra, shift=None, k=8, vectors=True):
    """(sigma, v): the eigenvalue of largest real part (dense), or of largest real part
    among the k nearest `shift` (sparse); v is None when vectors=False (dense only)."""
    if shift is None:
        w, V = eig_dense(pen, Ra, vectors)
    else:
        w, V = eig_near(pen, Ra, shift, k)
    j = int(np.argmax(w.real))
    return w[j], (V[:, j] if V is not None else None)


def critical_rayleigh(pen, bracket, shift=None, k=8, xtol=1e-12):
    """Onset of (m, class): the root of max Re sigma(Ra) in `bracket` (Brent).

    shift = None: dense QZ at every Ra.  shift = "auto": one dense QZ at the bracket's
    midpoint picks the rightmost eigenvalue, and Arnoldi near it serves the root search.

    Returns dict(Ra, sigma, omega, C, v, state): the neutral eigenvalue sigma = i omega
    (its real part is the root's residual), the drift C = -omega/m, the eigenvector v
    normalised to unit 2-norm with its largest T coefficient real and positive, and the
    corresponding canonical real state vector."""
    def g(Ra):
        return rightmost(pen, Ra, shift, k, vectors=False)[0].real

    lo, hi = bracket
    if isinstance(shift, str):
        shift = rightmost(pen, 0.5 * (lo + hi), vectors=False)[0]
    Ra = sopt.brentq(g, lo, hi, xtol=xtol * max(1.0, abs(hi)), rtol=4 * np.finfo(float).eps)
    sig, v = rightmost(pen, Ra, shift, k)
    tmask = np.zeros(pen.n, dtype=bool)
    for fl, l, o in pen.layout:
        if fl == "T":
            tmask[o:o + pen.shell.Nr] = True
    jt = int(np.argmax(np.where(tmask, np.abs(v), -1.0)))
    v = v / np.linalg.norm(v)
    v = v * (abs(v[jt]) / v[jt])
    omega = sig.imag
    C = -omega / pen.m if pen.m else 0.0
    return dict(Ra=Ra, sigma=sig, omega=omega, C=C, v=v, state=pen.state(v))


def onset(L, Nr, Ek, m, bracket, cls=1, Pr=1.0, eta=0.35, rotation=True, shift=None, k=8):
    """critical_rayleigh for mode m of the truncation (L, N_r) at (Ek, Pr, eta); cls = 1 is
    the equatorially symmetric class (f and T at l - m even, e at l - m odd)."""
    shell = Shell(L, max(int(m), 1), Nr, Ek, 1.0, Pr=Pr, eta=eta)
    pen = Pencil(shell, m, cls, rotation=rotation)
    out = critical_rayleigh(pen, bracket, shift, k)
    out["pencil"] = pen
    return out
