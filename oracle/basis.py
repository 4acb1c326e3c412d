"""Radial and angular basis tables of the oracle (plain FP64).

Radial direction (Sec. 3.1, Eq. expansion): every field is a sum of
Chebyshev polynomials T_k(x) of the shifted radius
x = (2r - r_out - r_in)/(r_out - r_in).  Equations are collocated at the
Gauss-Lobatto points x_j = cos(pi j/(N-1)); the 3/2 de-aliasing rule in r
(Sec. 3.1) uses N_d = ceil(3 N_r / 2) Gauss-Lobatto points.

Angular direction (Sec. 3.1, Eq. Ylm_norm): Y_l^m = N_l^m P_l^m(cos th) e^{i m phi}
with N_l^m = sqrt((2 - delta_m0)(2l+1)(l-m)!/(l+m)!) and no Condon-Shortley
phase.  Integrals over theta use Gauss-Legendre quadrature on nlat nodes.

Pins (tests/test_oracle_basis.py): Chebyshev values against cos(k arccos x)
and the closed-form endpoint derivatives; exact differentiation of random
polynomials; Gauss-Legendre exactness on monomials and, at n = 192 and 384,
on scipy's Legendre polynomials to the rounding level; P_l^m against
scipy.special.lpmv; discrete orthogonality up to L = 255; Unsold's sum rule
at L = 255; the scaled start against exact rational evaluation of the
Rodrigues form far below the double range; the recursions Eq. recu1 and
Eq. recu2 evaluated on the grid; dP/dtheta against finite differences.
"""
import decimal
import functools
import math

import numpy as np
from numpy.polynomial import chebyshev as _cheb


def shell_radii(eta):
    """Inner and outer radii for gap width 1 and radius ratio eta (Sec. 2.1)."""
    r_out = 1.0 / (1.0 - eta)
    r_in = eta / (1.0 - eta)
    return r_in, r_out


def lobatto_x(n):
    """Gauss-Lobatto points x_j = cos(pi j/(n-1)), j = 0..n-1 (x_0 = +1 is r_out)."""
    j = np.arange(n)
    return np.cos(np.pi * j / (n - 1))


def x_to_r(x, r_in, r_out):
    """Invert x = (2r - r_out - r_in)/(r_out - r_in) (Sec. 3.1)."""
    return r_in + 0.5 * (np.asarray(x) + 1.0) * (r_out - r_in)


def cheb_matrix(x, nk, order, r_in, r_out):
    """M[i, k] = d^order/dr^order of T_k evaluated at x_i, k < nk.

    Differentiation in r is 2/(r_out - r_in) times differentiation in x.
    """
    x = np.asarray(x, dtype=np.float64)
    scale = (2.0 / (r_out - r_in)) ** order
    out = np.empty((x.size, nk))
    for k in range(nk):
        c = np.zeros(nk)
        c[k] = 1.0
        d = _cheb.chebder(c, order) if order else c
        out[:, k] = _cheb.chebval(x, d) * scale
    return out


def dealias_nr(nr):
    """Number of radial points of the 3/2-rule de-aliased grid (Sec. 3.1)."""
    return -(-3 * nr // 2)


def nlat_for(L):
    """Gauss-Legendre latitudes: the smallest even count >= 3(L+1)/2.

    The paper lets SHTns pick an angular grid exact for quadratic terms
    (Sec. 3.1); 3(L+1)/2 nodes integrate exactly the triple products of
    degree <= 3L that a quadratic nonlinearity produces.
    """
    return 2 * ((3 * (L + 1) + 3) // 4)


def nphi_for(L, Ms):
    """Points per azimuthal sector: smallest 2^a 3^b >= 3K+1, K = floor(L/Ms)."""
    need = 3 * (L // Ms) + 1
    best = None
    a = 1
    while a < 4 * need:
        b = a
        while b < 4 * need:
            if b >= need and (best is None or b < best):
                best = b
            b *= 3
        a *= 2
    return best


def _legendre_pair_dec(n, x):
    """P_n(x), P_{n-1}(x) by Bonnet's recursion (k+1)P_{k+1} = (2k+1)x P_k - k P_{k-1}."""
    p0, p1 = type(x)(1), x
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    return p1, p0


@functools.lru_cache(maxsize=None)
def _gauss_legendre_nodes(n):
    """Nodes and weights of the n-point Gauss-Legendre rule, north first.

    Each node is a root of P_n found by Newton's method in 40-digit decimal
    arithmetic, started from the asymptotic guess cos(pi (i + 3/4)/(n + 1/2));
    its weight is w = 2 (1 - x^2) / (n P_{n-1}(x))^2 (at a root of P_n,
    (1 - x^2) P_n'(x) = n P_{n-1}(x)).  Node and weight are rounded to double
    only at the end, so both are correct to the last bit; double-precision
    Newton loses up to 1e-10 of the weights near the poles at n = 384 because
    P_n' is large there.
    """
    x = np.empty(n)
    w = np.empty(n)
    with decimal.localcontext() as ctx:
        ctx.prec = 40
        tol = decimal.Decimal(10) ** -36
        for i in range((n + 1) // 2):
            z = decimal.Decimal(math.cos(math.pi * (i + 0.75) / (n + 0.5)))
            for _ in range(100):
                pn, pm = _legendre_pair_dec(n, z)
                dp = n * (pm - z * pn) / (1 - z * z)
                dz = pn / dp
                z -= dz
                if abs(dz) < tol:
                    break
            else:
                raise RuntimeError("Gauss-Legendre Newton iteration did not converge")
            pn, pm = _legendre_pair_dec(n, z)
            one_m = (1 - z) * (1 + z)
            wi = 2 * one_m / (n * pm) ** 2
            x[i], w[i] = float(z), float(wi)
            x[n - 1 - i], w[n - 1 - i] = -x[i], w[i]
    if n % 2:
        x[n // 2] = 0.0
    return x, w


def gauss_legendre(n):
    """Gauss-Legendre nodes and weights on [-1, 1], ordered north (x ~ 1) first."""
    x, w = _gauss_legendre_nodes(n)
    return x.copy(), w.copy()


def gauss_legendre_sin(n):
    """sin(theta) = sqrt((1 - x)(1 + x)) at the (double) nodes of gauss_legendre(n).

    Formed from the rounded node itself (1 - x is exact for x >= 1/2), so that
    x^2 + sin^2 = 1 to rounding and the tables are values at one point.
    """
    x = _gauss_legendre_nodes(n)[0]
    return np.sqrt((1.0 - x) * (1.0 + x))


def plm_bar(lmax, m, x, s=None):
    """pbar_l^m(x) = sqrt((2l+1)(l-m)!/(l+m)!) P_l^m(x), rows l = m..lmax.

    No Condon-Shortley phase.  Three-term recursion in l at fixed m, started
    from pbar_m^m = prod_k sqrt((2k+1)/(2k)) (1-x^2)^{m/2} and
    pbar_{m+1}^m = sqrt(2m+3) x pbar_m^m.  ``s`` = sqrt(1 - x^2) may be given
    (as computed together with the nodes); otherwise it is formed from x.

    Scaled start: near the poles (1-x^2)^{m/2} leaves the double range for
    large m, so the start and the recursion carry a power-of-two exponent per
    node (values are kept in [2^-500, 2^500] by exact rescaling by 2^500) and
    are scaled back with ldexp at the end: entries below the double range
    become 0, the others keep full precision.
    """
    x = np.asarray(x, dtype=np.float64)
    if s is None:
        s = np.sqrt(np.maximum(0.0, (1.0 - x) * (1.0 + x)))
    s = np.asarray(s, dtype=np.float64)
    out = np.zeros((lmax - m + 1, x.size))
    if lmax < m:
        return out
    big = 2.0 ** 500
    e = np.zeros(x.size, dtype=np.int64)   # value = stored * 2^(500 e)
    pmm = np.ones_like(x)
    for k in range(1, m + 1):
        pmm = pmm * s * np.sqrt((2.0 * k + 1.0) / (2.0 * k))
        low = (pmm != 0.0) & (np.abs(pmm) < 1.0 / big)
        pmm = np.where(low, pmm * big, pmm)
        e = e - low
    v_prev = np.zeros_like(x)
    v = pmm
    out[0] = np.ldexp(v, 500 * e)
    if lmax == m:
        return out
    v_prev, v = v, x * np.sqrt(2.0 * m + 3.0) * v
    out[1] = np.ldexp(v, 500 * e)
    for l in range(m + 2, lmax + 1):
        a = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
        b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
        v_prev, v = v, a * (x * v - b * v_prev)
        high = (e < 0) & (np.abs(v) > big)
        v = np.where(high, v / big, v)
        v_prev = np.where(high, v_prev / big, v_prev)
        e = e + high
        out[l - m] = np.ldexp(v, 500 * e)
    return out


def dplm_bar_dtheta(lmax, m, x, s=None):
    """d pbar_l^m(cos theta) / d theta, rows l = m..lmax.

    Uses the ladder in m (not the recursion in l that the pins check):
      m = 0:  d pbar_l^0/dth = -sqrt(l(l+1)) pbar_l^1
      m > 0:  d pbar_l^m/dth = (sqrt((l+m)(l-m+1)) pbar_l^{m-1}
                                - sqrt((l+m+1)(l-m)) pbar_l^{m+1}) / 2
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((lmax - m + 1, x.size))
    up = plm_bar(lmax, m + 1, x, s) if m + 1 <= lmax else None  # rows l = m+1..
    if m == 0:
        for l in range(1, lmax + 1):
            out[l] = -np.sqrt(l * (l + 1.0)) * up[l - 1]
        return out
    down = plm_bar(lmax, m - 1, x, s)  # rows l = m-1..
    for l in range(m, lmax + 1):
        v = np.sqrt((l + m) * (l - m + 1.0)) * down[l - m + 1]
        if l >= m + 1:
            v = v - np.sqrt((l + m + 1.0) * (l - m)) * up[l - m - 1]
        out[l - m] = 0.5 * v
    return out


def ylm_norm_factor(m):
    """sqrt(2 - delta_m0): the paper's N_l^m over sqrt((2l+1)(l-m)!/(l+m)!)."""
    return np.sqrt(2.0) if m > 0 else 1.0
