"""Seeded synthetic inputs shared by the tests, smoke() and bench.py.

This module holds no arithmetic of the method: it only draws Gaussian numbers
and lays them out in the canonical state order
    [field e, f, T][pair (m, l): m = 0, Ms, ... <= L, l = m..L][k < Nr][re, im].
Both the oracle and the CUDA library receive the same arrays.

Perturbation recipe: amplitude
    amp * exp(-l/8) * exp(-k/6) * N(0, 1)
on the real and imaginary part of every allowed coefficient; imaginary parts
of m = 0 coefficients and the absent e_00, f_00 are zero.
"""
import numpy as np


def layout(L, Ms, Nr):
    """(pair_l, pair_m) arrays of the canonical pair order."""
    pl, pm = [], []
    for m in range(0, L + 1, Ms):
        for l in range(m, L + 1):
            pl.append(l)
            pm.append(m)
    return np.array(pl), np.array(pm)


def state_size(L, Ms, Nr):
    pl, _ = layout(L, Ms, Nr)
    return 3 * len(pl) * Nr * 2


def perturbation(L, Ms, Nr, seed, amp=1e-3, l_decay=8.0, k_decay=6.0):
    """Real canonical vector of a decaying Gaussian perturbation."""
    pl, pm = layout(L, Ms, Nr)
    P = len(pl)
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((3, P, Nr, 2))
    k = np.arange(Nr)
    w = amp * np.exp(-pl[:, None] / l_decay) * np.exp(-k[None, :] / k_decay)
    z *= w[None, :, :, None]
    z[:, pm == 0, :, 1] = 0.0
    z[0:2, pl == 0] = 0.0
    return z.reshape(-1)


def mode_seed(L, Ms, Nr, M, seed, amp=1e-2):
    """The perturbation recipe restricted to the azimuthal wavenumber m = M (a cos(M phi)-like
    seed for reaching a rotating wave by time stepping, as in Sec. 2.2)."""
    pl, pm = layout(L, Ms, Nr)
    z = perturbation(L, Ms, Nr, seed, amp=amp).reshape(3, len(pl), Nr, 2)
    z[:, pm != M] = 0.0
    return z.reshape(-1)


def random_vector(L, Ms, Nr, seed, amp=1.0):
    """A Gaussian direction vector with the same decay and zero pattern (for Jacobian tests)."""
    return perturbation(L, Ms, Nr, seed, amp=amp)


# Linear onset Ra_c of each workload's rotating wave (mode m = M, equatorially symmetric,
# Pr = 1, r_in/r_out = 0.35) at the workload's own truncation: the values that
# tests/golden/make_onset.py wrote to tests/golden/onset_workloads.txt from the oracle's
# linear analysis (tests/test_oracle_onset.py checks that the two tables agree).  The
# paper prints no onset values.
ONSET_RA = {
    "C1": 55.9041816078,
    "C2": 69.5958906601,
    "C3": 111.2929193930,
    "C4_m4": 118.4463565448,
    "C4_m6": 100.8089645706,
    "C4_m8": 90.3601771719,
    "C4_m10": 85.2962306339,
    "C4_m12": 85.8781358929,
    "C5": 219.0622885318,
}


def config(name):
    """Truncation and physical parameters of the named workloads.

    Ra is given as a multiple of the onset value when `ra_factor` is set; the
    absolute Ra used for timing runs is stated next to it.
    """
    table = {
        # L, Ms, Nr, Ek, dt, Ra
        "tiny": dict(L=7, Ms=4, Nr=10, Ek=1e-3, dt=1e-4, Ra=80.0),
        "C1": dict(L=31, Ms=4, Nr=24, Ek=1e-3, dt=1e-4, Ra=120.0),
        "C2": dict(L=63, Ms=8, Nr=48, Ek=1e-4, dt=2e-5, Ra=130.0),
        "C3": dict(L=127, Ms=12, Nr=64, Ek=1e-5, dt=5e-6, Ra=140.0),
        # C5 at 1.1 x the onset of its m = 8 wave
        "C5": dict(L=255, Ms=8, Nr=96, Ek=3e-6, dt=2e-6, Ra=1.1 * ONSET_RA["C5"]),
    }
    d = dict(table[name])
    d.update(Pr=1.0, eta=0.35)
    return d
