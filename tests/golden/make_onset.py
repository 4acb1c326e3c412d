"""Write onset_workloads.txt: the oracle's linear onset (oracle/onset.py) of the rotating
waves of the workloads, at their own truncations.

For each workload mode (Ek, m, L, N_r): the equatorially symmetric class; a dense QZ scan
of Ra = c Ek^(-1/3) on the coarsest truncation of the chain brackets the first crossing,
and each finer truncation repeats the root search with Arnoldi near the previous level's
neutral eigenvalue, in a bracket of +-15 % around its Ra_c.  Only the last level's values
are written.  Run from the repository root:

    python tests/golden/make_onset.py [NAME ...]

(several minutes of CPU time for C5; RSC_GOLDEN_OUT redirects the output file).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import onset as on  # noqa: E402
from oracle.shell import Shell  # noqa: E402

# name: (Ek, m, [(L, N_r) from coarse to the workload's own truncation])
WORKLOADS = {
    "C1": (1e-3, 4, [(31, 24)]),
    "C2": (1e-4, 8, [(31, 16), (47, 24), (63, 48)]),
    "C3": (1e-5, 12, [(47, 24), (79, 40), (127, 64)]),
    "C4_m4": (3e-5, 4, [(47, 24), (95, 48)]),
    "C4_m6": (3e-5, 6, [(47, 24), (95, 48)]),
    "C4_m8": (3e-5, 8, [(47, 24), (95, 48)]),
    "C4_m10": (3e-5, 10, [(47, 24), (95, 48)]),
    "C4_m12": (3e-5, 12, [(47, 24), (95, 48)]),
    "C5": (3e-6, 8, [(47, 24), (95, 40), (159, 64), (255, 96)]),
    "C5_m16": (3e-6, 16, [(63, 24), (127, 40), (191, 64), (255, 96)]),
    "C5_m24": (3e-6, 24, [(71, 24), (127, 40), (191, 64), (255, 96)]),
}
SCAN = (1.0, 1.5, 2.0, 2.5, 3.0, 4.0, 5.0, 6.0, 8.0, 11.0, 15.0)


def solve(name):
    Ek, m, levels = WORKLOADS[name]
    shift = Ra0 = None
    for L, Nr in levels:
        t0 = time.time()
        pen = on.Pencil(Shell(L, m, Nr, Ek, 1.0), m, 1)
        if shift is None:
            prev = None
            for c in SCAN:
                Ra = c * Ek ** (-1.0 / 3.0)
                sig = on.rightmost(pen, Ra, vectors=False)[0]
                if sig.real > 0:
                    break
                prev = Ra
            else:
                raise RuntimeError(f"{name}: no onset below {Ra}")
            if prev is None:
                raise RuntimeError(f"{name}: unstable at the first scan point")
            r = on.critical_rayleigh(pen, (prev, Ra), shift=sig, k=12)
        else:
            r = on.critical_rayleigh(pen, (0.85 * Ra0, 1.15 * Ra0), shift=shift, k=12)
        shift, Ra0 = r["sigma"], r["Ra"]
        print(f"{name} L={L} Nr={Nr} n={pen.n} Ra_c={r['Ra']:.10f} omega={r['omega']:.8f} "
              f"C={r['C']:.8f} ({time.time() - t0:.0f} s)", flush=True)
    return dict(Ek=Ek, m=m, L=L, Nr=Nr, Ra=r["Ra"], omega=r["omega"], C=r["C"])


def main(names):
    out = os.environ.get("RSC_GOLDEN_OUT", os.path.join(HERE, "onset_workloads.txt"))
    rows = {}
    if os.path.exists(out):
        for line in open(out):
            if line.strip() and not line.startswith("#"):
                rows[line.split()[0]] = line.rstrip("\n")
    for name in names:
        v = solve(name)
        rows[name] = (f"{name} {v['Ek']:.3e} {v['m']} {v['L']} {v['Nr']} {float(v['Ra']):.10f} "
                      f"{float(v['omega']):.8f} {float(v['C']):.8f}")
        with open(out, "w") as f:
            f.write("# Linear onset of the workloads' rotating waves (oracle/onset.py, written by\n"
                    "# tests/golden/make_onset.py): Pr = 1, r_in/r_out = 0.35, equatorially\n"
                    "# symmetric class.  Columns: name Ek m L N_r Ra_c omega C_c (C_c = -omega/m,\n"
                    "# the drift of the wave at onset in the convention U(phi - C t)).\n")
            for k in WORKLOADS:
                if k in rows:
                    f.write(rows[k] + "\n")


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
