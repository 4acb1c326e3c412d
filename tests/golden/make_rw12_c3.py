"""Write tests/golden/rw12_c3_oracle.txt: the oracle's rotating wave RW12 of Table 1 row 3
(Ek = 1e-5, Ra = 140, Pr = 1, r_in/r_out = 0.35, 12-fold symmetry) at the benchmark
truncation L = 127, N_r = 64, with its drift speed, kinetic energy and Nusselt numbers.

Calls only oracle/ (and the seeded-input layout): the conductive state plus the m = 12
seed of seeded_inputs.mode_seed(seed=4000, amp=1e-2) is time-stepped by the oracle's IMEX
Euler step (dt = 1e-4) until the m = 12 temperature amplitude settles, the drift is read
off its phase rate, and the oracle's Newton-GMRES (Secs. 3.3-3.4, dt = 200) converges the
wave to ||B(U) - U|| < 1e-10.  About half an hour on 8 cores.

    python tests/golden/make_rw12_c3.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import seeded_inputs as si  # noqa: E402
from oracle import krylov  # noqa: E402
from oracle.shell import Shell  # noqa: E402

L, Ms, Nr, Ek, Ra, M = 127, 12, 64, 1e-5, 140.0, 12
DT, CHUNK, MAX_STEPS = 1e-4, 100, 6000


def main():
    t0 = time.time()
    s = Shell(L, Ms, Nr, Ek, Ra)
    U = s.conductive_state() + si.mode_seed(L, Ms, Nr, M, seed=4000, amp=1e-2)
    pM = s.pair_index(M, M)
    prev, steps = None, 0
    while steps < MAX_STEPS:
        U = s.step(U, 0.0, DT, nsteps=CHUNK)
        steps += CHUNK
        amp = float(np.linalg.norm(s.to_complex(U)[2, pM]))
        print(f"step {steps}: |T_12| = {amp:.6e}  ({time.time() - t0:.0f} s)", flush=True)
        if prev is not None and amp > 1e-3 and abs(amp - prev) < 1e-4 * amp:
            break
        prev = amp
    U1 = s.step(U, 0.0, DT, nsteps=10)
    C0 = krylov.drift_estimate(s, U, U1, 10 * DT, M)
    J = krylov.phase_index(s, U, M)
    print(f"guess after {steps} steps: C0 = {C0:.6f}, J = {J}", flush=True)
    Uw, C, hist = krylov.newton(s, U, C0, J, dt=200.0, tol=1e-10, max_newton=10, kmax=400,
                                verbose=True)
    nu_in, nu_out = s.nusselt(Uw)
    ke = s.kinetic_energy(Uw)
    res = hist[-1]["residual"]
    out = os.environ.get("RSC_GOLDEN_OUT", os.path.join(HERE, "rw12_c3_oracle.txt"))
    with open(out, "w") as f:
        f.write("# The oracle's RW12 wave at L = 127, Ms = 12, N_r = 64, Ek = 1e-5, Ra = 140 (Table 1\n")
        f.write("# row 3 parameters at the benchmark truncation), written by make_rw12_c3.py from\n")
        f.write(f"# seeded_inputs.mode_seed(seed=4000, amp=1e-2), {steps} oracle steps of dt = {DT},\n")
        f.write(f"# Newton-GMRES at dt = 200: {len(hist) - 1} iterations, final ||B(U) - U|| = {res:.3e}.\n")
        f.write("# key value\n")
        f.write(f"C {float(C)!r}\nKE {float(ke)!r}\nNu_in {float(nu_in)!r}\n"
                f"Nu_out {float(nu_out)!r}\nresidual {float(res)!r}\n")
        f.write(f"phase_slot {J}\nnewton_iterations {len(hist) - 1}\n")
    print(f"wrote {out} after {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
