#!/usr/bin/env python
"""Benchmark of the Newton-GMRES hot path on one or more GB300s (one process per GPU).

Workload: the RW12 problem of Table 1 row 3 (Ek = 1e-5, Ra = 140, Pr = 1,
r_in/r_out = 0.35, 12-fold azimuthal symmetry) at truncation L = 127,
N_r = 64 (the low-Ekman configuration).  One bench step is one Newton
iteration of the rotating-wave solver (Secs. 3.3-3.4): the FP64 residual
B(U) - U at the pseudo-timestep dt = 200, a GMRES solve with a fixed number
of Jacobian actions (every row of the hot path: radial evaluation, Legendre
synthesis, azimuthal DFT, grid products, analysis, right-hand side, the
implicit-Coriolis chain solves, one-reduction MGS orthogonalisation), the Newton update and
the new residual.  The metric is Jacobian actions per second.

Inputs are synthetic and seeded: the conductive state plus a decaying
Gaussian perturbation; the state is reset from a device copy before every
step and L2 is flushed (a 256 MB write) between steps, outside the timed
interval of each step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference   # the FP64 CPU oracle on the host cores
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import seeded_inputs as si  # noqa: E402

WORKLOAD = dict(name="RW12 Ek=1e-5 Ra=140 (Table 1 row 3), L=127, Ms=12, Nr=64",
                L=127, Ms=12, Nr=64, Ek=1e-5, Ra=140.0, Pr=1.0, eta=0.35)
METRIC = "Jacobian actions/s in Newton-GMRES (timesteps/s, JVPs/s, Newton time at Ek=1e-5)"
UNIT = "JVP/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--krylov", type=int, default=200,
                    help="Jacobian actions per Newton iteration (the RW12 solve takes 208-216)")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-rw", action="store_true", help="skip the time-to-rotating-wave run")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-instances run")
    ap.add_argument("--no-fp64-arm", action="store_true",
                    help="skip the FP64-path and factorisation timings (profiling runs)")
    ap.add_argument("--chain-parts", type=int, default=1,
                    help="parts per chain of the mixed path's double-float solve after "
                         "autotuning (1: unpartitioned, the faster at RW12)")
    ap.add_argument("--tuning", default=None,
                    help="launch shapes as JSON (the line's `tuning`) instead of autotuning, so "
                         "that a profiled run uses the shapes of a measured one")
    ap.add_argument("--dt-study", default=None,
                    help="only run the Table 1 time-step study for the given rows (e.g. 0,1,2)")
    ap.add_argument("--configs-study", action="store_true",
                    help="only run the other configurations (C1, C2, C5 throughput, C2 wave, "
                         "mixed batched Newton)")
    ap.add_argument("--coriolis-study", action="store_true",
                    help="only run the implicit vs explicit Coriolis comparison (Sec. 5)")
    ap.add_argument("--resolution-study", action="store_true",
                    help="only run the resolution study of the RW12 drift (Table 1 row 3)")
    ap.add_argument("--implicit-solves", type=int, default=0,
                    help="only run this many implicit solves (rsc_implicit_solve, dt = 200) on "
                         "a context of the workload, for a profiler capture of the chain solve")
    ap.add_argument("--c5", action="store_true",
                    help="only run the large single instance (L = 255, N_r = 96): 1000 time "
                         "steps and one Newton iteration of 100 Jacobian actions per precision")
    ap.add_argument("--c5-steps", type=int, default=1000, help="time steps of --c5")
    ap.add_argument("--c5-krylov", type=int, default=100, help="Jacobian actions of --c5")
    ap.add_argument("--c5-precision", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--c5-wave-krylov", type=int, default=1000,
                    help="Jacobian actions per Newton iteration at most, for --c5-wave")
    ap.add_argument("--c5-wave", action="store_true",
                    help="with --c5: also converge the m = 8 rotating wave (time stepping from "
                         "the m = 8 seed until it settles, then Newton-GMRES to 1e-10) on "
                         "the mixed path and time it")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def cpu_oracle_sample(krylov, budget_s=25.0):
    """Time the FP64 oracle on a bounded sample of the same Newton iteration.

    Factorisation (done once per dt, as on the GPU) is excluded; one residual
    step and as many Jacobian actions as fit in the budget are timed, and the
    iteration time is 2 t_step + krylov t_jvp.
    """
    import numpy as np
    from oracle.shell import Shell
    w = WORKLOAD
    s = Shell(w["L"], w["Ms"], w["Nr"], w["Ek"], w["Ra"], w["Pr"], w["eta"])
    x = s.conductive_state() + si.perturbation(w["L"], w["Ms"], w["Nr"], seed=3000)
    u = si.random_vector(w["L"], w["Ms"], w["Nr"], seed=3001)
    s.factor(200.0)
    t0 = time.perf_counter()
    s.step(x, 0.0, 200.0)
    t_step = time.perf_counter() - t0
    gU = s.grid_fields(s.to_complex(x))
    n_jvp = 0
    t0 = time.perf_counter()
    while True:
        s.jvp(x, 0.0, None, u, 200.0, gU)
        n_jvp += 1
        if time.perf_counter() - t0 > budget_s - t_step or n_jvp >= krylov:
            break
    t_jvp = (time.perf_counter() - t0) / n_jvp
    t_iter = 2 * t_step + krylov * t_jvp
    return {"value": krylov / t_iter, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"1 FP64 step + {n_jvp} Jacobian actions of the same workload on the host "
                      f"(numpy/LAPACK, all cores); iteration time = 2 t_step + {krylov} t_jvp",
            "t_step_s": t_step, "t_jvp_s": t_jvp}


REF_ACTIONS_PER_STEP = 4


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, timed as it stands.  One step
    is REF_ACTIONS_PER_STEP Jacobian actions of the workload (the unit of the metric), each
    actually executed and timed; the oracle's factorisation and the base state's grid fields
    are built once before the warm-up, as on the GPU."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle.shell import Shell
    w = WORKLOAD
    s = Shell(w["L"], w["Ms"], w["Nr"], w["Ek"], w["Ra"], w["Pr"], w["eta"])
    x = s.conductive_state() + si.perturbation(w["L"], w["Ms"], w["Nr"], seed=3000)
    u = si.random_vector(w["L"], w["Ms"], w["Nr"], seed=3001)
    s.factor(200.0)
    gU = s.grid_fields(s.to_complex(x))
    times = []
    wall0 = time.perf_counter()
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for _ in range(REF_ACTIONS_PER_STEP):
            s.jvp(x, 0.5, None, u, 200.0, gU)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    wall = time.perf_counter() - wall0
    t = sum(times) / len(times)
    v = REF_ACTIONS_PER_STEP / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded perturbation of the conductive state)",
            "config": {"workload": w["name"],
                       "step": f"{REF_ACTIONS_PER_STEP} Jacobian actions (dt = 200) of the "
                               "FP64 oracle, all executed and timed",
                       "l2": "not applicable (CPU)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} timed steps of {REF_ACTIONS_PER_STEP} "
                                       "Jacobian actions each after "
                                       f"{args.warmup} warm-up steps (numpy/LAPACK on all "
                                       "host cores; factorisation excluded)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks(torch):
    """Peaks for the roofline: HBM and bf16 from MEASURED_PEAKS.json; FP64 / FP32 ALU from
    a cuBLAS DGEMM / SGEMM timed here on the same GPU."""
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        peaks["hbm_gbs"] = float(mp["hbm_gbs"])
        peaks["hbm_source"] = "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        peaks["hbm_gbs"] = 6800.0
        peaks["hbm_source"] = "fallback"
    for dt, key, N in ((torch.float64, "fp64_tflops", 4096), (torch.float32, "fp32_tflops", 8192)):
        a = torch.randn(N, N, dtype=dt, device="cuda")
        b = torch.randn(N, N, dtype=dt, device="cuda")
        for _ in range(2):
            a @ b
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(4):
            a @ b
        e1.record()
        torch.cuda.synchronize()
        peaks[key] = 2 * N ** 3 * 4 / (e0.elapsed_time(e1) * 1e-3) / 1e12
        del a, b
    torch.cuda.empty_cache()
    return peaks


# kernels whose arithmetic is FP64 on both paths; the transforms follow the path's precision
FP64_KERNELS = {"radial_eval", "rhs_assemble", "chain_gemv", "chain_sweep", "temp_solve",
                "gmres_dots", "gmres_axpy", "blas1"}


# DRAM bytes (read + write) per launch from one ncu capture of each kernel on this workload,
# keyed by (kernel class, arithmetic and chains): a figure holds only for the variant it was
# taken on
NCU_TRAFFIC_MB = {
    # k_chain_half_async: 95.3 + 2.9 MB; k_chain_out_async: 101.1 + 3.3 MB (mean per launch)
    ("chain_sweep", "fp64"): 101.3,
    # k_chain_half_df<2, 4>: 95.3 + 3.3 MB; k_chain_out_df<2, 4>: 101.1 + 3.3 MB (the two-warp
    # variant reads the same: 95.3 + 3.0 and 101.1 + 3.2 MB)
    ("chain_sweep", "df"): 101.5,
    # the sweeps over the odd-even reduced chains: k_chain_half_df<2, 4>: 45.5 + 0.0 MB,
    # k_chain_out_df<2, 4>: 51.3 + 18.7 MB
    ("chain_sweep", "df_cr"): 57.7,
    # k_cr_odd_df<8>: 49.9 + 1.3 MB, k_cr_even_df<8>: 51.4 + 2.0 MB, k_cr_back_df<8>: 50.7 + 1.0 MB
    ("chain_reduced", "df_cr"): 52.1,
}


def traffic_variant(name, precision, tuning, dfk):
    """The NCU_TRAFFIC_MB variant of a kernel class under this tuning."""
    if name not in dfk:
        return "fp64"
    if precision == "mixed" and tuning.get("chain_cr", 0) and name in ("chain_sweep", "chain_reduced"):
        return "df_cr"
    return "df"


def double_float_kernels(precision, tuning):
    """Kernel classes that run in double-float arithmetic (FP32 hi + lo pairs, Dot2 sums)
    under this tuning: the chain solve of the mixed path (chain_df) and the orthogonalisation
    against the split Krylov basis (krylov_split)."""
    out = set()
    if precision == "mixed" and tuning.get("chain_df", 0):
        out |= {"chain_sweep", "chain_gemv", "chain_reduced"}
    if tuning.get("krylov_split", 0):
        out |= {"gmres_dots", "gmres_axpy"}
    return out


def dtype_label(precision, tuning):
    """What the path computes in, from the tuning the run used."""
    if precision != "mixed":
        return "f64"
    parts = ["f32 transforms (tcgen05 3xTF32 Legendre sums) and Jacobian-action RHS"]
    parts.append("double-float e/f chain solve" if tuning.get("chain_df", 0)
                 else "f64 e/f chain solve")
    parts.append("double-float Krylov basis" if tuning.get("krylov_split", 0)
                 else "f64 Krylov basis")
    parts.append("f64 step / residual RHS, temperature solve and update")
    return " + ".join(parts)


def fp64_arm(torch, RotatingShell, w, K, nsteps=2):
    """The plain FP64 GPU path on the same workload (autotuned): Jacobian actions/s of one
    Newton iteration with K actions and IMEX Euler timesteps/s, CUDA events."""
    sh = RotatingShell(w["L"], w["Ms"], w["Nr"], w["Ek"], w["Ra"], w["Pr"], w["eta"])
    tuning = sh.autotune()
    U0 = sh.conductive_state() + torch.tensor(
        si.perturbation(w["L"], w["Ms"], w["Nr"], seed=3000), device="cuda")
    J = sh.phase_slot(w["Ms"], 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    U = U0.clone()
    sh.newton_rw(U, 0.5, J, tol=0.0, max_newton=1, kmax=K, gmres_tol=0.0)
    tot_ms, tot_act = 0.0, 0
    for _ in range(nsteps):
        U.copy_(U0)
        torch.cuda.synchronize()
        e0.record()
        _, rep, _ = sh.newton_rw(U, 0.5, J, tol=0.0, max_newton=1, kmax=K, gmres_tol=0.0)
        e1.record()
        torch.cuda.synchronize()
        tot_ms += e0.elapsed_time(e1)
        tot_act += rep["gmres_total"]
    U = U0.clone()
    sh.step(U, 0.0, 5e-6, nsteps=3)
    torch.cuda.synchronize()
    e0.record()
    sh.step(U, 0.0, 5e-6, nsteps=20)
    e1.record()
    torch.cuda.synchronize()
    tps = 20 / (e0.elapsed_time(e1) * 1e-3)
    sh.close()
    return {"jvps_per_s": tot_act / (tot_ms * 1e-3), "timesteps_per_s": tps,
            "ms_per_newton_iteration": tot_ms / nsteps, "tuning": tuning}


def factor_timing(torch, RotatingShell, w, dt=200.0):
    """Wall time of one factorisation of the implicit operator at dt (Sec. 3.2; Sec. 4.4
    refactorises at every new Ek) on the GPU (FP64 block LU kernels) and on the host."""
    out = {}
    for where, flag in (("gpu", 1), ("host", 0)):
        sh = RotatingShell(w["L"], w["Ms"], w["Nr"], w["Ek"], w["Ra"], w["Pr"], w["eta"])
        sh.set_tuning(dict(sh.tuning(), factor_gpu=flag))
        z = sh.new_state()
        sh.implicit_solve(z, dt)
        torch.cuda.synchronize()
        sec, on_gpu = sh.factor_time()
        out[where + "_s"] = sec
        out[where + "_ran_on_gpu"] = on_gpu
        sh.close()
        # the odd-even reduced chains of the mixed path's double-float solve
        sm = RotatingShell(w["L"], w["Ms"], w["Nr"], w["Ek"], w["Ra"], w["Pr"], w["eta"],
                           precision="mixed")
        sm.set_tuning(dict(sm.tuning(), factor_gpu=flag, chain_cr=1))
        sm.implicit_solve(sm.new_state(), dt)
        torch.cuda.synchronize()
        sec, on_gpu = sm.factor_time_cr()
        out["reduced_" + where + "_s"] = sec
        out["reduced_" + where + "_ran_on_gpu"] = on_gpu
        sm.close()
    out["host_cores"] = os.cpu_count()
    return out


def roofline(prof, peaks, precision, tuning):
    name = max(prof, key=lambda k: prof[k]["ms"])   # the only kernel timed in this pass
    p = prof[name]
    t = p["ms"] / max(1, p["launches"]) * 1e-3
    gbs = p["bytes"] / max(1, p["launches"]) / t / 1e9
    dfk = double_float_kernels(precision, tuning)
    if name in dfk:
        # FP64-equivalent flops carried out as FP32 pairs: no FP64 ALU bound applies; the
        # kernel reads its tables and vectors once, so HBM is the roofline
        out = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": gbs / peaks["hbm_gbs"], "peak_source": peaks["hbm_source"],
               "arithmetic": "double-float (FP32 hi + lo pairs, Dot2 sums)"}
    else:
        fp64 = name in FP64_KERNELS or precision == "fp64"
        alu_peak = peaks["fp64_tflops"] if fp64 else peaks["fp32_tflops"]
        tfs = p["flops"] / max(1, p["launches"]) / t / 1e12
        f_hbm = gbs / peaks["hbm_gbs"]
        f_alu = tfs / alu_peak
        if f_alu >= f_hbm:
            out = {"bound": "alu", "achieved": tfs, "peak": alu_peak, "unit": "TFLOP/s",
                   "frac": f_alu, "peak_source": ("FP64" if fp64 else "FP32") +
                   " cuBLAS GEMM timed in this run on this GPU (measured)",
                   "arithmetic": "FP64" if fp64 else "FP32"}
        else:
            out = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                   "frac": f_hbm, "peak_source": peaks["hbm_source"],
                   "arithmetic": "FP64" if fp64 else "FP32"}
    mb = NCU_TRAFFIC_MB.get((name, traffic_variant(name, precision, tuning, dfk)))
    out.update(kernel=name, traffic=mb * 1e6 if mb is not None else None,
               traffic_source="ncu dram__bytes_read.sum + dram__bytes_write.sum per launch"
               if mb is not None else None, avg_launch_ms=t * 1e3, launches=p["launches"],
               algorithmic_bytes_per_launch=p["bytes"] / max(1, p["launches"]),
               algorithmic_flops_per_launch=p["flops"] / max(1, p["launches"]))
    return out


def oracle_wave_rw12():
    """C, KE, Nu_in, Nu_out of the oracle's RW12 wave at L = 127, M_s = 12, N_r = 64
    (tests/golden/rw12_c3_oracle.txt, written by tests/golden/make_rw12_c3.py from the
    oracle alone)."""
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", "rw12_c3_oracle.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def newton_rw_measure(torch, RotatingShell, w, max_steps=40000, dt=2e-5):
    """Time-to-converged rotating wave at the workload's parameters (Table 1 row 3).

    The initial guess comes from time stepping an m = M_s seed (the route of
    Sec. 2.2) until the state stops changing relative to its drift; then
    Newton-GMRES (dt = 200, Sec. 3.3) is run from that guess on the FP64 path
    and on the mixed path, each autotuned first and timed end to end; the drift, kinetic
    energy and Nusselt numbers of both waves are compared with the oracle's wave.
    """
    M = w["Ms"]
    sh = RotatingShell(w["L"], w["Ms"], w["Nr"], w["Ek"], w["Ra"], w["Pr"], w["eta"],
                       precision="mixed")
    U = sh.conductive_state() + torch.tensor(
        si.mode_seed(w["L"], w["Ms"], w["Nr"], M, seed=4000, amp=1e-2), device="cuda")
    x = U.view(3, sh.P, w["Nr"], 2)
    pM = w["L"] + 1   # first pair of m = M (l = M)
    t0 = time.perf_counter()
    chunk = 500
    steps = 0
    prev_amp = None
    while steps < max_steps:
        sh.step(U, 0.0, dt, nsteps=chunk)
        steps += chunk
        amp = float(torch.linalg.norm(x[2, pM]).item())
        if prev_amp is not None and amp > 1e-3 and abs(amp - prev_amp) < 1e-3 * amp:
            break
        prev_amp = amp
    torch.cuda.synchronize()
    t_stepping = time.perf_counter() - t0
    a0 = x[2, pM].clone()
    sh.step(U, 0.0, dt, nsteps=10)
    a1 = x[2, pM]
    k = int(torch.argmax(a0[:, 0] ** 2 + a0[:, 1] ** 2).item())
    z0 = complex(a0[k, 0].item(), a0[k, 1].item())
    z1 = complex(a1[k, 0].item(), a1[k, 1].item())
    import cmath
    C0 = -cmath.phase(z1 / z0) / (M * 10 * dt)
    kstar = int(torch.argmax(torch.abs(x[2, pM, :, 0])).item())
    J = (((2 * sh.P + pM) * w["Nr"] + kstar) * 2 + 1)
    guess = U.clone()
    sh.close()
    out = {"time_stepping": {"steps": steps, "dt": dt, "seconds": t_stepping,
                             "precision": "mixed"}, "C0": C0, "phase_slot": J}
    ref = oracle_wave_rw12() if (w["L"], w["Ms"], w["Nr"]) == (127, 12, 64) else None
    for prec in ("fp64", "mixed"):
        s2 = RotatingShell(w["L"], w["Ms"], w["Nr"], w["Ek"], w["Ra"], w["Pr"], w["eta"],
                           precision=prec)
        s2.step(s2.new_state(), 0.0, 200.0, nsteps=1)   # factorise dt = 200 outside the timing
        s2.autotune()                                     # launch shapes, outside the timing
        Ur = guess.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        C, rep, st = s2.newton_rw(Ur, C0, J, tol=1e-10, max_newton=20, kmax=300,
                                  gmres_tol=1e-10, dt_newton=200.0)
        torch.cuda.synchronize()
        out[prec] = {"seconds": time.perf_counter() - t0, "status": st, "C": C,
                     "residual": rep["residual"], "newton_iterations": rep["iterations"],
                     "gmres_total": rep["gmres_total"], "gmres_per_newton": rep["gmres_history"],
                     "residual_history": rep["residual_history"]}
        ke, nu_in, nu_out = s2.diagnostics(Ur)
        out[prec].update(KE=ke, Nu_in=nu_in, Nu_out=nu_out)
        if ref:   # the oracle's wave at this truncation (drift, KE and Nu are phase-free)
            out[prec]["vs_oracle_wave"] = {
                k: abs(v - ref[k]) / abs(ref[k])
                for k, v in (("C", C), ("KE", ke), ("Nu_in", nu_in), ("Nu_out", nu_out))}
        out[prec + "_U"] = Ur
        s2.close()
    Uf, Um = out.pop("fp64_U"), out.pop("mixed_U")
    out["mixed_vs_fp64"] = {
        "drift_rel_diff": abs(out["mixed"]["C"] - out["fp64"]["C"]) / abs(out["fp64"]["C"]),
        "state_rel_diff": float((torch.linalg.norm(Um - Uf) / torch.linalg.norm(Uf)).item()),
        "speedup": out["fp64"]["seconds"] / out["mixed"]["seconds"]}
    out["paper_C_exact"] = 51.2817
    out["C_vs_paper_rel"] = abs(out["fp64"]["C"] - 51.2817) / 51.2817
    return out


def coriolis_study(torch, RotatingShell):
    """Sec. 5 comparison: Jacobian actions needed by Newton-GMRES for the same rotating wave
    with implicit Coriolis (the method) and explicit Coriolis (Eqs. expcor_e/f).

    Cases: RW4 at Ek = 1e-3, Ra = 120 (L = 31, N_r = 24) and the RW12 workload at Ek = 1e-5.
    Each case time-steps an m = M seed to the wave's basin, then solves with both schemes
    from the same guess (FP64 path, GMRES relative 1e-10, Newton 1e-10).
    """
    cases = [dict(name="RW4 Ek=1e-3 Ra=120 L=31 Nr=24", L=31, Ms=4, Nr=24, Ek=1e-3, Ra=120.0,
                  dt=2e-3, steps=2000),
             dict(name=WORKLOAD["name"], L=127, Ms=12, Nr=64, Ek=1e-5, Ra=140.0, dt=2e-5,
                  steps=8500)]
    out = []
    import cmath
    for c in cases:
        sh = RotatingShell(c["L"], c["Ms"], c["Nr"], c["Ek"], c["Ra"], precision="mixed")
        M = c["Ms"]
        U = sh.conductive_state() + torch.tensor(
            si.mode_seed(c["L"], c["Ms"], c["Nr"], M, seed=4000, amp=1e-2), device="cuda")
        sh.step(U, 0.0, c["dt"], nsteps=c["steps"])
        x = U.view(3, sh.P, c["Nr"], 2)
        pM = c["L"] + 1
        a0 = x[2, pM].clone()
        sh.step(U, 0.0, c["dt"], nsteps=10)
        a1 = x[2, pM]
        k = int(torch.argmax(a0[:, 0] ** 2 + a0[:, 1] ** 2).item())
        C0 = -cmath.phase(complex(a1[k, 0].item(), a1[k, 1].item()) /
                          complex(a0[k, 0].item(), a0[k, 1].item())) / (M * 10 * c["dt"])
        kstar = int(torch.argmax(torch.abs(x[2, pM, :, 0])).item())
        J = (((2 * sh.P + pM) * c["Nr"] + kstar) * 2 + 1)
        guess = U.clone()
        sh.close()
        row = {"case": c["name"]}
        for mode in ("implicit", "explicit"):
            s2 = RotatingShell(c["L"], c["Ms"], c["Nr"], c["Ek"], c["Ra"], coriolis=mode)
            Ur = guess.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            C, rep, st = s2.newton_rw(Ur, C0, J, tol=1e-10, max_newton=8, kmax=2048,
                                      gmres_tol=1e-10, dt_newton=200.0)
            torch.cuda.synchronize()
            row[mode] = {"status": st, "seconds": time.perf_counter() - t0, "C": C,
                         "newton_iterations": rep["iterations"], "jacobian_actions": rep["gmres_total"],
                         "gmres_per_newton": rep["gmres_history"], "residual": rep["residual"]}
            s2.close()
        row["actions_explicit_over_implicit"] = (row["explicit"]["jacobian_actions"] /
                                                 max(1, row["implicit"]["jacobian_actions"]))
        out.append(row)
    return out


def batch_measure(torch, Batch, count=16, reps=5):
    """Batched uneven instances: 32 continuation points at Ek = 3e-5 with azimuthal
    symmetries M_s = 4, 6, 8, 10, 12 (instance i has M_s = [4, 6, 8, 10, 12][i % 5], so 24, 16,
    12, 10 and 8 active m), L = 95, N_r = 48, Ra_i = linspace(1.05, 2.0, 32)_i x Ra_c(M_i),
    the linear onset of mode m = M_i at this truncation (seeded_inputs.ONSET_RA, from the
    oracle's linear analysis; the paper prints no onset values).
    16 Jacobian actions (Newton pseudo-step dt = 200) per instance per launch, all instances
    in one CUDA graph (rsc_batch_apply_jacobian), against the same actions issued instance
    by instance."""
    import numpy as np
    Ek = 3e-5
    ms_list = [4, 6, 8, 10, 12]
    inst = [dict(L=95, Ms=ms_list[i % 5], Nr=48, Ek=Ek,
                 Ra=float(f * si.ONSET_RA[f"C4_m{ms_list[i % 5]}"]), precision="mixed")
            for i, f in enumerate(np.linspace(1.05, 2.0, 32))]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    t0 = time.perf_counter()
    b = Batch(inst)
    t_create = time.perf_counter() - t0
    U, u, out, C, J = [], [], [], [], []
    for i, sh in enumerate(b.shells):
        d = inst[i]
        U.append(sh.conductive_state() + torch.tensor(
            si.perturbation(d["L"], d["Ms"], d["Nr"], seed=6000 + i), device="cuda"))
        u.append(torch.tensor(np.concatenate([si.random_vector(d["L"], d["Ms"], d["Nr"],
                                                               seed=7000 + 100 * i + q)
                                              for q in range(count)]), device="cuda"))
        out.append(torch.empty_like(u[-1]))
        C.append(0.0)
        J.append(None)
    t0 = time.perf_counter()
    tuning = b.autotune()
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    b.apply_jacobian(U, C, J, u, 200.0, out=out)     # factorisations and graph capture
    b.synchronize()
    t_first = time.perf_counter() - t0
    mem_gb = (free0 - torch.cuda.mem_get_info()[0]) / 1e9
    b.apply_jacobian(U, C, J, u, 200.0, out=out)
    b.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        b.apply_jacobian(U, C, J, u, 200.0, out=out)
    e1.record()
    torch.cuda.synchronize()
    t_graph = e0.elapsed_time(e1) / reps * 1e-3
    # the same actions instance by instance (each context's own per-action graph, on its own
    # stream; the device is synchronised after each instance so that they do not overlap)
    for i, sh in enumerate(b.shells):
        sh.apply_jacobian(U[i], 0.0, None, u[i], 200.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, sh in enumerate(b.shells):
        sh.apply_jacobian(U[i], 0.0, None, u[i], 200.0)
        torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    n_act = len(inst) * count
    b.close()
    return {"config": "32 instances, Ek=3e-5, L=95, Nr=48, Ms=[4,6,8,10,12][i%5], "
                      "Ra=linspace(1.05,2,32) x Ra_c(Ms) (linear onset of m = Ms), "
                      "16 actions each, mixed precision",
            "onset_Ra_by_Ms": {M: si.ONSET_RA[f"C4_m{M}"] for M in ms_list},
            "actions_per_launch": n_act, "graph_ms_per_launch": t_graph * 1e3,
            "jvps_per_s_batched": n_act / t_graph, "jvps_per_s_sequential": n_act / t_seq,
            "batching_speedup": t_seq / t_graph, "create_s": t_create, "autotune_s": t_tune,
            "tuning_by_Ms": {inst[i]["Ms"]: tuning[i] for i in range(5)},
            "first_launch_s_including_factorisation_and_capture": t_first,
            "device_memory_gb_after_first_launch": mem_gb,
            "factor_sets_per_dt": len(ms_list)}


def _wave_from_seed(torch, RotatingShell, c, precision="mixed", max_steps=60000):
    """Time-step an m = M seed (the route of Sec. 2.2) until the m = M temperature amplitude
    settles; return the state, the drift estimate from its phase rate and the phase slot J
    (Im T at l = m = M, k of the largest |Re T|)."""
    import cmath
    M = c["Ms"]
    sh = RotatingShell(c["L"], c["Ms"], c["Nr"], c["Ek"], c["Ra"], precision=precision)
    U = sh.conductive_state() + torch.tensor(
        si.mode_seed(c["L"], c["Ms"], c["Nr"], M, seed=4000, amp=1e-2), device="cuda")
    x = U.view(3, sh.P, c["Nr"], 2)
    pM = c["L"] + 1   # first pair of m = M (l = M)
    steps, prev, chunk = 0, None, 500
    while steps < max_steps:
        sh.step(U, 0.0, c["seed_dt"], nsteps=chunk)
        steps += chunk
        amp = float(torch.linalg.norm(x[2, pM]).item())
        if prev is not None and amp > 1e-3 and abs(amp - prev) < 1e-4 * amp:
            break
        prev = amp
    a0 = x[2, pM].clone()
    sh.step(U, 0.0, c["seed_dt"], nsteps=10)
    a1 = x[2, pM]
    k = int(torch.argmax(a0[:, 0] ** 2 + a0[:, 1] ** 2).item())
    C0 = -cmath.phase(complex(a1[k, 0].item(), a1[k, 1].item()) /
                      complex(a0[k, 0].item(), a0[k, 1].item())) / (M * 10 * c["seed_dt"])
    kstar = int(torch.argmax(torch.abs(x[2, pM, :, 0])).item())
    J = (((2 * sh.P + pM) * c["Nr"] + kstar) * 2 + 1)
    guess = U.clone()
    sh.close()
    return guess, C0, J, steps


def dt_study(torch, RotatingShell, rows=(0, 1, 2)):
    """Table 1 / Fig. 12 (Sec. 5): relative error of the drift speed obtained by second-order
    time stepping (rsc_step2) with implicit and with explicit Coriolis, against the exact
    speed from Newton's method, as a function of dt; the dt at which explicit time stepping
    diverges, and the largest dt whose implicit error stays below 2 %.

    Each wave is converged by Newton-GMRES (FP64, residual 1e-10) at the resolution of its
    Table 1 row; time stepping then starts from it in the laboratory frame, runs two wave
    periods (one for the explicit stability scan) to settle, and the speed is the
    least-squares slope of the unwrapped phase of the slot-J coefficient over the next two
    periods (one), C = -(d phase/dt)/M.  Transforms run in
    the mixed precision (their 1e-6 error is far below the errors measured here)."""
    import math
    import numpy as np
    table1 = [
        dict(name="RW4 Ek=1e-3 Ra=120 (Table 1 row 1), L=47, Nr=46", L=47, Ms=4, Nr=46,
             Ek=1e-3, Ra=120.0, seed_dt=2e-3, paper=dict(C=-2.7647, explicit_diverges=4.0e-4,
                                                          two_percent=1.1e-3),
             dts=dict(implicit=[2e-4, 5e-4, 1e-3, 2e-3, 3e-3, 5e-3, 8e-3],
                      explicit=[2e-4, 3e-4, 4e-4, 5e-4, 6e-4])),
        dict(name="RW8 Ek=1e-4 Ra=130 (Table 1 row 2), L=52, Nr=60", L=52, Ms=8, Nr=60,
             Ek=1e-4, Ra=130.0, seed_dt=2e-4, paper=dict(C=3.9998, explicit_diverges=2.0e-5,
                                                         two_percent=1.9e-4),
             dts=dict(implicit=[2e-5, 5e-5, 1e-4, 2e-4, 4e-4, 8e-4, 1.5e-3],
                      explicit=[1e-5, 1.5e-5, 2e-5, 2.5e-5, 3e-5])),
        dict(name="RW12 Ek=1e-5 Ra=140 (Table 1 row 3), L=89, Nr=76", L=89, Ms=12, Nr=76,
             Ek=1e-5, Ra=140.0, seed_dt=2e-5, paper=dict(C=51.2817, explicit_diverges=1.6e-6,
                                                         two_percent=2.8e-5),
             dts=dict(implicit=[2e-6, 6e-6, 1.2e-5, 2.4e-5, 5e-5, 1e-4, 2e-4, 4e-4, 8e-4],
                      explicit=[1e-6, 1.5e-6, 2e-6, 2.5e-6, 3e-6])),
    ]
    out = []
    for ri in rows:
        c = table1[ri]
        M = c["Ms"]
        t0 = time.perf_counter()
        guess, C0, J, seed_steps = _wave_from_seed(torch, RotatingShell, c)
        sN = RotatingShell(c["L"], c["Ms"], c["Nr"], c["Ek"], c["Ra"])
        Ustar = guess.clone()
        Cx, rep, st = sN.newton_rw(Ustar, C0, J, tol=1e-10, max_newton=20, kmax=600,
                                   gmres_tol=1e-10, dt_newton=200.0)
        sN.close()
        row = {"case": c["name"], "C_exact": Cx, "newton_status": st, "newton_residual": rep["residual"],
               "seed_steps": seed_steps, "paper": c["paper"]}
        period = 2.0 * math.pi / (M * abs(Cx))
        for mode in ("implicit", "explicit"):
            sh = RotatingShell(c["L"], c["Ms"], c["Nr"], c["Ek"], c["Ra"], precision="mixed",
                               coriolis=mode)
            pts = []
            # implicit: settle 2 periods, measure 2; explicit (stability): 1 and 1
            p_settle, p_meas = (2.0, 2.0) if mode == "implicit" else (1.0, 1.0)
            for dt in c["dts"][mode]:
                U = Ustar.clone()
                n0 = float(torch.linalg.norm(U).item())
                n_settle = max(1, int(math.ceil(p_settle * period / dt)))
                n_meas = max(32, int(math.ceil(p_meas * period / dt)))
                every = max(1, n_meas // int(64 * p_meas))
                sh.step2(U, dt, nsteps=n_settle)
                ts, ph, diverged = [], [], False
                for q in range(0, n_meas + 1, every):
                    if q:
                        sh.step2(U, dt, nsteps=every)
                    v = U[J - 1:J + 1].cpu().numpy()
                    nrm = float(torch.linalg.norm(U).item())
                    if not np.all(np.isfinite(v)) or not math.isfinite(nrm) or nrm > 1e3 * n0:
                        diverged = True
                        break
                    ts.append(q * dt)
                    ph.append(math.atan2(v[1], v[0]))
                if diverged:
                    pts.append({"dt": dt, "diverged": True})
                    continue
                slope = float(np.polyfit(np.array(ts), np.unwrap(np.array(ph)), 1)[0])
                Cdt = -slope / M
                pts.append({"dt": dt, "C_dt": Cdt, "rel_error": abs(Cdt - Cx) / abs(Cx),
                            "diverged": False})
            sh.close()
            row[mode] = pts
        ok = [p for p in row["explicit"] if p["diverged"]]
        row["explicit_diverges_at"] = min(p["dt"] for p in ok) if ok else None
        below = [p["dt"] for p in row["implicit"] if not p["diverged"] and p["rel_error"] < 0.02]
        row["implicit_largest_dt_below_2pct"] = max(below) if below else None
        if row["explicit_diverges_at"] and row["implicit_largest_dt_below_2pct"]:
            row["ratio"] = row["implicit_largest_dt_below_2pct"] / row["explicit_diverges_at"]
        row["seconds"] = time.perf_counter() - t0
        out.append(row)
        print(json.dumps({"dt_study_row": row}), flush=True)
    return out


def resolution_study(torch, RotatingShell):
    """Table 1 row 3 (RW12, Ek = 1e-5, Ra = 140) at several truncations: the wave is
    converged on the FP64 path at L = 127, N_r = 64 from a time-stepped m = 12 seed, then
    carried by zero-fill regridding (rsc_regrid) to every (L, N_r) of the grid and converged
    again by FP64 Newton-GMRES (residual 1e-10).  The drift C, kinetic energy and Nusselt
    numbers show whether C settles with resolution, and where the paper's resolution
    (N_r = 76, N_theta = 136: L = 89) sits."""
    w = dict(WORKLOAD)
    c = dict(L=127, Ms=12, Nr=64, Ek=w["Ek"], Ra=w["Ra"], seed_dt=2e-5)
    guess, C0, J, seed_steps = _wave_from_seed(torch, RotatingShell, c)
    base = RotatingShell(127, 12, 64, w["Ek"], w["Ra"])
    Ub = guess.clone()
    Cb, rep, st = base.newton_rw(Ub, C0, J, tol=1e-10, max_newton=20, kmax=600, gmres_tol=1e-10)
    out = {"seed_steps": seed_steps, "base": {"L": 127, "Nr": 64, "C": Cb, "status": st,
                                              "residual": rep["residual"]}, "points": []}
    grid = [(89, 64), (89, 76), (89, 96), (107, 76), (127, 64), (127, 76), (127, 96),
            (159, 64), (159, 76), (159, 96), (191, 96)]
    for L, Nr in grid:
        t0 = time.perf_counter()
        sh = RotatingShell(L, 12, Nr, w["Ek"], w["Ra"])
        U = sh.regrid_from(base, Ub)
        x = U.view(3, sh.P, Nr, 2)
        pM = L + 1
        kstar = int(torch.argmax(torch.abs(x[2, pM, :, 0])).item())
        Jt = sh.phase_slot(12, kstar)
        C, rep, st = sh.newton_rw(U, Cb, Jt, tol=1e-10, max_newton=20, kmax=600,
                                  gmres_tol=1e-10)
        ke, nui, nuo = sh.diagnostics(U)
        cheb, shs = sh.spectral_tail(U)
        row = {"L": L, "Nr": Nr, "C": C, "KE": ke, "Nu_in": nui, "Nu_out": nuo,
               "status": st, "residual": rep["residual"], "newton_iterations": rep["iterations"],
               "jacobian_actions": rep["gmres_total"], "cheb_tail": cheb, "sh_tail": shs,
               "seconds": time.perf_counter() - t0}
        out["points"].append(row)
        print(json.dumps({"resolution_point": row}), flush=True)
        sh.close()
    base.close()
    out["paper_C_exact"] = 51.2817
    return out


def c5_run(torch, RotatingShell, nsteps=1000, krylov=100, precisions=("mixed", "fp64"),
           wave=False, tuning=None, wave_krylov=1000):
    """The large single instance (Ek = 3e-6, Pr = 1, r_in/r_out = 0.35, L = 255, M_s = 8,
    N_r = 96, dt = 2e-6, Ra = 1.1 Ra_c of m = 8): from the m = 8 seed, `nsteps` IMEX Euler
    steps timed with CUDA events, then one Newton iteration (FP64 residual at dt = 200, GMRES
    with `krylov` Jacobian actions, update, FP64 residual) on the stepped state, for the
    mixed and the FP64 path, each autotuned; and the per-kernel time of one traced Newton
    iteration.  wave: the m = 8 rotating wave converged on the mixed path (time stepping at
    dt = 2e-5 from the seed until the m = 8 temperature amplitude settles, then Newton-GMRES
    to a residual of 1e-10 with GMRES of at most wave_krylov actions per Newton iteration),
    with the time of each part.  tuning: fixed launch shapes (JSON)
    instead of autotuning, so that a profiled run holds only the measured work."""
    c = si.config("C5")
    out = {"config": f"C5: Ek=3e-6, L=255, Ms=8, Nr=96, dt=2e-6, Ra={c['Ra']:.4f} "
                     f"(1.1 x onset of m = 8, {si.ONSET_RA['C5']:.4f})", "n": None}
    for prec in precisions:
        sh = RotatingShell(c["L"], 8, c["Nr"], c["Ek"], c["Ra"], precision=prec)
        if tuning:
            sh.set_tuning(json.loads(tuning))
            tun = sh.tuning()
        else:
            tun = sh.autotune()
        U = sh.conductive_state() + torch.tensor(
            si.mode_seed(c["L"], 8, c["Nr"], 8, seed=5000, amp=1e-2), device="cuda")
        sh.step(U, 0.0, c["dt"], nsteps=3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        sh.step(U, 0.0, c["dt"], nsteps=nsteps)
        e1.record()
        torch.cuda.synchronize()
        t_steps = e0.elapsed_time(e1) * 1e-3
        J = sh.phase_slot(8, 1)
        U1 = U.clone()
        sh.newton_rw(U1, 0.0, J, tol=0.0, max_newton=1, kmax=krylov, gmres_tol=0.0)  # warm-up
        U1 = U.clone()
        torch.cuda.synchronize()
        e0.record()
        _, rep, _ = sh.newton_rw(U1, 0.0, J, tol=0.0, max_newton=1, kmax=krylov, gmres_tol=0.0)
        e1.record()
        torch.cuda.synchronize()
        t_newton = e0.elapsed_time(e1) * 1e-3
        sh.profile(True)
        U1 = U.clone()
        sh.newton_rw(U1, 0.0, J, tol=0.0, max_newton=1, kmax=krylov, gmres_tol=0.0)
        prof = {k: round(v["ms"], 3) for k, v in sh.profile_report().items() if v["launches"]}
        sh.profile(False)
        ke, nui, nuo = sh.diagnostics(U)
        fac_s, fac_gpu = sh.factor_time()
        out["n"] = sh.n
        out[prec] = {"timesteps_per_s": nsteps / t_steps, "seconds_1000_steps": t_steps,
                     "newton_iteration_s": t_newton, "jvps_per_s": rep["gmres_total"] / t_newton,
                     "jacobian_actions": rep["gmres_total"], "residual_after": rep["residual"],
                     "KE_after_steps": ke, "kernel_ms_per_newton_iteration": prof,
                     "last_factorisation_s": fac_s, "factorisation_on_gpu": fac_gpu,
                     "tuning": tun}
        sh.close()
        print(json.dumps({"c5_" + prec: out[prec]}), flush=True)
    if wave:
        cw = dict(L=c["L"], Ms=8, Nr=c["Nr"], Ek=c["Ek"], Ra=c["Ra"], seed_dt=2e-5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        guess, C0, J, steps = _wave_from_seed(torch, RotatingShell, cw, "mixed", max_steps=150000)
        torch.cuda.synchronize()
        t_seed = time.perf_counter() - t0
        sh = RotatingShell(c["L"], 8, c["Nr"], c["Ek"], c["Ra"], precision="mixed")
        sh.autotune()
        U = guess.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        C, rep, st = sh.newton_rw(U, C0, J, tol=1e-10, max_newton=16, kmax=wave_krylov,
                                  gmres_tol=1e-10)
        torch.cuda.synchronize()
        t_newton = time.perf_counter() - t0
        ke, nui, nuo = sh.diagnostics(U)
        out["wave"] = {"seed_dt": 2e-5, "seed_steps": steps, "seed_s": t_seed, "C_seed": C0,
                       "newton_s": t_newton, "status": st, "C": C, "KE": ke, "Nu_in": nui,
                       "Nu_out": nuo, "newton_iterations": rep["iterations"],
                       "jacobian_actions": rep["gmres_total"], "residual": rep["residual"],
                       "residual_history": rep["residual_history"],
                       "gmres_per_newton": rep["gmres_history"], "krylov_cap": wave_krylov,
                       "time_to_wave_s": t_seed + t_newton}
        sh.close()
        print(json.dumps({"c5_wave": out["wave"]}), flush=True)
    if "mixed" in out and "fp64" in out:
        out["mixed_over_fp64"] = {
            "timesteps": out["mixed"]["timesteps_per_s"] / out["fp64"]["timesteps_per_s"],
            "jvps": out["mixed"]["jvps_per_s"] / out["fp64"]["jvps_per_s"]}
    return out


def _throughput(torch, RotatingShell, c, precision, krylov, nsteps):
    """Time steps/s (IMEX Euler, lab frame) and Jacobian actions/s (one Newton iteration with
    `krylov` actions) of one configuration, after autotuning; CUDA events, 2 warm-ups."""
    sh = RotatingShell(c["L"], c["Ms"], c["Nr"], c["Ek"], c["Ra"], precision=precision)
    sh.autotune()
    U0 = sh.conductive_state() + torch.tensor(
        si.perturbation(c["L"], c["Ms"], c["Nr"], seed=5000), device="cuda")
    U = U0.clone()
    sh.step(U, 0.0, c["dt"], nsteps=2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    sh.step(U, 0.0, c["dt"], nsteps=nsteps)
    e1.record()
    torch.cuda.synchronize()
    tps = nsteps / (e0.elapsed_time(e1) * 1e-3)
    J = sh.phase_slot(c["Ms"], 1)
    for rep in range(3):
        U = U0.clone()
        torch.cuda.synchronize()
        e0.record()
        _, r, _ = sh.newton_rw(U, 0.5, J, tol=0.0, max_newton=1, kmax=krylov, gmres_tol=0.0)
        e1.record()
        torch.cuda.synchronize()
    jvps = r["gmres_total"] / (e0.elapsed_time(e1) * 1e-3)
    sh.close()
    return {"timesteps_per_s": tps, "jvps_per_s": jvps, "krylov": krylov, "n": sh.n}


def configs_study(torch, RotatingShell, Batch):
    """The other configurations: throughput at C1 (L = 31), C2 (L = 63) and C5 (L = 255,
    N_r = 96), FP64 and mixed; the C2 rotating wave (RW8, Ek = 1e-4, Ra = 130) solved by
    Newton on both paths with the mixed path's errors in drift, kinetic energy and Nusselt
    numbers against the FP64 solution; and the mixed batched Newton (rsc_batch_newton_rw) on
    four RW4 continuation points against FP64 single solves."""
    out = {"throughput": []}
    for name in ("C1", "C2", "C5"):
        c = si.config(name)
        c.update(Ms={"C1": 4, "C2": 8, "C5": 8}[name])
        row = {"config": name, "L": c["L"], "Ms": c["Ms"], "Nr": c["Nr"]}
        for prec in ("fp64", "mixed"):
            row[prec] = _throughput(torch, RotatingShell, c, prec,
                                    krylov=100, nsteps=200 if name != "C5" else 50)
        out["throughput"].append(row)
        print(json.dumps({"configs_row": row}), flush=True)
    # C2 rotating wave: FP64 vs mixed Newton from the same time-stepped guess
    c = dict(si.config("C2"), Ms=8, seed_dt=2e-4)
    guess, C0, J, seed_steps = _wave_from_seed(torch, RotatingShell, c)
    rw = {"config": "C2 RW8 Ek=1e-4 Ra=130 L=63 Nr=48", "seed_steps": seed_steps}
    states = {}
    for prec in ("fp64", "mixed"):
        sh = RotatingShell(c["L"], c["Ms"], c["Nr"], c["Ek"], c["Ra"], precision=prec)
        sh.autotune()
        sh.step(sh.new_state(), 0.0, 200.0, nsteps=1)
        U = guess.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Cx, rep, st = sh.newton_rw(U, C0, J, tol=1e-10, max_newton=20, kmax=400,
                                   gmres_tol=1e-10, dt_newton=200.0)
        torch.cuda.synchronize()
        ke, nui, nuo = sh.diagnostics(U)
        rw[prec] = {"seconds": time.perf_counter() - t0, "status": st, "C": Cx, "KE": ke,
                    "Nu_in": nui, "Nu_out": nuo, "residual": rep["residual"],
                    "newton_iterations": rep["iterations"], "jacobian_actions": rep["gmres_total"]}
        states[prec] = U
        sh.close()
    f, m = rw["fp64"], rw["mixed"]
    rw["mixed_vs_fp64"] = {
        "drift_rel": abs(m["C"] - f["C"]) / abs(f["C"]), "KE_rel": abs(m["KE"] - f["KE"]) / f["KE"],
        "Nu_in_rel": abs(m["Nu_in"] - f["Nu_in"]) / f["Nu_in"],
        "Nu_out_rel": abs(m["Nu_out"] - f["Nu_out"]) / f["Nu_out"],
        "state_rel": float((torch.linalg.norm(states["mixed"] - states["fp64"]) /
                            torch.linalg.norm(states["fp64"])).item()),
        "speedup": f["seconds"] / m["seconds"]}
    rw["paper_C_exact"] = 3.9998
    out["rw_C2"] = rw
    print(json.dumps({"rw_C2": rw}), flush=True)
    # mixed batched Newton on four RW4 continuation points
    c = dict(si.config("C1"), Ms=4, seed_dt=2e-3)
    guess, C0, J, _ = _wave_from_seed(torch, RotatingShell, c)
    Ras = [120.0, 121.0, 122.0, 123.0]
    b = Batch([dict(L=c["L"], Ms=4, Nr=c["Nr"], Ek=c["Ek"], Ra=Ra, precision="mixed") for Ra in Ras])
    b.autotune()
    Ub = [guess.clone() for _ in Ras]
    t0 = time.perf_counter()
    Cb, reps, sts = b.newton_rw(Ub, [C0] * 4, [J] * 4, tol=1e-10, max_newton=12, kmax=300)
    b.synchronize()
    t_batch = time.perf_counter() - t0
    b.close()
    bat = {"config": "4 RW4 points, Ek=1e-3, L=31, Nr=24, Ra=120..123, mixed, concurrent",
           "seconds": t_batch, "status": sts, "residuals": [r["residual"] for r in reps]}
    drift_rel = []
    for i, Ra in enumerate(Ras):
        sh = RotatingShell(c["L"], 4, c["Nr"], c["Ek"], Ra, precision="fp64")
        U = guess.clone()
        Cf, rep, st = sh.newton_rw(U, C0, J, tol=1e-10, max_newton=12, kmax=300)
        drift_rel.append(abs(Cb[i] - Cf) / abs(Cf))
        sh.close()
    bat["drift_rel_vs_fp64"] = drift_rel
    out["batch_mixed_newton"] = bat
    print(json.dumps({"batch_mixed_newton": bat}), flush=True)
    return out


def replica_throughput(torch, dist, units, seconds, device):
    """Whole-job throughput of independent replicas: the units every rank processed, summed,
    over the slowest rank's time (seconds).  dist = None on a single rank.  The two
    reductions run on tensors on `device` (the rank's GPU under NCCL, the CPU under gloo)."""
    if dist is None:
        return units / seconds, units, seconds
    u = torch.tensor([float(units)], device=device, dtype=torch.float64)
    t = torch.tensor([float(seconds)], device=device, dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()) / float(t.item()), float(u.item()), float(t.item())


def run_gpu(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    __graft_entry__.build()
    from paper_2508_16635_gb300 import RotatingShell
    from paper_2508_16635_gb300.rsc import KERNELS

    w = WORKLOAD
    if args.dt_study is not None:
        if rank == 0:
            rows = tuple(int(r) for r in args.dt_study.split(","))
            print(json.dumps({"dt_study": dt_study(torch, RotatingShell, rows)}), flush=True)
        return 0
    if args.configs_study:
        if rank == 0:
            from paper_2508_16635_gb300 import Batch
            print(json.dumps({"configs_study": configs_study(torch, RotatingShell, Batch)}),
                  flush=True)
        return 0
    if args.coriolis_study:
        if rank == 0:
            print(json.dumps({"coriolis_study": coriolis_study(torch, RotatingShell)}), flush=True)
        return 0
    if args.c5:
        if rank == 0:
            precs = ("mixed", "fp64") if args.c5_precision == "both" else (args.c5_precision,)
            print(json.dumps({"c5": c5_run(torch, RotatingShell, args.c5_steps, args.c5_krylov,
                                           precs, wave=args.c5_wave, tuning=args.tuning,
                                           wave_krylov=args.c5_wave_krylov)}),
                  flush=True)
        return 0
    if args.implicit_solves:
        if rank == 0:
            sh = RotatingShell(w["L"], w["Ms"], w["Nr"], w["Ek"], w["Ra"], w["Pr"], w["eta"],
                               precision=args.precision)
            if args.tuning:
                sh.set_tuning(json.loads(args.tuning))
            b = torch.tensor(si.random_vector(w["L"], w["Ms"], w["Nr"], seed=3003), device="cuda")
            for _ in range(args.implicit_solves):
                x = sh.implicit_solve(b, 200.0)
            torch.cuda.synchronize()
            print(json.dumps({"implicit_solves": args.implicit_solves, "tuning": sh.tuning(),
                              "norm": float(torch.linalg.norm(x).item())}), flush=True)
            sh.close()
        return 0
    if args.resolution_study:
        if rank == 0:
            print(json.dumps({"resolution_study": resolution_study(torch, RotatingShell)}),
                  flush=True)
        return 0
    peaks = measured_peaks(torch)
    sh = RotatingShell(w["L"], w["Ms"], w["Nr"], w["Ek"], w["Ra"], w["Pr"], w["eta"],
                       precision=args.precision)
    if args.tuning:             # fixed shapes (a profiler distorts the autotuner's timings)
        sh.set_tuning(json.loads(args.tuning))
        tuning = sh.tuning()
    else:
        tuning = sh.autotune()  # launch shapes picked by timing, before any measurement
        if args.precision == "mixed" and args.chain_parts > 1:
            # partitioned chains for the double-float solve (factorised in the warm-up)
            sh.set_tuning(dict(tuning, chain_parts=args.chain_parts))
            tuning = sh.tuning()
    U0 = sh.conductive_state() + torch.tensor(
        si.perturbation(w["L"], w["Ms"], w["Nr"], seed=3000 + rank), device="cuda")
    # phase slot: Im of the T coefficient (l = m = 12, k*) with k* = argmax |Re|
    x = U0.view(3, sh.P, w["Nr"], 2)
    p12 = (w["L"] + 1)  # first pair of m = 12
    kstar = int(torch.argmax(torch.abs(x[2, p12, :, 0])).item())
    J = (((2 * sh.P + p12) * w["Nr"] + kstar) * 2 + 1)
    U = U0.clone()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    K = args.krylov

    def one_step():
        return sh.newton_rw(U, 0.5, J, tol=0.0, max_newton=1, kmax=K, gmres_tol=0.0)

    for _ in range(args.warmup):
        U.copy_(U0)
        one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = sh.launch_count()
    gmres_total = 0
    sh.profile(False)     # timed region: Jacobian actions replay their CUDA graph
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            U.copy_(U0)
            flush.zero_()
            ev[i][0].record()
            _, rep, _ = one_step()
            ev[i][1].record()
            gmres_total += rep["gmres_total"]
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    launches = sh.launch_count() - launches0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    # JVPs per second of all ranks: the actions every rank ran over the slowest rank's time
    value, _, slowest_s = replica_throughput(torch, dist, gmres_total / args.steps, ms * 1e-3,
                                             torch.device("cuda", local))
    ms = slowest_s * 1e3
    # traced passes over the same iteration (individual launches, CUDA events on the
    # context stream): one with every kernel for the breakdown, then one timing only
    # the dominant kernel for the roofline
    sh.profile(True)
    U.copy_(U0)
    flush.zero_()
    one_step()
    prof_all = sh.profile_report()
    dom = max(prof_all, key=lambda k: prof_all[k]["ms"])
    sh.profile(True, kernels=[dom])
    for i in range(args.steps):
        U.copy_(U0)
        flush.zero_()
        one_step()
    prof = sh.profile_report()
    sh.profile(False)
    jvps_per_step = gmres_total / args.steps

    # per-kernel cost of one Jacobian action and of one FP64 residual step
    ub = torch.tensor(si.random_vector(w["L"], w["Ms"], w["Nr"], seed=3002), device="cuda")
    ubatch = ub.repeat(10)
    outb = torch.empty_like(ubatch)
    sh.apply_jacobian(U0, 0.5, J, ubatch, 200.0, out=outb)
    sh.profile(True)
    sh.apply_jacobian(U0, 0.5, J, ubatch, 200.0, out=outb)
    prof_jvp = {k: round(v["ms"] / 10, 5) for k, v in sh.profile_report().items() if v["launches"]}
    sh.profile(False)
    shf = RotatingShell(w["L"], w["Ms"], w["Nr"], w["Ek"], w["Ra"], w["Pr"], w["eta"])
    Uf = U0.clone()
    shf.step(Uf, 0.5, 200.0)
    shf.profile(True)
    shf.step(Uf, 0.5, 200.0, nsteps=2)
    prof_step64 = {k: round(v["ms"] / 2, 5) for k, v in shf.profile_report().items() if v["launches"]}
    shf.close()

    # plain time stepping (timesteps/s) on the same workload
    Us = U0.clone()
    sh.step(Us, 0.0, 5e-6, nsteps=3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sh.step(Us, 0.0, 5e-6, nsteps=20)
    e1.record()
    torch.cuda.synchronize()
    steps_per_s = 20 / (e0.elapsed_time(e1) * 1e-3)

    # end to end through the C ABI with host buffers (copies inside the call)
    import numpy as np
    host = np.ascontiguousarray(U0.cpu().numpy())
    e2e_times = []
    for i in range(max(2, min(3, args.steps))):
        h = host.copy()
        t0 = time.perf_counter()
        _, rep2, _ = sh.newton_rw_host(h, 0.5, J, tol=0.0, max_newton=1, kmax=K, gmres_tol=0.0)
        e2e_times.append((time.perf_counter() - t0, rep2["gmres_total"]))
    e2e_v, _, e2e_t = replica_throughput(torch, dist, sum(g for _, g in e2e_times) / len(e2e_times),
                                         sum(t for t, _ in e2e_times) / len(e2e_times),
                                         torch.device("cuda", local))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": dtype_label(args.precision, tuning),
            "data": "synthetic (seeded perturbation of the conductive state)",
            "config": {"workload": w["name"], "precision": args.precision,
                       "onset_Ra": si.ONSET_RA["C3"],
                       "Ra_over_onset": w["Ra"] / si.ONSET_RA["C3"],
                       "step": f"1 Newton iteration: FP64 residual, GMRES with {K} Jacobian "
                               f"actions (one-reduction MGS), update, FP64 residual",
                       "krylov_per_iteration": K, "parallelism": f"replicas x{world}",
                       "l2": "flushed between steps (256 MB write, outside the timed interval)"},
            "timesteps_per_s": steps_per_s,
            "jvps_per_step": jvps_per_step,
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": 8 * sh.n,
                    "d2h_bytes_per_step": 8 * sh.n, "ms_per_step": e2e_t * 1e3},
            "gpu_launches": int(launches),
            "tuning": tuning,
            "kernel_ms_per_step": {k: round(v["ms"], 4) for k, v in prof_all.items()},
            "kernel_ms_per_jacobian_action": prof_jvp,
            "kernel_ms_per_fp64_step": prof_step64,
            "roofline": roofline(prof, peaks, args.precision, tuning),
            "peaks": {k: v for k, v in peaks.items()},
            "clocks": clk.summary(),
            "wall_s_timed_region": wall,
        }
        if not args.no_fp64_arm:
            line["factorisation"] = factor_timing(torch, RotatingShell, w)
        if args.precision == "mixed" and not args.no_fp64_arm:
            line["fp64_path"] = fp64_arm(torch, RotatingShell, w, K)
            line["mixed_over_fp64_jvps"] = value / world / line["fp64_path"]["jvps_per_s"]
        if not args.no_rw:
            line["newton_rw"] = newton_rw_measure(torch, RotatingShell, w)
        if not args.no_batch:
            from paper_2508_16635_gb300 import Batch
            line["batch"] = batch_measure(torch, Batch)
        if not args.no_baseline:
            line["cpu_baseline"] = cpu_oracle_sample(K)
        print(json.dumps(line), flush=True)
    sh.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
