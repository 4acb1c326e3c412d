"""Host logic of bench.py's roofline entry (no GPU): which kernels count as double-float,
which bound a kernel is reported against, and which ncu traffic figure applies."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6800.0, "hbm_source": "measured", "fp64_tflops": 1.1, "fp32_tflops": 70.0}


def prof_of(name, ms, launches, nbytes, flops):
    return {name: {"ms": ms, "launches": launches, "bytes": nbytes * launches,
                   "flops": flops * launches}}


def test_double_float_kernels_follow_the_tuning():
    t = {"chain_df": 4, "krylov_split": 1}
    assert bench.double_float_kernels("mixed", t) == {"chain_sweep", "chain_gemv", "chain_reduced",
                                                       "gmres_dots", "gmres_axpy"}
    # the FP64 path never runs the double-float chain solve; its GMRES may use the split basis
    assert bench.double_float_kernels("fp64", t) == {"gmres_dots", "gmres_axpy"}
    assert bench.double_float_kernels("mixed", {"chain_df": 0, "krylov_split": 0}) == set()


def test_double_float_sweeps_are_reported_against_hbm_with_their_traffic():
    # 101.1 MB per launch in 68.5 us: 1.476 TB/s
    prof = prof_of("chain_sweep", 0.0685 * 100, 100, 101.1e6, 49e6)
    r = bench.roofline(prof, PEAKS, "mixed", {"chain_df": 4, "krylov_split": 1})
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(101.1e6 / 68.5e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0)
    assert r["traffic"] == pytest.approx(101.5e6)          # the double-float capture
    assert r["arithmetic"].startswith("double-float")


def test_reduced_chain_sweeps_take_their_own_capture():
    # the sweeps over the odd-even reduced chains read half the blocks: 51.5 MB in 40.4 us
    prof = prof_of("chain_sweep", 0.0404 * 100, 100, 51.5e6, 25e6)
    r = bench.roofline(prof, PEAKS, "mixed", {"chain_df": 4, "krylov_split": 1, "chain_cr": 1})
    assert r["bound"] == "hbm" and r["traffic"] == pytest.approx(57.7e6)
    assert r["frac"] == pytest.approx(51.5e6 / 40.4e-6 / 1e9 / 6800.0)
    prof = prof_of("chain_reduced", 0.025 * 30, 30, 52e6, 33e6)
    r = bench.roofline(prof, PEAKS, "mixed", {"chain_df": 4, "krylov_split": 1, "chain_cr": 1})
    assert r["arithmetic"].startswith("double-float") and r["traffic"] == pytest.approx(52.1e6)


def test_fp64_sweeps_keep_the_fp64_bound_and_their_own_traffic():
    # 49 MFLOP in 117 us is 0.42 TFLOP/s (38 % of FP64), 0.86 TB/s (13 % of HBM): ALU-bound
    prof = prof_of("chain_sweep", 0.117 * 10, 10, 101.1e6, 49e6)
    r = bench.roofline(prof, PEAKS, "mixed", {"chain_df": 0, "krylov_split": 1})
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == 1.1 and r["arithmetic"] == "FP64"
    assert r["frac"] == pytest.approx(49e6 / 117e-6 / 1e12 / 1.1)
    assert r["traffic"] == pytest.approx(101.3e6)          # the FP64 capture


def test_a_kernel_without_a_capture_reports_no_traffic():
    prof = prof_of("fft_products", 0.05, 1, 30e6, 0.3e9)
    r = bench.roofline(prof, PEAKS, "mixed", {"chain_df": 4, "krylov_split": 1})
    assert r["traffic"] is None and r["traffic_source"] is None
    assert r["arithmetic"] == "FP32" and r["peak"] in (70.0, 6800.0)


def test_dtype_label_says_what_ran():
    assert bench.dtype_label("fp64", {"chain_df": 4, "krylov_split": 1}) == "f64"
    lab = bench.dtype_label("mixed", {"chain_df": 2, "krylov_split": 1})
    assert "double-float e/f chain solve" in lab and "double-float Krylov basis" in lab
    lab = bench.dtype_label("mixed", {"chain_df": 0, "krylov_split": 0})
    assert "f64 e/f chain solve" in lab and "f64 Krylov basis" in lab


def _replica_rank(rank, world, port, out):
    """One gloo rank on the CPU: rank r ran r + 1 units in 0.5 + r seconds."""
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        v, units, secs = bench.replica_throughput(torch, dist, rank + 1, 0.5 + rank,
                                                  torch.device("cpu"))
        out[rank] = (v, units, secs)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_throughput_sums_units_over_the_slowest_rank():
    """bench.py with N > 1: the whole-job value is the units of all ranks over the slowest
    rank's time (world_size 2 over gloo on the CPU); a single rank reduces to units / time."""
    import socket
    import torch
    import torch.multiprocessing as mp
    assert bench.replica_throughput(torch, None, 200, 0.08, None) == (2500.0, 200, 0.08)
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_replica_rank, args=(2, port, out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    for r in (0, 1):
        v, units, secs = res[r]
        assert units == 3.0 and secs == 1.5
        assert v == pytest.approx(2.0)
