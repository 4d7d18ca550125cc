#!/usr/bin/env python3
"""Benchmark of the all-at-once heat solve with the block epsilon-circulant
preconditioner on GB300.

Workload: 2D heat equation on the unit square, 255 x 255 interior grid,
T = 1, N = 256 backward-Euler steps (16,646,400 space-time unknowns),
eps = sqrt(tau) = 1/16, seeded U[-1,1] source and an 8 x 8 random sine-series
u0.  One step = one solve of L u = f to RES = ||f - L u|| / ||f|| <= 1e-8 by
right-preconditioned GMRES(30) with the FP64 sine-transform P_eps^{-1}, f
resident on the device.  Metric: space-time unknowns per second.

`--form fp32` times the mixed-precision form (FP32 P_eps^{-1} in FP64 FGMRES)
on the same workload instead.

Run: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run; every rank solves its own copy
of the workload (independent problems, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

M_SIDE = 255
N_STEPS = 256
EPS = 1.0 / 16.0                     # sqrt(tau)
RTOL = 1e-8
RESTART = 30
METRIC = "space-time unknowns/s solved to 1e-8 rel. residual"
UNIT = "unknowns/s"

# Algorithmic work per space-time unknown of each kernel at this workload
# (n = 256 sine-transform length, N = 256 time steps).  A DST-I pass counts a
# real FFT of length 2n: 2.5 log2(2n) flops; the time pass a real FFT and its
# inverse plus the divide and scalings: 2 x 2.5 log2 N + 8; the stencil 7
# flops.  Bytes are one read and one write of the vector in the kernel's
# storage type.
LOG2N = math.log2(M_SIDE + 1)
LOG2T = math.log2(N_STEPS)
ALGO = {
    "dst_rows_kernel": {"flops": 2.5 * (LOG2N + 1)},
    "dst_cols_kernel": {"flops": 2.5 * (LOG2N + 1)},
    "time_pass_kernel": {"flops": 5.0 * LOG2T + 8.0},
    "apply_L_kernel": {"flops": 7.0},
}
BYTES_PER_UNIT = {"fp64": {"dst_rows_kernel": 16.0, "dst_cols_kernel": 16.0, "time_pass_kernel": 16.0,
                           "apply_L_kernel": 16.0},
                  "fp32": {"dst_rows_kernel": 12.0, "dst_cols_kernel": 8.0, "time_pass_kernel": 8.0,
                           "apply_L_kernel": 16.0}}
# FP64 FMA peak of GB300 from unit counts: 2 FP64 FMA / clock / SM x 152 SMs x
# 2.07 GHz x 2 flops = 1.26 TFLOP/s (a throughput probe measured 1.20 TFLOP/s
# at 1.99 GHz).  FP32: 128 lanes / SM -> 80.5 TFLOP/s.
FP64_PEAK_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12
# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture
# of each kernel at this workload (see profiles/); None = not captured for the
# current build of the kernel.
NCU_TRAFFIC = {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--form", choices=("fp64", "fp32"), default="fp64",
                    help="preconditioner arithmetic of the headline number")
    ap.add_argument("--no-other-form", action="store_true",
                    help="skip measuring the other preconditioner form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-case", choices=("pinv_fp64", "pinv_fp32", "solve_fp32"), default=None,
                    help="run a small bounded case for an ncu capture and exit (no JSON line)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "of measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "of fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(form: str):
    return {
        "workload": f"heat2d {M_SIDE}x{M_SIDE} interior grid, N={N_STEPS} backward-Euler steps, T=1, "
                    f"eps=sqrt(tau)=1/16, {'FP64' if form == 'fp64' else 'FP32'} sine-transform "
                    f"P_eps^-1, right-preconditioned FGMRES"
                    f"({RESTART}), stop at ||f-Lu||/||f|| <= 1e-8",
        "unknowns": M_SIDE * M_SIDE * N_STEPS,
        "grid": [M_SIDE, M_SIDE],
        "N": N_STEPS,
        "eps": EPS,
        "preconditioner": form,
        "l2": "inputs larger than L2: each vector is 133 MB > 129 MB L2, Krylov basis 4 GB",
    }


def cpu_baseline_sample(case):
    """The oracle's solver for u (sequential backward-Euler stepping, the
    definition of the all-at-once solution) timed on the full workload."""
    import numpy as np
    import scipy.sparse as sp

    import oracle as O
    K = O.fd_stiffness(2, case.m)
    M = sp.identity(K.shape[0], format="csr")
    f = O.build_rhs(case.u0, case.fsrc, case.tau)
    t0 = time.perf_counter()
    O.timestep_solve(f, M, K, case.tau)
    dt = time.perf_counter() - t0
    return {"value": case.U / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one full solve of the workload ({case.U} unknowns) by the oracle's "
                      f"sequential backward-Euler stepping (one sparse LU, SuperLU, single thread): "
                      f"{dt:.2f} s",
            "host_cores": os.cpu_count(), "cpu": platform.processor() or platform.machine()}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import numpy as np
    import scipy.sparse as sp

    import oracle as O
    from workloads import heat_case_2d
    case = heat_case_2d(seed=2, m=M_SIDE, N=N_STEPS, eps=EPS)
    K = O.fd_stiffness(2, case.m)
    M = sp.identity(K.shape[0], format="csr")
    f = O.build_rhs(case.u0, case.fsrc, case.tau)
    ns = 64                                            # slices per step: a bounded sample
    sample = f[:ns]
    for _ in range(args.warmup):
        O.timestep_solve(sample, M, K, case.tau)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.timestep_solve(sample, M, K, case.tau)
    dt = (time.perf_counter() - t0) / args.steps
    value = ns * case.J / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded U[-1,1] source, 8x8 random sine-series u0)",
        "config": workload_config("fp64"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"first {ns} of {N_STEPS} time slices per step, solved by the "
                                   f"oracle's sequential backward-Euler stepping (SuperLU, one thread)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_form(form, case, args, ws, local, dist):
    """Time K solves of the workload with one preconditioner form.  Returns the
    per-step time (max over ranks), the live per-kernel event times, the
    launch count, the clocks seen and the host-buffer (end-to-end) time."""
    import torch
    from paper_2002_01108_gb300 import Problem

    # Z is stored in both forms: with a fixed preconditioner FGMRES gives the
    # same iterates as right-preconditioned GMRES and saves the final apply.
    prob = Problem(2, M_SIDE, N_STEPS, precision=form, max_restart=RESTART, flexible=True,
                   host_io=True)
    prob.set_eps(EPS)
    f = prob.build_rhs(torch.from_numpy(case.u0).cuda(), torch.from_numpy(case.fsrc).cuda())
    u = torch.empty_like(f)
    solve_kw = dict(restart=RESTART, rtol=RTOL, maxit=1000, flexible=True)
    for _ in range(args.warmup):
        prob.gmres_solve(f, u, **solve_kw)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    launches0 = prob.launches
    prob.profile_start(1 << 16)
    stream = prob.stream
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = []
    for _ in range(args.steps):
        _, info = prob.gmres_solve(f, u, **solve_kw)
        infos.append(info)
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms_step = ev0.elapsed_time(ev1) / args.steps
    kernels = prob.profile_stop()
    launches = prob.launches - launches0
    clocks = sampler.stop()
    if ws > 1:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())

    # end to end through the host-buffer entry point: H2D of f, solve, D2H of u
    f_host = f.cpu().pin_memory()
    u_host = torch.empty_like(f_host).pin_memory()
    prob.gmres_solve_host(f_host, u_host, **solve_kw)
    e2e = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        prob.gmres_solve_host(f_host, u_host, **solve_kw)
        e2e.append(time.perf_counter() - t0)
    e2e_s = sum(e2e) / len(e2e)
    if ws > 1:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    U = prob.U
    prob.close()
    return {"U": U, "ms_step": ms_step, "kernels": kernels, "launches": launches,
            "clocks": clocks, "info": infos[-1], "e2e_s": e2e_s,
            "e2e_samples_ms": [round(x * 1e3, 3) for x in e2e]}


def roofline(form, kernels, U):
    dom = max(kernels.items(), key=lambda kv: kv[1][1])[0]
    dom_n, dom_ms = kernels[dom]
    avg_ms = dom_ms / max(dom_n, 1)
    peaks, peak_src = measured_peaks()
    if form == "fp64" and dom in ALGO:
        achieved = ALGO[dom]["flops"] * U / (avg_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "FP64 FMA units x clock (2/clk/SM x 152 SMs x 2.07 GHz)",
                "algorithmic_per_unit": f"{ALGO[dom]['flops']:.1f} flop", "units_per_launch": U}
    else:
        bpu = BYTES_PER_UNIT[form].get(dom, 16.0)
        achieved = bpu * U / (avg_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "peak_source": peak_src,
                "algorithmic_per_unit": f"{bpu:.0f} B", "units_per_launch": U}
    roof["avg_launch_ms"] = avg_ms
    roof["traffic"] = NCU_TRAFFIC.get((dom, form))
    return roof


def kernel_table(kernels):
    total_ms = sum(ms for _, ms in kernels.values())
    return {name: {"launches": n, "ms": round(ms, 4),
                   "share": round(ms / total_ms, 4) if total_ms else None}
            for name, (n, ms) in sorted(kernels.items(), key=lambda kv: -kv[1][1])}


def run_gpu(args):
    import torch

    ws, rank, local = dist_setup()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2002_01108_gb300 import build as bec_build
    if rank == 0:
        bec_build.build()
    if ws > 1:
        dist.barrier()
    from workloads import heat_case_2d

    case = heat_case_2d(seed=2, m=M_SIDE, N=N_STEPS, eps=EPS)
    form = args.form
    r = measure_form(form, case, args, ws, local, dist)
    U = r["U"]
    line = {
        "metric": METRIC, "value": ws * U / (r["ms_step"] / 1e3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded U[-1,1] source, 8x8 random sine-series u0)",
        "config": dict(workload_config(form), iterations=r["info"]["iters"],
                       true_relres=r["info"]["true_relres"],
                       parallelism=f"{ws} independent replicas"),
        "roofline": roofline(form, r["kernels"], U),
        "e2e": {"value": ws * U / r["e2e_s"], "unit": UNIT, "h2d_bytes_per_step": U * 8,
                "d2h_bytes_per_step": U * 8, "ms_per_step": r["e2e_s"] * 1e3,
                "samples_ms": r["e2e_samples_ms"]},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "kernels": kernel_table(r["kernels"]),
        "paper_context": "Table table1 (N=256, 255^2, Q1, a=1e-5): 12.54 s MATLAB on 2x Xeon E5-2690 v4 "
                         "= 1.33e6 unknowns/s (different discretisation and tolerance)",
    }
    if not args.no_other_form:
        other = "fp32" if form == "fp64" else "fp64"
        o = measure_form(other, case, args, ws, local, dist)
        line["forms"] = {other + "_preconditioner": {
            "value": ws * U / (o["ms_step"] / 1e3), "unit": UNIT, "ms_per_step": o["ms_step"],
            "iterations": o["info"]["iters"], "true_relres": o["info"]["true_relres"],
            "e2e_value": ws * U / o["e2e_s"], "gpu_launches": o["launches"], "clocks": o["clocks"],
            "roofline": roofline(other, o["kernels"], U), "kernels": kernel_table(o["kernels"]),
            "note": "same workload and tolerance; FP32/complex64 P_eps^-1 inside FP64 FGMRES"
                    if other == "fp32" else "same workload; plain FP64 form"}}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(case)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_ncu_case(which: str):
    """A bounded workload for profiler captures: the benchmark problem with a
    two-vector Krylov basis (under 1 GB on the device), three P_eps^{-1}
    applies and two stencil applies, or one short FGMRES solve."""
    import torch
    torch.cuda.set_device(0)
    from paper_2002_01108_gb300 import Problem
    from paper_2002_01108_gb300 import build as bec_build
    from workloads import heat_case_2d
    bec_build.build()
    case = heat_case_2d(seed=2, m=M_SIDE, N=N_STEPS, eps=EPS)
    form = "fp64" if which == "pinv_fp64" else "fp32"
    with Problem(2, M_SIDE, N_STEPS, precision=form, max_restart=2, flexible=form == "fp32") as p:
        p.set_eps(EPS)
        f = p.build_rhs(torch.from_numpy(case.u0).cuda(), torch.from_numpy(case.fsrc).cuda())
        if which == "solve_fp32":
            p.gmres_solve(f, restart=2, maxit=2, rtol=RTOL, flexible=True)
        else:
            z = torch.empty_like(f)
            for _ in range(3):
                p.apply_Pinv(f, z)
            y = torch.empty_like(f)
            for _ in range(2):
                p.apply_A(z, y)
        torch.cuda.synchronize()
    print(f"ncu case {which} done")
    return 0


def main():
    args = parse()
    if args.ncu_case:
        return run_ncu_case(args.ncu_case)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
