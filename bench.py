#!/usr/bin/env python3
"""BDDC-PCG time-to-solution on one GB300.

Workload: Poisson on the 64^3-cell bumpy sphere (6 seeded bumps, sub-cell
shift forcing cut fractions down to ~1e-6), 8^3-cell subdomain blocks, random
nodal source, Neumann on the cut boundary, stiffness weighting, variant-1
coarse objects, BDDC(cef), PCG to |r| < 1e-8 |b|.

One step = one complete solve from the device-resident nodal level set and
source: ufe_mesh_create -> ufe_assemble -> ufe_bddc_setup -> ufe_pcg_solve.
`value` is the mean time-to-solution per problem in mixed precision; the FP64
form of the same step is reported beside it.  L2 is flushed between steps.

Under torchrun each rank solves its own seeded replica (no collective on the
data path): weak scaling, value = max-over-ranks step time / problems per step.

--impl reference times the FP64 CPU oracle (the comparison implementation of
this project) on the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BDDC-PCG time-to-solution (s) and DOF-iters/s at rtol 1e-8, mixed vs FP64 on 1 GB300"
RTOL = 1e-8

# ALU peaks from unit counts and clocks (no measured FP32/FP64 SIMT peak is available):
# FP64 1.25 TFLOP/s nominal for GB300; FP32 SIMT 152 SMs x 128 lanes x 2 flop x 2.07 GHz.
PEAK_FP64_TFLOPS = 1.25
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes per launch of the dominant kernel from one ncu capture (summarised in
# profiles/launches_bumpy64_mixed_step.md); None once the kernel has changed since the
# counters were taken.
TRAFFIC_BYTES_PER_LAUNCH = {"gj_update_f64": 4.84e6, "gj_update_f32": None}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# oracle timing (the CPU baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def oracle_time_to_solution(seed, solves=1):
    """Time the FP64 oracle on the full workload: every set-up phase once, then
    `solves` PCG solves.  Returns phase times (s), iterations and DOFs."""
    from oracle.assembly import System
    from oracle.bddc import BDDC
    from oracle.integration import Integration
    from oracle.mesh import Mesh
    from oracle.pcg import pcg
    from paper_1703_06323_gb300 import inputs

    p = inputs.bumpy_sphere(seed)
    t = {}
    t0 = time.perf_counter()
    m = Mesh(p)
    m.objects("v1")
    t["mesh"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    integ = Integration(m, p)
    t["integration"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    sysm = System(m, integ, p)
    t["assembly"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    B = BDDC(m, integ, sysm, weighting="stiffness", objects="v1", coarse="cef")
    t["bddc_setup"] = time.perf_counter() - t0
    solve_times, its = [], 0
    for _ in range(solves):
        t0 = time.perf_counter()
        res = pcg(sysm.apply, sysm.b, B.apply, rtol=RTOL, maxit=2000)
        solve_times.append(time.perf_counter() - t0)
        its = res["iterations"]
    return {"phases": t, "solve_times": solve_times, "iterations": its, "n_dof": int(m.n_dof)}


def _oracle_worker_entry(seed, solves, out_path):
    res = oracle_time_to_solution(seed, solves)
    with open(out_path, "w") as fh:
        json.dump(res, fh)


def spawn_oracle(seed, solves, out_path):
    """Run the oracle in a spawned single-threaded process (BLAS pinned to 1 thread)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", f"{seed}:{solves}:{out_path}"]
    return subprocess.Popen(cmd, env=env, stdout=subprocess.DEVNULL, stderr=subprocess.PIPE)


def run_reference(args, rank):
    if rank != 0:
        return
    out = os.path.join("/tmp", f"ufe_oracle_ref_{os.getpid()}.json")
    solves = args.warmup + args.steps
    proc = spawn_oracle(args.seed, solves, out)
    _, err = proc.communicate()
    if proc.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": f"oracle failed: {err.decode()[-300:]}"}))
        return
    r = json.load(open(out))
    setup = sum(r["phases"].values())
    timed = r["solve_times"][args.warmup:]
    per_step = setup + statistics.mean(timed)
    sample = ("full workload; set-up phases timed once, then warmup+steps PCG solves; "
              "value = set-up + mean timed solve")
    line = {
        "impl": "reference", "metric": METRIC, "value": per_step, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "bumpy_sphere_64^3_cells_8^3_blocks", "rtol": RTOL, "weighting": "stiffness",
                   "objects": "v1", "coarse": "cef", "precision": "fp64"},
        "iterations": r["iterations"], "phases_s": r["phases"],
        "cpu_baseline": {"value": per_step, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": per_step, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def hbm_peak_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def per_iteration_roofline(U, p, phi_d, f_d, stream, flush, reps=20):
    """HBM roofline of the per-iteration kernels (mixed precision): CUDA-event timing of
    each kernel over `reps` preconditioner + operator applications, L2 flushed before
    each application; algorithmic bytes = the operator storage each kernel must read
    (BDDC info) plus 8 bytes per local vector entry it gathers or writes."""
    import torch
    peak, src = hbm_peak_gbs()
    mesh = U.ufe_mesh_create(p.box_lo, p.box_hi, p.cells, p.sub_cells, phi_d, p.dirichlet_face_mask, p.pin_node,
                             stream=stream.cuda_stream)
    sysh = bddc = None
    try:
        minfo = U.ufe_mesh_get_info(mesh)
        n = minfo["n_dof"]
        sysh = U.ufe_assemble(mesh, None, f_d, None, None)
        bddc = U.ufe_bddc_setup(sysh, U.WEIGHT_STIFFNESS, U.OBJECTS_VARIANT1, U.COARSE_CEF, U.PREC_MIXED)
        bi = U.ufe_bddc_get_info(bddc)
        g = torch.Generator(device="cpu").manual_seed(1)
        r = torch.randn(n, dtype=torch.float64, generator=g).to(phi_d.device)
        for _ in range(3):
            U.ufe_bddc_apply(bddc, r)
            U.ufe_system_apply(sysh, r)
        U.ufe_timing_reset()
        U.ufe_timing_enable(True)
        for _ in range(reps):
            flush.fill_(1.0)
            U.ufe_bddc_apply(bddc, r)
            U.ufe_system_apply(sysh, r)
        U.ufe_timing_enable(False)
        ni, ng, nc = bi["interior_slots"], bi["interface_slots"], bi["n_coarse"]
        gi, ig = 12 * 27 * ng, 12 * 27 * ni
        bytes_ = {
            "prec_interior": bi["bytes_interior_inverse"] + gi + 8 * ni + 8 * ng,
            "prec_neumann": bi["bytes_neumann"] + bi["bytes_coarse_basis"] + 24 * ng,
            "coarse_solve": bi["bytes_coarse_inverse"] + 16 * nc,
            "prec_prolong": bi["bytes_coarse_basis"] + 16 * ng,
            "prec_final": bi["bytes_interior_inverse"] + ig + 16 * ng + 16 * ni,
            "apply": 16 * n + 4 * minfo["n_nodes"] + minfo["n_cells"] + 512 * minfo["n_cut_cells"],
        }
        out = {"peak_gbs": peak, "peak_source": src, "l2": "flushed before each application", "reps": reps}
        for k, b in bytes_.items():
            ms, cnt = U.ufe_timing_get(k)
            us = 1e3 * ms / max(cnt, 1)
            gbs = b / (us * 1e-6) / 1e9 if us > 0 else None
            out[k] = {"us": us, "bytes": int(b), "gbs": gbs, "frac": gbs / peak if gbs else None}
        U.ufe_timing_reset()
        return out
    finally:
        if bddc is not None:
            U.ufe_bddc_destroy(bddc)
        if sysh is not None:
            U.ufe_system_destroy(sysh)
        U.ufe_mesh_destroy(mesh)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world):
    import numpy as np
    import torch

    from paper_1703_06323_gb300 import build_ext, inputs
    build_ext.build()
    from paper_1703_06323_gb300 import ufe as U

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    oracle_proc, oracle_out = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        oracle_out = os.path.join("/tmp", f"ufe_oracle_cpu_{os.getpid()}.json")
        oracle_proc = spawn_oracle(args.seed, 1, oracle_out)

    p = inputs.bumpy_sphere(args.seed + rank)
    phi_d = torch.from_numpy(p.phi).to(dev)
    f_d = torch.from_numpy(p.f).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2

    def step(precision, host=False):
        if host:
            phi, f = p.phi, p.f
        else:
            phi, f = phi_d, f_d
        mesh = U.ufe_mesh_create(p.box_lo, p.box_hi, p.cells, p.sub_cells, phi, p.dirichlet_face_mask, p.pin_node,
                                 stream=stream.cuda_stream)
        sysh = bddc = None
        try:
            n = U.ufe_mesh_get_info(mesh)["n_dof"]
            sysh = U.ufe_assemble(mesh, None, f, None, None)
            bddc = U.ufe_bddc_setup(sysh, U.WEIGHT_STIFFNESS, U.OBJECTS_VARIANT1, U.COARSE_CEF,
                                    U.PREC_MIXED if precision == "mixed" else U.PREC_FP64)
            x = np.zeros(n) if host else torch.zeros(n, dtype=torch.float64, device=dev)
            _, info = U.ufe_pcg_solve(sysh, bddc, None, x, rtol=RTOL, maxit=1000)
            binfo = U.ufe_bddc_get_info(bddc)
        finally:
            if bddc is not None:
                U.ufe_bddc_destroy(bddc)
            if sysh is not None:
                U.ufe_system_destroy(sysh)
            U.ufe_mesh_destroy(mesh)
        return n, info, binfo, x

    def timed(precision, k, launches=False):
        times, infos = [], []
        l0 = U.ufe_kernel_launches()
        for _ in range(k):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            n, info, binfo, _ = step(precision)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            infos.append((n, info, binfo))
        nl = U.ufe_kernel_launches() - l0
        return times, infos, nl

    for _ in range(args.warmup):
        step("mixed")
        if args.fp64_steps > 0:
            step("fp64")
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    U.ufe_timing_reset()
    U.ufe_timing_enable(True)
    t_mixed, i_mixed, launches = timed("mixed", args.steps)
    U.ufe_timing_enable(False)
    kt = {k: U.ufe_timing_get(k) for k in ("gj_update_f64", "gj_update_f32", "integrate_cut")}
    kt_extra = {k: U.ufe_timing_get(k)[0] / args.steps for k in ("gj_lookahead_f64", "gj_lookahead_f32",
                                                                   "gj_panel_f64", "gj_panel_f32")}
    phases = {k: U.ufe_timing_get(k)[0] / args.steps for k in
              ("phase_mesh", "phase_assemble", "phase_objects", "phase_local", "phase_factor", "phase_coarse",
               "phase_solve")}
    U.ufe_timing_reset()
    clk_stats = clk.stop()
    t_fp64, i_fp64, _ = timed("fp64", args.fp64_steps) if args.fp64_steps > 0 else ([float("nan")], [None], 0)
    if world > 1:
        torch.distributed.barrier()

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e_times = []
    for _ in range(max(0, min(args.steps, args.e2e_steps))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n, info, _, x_host = step("mixed", host=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)

    per_iter = per_iteration_roofline(U, p, phi_d, f_d, stream, flush) if rank == 0 else None

    mean_mixed = statistics.mean(t_mixed)
    mean_fp64 = statistics.mean(t_fp64)
    if world > 1:
        mean_mixed, mean_fp64, e2e_mean = max_over_ranks([mean_mixed, mean_fp64, statistics.mean(e2e_times)], dev)
    else:
        e2e_mean = statistics.mean(e2e_times) if e2e_times else float("nan")
    if rank != 0:
        return

    n, info, binfo = i_mixed[-1]
    its = info["iterations"]
    solve_s = statistics.mean(i[1]["solve_ms"] for i in i_mixed) / 1e3
    setup_s = statistics.mean(i[2]["setup_ms"] for i in i_mixed) / 1e3
    if i_fp64[-1] is not None:
        n64, info64, binfo64 = i_fp64[-1]
    else:
        n64, info64 = n, {"iterations": 0, "true_rel_residual": None}

    # roofline of the dominant instrumented kernel (the Gauss-Jordan update steps are
    # ALU bound: symmetric inversion of an n x n matrix takes n^3 flops)
    flops = {"gj_update_f64": binfo["inverse_flops_coarse"], "gj_update_f32": binfo["inverse_flops_local"]}
    peaks = {"gj_update_f64": PEAK_FP64_TFLOPS, "gj_update_f32": PEAK_FP32_TFLOPS}
    dom = max(flops, key=lambda k: kt[k][0])
    ms_tot, n_launch = kt[dom]
    per_launch_flops = flops[dom] * args.steps / max(n_launch, 1)
    avg_s = ms_tot / 1e3 / max(n_launch, 1)
    achieved = per_launch_flops / avg_s / 1e12 if avg_s > 0 else None
    roofline = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peaks[dom], "unit": "TFLOP/s",
                "frac": achieved / peaks[dom] if achieved else None, "traffic": TRAFFIC_BYTES_PER_LAUNCH[dom],
                "peak_source": "derived from unit counts and clocks (FP64: 1.25 TFLOP/s nominal)",
                "launches": n_launch, "avg_launch_us": avg_s * 1e6,
                "kernel_ms_per_step": dict({k: v[0] / args.steps for k, v in kt.items()}, **kt_extra)}

    line = {
        "metric": METRIC,
        "value": mean_mixed / world,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": mean_mixed * 1e3,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "bumpy_sphere_64^3_cells_8^3_blocks", "rtol": RTOL, "precision": "mixed",
                   "weighting": "stiffness", "objects": "v1", "coarse": "cef", "n_dof": n,
                   "problems_per_step": world, "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": "replicas" if world > 1 else "single"},
        "iterations": its,
        "dof_iters_per_s": n * its / (mean_mixed),
        "solve_dof_iters_per_s": n * its / solve_s if solve_s > 0 else None,
        "setup_s_device": setup_s,
        "solve_s_device": solve_s,
        "n_coarse": binfo["n_coarse"],
        "fp64": {"value": mean_fp64 / world, "unit": "s", "iterations": info64["iterations"],
                 "dof_iters_per_s": n64 * info64["iterations"] / mean_fp64 if mean_fp64 == mean_fp64 else None,
                 "true_rel_residual": info64["true_rel_residual"]},
        "true_rel_residual": info["true_rel_residual"],
        "gpu_launches": launches,
        "phase_ms": phases,
        "roofline": roofline,
        "per_iteration_roofline": per_iter,
        "clocks": clk_stats,
        "e2e": {"value": e2e_mean / world, "unit": "s",
                "h2d_bytes_per_step": int(p.phi.nbytes + p.f.nbytes + 8 * n),
                "d2h_bytes_per_step": int(8 * n)},
    }
    if oracle_proc is not None:
        _, err = oracle_proc.communicate()
        if oracle_proc.returncode == 0:
            r = json.load(open(oracle_out))
            total = sum(r["phases"].values()) + r["solve_times"][0]
            line["cpu_baseline"] = {"value": total, "unit": "s", "cores": 1, "kind": "oracle",
                                    "sample": "one complete time-to-solution of the same workload (seed "
                                              f"{args.seed}), BLAS pinned to 1 thread",
                                    "phases_s": r["phases"], "iterations": r["iterations"]}
        else:
            line["cpu_baseline"] = {"value": None, "unit": "s", "cores": 1, "kind": "oracle",
                                    "sample": f"oracle failed: {err.decode()[-200:]}"}
    print(json.dumps(line))


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over all ranks of the process group
    (every rank receives it): the job's step time is that of its slowest rank."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t]


def main():
    args = parse_args()
    if args.oracle_worker:
        seed, solves, out = args.oracle_worker.split(":", 2)
        _oracle_worker_entry(int(seed), int(solves), out)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
