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

# DRAM bytes per launch of a kernel from one ncu capture of the same command
# (dram__bytes_read.sum + dram__bytes_write.sum); a kernel missing here (or changed
# since its capture) reports traffic null.
TRAFFIC_BYTES_PER_LAUNCH = {"gj_update_f64": 2.85e6}
# nominal dense tensor rates (PFLOP/s) that scale a measured bf16 peak to another dtype
NOMINAL_TENSOR = {"bf16": 2.25, "tf32": 1.1}


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
    ap.add_argument("--no-extra", action="store_true", help="skip the batched-set and adjoint workloads")
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# oracle timing (the CPU baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_time_to_solution(p, pool=None):
    """One complete FP64 oracle time-to-solution of problem p: mesh and objects, cut-cell
    integration (over the cut cells on `pool`'s workers when given), assembly, BDDC
    set-up, PCG.  Returns the phase times (s), iterations and DOFs."""
    from oracle.assembly import System
    from oracle.bddc import BDDC
    from oracle.integration import Integration
    from oracle.mesh import Mesh
    from oracle.pcg import pcg

    t = {}
    t0 = time.perf_counter()
    m = Mesh(p)
    m.objects("v1")
    t["mesh"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    mapper = None if pool is None else (lambda fn, args: pool.starmap(fn, args, chunksize=64))
    integ = Integration(m, p, map_fn=mapper)
    t["integration"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    sysm = System(m, integ, p)
    t["assembly"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    B = BDDC(m, integ, sysm, weighting="stiffness", objects="v1", coarse="cef")
    t["bddc_setup"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = pcg(sysm.apply, sysm.b, B.apply, rtol=RTOL, maxit=2000)
    t["pcg"] = time.perf_counter() - t0
    return {"phases": t, "total": sum(t.values()), "iterations": res["iterations"], "n_dof": int(m.n_dof)}


def _oracle_worker_entry(spec, out_path):
    """`runs` complete time-to-solutions of the bench workload with `workers` processes
    (1: this process alone)."""
    seed, runs, workers = (int(v) for v in spec.split(","))
    from paper_1703_06323_gb300 import inputs
    p = inputs.bumpy_sphere(seed)
    pool = None
    if workers > 1:
        pool = mp.get_context("spawn").Pool(workers)
        pool.starmap(max, [(1, 2)] * workers)   # workers started before the timing
    try:
        res = [oracle_time_to_solution(p, pool) for _ in range(runs)]
    finally:
        if pool is not None:
            pool.terminate()
    with open(out_path, "w") as fh:
        json.dump({"runs": res, "workers": workers}, fh)


def run_oracle(seed, runs, workers):
    """Run the oracle in a child process with BLAS pinned to one thread per process;
    returns (result dict, error text)."""
    out = os.path.join("/tmp", f"ufe_oracle_{os.getpid()}_{workers}_{runs}.json")
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", f"{seed},{runs},{workers}:{out}"]
    proc = subprocess.run(cmd, env=env, stdout=subprocess.DEVNULL, stderr=subprocess.PIPE)
    if proc.returncode != 0:
        return None, proc.stderr.decode()[-300:]
    with open(out) as fh:
        r = json.load(fh)
    os.unlink(out)
    return r, ""


def run_reference(args, rank):
    """The reference arm: the FP64 oracle on every host core, one complete
    time-to-solution of the bench workload per step (warmup + steps runs)."""
    if rank != 0:
        return
    cores = host_cores()
    r, err = run_oracle(args.seed, args.warmup + args.steps, cores)
    if r is None:
        print(json.dumps({"impl": "reference", "unavailable": f"oracle failed: {err}"}))
        return
    timed = r["runs"][args.warmup:]
    per_step = statistics.mean(x["total"] for x in timed)
    phases = {k: statistics.mean(x["phases"][k] for x in timed) for k in timed[0]["phases"]}
    sample = (f"each step one complete time-to-solution of the workload (seed {args.seed}): mesh, "
              f"integration over {cores} processes, assembly, BDDC set-up, PCG; value = mean over the timed steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": per_step, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "bumpy_sphere_64^3_cells_8^3_blocks", "rtol": RTOL, "weighting": "stiffness",
                   "objects": "v1", "coarse": "cef", "precision": "fp64"},
        "iterations": timed[-1]["iterations"], "phases_s": phases,
        "cpu_baseline": {"value": per_step, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
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


def measured_peaks():
    """Measured peaks of the GB300s (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d.get("bf16_tflops", 1900.0)),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d.get("bf16_tflops", 1700.0))),
                "source": "measured"}
    except (OSError, KeyError, ValueError, TypeError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def per_iteration_roofline(U, p, phi_d, f_d, stream, flush, peaks, reps=20):
    """Per-iteration kernels (mixed precision): CUDA-event time per launch over `reps`
    preconditioner + operator applications, L2 flushed before each application.
    Algorithmic bytes per launch = the stored operators each kernel must read (dense
    explicit inverses, as stored: BDDC info) plus 8 bytes per local vector entry it
    gathers or writes; the operator apply reads x, writes y, the DOF map and the 36
    unique entries of each cut-cell matrix."""
    import torch
    peak = peaks["hbm_gbs"]
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
            "apply": 16 * n + 4 * minfo["n_nodes"] + minfo["n_cells"] + 36 * 8 * minfo["n_cut_cells"],
        }
        out = {"peak_gbs": peak, "peak_source": peaks["source"], "l2": "flushed before each application",
               "reps": reps}
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


def kuhn_subtets(phi, cells):
    """Clipped sub-tetrahedra of the cut cells' Kuhn tets (host count from the nodal level
    set): a Kuhn tet with k inside vertices gives 1 (k = 1) or 3 (k = 2, 3) sub-tets; one
    with 0 or 4 needs no quadrature."""
    import numpy as np
    nx, ny, nz = cells
    ph = phi.reshape(nz + 1, ny + 1, nx + 1)
    neg = ph < 0.0
    v = [neg[dz:dz + nz, dy:dy + ny, dx:dx + nx].ravel() for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
    total = 0
    for a, b in ((0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1)):
        verts = (0, 1 << a, (1 << a) | (1 << b), 7)
        k = sum(v[i].astype(np.int64) for i in verts)
        total += int((k == 1).sum() + 3 * ((k == 2) | (k == 3)).sum())
    return total


def roofline_block(kt, n_steps, binfo, per_iter, iterations, fma, peaks, n_subtets):
    """Roofline of the dominant kernel: the candidate with the largest device time per
    step among every instrumented kernel.  Algorithmic work per launch:
    * Gauss-Jordan update launches (local inverses in FP32 / coarse inverse in FP64):
      the Cholesky factorisation count n^3/3 of every inverted matrix, spread evenly over
      that precision's update launches (the look-ahead, panel and diagonal launches of the
      same inversions are listed with their time only);
    * cut-cell integration: 27 moment FMAs (54 flops) at each of the 35 points of every
      clipped sub-tetrahedron;
    * per-iteration kernels: the bytes of per_iteration_roofline, timed once per PCG
      iteration plus the initial preconditioner application."""
    # the tensor-core update launches are timed inside the long bench step: the sustained
    # bf16 figure, scaled to tf32 by the nominal ratio
    tf32 = peaks["bf16_tflops_sustained"] * NOMINAL_TENSOR["tf32"] / NOMINAL_TENSOR["bf16"]
    f32_on_tc = binfo.get("local_tensor_cores", 0) == 1
    local_flops = binfo["inverse_flops_local"] / 3.0
    coarse_flops = binfo["inverse_flops_coarse"] / 3.0
    f64_flops = coarse_flops + (local_flops if binfo["fp64_refactor"] else 0.0)
    rows = []

    def add(name, ms_step, launches_step, work, bound, unit, peak, peak_source):
        if ms_step <= 0 or launches_step <= 0:
            return
        row = {"kernel": name, "ms_per_step": ms_step, "launches_per_step": launches_step,
               "avg_launch_us": 1e3 * ms_step / launches_step}
        if work is not None:
            achieved = work / launches_step / (row["avg_launch_us"] * 1e-6)
            achieved = achieved / 1e12 if unit == "TFLOP/s" else achieved / 1e9
            row.update({"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                        "peak_source": peak_source, "work_per_launch": work / launches_step})
        rows.append(row)

    fma_src = "FMA-loop probe (ufe_probe_fma_rate) measured in this run"
    for name, (ms, cnt) in kt.items():
        ms_step, l_step = ms / n_steps, cnt / n_steps
        if name == "gj_update_f64":
            add(name, ms_step, l_step, f64_flops, "alu", "TFLOP/s", fma["fp64"], fma_src)
        elif name == "gj_update_f32":
            if f32_on_tc:
                add(name, ms_step, l_step, 0.0 if binfo["fp64_refactor"] else local_flops, "tensor", "TFLOP/s",
                    tf32, f"{peaks['source']} sustained bf16 peak x nominal tf32/bf16 ({NOMINAL_TENSOR['tf32']}/"
                          f"{NOMINAL_TENSOR['bf16']})")
            else:
                add(name, ms_step, l_step, 0.0 if binfo["fp64_refactor"] else local_flops, "alu", "TFLOP/s",
                    fma["fp32"], fma_src)
        elif name == "integrate_cut":
            add(name, ms_step, l_step, 54.0 * 35 * n_subtets, "alu", "TFLOP/s", fma["fp64"], fma_src)
        else:
            add(name, ms_step, l_step, None, None, None, None, None)
    if per_iter:
        for k in ("prec_interior", "prec_neumann", "coarse_solve", "prec_prolong", "prec_final", "apply"):
            d = per_iter.get(k)
            if not d or not d["us"]:
                continue
            launches = iterations + 1
            add(k, d["us"] * launches / 1e3, launches, d["bytes"] * launches, "hbm", "GB/s", per_iter["peak_gbs"],
                per_iter["peak_source"])
    rows.sort(key=lambda r: -r["ms_per_step"])
    dom = next(r for r in rows if "achieved" in r)
    traffic = TRAFFIC_BYTES_PER_LAUNCH.get(dom["kernel"])
    out = {"kernel": dom["kernel"], "bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"],
           "unit": dom["unit"], "frac": dom["frac"], "traffic": traffic, "peak_source": dom["peak_source"],
           "launches_per_step": dom["launches_per_step"], "avg_launch_us": dom["avg_launch_us"],
           "work_per_launch": dom["work_per_launch"], "kernels": rows}
    return out


def adjoint_workload(U, dev, stream, flush, precision, reps=2, coarse_solver="auto", keep_corners=False):
    """Config-5 style adjoint workload (128^3 background cells, 16^3 subdomains, sphere of
    radius 0.45, per-cell kappa = exp(GRF)): mesh, assembly, BDDC set-up, forward solve
    and adjoint solve with the per-cell gradient, timed by CUDA events; returns the mean
    time and the solve details."""
    import torch
    from paper_1703_06323_gb300 import autograd as AG
    from paper_1703_06323_gb300 import inputs
    from paper_1703_06323_gb300.solver import Solver
    if not hasattr(adjoint_workload, "problem"):
        adjoint_workload.problem = inputs.coefficient_sphere(0, 128)
    p = adjoint_workload.problem
    arrays = {"phi": torch.from_numpy(p.phi).to(dev), "f": torch.from_numpy(p.f).to(dev),
              "g": torch.from_numpy(p.dirichlet_values).to(dev), "kappa": torch.from_numpy(p.kappa).to(dev)}
    w = AG.lumped_mass(p, dev)
    ud_nodes = torch.from_numpy(p.meta["u_d"]).to(dev)
    times, last = [], None
    for rep in range(reps + 1):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with Solver(p, precision=precision, arrays=dict(arrays), stream=stream.cuda_stream,
                    coarse_solver=coarse_solver, coarse_keep_corners=keep_corners) as S:
            u = torch.zeros(S.n_dof, dtype=torch.float64, device=dev)
            _, fi = U.ufe_pcg_solve(S.system, S.bddc, None, u, rtol=RTOL, maxit=2000)
            dof = torch.from_numpy(U.ufe_mesh_get_dof_map(S.mesh)).to(dev).long()
            node_of_dof = torch.empty(S.n_dof, dtype=torch.long, device=dev)
            sel = dof >= 0
            node_of_dof[dof[sel]] = torch.nonzero(sel).squeeze(1)
            lam = torch.zeros_like(u)
            g = torch.empty(p.kappa.size, dtype=torch.float64, device=dev)
            ai = U.ufe_adjoint(S.system, S.bddc, u, w * (u - ud_nodes[node_of_dof]), lam, g, rtol=RTOL,
                               maxit=2000)
            e1.record(stream)
            torch.cuda.synchronize()
            info = (S.n_dof, S.info["n_subdomains"], S.bddc_info["n_coarse"], fi, ai, S.bddc_info)
        if rep > 0:
            times.append(e0.elapsed_time(e1) / 1e3)
        last = info
    n, nsub, nc, fi, ai, bi = last
    return {"value": statistics.mean(times), "unit": "s", "reps": reps, "n_dof": n, "subdomains": nsub,
            "n_coarse": nc, "forward_iterations": fi["iterations"], "adjoint_iterations": ai["iterations"],
            "forward_true_rel_residual": fi["true_rel_residual"], "setup_ms": bi["setup_ms"],
            "forward_solve_ms": fi["solve_ms"], "coarse_solver": bi["coarse_solver"],
            "level2_subdomains": bi["level2_subdomains"], "level3_coarse": bi["level3_coarse"]}


def elastic_workload(U, dev, stream, flush, precision, reps=2, coarse_solver="auto"):
    """Config-3 elasticity workload (the 96^3 union of 8 seeded spheres, 8^3 subdomains,
    3 DOFs per node): mesh, assembly, BDDC set-up and solve at rtol 1e-8 from device
    inputs, timed by CUDA events; returns the mean time-to-solution and the details."""
    import numpy as np
    import torch
    from paper_1703_06323_gb300 import inputs
    from paper_1703_06323_gb300.solver import Solver
    if not hasattr(elastic_workload, "problem"):
        elastic_workload.problem = inputs.elastic_spheres(0)
    p = elastic_workload.problem
    arrays = {"phi": torch.from_numpy(p.phi).to(dev), "f": torch.from_numpy(np.ascontiguousarray(p.f)).to(dev),
              "g": torch.from_numpy(np.ascontiguousarray(p.dirichlet_values)).to(dev)}
    times, last = [], None
    for rep in range(reps + 1):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with Solver(p, precision=precision, arrays=dict(arrays), stream=stream.cuda_stream,
                    coarse_solver=coarse_solver) as S:
            x = torch.zeros(S.n_dof, dtype=torch.float64, device=dev)
            _, fi = U.ufe_pcg_solve(S.system, S.bddc, None, x, rtol=RTOL, maxit=2000)
            e1.record(stream)
            torch.cuda.synchronize()
            bi = S.bddc_info
            info = (S.n_dof, S.info["n_subdomains"], bi["n_coarse"], bi["setup_ms"], bi["fp64_subdomains"], fi,
                    bi["level3_coarse"])
        if rep > 0:
            times.append(e0.elapsed_time(e1) / 1e3)
        last = info
    n, nsub, nc, setup_ms, n64, fi, n3 = last
    return {"value": statistics.mean(times), "unit": "s", "reps": reps, "n_dof": n, "subdomains": nsub,
            "n_coarse": nc, "setup_s_device": setup_ms / 1e3, "solve_s_device": fi["solve_ms"] / 1e3,
            "fp64_subdomains": n64, "iterations": fi["iterations"], "true_rel_residual": fi["true_rel_residual"],
            "level3_coarse": n3}


def batched_workload(U, dev, stream, flush, reps=2):
    """Config-4 style batched set (256 seeded spheres on 24^3..64^3 background meshes,
    mixed precision): set-up of every problem, then one ufe_pcg_solve_batched over all
    of them (first call builds the solve graphs; the repeats reuse them)."""
    import torch
    from paper_1703_06323_gb300 import inputs
    from paper_1703_06323_gb300.solver import Solver
    ps = inputs.batched_spheres(count=256, seed=0)
    arrays = [{"phi": torch.from_numpy(p.phi).to(dev), "f": torch.from_numpy(p.f).to(dev),
               "g": torch.from_numpy(p.dirichlet_values).to(dev)} for p in ps]
    torch.cuda.synchronize()
    solvers = []
    try:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for p, a in zip(ps, arrays):
            solvers.append(Solver(p, precision="mixed", arrays=a, stream=stream.cuda_stream))
        e1.record(stream)
        torch.cuda.synchronize()
        setup_s = e0.elapsed_time(e1) / 1e3
        solve_times, infos = [], None
        for rep in range(reps + 1):
            xs = [torch.zeros(S.n_dof, dtype=torch.float64, device=dev) for S in solvers]
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0.record(stream)
            st, infos = U.ufe_pcg_solve_batched([S.system for S in solvers], [S.bddc for S in solvers], None, xs,
                                                rtol=RTOL, maxit=1000)
            e1.record(stream)
            torch.cuda.synchronize()
            solve_times.append(e0.elapsed_time(e1) / 1e3)
        dofs = [S.n_dof for S in solvers]
        its = [i["iterations"] for i in infos]
        solve = statistics.mean(solve_times[1:])
        return {"problems": len(ps), "total_dofs": int(sum(dofs)), "setup_s": setup_s,
                "solve_s_first_call": solve_times[0], "solve_s": solve, "unit": "s",
                "time_to_solution_s": setup_s + solve,
                "dof_iters_per_s": float(sum(d * i for d, i in zip(dofs, its))) / solve,
                "iterations_min_median_max": [min(its), int(statistics.median(its)), max(its)],
                "all_converged": all(i["converged"] == 1 for i in infos),
                "max_true_rel_residual": max(i["true_rel_residual"] for i in infos)}
    finally:
        for S in solvers:
            S.close()


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

    p = inputs.bumpy_sphere(args.seed + rank)
    phi_d = torch.from_numpy(p.phi).to(dev)
    f_d = torch.from_numpy(p.f).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2

    def step(precision, host=False, coarse_solver=0, keep_corners=0):
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
                                    U.PREC_MIXED if precision == "mixed" else U.PREC_FP64, coarse_solver, 0,
                                    keep_corners)
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

    def timed(precision, k):
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
    kt = {k: U.ufe_timing_get(k) for k in ("gj_update_f64", "gj_update_f32", "gj_lookahead_f64", "gj_lookahead_f32",
                                           "gj_panel_f64", "gj_panel_f32", "gj_diag_f64", "gj_diag_f32",
                                           "integrate_cut")}
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

    mean_mixed = statistics.mean(t_mixed)
    mean_fp64 = statistics.mean(t_fp64)
    if world > 1:
        mean_mixed, mean_fp64, e2e_mean = max_over_ranks([mean_mixed, mean_fp64, statistics.mean(e2e_times)], dev)
    else:
        e2e_mean = statistics.mean(e2e_times) if e2e_times else float("nan")
    if rank != 0:
        return

    peaks = measured_peaks()
    per_iter = per_iteration_roofline(U, p, phi_d, f_d, stream, flush, peaks)
    fma = {"fp64": U.ufe_probe_fma_rate("fp64", stream.cuda_stream),
           "fp32": U.ufe_probe_fma_rate("fp32", stream.cuda_stream)}
    extra = {}
    if not args.no_extra and world == 1:
        # the same workload with the three-level method (the coarse problem preconditioned
        # by BDDC over groups of 2^3 blocks instead of inverted)
        tl = {}
        for prec, keep in (("mixed", 0), ("fp64", 0), ("mixed_keep_corners", 1)):
            pr = prec.split("_")[0]
            step(pr, coarse_solver=U.COARSE_SOLVER_BDDC, keep_corners=keep)
            ts = []
            for _ in range(5):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, tinfo, tb, _ = step(pr, coarse_solver=U.COARSE_SOLVER_BDDC, keep_corners=keep)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            tl[prec] = {"ms_per_step": statistics.mean(ts), "iterations": tinfo["iterations"],
                        "setup_ms": tb["setup_ms"], "solve_ms": tinfo["solve_ms"],
                        "true_rel_residual": tinfo["true_rel_residual"],
                        "level2_subdomains": tb["level2_subdomains"], "level3_coarse": tb["level3_coarse"]}
        extra["three_level"] = tl
        extra["adjoint_128^3"] = {prec: adjoint_workload(U, dev, stream, flush, prec) for prec in ("mixed", "fp64")}
        extra["adjoint_128^3"]["mixed_three_level"] = adjoint_workload(U, dev, stream, flush, "mixed",
                                                                       coarse_solver="bddc")
        extra["adjoint_128^3"]["mixed_three_level_keep_corners"] = adjoint_workload(
            U, dev, stream, flush, "mixed", coarse_solver="bddc", keep_corners=True)
        extra["batched_256"] = batched_workload(U, dev, stream, flush)
        extra["elastic_96^3"] = {prec: elastic_workload(U, dev, stream, flush, prec) for prec in ("mixed", "fp64")}
        extra["elastic_96^3"]["mixed_three_level"] = elastic_workload(U, dev, stream, flush, "mixed",
                                                                      coarse_solver="bddc")

    n, info, binfo = i_mixed[-1]
    its = info["iterations"]
    solve_s = statistics.mean(i[1]["solve_ms"] for i in i_mixed) / 1e3
    setup_s = statistics.mean(i[2]["setup_ms"] for i in i_mixed) / 1e3
    if i_fp64[-1] is not None:
        n64, info64, binfo64 = i_fp64[-1]
    else:
        n64, info64 = n, {"iterations": 0, "true_rel_residual": None}
    roofline = roofline_block(kt, args.steps, binfo, per_iter, its, fma, peaks, kuhn_subtets(p.phi, p.cells))

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
        "launch_shape": {"cluster_ctas": binfo["prec_cluster"], "row_stages": binfo["prec_stages"],
                         "chosen_by": "UFE_PREC_SHAPE" if os.environ.get("UFE_PREC_SHAPE") else "tuner"},
        "fp64": {"value": mean_fp64 / world, "unit": "s", "iterations": info64["iterations"],
                 "dof_iters_per_s": n64 * info64["iterations"] / mean_fp64 if mean_fp64 == mean_fp64 else None,
                 "true_rel_residual": info64["true_rel_residual"]},
        "true_rel_residual": info["true_rel_residual"],
        "gpu_launches": launches,
        "phase_ms": phases,
        "roofline": roofline,
        "fma_peaks_tflops": fma,
        "per_iteration_roofline": per_iter,
        "clocks": clk_stats,
        "e2e": {"value": e2e_mean / world, "unit": "s",
                "h2d_bytes_per_step": int(p.phi.nbytes + p.f.nbytes + 8 * n),
                "d2h_bytes_per_step": int(8 * n)},
    }
    line.update(extra)
    # the CPU baseline runs after every GPU measurement (no host core busy meanwhile)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.seed)
    print(json.dumps(line))


def cpu_baseline(seed):
    """The FP64 oracle on the host: one complete time-to-solution of the same workload on
    one core, then one with the cut-cell integration spread over every host core."""
    cores = host_cores()
    r1, err1 = run_oracle(seed, 1, 1)
    rn, errn = run_oracle(seed, 1, cores) if cores > 1 else (None, "one host core")
    if r1 is None:
        return {"value": None, "unit": "s", "cores": 1, "kind": "oracle", "sample": f"oracle failed: {err1}"}
    one = r1["runs"][0]
    out = {"value": one["total"], "unit": "s", "cores": 1, "kind": "oracle",
           "sample": f"one complete time-to-solution of the same workload (seed {seed}), one process, BLAS on 1 "
                     "thread", "phases_s": one["phases"], "iterations": one["iterations"], "host_cores": cores}
    if rn is not None:
        r = rn["runs"][0]
        out["n_core"] = {"value": r["total"], "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": f"the same, cut-cell integration over {cores} processes", "phases_s": r["phases"]}
    else:
        out["n_core"] = {"value": None, "cores": cores, "sample": errn}
    return out


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
        spec, out = args.oracle_worker.split(":", 1)
        _oracle_worker_entry(spec, out)
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
