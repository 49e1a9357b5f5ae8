#!/usr/bin/env python
"""Benchmark of the Basic-Scheme solver on the anisotropic dlVP workload.

Workload (the configuration the headline metric is quoted on): M = [[128,32],[0,128]] (m = 16384,
Smith grid 32 x 512), de la Vallee Poussin generator with plateau |u| <= 0.25
and ramp to 0.75, 20 random non-overlapping disks (radii U[0.03,0.08], seed 2)
at contrast 100, nu = 0.3, the 3 Mandel unit strains, Cauchy tolerance 1e-6.

One step = one complete solve of that workload: the Gamma^p table build
(fh_set_reference), every fixed-point iteration of all 3 load cases until each
reaches r <= 1e-6, and the FP64 mean-stress / C_eff reduction.  The metric is
voxel-iterations/s = sum over loads of m * iterations / time; time-to-1e-6 is
the per-step time.  Three precision modes are run: plain FP64, FP32 bulk
stages, and mixed (FP32 iterations, then one FP64 step); each reports its C_eff
error against the converged FP64 oracle (tests/golden/ceff_dlvp_sheared.txt).
The headline is the mode selected with --mode (default: mixed, the fastest mode
whose C_eff meets 1e-6).

The line also carries the batched 2-D workload (512 microstructures) and the
3-D box-spline workload (M = diag(128,128,128), 6 loads: time to 1e-6 per
precision mode and the HBM roofline of each pass of one iteration).

Prints one JSON line (rank 0).  --impl reference runs the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

# The FP64 CPU oracle (the reference arm and the cpu_baseline leg) is timed on
# one host thread: pin numpy's BLAS before numpy loads, so that "cores": 1 in
# the JSON line is what actually ran (its threaded GEMMs on small tiles were
# slower anyway).
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "voxel-iterations/s & time-to-1e-6 residual: batched/mixed/learned vs plain FP64"
UNIT = "voxel-iterations/s"
WORKLOAD = ("dlvp_sheared: M=[[128,32],[0,128]] (m=16384, grid 32x512), dlVP plateau 0.25 ramp 0.5, "
            "20 disks r~U[0.03,0.08] contrast 100, 3 Mandel unit loads, Cauchy tol 1e-6")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-cluster", type=int, default=0)
    ap.add_argument("--no-box3d", action="store_true")
    ap.add_argument("--only-box3d", action="store_true",
                    help="run only the 3-D box-spline section (prints its JSON object)")
    ap.add_argument("--box3d-n", type=int, default=128, help="grid size of the 3-D section")
    ap.add_argument("--box3d-modes", default="mixed,fp32,fp64",
                    help="precision modes of the 3-D section (comma-separated)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------

def oracle_problem(w):
    from oracle import generators as OG, green as OGr, material as OM, scheme as OS
    T = OS.SNFTransform(w["M"])
    ids = W.phase_ids(T.points / T.D, w["centres"], w["radii"])
    lm = [OM.lame(E, nu) for E, nu in w["phases"]]
    Cp = np.stack([OM.isotropic_mandel(l, m, 2) for l, m in lm])
    l0, m0 = OM.reference_medium_ms([l for l, _ in lm], [m for _, m in lm])
    C0 = OM.isotropic_mandel(l0, m0, 2)
    Gp = OGr.gamma_p_table(w["M"], OG.Generator("dlvp", alpha=w["generator"]["alpha"]), C0, T.freqs)
    return T, Gp, Cp[ids], C0


def oracle_sample(w, seconds, max_iter=5000):
    """Time the oracle as it stands on one load case, iterating until `seconds` elapse."""
    from oracle import scheme as OS
    T, Gp, C, C0 = oracle_problem(w)
    e0 = np.eye(3)[:1]
    n = 8
    t0 = time.perf_counter()
    OS.solve(T, Gp, C, C0, e0, tol=0.0, max_iter=n)
    dt = time.perf_counter() - t0
    n = int(min(max_iter, max(8, seconds / max(dt / 8, 1e-6))))
    t0 = time.perf_counter()
    OS.solve(T, Gp, C, C0, e0, tol=0.0, max_iter=n)
    dt = time.perf_counter() - t0
    return {"value": T.m * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"load 1 of 3, {n} fixed-point iterations of the FP64 oracle (numpy FFT on the "
                      f"Smith grid), {dt:.1f} s single-threaded"}


def run_reference(args, rank):
    if rank != 0:
        return
    w = W.dlvp_sheared()
    from oracle import scheme as OS
    T, Gp, C, C0 = oracle_problem(w)
    e0 = np.eye(3)[:1]
    iters = 30
    for _ in range(args.warmup):
        OS.solve(T, Gp, C, C0, e0, tol=0.0, max_iter=iters)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        OS.solve(T, Gp, C, C0, e0, tol=0.0, max_iter=iters)
    dt = time.perf_counter() - t0
    value = T.m * iters * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": f"{iters} oracle iterations of one load case (bounded sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{iters} iterations x {args.steps} steps, load 1 of 3"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU clocks sampled during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) != 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def reduce_over_ranks(dist, total_ms, vox, device):
    """Whole-job numbers of independent replicas: the slowest rank's time and the
    voxel-iterations of all ranks (no collective touches the solver's data)."""
    import torch
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    v = torch.tensor([float(vox)], device=device, dtype=torch.float64)
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return float(t.item()), int(v.item())


def ceff_reference():
    path = os.path.join(ROOT, "tests", "golden", "ceff_dlvp_sheared.txt")
    return np.loadtxt(path) if os.path.exists(path) else None


def flops_per_launch(g, nload, kind):
    """Algorithmic FLOPs of one launch of a pass (5 N log2 N per complex FFT of
    length N, half that for a real one; n_v^2 FMAs per point for the stress,
    4 n_v^2 flops per half-spectrum frequency for the Green step)."""
    nv, L, dims = g["nv"], g["L"], g["dims"]
    m = g["m"]
    nrows = m // L
    if kind == "row":
        fft = nv * 2 * 2.5 * L * math.log2(L) * nrows
        pw = m * (2 * nv * nv + 6 * nv)
        return nload * (fft + pw)
    N0 = dims[0]
    nhalf = g["nhalf"]
    fft = nv * 2 * 5 * N0 * math.log2(N0) * (nhalf // N0)
    return nload * (fft + nhalf * 4 * nv * nv)


def run_gpu(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    import paper_1701_04685_gb300 as fh
    fh.library()
    dist = None
    if world > 1:
        import torch.distributed as dist
    w = W.dlvp_sheared()
    p = fh.Pattern(w["M"])
    ids = W.phase_ids(p.points(), w["centres"], w["radii"])
    Cp = np.stack([fh.isotropic_stiffness(*fh.lame(E, nu), 2) for E, nu in w["phases"]])
    eps0 = np.eye(3)
    stream = torch.cuda.current_stream().cuda_stream
    s = fh.Solver(p, fh.generator("dlvp", alpha=w["generator"]["alpha"]), 3, stream)
    s.set_stiffness_phases(ids, Cp)
    prec = {"fp64": fh.FH_PREC_FP64, "fp32": fh.FH_PREC_FP32, "mixed": fh.FH_PREC_MIXED}
    Cref = ceff_reference()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2

    def step(mode):
        s.set_reference(None)                     # Gamma^p table (FP64, on the device)
        return s.solve(eps0, tol=args.tol, max_iter=20000, precision=prec[mode])

    results = {}
    clocks = None
    for mode in ("fp64", "fp32", "mixed"):
        for _ in range(args.warmup):
            step(mode)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if mode == args.mode and local_rank == 0:
            clocks = Clocks(local_rank)
        times, vox, launches, iters, path = [], 0, 0, None, None
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()                         # L2 flushed between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            out = step(mode)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            vox += int(np.sum(out["iterations"])) * p.m
            launches += out["kernel_launches"] + 1  # + the table-build kernel
            iters = out["iterations"]
            path = (out["path"], out["cluster"])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
        if mode == args.mode and clocks is not None:
            clocks = clocks.stop()
        total_ms = float(np.sum(times))
        if dist:
            total_ms, vox = reduce_over_ranks(dist, total_ms, vox, "cuda")
        ce = s.get_ceff()
        results[mode] = {"value": vox / (total_ms * 1e-3), "ms_per_step": total_ms / args.steps,
                         "iterations": [int(x) for x in iters], "gpu_launches": launches,
                         "path": "cluster-resident" if path[0] == 2 else "whole-GPU passes",
                         "cluster_size": path[1], "ceff": ce.tolist(), "wall_s": wall,
                         "ceff_rel_err_vs_converged_oracle":
                             None if Cref is None else float(np.linalg.norm(ce - Cref) / np.linalg.norm(Cref))}

    # e2e: through the public API with host buffers (pinned), copies inside the timed region
    head = args.mode
    ph_host = torch.from_numpy(ids).pin_memory()
    E_host = torch.empty((3, 3, p.m), dtype=torch.float64).pin_memory()
    for _ in range(2):
        s.set_stiffness_phases(ph_host, Cp)
        step(head)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_vox = 0
    for _ in range(args.steps):
        s.set_stiffness_phases(ph_host, Cp)     # H2D: phase ids
        out = step(head)
        for L in range(3):
            s.get_strain(L, E_host[L])          # D2H: strain fields
        s.get_ceff()
        e2e_vox += int(np.sum(out["iterations"])) * p.m
    torch.cuda.synchronize()
    e2e_t = time.perf_counter() - t0
    e2e = {"value": e2e_vox / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(p.m + 9 * 8 * 2 + Cp.nbytes),
           "d2h_bytes_per_step": int(E_host.numel() * 8 + 9 * 8)}

    # roofline of the dominant kernel of the headline mode, timed live with CUDA
    # events on the solver's stream (fh_solve's elapsed_ms, or fh_profile_passes)
    bulk = "fp64" if head == "fp64" else "fp32"
    g = {"nv": 3, "L": p.dims[-1], "dims": p.dims, "m": p.m, "nhalf": len(p.half_freqs())}
    per_iter = flops_per_launch(g, 1, "row") + flops_per_launch(g, 1, "green")
    peak = measured_fp_peak(bulk)
    if results[bulk]["path"] == "cluster-resident":
        out = s.solve(eps0, tol=args.tol, max_iter=20000, precision=prec[bulk])
        flops = per_iter * float(np.sum(out["iterations"]))
        dur_ms = out["elapsed_ms"]
        kernel = f"cluster_solve_2d<{'float' if bulk == 'fp32' else 'double'},3,{out['cluster']}> (one launch per solve, one cluster per load)"
        passes = None
    else:
        step(bulk)
        ms = s.profile_passes(3, prec[bulk], reps=50)
        kinds = [("row_pass", ms[0], flops_per_launch(g, 3, "row")),
                 ("line_pass_green", ms[1], flops_per_launch(g, 3, "green"))]
        dom = max(kinds, key=lambda k: k[1])
        kernel, dur_ms, flops = dom[0], dom[1], dom[2]
        passes = {k[0]: k[1] for k in kinds}
    achieved = flops / (dur_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak["tflops"],
                "unit": "TFLOP/s", "frac": achieved / peak["tflops"], "traffic": None,
                "peak_source": peak["source"] + " (of measured)", "duration_ms": dur_ms,
                "algorithmic_flops": flops, "passes_ms": passes}
    return results, e2e, roofline, clocks


def run_batched(fh, steps, cluster):
    """The batched workload: 512 seeded two-phase 2-D microstructures with N in
    {64,96,128,192,256} (half diagonal, half sheared M), 3 loads each, mixed
    precision to r <= 1e-6, solved with one fh_solve_batch call per step;
    compared with solving the same solvers one after another."""
    import torch
    solvers, ms = [], []
    t0 = time.perf_counter()
    for i in range(512):
        w = W.batch2d_item(i)
        p = fh.Pattern(w["M"])
        ids = W.phase_ids(p.points(), w["centres"], w["radii"])
        Cp = np.stack([fh.isotropic_stiffness(*fh.lame(E, nu), 2) for E, nu in w["phases"]])
        s = fh.Solver(p, fh.generator("dirichlet"), 3, torch.cuda.current_stream().cuda_stream)
        s.set_stiffness_phases(ids, Cp)
        s.set_reference(None)
        solvers.append(s)
        ms.append(p.m)
    setup = time.perf_counter() - t0
    eps = [np.eye(3)] * len(solvers)
    fh.solve_batch(solvers, eps, tol=1e-6, precision=fh.FH_PREC_MIXED, cluster=cluster)   # warm-up
    torch.cuda.synchronize()
    times, vox, launches = [], 0, 0
    for _ in range(steps):
        t0 = time.perf_counter()
        rc, outs = fh.solve_batch(solvers, eps, tol=1e-6, precision=fh.FH_PREC_MIXED, cluster=cluster)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        vox += sum(m * int(np.sum(o["iterations"])) for m, o in zip(ms, outs))
        launches += sum(o["kernel_launches"] + 1 for o in outs)
    t0 = time.perf_counter()
    seq_vox = 0
    for s, m in zip(solvers, ms):
        o = s.solve(np.eye(3), tol=1e-6, max_iter=20000, precision=fh.FH_PREC_MIXED, cluster=cluster)
        seq_vox += m * int(np.sum(o["iterations"]))
    torch.cuda.synchronize()
    seq = time.perf_counter() - t0
    paths = {}
    for o in outs:
        k = f"path{o['path']}/cluster{o['cluster']}"
        paths[k] = paths.get(k, 0) + 1
    for s in solvers:
        s.close()
    return {"workload": "batch2d: 512 microstructures, N in {64,96,128,192,256}, diag and sheared M, "
                        "Dirichlet, contrast log-U[5,200], 3 loads each, mixed precision, tol 1e-6",
            "value": vox / sum(times), "unit": UNIT, "ms_per_step": 1e3 * sum(times) / steps, "steps": steps,
            "points": int(sum(ms)), "status": int(rc), "launch_configs": paths,
            "sequential_value": seq_vox / seq, "sequential_ms": 1e3 * seq, "setup_s": setup,
            "timing": "host wall clock around fh_solve_batch (synchronous), L2 not flushed (1.6 M points x 3 "
                      "loads, working set > L2)", "gpu_launches": launches}


def hbm_peak():
    """Measured copy bandwidth of the GB300s (GB/s), else the fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (of fallback)"


def run_box3d(fh, args):
    """The 3-D workload: M = diag(n,n,n) (n = 128: m = 2 097 152), tensor-product
    box spline of order 2 with alias radius 4, 50 spheres (seed 3) at contrast
    50, the 6 Mandel unit loads.  The Gamma^p table is built once (a one-off
    precompute, timed separately); one step is one solve of all 6 loads to
    r <= tol.  Mixed and FP32 run `steps` steps, FP64 one.  Then the passes of
    one iteration are timed alone (fh_profile_passes, CUDA events) and divided
    into the bytes each must move: the HBM roofline of the 3-D kernels."""
    import torch
    n = args.box3d_n
    w = W.box3d(n=n)
    p = fh.Pattern(w["M"])
    ids = W.phase_ids(p.points(), w["centres"], w["radii"])
    Cp = np.stack([fh.isotropic_stiffness(*fh.lame(E, nu), 3) for E, nu in w["phases"]])
    stream = torch.cuda.current_stream().cuda_stream
    s = fh.Solver(p, fh.tensor_boxspline(3, 2, 4), 6, stream)
    s.set_stiffness_phases(ids, Cp)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.set_reference(None)
    e1.record()
    e1.synchronize()
    table_ms = e0.elapsed_time(e1)
    eps0 = np.eye(6)
    prec = {"fp64": fh.FH_PREC_FP64, "fp32": fh.FH_PREC_FP32, "mixed": fh.FH_PREC_MIXED}
    modes, launches = {}, 0
    wanted = [m for m in ("mixed", "fp32", "fp64") if m in args.box3d_modes.split(",")]
    for mode, steps in [(m, args.steps if m != "fp64" else 1) for m in wanted]:
        s.solve(eps0, tol=0.0, max_iter=5, precision=prec[mode])      # warm-up (graph capture)
        times, out = [], None
        for _ in range(steps):
            e0.record()
            out = s.solve(eps0, tol=args.tol, max_iter=20000, precision=prec[mode])
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        it = [int(x) for x in out["iterations"]]
        modes[mode] = {"time_to_tol_ms": float(np.median(times)), "iterations": it,
                       "ms_per_iteration": float(np.median(times)) / max(it),
                       "voxel_iterations_per_s": p.m * sum(it) / (float(np.median(times)) * 1e-3),
                       "status": int(out["status"]), "load_status": [int(x) for x in out["load_status"]],
                       "ceff": s.get_ceff().tolist()}
        if mode == "mixed":
            launches = out["kernel_launches"]
    if "fp64" in modes:
        C64 = np.array(modes["fp64"]["ceff"])
        for mode in modes:
            if mode != "fp64":
                modes[mode]["ceff_rel_err_vs_fp64"] = float(np.linalg.norm(np.array(modes[mode]["ceff"]) - C64)
                                                            / np.linalg.norm(C64))
    # per-pass roofline
    nhalf = len(p.half_freqs())
    peak, peak_src = hbm_peak()
    passes = {}
    for mode, rb, cb in [x for x in (("fp32", 4, 8), ("fp64", 8, 16)) if x[0] in wanted]:
        s.solve(eps0, tol=0.0, max_iter=3, precision=prec[mode])
        ms = s.profile_passes(6, prec[mode], reps=20)
        spec = 6 * 6 * nhalf * cb                       # all loads' half spectra, one way
        field = 6 * 6 * p.m * rb                        # all loads' strain fields, one way
        table = 21 * nhalf * rb
        bytes_ = {"row_pass": 2 * spec + 2 * field + p.m, "axis0_green_pass": 2 * spec + table,
                  "axis1_forward_pass": 2 * spec, "axis1_inverse_pass": 2 * spec}
        names = list(bytes_)
        passes[mode] = {k: {"ms": float(ms[i]), "bytes": int(bytes_[k]),
                            "gbs": bytes_[k] / (ms[i] * 1e-3) / 1e9,
                            "frac_of_hbm": bytes_[k] / (ms[i] * 1e-3) / 1e9 / peak} for i, k in enumerate(names)}
        tot_b = sum(bytes_.values())
        tot_ms = float(sum(ms))
        # the method's own minimum per iteration: read and write every strain
        # field once, the phase ids and the table once
        algo = 6 * 6 * p.m * rb * 2 + p.m + table
        passes[mode]["iteration"] = {"ms": tot_ms, "bytes": int(tot_b), "gbs": tot_b / (tot_ms * 1e-3) / 1e9,
                                     "frac_of_hbm": tot_b / (tot_ms * 1e-3) / 1e9 / peak,
                                     "algorithmic_bytes": int(algo),
                                     "algorithmic_gbs": algo / (tot_ms * 1e-3) / 1e9}
    s.close()
    return {"workload": f"box3d: M=diag({n},{n},{n}) (m={p.m}, grid {p.dims}), box spline order 2 alias radius 4 "
                        f"(729 aliases), 50 spheres r~U[0.05,0.1] seed 3, contrast 50, 6 Mandel unit loads, "
                        f"tol {args.tol}",
            "table_build_ms": table_ms, "modes": modes, "passes": passes, "hbm_peak_gbs": peak,
            "hbm_peak_source": peak_src, "gpu_launches_mixed_step": launches,
            "timing": "CUDA events on the solver's stream; working set (1.2 GB FP32) larger than L2"}


def measured_fp_peak(mode):
    """Dense peak of the arithmetic type measured here with cuBLAS (DGEMM / SGEMM without TF32)."""
    import torch
    dt = torch.float64 if mode == "fp64" else torch.float32
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    n = 8192 if mode == "fp64" else 8192
    a = torch.randn(n, n, dtype=dt, device="cuda")
    b = torch.randn(n, n, dtype=dt, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    torch.backends.cuda.matmul.allow_tf32 = prev
    del a, b
    return {"tflops": 2 * n ** 3 / (best * 1e-3) / 1e12,
            "source": f"measured here: cuBLAS {'DGEMM' if mode == 'fp64' else 'SGEMM (no TF32)'} {n}^3, best of 5"}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    from paper_1701_04685_gb300 import build
    build.build()
    if args.only_box3d:
        import torch
        torch.cuda.set_device(local_rank)
        import paper_1701_04685_gb300 as fh
        box = run_box3d(fh, args)
        if rank == 0:
            print(json.dumps({"box3d": box}), flush=True)
        return
    results, e2e, roofline, clocks = run_gpu(args, rank, world, local_rank)
    batched = None
    if not args.no_batched:
        import paper_1701_04685_gb300 as fh
        batched = run_batched(fh, min(args.steps, 3), args.batch_cluster)
    box = None
    if not args.no_box3d:
        import paper_1701_04685_gb300 as fh
        box = run_box3d(fh, args)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = oracle_sample(W.dlvp_sheared(), args.cpu_seconds)
    head = results[args.mode]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.mode == "fp64" else "f32",
        "precision_mode": args.mode,
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "mode": args.mode, "tol": args.tol,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "iterations_per_load": head["iterations"]},
        "time_to_tol_ms": head["ms_per_step"],
        "modes": results,
        "batched": batched,
        "box3d": box,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": head["gpu_launches"],
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
