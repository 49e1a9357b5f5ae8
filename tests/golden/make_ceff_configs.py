"""Write converged FP64 oracle C_eff of the 3-D, batched and learned-start workloads.

Calls only the oracle (and the seeded geometry of ``workloads``).  For every
microstructure the oracle's fixed point (Eq. (pde_coefficients), Sec. 4) is run
per load case, first to the Cauchy residual 1e-6 of the benchmark (the C_eff
and iteration counts at that stop are stored too), then continued from that
iterate to r <= 1e-11, far below the benchmark tolerance; the stored
"converged" C_eff is <C:(E+eps0)> of that last iterate (Sec. 3.1).

  box3d   M = diag(128,128,128), tensor box spline of order 2, alias radius 4,
          50 spheres, contrast 50, 6 loads            -> ceff_box3d.txt
  batch   20 of the 512 batched 2-D microstructures: for each N in
          {64,96,128,192,256} and each shape (diagonal, sheared), the items
          of lowest and highest contrast; Dirichlet, 3 loads -> ceff_batch2d.txt
  fno3d   held-out seeds 100000..100003 of the learned-start workload,
          M = diag(64,64,64), Dirichlet, 6 loads      -> ceff_fno3d.txt

Usage: python tests/golden/make_ceff_configs.py box3d|batch|fno3d [--procs N]
The work is spread over processes (spawn); the 3-D runs take tens of minutes.
``tests/parity.py::read_golden_blocks`` parses the files.
"""
import argparse
import multiprocessing as mp
import os
import sys
import tempfile

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import generators as OG, green as OGr, material as OM, scheme as OS  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
TOL_BENCH = 1e-6
TOL_CONVERGED = 1e-11
MAX_ITER = 200000


def oracle_generator(spec, d):
    if spec["kind"] == "dirichlet":
        return OG.Generator("dirichlet")
    if spec["kind"] == "dlvp":
        return OG.Generator("dlvp", alpha=spec["alpha"])
    return OG.Generator("boxspline", xi=OG.tensor_boxspline_xi(d, spec["order"]), radius=spec["radius"])


def materials(w):
    d = w["d"]
    lm = [OM.lame(E, nu) for E, nu in w["phases"]]
    Cp = np.stack([OM.isotropic_mandel(l, m, d) for l, m in lm])
    l0, m0 = OM.reference_medium_ms([l for l, _ in lm], [m for _, m in lm])
    return Cp, OM.isotropic_mandel(l0, m0, d)


def _table_chunk(args):
    M, spec, d, C0, fpath, lo, hi = args
    freqs = np.load(fpath, mmap_mode="r")[lo:hi]
    return lo, OGr.gamma_p_table(M, oracle_generator(spec, d), C0, np.array(freqs))


def _solve_loads(args):
    """Both stops of the oracle for the given loads of one microstructure."""
    w, loads, gp_path = args
    d = w["d"]
    nv = 3 if d == 2 else 6
    T = OS.SNFTransform(w["M"])
    Cp, C0 = materials(w)
    ids = W.phase_ids(T.points / T.D, w["centres"], w["radii"])
    if gp_path is None:
        Gp = OGr.gamma_p_table(w["M"], oracle_generator(w["generator"], d), C0, T.freqs)
    else:
        Gp = np.load(gp_path, mmap_mode="r")
    C = Cp[ids]
    out = []
    for L in loads:
        e0 = np.eye(nv)[L:L + 1]
        a = OS.solve(T, Gp, C, C0, e0, tol=TOL_BENCH, max_iter=MAX_ITER)
        b = OS.solve(T, Gp, C, C0, e0, tol=TOL_CONVERGED, max_iter=MAX_ITER, E_init=a["E"])
        out.append((L, int(a["iters"][0]), a["mean_stress"][0], int(a["iters"][0] + b["iters"][0]),
                    float(b["resid"][0][-1]), b["mean_stress"][0]))
    return out


def _assemble(w, rows):
    nv = 3 if w["d"] == 2 else 6
    rows = sorted(rows)
    S_bench = np.stack([r[2] for r in rows])
    S_conv = np.stack([r[5] for r in rows])
    return {"iters_bench": [r[1] for r in rows], "iters_conv": [r[3] for r in rows],
            "resid_conv": [r[4] for r in rows],
            "ceff_bench": OS.effective_stiffness(S_bench, np.eye(nv)),
            "ceff_conv": OS.effective_stiffness(S_conv, np.eye(nv))}


def _write_block(f, name, res):
    f.write(f"[{name}]\n")
    f.write("iterations_to_1e-6 " + " ".join(str(i) for i in res["iters_bench"]) + "\n")
    f.write("iterations_to_1e-11 " + " ".join(str(i) for i in res["iters_conv"]) + "\n")
    f.write("ceff_converged\n")
    for row in res["ceff_conv"]:
        f.write(" ".join(f"{v:.17e}" for v in row) + "\n")
    f.write("ceff_at_1e-6\n")
    for row in res["ceff_bench"]:
        f.write(" ".join(f"{v:.17e}" for v in row) + "\n")


def run_box3d(procs):
    w = W.box3d()
    T = OS.SNFTransform(w["M"])
    _, C0 = materials(w)
    tmp = tempfile.mkdtemp(prefix="ceff_box3d_")
    fpath = os.path.join(tmp, "freqs.npy")
    np.save(fpath, T.freqs)
    n, step = T.m, 16384
    Gp = np.lib.format.open_memmap(os.path.join(tmp, "gp.npy"), mode="w+", dtype=np.float64, shape=(n, 6, 6))
    ctx = mp.get_context("spawn")
    jobs = [(w["M"], w["generator"], 3, C0, fpath, lo, min(n, lo + step)) for lo in range(0, n, step)]
    with ctx.Pool(procs) as pool:
        for lo, block in pool.imap_unordered(_table_chunk, jobs):
            Gp[lo:lo + len(block)] = block
    Gp.flush()
    del Gp
    with ctx.Pool(min(procs, 6)) as pool:
        parts = pool.map(_solve_loads, [(w, [L], os.path.join(tmp, "gp.npy")) for L in range(6)])
    res = _assemble(w, [r for p in parts for r in p])
    path = os.path.join(HERE, "ceff_box3d.txt")
    with open(path, "w") as f:
        f.write("# C_eff (Mandel 6x6) of workloads.box3d (M=diag(128,128,128), box spline order 2, alias radius 4,\n"
                "# 50 spheres seed 3, contrast 50) from the FP64 oracle: per load, the fixed point stopped at\n"
                "# r <= 1e-6 and continued to r <= 1e-11.  Written by tests/golden/make_ceff_configs.py box3d\n")
        _write_block(f, "box3d", res)
    print(path)


def batch_selection():
    """Items of lowest and highest contrast for every (N, shape) of the 512 batched workloads."""
    groups = {}
    for i in range(512):
        w = W.batch2d_item(i)
        key = (w["M"][0][0], w["M"][0][1] != 0)
        c = w["phases"][1][0]
        groups.setdefault(key, []).append((c, i))
    sel = set()
    for key in sorted(groups):
        g = sorted(groups[key])
        sel.add(g[0][1])
        sel.add(g[-1][1])
    return sorted(sel)


def run_batch(procs):
    items = batch_selection()
    ctx = mp.get_context("spawn")
    jobs = [(W.batch2d_item(i), [L], None) for i in items for L in range(3)]
    with ctx.Pool(procs) as pool:
        parts = pool.map(_solve_loads, jobs, chunksize=1)
    path = os.path.join(HERE, "ceff_batch2d.txt")
    with open(path, "w") as f:
        f.write("# C_eff (Mandel 3x3) of 20 items of workloads.batch2d_item (Dirichlet, 3 loads): for each N and\n"
                "# shape the lowest- and highest-contrast item; FP64 oracle stopped at r <= 1e-6 and continued\n"
                "# to r <= 1e-11.  Written by tests/golden/make_ceff_configs.py batch\n")
        for k, i in enumerate(items):
            w = W.batch2d_item(i)
            res = _assemble(w, [r for p in parts[3 * k:3 * k + 3] for r in p])
            _write_block(f, f"item {i} M={w['M']} contrast={w['phases'][1][0]:.6g}", res)
    print(path)


FNO_SEEDS = [100000, 100001, 100002, 100003]


def run_fno3d(procs):
    ctx = mp.get_context("spawn")
    jobs = [(W.fno3d_item(s), [L], None) for s in FNO_SEEDS for L in range(6)]
    with ctx.Pool(procs) as pool:
        parts = pool.map(_solve_loads, jobs, chunksize=1)
    path = os.path.join(HERE, "ceff_fno3d.txt")
    with open(path, "w") as f:
        f.write("# C_eff (Mandel 6x6) of held-out learned-start workloads workloads.fno3d_item(seed)\n"
                "# (M=diag(64,64,64), Dirichlet, 6 loads); FP64 oracle stopped at r <= 1e-6 and continued to\n"
                "# r <= 1e-11.  Written by tests/golden/make_ceff_configs.py fno3d\n")
        for k, s in enumerate(FNO_SEEDS):
            w = W.fno3d_item(s)
            res = _assemble(w, [r for p in parts[6 * k:6 * k + 6] for r in p])
            _write_block(f, f"seed {s} contrast={w['phases'][1][0]:.6g}", res)
    print(path)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["box3d", "batch", "fno3d"])
    ap.add_argument("--procs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    a = ap.parse_args()
    {"box3d": run_box3d, "batch": run_batch, "fno3d": run_fno3d}[a.what](a.procs)
