"""Sweep of the de la Vallee Poussin parameter alpha (the paper's numerical
section varies alpha between the modified Dirichlet kernel, alpha = 0, and the
Fejer kernel, alpha = 1/2).

For each alpha the solver builds the periodised Green operator of the dlVP
generator with equal half ramp widths in every direction, solves all loads of
one microstructure to a Cauchy tolerance, and records the effective stiffness,
the iteration counts and the solve time.  The paper compares each alpha's
effective quantities with an analytic (Hashin) solution; that solution's
inputs are not available here, so the sweep reports the effective stiffness
itself and its change relative to alpha = 0.

Run ``python -m paper_1701_04685_gb300.alpha_sweep`` for the default sweep on
the anisotropic benchmark pattern (M = [[128, 32], [0, 128]], 20 disks at
contrast 100), alpha = 0, 0.05, ..., 0.5, FP64, tolerance 1e-8.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

import workloads as W

from . import FH_PREC_FP64, FH_PREC_FP32, FH_PREC_MIXED, Pattern, Solver, generator, isotropic_stiffness, lame


def sweep(w, alphas, tol=1e-8, precision=FH_PREC_FP64, max_iter=20000, stream=0):
    """One solve per alpha of workload `w` (a dict with M, phases, centres,
    radii); returns a list of {alpha, ceff, iterations, status, ms}."""
    d = len(w["M"])
    nv = 3 if d == 2 else 6
    p = Pattern(w["M"])
    ids = W.phase_ids(p.points(), w["centres"], w["radii"])
    Cp = np.stack([isotropic_stiffness(*lame(E, nu), d) for E, nu in w["phases"]])
    rows = []
    for a in alphas:
        s = Solver(p, generator("dlvp", alpha=[float(a)] * d), nv, stream)
        s.set_stiffness_phases(ids, Cp)
        s.set_reference(None)
        t0 = time.perf_counter()
        out = s.solve(np.eye(nv), tol=tol, max_iter=max_iter, precision=precision)
        ms = 1e3 * (time.perf_counter() - t0)
        rows.append({"alpha": float(a), "ceff": s.get_ceff().tolist(),
                     "iterations": [int(i) for i in out["iterations"]], "status": int(out["status"]),
                     "ms": ms})
        s.close()
    C0 = np.array(rows[0]["ceff"])
    for r in rows:
        r["ceff_change_vs_first"] = float(np.linalg.norm(np.array(r["ceff"]) - C0) / np.linalg.norm(C0))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--alphas", default="0,0.05,0.1,0.15,0.2,0.25,0.3,0.35,0.4,0.45,0.5")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    prec = {"fp64": FH_PREC_FP64, "fp32": FH_PREC_FP32, "mixed": FH_PREC_MIXED}[a.precision]
    rows = sweep(W.dlvp_sheared(), [float(x) for x in a.alphas.split(",")], tol=a.tol, precision=prec)
    for r in rows:
        C = np.array(r["ceff"])
        print(json.dumps({"alpha": r["alpha"], "C11": C[0, 0], "C22": C[1, 1], "C12": C[0, 1], "C33": C[2, 2],
                          "change_vs_alpha0": r["ceff_change_vs_first"], "iterations": r["iterations"],
                          "ms": round(r["ms"], 2)}), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rows, f)


if __name__ == "__main__":
    main()
