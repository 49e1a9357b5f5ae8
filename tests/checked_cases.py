"""Small solves over every kernel family of the solver, for the checked build.

``run_cases(fh)`` runs them with whatever library the binding loaded and
returns the results by name; run as a script (``python checked_cases.py
OUT.npz`` with FH_CHECKED=1) it loads the checked build, records the self
test of the index checks, and saves the results for the test in
``test_gpu_checked.py`` to compare with the normal build."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import workloads as W  # noqa: E402
from parity import product_generator  # noqa: E402


def _solver(fh, M, gen, phases, centres, radii, nload):
    p = fh.Pattern(M)
    d = len(M)
    ids = W.phase_ids(p.points(), np.asarray(centres, float).reshape(-1, d), np.asarray(radii, float))
    Cp = np.stack([fh.isotropic_stiffness(*fh.lame(E, nu), d) for E, nu in phases])
    s = fh.Solver(p, gen, nload)
    s.set_stiffness_phases(ids, Cp)
    s.set_reference(None)
    return s, p


def _collect(out, name, s, nload, res):
    out[name + "/E"] = np.stack([s.get_strain(L) for L in range(nload)])
    out[name + "/iters"] = np.asarray(res["iterations"])
    out[name + "/hist"] = np.concatenate([s.get_residuals(L) for L in range(nload)])


def run_cases(fh):
    out = {}
    ball2 = (np.full((1, 2), 0.07), [0.27])
    ball3 = (np.full((1, 3), 0.07), [0.3])
    two = [(1.0, 0.3), (20.0, 0.3)]
    # 2-D: the cluster solve (default path) and the whole-GPU passes
    for path, prec in ((0, 0), (1, 0), (0, 1)):
        s, _ = _solver(fh, [[32, 8], [0, 32]], fh.generator("dlvp", alpha=[0.25, 0.2]), two, *ball2, 3)
        r = s.solve(np.eye(3), tol=0.0, max_iter=12, precision=prec, path=path)
        _collect(out, f"2d_path{path}_prec{prec}", s, 3, r)
        s.close()
    # 3-D block passes (FP64) on a sheared pattern, FP32 rows of 64 / 128 with
    # the two-step and the warp-exchange column passes
    cases3 = [
        ("3d_sheared_fp64", [[6, 2, 0], [0, 6, 2], [0, 0, 10]], fh.generator("dlvp", alpha=[0.2, 0.3, 0.1]), 0, 0),
        ("3d_cube32_fp32", [[32, 0, 0], [0, 32, 0], [0, 0, 32]], fh.generator("dlvp", alpha=[0.25] * 3), 1, 0),
        ("3d_cube64_fp32", [[64, 0, 0], [0, 64, 0], [0, 0, 64]], fh.generator("dirichlet"), 1, 0),
        ("3d_cube64_fp32_warpcols", [[64, 0, 0], [0, 64, 0], [0, 0, 64]], fh.generator("dirichlet"), 1, 7),
        ("3d_rows128_fp32", [[2, 0, 0], [0, 4, 0], [0, 0, 128]], fh.generator("dirichlet"), 1, 0),
    ]
    for name, M, gen, prec, tune in cases3:
        s, _ = _solver(fh, M, gen, two, *ball3, 2)
        eps0 = np.eye(6)[[0, 3]]
        r = s.solve(eps0, tol=0.0, max_iter=8, precision=prec, tune=tune)
        _collect(out, name, s, 2, r)
        s.close()
    # BiCGStab (FP64 and FP32) on the passes
    for prec in (0, 1):
        s, _ = _solver(fh, [[8, 0, 0], [0, 8, 0], [0, 0, 64]], fh.generator("dlvp", alpha=[0.25] * 3), two, *ball3, 2)
        r = s.solve(np.eye(6)[[1, 4]], tol=0.0, max_iter=5, precision=prec, method=1)
        _collect(out, f"bicgstab_prec{prec}", s, 2, r)
        s.close()
    # a batch of 2-D solvers (cluster task queue)
    solvers = []
    for i in range(3):
        w = W.batch2d_item(i)
        s, _ = _solver(fh, w["M"], product_generator(fh, w["generator"], 2), w["phases"], w["centres"], w["radii"], 3)
        solvers.append(s)
    rc, res = fh.solve_batch(solvers, [np.eye(3)] * 3, tol=0.0, max_iter=6, precision=0)
    for i, (s, r) in enumerate(zip(solvers, res)):
        _collect(out, f"batch{i}", s, 3, r)
        s.close()
    # point-by-point stiffness (more than 16 matrices), FP64 and FP32
    rng = np.random.default_rng(3)
    for prec in (0, 1):
        p = fh.Pattern([[16, 0, 0], [0, 16, 0], [0, 0, 32]])
        s = fh.Solver(p, fh.generator("dirichlet"), 1)
        Ey = 1.0 + 9.0 * rng.random(p.m)
        C = np.stack([fh.isotropic_stiffness(*fh.lame(E, 0.3), 3) for E in Ey])
        s.set_stiffness_field(C)
        s.set_reference(None)
        r = s.solve(np.eye(6)[[2]], tol=0.0, max_iter=6, precision=prec)
        _collect(out, f"field_prec{prec}", s, 1, r)
        s.close()
    return out


def main(path):
    import paper_1701_04685_gb300 as fh
    out = {"checked": np.asarray(int(fh.checked_build()))}
    rc, msg = fh.check_selftest()
    out["selftest_status"] = np.asarray(rc)
    out["selftest_message"] = np.asarray(msg)
    out.update(run_cases(fh))
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])
