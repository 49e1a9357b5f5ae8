"""Learned starting strain for the Basic Scheme: data, training, evaluation.

The Fourier neural operator of ``fh_fno_*`` is trained on strain fields that
the solver itself produces for seeded random-sphere microstructures (3-D,
M = diag(n, n, n), Dirichlet kernel), then used as the starting strain of the
fixed point or of BiCGStab.  The solve still runs to the same Cauchy
tolerance, so the network can only save iterations; the zero start is the
fallback: for each solver method a validation split of held-out seeds decides
whether the learned start pays (mean time to tolerance, inference included),
and the other seeds report what that choice gives.

The solution is linear in the macroscopic strain, E = sum_j eps0_j E^(j), so
the network maps the modulus field log10 E(x) (one input channel) to the six
unit-load fields E^(j) at once (36 output channels, load-major); the start for
a macroscopic strain eps0 is the corresponding combination.

Workload (``workloads.fno3d_item``): spheres with radii U[0.06, 0.12] added
until a volume fraction drawn from U[0.1, 0.35], contrast U[10, 100], nu = 0.3.
Every microstructure is solved for the six Mandel unit strains at once, which
gives six training solutions per solve.

Run ``python -m paper_1701_04685_gb300.learned_start --n 64 --train 683 --test 256``
for the full experiment (4098 training solutions, 256 held-out seeds x 6 loads).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

import workloads as W

from . import (FH_PREC_MIXED, FNO, Pattern, Solver, generator, get_strain_f32, isotropic_stiffness, lame,
               set_strain_f32)


def init_params(net, rng):
    """Scaled random initial weights (parameter order of fh_fno_set_params)."""
    W, cin, cout, L, m = net.width, net.cin, net.cout, net.layers, net.modes
    nm = 4 * m ** 3
    parts = [rng.standard_normal(W * cin) / np.sqrt(cin), np.zeros(W),
             rng.standard_normal(L * W * W) / np.sqrt(W), np.zeros(L * W),
             rng.standard_normal(L * nm * W * W) / W, rng.standard_normal(L * nm * W * W) / W,
             0.1 * rng.standard_normal(cout * W) / np.sqrt(W), np.zeros(cout)]
    flat = np.concatenate(parts).astype(np.float32)
    assert flat.size == net.nparam
    net.set_params(flat)


def make_solver(item, stream=0):
    p = Pattern(item["M"])
    ids = W.phase_ids(p.points(), item["centres"], item["radii"])
    Cp = np.stack([isotropic_stiffness(*lame(E, nu), 3) for E, nu in item["phases"]])
    s = Solver(p, generator("dirichlet"), 6, stream)
    s.set_stiffness_phases(ids, Cp)
    s.set_reference(None)
    logE = np.log10([E for E, _ in item["phases"]])
    return s, ids, logE


def generate(net, seeds, n, tol=1e-6, method=0):
    """Inputs (S, 1, n^3) and targets (S, 36, n^3) on the device, one sample per seed
    holding the six unit-load solutions (solved with the given method: the fixed
    point or BiCGStab give the same solution to the tolerance)."""
    import torch
    S = len(seeds)
    X = torch.empty((S, 1, n ** 3), dtype=torch.float32, device="cuda")
    T = torch.empty((S, 36, n ** 3), dtype=torch.float32, device="cuda")
    iters = []
    for j, seed in enumerate(seeds):
        s, ids, logE = make_solver(W.fno3d_item(seed, n=n))
        out = s.solve(np.eye(6), tol=tol, max_iter=20000, precision=FH_PREC_MIXED, method=method)
        iters.append([int(i) for i in out["iterations"]])
        net.make_input(torch.from_numpy(ids).cuda(), logE, np.zeros(6), X[j])
        for L in range(6):
            get_strain_f32(s, L, T[j, 6 * L:6 * L + 6])
        s.close()
    return X, T, np.array(iters)


def train(net, X, T, epochs, lr=2e-3, batch=4, seed=0, log=None):
    rng = np.random.default_rng(seed)
    S = X.shape[0]
    step, hist = 0, []
    for ep in range(epochs):
        perm = rng.permutation(S)
        tot = 0.0
        for b0 in range(0, S - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb = X[idx].contiguous()
            tb = T[idx].contiguous()
            net.zero_grad()
            tot += net.loss_grad(xb, tb)
            step += 1
            lr_t = lr * 0.5 * (1 + np.cos(np.pi * min(1.0, step / max(1, epochs * (S // batch)))))
            net.adam_step(lr_t, step)
        hist.append(tot / max(1, S // batch))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def evaluate(net, seeds, n, tol=1e-6, methods=(0,)):
    """Iterations and time to tolerance per held-out seed, zero start vs learned start,
    for each solver method (0: the fixed point, 1: BiCGStab), mixed precision."""
    import torch
    rows = []
    x = torch.empty((1, 1, n ** 3), dtype=torch.float32, device="cuda")
    y = torch.empty((1, 36, n ** 3), dtype=torch.float32, device="cuda")
    for seed in seeds:
        s, ids, logE = make_solver(W.fno3d_item(seed, n=n))
        ph = torch.from_numpy(ids).cuda()
        row = {"seed": int(seed)}
        for method in methods:
            z = s.solve(np.eye(6), tol=tol, max_iter=20000, precision=FH_PREC_MIXED, method=method)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            net.make_input(ph, logE, np.zeros(6), x[0])
            net.forward(x, y)
            for L in range(6):                       # unit load L: its block of six channels
                set_strain_f32(s, L, y[0, 6 * L:6 * L + 6])
            torch.cuda.synchronize()
            t_inf = time.perf_counter() - t0
            lrn = s.solve(np.eye(6), tol=tol, max_iter=20000, precision=FH_PREC_MIXED, init=1, method=method)
            row[f"m{method}"] = {"iters_zero": [int(i) for i in z["iterations"]],
                                 "iters_learned": [int(i) for i in lrn["iterations"]],
                                 "ms_zero": z["elapsed_ms"], "ms_learned": lrn["elapsed_ms"] + 1e3 * t_inf,
                                 "ms_inference": 1e3 * t_inf}
        rows.append(row)
        s.close()
    return rows


def summary(rows, methods=(0,), val=0):
    """Means over seeds and loads per method, and the start a validation split selects.

    The first ``val`` seeds choose, per method, the start (learned or zero) with
    the smaller mean time to tolerance (inference included); the remaining seeds
    report what that choice gives: the fallback to the zero start is taken
    whenever the network does not pay on held-out data."""
    out = {"seeds": len(rows), "loads": 6, "validation_seeds": val}
    for m in methods:
        def mean(key, rs):
            return float(np.mean([np.mean(r[f"m{m}"][key]) for r in rs]))
        va, te = rows[:val], (rows[val:] if val < len(rows) else rows)
        use_learned = bool(val > 0 and mean("ms_learned", va) < mean("ms_zero", va))
        pick = "learned" if use_learned else "zero"
        out[f"method{m}"] = {
            "mean_iters_zero": mean("iters_zero", rows), "mean_iters_learned": mean("iters_learned", rows),
            "iteration_saving": 1 - mean("iters_learned", rows) / mean("iters_zero", rows),
            "mean_ms_zero": mean("ms_zero", rows), "mean_ms_learned_incl_inference": mean("ms_learned", rows),
            "time_saving": 1 - mean("ms_learned", rows) / mean("ms_zero", rows),
            "policy_start": pick,
            "test_mean_iters_zero": mean("iters_zero", te), "test_mean_iters_policy": mean(f"iters_{pick}", te),
            "test_mean_ms_zero": mean("ms_zero", te), "test_mean_ms_policy": mean(f"ms_{pick}", te)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--train", type=int, default=683, help="training microstructures (x6 loads)")
    ap.add_argument("--test", type=int, default=256)
    ap.add_argument("--width", type=int, default=32)
    ap.add_argument("--modes", type=int, default=12)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--methods", default="0,1", help="solver methods to evaluate (0 fixed point, 1 BiCGStab)")
    ap.add_argument("--val", type=int, default=32, help="held-out seeds that choose the start per method")
    ap.add_argument("--gen-method", type=int, default=1, help="solver method producing the training solutions")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    methods = tuple(int(v) for v in a.methods.split(","))
    import torch
    log = lambda s: print(s, flush=True)  # noqa: E731
    net = FNO(a.n, 1, 36, a.width, min(a.modes, a.n // 2), a.layers, max_batch=a.batch)
    init_params(net, np.random.default_rng(1234))
    t0 = time.perf_counter()
    X, T, it_train = generate(net, range(a.train), a.n, method=a.gen_method)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    log(f"generated {6 * X.shape[0]} solutions in {t_gen:.1f} s (mean iterations {it_train.mean():.1f})")
    t0 = time.perf_counter()
    hist = train(net, X, T, a.epochs, a.lr, a.batch, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    log(f"trained {a.epochs} epochs in {t_train:.1f} s")
    del X, T
    rows = evaluate(net, range(100000, 100000 + a.test), a.n, methods=methods)
    res = {"config": vars(a), "generate_s": t_gen, "train_s": t_train, "loss_history": hist,
           "summary": summary(rows, methods, a.val)}
    log(json.dumps(res["summary"]))
    if a.out:
        with open(a.out, "w") as f:
            json.dump({**res, "rows": rows}, f)


if __name__ == "__main__":
    main()
