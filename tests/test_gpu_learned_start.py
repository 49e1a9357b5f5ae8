"""Learned start: trained on the solver's own solutions, used as the starting strain.

A small network (16^3 grid, width 16, 4 modes, 3 layers) is trained on strain
fields the solver produced for 48 seeded random-sphere microstructures (x 6
unit loads) and used as the starting strain of the fixed point and of
BiCGStab on 8 unseen seeds.  The solve still iterates to r <= 1e-6, so the
network may change the iteration count but not the answer: every
learned-start solve converges with the same C_eff as the zero start.  The
start a validation split of the held-out seeds selects is the one the test
seeds then use, and it never does worse than the zero start on the validation
seeds: the fallback to the zero start is taken exactly when the network does
not pay there."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_learned_start_converges_to_the_same_answer_and_the_policy_follows_the_gain():
    import torch
    assert torch.cuda.is_available()
    from paper_1701_04685_gb300 import build
    build.build()
    import paper_1701_04685_gb300 as fh
    import workloads as W
    from paper_1701_04685_gb300 import learned_start as LS
    n = 16
    net = fh.FNO(n, 1, 36, 16, 4, 3, max_batch=4)
    LS.init_params(net, np.random.default_rng(0))
    X, T, _ = LS.generate(net, range(48), n)
    hist = LS.train(net, X, T, epochs=60, lr=5e-3, batch=4)
    assert hist[-1] < 0.6 * hist[0]
    methods = (0, 1)
    rows = LS.evaluate(net, range(100000, 100008), n, methods=methods)
    s = LS.summary(rows, methods, val=4)
    print("learned start:", s)
    for m in methods:
        r = s[f"method{m}"]
        va = rows[:4]
        zero = np.mean([np.mean(q[f"m{m}"]["ms_zero"]) for q in va])
        lrn = np.mean([np.mean(q[f"m{m}"]["ms_learned"]) for q in va])
        assert r["policy_start"] == ("learned" if lrn < zero else "zero")
        picked = {"learned": lrn, "zero": zero}[r["policy_start"]]
        assert picked <= zero
        if r["policy_start"] == "zero":
            assert r["test_mean_iters_policy"] == r["test_mean_iters_zero"]
    # same answer from either start, for both methods
    x = torch.empty((1, 1, n ** 3), dtype=torch.float32, device="cuda")
    y = torch.empty((1, 36, n ** 3), dtype=torch.float32, device="cuda")
    for seed, method in ((100000, 0), (100003, 1)):
        sv, ids, logE = LS.make_solver(W.fno3d_item(seed, n=n))
        z = sv.solve(np.eye(6), tol=1e-8, max_iter=20000, precision=fh.FH_PREC_FP64, method=method)
        C0 = sv.get_ceff()
        net.make_input(torch.from_numpy(ids).cuda(), logE, np.zeros(6), x[0])
        net.forward(x, y)
        for L in range(6):
            fh.set_strain_f32(sv, L, y[0, 6 * L:6 * L + 6])
        o = sv.solve(np.eye(6), tol=1e-8, max_iter=20000, precision=fh.FH_PREC_FP64, init=1, method=method)
        assert o["status"] == 0 and z["status"] == 0
        assert np.abs(sv.get_ceff() - C0).max() / np.abs(C0).max() < 1e-6
        sv.close()
