"""Learned start: trained on the solver's own solutions, used as the starting strain.

A small network (16^3 grid, width 16, 4 modes, 3 layers) is trained on strain
fields the solver produced for 48 seeded random-sphere microstructures (x 6
unit loads) and used as the starting strain on 6 unseen seeds.  The scheme
still iterates to r <= 1e-6, so the network may change the iteration count but
not the answer: the test checks that every learned-start solve converges to the
same tolerance with the same C_eff as the zero start, and reports the iteration
counts of both starts (the gain is measured, not assumed)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_learned_start_converges_to_the_same_answer_and_reports_the_gain():
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
    rows = LS.evaluate(net, range(100000, 100006), n)
    s = LS.summary(rows)
    print("learned start:", s)
    assert s["mean_iters_zero"] > 0 and s["mean_iters_learned"] > 0
    # same answer from either start
    x = torch.empty((1, 1, n ** 3), dtype=torch.float32, device="cuda")
    y = torch.empty((1, 36, n ** 3), dtype=torch.float32, device="cuda")
    for seed in (100000, 100003):
        sv, ids, logE = LS.make_solver(W.fno3d_item(seed, n=n))
        z = sv.solve(np.eye(6), tol=1e-8, max_iter=20000, precision=fh.FH_PREC_FP64)
        C0 = sv.get_ceff()
        net.make_input(torch.from_numpy(ids).cuda(), logE, np.zeros(6), x[0])
        net.forward(x, y)
        for L in range(6):
            fh.set_strain_f32(sv, L, y[0, 6 * L:6 * L + 6])
        o = sv.solve(np.eye(6), tol=1e-8, max_iter=20000, precision=fh.FH_PREC_FP64, init=1)
        assert o["status"] == 0 and z["status"] == 0
        assert np.abs(sv.get_ceff() - C0).max() / np.abs(C0).max() < 1e-6
        sv.close()
