"""Batched solves (fh_solve_batch) over microstructures of uneven pattern sizes."""
import numpy as np
import pytest

import workloads as W
from parity import Case, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fh():
    import torch
    assert torch.cuda.is_available()
    from paper_1701_04685_gb300 import build
    build.build()
    import paper_1701_04685_gb300 as fh
    return fh


def _items(idx):
    return [W.batch2d_item(i) for i in idx]


def test_batch_equals_individual_solves(fh):
    """Every solver of a heterogeneous batch (sizes 64^2..256^2, diagonal and sheared M)
    reaches bitwise the same strain as when it is solved alone."""
    ws = _items(range(8))
    cases = [Case.from_workload(w) for w in ws]
    solvers = [c.product(fh) for c in cases]
    eps0 = [c.eps0 for c in cases]
    rc, outs = fh.solve_batch(solvers, eps0, tol=0.0, max_iter=30, precision=fh.FH_PREC_FP64)
    batched = [[s.get_strain(L).copy() for L in range(3)] for s in solvers]
    for s, c, b, o in zip(solvers, cases, batched, outs):
        alone = s.solve(c.eps0, tol=0.0, max_iter=30, precision=fh.FH_PREC_FP64)
        assert list(o["iterations"]) == list(alone["iterations"]) == [30, 30, 30]
        for L in range(3):
            assert np.array_equal(s.get_strain(L), b[L])


def test_batch_matches_oracle(fh):
    """Two batch members checked element by element against the FP64 oracle."""
    ws = _items([0, 1, 2, 3])
    cases = [Case.from_workload(w) for w in ws]
    solvers = [c.product(fh) for c in cases]
    fh.solve_batch(solvers, [c.eps0 for c in cases], tol=0.0, max_iter=20, precision=fh.FH_PREC_FP64)
    for k in (0, 1):
        ref = cases[k].oracle_solve(tol=0.0, max_iter=20)
        assert cases[k].strain_error(solvers[k], ref["E"]) < 1e-10


def test_batch_mixed_converges(fh):
    """Mixed-precision batch to r <= 1e-6: every load converges, C_eff symmetric and
    positive definite, and every load's last (FP64) Cauchy residual meets the tolerance
    the batch was solved to."""
    ws = _items(range(12))
    cases = [Case.from_workload(w) for w in ws]
    solvers = [c.product(fh) for c in cases]
    rc, outs = fh.solve_batch(solvers, [c.eps0 for c in cases], tol=1e-6, max_iter=20000,
                              precision=fh.FH_PREC_MIXED)
    assert rc == 0
    for s, o in zip(solvers, outs):
        assert np.all(o["load_status"] == 0)
        assert np.all(o["residual"] <= 1e-6)
        C = s.get_ceff()
        assert rel(C, C.T) < 1e-5
        assert np.linalg.eigvalsh(0.5 * (C + C.T)).min() > 0


def test_batch_rejects_duplicates_and_bad_args(fh):
    c = Case.from_workload(W.batch2d_item(0))
    s = c.product(fh)
    with pytest.raises(fh.FhError):
        fh.solve_batch([s, s], [c.eps0, c.eps0], tol=0.0, max_iter=2)
    with pytest.raises(fh.FhError):
        fh.solve_batch([s], [c.eps0], tol=-1.0, max_iter=2)
