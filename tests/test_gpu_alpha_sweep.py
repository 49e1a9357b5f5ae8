"""The dlVP alpha sweep (paper_1701_04685_gb300.alpha_sweep) against the oracle:
alpha = 0 is the modified Dirichlet kernel, and the converged effective
stiffness at each alpha of a small sheared pattern agrees with the oracle's."""
import numpy as np
import pytest

from oracle import scheme as OS
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


def _workload():
    return {"M": [[16, 4], [0, 20]], "phases": [(1.0, 0.3), (25.0, 0.3)],
            "centres": np.array([[0.1, -0.05], [-0.3, 0.25]]), "radii": np.array([0.22, 0.12])}


def test_alpha_zero_is_the_modified_dirichlet_kernel(fh):
    """Half ramp width 0 gives g = 1 inside, 1/2 on the boundary of the
    frequency cube: the same Gamma^p table and the same solution as the
    Dirichlet generator (modified on the boundary)."""
    w = _workload()
    a = Case(w["M"], {"kind": "dlvp", "alpha": [0.0, 0.0]}, w["phases"], w["centres"], w["radii"])
    b = Case(w["M"], {"kind": "dirichlet"}, w["phases"], w["centres"], w["radii"])
    sa, sb = a.product(fh), b.product(fh)
    assert rel(sa.get_green(), sb.get_green()) < 1e-14
    sa.solve(a.eps0, tol=1e-10, max_iter=5000)
    sb.solve(b.eps0, tol=1e-10, max_iter=5000)
    assert rel(sa.get_ceff(), sb.get_ceff()) < 1e-12


def test_sweep_effective_stiffness_matches_oracle(fh):
    from paper_1701_04685_gb300 import alpha_sweep
    w = _workload()
    alphas = [0.1, 0.3, 0.5]
    rows = alpha_sweep.sweep(w, alphas, tol=1e-12, precision=fh.FH_PREC_FP64)
    for r, a in zip(rows, alphas):
        assert r["status"] == 0
        case = Case(w["M"], {"kind": "dlvp", "alpha": [a, a]}, w["phases"], w["centres"], w["radii"])
        ref = case.oracle_solve(tol=1e-12, max_iter=5000)
        Co = OS.effective_stiffness(ref["mean_stress"], case.eps0)
        C = np.array(r["ceff"])
        assert rel(C, Co) < 1e-9, (a, rel(C, Co))
        assert rel(C, C.T) < 1e-9
    # the generator changes the discretisation: distinct alphas, distinct C_eff
    assert rows[-1]["ceff_change_vs_first"] > 1e-6
