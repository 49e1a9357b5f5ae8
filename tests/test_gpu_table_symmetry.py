"""GPU: the closed-form Gamma^p table where the axes of the pattern are
interchangeable, against the FP64 oracle's table (Def. gamma_tilde_fourier).

For M = diag(N, N, N) up to signs, an isotropic C0 and the same per-axis symbol
on every axis, permuting the geometric axes maps the alias set and its weights
onto themselves, so the table kernel sums the aliases of one frequency out of
each permutation class and writes the others with the moments' exponents
permuted.  These cases cover odd and even N (the modified Dirichlet boundary
weights at N/2), dlVP, box splines, a negative diagonal entry, and two patterns
where the symmetry does not hold (unequal ramps, unequal direction counts), which
keep the per-frequency sums.  Bar: 1e-12 relative on the whole table.
"""
import numpy as np
import pytest

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


def _eye3(n, s=(1, 1, 1)):
    return [[s[0] * n, 0, 0], [0, s[1] * n, 0], [0, 0, s[2] * n]]


XI_UNEQUAL = np.array([[1, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]], float)   # e0 twice, e1 and e2 once

CASES = [
    ("dirichlet_odd9", _eye3(9), {"kind": "dirichlet"}),
    ("dirichlet_even8", _eye3(8), {"kind": "dirichlet"}),
    ("dlvp_equal8", _eye3(8), {"kind": "dlvp", "alpha": [0.25, 0.25, 0.25]}),
    ("box2_r3_n10", _eye3(10), {"kind": "boxspline", "order": 2, "radius": 3}),
    ("box1_r2_negative6", _eye3(6, (-1, 1, 1)), {"kind": "boxspline", "order": 1, "radius": 2}),
    ("dlvp_unequal8", _eye3(8), {"kind": "dlvp", "alpha": [0.25, 0.2, 0.25]}),
    ("box_unequal_counts6", _eye3(6), {"kind": "boxspline", "xi": XI_UNEQUAL, "radius": 2}),
]


@pytest.mark.parametrize("spec", CASES, ids=[c[0] for c in CASES])
def test_symmetric_table_matches_oracle(fh, spec):
    name, M, gen = spec
    case = Case(M, gen, [(1.0, 0.3), (20.0, 0.3)], np.full((1, 3), 0.07), np.array([0.3]))
    s = case.product(fh)
    fp = case.freq_perm(case.pattern)
    Gg = s.get_green()
    Go = case.Gp[fp]
    assert rel(Gg, Go) < 1e-12
    s.close()
