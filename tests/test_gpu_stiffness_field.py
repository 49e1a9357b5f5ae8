"""fh_set_stiffness_field: a point-by-point stiffness field gives exactly the
solve of the equivalent phase ids and table, from host and device memory;
more than 16 distinct matrices are refused and leave the solver unchanged."""
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


def _case():
    return Case([[24, 4], [0, 20]], {"kind": "dlvp", "alpha": [0.2, 0.3]}, [(1.0, 0.3), (30.0, 0.25)],
                np.array([[0.1, -0.2]]), np.array([0.3]))


def test_field_equals_phases_host_and_device(fh):
    import torch
    case = _case()
    s = case.product(fh)
    ids = case.ids[case.perm]                       # product storage order
    mats = np.stack([fh.isotropic_stiffness(*fh.lame(E, nu), 2) for E, nu in case.phases])
    s.solve(case.eps0, tol=0.0, max_iter=20)
    E_ref = [s.get_strain(L).copy() for L in range(3)]
    C_ref = s.get_ceff()
    field = np.ascontiguousarray(mats[ids])         # (m, 3, 3)
    for f in (field, torch.from_numpy(field).cuda()):
        s.set_stiffness_field(f)
        s.set_reference(None)
        s.solve(case.eps0, tol=0.0, max_iter=20)
        for L in range(3):
            assert np.array_equal(s.get_strain(L), E_ref[L])
        assert np.array_equal(s.get_ceff(), C_ref)


def test_field_with_many_phases_matches_oracle(fh):
    """Five isotropic materials assigned point by point (more phases than the
    workloads use): FP64 parity with the oracle after 25 iterations."""
    from oracle import green as OGr, material as OM, scheme as OS
    case = _case()
    s = case.product(fh)
    rng = np.random.default_rng(5)
    Es = [1.0, 3.0, 7.0, 15.0, 40.0]
    ids_o = rng.integers(0, 5, size=case.D)        # oracle order
    lm = [OM.lame(E, 0.3) for E in Es]
    Cp_o = np.stack([OM.isotropic_mandel(l, m, 2) for l, m in lm])
    l0, m0 = OM.reference_medium_ms([l for l, _ in lm], [m for _, m in lm])
    C0_o = OM.isotropic_mandel(l0, m0, 2)
    Gp = OGr.gamma_p_table(case.M, case.gen_o, C0_o, case.T.freqs)
    ref = OS.solve(case.T, Gp, Cp_o[ids_o], C0_o, case.eps0, tol=0.0, max_iter=25)
    mats = np.stack([fh.isotropic_stiffness(*fh.lame(E, 0.3), 2) for E in Es])
    s.set_stiffness_field(np.ascontiguousarray(mats[ids_o[case.perm]]))
    s.set_reference(None)
    out = s.solve(case.eps0, tol=0.0, max_iter=25)
    assert case.strain_error(s, ref["E"]) < 1e-10
    assert rel(out["mean_stress"], ref["mean_stress"]) < 1e-10


def test_more_than_16_distinct_matrices_is_refused(fh):
    case = _case()
    s = case.product(fh)
    s.solve(case.eps0, tol=0.0, max_iter=10)
    E_ref = s.get_strain(0).copy()
    mats = np.stack([fh.isotropic_stiffness(*fh.lame(1.0 + k, 0.3), 2) for k in range(17)])
    ids = np.arange(case.D) % 17
    with pytest.raises(fh.FhError) as e:
        s.set_stiffness_field(np.ascontiguousarray(mats[ids]))
    assert e.value.status == -8
    s.solve(case.eps0, tol=0.0, max_iter=10)      # the earlier stiffness is still in place
    assert np.array_equal(s.get_strain(0), E_ref)
