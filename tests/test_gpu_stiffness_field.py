"""fh_set_stiffness_field: a point-by-point stiffness field gives exactly the
solve of the equivalent phase ids and table, from host and device memory; a
field with more than 16 distinct matrices (a graded material) is solved point
by point and matches the oracle, which takes C(x) per point anyway."""
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


def _graded_field(case, rng):
    """A continuously varying isotropic material: Young's modulus 1 + 20 (1 + sin)
    / 2 along a direction plus 5 % noise, Poisson ratio 0.2..0.35 (every point
    distinct)."""
    y = case.T.points / case.T.D                      # oracle order
    t = 0.5 * (1 + np.sin(2 * np.pi * (y[:, 0] + 2 * y[:, 1])))
    E = (1.0 + 20.0 * t) * (1 + 0.05 * rng.standard_normal(len(y)))
    nu = 0.2 + 0.15 * rng.random(len(y))
    return E, nu


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 5e-5)])
def test_graded_field_is_solved_point_by_point(fh, prec, tol):
    """Every point its own matrix: FP64 parity with the oracle after 25 iterations
    (FP32 within its tracking bound), mean stresses included; the reference medium
    follows the Moulinec-Suquet rule over all points."""
    from oracle import green as OGr, material as OM, scheme as OS
    case = _case()
    s = case.product(fh)
    E, nu = _graded_field(case, np.random.default_rng(7))
    lm = [OM.lame(e, n) for e, n in zip(E, nu)]
    C_o = np.stack([OM.isotropic_mandel(l, m, 2) for l, m in lm])
    l0, m0 = OM.reference_medium_ms([l for l, _ in lm], [m for _, m in lm])
    C0_o = OM.isotropic_mandel(l0, m0, 2)
    Gp = OGr.gamma_p_table(case.M, case.gen_o, C0_o, case.T.freqs)
    ref = OS.solve(case.T, Gp, C_o, C0_o, case.eps0, tol=0.0, max_iter=25)
    mats = np.stack([fh.isotropic_stiffness(*fh.lame(e, n), 2) for e, n in zip(E, nu)])
    s.set_stiffness_field(np.ascontiguousarray(mats[case.perm]))
    s.set_reference(None)
    out = s.solve(case.eps0, tol=0.0, max_iter=25, precision=prec)
    assert case.strain_error(s, ref["E"]) < tol
    assert rel(out["mean_stress"], ref["mean_stress"]) < tol
    with pytest.raises(fh.FhError) as e:
        s.solve(case.eps0, tol=0.0, max_iter=2, path=2)
    assert e.value.status == -8


def test_graded_field_3d_warp_grid_and_krylov(fh):
    """A 3-D grid whose FP32 solves otherwise take the warp and plane passes: with a
    point-by-point field the block row pass runs instead, in both methods."""
    from oracle import green as OGr, krylov as OK, material as OM, scheme as OS
    case = Case([[4, 0, 0], [0, 32, 0], [0, 0, 32]], {"kind": "dlvp", "alpha": [0.25, 0.25, 0.25]},
                [(1.0, 0.3), (10.0, 0.3)], np.array([[0.1, 0.0, -0.1]]), np.array([0.3]))
    s = case.product(fh)
    y = case.T.points / case.T.D
    E = 1.0 + 9.0 * (0.5 + 0.5 * np.cos(2 * np.pi * y[:, 2])) + 0.01 * np.arange(len(y)) / len(y)
    lm = [OM.lame(e, 0.3) for e in E]
    C_o = np.stack([OM.isotropic_mandel(l, m, 3) for l, m in lm])
    l0, m0 = OM.reference_medium_ms([l for l, _ in lm], [m for _, m in lm])
    C0_o = OM.isotropic_mandel(l0, m0, 3)
    Gp = OGr.gamma_p_table(case.M, case.gen_o, C0_o, case.T.freqs)
    mats = np.stack([fh.isotropic_stiffness(*fh.lame(e, 0.3), 3) for e in E])
    s.set_stiffness_field(np.ascontiguousarray(mats[case.perm]))
    s.set_reference(None)
    ref = OS.solve(case.T, Gp, C_o, C0_o, case.eps0, tol=0.0, max_iter=15)
    s.solve(case.eps0, tol=0.0, max_iter=15, precision=1)
    assert case.strain_error(s, ref["E"]) < 5e-5
    s.solve(case.eps0, tol=0.0, max_iter=15, precision=0)
    assert case.strain_error(s, ref["E"]) < 1e-10
    kr = np.stack([OK.bicgstab(case.T, Gp, C_o, C0_o, case.eps0[L], tol=0.0, max_iter=6)["E"] for L in range(6)])
    s.solve(case.eps0, tol=0.0, max_iter=6, method=1)
    assert case.strain_error(s, kr) < 1e-9
