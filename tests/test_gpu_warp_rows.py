"""The FP32 warp-per-row and warp-per-column passes of 3-D grids (axes of 32,
64, 128 or 256 points) against the FP64 oracle: fixed-iteration tracking for
every row and column length, grids with fewer rows than a block has warps,
one- and two-axis Smith grids, axes that mix the warp and block passes, the
variational form, resumption, and full-size sampled iterations.
"""
import numpy as np
import pytest

import workloads as W
from oracle import scheme as OS
from parity import Case, rel, sampled_iteration_check

pytestmark = pytest.mark.gpu

# FP32 bulk stages, 25 iterations: rounding of order eps32 * log2(m) per
# iteration, damped by the contraction (the bound of the 2-D FP32 tests)
TOL32 = 5e-5
FP32 = 1


@pytest.fixture(scope="module")
def fh():
    import torch
    assert torch.cuda.is_available()
    from paper_1701_04685_gb300 import build
    build.build()
    import paper_1701_04685_gb300 as fh
    return fh


def _ball(r=0.3):
    return np.full((1, 3), 0.07), np.array([r])


# (name, M, generator, phases, inclusions, Smith dims)
WARP_CASES = [
    ("L32_three_axes", [[4, 0, 0], [0, 8, 0], [0, 0, 32]], {"kind": "dirichlet"},
     [(1.0, 0.3), (10.0, 0.3)], _ball(), [4, 8, 32]),
    ("L32_sheared", [[4, 2, 0], [0, 8, 0], [0, 0, 32]], {"kind": "dlvp", "alpha": [0.2, 0.3, 0.1]},
     [(1.0, 0.3), (15.0, 0.25)], _ball(0.25), [2, 16, 32]),
    ("L64_two_axes_8_rows", [[2, 1, 0], [0, 4, 0], [0, 0, 64]], {"kind": "boxspline", "order": 2, "radius": 2},
     [(2.0, 0.3), (30.0, 0.2)], _ball(), [8, 64]),
    ("L128", [[2, 0, 0], [0, 4, 0], [0, 0, 128]], {"kind": "dirichlet"},
     [(1.0, 0.3), (20.0, 0.3)], _ball(0.2), [2, 4, 128]),
    ("L256_four_rows", [[2, 0, 0], [0, 2, 0], [0, 0, 256]], {"kind": "dlvp", "alpha": [0.25, 0.25, 0.25]},
     [(1.0, 0.3), (8.0, 0.3)], _ball(0.3), [2, 2, 256]),
    ("L64_single_row", [[1, 0, 0], [0, 1, 0], [0, 0, 64]], {"kind": "dirichlet"},
     [(1.0, 0.3), (5.0, 0.3)], _ball(0.3), [64]),
    # warp-per-column passes: every axis, only the middle axis, a sheared grid
    ("cols32_cube", [[32, 0, 0], [0, 32, 0], [0, 0, 32]], {"kind": "dlvp", "alpha": [0.25, 0.25, 0.25]},
     [(1.0, 0.3), (25.0, 0.3)], _ball(0.2), [32, 32, 32]),
    ("cols_middle_axis", [[32, 0, 0], [0, 8, 0], [0, 0, 64]], {"kind": "dirichlet"},
     [(1.0, 0.3), (10.0, 0.25)], _ball(0.3), [8, 32, 64]),
    ("cols_sheared", [[32, 8, 0], [0, 32, 0], [0, 0, 32]], {"kind": "boxspline", "order": 2, "radius": 2},
     [(1.0, 0.3), (40.0, 0.3)], _ball(0.25), [8, 32, 128]),
    ("cols64", [[32, 0, 0], [0, 64, 0], [0, 0, 64]], {"kind": "dirichlet"},
     [(1.0, 0.3), (50.0, 0.3)], _ball(0.15), [32, 64, 64]),
    # every column pass of 64 points, the Green step's included
    ("cols64_cube", [[64, 0, 0], [0, 64, 0], [0, 0, 64]], {"kind": "dlvp", "alpha": [0.2, 0.25, 0.3]},
     [(1.0, 0.3), (20.0, 0.25)], _ball(0.27), [64, 64, 64]),
    # ragged tiles: 4 x 17 = 68 columns of 32 points (the last tile holds 4),
    # and a two-axis grid whose Green pass has 33 columns of 64 points
    ("cols32_ragged", [[4, 0, 0], [0, 32, 0], [0, 0, 32]], {"kind": "boxspline", "order": 2, "radius": 2},
     [(1.0, 0.3), (25.0, 0.3)], _ball(0.3), [4, 32, 32]),
    ("cols64_two_axes_ragged", [[2, 1, 0], [0, 32, 0], [0, 0, 64]], {"kind": "dlvp", "alpha": [0.25, 0.2, 0.15]},
     [(1.0, 0.3), (15.0, 0.3)], _ball(0.25), [64, 64]),
]
IDS = [c[0] for c in WARP_CASES]


def _case(spec):
    name, M, gen, phases, (c, r), _ = spec
    return Case(M, gen, phases, c, r)


@pytest.mark.parametrize("spec", WARP_CASES, ids=IDS)
def test_smith_grid_is_the_intended_one(fh, spec):
    assert fh.Pattern(spec[1]).dims == spec[5]


@pytest.mark.parametrize("spec", WARP_CASES, ids=IDS)
def test_fp32_warp_rows_track_fp64_oracle(fh, spec):
    case = _case(spec)
    s = case.product(fh)
    n = 25
    out = s.solve(case.eps0, tol=0.0, max_iter=n, precision=FP32)
    ref = case.oracle_solve(tol=0.0, max_iter=n)
    assert list(out["iterations"]) == [n] * case.nload
    assert case.strain_error(s, ref["E"]) < TOL32
    assert rel(out["mean_stress"], ref["mean_stress"]) < TOL32
    for L in range(case.nload):
        # early residuals well above the FP32 rounding of E agree; where the
        # oracle's iteration is exact (a laminate's update vanishes) the FP32
        # residual is rounding-sized
        r_ref = np.asarray(ref["resid"][L][:10])
        r_gpu = s.get_residuals(L)[:len(r_ref)]
        big = r_ref > 1e-5
        if big.any():
            assert rel(r_gpu[big], r_ref[big]) < 1e-3
        assert np.all(r_gpu[~big] < 1e-5)


@pytest.mark.parametrize("spec", [WARP_CASES[1], WARP_CASES[3]], ids=[IDS[1], IDS[3]])
def test_fp32_warp_rows_variational_form(fh, spec):
    """E <- E - Gamma^p C (E + eps0) (the oracle's form B): the first pass
    transforms C (E + eps0) and every later pass adds the update to E."""
    case = _case(spec)
    s = case.product(fh)
    n = 25
    out = s.solve(case.eps0, tol=0.0, max_iter=n, precision=FP32, form=1)
    ref = OS.solve(case.T, case.Gp, case.Cp_o[case.ids], case.C0_o, case.eps0, tol=0.0, max_iter=n, form="B")
    assert case.strain_error(s, ref["E"]) < TOL32
    assert rel(out["mean_stress"], ref["mean_stress"]) < TOL32


def test_fp32_warp_rows_resume_is_bitwise_identical(fh):
    case = _case(WARP_CASES[3])
    s = case.product(fh)
    s.solve(case.eps0, tol=0.0, max_iter=20, precision=FP32)
    E20 = [s.get_strain(L).copy() for L in range(case.nload)]
    s.solve(case.eps0, tol=0.0, max_iter=12, precision=FP32)
    s.solve(case.eps0, tol=0.0, max_iter=8, init=1, precision=FP32)
    for L in range(case.nload):
        assert np.array_equal(s.get_strain(L), E20[L])


def test_fp32_warp_rows_subset_of_loads(fh):
    """Two loads on a solver made for six: the grid is sized for the loads of
    the call; the second load is tiny (1e-9)."""
    case = _case(WARP_CASES[0])
    s = case.product(fh)
    eps0 = np.stack([case.eps0[0], 1e-9 * case.eps0[3]])
    ref = case.oracle_solve(tol=0.0, max_iter=15, eps0=eps0)
    out = s.solve(eps0, tol=0.0, max_iter=15, precision=FP32)
    assert list(out["iterations"]) == [15, 15]
    for L in range(2):
        Eg = s.get_strain(L)
        Eo = ref["E"][L][case.perm].T
        assert np.abs(Eg - Eo).max() / np.abs(Eo + eps0[L][:, None]).max() < TOL32


def test_fp32_columns_of_128_track_oracle(fh):
    """M = diag(128,128,128), Dirichlet kernel, two loads: every column pass
    and the Green step on columns of 128 points, element by element after 5
    FP32 iterations."""
    case = Case([[128, 0, 0], [0, 128, 0], [0, 0, 128]], {"kind": "dirichlet"}, [(1.0, 0.3), (30.0, 0.3)],
                *_ball(0.3), nload=2)
    case.eps0 = np.stack([np.eye(6)[1], np.eye(6)[4]])
    s = case.product(fh)
    n = 5
    out = s.solve(case.eps0, tol=0.0, max_iter=n, precision=FP32)
    ref = case.oracle_solve(tol=0.0, max_iter=n)
    assert list(out["iterations"]) == [n, n]
    assert case.strain_error(s, ref["E"]) < 2e-5
    assert rel(out["mean_stress"], ref["mean_stress"]) < 2e-5
    for L in range(2):
        assert rel(s.get_residuals(L)[:n], np.asarray(ref["resid"][L][:n])) < 1e-4
    s.close()


def test_two_step_and_warp_exchange_column_passes_agree(fh):
    """The column passes of 64 points in the two-step form (the default) and in
    the warp-exchange form (autotuner candidate 5, tune = 7) give the same
    iterates to FP32 rounding."""
    case = _case([c for c in WARP_CASES if c[0] == "cols64_cube"][0])
    s = case.product(fh)
    n = 20
    s.solve(case.eps0, tol=0.0, max_iter=n, precision=FP32, tune=2)
    Ea = [s.get_strain(L).copy() for L in range(case.nload)]
    s.solve(case.eps0, tol=0.0, max_iter=n, precision=FP32, tune=7)
    for L in range(case.nload):
        Eb = s.get_strain(L)
        assert np.abs(Ea[L] - Eb).max() / np.abs(Eb + case.eps0[L][:, None]).max() < 3e-6
    s.close()


def test_full_size_box3d_fp32_iteration_sampled(fh):
    """M = diag(128,128,128) (rows of 128 points), box spline of order 2 with
    alias radius 4, 6 loads: one FP32 iteration at 300 sampled frequencies."""
    sampled_iteration_check(fh, W.box3d(), loads=[0, 4], n_prev=3, nsample=300, seed=9, tol=2e-5, precision=FP32)


def test_full_size_column_axis_of_256_sampled(fh):
    """M = diag(32, 256, 256): a column axis and rows of 256 points, random
    spheres, Dirichlet kernel: one FP32 iteration at 300 sampled frequencies."""
    rng = np.random.default_rng(11)
    c, r = W.random_inclusions(rng, 3, 12, 0.05, 0.1)
    w = {"M": [[32, 0, 0], [0, 256, 0], [0, 0, 256]], "generator": {"kind": "dirichlet"},
         "phases": [(1.0, 0.3), (30.0, 0.3)], "centres": c, "radii": r}
    assert fh.Pattern(w["M"]).dims == [32, 256, 256]
    sampled_iteration_check(fh, w, loads=[1, 5], n_prev=3, nsample=300, seed=12, tol=2e-5, precision=FP32)


def test_full_size_fno3d_fp32_iteration_sampled(fh):
    """M = diag(64,64,64) (rows of 64 points), Dirichlet kernel: one FP32 iteration sampled."""
    sampled_iteration_check(fh, W.fno3d_item(100001), loads=[2, 3], n_prev=4, nsample=300, seed=10, tol=2e-5,
                            precision=FP32)


# ---------------------------------------------------------------------------
# the fused plane pass (path 3; FP32 3-D grids with axis-1 and axis-2 lengths
# in {32, 64, 128}): axes 1 and 2 and the constitutive stage in one kernel per
# plane, an iteration = plane pass + axis-0 pass; path 1 runs the four passes
# ---------------------------------------------------------------------------
PLANE_CASES = [WARP_CASES[6], WARP_CASES[7], WARP_CASES[8], WARP_CASES[9]]
PLANE_IDS = [c[0] for c in PLANE_CASES]


@pytest.mark.parametrize("spec", PLANE_CASES, ids=PLANE_IDS)
def test_plane_pass_is_taken_and_agrees_with_four_passes(fh, spec):
    """The plane pass runs two kernels per iteration (the four-pass path four);
    after 20 FP32 iterations both paths agree to FP32 rounding, and both track
    the FP64 oracle."""
    case = _case(spec)
    s = case.product(fh)
    n = 20
    a = s.solve(case.eps0, tol=0.0, max_iter=n, precision=FP32, path=3)
    Ea = [s.get_strain(L).copy() for L in range(case.nload)]
    ha = [s.get_residuals(L) for L in range(case.nload)]
    b = s.solve(case.eps0, tol=0.0, max_iter=n, precision=FP32, path=1)
    # launches: 2 + (iterations of the replayed graph chunks) x (kernels per iteration)
    assert 2 * (a["kernel_launches"] - 2) == b["kernel_launches"] - 2
    for L in range(case.nload):
        Eb = s.get_strain(L)
        assert np.abs(Ea[L] - Eb).max() / np.abs(Eb + case.eps0[L][:, None]).max() < 3e-6
        hb = s.get_residuals(L)
        big = hb > 1e-5
        assert rel(ha[L][big], hb[big]) < 1e-3
    ref = case.oracle_solve(tol=0.0, max_iter=n)
    s.solve(case.eps0, tol=0.0, max_iter=n, precision=FP32, path=3)
    assert case.strain_error(s, ref["E"]) < TOL32
    assert rel(a["mean_stress"], ref["mean_stress"]) < TOL32


def test_plane_pass_variational_form(fh):
    case = _case(WARP_CASES[7])
    s = case.product(fh)
    n = 25
    out = s.solve(case.eps0, tol=0.0, max_iter=n, precision=FP32, form=1, path=3)
    ref = OS.solve(case.T, case.Gp, case.Cp_o[case.ids], case.C0_o, case.eps0, tol=0.0, max_iter=n, form="B")
    assert case.strain_error(s, ref["E"]) < TOL32
    assert rel(out["mean_stress"], ref["mean_stress"]) < TOL32


def test_plane_pass_resume_and_per_load_stop(fh):
    """Resuming is bitwise; at a tolerance every load stops on its own, within one
    iteration of the four-pass path (the residuals differ by FP32 rounding)."""
    case = _case(WARP_CASES[9])
    s = case.product(fh)
    s.solve(case.eps0, tol=0.0, max_iter=16, precision=FP32, path=3)
    E16 = [s.get_strain(L).copy() for L in range(case.nload)]
    s.solve(case.eps0, tol=0.0, max_iter=9, precision=FP32, path=3)
    s.solve(case.eps0, tol=0.0, max_iter=7, init=1, precision=FP32, path=3)
    for L in range(case.nload):
        assert np.array_equal(s.get_strain(L), E16[L])
    a = s.solve(case.eps0, tol=1e-5, max_iter=5000, precision=FP32, path=3)
    b = s.solve(case.eps0, tol=1e-5, max_iter=5000, precision=FP32, path=1)
    assert a["status"] == 0 and b["status"] == 0
    assert np.all(np.abs(a["iterations"] - b["iterations"]) <= 1), (a["iterations"], b["iterations"])
