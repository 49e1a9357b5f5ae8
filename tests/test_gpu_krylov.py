"""BiCGStab on the GPU (fh_solve_opts.method = 1) against the oracle's BiCGStab.

The discrete equation of the fixed point, (I + Gamma^p (C - C0)) E =
-Gamma^p (C - C0) eps0, solved by BiCGStab (van der Vorst, 1992) with the
operator applied by the same passes as the Basic Scheme.  In FP64 the iterates
after a fixed number of iterations match ``oracle.krylov.bicgstab`` element by
element; at a tolerance the solve stops where one fixed-point step from its
result is below that tolerance (the stopping rules coincide), and the C_eff of
the benchmark workloads agrees with the converged oracle to 1e-6."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import krylov as OK
from parity import Case, frob_rel, read_golden_blocks

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL64 = 1e-9


@pytest.fixture(scope="module")
def fh():
    import torch
    assert torch.cuda.is_available()
    from paper_1701_04685_gb300 import build
    build.build()
    import paper_1701_04685_gb300 as fh
    return fh


def _disk(d, r=0.27):
    return np.full((1, d), 0.07), np.array([r])


CASES = [
    ("disk32_dirichlet", [[32, 0], [0, 32]], {"kind": "dirichlet"}, [(1.0, 0.3), (10.0, 0.3)], _disk(2, 0.2523)),
    ("sheared_odd_dlvp", [[9, 3], [0, 15]], {"kind": "dlvp", "alpha": [0.25, 0.1]}, [(1.0, 0.3), (20.0, 0.25)], _disk(2)),
    ("quincunx_box", [[8, 8], [-8, 8]], {"kind": "boxspline", "order": 2, "radius": 3}, [(2.0, 0.3), (30.0, 0.2)], _disk(2)),
    ("grid3d_three_axes", [[2, 0, 0], [0, 4, 0], [0, 0, 8]], {"kind": "dirichlet"}, [(1.0, 0.3), (10.0, 0.3)], _disk(3, 0.3)),
    ("box3d_small", [[12, 0, 0], [0, 12, 0], [0, 0, 12]], {"kind": "boxspline", "order": 2, "radius": 2},
     [(1.0, 0.3), (50.0, 0.3)], _disk(3, 0.25)),
    ("sheared3d_dlvp", [[6, 2, 0], [0, 6, 2], [0, 0, 10]], {"kind": "dlvp", "alpha": [0.2, 0.3, 0.1]},
     [(1.0, 0.3), (15.0, 0.3)], _disk(3, 0.3)),
    # FP32 3-D grid with rows of 64 points: the warp row kernel
    ("rows64_warp", [[8, 0, 0], [0, 8, 0], [0, 0, 64]], {"kind": "dlvp", "alpha": [0.25, 0.25, 0.25]},
     [(1.0, 0.3), (20.0, 0.3)], _disk(3, 0.3)),
]


def _case(spec):
    name, M, gen, phases, (c, r) = spec
    return Case(M, gen, phases, c, r)


def _oracle_bicgstab(case, n):
    C = case.Cp_o[case.ids]
    return np.stack([OK.bicgstab(case.T, case.Gp, C, case.C0_o, case.eps0[L], tol=0.0, max_iter=n)["E"]
                     for L in range(case.nload)])


@pytest.mark.parametrize("spec", CASES, ids=[c[0] for c in CASES])
def test_bicgstab_iterates_match_oracle(fh, spec):
    """FP64: every load's iterate after 8 BiCGStab iterations (16 operator
    applications), element by element against the oracle's BiCGStab."""
    case = _case(spec)
    s = case.product(fh)
    n = 8
    out = s.solve(case.eps0, tol=0.0, max_iter=n, method=1)
    assert list(out["iterations"]) == [n] * case.nload
    ref = _oracle_bicgstab(case, n)
    assert case.strain_error(s, ref) < TOL64
    s.close()


@pytest.mark.parametrize("spec", [CASES[4], CASES[6]], ids=["box3d_small", "rows64_warp"])
def test_bicgstab_fp32_tracks_oracle(fh, spec):
    """FP32 fields (double-float dot products): 5 iterations within 5e-5 of the FP64 oracle."""
    case = _case(spec)
    s = case.product(fh)
    s.solve(case.eps0, tol=0.0, max_iter=5, method=1, precision=fh.FH_PREC_FP32)
    assert case.strain_error(s, _oracle_bicgstab(case, 5)) < 5e-5
    s.close()


def test_bicgstab_stop_rule_is_the_cauchy_criterion(fh):
    """After BiCGStab stops at tol, one fixed-point step from its result moves E by
    at most tol |E + eps0| (up to the recursive residual's rounding)."""
    case = _case(CASES[1])
    s = case.product(fh)
    tol = 1e-8
    out = s.solve(case.eps0, tol=tol, max_iter=2000, method=1)
    assert out["status"] == 0 and np.all(out["residual"] <= tol)
    h = s.get_residuals(0)
    assert len(h) == out["iterations"][0] and h[-1] <= tol
    step = s.solve(case.eps0, tol=0.0, max_iter=1, init=1, path=1)
    assert np.all(step["residual"] <= 1.01 * tol), step["residual"]
    s.close()


@pytest.mark.parametrize("prec,tol,bound", [("fp64", 1e-6, 2e-6), ("fp64", 2e-7, 1e-6), ("mixed", 1e-6, 1e-6)])
def test_bicgstab_benchmark_ceff(fh, prec, tol, bound):
    """The 2-D benchmark workload (dlVP, [[128,32],[0,128]], contrast 100): C_eff
    against the converged oracle, with fewer operator applications than the fixed
    point needs iterations.  At the same residual 1e-6 the FP64 BiCGStab result's
    C_eff is 1.1e-6 off (the fixed point's 9e-8: its remaining error lies in
    directions the mean stress hardly sees); 2e-7 brings it within 1e-6, and the
    mixed mode (FP32 BiCGStab to tol / 2, then FP64 fixed-point steps) meets 1e-6
    at 1e-6."""
    P = {"fp64": fh.FH_PREC_FP64, "mixed": fh.FH_PREC_MIXED}[prec]
    case = Case.from_workload(W.dlvp_sheared())
    s = case.product(fh)
    fp = s.solve(case.eps0, tol=1e-6, max_iter=20000, precision=P, path=1)
    kr = s.solve(case.eps0, tol=tol, max_iter=20000, precision=P, method=1)
    assert kr["status"] == 0
    Cref = np.loadtxt(os.path.join(GOLDEN, "ceff_dlvp_sheared.txt"))
    err = frob_rel(s.get_ceff(), Cref)
    print(f"{prec} tol {tol}: BiCGStab iterations {list(kr['iterations'])} (fixed point to 1e-6 "
          f"{list(fp['iterations'])}), C_eff error {err:.3e}")
    assert err < bound
    assert np.all(2 * kr["iterations"] < fp["iterations"])
    s.close()


def test_bicgstab_box3d_ceff(fh):
    """128^3 box spline workload, mixed BiCGStab to r <= 1e-6: C_eff within 1e-6 of
    the converged oracle."""
    ref = read_golden_blocks(os.path.join(GOLDEN, "ceff_box3d.txt"))["box3d"]
    case = Case.from_workload(W.box3d())
    s = case.product(fh)
    out = s.solve(case.eps0, tol=1e-6, max_iter=20000, precision=fh.FH_PREC_MIXED, method=1)
    assert out["status"] == 0
    err = frob_rel(s.get_ceff(), ref["ceff_converged"])
    print(f"box3d mixed BiCGStab: iterations {list(out['iterations'])}, C_eff error {err:.3e}")
    assert err < 1e-6
    s.close()


def test_bicgstab_batch_equals_individual_solves(fh):
    ws = [W.batch2d_item(i) for i in range(3)]
    cases = [Case.from_workload(w) for w in ws]
    solvers = [c.product(fh) for c in cases]
    rc, outs = fh.solve_batch(solvers, [c.eps0 for c in cases], tol=0.0, max_iter=6, precision=fh.FH_PREC_FP64,
                              method=1)
    got = [[s.get_strain(L).copy() for L in range(3)] for s in solvers]
    for s, c, g in zip(solvers, cases, got):
        s.solve(c.eps0, tol=0.0, max_iter=6, method=1)
        for L in range(3):
            assert np.array_equal(s.get_strain(L), g[L])
        s.close()


def test_bicgstab_argument_errors(fh):
    case = _case(CASES[0])
    s = case.product(fh)
    with pytest.raises(fh.FhError) as e:
        s.solve(case.eps0, tol=0.0, max_iter=2, method=1, path=2)
    assert e.value.status == -8
    with pytest.raises(fh.FhError) as e:
        s.solve(case.eps0, tol=0.0, max_iter=2, method=1, form=1)
    assert e.value.status == -1
    with pytest.raises(fh.FhError) as e:
        s.solve(case.eps0, tol=0.0, max_iter=2, method=2)
    assert e.value.status == -1
    s.close()
