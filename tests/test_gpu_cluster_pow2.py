"""The cluster-resident solve on power-of-two 2-D grids against the oracle.

These grids take the kernel variant with radix-2/4/8 stages only (16 warps
per CTA, a control warp that takes the stop decision of the previous
iteration while the others run the column phase) and, in FP32, the one-warp
register FFTs for lines of 32..512 points.  FP64: strain, residual history
and mean stress within 1e-10 of the oracle after 25 iterations; FP32 within
the FP32 tracking bound.
"""
import numpy as np
import pytest

from parity import Case, rel

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 5e-5


@pytest.fixture(scope="module")
def fh():
    import torch
    assert torch.cuda.is_available()
    from paper_1701_04685_gb300 import build
    build.build()
    import paper_1701_04685_gb300 as fh
    return fh


def _disk(r=0.27):
    return np.full((1, 2), 0.07), np.array([r])


# (name, M, generator, phases, inclusion, Smith dims): rows of 64..512 points,
# columns of 16..64 points
POW2 = [
    ("rows64_cols64", [[64, 0], [0, 64]], {"kind": "dirichlet"}, [(1.0, 0.3), (10.0, 0.3)], _disk(), [64, 64]),
    ("rows128_cols32", [[32, 0], [0, 128]], {"kind": "dlvp", "alpha": [0.25, 0.25]},
     [(1.0, 0.3), (20.0, 0.25)], _disk(0.2), [32, 128]),
    ("rows256_cols32", [[32, 0], [0, 256]], {"kind": "boxspline", "order": 2, "radius": 2},
     [(1.0, 0.3), (30.0, 0.3)], _disk(0.3), [32, 256]),
    ("rows512_cols32_sheared", [[128, 32], [0, 128]], {"kind": "dirichlet"},
     [(1.0, 0.3), (100.0, 0.3)], _disk(0.15), [32, 512]),
    ("rows256_cols16_sheared", [[64, 16], [0, 64]], {"kind": "dlvp", "alpha": [0.2, 0.3]},
     [(2.0, 0.3), (25.0, 0.2)], _disk(0.25), [16, 256]),
]
IDS = [c[0] for c in POW2]
CLUSTERS = [8, 16]


def _case(spec):
    name, M, gen, phases, (c, r), _ = spec
    return Case(M, gen, phases, c, r)


def _solve(fh, s, case, n, prec, cs):
    try:
        return s.solve(case.eps0, tol=0.0, max_iter=n, precision=prec, path=2, cluster=cs)
    except fh.FhError as e:
        if e.status == -8:
            pytest.skip("fields do not fit in a cluster of this size")
        raise


@pytest.mark.parametrize("cs", CLUSTERS)
@pytest.mark.parametrize("spec", POW2, ids=IDS)
def test_fp64_cluster_pow2_matches_oracle(fh, spec, cs):
    case = _case(spec)
    s = case.product(fh)
    assert case.pattern.dims == spec[5]
    n = 25
    out = _solve(fh, s, case, n, fh.FH_PREC_FP64, cs)
    assert out["path"] == 2 and out["cluster"] == cs
    ref = case.oracle_solve(tol=0.0, max_iter=n)
    assert list(out["iterations"]) == [n] * case.nload
    assert case.strain_error(s, ref["E"]) < TOL64
    for L in range(case.nload):
        assert rel(s.get_residuals(L), ref["resid"][L]) < 1e-9
    assert rel(out["mean_stress"], ref["mean_stress"]) < TOL64


@pytest.mark.parametrize("cs", CLUSTERS)
@pytest.mark.parametrize("spec", POW2, ids=IDS)
def test_fp32_cluster_pow2_tracks_oracle(fh, spec, cs):
    case = _case(spec)
    s = case.product(fh)
    n = 25
    out = _solve(fh, s, case, n, fh.FH_PREC_FP32, cs)
    ref = case.oracle_solve(tol=0.0, max_iter=n)
    assert case.strain_error(s, ref["E"]) < TOL32
    assert rel(out["mean_stress"], ref["mean_stress"]) < TOL32


def test_stop_decision_at_tolerance_matches_the_pass_path(fh):
    """The control warp's stop decision (taken one iteration late, while the
    next column phase runs) stops each load at the same iteration and with
    the same residual history as the pass path, whose last block decides."""
    case = _case(POW2[1])
    s = case.product(fh)
    a = s.solve(case.eps0, tol=1e-7, max_iter=5000, path=1)
    ha = [s.get_residuals(L) for L in range(case.nload)]
    b = s.solve(case.eps0, tol=1e-7, max_iter=5000, path=2, cluster=16)
    assert list(a["iterations"]) == list(b["iterations"])
    for L in range(case.nload):
        hb = s.get_residuals(L)
        assert len(hb) == len(ha[L])
        assert rel(hb, ha[L]) < 1e-9
    assert rel(b["mean_stress"], a["mean_stress"]) < TOL64
