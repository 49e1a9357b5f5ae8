"""GPU: the constitutive stage tau = (C - C0):(E + eps0) of Eq. (pde_coefficients)
in the 3-D row passes, against the FP64 oracle after a fixed number of
iterations.

Phase matrices with the zero pattern of isotropic, cubic and orthotropic
materials in the grid axes (no normal-shear coupling, diagonal shear block) take
the decoupled form of the stage (12 of the 36 products, summed in the order of
the full product); a fully anisotropic phase takes all 36.  The grid's rows of
32 points take the warp row pass in FP32 and the two-step row pass in FP64.
Bars: 1e-10 relative in FP64, 5e-5 in FP32 (the FP32 tracking bound of the
other parity tests).
"""
import numpy as np
import pytest

import workloads as W
from oracle import generators as OG, green as OGr, material as OM, scheme as OS
from parity import rel

pytestmark = pytest.mark.gpu

M = [[16, 0, 0], [0, 32, 0], [0, 0, 32]]
NITER = 20


@pytest.fixture(scope="module")
def fh():
    import torch
    assert torch.cuda.is_available()
    from paper_1701_04685_gb300 import build
    build.build()
    import paper_1701_04685_gb300 as fh
    return fh


def _orthotropic(rng):
    """Normal block SPD with coupling, shear block diagonal, no normal-shear terms."""
    A = rng.standard_normal((3, 3))
    C = np.zeros((6, 6))
    C[:3, :3] = 2.0 * (A @ A.T) + 6.0 * np.eye(3)
    C[3:, 3:] = np.diag(rng.uniform(3.0, 8.0, 3))
    return C


def _anisotropic(rng):
    A = rng.standard_normal((6, 6))
    return A @ A.T + 6.0 * np.eye(6)


@pytest.fixture(scope="module")
def setup():
    T = OS.SNFTransform(M)
    centres, radii = np.array([[0.05, -0.1, 0.02]]), np.array([0.3])
    ids = W.phase_ids(T.points / T.D, centres, radii)
    C0 = OM.isotropic_mandel(1.0, 5.0, 3)   # 2 C0 above every phase matrix: a contraction
    Gp = OGr.gamma_p_table(M, OG.Generator("dirichlet"), C0, T.freqs)
    return T, ids, centres, radii, C0, Gp


@pytest.mark.parametrize("inclusion", ["orthotropic", "anisotropic"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_constitutive_stage_matches_oracle(fh, setup, inclusion, prec):
    T, ids, centres, radii, C0, Gp = setup
    rng = np.random.default_rng(11)
    Cm = OM.isotropic_mandel(*OM.lame(1.0, 0.3), 3)
    Ci = _orthotropic(rng) if inclusion == "orthotropic" else _anisotropic(rng)
    Cp = np.stack([Cm, Ci])
    eps0 = np.eye(6)
    ref = OS.solve(T, Gp, Cp[ids], C0, eps0, tol=0.0, max_iter=NITER)
    p = fh.Pattern(M)
    idx = {tuple(a): i for i, a in enumerate(T.points.tolist())}
    perm = np.array([idx[tuple(a)] for a in p.numerators().tolist()])
    s = fh.Solver(p, fh.generator("dirichlet"), 6, 0)
    s.set_stiffness_phases(ids[perm], Cp)
    s.set_reference(C0)
    P = fh.FH_PREC_FP64 if prec == "fp64" else fh.FH_PREC_FP32
    out = s.solve(eps0, tol=0.0, max_iter=NITER, precision=P)
    assert list(out["iterations"]) == [NITER] * 6
    worst = 0.0
    for L in range(6):
        Eg = s.get_strain(L)
        Eo = ref["E"][L][perm].T
        worst = max(worst, np.abs(Eg - Eo).max() / np.abs(Eo + eps0[L][:, None]).max())
    bound = 1e-10 if prec == "fp64" else 5e-5
    print(f"{inclusion} {prec}: strain error {worst:.3e}")
    assert worst < bound
    assert rel(out["mean_stress"], ref["mean_stress"]) < bound
    s.close()


def _iso_case(fh, setup):
    T, ids, centres, radii, C0, Gp = setup
    p = fh.Pattern(M)
    idx = {tuple(a): i for i, a in enumerate(T.points.tolist())}
    perm = np.array([idx[tuple(a)] for a in p.numerators().tolist()])
    Cp = np.stack([OM.isotropic_mandel(*OM.lame(E, 0.3), 3) for E in (1.0, 12.0)])
    s = fh.Solver(p, fh.generator("dirichlet"), 6, 0)
    s.set_stiffness_phases(ids[perm], Cp)
    s.set_reference(None)
    return s


def test_mixed_mode_equals_fp32_then_fp64(fh, setup):
    """Mixed precision (Sec. 4's fixed point in FP32 to the tolerance, then in FP64
    to the same tolerance) gives the bits of an FP32 solve followed by an FP64 solve
    that continues from its strain: the FP64 phase's first row pass, which stops
    after the E update and the residual, leaves the same E."""
    s = _iso_case(fh, setup)
    eps0 = np.eye(6)
    mixed = s.solve(eps0, tol=1e-6, max_iter=5000, precision=fh.FH_PREC_MIXED)
    Em = [s.get_strain(L).copy() for L in range(6)]
    a = s.solve(eps0, tol=1e-6, max_iter=5000, precision=fh.FH_PREC_FP32)
    b = s.solve(eps0, tol=1e-6, max_iter=5000, precision=fh.FH_PREC_FP64, init=1)
    assert list(mixed["iterations"]) == [i + j for i, j in zip(a["iterations"], b["iterations"])]
    for L in range(6):
        assert np.array_equal(s.get_strain(L), Em[L])
    assert np.array_equal(np.asarray(b["mean_stress"]), np.asarray(mixed["mean_stress"]))
    s.close()


def test_mixed_mode_polish_of_several_iterations(fh, setup):
    """A tolerance below the FP32 rounding floor: the FP32 phase stops on its stall
    rule and the FP64 phase runs several iterations (the spectra rebuilt after its
    first row pass); the result meets the FP64 solve at the same tolerance."""
    s = _iso_case(fh, setup)
    eps0 = np.eye(6)
    ref = s.solve(eps0, tol=1e-10, max_iter=5000, precision=fh.FH_PREC_FP64)
    E64 = [s.get_strain(L).copy() for L in range(6)]
    C64 = s.get_ceff()
    mixed = s.solve(eps0, tol=1e-10, max_iter=5000, precision=fh.FH_PREC_MIXED)
    assert mixed["status"] == 0 and ref["status"] == 0
    for L in range(6):
        assert np.abs(s.get_strain(L) - E64[L]).max() < 1e-8
    assert rel(s.get_ceff(), C64) < 1e-9
    s.close()
