"""Pins of the Krylov oracle (conjugate gradients on the Galerkin form for the
Dirichlet kernel, GMRES on the fixed point's linear system for every
generator): both return the solution the fixed point of Eq. (pde_coefficients)
converges to, conjugate gradients decrease the energy norm of the error
monotonically, and at high contrast they need far fewer operator applications
than the fixed point."""
import numpy as np
import pytest

import workloads as W
from oracle import generators as G
from oracle import green, krylov, material, scheme

M_ODD = [[25, 6], [0, 27]]          # det 675: no boundary frequencies, Gamma^p I is a projection


def _problem(M, gen, contrast, r=0.3):
    T = scheme.SNFTransform(M)
    d = len(M)
    ids = W.phase_ids(T.points / T.D, np.array([[0.1, -0.05]]), np.array([r]))
    lm = [material.lame(1.0, 0.3), material.lame(contrast, 0.25)]
    Cp = np.stack([material.isotropic_mandel(l, m, d) for l, m in lm])
    l0, m0 = material.reference_medium_ms([l for l, _ in lm], [m for _, m in lm])
    C0 = material.isotropic_mandel(l0, m0, d)
    return T, Cp[ids], C0, green.gamma_p_table(M, gen, C0, T.freqs)


E0 = np.array([0.4, -0.1, 0.7])


def _fixed_point(T, C, C0, Gp, tol=1e-14):
    return scheme.solve(T, Gp, C, C0, E0[None], tol=tol, max_iter=50000)["E"][0]


def test_cg_reaches_the_fixed_points_solution():
    gen = G.Generator("dirichlet")
    T, C, C0, Gp = _problem(M_ODD, gen, 20.0)
    P = green.gamma_p_table(M_ODD, gen, np.eye(3), T.freqs)
    star = _fixed_point(T, C, C0, Gp)
    out = krylov.cg(T, P, C, E0, tol=1e-13, max_iter=2000)
    assert np.abs(out["E"] - star).max() / np.abs(star).max() < 1e-10
    assert abs(out["E"].mean(axis=0)).max() < 1e-13          # zero-mean fluctuation


@pytest.mark.parametrize("gen", [G.Generator("dirichlet"), G.Generator("dlvp", alpha=[0.25, 0.25]),
                                 G.Generator("boxspline", xi=G.tensor_boxspline_xi(2, 2), radius=3)],
                         ids=lambda g: g.kind)
def test_gmres_reaches_the_fixed_points_solution(gen):
    T, C, C0, Gp = _problem(M_ODD, gen, 20.0)
    star = _fixed_point(T, C, C0, Gp)
    out = krylov.gmres(T, Gp, C, C0, E0, tol=1e-13, max_iter=400)
    assert out["resid"][-1] <= 1e-13
    assert np.abs(out["E"] - star).max() / np.abs(star).max() < 1e-10


@pytest.mark.parametrize("gen", [G.Generator("dirichlet"), G.Generator("dlvp", alpha=[0.25, 0.25]),
                                 G.Generator("boxspline", xi=G.tensor_boxspline_xi(2, 2), radius=3)],
                         ids=lambda g: g.kind)
def test_bicgstab_reaches_the_fixed_points_solution(gen):
    """BiCGStab reaches the fixed point's solution for every generator."""
    T, C, C0, Gp = _problem(M_ODD, gen, 20.0)
    star = _fixed_point(T, C, C0, Gp)
    out = krylov.bicgstab(T, Gp, C, C0, E0, tol=1e-13, max_iter=500)
    assert out["resid"][-1] <= 1e-13
    assert np.abs(out["E"] - star).max() / np.abs(star).max() < 1e-10


def test_cg_refuses_tables_that_are_not_projections():
    """On an even determinant the Dirichlet table averages two aliases at the
    boundary frequencies, Gamma^p (C0 = I) is no projection, and CG is refused;
    BiCGStab still reaches the fixed point's solution there."""
    gen = G.Generator("dirichlet")
    M = [[16, 0], [0, 16]]
    T, C, C0, Gp = _problem(M, gen, 100.0)
    P = green.gamma_p_table(M, gen, np.eye(3), T.freqs)
    with pytest.raises(ValueError):
        krylov.cg(T, P, C, E0)
    star = _fixed_point(T, C, C0, Gp)
    out = krylov.bicgstab(T, Gp, C, C0, E0, tol=1e-12, max_iter=500)
    assert np.abs(out["E"] - star).max() / np.abs(star).max() < 1e-9


def test_cg_error_energy_decreases_monotonically():
    """CG minimises the energy norm sqrt(e . C e) of the error over the growing
    Krylov space, so it never increases (a wrong step length or direction
    update breaks this)."""
    gen = G.Generator("dirichlet")
    T, C, C0, Gp = _problem(M_ODD, gen, 50.0)
    P = green.gamma_p_table(M_ODD, gen, np.eye(3), T.freqs)
    star = krylov.cg(T, P, C, E0, tol=1e-14, max_iter=3000)["E"]
    energy = []
    for k in range(1, 30):
        e = krylov.cg(T, P, C, E0, tol=0.0, max_iter=k)["E"] - star
        energy.append(float(np.sum(e * np.einsum("mab,mb->ma", C, e))))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(energy, energy[1:]))
    assert energy[-1] < 1e-3 * energy[0]


def test_homogeneous_medium_has_zero_fluctuation():
    """Constant C: the right-hand side is the projection of a constant field,
    zero up to FFT rounding, and both solvers return E = 0 to rounding."""
    gen = G.Generator("dirichlet")
    T = scheme.SNFTransform(M_ODD)
    C = np.broadcast_to(material.isotropic_mandel(2.0, 1.5, 2), (T.m, 3, 3)).copy()
    P = green.gamma_p_table(M_ODD, gen, np.eye(3), T.freqs)
    assert np.abs(krylov.cg(T, P, C, E0, max_iter=5)["E"]).max() < 1e-14
    C0 = material.isotropic_mandel(1.0, 1.0, 2)
    Gp = green.gamma_p_table(M_ODD, gen, C0, T.freqs)
    assert np.abs(krylov.gmres(T, Gp, C, C0, E0, max_iter=5)["E"]).max() < 1e-14


def test_krylov_needs_fewer_applications_at_high_contrast():
    """Contrast 100: operator applications until the error is below 1e-6 of the
    solution, fixed point against conjugate gradients."""
    gen = G.Generator("dirichlet")
    T, C, C0, Gp = _problem(M_ODD, gen, 100.0)
    P = green.gamma_p_table(M_ODD, gen, np.eye(3), T.freqs)
    star = _fixed_point(T, C, C0, Gp)
    scale = np.abs(star).max()

    def first_below(run):
        for k in range(1, 3000):
            if np.abs(run(k) - star).max() <= 1e-6 * scale:
                return k
        return None

    E = np.zeros((T.m, 3))
    n_fp = None
    for k in range(1, 5000):
        E = scheme.solve(T, Gp, C, C0, E0[None], tol=0.0, max_iter=1, E_init=E[None])["E"][0]
        if np.abs(E - star).max() <= 1e-6 * scale:
            n_fp = k
            break
    n_cg = first_below(lambda k: krylov.cg(T, P, C, E0, tol=0.0, max_iter=k)["E"])
    assert n_fp is not None and n_cg is not None
    assert 3 * n_cg < n_fp
