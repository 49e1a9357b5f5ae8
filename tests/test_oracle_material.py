"""Pins of the oracle's Mandel / Voigt conversions (Sec. 3.1 tensor conventions).

The Voigt form used for reporting C_eff pairs stresses sigma_ij with
engineering strains (eps_ii, 2 eps_ij): sigma_V = C_V eps_V.  These tests fix
``material.mandel_to_voigt`` by that defining relation, computed through the
fourth-order tensor, and by the textbook isotropic matrix."""
import numpy as np
import pytest

from oracle import material as M


def _voigt_strain(e, d):
    return np.array([e[i, j] * (1.0 if i == j else 2.0) for i, j in M.PAIRS[d]])


def _voigt_stress(s, d):
    return np.array([s[i, j] for i, j in M.PAIRS[d]])


@pytest.mark.parametrize("d", [2, 3])
def test_voigt_matrix_maps_engineering_strain_to_stress(d):
    rng = np.random.default_rng(11 + d)
    n = M.nv(d)
    A = rng.standard_normal((n, n))
    Cm = A @ A.T + n * np.eye(n)                 # any symmetric Mandel stiffness
    C4 = M.mandel_to_tensor4(Cm, d)
    Cv = M.mandel_to_voigt(Cm, d)
    for _ in range(5):
        e = rng.standard_normal((d, d))
        e = 0.5 * (e + e.T)
        sigma = np.einsum("ijkl,kl->ij", C4, e)
        assert np.allclose(_voigt_stress(sigma, d), Cv @ _voigt_strain(e, d), rtol=1e-13, atol=1e-13)
    assert np.allclose(Cv, Cv.T)


@pytest.mark.parametrize("d", [2, 3])
def test_isotropic_voigt_matrix(d):
    lam, mu = 1.7, 0.45
    Cv = M.mandel_to_voigt(M.isotropic_mandel(lam, mu, d), d)
    n = M.nv(d)
    ref = np.zeros((n, n))
    ref[:d, :d] = lam
    ref[np.arange(d), np.arange(d)] = lam + 2 * mu
    ref[np.arange(d, n), np.arange(d, n)] = mu   # shear: sigma_12 = mu * gamma_12
    assert np.allclose(Cv, ref, rtol=1e-14, atol=1e-14)
