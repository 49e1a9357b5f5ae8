"""Fixed-point iteration on the discretised Lippmann-Schwinger equation.

Test infrastructure (see ``oracle/__init__.py``): not used by the product.

Thm. pde_discretization, Eq. (pde_coefficients) of arXiv 1701.04685: the pattern
values E_y of the strain fluctuation satisfy

    E_y + Gamma^p_y (C(y) - C0) : (E_y + eps0) = 0,     y in P(M),

where Gamma^p acts as the Fourier multiplier Gamma^p_h of Def.
gamma_tilde_fourier on the pattern DFT.  Sec. 4 solves it by the fixed-point
iteration of Moulinec & Suquet (1998) up to a relative Cauchy criterion.  One
step of the iteration ("form A"):

    tau   = (C - C0) : (E + eps0)                    pointwise on P(M)
    tau^  = sum_y tau_y exp(-2 pi i h^T y)           pattern DFT, h in G(M^T)
    E^_h  = -Gamma^p_h tau^_h,   E^_0 = 0            mean strain stays eps0
    E     = (1/m) sum_h E^_h exp(+2 pi i h^T y)      inverse pattern DFT
    r     = ||E_new - E_old|| / ||E_new + eps0||     Frobenius l2 over P(M)

The effective stiffness (Sec. 3.1) is read as C_eff : eps0 = <C : (E + eps0)>,
the mean over the pattern points.  ``form='B'`` is the classic
strain-update form eps <- eps - Gamma^p C eps with mean eps0, which equals
form A exactly when Gamma^p C0 is a projection (Remark constants).

Two interchangeable DFT routes: ``BruteTransform`` multiplies by the literal
matrix of Eq. (Fouriermatrix) over the enumerated P(M) and G(M^T);
``SNFTransform`` uses numpy's FFT on the Smith-normal-form grid.
"""
from __future__ import annotations

import numpy as np

from . import lattice


class BruteTransform:
    """Literal pattern DFT over the enumerated P(M), G(M^T) (small m only)."""

    def __init__(self, M):
        self.points, self.D = lattice.pattern(M)
        self.freqs = lattice.generating_set(M)
        P = lattice.dft_phases(self.points, self.D, self.freqs)
        self.W = np.exp(-2j * np.pi * (P / self.D))  # rows h, cols y
        self.m = self.D

    def fwd(self, x):
        return np.tensordot(self.W, x, axes=([1], [0]))

    def inv(self, X):
        return np.tensordot(self.W.conj().T, X, axes=([1], [0])) / self.m


class SNFTransform:
    """Pattern DFT as a d-dimensional FFT on the Smith-normal-form grid.

    ``workers`` = None uses numpy's FFT; an integer uses scipy.fft (the same
    pocketfft algorithm) with that many threads, for timing the oracle on all
    host cores.  Both compute the same plain DFT."""

    def __init__(self, M, workers=None):
        g = lattice.snf_grid(M)
        self.dims = g["dims"]
        self.points = g["points"]
        self.freqs = g["freqs"]
        self.D = g["D"]
        self.m = self.D
        self.workers = workers

    def _fftn(self, x, inverse):
        axes = tuple(range(len(self.dims)))
        if self.workers is None:
            return (np.fft.ifftn if inverse else np.fft.fftn)(x, axes=axes)
        import scipy.fft
        return (scipy.fft.ifftn if inverse else scipy.fft.fftn)(x, axes=axes, workers=self.workers)

    def fwd(self, x):
        y = self._fftn(x.reshape(self.dims + list(x.shape[1:])), False)
        return y.reshape(x.shape)

    def inv(self, X):
        y = self._fftn(X.reshape(self.dims + list(X.shape[1:])), True)
        return y.reshape(X.shape)


def _norm(x):
    return np.sqrt(np.sum(np.abs(x) ** 2))


def solve(transform, Gp, C, C0m, eps0, tol=0.0, max_iter=100, form="A",
          E_init=None, complex_iterate=False):
    """Run the fixed point for every load case separately.

    Gp: (m, n_v, n_v) aligned with ``transform.freqs``; C: (m, n_v, n_v) aligned
    with ``transform.points``; eps0: (n_L, n_v) Mandel.  Iteration n computes
    E_n and r_n; it stops after the first n with r_n <= tol, or at max_iter.
    """
    eps0 = np.atleast_2d(np.asarray(eps0, dtype=float))
    nL, nvv = eps0.shape
    m = transform.m
    zero = np.where(np.all(transform.freqs == 0, axis=1))[0]
    assert len(zero) == 1
    dC = C - C0m[None, :, :]
    Es, iters, hist, imag = [], [], [], []
    for L in range(nL):
        e0 = eps0[L][None, :]
        E = np.zeros((m, nvv)) if E_init is None else np.array(E_init[L], dtype=float)
        if complex_iterate:
            E = E.astype(complex)
        rs = []
        imax = 0.0
        n = 0
        for n in range(1, max_iter + 1):
            if form == "A":
                tau = np.einsum("mab,mb->ma", dC, E + e0)
                tau_h = transform.fwd(tau)
                E_h = -np.einsum("mab,mb->ma", Gp, tau_h)
                E_h[zero] = 0.0
                E_new = transform.inv(E_h)
            elif form == "B":
                eps = E + e0
                sig_h = transform.fwd(np.einsum("mab,mb->ma", C, eps))
                eps_h = transform.fwd(eps.astype(complex))
                new_h = eps_h - np.einsum("mab,mb->ma", Gp, sig_h)
                new_h[zero] = m * e0
                E_new = transform.inv(new_h) - e0
            else:
                raise ValueError(form)
            if not complex_iterate:
                imax = max(imax, float(np.max(np.abs(E_new.imag))))
                E_new = E_new.real
            r = _norm(E_new - E) / _norm(E_new + e0)
            rs.append(r)
            E = E_new
            if r <= tol:
                break
        Es.append(E)
        iters.append(n)
        hist.append(np.array(rs))
        imag.append(imax)
    Es = np.stack(Es)
    mean_stress = np.stack([np.mean(np.einsum("mab,mb->ma", C, Es[L] + eps0[L][None, :]), axis=0)
                            for L in range(nL)])
    return {"E": Es, "iters": np.array(iters), "resid": hist,
            "mean_stress": mean_stress, "imag_max": np.array(imag)}


def effective_stiffness(mean_stress, eps0):
    """C_eff from <sigma>_L = C_eff eps0_L for n_v independent load cases."""
    S = np.asarray(mean_stress)
    E0 = np.asarray(eps0, dtype=float)
    return np.linalg.solve(E0, S).T


def apply_operator(transform, Gp, field):
    """Gamma^p applied to a real field (m, n_v): inverse DFT of Gamma^p_h times the DFT."""
    F = transform.fwd(field)
    return transform.inv(np.einsum("mab,mb->ma", Gp, F))
