"""Mandel layout of Sym_d and SSym_d, isotropic stiffness, reference medium.

Test infrastructure (see ``oracle/__init__.py``): not used by the product.

Sec. 3.1 of arXiv 1701.04685 equips Sym_d(R) with the Frobenius inner product
and takes stiffness tensors in SSym_d (minor and major symmetry).  The Mandel
vector v of a symmetric matrix S stores the diagonal entries as they are and
each off-diagonal pair scaled by sqrt(2), so that the Frobenius product of two
symmetric matrices equals the Euclidean product of their Mandel vectors, and a
tensor in SSym_d becomes a symmetric n_v x n_v matrix (n_v = 3 for d = 2,
n_v = 6 for d = 3).

Component order: d = 2: (11, 22, 12); d = 3: (11, 22, 33, 23, 13, 12).
"""
from __future__ import annotations

import numpy as np

PAIRS = {
    2: [(0, 0), (1, 1), (0, 1)],
    3: [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)],
}


def nv(d):
    return len(PAIRS[d])


def scale(d):
    """sqrt(2) on off-diagonal pairs, 1 on the diagonal."""
    return np.array([1.0 if i == j else np.sqrt(2.0) for i, j in PAIRS[d]])


def sym_to_mandel(S):
    S = np.asarray(S)
    d = S.shape[-1]
    return np.stack([S[..., i, j] * (1.0 if i == j else np.sqrt(2.0)) for i, j in PAIRS[d]], axis=-1)


def mandel_to_sym(v, d):
    v = np.asarray(v)
    S = np.zeros(v.shape[:-1] + (d, d), dtype=v.dtype)
    for a, (i, j) in enumerate(PAIRS[d]):
        val = v[..., a] / (1.0 if i == j else np.sqrt(2.0))
        S[..., i, j] = val
        S[..., j, i] = val
    return S


def tensor4_to_mandel(C4):
    d = C4.shape[0]
    s = scale(d)
    P = PAIRS[d]
    n = len(P)
    Cm = np.zeros((n, n))
    for a, (i, j) in enumerate(P):
        for b, (k, l) in enumerate(P):
            Cm[a, b] = s[a] * s[b] * C4[i, j, k, l]
    return Cm


def mandel_to_tensor4(Cm, d):
    C4 = np.zeros((d, d, d, d))
    s = scale(d)
    P = PAIRS[d]
    for a, (i, j) in enumerate(P):
        for b, (k, l) in enumerate(P):
            v = Cm[a, b] / (s[a] * s[b])
            for (p, q) in {(i, j), (j, i)}:
                for (r, t) in {(k, l), (l, k)}:
                    C4[p, q, r, t] = v
    return C4


def isotropic_tensor4(lam, mu, d):
    """C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk)."""
    I = np.eye(d)
    return (lam * np.einsum("ij,kl->ijkl", I, I)
            + mu * (np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I)))


def isotropic_mandel(lam, mu, d):
    return tensor4_to_mandel(isotropic_tensor4(lam, mu, d))


def lame(E, nu):
    """Lame constants of an isotropic solid (3-D formulas, also used for plane strain)."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def reference_medium_ms(lams, mus):
    """Reference medium of Moulinec & Suquet (1998): midpoints of the phase Lame ranges.

    The paper never states C0; this is the reading shared with the product.
    Pinned to its defining property: per isotropic eigenspace the eigenvalues
    of C0^-1 C over the phases span an interval centred on 1.
    """
    return 0.5 * (min(lams) + max(lams)), 0.5 * (min(mus) + max(mus))


def mandel_to_voigt(Cm, d):
    s = scale(d)
    return Cm / np.outer(s, s)
