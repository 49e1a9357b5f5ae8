"""Generator symbols and orthonormalised alias weights.

Test infrastructure (see ``oracle/__init__.py``): not used by the product.

The space of translates V^f_M is fixed by the Fourier coefficients c_k(f) of
its generator f.  arXiv 1701.04685 uses three families, all of the form
c_k(f) = const * g(M^{-T} k):

* Dirichlet kernel D_M (Sec. 2.2): g = indicator of [-1/2,1/2)^d.  Its
  alpha -> 0 limit, the modified Dirichlet kernel, puts g = 1/2 on each
  boundary coordinate |u_i| = 1/2 (kind ``dirichlet``: the reading used by
  the product, because it makes the symbol even); ``dirichlet_literal`` is the
  half-open indicator itself.
* de la Vallee Poussin means (Def. dlVP): g a per-axis trapezoid.  The
  parameter ``alpha[i]`` in [0, 1/2] is half the ramp width, as in the
  numerical section (alpha = 1/2 is the Fejer kernel, alpha = 0 the modified
  Dirichlet kernel): g_i(x) = 1 for |x| <= 1/2 - alpha_i, 0 for
  |x| >= 1/2 + alpha_i, linear in between.
* periodised pattern box splines (Sec. 2.2): c_k(B_Xi) = prod_xi sinc(pi xi^T k),
  scaled by M: g(u) = prod_{xi in Xi} sinc(pi xi^T u).

Lemma FI:Props (iii): the translates are orthonormal iff
sum_z |c_{h + M^T z}(f)|^2 = 1/m.  Orthonormalising divides by that sum, so the
weight of alias z of frequency h (u = M^{-T} h) is

    w_z(h) = g(u + z)^2 / sum_{z'} g(u + z')^2,

the factor that multiplies Gamma^0 in Def. gamma_tilde_fourier.  The sum runs
over the aliases with |u_i + z_i| <= R + 1/2 for every i (R is the truncation
radius of the box spline): z_i in {-R..R}, plus z_i = R + 1 where u_i = -1/2.
The paper only says the box-spline bracket sums are precomputed with finitely
many terms (33^2 in Sec. 4.2); truncating to a cube that is symmetric in
M^{-T} k keeps Gamma^p_{-h} = Gamma^p_h, so Gamma^p maps real fields to real
fields.  For the frequency-compact symbols (Dirichlet, dlVP) nothing is cut.
"""
from __future__ import annotations

import itertools

import numpy as np


class Generator:
    def __init__(self, kind, alpha=None, xi=None, radius=None):
        assert kind in ("dirichlet", "dirichlet_literal", "dlvp", "boxspline")
        self.kind = kind
        self.alpha = None if alpha is None else np.asarray(alpha, dtype=float)
        self.xi = None if xi is None else np.asarray(xi, dtype=float)  # (d, s)
        if radius is None:
            # frequency-compact symbols vanish beyond |u_i| = 1, so |z_i| <= 1
            # already covers every nonzero alias; 2 is taken to be safe.
            radius = 2
        self.radius = int(radius)

    def __repr__(self):
        return f"Generator({self.kind}, alpha={self.alpha}, radius={self.radius})"


def tensor_boxspline_xi(d, order):
    """Xi with ``order`` copies of every unit vector (tensor-product B-spline)."""
    return np.concatenate([np.eye(d)] * order, axis=1)


def alias_set(d, radius):
    """Candidate shifts z in {-R..R+1}^d; ``alias_mask`` keeps |u + z| <= R + 1/2."""
    return np.array(list(itertools.product(range(-radius, radius + 2), repeat=d)), dtype=np.int64)


def alias_mask(unum, Z, D, radius):
    """True where every |u_i + z_i| <= R + 1/2 (u = unum / D), evaluated exactly."""
    t = np.abs(2 * (np.asarray(unum, dtype=np.int64)[..., None, :] + D * Z))
    return np.all(t <= (2 * radius + 1) * D, axis=-1)


def symbol(gen, unum, D):
    """g(u) at u = unum / D; ``unum`` integer (..., d).  Boundary tests are exact."""
    unum = np.asarray(unum, dtype=np.int64)
    u = unum / D
    if gen.kind == "dirichlet_literal":
        inside = (2 * unum >= -D) & (2 * unum < D)
        return np.prod(inside.astype(float), axis=-1)
    if gen.kind == "dirichlet" or (gen.kind == "dlvp" and np.all(gen.alpha == 0)):
        two = np.abs(2 * unum)
        per = np.where(two < D, 1.0, np.where(two == D, 0.5, 0.0))
        return np.prod(per, axis=-1)
    if gen.kind == "dlvp":
        a = gen.alpha
        per = []
        for i in range(u.shape[-1]):
            if a[i] == 0:
                two = np.abs(2 * unum[..., i])
                per.append(np.where(two < D, 1.0, np.where(two == D, 0.5, 0.0)))
            else:
                per.append(np.clip((0.5 + a[i] - np.abs(u[..., i])) / (2 * a[i]), 0.0, 1.0))
        return np.prod(np.stack(per, axis=-1), axis=-1)
    if gen.kind == "boxspline":
        t = np.tensordot(u, gen.xi, axes=([-1], [0]))  # (..., s) = xi^T u
        # np.sinc(x) = sin(pi x)/(pi x); its zeros at the nonzero integers are
        # taken exactly (floating sin(pi n) is ~1e-16, not 0).
        s = np.where((t == np.round(t)) & (t != 0), 0.0, np.sinc(t))
        return np.prod(s, axis=-1)
    raise ValueError(gen.kind)


def alias_weights(gen, unum, D):
    """Orthonormalised weights w_z for one frequency: returns (Z, w) with sum w = 1."""
    d = len(unum)
    Z = alias_set(d, gen.radius)
    Z = Z[alias_mask(unum, Z, D, gen.radius)]
    g = symbol(gen, np.asarray(unum, dtype=np.int64)[None, :] + D * Z, D)
    s = np.sum(g * g)
    if s <= 0:
        raise ValueError("orthonormalisation impossible: the alias sum of |c_k(f)|^2 vanishes")
    return Z, (g * g) / s
