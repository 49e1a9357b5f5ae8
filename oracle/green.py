"""Green operator Gamma^0 and periodised Green operator Gamma^p (Mandel form).

Test infrastructure (see ``oracle/__init__.py``): not used by the product.

* Def. projection, Eq. (gamma) of arXiv 1701.04685: the Fourier coefficient of
  Gamma^0 at k is grad_k (conj(grad_k)^T C0 grad_k)^{-1} conj(grad_k)^T with the
  symmetrised gradient grad_k c = (i/2)(k c^T + c k^T).  Written out, with the
  acoustic tensor K_ik(k) = C0_ijkl k_j k_l,

      Gamma^0(k) : tau = sym(k (x) K(k)^{-1} tau k),     Gamma^0(0) = 0.

  ``gamma0`` evaluates this for any elliptic C0.  ``gamma0_isotropic`` is the
  textbook closed form for an isotropic C0 (Moulinec & Suquet 1998), kept as
  an independent pin.
* Def. gamma_tilde_fourier: Gamma^p_h = m [ {Gamma^0_k |c_k(f)|^2} ]^M_h for
  h in G(M^T).  With orthonormal translates this is the convex combination
  sum_z w_z(h) Gamma^0(h + M^T z) with the weights of ``generators``.
"""
from __future__ import annotations

import numpy as np

from . import generators as gen_mod
from . import lattice
from . import material


def gamma0(k, C0m):
    """Gamma^0(k) as n_v x n_v Mandel matrices; k of shape (d,) or (n, d)."""
    k = np.asarray(k, dtype=float)
    single = k.ndim == 1
    k = np.atleast_2d(k)
    n, d = k.shape
    nvv = material.nv(d)
    out = np.zeros((n, nvv, nvv))
    nz = np.any(k != 0, axis=1)
    if not np.any(nz):
        return out[0] if single else out
    kk = k[nz]
    C4 = material.mandel_to_tensor4(C0m, d)
    K = np.einsum("ijkl,nj,nl->nik", C4, kk, kk)
    N = np.linalg.inv(K)
    cols = []
    for b in range(nvv):
        e = np.zeros(nvv)
        e[b] = 1.0
        tau = material.mandel_to_sym(e, d)
        a = np.einsum("nip,pq,nq->ni", N, tau, kk)          # K^{-1} tau k
        G = 0.5 * (np.einsum("ni,nj->nij", kk, a) + np.einsum("ni,nj->nij", a, kk))
        cols.append(material.sym_to_mandel(G))
    out[nz] = np.stack(cols, axis=-1)
    return out[0] if single else out


def gamma0_isotropic(k, lam0, mu0):
    """Closed form for isotropic C0:
    Gamma_khij = [d_ki x_h x_j + d_hi x_k x_j + d_kj x_h x_i + d_hj x_k x_i] / (4 mu0 |x|^2)
                 - (lam0 + mu0) / (mu0 (lam0 + 2 mu0)) x_i x_j x_k x_h / |x|^4."""
    x = np.asarray(k, dtype=float)
    d = len(x)
    if not np.any(x):
        return np.zeros((material.nv(d), material.nv(d)))
    I = np.eye(d)
    n2 = x @ x
    G = (np.einsum("ki,h,j->khij", I, x, x) + np.einsum("hi,k,j->khij", I, x, x)
         + np.einsum("kj,h,i->khij", I, x, x) + np.einsum("hj,k,i->khij", I, x, x)) / (4 * mu0 * n2)
    G -= (lam0 + mu0) / (mu0 * (lam0 + 2 * mu0)) * np.einsum("i,j,k,h->khij", x, x, x, x) / n2 ** 2
    return material.tensor4_to_mandel(G)


def gamma_p(M, gen, C0m, h):
    """Gamma^p_h = sum_z w_z(h) Gamma^0(h + M^T z) for one frequency h (integer vector)."""
    L = lattice.Lattice(M)
    unum = L.freq_numerator([int(v) for v in h])
    Z, w = gen_mod.alias_weights(gen, unum, L.D)
    Mt = np.array(lattice.transpose(L.M), dtype=np.int64)
    keep = w > 0
    ks = np.asarray(h, dtype=np.int64)[None, :] + Z[keep] @ Mt.T
    return np.einsum("z,zab->ab", w[keep], gamma0(ks, C0m))


def gamma_p_table(M, gen, C0m, freqs):
    """Gamma^p at every frequency of ``freqs`` (m, d): returns (m, n_v, n_v).

    The same sum as ``gamma_p``, evaluated for all frequencies at once.
    """
    L = lattice.Lattice(M)
    D = L.D
    freqs = np.asarray(freqs, dtype=np.int64)
    n, d = freqs.shape
    adjT = np.array(L.adjT, dtype=np.int64)
    Mt = np.array(lattice.transpose(L.M), dtype=np.int64)
    unum = L.sign * (freqs @ adjT.T)                     # numerators of M^{-T} h
    Z = gen_mod.alias_set(d, gen.radius)
    keep = gen_mod.alias_mask(unum, Z, D, gen.radius)                    # (n, nz)
    g = np.stack([gen_mod.symbol(gen, unum + D * z, D) for z in Z], axis=0)  # (nz, n)
    g = g * keep.T
    s = np.sum(g * g, axis=0)
    if np.any(s <= 0):
        raise ValueError("orthonormalisation impossible: the alias sum of |c_k(f)|^2 vanishes")
    w = g * g / s
    nvv = material.nv(d)
    out = np.zeros((n, nvv, nvv))
    for iz, z in enumerate(Z):
        sel = w[iz] > 0
        if not np.any(sel):
            continue
        ks = freqs[sel] + (Mt @ z)[None, :]
        out[sel] += w[iz][sel][:, None, None] * gamma0(ks, C0m)
    return out
