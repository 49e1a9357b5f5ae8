"""Krylov solvers for the discrete equation of the fixed point (not the paper's
iteration).

Test infrastructure (see ``oracle/__init__.py``): not used by the product.

The paper solves Eq. (pde_coefficients) with the fixed point of Sec. 4 and
names Krylov methods, in its introduction, as faster solvers of the same
discretised Lippmann-Schwinger equation.  The functions here return the unique
solution E of the linear system that the fixed point converges to, so they
are pinned against ``scheme.solve``:

* ``cg`` -- Dirichlet kernel.  With C0 = I (the Mandel identity) the table of
  Gamma^p is the Euclidean-orthogonal projection P onto compatible zero-mean
  strain fields (Remark constants, pinned on odd-determinant patterns), and the
  fixed point's equation is the Galerkin condition P C (E + eps0) = 0 with E in
  range(P).  On range(P) the map E -> P C E is symmetric positive definite, so
  conjugate gradients (Hestenes & Stiefel, 1952) apply:
      r_0 = -P C eps0,  p_0 = r_0;
      a_k = (r_k . r_k) / (p_k . P C p_k),  E_{k+1} = E_k + a_k p_k,
      r_{k+1} = r_k - a_k P C p_k,  p_{k+1} = r_{k+1} + (|r_{k+1}|^2 / |r_k|^2) p_k;
  stopping when |r_k| <= tol |r_0|.
* ``gmres`` -- any generator and reference medium:
      (I + Gamma^p (C - C0)) E = -Gamma^p (C - C0) eps0,
  by GMRES (Saad & Schultz, 1986) without restarts: an Arnoldi basis by
  modified Gram-Schmidt, the coefficients from the small least-squares problem
  min |beta e_1 - H y|, stopping when its residual is <= tol |b|.
* ``bicgstab`` -- the same system as ``gmres`` with BiCGStab (van der Vorst,
  1992), which keeps a fixed number of fields instead of a growing basis:
      r_0 = b - A E_0, rhat = r_0, rho = alpha = omega = 1, v = p = 0;
      rho' = rhat . r,  beta = (rho' / rho)(alpha / omega),
      p = r + beta (p - omega v),  v = A p,  alpha = rho' / (rhat . v),
      s = r - alpha v,  t = A s,  omega = (t . s) / (t . t),
      E += alpha p + omega s,  r = s - omega t;
  stopping when |r| <= tol |b|.  Two operator applications per iteration.

Fields are real (m, n_v) Mandel arrays in the transform's point order; the dot
product is the Euclidean one over all points and components (Sec. 3.1's
Frobenius product in Mandel form).
"""
from __future__ import annotations

import numpy as np


def apply_multiplier(transform, table, field):
    """Real part of the Fourier multiplier ``table`` (m, n_v, n_v) applied to a
    real field (m, n_v); the symbols used here are even, so the imaginary part
    is rounding only."""
    F = transform.fwd(field)
    return transform.inv(np.einsum("mab,mb->ma", table, F)).real


def _stress(C, E):
    return np.einsum("mab,mb->ma", C, E)


def cg(transform, P_table, C, eps0, tol=1e-10, max_iter=1000):
    """Conjugate gradients on P C (E + eps0) = 0, E in range(P), one load case.

    P_table: Gamma^p of the Dirichlet kernel built with C0 = I; C: (m, n_v, n_v);
    eps0: (n_v,).  Returns {"E", "iters", "resid"} with resid[k] = |r_k| / |r_0|.
    The table must be a projection at every frequency (Dirichlet kernel, odd
    determinant: on even determinants the boundary frequencies average two
    aliases and CG does not reach the solution); otherwise ValueError."""
    if np.abs(np.einsum("mab,mbc->mac", P_table, P_table) - P_table).max() > 1e-12:
        raise ValueError("cg needs Gamma^p (C0 = I) to be a projection: Dirichlet kernel, odd determinant")
    e0 = np.asarray(eps0, dtype=float)[None, :]
    K = lambda x: apply_multiplier(transform, P_table, _stress(C, x))
    r = -K(np.broadcast_to(e0, (transform.m, e0.shape[1])).copy())
    E = np.zeros_like(r)
    p = r.copy()
    rr = float(np.sum(r * r))
    r0 = np.sqrt(rr)
    hist = [1.0]
    k = 0
    if r0 == 0.0:
        return {"E": E, "iters": 0, "resid": np.array(hist)}
    for k in range(1, max_iter + 1):
        Kp = K(p)
        a = rr / float(np.sum(p * Kp))
        E += a * p
        r -= a * Kp
        rr_new = float(np.sum(r * r))
        hist.append(np.sqrt(rr_new) / r0)
        if hist[-1] <= tol:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return {"E": E, "iters": k, "resid": np.array(hist)}


def gmres(transform, Gp, C, C0m, eps0, tol=1e-10, max_iter=500):
    """GMRES on (I + Gamma^p (C - C0)) E = -Gamma^p (C - C0) eps0, one load case.

    Returns {"E", "iters", "resid"} with resid[k] = |b - A E_k| / |b| from the
    least-squares problem."""
    m = transform.m
    e0 = np.asarray(eps0, dtype=float)[None, :]
    dC = C - C0m[None, :, :]
    A = lambda x: x + apply_multiplier(transform, Gp, _stress(dC, x))
    b = -apply_multiplier(transform, Gp, _stress(dC, np.broadcast_to(e0, (m, e0.shape[1])).copy()))
    beta = np.sqrt(float(np.sum(b * b)))
    if beta == 0.0:
        return {"E": np.zeros_like(b), "iters": 0, "resid": np.array([0.0])}
    V = [b / beta]
    H = np.zeros((max_iter + 1, max_iter))
    hist = [1.0]
    y = np.zeros(0)
    k = 0
    for k in range(1, max_iter + 1):
        w = A(V[k - 1])
        for i in range(k):
            H[i, k - 1] = float(np.sum(V[i] * w))
            w = w - H[i, k - 1] * V[i]
        H[k, k - 1] = np.sqrt(float(np.sum(w * w)))
        rhs = np.zeros(k + 1)
        rhs[0] = beta
        y = np.linalg.lstsq(H[:k + 1, :k], rhs, rcond=None)[0]
        res = np.linalg.norm(rhs - H[:k + 1, :k] @ y) / beta
        hist.append(res)
        if res <= tol or H[k, k - 1] == 0.0:
            break
        V.append(w / H[k, k - 1])
    E = sum(y[i] * V[i] for i in range(len(y)))
    return {"E": E, "iters": k, "resid": np.array(hist)}


def bicgstab(transform, Gp, C, C0m, eps0, tol=1e-10, max_iter=1000):
    """BiCGStab on (I + Gamma^p (C - C0)) E = -Gamma^p (C - C0) eps0, one load
    case.  Returns {"E", "iters", "resid"} with resid[k] = |r_k| / |b|."""
    m = transform.m
    e0 = np.asarray(eps0, dtype=float)[None, :]
    dC = C - C0m[None, :, :]
    A = lambda x: x + apply_multiplier(transform, Gp, _stress(dC, x))
    b = -apply_multiplier(transform, Gp, _stress(dC, np.broadcast_to(e0, (m, e0.shape[1])).copy()))
    bn = np.sqrt(float(np.sum(b * b)))
    E = np.zeros_like(b)
    if bn == 0.0:
        return {"E": E, "iters": 0, "resid": np.array([0.0])}
    r = b.copy()
    rhat = r.copy()
    rho = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    hist = [1.0]
    k = 0
    for k in range(1, max_iter + 1):
        rho_new = float(np.sum(rhat * r))
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = A(p)
        alpha = rho_new / float(np.sum(rhat * v))
        s = r - alpha * v
        t = A(s)
        omega = float(np.sum(t * s)) / float(np.sum(t * t))
        E += alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        hist.append(np.sqrt(float(np.sum(r * r))) / bn)
        if hist[-1] <= tol:
            break
    return {"E": E, "iters": k, "resid": np.array(hist)}
