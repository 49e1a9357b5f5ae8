"""Pattern P(M), generating set G(M^T) and the pattern DFT, in exact integers.

Test infrastructure (see ``oracle/__init__.py``): not used by the product.

Paper passages followed (arXiv 1701.04685):
* Sec. 2.1, the lattice Lambda(M) = M^{-1} Z^d and the pattern P(M) as the
  congruence representatives of Lambda(M) modulo 1 in the half-open symmetric
  cube [-1/2, 1/2)^d; |P(M)| = |G(M^T)| = |det M| = m.
* Sec. 2.1, generating set G(M) = M P(M) (so G(M^T) = M^T P(M^T)).
* Sec. 2.1, Eq. (Fouriermatrix): F(M) = m^{-1/2} (exp(-2 pi i h^T y))_{h,y}.

Every point y is stored exactly as an integer numerator vector ``a`` with
y = a / D, D = |det M|; every frequency h is an integer vector.

The Smith-normal-form map (``smith``, ``snf_grid``) is an independent route to
the same DFT, used by the O(m log m) variant of the oracle; tests pin it to
the literal matrix of Eq. (Fouriermatrix).
"""
from __future__ import annotations

import numpy as np


def det_int(M):
    """Exact integer determinant (d <= 3)."""
    M = [[int(v) for v in row] for row in M]
    d = len(M)
    if d == 1:
        return M[0][0]
    if d == 2:
        return M[0][0] * M[1][1] - M[0][1] * M[1][0]
    if d == 3:
        a, b, c = M
        return (a[0] * (b[1] * c[2] - b[2] * c[1])
                - a[1] * (b[0] * c[2] - b[2] * c[0])
                + a[2] * (b[0] * c[1] - b[1] * c[0]))
    raise ValueError("d must be 1, 2 or 3")


def adjugate(M):
    """Exact integer adjugate, adj(M) M = det(M) I."""
    M = [[int(v) for v in row] for row in M]
    d = len(M)
    if d == 1:
        return [[1]]
    adj = [[0] * d for _ in range(d)]
    for i in range(d):
        for j in range(d):
            minor = [[M[r][c] for c in range(d) if c != j] for r in range(d) if r != i]
            adj[j][i] = (-1) ** (i + j) * det_int(minor)
    return adj


def _matvec(A, v):
    return [sum(int(A[i][k]) * int(v[k]) for k in range(len(v))) for i in range(len(A))]


def transpose(M):
    return [list(r) for r in zip(*M)]


def reduce_half_open(num, D):
    """Reduce numerators a (y = a/D) modulo D into -D <= 2a < D, i.e. y in [-1/2,1/2)."""
    num = np.asarray(num, dtype=object) if isinstance(num, list) else num
    return num - D * ((2 * num + D) // (2 * D))


class Lattice:
    """Exact description of Lambda(M) for one regular integer matrix M."""

    def __init__(self, M):
        self.M = [[int(v) for v in row] for row in M]
        self.d = len(self.M)
        det = det_int(self.M)
        if det == 0:
            raise ValueError("M is singular")
        self.sign = 1 if det > 0 else -1
        self.D = abs(det)                      # m = |det M|
        self.adj = adjugate(self.M)
        self.adjT = adjugate(transpose(self.M))  # adj(M^T)

    # y = M^{-1} j  ->  numerator  sign * adj(M) j  over D
    def point_numerator(self, j):
        return [self.sign * v for v in _matvec(self.adj, j)]

    # u = M^{-T} h  ->  numerator  sign * adj(M^T) h  over D
    def freq_numerator(self, h):
        return [self.sign * v for v in _matvec(self.adjT, h)]


def pattern(M):
    """P(M) in [-1/2,1/2)^d as an (m, d) int64 array of numerators over D.

    Built as the subgroup of (R/Z)^d generated by the columns of M^{-1}: the
    lattice M^{-1} Z^d modulo 1 is exactly that subgroup.  Returns (A, D).
    """
    L = Lattice(M)
    d, D = L.d, L.D
    gens = []
    for i in range(d):
        e = [0] * d
        e[i] = 1
        a = L.point_numerator(e)
        gens.append(tuple(int(x - D * ((2 * x + D) // (2 * D))) for x in a))
    zero = tuple([0] * d)
    seen = {zero}
    frontier = [zero]
    while frontier:
        nxt = []
        for p in frontier:
            for g in gens:
                q = tuple(int((p[k] + g[k]) - D * ((2 * (p[k] + g[k]) + D) // (2 * D)))
                          for k in range(d))
                if q not in seen:
                    seen.add(q)
                    nxt.append(q)
        frontier = nxt
    A = np.array(sorted(seen), dtype=np.int64).reshape(-1, d)
    return A, D


def generating_set(M):
    """G(M^T) = M^T P(M^T) as an (m, d) int64 array: all k with M^{-T} k in [-1/2,1/2)^d."""
    Mt = transpose([[int(v) for v in row] for row in M])
    A, D = pattern(Mt)
    # h = M^T y with y = a / D  ->  integer
    Mt_np = np.array(Mt, dtype=object)
    H = (Mt_np.dot(A.astype(object).T)).T
    assert all(int(v) % D == 0 for v in H.flat)
    return (H // D).astype(np.int64)


def reduce_freq(M, h):
    """Representative of h modulo M^T Z^d inside G(M^T) (exact)."""
    L = Lattice(M)
    u = L.freq_numerator(list(h))
    z = [(2 * x + L.D) // (2 * L.D) for x in u]
    Mt = transpose(L.M)
    return [int(h[i]) - sum(Mt[i][k] * z[k] for k in range(L.d)) for i in range(L.d)]


def dft_phases(points, D, freqs):
    """Integer phase table P[h, y] = (h^T a) mod D so that exp(-2 pi i h^T y) = exp(-2 pi i P/D)."""
    P = (freqs.astype(object).dot(points.astype(object).T)) % D
    return P.astype(np.int64)


def fourier_matrix(M, points=None, freqs=None):
    """Eq. (Fouriermatrix): F(M) = m^{-1/2} (exp(-2 pi i h^T y)) rows h in G(M^T), cols y in P(M)."""
    if points is None:
        points, D = pattern(M)
    else:
        D = abs(det_int(M))
    if freqs is None:
        freqs = generating_set(M)
    P = dft_phases(points, D, freqs)
    return np.exp(-2j * np.pi * (P / D)) / np.sqrt(D), points, freqs


# --------------------------------------------------------------------------
# Smith normal form route (used by the O(m log m) variant of the oracle)
# --------------------------------------------------------------------------

def smith(M):
    """Smith normal form U M V = diag(d_1..d_d), d_i | d_{i+1}, d_i > 0.

    Plain elimination with integer row operations (recorded in U) and column
    operations (recorded in V).  Returns (U, diag list, V) as Python int lists.
    """
    A = [[int(v) for v in row] for row in M]
    d = len(A)
    U = [[int(i == j) for j in range(d)] for i in range(d)]
    V = [[int(i == j) for j in range(d)] for i in range(d)]

    def row_add(dst, src, q):  # row_dst += q * row_src
        for c in range(d):
            A[dst][c] += q * A[src][c]
            U[dst][c] += q * U[src][c]

    def col_add(dst, src, q):  # col_dst += q * col_src
        for r in range(d):
            A[r][dst] += q * A[r][src]
            V[r][dst] += q * V[r][src]

    for t in range(d):
        while True:
            piv = None
            for i in range(t, d):
                for j in range(t, d):
                    if A[i][j] != 0 and (piv is None or abs(A[i][j]) < abs(A[piv[0]][piv[1]])):
                        piv = (i, j)
            if piv is None:
                raise ValueError("M is singular")
            i, j = piv
            A[t], A[i] = A[i], A[t]
            U[t], U[i] = U[i], U[t]
            for r in range(d):
                A[r][t], A[r][j] = A[r][j], A[r][t]
                V[r][t], V[r][j] = V[r][j], V[r][t]
            clean = True
            for i in range(t + 1, d):
                q = A[i][t] // A[t][t]
                if q:
                    row_add(i, t, -q)
                if A[i][t] != 0:
                    clean = False
            for j in range(t + 1, d):
                q = A[t][j] // A[t][t]
                if q:
                    col_add(j, t, -q)
                if A[t][j] != 0:
                    clean = False
            if not clean:
                continue
            bad = None
            for i in range(t + 1, d):
                for j in range(t + 1, d):
                    if A[i][j] % A[t][t] != 0:
                        bad = i
            if bad is not None:
                row_add(t, bad, 1)
                continue
            break
        if A[t][t] < 0:
            for c in range(d):
                A[t][c] = -A[t][c]
                U[t][c] = -U[t][c]
    return U, [A[i][i] for i in range(d)], V


def int_inverse_unimodular(U):
    det = det_int(U)
    assert abs(det) == 1
    adj = adjugate(U)
    return [[det * adj[i][j] for j in range(len(U))] for i in range(len(U))]


def snf_grid(M):
    """Grid form of the pattern DFT via the Smith normal form.

    Returns dict with ``dims`` (d_1..d_d), ``points`` (m, d) numerators over D of
    y(n) = M^{-1} U^{-1} n reduced to [-1/2,1/2)^d for n in C-order over the
    grid, and ``freqs`` (m, d) of h(l) = V^{-T} l reduced to G(M^T), l in
    C-order.  With these, exp(-2 pi i h^T y) = exp(-2 pi i sum_i l_i n_i / d_i)
    because h^T M^{-1} U^{-1} n = l^T (U M V)^{-1} n.
    """
    U, dims, V = smith(M)
    L = Lattice(M)
    D = L.D
    Uinv = np.array(int_inverse_unimodular(U), dtype=np.int64)
    Vinv = np.array(int_inverse_unimodular(V), dtype=np.int64)
    adj = np.array(L.adj, dtype=np.int64)
    adjT = np.array(L.adjT, dtype=np.int64)
    Mn = np.array(L.M, dtype=np.int64)
    idx = np.indices(dims).reshape(len(dims), -1).T.astype(np.int64)  # C-order
    j = idx @ Uinv.T                      # j = U^{-1} n
    a = L.sign * (j @ adj.T)              # numerator of M^{-1} j
    a = a - D * ((2 * a + D) // (2 * D))  # reduce into [-1/2, 1/2)
    h = idx @ Vinv                        # h = V^{-T} l  (row form)
    u = L.sign * (h @ adjT.T)             # numerator of M^{-T} h
    z = (2 * u + D) // (2 * D)
    h = h - z @ Mn                        # h - M^T z (row form)
    return {"dims": list(dims), "U": U, "V": V, "D": D,
            "points": a, "freqs": h}
