"""Pins of the oracle's lattice layer (Sec. 2.1): pattern, generating set, pattern DFT."""
import itertools
import os

import numpy as np
import pytest

from oracle import lattice

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pattern_counts.txt")

SMALL_MATS = [
    [[4, 0], [0, 6]],
    [[3, 1], [0, 5]],
    [[4, -2], [4, 14]],
    [[5, 2], [-3, 4]],
    [[2, 1], [1, 3]],
    [[3, 1, 0], [0, 2, 1], [1, 0, 3]],
    [[2, 0, 0], [0, 3, 0], [0, 0, 4]],
    [[4, 2, 0], [0, 4, 2], [0, 0, 4]],
]


def _brute_pattern(M):
    """Exhaustive search: all a/D in [-1/2,1/2)^d with M a in D Z^d."""
    Mn = np.array(M, dtype=np.int64)
    d = len(M)
    D = abs(int(round(np.linalg.det(Mn))))
    out = set()
    for a in itertools.product(range(-(D // 2) - 1, D // 2 + 1), repeat=d):
        a = np.array(a)
        if np.any(2 * a < -D) or np.any(2 * a >= D):
            continue
        if np.all((Mn @ a) % D == 0):
            out.add(tuple(int(v) for v in a))
    return out, D


def _read_golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, mat, count, cite = [s.strip() for s in line.split(";")]
        M = [[int(v) for v in r.split()] for r in mat.split("|")]
        rows.append((name, M, int(count), cite))
    return rows


@pytest.mark.parametrize("M", SMALL_MATS)
def test_pattern_equals_exhaustive_search(M):
    A, D = lattice.pattern(M)
    ref, D2 = _brute_pattern(M)
    assert D == D2
    assert set(map(tuple, A.tolist())) == ref
    assert len(A) == D


@pytest.mark.parametrize("M", SMALL_MATS)
def test_generating_set(M):
    H = lattice.generating_set(M)
    D = abs(lattice.det_int(M))
    assert len(H) == D == len(set(map(tuple, H.tolist())))
    L = lattice.Lattice(M)
    for h in H:
        u = L.freq_numerator(list(h))
        assert all(-D <= 2 * x < D for x in u)          # M^{-T} h in [-1/2,1/2)^d
        assert lattice.reduce_freq(M, h) == list(h)     # already reduced


@pytest.mark.parametrize("row", _read_golden(), ids=lambda r: r[0])
def test_printed_pattern_counts(row):
    name, M, count, cite = row
    assert abs(lattice.det_int(M)) == count
    if count <= 8192:
        assert len(lattice.pattern(M)[0]) == count
        assert len(lattice.generating_set(M)) == count


@pytest.mark.parametrize("M", SMALL_MATS)
def test_fourier_matrix_unitary(M):
    F, _, _ = lattice.fourier_matrix(M)
    assert np.allclose(F @ F.conj().T, np.eye(len(F)), atol=1e-13)


@pytest.mark.parametrize("M", SMALL_MATS + [[[128, 32], [0, 128]], [[64, 64], [-64, 64]]])
def test_smith_form(M):
    U, dims, V = lattice.smith(M)
    A = np.array(U, dtype=object) @ np.array(M, dtype=object) @ np.array(V, dtype=object)
    assert np.all(A == np.diag(dims))
    assert abs(lattice.det_int(U)) == 1 and abs(lattice.det_int(V)) == 1
    assert all(x > 0 for x in dims)
    assert all(dims[i + 1] % dims[i] == 0 for i in range(len(dims) - 1))
    assert int(np.prod(dims)) == abs(lattice.det_int(M))


def determinantal_divisors(M):
    """Smith invariants from their definition: d_1 ... d_k = gcd of all k x k minors."""
    import itertools
    from math import gcd
    d = len(M)
    out, prev = [], 1
    for k in range(1, d + 1):
        g = 0
        for rows in itertools.combinations(range(d), k):
            for cols in itertools.combinations(range(d), k):
                g = gcd(g, abs(lattice.det_int([[M[i][j] for j in cols] for i in rows])))
        out.append(g // prev)
        prev = g
    return out


def test_smith_form_equals_determinantal_divisors(rng):
    """Random integer matrices: the diagonal of the oracle's Smith form is the
    sequence of determinantal divisor quotients, and U M V = diag."""
    n = 0
    while n < 200:
        d = int(rng.integers(2, 4))
        M = rng.integers(-15, 16, size=(d, d)).tolist()
        if lattice.det_int(M) == 0:
            continue
        n += 1
        U, dims, V = lattice.smith(M)
        assert dims == determinantal_divisors(M)
        A = np.array(U, dtype=object) @ np.array(M, dtype=object) @ np.array(V, dtype=object)
        assert np.all(A == np.diag(dims))


def test_paper_snf_shapes():
    assert lattice.smith([[128, 32], [0, 128]])[1] == [32, 512]
    assert lattice.smith([[64, 64], [-64, 64]])[1] == [64, 128]
    assert lattice.smith([[128, 272], [0, 128]])[1] == [16, 1024]


@pytest.mark.parametrize("M", SMALL_MATS)
def test_snf_grid_dft_equals_literal_matrix(M, rng):
    """The FFT on the Smith grid is the pattern DFT of Eq. (Fouriermatrix)."""
    g = lattice.snf_grid(M)
    A, D = lattice.pattern(M)
    H = lattice.generating_set(M)
    pidx = {tuple(p): i for i, p in enumerate(A.tolist())}
    hidx = {tuple(h): i for i, h in enumerate(H.tolist())}
    perm_y = np.array([pidx[tuple(p)] for p in g["points"].tolist()])
    perm_h = np.array([hidx[tuple(h)] for h in g["freqs"].tolist()])
    assert sorted(perm_y) == list(range(D)) and sorted(perm_h) == list(range(D))
    x = rng.standard_normal(D) + 1j * rng.standard_normal(D)
    F, _, _ = lattice.fourier_matrix(M, A, H)
    lit = np.sqrt(D) * (F @ x)                               # indexed like H
    fast = np.fft.fftn(x[perm_y].reshape(g["dims"])).reshape(-1)  # indexed like g["freqs"]
    assert np.allclose(fast, lit[perm_h], atol=1e-10 * np.sqrt(D))


@pytest.mark.parametrize("M", [[[4, 0], [0, 6]], [[3, 1], [0, 5]], [[5, 2], [-3, 4]],
                               [[3, 1, 0], [0, 2, 1], [1, 0, 3]]])
def test_aliasing_lemma(M, rng):
    """Lemma Aliasing: c^M_h(f) = sum_z c_{h + M^T z}(f) for a trigonometric polynomial f."""
    d = len(M)
    A, D = lattice.pattern(M)
    H = lattice.generating_set(M)
    ks = np.array(list(itertools.product(range(-7, 8), repeat=d)))
    ck = rng.standard_normal(len(ks)) + 1j * rng.standard_normal(len(ks))
    y = A / D
    f = (np.exp(1j * 2 * np.pi * (y @ ks.T)) * ck[None, :]).sum(axis=1)  # f(2 pi y)
    F, _, _ = lattice.fourier_matrix(M, A, H)
    cM = (F @ f) / np.sqrt(D)                                            # (1/m) sum_y f e^{-2pi i h.y}
    expect = np.zeros(len(H), dtype=complex)
    hidx = {tuple(h): i for i, h in enumerate(H.tolist())}
    for k, c in zip(ks, ck):
        expect[hidx[tuple(lattice.reduce_freq(M, k))]] += c
    assert np.allclose(cM, expect, atol=1e-11)
