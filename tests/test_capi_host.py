"""C-ABI checks that need no GPU: the library loads, exports every declared entry
point, and its host-side lattice maps agree with the oracle's enumeration."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import lattice
from test_oracle_lattice import determinantal_divisors

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fh():
    from paper_1701_04685_gb300 import build
    build.build()
    import paper_1701_04685_gb300 as fh
    fh.library()
    return fh


def _declared():
    src = open(os.path.join(ROOT, "include", "fftHomog.h")).read()
    return sorted(set(re.findall(r"\b(fh_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(fh):
    lib = ctypes.CDLL(fh.LIB)
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert set(fh.exported_symbols()) == set(names)


MATS = [[[128, 32], [0, 128]], [[4, -2], [4, 14]], [[3, 1, 0], [0, 2, 1], [1, 0, 3]],
        [[64, 64], [-64, 64]], [[9, 3], [0, 15]], [[6, 0, 0], [0, 10, 0], [0, 0, 12]],
        [[32, 0], [0, 32]], [[128, 272], [0, 128]]]


@pytest.mark.parametrize("M", MATS)
def test_pattern_maps_match_oracle(fh, M):
    p = fh.Pattern(M)
    D = abs(lattice.det_int(M))
    assert p.m == D and int(np.prod(p.dims)) == D
    A = p.numerators()
    ref, _ = lattice.pattern(M)
    assert sorted(map(tuple, A.tolist())) == sorted(map(tuple, ref.tolist()))
    assert np.allclose(p.points(), A / D, rtol=0, atol=0)
    H = p.half_freqs()
    G = set(map(tuple, lattice.generating_set(M).tolist()))
    assert all(tuple(h) in G for h in H)
    assert len(set(map(tuple, H.tolist()))) == len(H)


@pytest.mark.parametrize("M", MATS)
def test_storage_grid_carries_the_pattern_dft(fh, M, rng):
    """exp(-2 pi i h^T y) = exp(-2 pi i sum_k l_k n_k / dims_k) for stored points and
    stored half-spectrum frequencies (Eq. (Fouriermatrix) on the storage grid)."""
    p = fh.Pattern(M)
    D = p.m
    A = p.numerators()
    H = p.half_freqs()
    dims = p.dims
    hl = dims[-1] // 2 + 1
    half_shape = dims[:-1] + [hl]
    for _ in range(300):
        i = int(rng.integers(D))
        f = int(rng.integers(len(H)))
        n = np.unravel_index(i, dims)
        l = np.unravel_index(f, half_shape)
        lhs = int(H[f].astype(object).dot(A[i].astype(object))) % D
        rhs = sum(int(l[k]) * int(n[k]) * (D // dims[k]) for k in range(len(dims))) % D
        assert lhs == rhs


def _unimodular(rng, d):
    U = np.eye(d, dtype=np.int64)
    for _ in range(6):
        i, j = rng.choice(d, size=2, replace=False)
        E = np.eye(d, dtype=np.int64)
        E[i, j] = int(rng.integers(-2, 3))
        U = U @ E
    return U


def _random_matrices(rng, count):
    """Random integer matrices (mostly one Smith axis), plus U diag(s) V with
    random unimodular U, V and divisor chains s, which have 2 or 3 Smith axes."""
    out = []
    while len(out) < count:
        d = int(rng.integers(2, 4))
        M = rng.integers(-9, 10, size=(d, d))
        det = abs(lattice.det_int(M.tolist()))
        if 0 < det <= 1500:
            out.append(M.tolist())
    for _ in range(count // 2):
        d = int(rng.integers(2, 4))
        s = [int(rng.integers(2, 5))]
        while len(s) < d:
            s.append(s[-1] * int(rng.integers(1, 4)))
        M = _unimodular(rng, d) @ np.diag(s) @ _unimodular(rng, d)
        out.append(M.tolist())
    return out


def test_random_integer_matrices_match_oracle(fh):
    """The exact int64 Smith-form map on random unimodular-equivalence classes:
    the library's points and half-spectrum frequencies are P(M) and a subset of
    G(M^T) as the oracle enumerates them by brute force, the storage grid has
    |det M| points, and the DFT phase identity of Eq. (Fouriermatrix) holds on
    sampled pairs."""
    rng = np.random.default_rng(77)
    for M in _random_matrices(rng, 40):
        p = fh.Pattern(M)
        D = abs(lattice.det_int(M))
        assert p.m == D and int(np.prod(p.dims)) == D
        A = p.numerators()
        ref, _ = lattice.pattern(M)
        assert sorted(map(tuple, A.tolist())) == sorted(map(tuple, ref.tolist()))
        H = p.half_freqs()
        G = set(map(tuple, lattice.generating_set(M).tolist()))
        assert all(tuple(h) in G for h in H)
        dims = p.dims
        assert dims == [s for s in determinantal_divisors(M) if s > 1]
        assert len(H) == int(np.prod(dims[:-1])) * (dims[-1] // 2 + 1)
        half_shape = dims[:-1] + [dims[-1] // 2 + 1]
        for _ in range(50):
            i = int(rng.integers(D))
            f = int(rng.integers(len(H)))
            n = np.unravel_index(i, dims)
            l = np.unravel_index(f, half_shape)
            lhs = int(H[f].astype(object).dot(A[i].astype(object))) % D
            rhs = sum(int(l[k]) * int(n[k]) * (D // dims[k]) for k in range(len(dims))) % D
            assert lhs == rhs


@pytest.mark.parametrize("M", [[[1, 0], [0, 1]], [[1, 0, 0], [0, 1, 0], [0, 0, 1]], [[0, 1], [1, 0]],
                               [[2, 1], [1, 1]], [[1, 0], [0, 7]], [[-3, 0, 0], [0, 1, 0], [0, 0, -5]]])
def test_degenerate_patterns(fh, M):
    """Unimodular M (a single point, det +-1) and patterns with trivial Smith
    factors or negative determinants: one storage axis (of length 1 for m = 1)
    and the oracle's points and frequencies."""
    p = fh.Pattern(M)
    D = abs(lattice.det_int(M))
    assert p.m == D and int(np.prod(p.dims)) == D and len(p.dims) >= 1
    ref, _ = lattice.pattern(M)
    assert sorted(map(tuple, p.numerators().tolist())) == sorted(map(tuple, ref.tolist()))
    H = p.half_freqs()
    assert len(H) == int(np.prod(p.dims[:-1])) * (p.dims[-1] // 2 + 1)
    G = set(map(tuple, lattice.generating_set(M).tolist()))
    assert all(tuple(h) in G for h in H)
    if D == 1:
        assert p.dims == [1] and np.all(p.points() == 0) and np.all(H == 0)


def test_error_codes_without_gpu(fh):
    with pytest.raises(fh.FhError) as e:
        fh.Pattern([[2, 4], [1, 2]])
    assert e.value.status == -2          # FH_ERR_SINGULAR_M
    with pytest.raises(fh.FhError) as e:
        fh.Pattern([[1 << 21, 0], [0, 3]])
    assert e.value.status == -3          # FH_ERR_OVERFLOW
    with pytest.raises(fh.FhError) as e:
        fh.Pattern([[1 << 16, 0], [0, 1 << 16]])          # |det M| = 2^32
    assert e.value.status == -3
    for M in ([[8192, 0], [0, 1]], [[64, 0], [0, 8192]]):   # a Smith axis longer than 4096
        with pytest.raises(fh.FhError) as e:
            fh.Solver(fh.Pattern(M), fh.generator("dirichlet"), 3)
        assert e.value.status == -8
    for M in ([[1, 0], [0, 1]], [[2, 1], [1, 1]]):   # |det M| = 1: one point, nothing to solve
        with pytest.raises(fh.FhError) as e:
            fh.Solver(fh.Pattern(M), fh.generator("dirichlet"), 3)
        assert e.value.status == -8
    p = fh.Pattern([[8, 0], [0, 8]])
    with pytest.raises(fh.FhError) as e:
        fh.Solver(p, fh.generator("dlvp", alpha=[0.7, 0.1]), 3)
    assert e.value.status == -1          # alpha outside [0, 1/2]
    with pytest.raises(fh.FhError) as e:
        fh.Solver(p, fh.generator("dirichlet"), 17)
    assert e.value.status == -1          # nload_max > FH_MAX_LOADS


def test_status_strings(fh):
    """Every status of the header has its own message; other values map to one fallback."""
    lib = fh.library()
    codes = range(-9, 4)
    msgs = [lib.fh_status_string(c).decode() for c in codes]
    assert all(msgs) and len(set(msgs)) == len(msgs)
    assert lib.fh_status_string(0).decode() == "ok"
    assert lib.fh_status_string(99).decode() == lib.fh_status_string(-99).decode() not in msgs
