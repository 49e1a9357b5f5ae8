"""Pins of the oracle's generator weights, Gamma^0 and Gamma^p (Sec. 2.2, 3.1, 3.2)."""
import itertools

import numpy as np
import pytest

from oracle import generators as G
from oracle import green, lattice, material


def _random_spd_mandel(rng, d):
    """A random anisotropic stiffness in SSym_d (Mandel, symmetric positive definite)."""
    n = material.nv(d)
    A = rng.standard_normal((n, n))
    return A @ A.T + n * np.eye(n)


def _gens(d):
    return [
        G.Generator("dirichlet"),
        G.Generator("dlvp", alpha=[0.25] * d),
        G.Generator("dlvp", alpha=[0.45] + [0.1] * (d - 1)),
        G.Generator("dlvp", alpha=[0.5] * d),
        G.Generator("boxspline", xi=G.tensor_boxspline_xi(d, 2), radius=3),
    ]


# ----------------------------------------------------------------- generators

@pytest.mark.parametrize("alpha", [0.0, 0.1, 0.25, 0.45, 0.5])
def test_dlvp_is_admissible(alpha, rng):
    """Sec. 2.2 admissibility: g >= 0, g > 0 on [-1/2,1/2)^d, sum_z g(x+z) = 1."""
    gen = G.Generator("dlvp", alpha=[alpha, alpha])
    D = 1 << 20
    for _ in range(200):
        unum = rng.integers(-D // 2, D // 2, size=2)
        Z = G.alias_set(2, 3)
        g = G.symbol(gen, unum[None, :] + D * Z, D)
        assert np.all(g >= 0)
        assert abs(g.sum() - 1.0) < 1e-14
        assert G.symbol(gen, unum[None, :], D)[0] > 0


def test_dlvp_fejer_is_triangle(rng):
    gen = G.Generator("dlvp", alpha=[0.5, 0.5])
    D = 1 << 16
    unum = rng.integers(-D, D, size=(100, 2))
    u = unum / D
    expect = np.prod(np.clip(1 - np.abs(u), 0, None), axis=1)
    assert np.allclose(G.symbol(gen, unum, D), expect, atol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_dlvp_at_most_2d_aliases(d, rng):
    """Sec. 3.2: for dlVP means each alias sum has at most 2^d terms (4 in 2-D)."""
    D = 997
    for alpha in (0.1, 0.25, 0.5):
        gen = G.Generator("dlvp", alpha=[alpha] * d)
        for _ in range(100):
            unum = rng.integers(-(D // 2), D // 2 + 1, size=d)
            unum = np.where(2 * unum >= D, unum - D, unum)
            _, w = G.alias_weights(gen, unum, D)
            assert np.count_nonzero(w) <= 2 ** d
            assert abs(w.sum() - 1) < 1e-14


def test_boxspline_closed_form_sums(rng):
    """Periodised B-spline identities: sum_z sinc^2(pi(u+z)) = 1, sum_z sinc^4 = (2+cos 2 pi u)/3.

    With the sums truncated at |z| <= r the deficit is bounded by the tail,
    < 2/(pi^2 (r - 1/2)) for sinc^2 and < 2/(3 pi^4 (r - 1/2)^3) for sinc^4."""
    for r in (4, 16):
        z = np.arange(-r, r + 1)
        for u in rng.uniform(-0.5, 0.5, 50):
            s2 = np.sum(np.sinc(u + z) ** 2)
            s4 = np.sum(np.sinc(u + z) ** 4)
            assert 0 <= 1 - s2 < 2 / (np.pi ** 2 * (r - 0.5))
            assert 0 <= (2 + np.cos(2 * np.pi * u)) / 3 - s4 < 2 / (3 * np.pi ** 4 * (r - 0.5) ** 3)
    # the generator symbol is that product: Xi = (I, I) gives prod_i sinc^2(pi u_i)
    gen = G.Generator("boxspline", xi=G.tensor_boxspline_xi(2, 2), radius=4)
    D = 1000
    unum = np.array([[137, -411]])
    assert np.allclose(G.symbol(gen, unum, D), np.sinc(0.137) ** 2 * np.sinc(-0.411) ** 2)


def test_three_direction_boxspline_alias_sum(rng):
    """Non-tensor directions: for Xi = (e1, e2, e1 + e2) (the Courant hat on the
    three-direction mesh) Poisson summation turns sum_z g(u + z)^2 into the
    Fourier series of the hat's autocorrelation sampled on Z^2: 1/2 at 0 and
    1/12 at the six neighbours +-e1, +-e2, +-(e1 + e2), i.e.
    1/2 + (cos 2 pi u1 + cos 2 pi u2 + cos 2 pi (u1 + u2)) / 6.  The sum over
    |z_i| <= 150 misses a tail below 1e-8 (largest along z1 = -z2, where the
    terms fall like 1 / (pi^4 k^4))."""
    xi = np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 1.0]])
    gen = G.Generator("boxspline", xi=xi, radius=4)
    D, R = 1000, 150
    z = np.stack(np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1), indexing="ij"), -1).reshape(-1, 2)
    for _ in range(6):
        un = rng.integers(-D // 2, D // 2, size=2)
        g = G.symbol(gen, un[None, :] + D * z, D)
        u = un / D
        closed = 0.5 + (np.cos(2 * np.pi * u[0]) + np.cos(2 * np.pi * u[1]) + np.cos(2 * np.pi * u.sum())) / 6
        assert 0 <= closed - np.sum(g * g) < 1e-8
        _, w = G.alias_weights(gen, un, D)
        assert np.all(w >= 0) and abs(w.sum() - 1) < 1e-14


@pytest.mark.parametrize("d", [2, 3])
def test_weights_orthonormalise(d, rng):
    """Lemma FI:Props (iii): after normalisation sum_z |c_{h+M^T z}|^2 = 1/m."""
    D = 501
    for gen in _gens(d):
        for _ in range(30):
            unum = rng.integers(-(D // 2), D // 2 + 1, size=d)
            Z, w = G.alias_weights(gen, unum, D)
            g = G.symbol(gen, unum[None, :] + D * Z, D)
            c2 = g * g / D / np.sum(g * g / D)   # |c_k|^2 with c_k ~ g / sqrt(m), normalised
            assert abs(np.sum(c2) - 1.0) < 1e-14   # m * sum |c|^2 / m
            assert np.allclose(w, c2)
            assert np.all(w >= 0)


# ----------------------------------------------------------------- Gamma^0

@pytest.mark.parametrize("d", [2, 3])
def test_gamma0_matches_isotropic_closed_form(d, rng):
    for _ in range(20):
        lam0, mu0 = rng.uniform(0.5, 5.0, 2)
        C0 = material.isotropic_mandel(lam0, mu0, d)
        k = rng.integers(-9, 10, size=d)
        if not np.any(k):
            continue
        assert np.allclose(green.gamma0(k, C0), green.gamma0_isotropic(k, lam0, mu0), atol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_gamma0_is_C0_orthogonal_projection_onto_compatible_strains(d, rng):
    """Remark Gamma_identity: Gamma^0 C0 keeps every compatible strain sym(k (x) a)
    and annihilates every strain whose stress C0 gamma is divergence-free at k."""
    for _ in range(20):
        C0 = _random_spd_mandel(rng, d)
        k = rng.standard_normal(d)
        P = green.gamma0(k, C0) @ C0
        a = rng.standard_normal(d)
        comp = material.sym_to_mandel(0.5 * (np.outer(k, a) + np.outer(a, k)))
        assert np.allclose(P @ comp, comp, atol=1e-12)
        # stresses s with s k = 0 are a (n_v - d)-dim space; gamma = C0^{-1} s
        basis = []
        for b in range(material.nv(d)):
            e = np.zeros(material.nv(d))
            e[b] = 1
            basis.append(material.mandel_to_sym(e, d) @ k)
        A = np.stack(basis, axis=1)                  # s (Mandel) -> s k
        _, _, Vt = np.linalg.svd(A)
        for s in Vt[d:]:
            gam = np.linalg.solve(C0, s)
            assert np.allclose(P @ gam, 0, atol=1e-12)
        assert np.allclose(P @ P, P, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_gamma0_symmetric_homogeneous_bounded(d, rng):
    C0 = _random_spd_mandel(rng, d)
    l = np.linalg.eigvalsh(C0)[0]
    for _ in range(20):
        k = rng.standard_normal(d)
        G0 = green.gamma0(k, C0)
        assert np.allclose(G0, G0.T, atol=1e-14)
        assert np.allclose(G0, green.gamma0(3.7 * k, C0), atol=1e-14)
        assert np.linalg.norm(G0, 2) <= 1 / l * (1 + 1e-12)   # ||Gamma^0_k|| <= 1/l
    assert np.all(green.gamma0(np.zeros(d), C0) == 0)


# ----------------------------------------------------------------- Gamma^p

ODD_MATS = [[[15, 0], [0, 15]], [[15, 4], [0, 17]], [[5, 0, 0], [0, 5, 0], [0, 0, 5]]]


def _C0(d):
    return material.isotropic_mandel(1.9, 0.8, d)


@pytest.mark.parametrize("M", ODD_MATS)
def test_dirichlet_gamma_p_equals_gamma0(M):
    """Thm CoincidenceGamma0GammaP: for D_M the periodised operator is Gamma^0 on G(M^T)."""
    d = len(M)
    H = lattice.generating_set(M)
    Gp = green.gamma_p_table(M, G.Generator("dirichlet"), _C0(d), H)
    G0 = green.gamma0(H, _C0(d))
    assert np.abs(Gp - G0).max() < 1e-15


@pytest.mark.parametrize("M", ODD_MATS)
def test_projection_iff_dirichlet(M):
    """Thm (Gamma_projection): Gamma^p C0 is a projection iff the space is V^{D_M}."""
    d = len(M)
    C0 = _C0(d)
    H = lattice.generating_set(M)
    for gen in _gens(d):
        Gp = green.gamma_p_table(M, gen, C0, H)
        P = Gp @ C0
        defect = np.abs(np.einsum("hab,hbc->hac", P, P) - P).max()
        if gen.kind == "dirichlet":
            assert defect < 1e-13
        else:
            assert defect > 1e-3, gen


@pytest.mark.parametrize("M", ODD_MATS + [[[8, 0], [0, 8]], [[4, -2], [4, 14]]])
def test_gamma_p_bounded_symmetric_zero_mean(M, rng):
    """Thm (boundedness): ||Gamma^p C0 gamma||^2 <= (u/l) ||gamma||^2, read per frequency;
    Gamma^p_h symmetric (adjointness theorem); Gamma^p_0 = 0."""
    d = len(M)
    C0 = _random_spd_mandel(rng, d)
    ev = np.linalg.eigvalsh(C0)
    H = lattice.generating_set(M)
    izero = int(np.where(np.all(H == 0, axis=1))[0][0])
    for gen in _gens(d):
        Gp = green.gamma_p_table(M, gen, C0, H)
        assert np.all(Gp[izero] == 0)
        assert np.abs(Gp - np.transpose(Gp, (0, 2, 1))).max() < 1e-14
        norms = np.linalg.norm(Gp @ C0, ord=2, axis=(1, 2))
        assert norms.max() ** 2 <= ev[-1] / ev[0] * (1 + 1e-12)


@pytest.mark.parametrize("M", [[[8, 0], [0, 8]], [[4, -2], [4, 14]], [[6, 2], [0, 4]], [[128, 32], [0, 128]]])
def test_gamma_p_even_symbol_gives_real_operator(M):
    """The symmetric readings give Gamma^p_{-h} = Gamma^p_h (a real operator); the literal
    half-open Dirichlet indicator does not on even-det patterns (boundary frequencies)."""
    d = len(M)
    C0 = _C0(d)
    H = lattice.generating_set(M)
    if len(H) > 4096:
        H = H[::37]
    Hn = np.array([lattice.reduce_freq(M, -h) for h in H])
    for gen in (G.Generator("dirichlet"), G.Generator("dlvp", alpha=[0.25, 0.25]),
                G.Generator("boxspline", xi=G.tensor_boxspline_xi(2, 2), radius=3)):
        a = green.gamma_p_table(M, gen, C0, H)
        b = green.gamma_p_table(M, gen, C0, Hn)
        assert np.abs(a - b).max() < 1e-14


def test_literal_dirichlet_is_not_even():
    """On an even grid the half-open indicator treats u_i = -1/2 and +1/2 differently,
    so Gamma^p_{-h} != Gamma^p_h at boundary frequencies such as h = (-4, 1) for
    M = diag(8, 8): a real field would get a complex update.  This is why the
    product uses the modified (even) Dirichlet symbol."""
    M = [[8, 0], [0, 8]]
    C0 = _C0(2)
    lit = G.Generator("dirichlet_literal")
    h = np.array([[-4, 1]])
    hn = np.array([lattice.reduce_freq(M, -h[0])])
    assert hn.tolist() == [[-4, -1]]
    a = green.gamma_p_table(M, lit, C0, h)
    b = green.gamma_p_table(M, lit, C0, hn)
    assert np.abs(a - b).max() > 1e-3
    sym = G.Generator("dirichlet")
    assert np.abs(green.gamma_p_table(M, sym, C0, h) - green.gamma_p_table(M, sym, C0, hn)).max() < 1e-15


# ------------------------------------------------ symmetry of the cubic pattern

_PAIRS3 = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]   # Mandel order in 3-D


def _mandel_index(i, j):
    return _PAIRS3.index((min(i, j), max(i, j)))


@pytest.mark.parametrize("gen", [G.Generator("dirichlet"), G.Generator("dlvp", alpha=[0.3] * 3),
                                 G.Generator("boxspline", xi=G.tensor_boxspline_xi(3, 2), radius=2)],
                         ids=["dirichlet", "dlvp", "boxspline"])
def test_gamma_p_follows_axis_permutations_and_mirrors(gen, rng):
    """M = diag(N, N, N), an isotropic C0 and the same symbol on every axis: a
    rotation R that permutes or mirrors the axes maps the alias set onto itself
    and keeps the weights (Def. gamma_tilde_fourier), and Gamma^0 of an
    isotropic C0 is covariant, so Gamma^p(R h)_ijkl = R_ia R_jb R_kc R_ld
    Gamma^p(h)_abcd.  In Mandel form a permutation relabels the components and a
    mirror of axis g flips the sign of the entries whose index pairs hold g an
    odd number of times."""
    N = 6
    M = [[N, 0, 0], [0, N, 0], [0, 0, N]]
    C0 = material.isotropic_mandel(2.0, 1.5, 3)
    for _ in range(6):
        h = rng.integers(-N // 2, N // 2, size=3)
        Gh = green.gamma_p(M, gen, C0, h)
        scale = np.abs(Gh).max()
        for perm in itertools.permutations(range(3)):
            hp = h[list(perm)]                     # (R h)_g = h_perm(g)
            A = [_mandel_index(perm[i], perm[j]) for i, j in _PAIRS3]
            assert np.abs(green.gamma_p(M, gen, C0, hp) - Gh[np.ix_(A, A)]).max() <= 1e-13 * scale
        for g in range(3):
            if h[g] == -N // 2:                    # -h_g would leave the reduced set
                continue
            hm = h.copy()
            hm[g] = -h[g]
            s = np.array([-1.0 if (i == g) != (j == g) else 1.0 for i, j in _PAIRS3])
            assert np.abs(green.gamma_p(M, gen, C0, hm) - np.outer(s, s) * Gh).max() <= 1e-13 * scale
