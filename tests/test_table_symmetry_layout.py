"""CPU model of the index and sign arithmetic of the Gamma^p table kernel's
axis-permutation symmetry (green_table_iso<3> with cubic = 1).

On a pattern M = diag(+-N, +-N, +-N) with the same per-axis symbol on every
axis (Def. gamma_tilde_fourier with a product symbol), the alias sums of the
fourth moments B_e = sum_z w_z prod_g k_g^(e_g) / |k|^4 (k = h + M^T z) at a
frequency whose |h_g| are permuted are the moments at h with their exponents
permuted.  The kernel sums the aliases once for each storage triple
N/2 >= l0 >= l1 >= l2 >= 0 (the thread index decoded through tetrahedral
numbers), and writes every distinct permutation of the triple: the moments at
the permuted frequency h' are B[src] with src_{ax(g)} = e_g, ax the geometric
axis map |h'_g| = |h_{ax(g)}|, times (-1)^(sum over negative h_g of src_g plus
sum over negative h'_g of e_g).  This model restates those steps and checks,
on small grids: every stored quadrant frequency is written exactly once, and
the permuted moments equal moments summed directly at the permuted frequency
(brute force over the alias set).  It shares no code with the kernel or the
oracle."""
import itertools
import math

import numpy as np
import pytest

# accumulation order of the kernel's 15 fourth moments: exponents (e1, e2), e0 = 4 - e1 - e2
E12 = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2), (4, 0), (3, 1), (2, 2), (0, 3),
       (1, 3), (0, 4)]
EXP = [(4 - a - b, a, b) for a, b in E12]
INDEX = {e: t for t, e in enumerate(EXP)}


def tet3(a):
    return a * (a + 1) * (a + 2) // 6


def decode(idx):
    """Thread index -> (l0, l1, l2) with l0 >= l1 >= l2, as the kernel does it."""
    a = int(math.floor((6.0 * idx) ** (1.0 / 3.0))) if idx > 0 else 0
    while tet3(a + 1) <= idx:
        a += 1
    while a > 0 and tet3(a) > idx:
        a -= 1
    r = idx - tet3(a)
    b = int((math.sqrt(8.0 * r + 1.0) - 1.0) * 0.5)
    while (b + 1) * (b + 2) // 2 <= r:
        b += 1
    while b > 0 and b * (b + 1) // 2 > r:
        b -= 1
    return a, b, r - b * (b + 1) // 2


def distinct_perms(L):
    seen = []
    for p in [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]:
        lp = (L[p[0]], L[p[1]], L[p[2]])
        if lp not in seen:
            seen.append(lp)
    return seen


@pytest.mark.parametrize("N", [2, 3, 8, 9, 12, 31, 128])
def test_every_quadrant_frequency_written_once(N):
    n = N // 2 + 1
    count = {}
    for idx in range(tet3(n)):
        L = decode(idx)
        assert n - 1 >= L[0] >= L[1] >= L[2] >= 0
        for lp in distinct_perms(L):
            count[lp] = count.get(lp, 0) + 1
    assert len(count) == n ** 3
    assert set(count.values()) == {1}


def reduce_h(l, N, fmap, mdiag):
    """storage triple -> geometric frequency h, reduced so that the numerator of
    u = M^-T h (u_g = h_g / M_gg in units of 1/N) lies in [-N/2, N/2)"""
    h = [sum(l[k] * fmap[k][g] for k in range(3)) for g in range(3)]
    out = []
    for g in range(3):
        sg = 1 if mdiag[g] > 0 else -1
        u = ((h[g] * sg + N // 2) % N) - N // 2
        out.append(u * sg)
    return out


def axis_weights(u, N, R, s):
    """aliases z with |u/N + z| <= R + 1/2 and weights sinc(pi (u/N + z))^(2 s), normalised"""
    zs, ws = [], []
    for z in range(-R, R + 2):
        v = u / N + z
        if abs(2 * v) > 2 * R + 1:
            continue
        g = 1.0 if v == 0 else (0.0 if v == round(v) else math.sin(math.pi * v) / (math.pi * v))
        g = g ** s
        if g == 0.0:
            continue
        zs.append(z)
        ws.append(g * g)
    S = sum(ws)
    return zs, [w / S for w in ws]


def moments(h, N, R, s, Mdiag):
    per = [axis_weights(h[g] * (1 if Mdiag[g] > 0 else -1), N, R, s) for g in range(3)]
    B = np.zeros(15)
    for (z0, w0), (z1, w1), (z2, w2) in itertools.product(*[list(zip(*p)) for p in per]):
        k = np.array([h[0] + Mdiag[0] * z0, h[1] + Mdiag[1] * z1, h[2] + Mdiag[2] * z2], float)
        r2 = k @ k
        if r2 == 0.0:
            continue
        q = w0 * w1 * w2 / r2 ** 2
        for t, e in enumerate(EXP):
            B[t] += q * k[0] ** e[0] * k[1] ** e[1] * k[2] ** e[2]
    return B


def permuted(B, h, hp):
    ax, used = [-1] * 3, [False] * 3
    for g in range(3):
        for g2 in range(3):
            if ax[g] < 0 and not used[g2] and abs(h[g2]) == abs(hp[g]):
                ax[g], used[g2] = g2, True
    assert min(ax) >= 0
    out = np.zeros(15)
    for t, e in enumerate(EXP):
        src = [0, 0, 0]
        for g in range(3):
            src[ax[g]] = e[g]
        par = sum((src[g] if h[g] < 0 else 0) + (e[g] if hp[g] < 0 else 0) for g in range(3))
        v = B[INDEX[tuple(src)]]
        out[t] = -v if par & 1 else v
    return out


@pytest.mark.parametrize("N,R,s", [(8, 2, 2), (9, 1, 1), (6, 3, 2)])
@pytest.mark.parametrize("fmap,mdiag", [
    (np.eye(3, dtype=int), (1, 1, 1)),
    (np.array([[0, -1, 0], [0, 0, 1], [1, 0, 0]]), (1, 1, 1)),
    (np.eye(3, dtype=int), (-1, 1, 1)),
])
def test_permuted_moments_equal_direct_sums(N, R, s, fmap, mdiag):
    rng = np.random.default_rng(N * 100 + R)
    n = N // 2 + 1
    Md = [m * N for m in mdiag]
    for idx in rng.choice(tet3(n), size=min(tet3(n), 12), replace=False):
        L = decode(int(idx))
        h = reduce_h(L, N, fmap, mdiag)
        B = moments(h, N, R, s, Md)
        for lp in distinct_perms(L):
            hp = reduce_h(lp, N, fmap, mdiag)
            direct = moments(hp, N, R, s, Md)
            got = permuted(B, h, hp)
            assert np.abs(got - direct).max() <= 1e-13 * max(np.abs(direct).max(), 1e-300)
