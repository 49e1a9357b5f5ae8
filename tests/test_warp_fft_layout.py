"""CPU model of the index arithmetic of the one-warp line FFTs (warprow.cuh).

A line of L = 32 P points sits in a warp as lane l, register j -> point
l + 32 j.  The forward transform does a P-point DFT in each lane's registers,
multiplies register q of lane l by w_L^(l q), and finishes with a 32-point DFT
across the lanes in five exchange stages (decimation in frequency, lane
distance h = 16, 8, 4, 2, 1).  For P >= 2 the kernels use the paired form:
registers 2k and 2k+1 hold two independent lane DFTs; in stage h the lower
lane of a pair keeps the first and sends the second, the upper lane the
reverse, and the sign of the butterfly folds into its twiddle.  The frequency
that lane l, register q holds afterwards is

    P = 1:   q + P bitrev5(l)
    P >= 2:  2 (q >> 1) + (l >> 4) + P bitrev5(((l & 15) << 1) | (q & 1))

and the inverse takes that layout back to natural order.  This model follows
the kernels' stage order and exchange rule and checks both layouts against
numpy's FFT; the 16-point register DFT is checked as the 4 x 4 split the
kernels use.  It shares no code with either the kernels or the oracle."""
import numpy as np
import pytest


def bitrev5(v):
    return int(f"{v:05b}"[::-1], 2)


def warp_freq(lane, q, P):
    if P >= 2:
        return 2 * (q >> 1) + (lane >> 4) + P * bitrev5(((lane & 15) << 1) | (q & 1))
    return q + P * bitrev5(lane)


def _twiddle(L, k, sign):
    return np.exp(sign * 2j * np.pi * k / L)


def _register_stage(x, P):
    """Natural order -> per-lane P-point DFT times w_L^(l q): v[l][q]."""
    L = 32 * P
    v = np.array([[x[l + 32 * j] for j in range(P)] for l in range(32)], complex)
    F = np.exp(-2j * np.pi * np.outer(np.arange(P), np.arange(P)) / P)
    v = v @ F.T
    return v * _twiddle(L, np.outer(np.arange(32), np.arange(P)), -1)


def forward(x, P):
    L = 32 * P
    v = _register_stage(x, P)
    for h in (16, 8, 4, 2, 1):
        n = v.copy()
        for l in range(32):
            up = (l & h) != 0
            tw = _twiddle(L, (l & (h - 1)) * (L // (2 * h)), -1) if h > 1 else 1.0
            w = -tw if up else tw            # butterfly sign folded into the twiddle
            p = l ^ h
            if P == 1:                       # plain form: lower lane a + b, upper (a - b) tw
                a, b = (v[p][0], v[l][0]) if up else (v[l][0], v[p][0])
                n[l][0] = (a - b) * tw if up else a + b
                continue
            for k in range(P // 2):
                keep = v[l][2 * k + 1] if up else v[l][2 * k]
                recv = v[p][2 * k] if (p & h) else v[p][2 * k + 1]
                n[l][2 * k], n[l][2 * k + 1] = keep + recv, (keep - recv) * w
        v = n
    X = np.zeros(L, complex)
    for l in range(32):
        for q in range(P):
            X[warp_freq(l, q, P)] = v[l][q]
    return X


def inverse_pairs(X, P):
    """Unnormalised inverse from the paired layout (P >= 2) to natural order."""
    L = 32 * P
    v = np.array([[X[warp_freq(l, q, P)] for q in range(P)] for l in range(32)], complex)
    for h in (1, 2, 4, 8, 16):
        keep = np.zeros_like(v)
        sent = np.zeros_like(v)
        for l in range(32):
            up = (l & h) != 0
            w = (_twiddle(L, (l & (h - 1)) * (L // (2 * h)), +1) if h > 1 else 1.0) * (-1 if up else 1)
            for k in range(P // 2):
                u = v[l][2 * k + 1] * w
                keep[l][2 * k], sent[l][2 * k] = v[l][2 * k] + u, v[l][2 * k] - u
        n = v.copy()
        for l in range(32):
            up = (l & h) != 0
            for k in range(P // 2):
                recv = sent[l ^ h][2 * k]
                n[l][2 * k], n[l][2 * k + 1] = (recv, keep[l][2 * k]) if up else (keep[l][2 * k], recv)
        v = n
    v = v * _twiddle(L, np.outer(np.arange(32), np.arange(P)), +1)
    F = np.exp(2j * np.pi * np.outer(np.arange(P), np.arange(P)) / P)
    v = v @ F.T
    x = np.zeros(L, complex)
    for l in range(32):
        for j in range(P):
            x[l + 32 * j] = v[l][j]
    return x


@pytest.mark.parametrize("P", [1, 2, 4, 8, 16])
def test_forward_layout_is_the_dft(P, rng):
    x = rng.standard_normal(32 * P) + 1j * rng.standard_normal(32 * P)
    assert np.allclose(forward(x, P), np.fft.fft(x), rtol=0, atol=1e-9 * np.sqrt(32 * P))


@pytest.mark.parametrize("P", [1, 2, 4, 8, 16])
def test_layout_is_a_permutation(P):
    assert sorted(warp_freq(l, q, P) for l in range(32) for q in range(P)) == list(range(32 * P))


@pytest.mark.parametrize("P", [2, 4, 8, 16])
def test_inverse_from_paired_layout(P, rng):
    L = 32 * P
    X = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    assert np.allclose(inverse_pairs(X, P), np.fft.ifft(X) * L, rtol=0, atol=1e-9 * L)


def test_sixteen_point_register_dft_as_4x4():
    """X[k1 + 4 k2] = sum_n2 w16^(n2 k1) w4^(n2 k2) sum_n1 x[4 n1 + n2] w4^(n1 k1), both signs."""
    rng = np.random.default_rng(5)
    for sign in (-1, +1):
        x = rng.standard_normal(16) + 1j * rng.standard_normal(16)
        w4 = lambda e: np.exp(sign * 2j * np.pi * e / 4)
        w16 = lambda e: np.exp(sign * 2j * np.pi * e / 16)
        y = [[sum(x[4 * n1 + n2] * w4(n1 * k1) for n1 in range(4)) * w16(n2 * k1) for k1 in range(4)]
             for n2 in range(4)]
        X = np.zeros(16, complex)
        for k1 in range(4):
            for k2 in range(4):
                X[k1 + 4 * k2] = sum(y[n2][k1] * w4(n2 * k2) for n2 in range(4))
        ref = np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * 16
        assert np.allclose(X, ref)
