"""Pins of the FNO oracle (the learned start's network, forward only)."""
import numpy as np
import pytest

from oracle import fno


def _direct_spectral(v, R, m):
    """K v by explicit sums over the kept modes (no FFT)."""
    C, N = v.shape[0], v.shape[1]
    ix = fno.mode_index(N, m)
    g = np.arange(N)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    out = np.zeros((R.shape[3], N, N, N))
    for a, kx in enumerate(ix):
        for b, ky in enumerate(ix):
            for kz in range(m):
                ph = np.exp(-2j * np.pi * (kx * X + ky * Y + kz * Z) / N)
                vh = np.array([np.sum(v[c] * ph) for c in range(C)])
                c_out = R[a, b, kz] @ vh
                w = 1.0 if kz == 0 else 2.0
                for o in range(R.shape[3]):
                    out[o] += w * np.real(c_out[o] * np.conj(ph)) / N ** 3
    return out


def test_spectral_equals_direct_sums(rng):
    N, m, C = 6, 2, 2
    v = rng.standard_normal((C, N, N, N))
    R = rng.standard_normal((2 * m, 2 * m, m, 3, C)) + 1j * rng.standard_normal((2 * m, 2 * m, m, 3, C))
    assert np.allclose(fno.spectral(v, R, m), _direct_spectral(v, R, m), atol=1e-12)


def test_identity_weights_keep_band_modes(rng):
    """With R = identity, K keeps real Fourier modes inside the band, removes modes
    outside it, and on the kz = 0 plane keeps half of a mode whose partner -k lies
    outside the asymmetric range {-m..m-1} (the real part of a one-sided sum)."""
    N, m, C = 8, 2, 1
    R = np.zeros((2 * m, 2 * m, m, C, C), dtype=complex)
    R[..., 0, 0] = 1.0
    g = np.arange(N)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    mode = lambda kx, ky, kz: np.cos(2 * np.pi * (kx * X + ky * Y + kz * Z) / N)[None]
    for k in [(1, -2, 1), (0, 0, 1), (-2, -2, 1), (1, -1, 0), (0, 0, 0)]:
        assert np.allclose(fno.spectral(mode(*k), R, m), mode(*k), atol=1e-12), k
    for k in [(3, 0, 1), (0, 3, 0), (1, 1, 2)]:
        assert np.allclose(fno.spectral(mode(*k), R, m), 0.0, atol=1e-12), k
    assert np.allclose(fno.spectral(mode(-2, 0, 0), R, m), 0.5 * mode(-2, 0, 0), atol=1e-12)
    assert np.allclose(fno.spectral(mode(1, -2, 0), R, m), 0.5 * mode(1, -2, 0), atol=1e-12)
    assert np.allclose(fno.spectral(mode(0, 2, 0), R, m), 0.5 * mode(0, 2, 0), atol=1e-12)


def test_gelu_values():
    assert fno.gelu(np.array(0.0)) == 0.0
    assert np.isclose(fno.gelu(np.array(1.0)), 0.8413447460685429, atol=1e-15)
    assert np.isclose(fno.gelu(np.array(-1.0)), -0.15865525393145707, atol=1e-15)
    assert np.isclose(fno.gelu(np.array(8.0)), 8.0, atol=1e-12)


def test_flat_round_trip(rng):
    p = fno.Params(7, 6, 4, 2, 2)
    flat = rng.standard_normal(p.flat().size)
    p.set_flat(flat)
    assert np.array_equal(p.flat(), flat)


def test_zero_network_outputs_the_bias():
    p = fno.Params(7, 6, 4, 2, 2)
    p.q[:] = np.arange(6)
    x = np.ones((7, 4, 4, 4))
    y = fno.forward(p, x)
    assert np.allclose(y, np.arange(6)[:, None, None, None])
