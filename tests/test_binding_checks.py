"""The Python binding refuses buffers of the wrong size, dtype or layout with
ValueError before any C entry point runs (the C side cannot see buffer sizes
and would read or write past them).  No GPU: the objects are made without
their C handles, and every check fires before a library call."""
import numpy as np
import pytest

import paper_1701_04685_gb300 as fh

torch = pytest.importorskip("torch")


def _solver(nv=3, m=64):
    s = fh.Solver.__new__(fh.Solver)
    s._h = None
    s.nv, s.m, s.d = nv, m, 2 if nv == 3 else 3
    return s


def _fno(n=4, cin=7, cout=6):
    f = fh.FNO.__new__(fh.FNO)
    f._h = None
    f.n, f.cin, f.cout, f.nparam = n, cin, cout, 10
    return f


def test_stiffness_inputs():
    s = _solver()
    Cp = np.stack([np.eye(3)] * 2)
    with pytest.raises(ValueError):
        s.set_stiffness_phases(np.zeros(63, np.uint8), Cp)
    with pytest.raises(ValueError):
        s.set_stiffness_phases(np.zeros(64, np.uint8), np.eye(3))
    with pytest.raises(ValueError):
        s.set_stiffness_phases(np.full(64, 256), Cp)
    with pytest.raises(ValueError):
        s.set_stiffness_phases(torch.zeros(64, dtype=torch.int64), Cp)
    with pytest.raises(ValueError):
        s.set_stiffness_field(np.zeros((64, 3, 2)))
    with pytest.raises(ValueError):
        s.set_stiffness_field(torch.zeros((64, 3, 3), dtype=torch.float32))
    with pytest.raises(ValueError):
        s.set_reference(np.eye(2))


def test_strain_buffers():
    s = _solver(nv=6, m=8)
    with pytest.raises(ValueError):
        s.solve(np.eye(3))
    with pytest.raises(ValueError):
        s.get_strain(0, np.empty((6, 8), np.float32))
    with pytest.raises(ValueError):
        s.get_strain(0, torch.empty((6, 7), dtype=torch.float64))
    with pytest.raises(ValueError):
        s.get_strain(0, torch.empty((8, 6), dtype=torch.float64).t())
    with pytest.raises(ValueError):
        s.set_strain(0, np.zeros(47))
    with pytest.raises(ValueError):
        fh.get_strain_f32(s, 0, torch.empty((6, 8), dtype=torch.float64))
    with pytest.raises(ValueError):
        fh.set_strain_f32(s, 0, torch.empty((6, 9), dtype=torch.float32))
    with pytest.raises(ValueError):
        fh.solve_batch([s], [np.eye(6), np.eye(6)])
    with pytest.raises(ValueError):
        fh.solve_batch([s], [np.eye(3)])


def test_fno_buffers():
    f = _fno()
    x = torch.empty((2, 7, 64))
    with pytest.raises(ValueError):
        f.forward(x, torch.empty((2, 5, 64)))
    with pytest.raises(ValueError):
        f.forward(np.empty((2, 7, 64), np.float32), torch.empty((2, 6, 64)))
    with pytest.raises(ValueError):
        f.loss_grad(torch.empty((2, 7, 63)), torch.empty((2, 6, 64)))
    with pytest.raises(ValueError):
        f.make_input(torch.zeros(64, dtype=torch.uint8), [0.0, 1.0], np.zeros(3), torch.empty((7, 64)))
    with pytest.raises(ValueError):
        f.make_input(torch.zeros(63, dtype=torch.uint8), [0.0, 1.0], np.zeros(6), torch.empty((7, 64)))
    with pytest.raises(ValueError):
        f.set_params(np.zeros(9))


def test_valid_buffers_pass_unchanged():
    t = torch.empty((3, 64), dtype=torch.float64)
    assert fh._buf(t, 192, np.float64, "t") is t
    a = np.empty((3, 64))
    assert fh._buf(a, 192, np.float64, "a", writable=True) is a
    b = fh._buf([[1, 2], [3, 4]], 4, np.float64, "b")
    assert b.dtype == np.float64 and b.flags["C_CONTIGUOUS"]


def test_pattern_matrix_shape():
    for M in ([[1, 2, 3], [4, 5, 6]], [[1, 0], [0, 1], [1, 1]], [4], [[[1]]], np.eye(4, dtype=int)):
        with pytest.raises(ValueError):
            fh.Pattern(M)
