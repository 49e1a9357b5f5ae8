"""The allocation-free mean-stress entry point, called through the C ABI.

fh_mean_stress_noalloc serves callers that cannot allocate device memory when
they need the result (real-time loops where an allocation could block or fail,
applications whose device memory belongs to their own fixed-budget allocator):
its scratch is a fixed array inside the library.  This test checks it against
the mean stresses that the regular fh_solve entry point returns, on two calls
in a row (the second call reuses the array the first one left behind).  The
file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from parity import Case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fh():
    import torch
    assert torch.cuda.is_available()
    from paper_1701_04685_gb300 import build
    build.build()
    import paper_1701_04685_gb300 as fh
    lib = fh.library()
    f = lib.fh_mean_stress_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                  C.c_void_p, C.c_void_p, C.c_void_p]
    return fh


def _call(fh, d, m, nload, E, phase, Cp, eps0, out):
    lib = fh.library()
    return lib.fh_mean_stress_noalloc(d, m, nload, C.c_void_p(E.data_ptr()), C.c_void_p(phase.data_ptr()),
                                      Cp.shape[0], C.c_void_p(Cp.ctypes.data), C.c_void_p(eps0.ctypes.data),
                                      C.c_void_p(out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()),
                                      None)


@pytest.mark.parametrize("M", [[[9, 3], [0, 15]], [[6, 2, 0], [0, 6, 2], [0, 0, 10]]])
def test_noalloc_mean_stress_matches_solver(fh, M):
    import torch
    d = len(M)
    case = Case(M, {"kind": "dlvp", "alpha": [0.25] * d}, [(1.0, 0.3), (20.0, 0.25)],
                np.full((1, d), 0.07), np.array([0.3]))
    s = case.product(fh)
    out = s.solve(case.eps0, tol=0.0, max_iter=30)        # regular entry point
    nv, m, nload = case.nv, case.D, case.nload
    E = torch.empty((nload, nv, m), dtype=torch.float64, device="cuda")
    for L in range(nload):
        s.get_strain(L, E[L])
    phase = torch.from_numpy(case.ids[case.perm]).cuda()
    Cp = np.ascontiguousarray(np.stack([fh.isotropic_stiffness(*fh.lame(Ey, nu), d) for Ey, nu in case.phases]))
    eps0 = np.ascontiguousarray(case.eps0)
    ref = out["mean_stress"]
    for call in range(2):                                  # two calls in a row share the array
        host = np.full((nload, nv), np.nan)
        assert _call(fh, d, m, nload, E, phase, Cp, eps0, host) == 0
        assert np.abs(host - ref).max() <= 1e-12 * np.abs(ref).max()
    dev = torch.full((nload, nv), float("nan"), dtype=torch.float64, device="cuda")
    assert _call(fh, d, m, nload, E, phase, Cp, eps0, dev) == 0
    assert np.abs(dev.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_noalloc_rejects_too_many_loads(fh):
    import torch
    m, nv = 64, 3
    E = torch.zeros((17, nv, m), dtype=torch.float64, device="cuda")
    phase = torch.zeros(m, dtype=torch.uint8, device="cuda")
    Cp = np.ascontiguousarray(fh.isotropic_stiffness(1.0, 1.0, 2)[None])
    eps0 = np.zeros((17, nv))
    out = np.zeros((17, nv))
    assert _call(fh, 2, m, 17, E, phase, Cp, eps0, out) == -1
    assert b"16" in fh.library().fh_last_error()


def test_noalloc_rejects_phase_id_out_of_range(fh):
    """An id equal to nphase is reported as FH_ERR_ARG and never used as an index."""
    import torch
    m, nv = 300, 3
    E = torch.zeros((1, nv, m), dtype=torch.float64, device="cuda")
    ids = np.zeros(m, dtype=np.uint8)
    ids[123] = 2                                           # nphase = 2 below
    phase = torch.from_numpy(ids).cuda()
    Cp = np.ascontiguousarray(np.stack([fh.isotropic_stiffness(1.0, 1.0, 2)] * 2))
    eps0 = np.ascontiguousarray(np.eye(nv)[:1])
    out = np.zeros((1, nv))
    assert _call(fh, 2, m, 1, E, phase, Cp, eps0, out) == -1
    assert b"phase id" in fh.library().fh_last_error()
    ids[123] = 1                                           # the next call starts clean
    phase = torch.from_numpy(ids).cuda()
    assert _call(fh, 2, m, 1, E, phase, Cp, eps0, out) == 0
    assert np.allclose(out[0], Cp[0] @ eps0[0], rtol=1e-14, atol=0)
