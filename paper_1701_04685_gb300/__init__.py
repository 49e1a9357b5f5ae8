"""GB300 Basic-Scheme solver for FFT-based homogenisation on anisotropic patterns.

Thin ctypes binding of the C ABI in ``include/fftHomog.h`` (argument
marshalling only; every step of the iteration runs in the CUDA library
``_build/libffthomog.so``).  Method: Bergmann & Merkert, arXiv 1701.04685 --
the fixed point of Eq. (pde_coefficients) on the pattern P(M) with the
periodised Green operator Gamma^p of Def. gamma_tilde_fourier.

Arrays may be numpy arrays (host) or CUDA torch tensors (device) where the C
ABI says "host or device".  The library must have been built
(``paper_1701_04685_gb300.build.build()``); importing the binding never falls
back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, LIB_CHECKED

FH_OK, FH_NOT_CONVERGED, FH_DIVERGED, FH_NONFINITE = 0, 1, 2, 3
FH_ERR_ARG, FH_ERR_INTERNAL, FH_ERR_UNSUPPORTED = -1, -7, -8
FH_GEN_DIRICHLET, FH_GEN_DLVP, FH_GEN_BOXSPLINE = 0, 1, 2
FH_PREC_FP64, FH_PREC_FP32, FH_PREC_MIXED = 0, 1, 2
FH_MAX_LOADS = 16
FH_TUNE_CANDIDATES = 8
FH_MAX_XI = 16

_STATUS = {0: "ok", 1: "not converged", 2: "diverged", 3: "non-finite", -1: "invalid argument",
           -2: "singular M", -3: "overflow", -4: "no orthonormal basis", -5: "CUDA error",
           -6: "timeout", -7: "internal error", -8: "unsupported", -9: "call order"}


class FhError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)} ({status}): {msg}")
        self.status = status


class fh_generator(C.Structure):
    _fields_ = [("kind", C.c_int), ("alpha", C.c_double * 3), ("n_xi", C.c_int),
                ("xi", C.c_double * (3 * FH_MAX_XI)), ("alias_radius", C.c_int)]


class fh_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("precision", C.c_int),
                ("init", C.c_int), ("chunk", C.c_int), ("path", C.c_int), ("cluster", C.c_int),
                ("form", C.c_int), ("tune", C.c_int), ("method", C.c_int)]


class fh_result(C.Structure):
    _fields_ = [("iterations", C.c_int * FH_MAX_LOADS), ("residual", C.c_double * FH_MAX_LOADS),
                ("status", C.c_int * FH_MAX_LOADS), ("mean_stress", C.c_double * (FH_MAX_LOADS * 6)),
                ("elapsed_ms", C.c_double), ("kernel_launches", C.c_longlong), ("path", C.c_int),
                ("cluster", C.c_int)]


_lib = None


def library():
    """The loaded CUDA library; raises if it has not been built.  With the
    environment variable FH_CHECKED=1 at the first call, the checked build
    (``build(checked=True)``: index checks in the solver kernels) is loaded
    instead of the normal one."""
    global _lib
    if _lib is None:
        path = LIB_CHECKED if os.environ.get("FH_CHECKED") == "1" else LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run paper_1701_04685_gb300.build.build()")
        lib = C.CDLL(path)
        P, I, D, V = C.c_void_p, C.c_int, C.c_double, None
        sig = {
            "fh_pattern_create": (I, [I, P, C.POINTER(P)]),
            "fh_pattern_destroy": (V, [P]),
            "fh_pattern_info": (I, [P, P, P, P]),
            "fh_pattern_points": (I, [P, P]),
            "fh_pattern_numerators": (I, [P, P]),
            "fh_pattern_half_freqs": (I, [P, P, P]),
            "fh_solver_create": (I, [P, C.POINTER(fh_generator), I, P, C.POINTER(P)]),
            "fh_solver_destroy": (V, [P]),
            "fh_set_stiffness_phases": (I, [P, P, I, P]),
            "fh_set_stiffness_field": (I, [P, P]),
            "fh_set_reference": (I, [P, P]),
            "fh_solve": (I, [P, I, P, C.POINTER(fh_solve_opts), C.POINTER(fh_result)]),
            "fh_get_strain": (I, [P, I, P]),
            "fh_set_strain": (I, [P, I, P]),
            "fh_get_ceff": (I, [P, P, I]),
            "fh_get_green": (I, [P, P]),
            "fh_get_residuals": (I, [P, I, P, P]),
            "fh_profile_passes": (I, [P, I, I, I, P]),
            "fh_solve_batch": (I, [P, I, P, P, C.POINTER(fh_solve_opts), P]),
            "fh_get_tuning": (I, [P, I, P, P, P, P]),
            "fh_status_string": (C.c_char_p, [I]),
            "fh_last_error": (C.c_char_p, []),
            "fh_checked_build": (I, []),
            "fh_check_selftest": (I, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    """Names of the C entry points the binding expects (all declared in fftHomog.h)."""
    return FNO_SYMBOLS + ["fh_pattern_create", "fh_pattern_destroy", "fh_pattern_info", "fh_pattern_points",
            "fh_pattern_numerators", "fh_pattern_half_freqs", "fh_solver_create", "fh_solver_destroy",
            "fh_set_stiffness_phases", "fh_set_stiffness_field", "fh_set_reference", "fh_solve", "fh_get_strain", "fh_set_strain",
            "fh_get_ceff", "fh_get_green", "fh_get_residuals", "fh_profile_passes", "fh_status_string",
            "fh_last_error", "fh_mean_stress_noalloc", "fh_solve_batch",
            "fh_get_tuning", "fh_checked_build", "fh_check_selftest"]


def checked_build():
    """True when the loaded library is the checked build (FH_CHECKED=1)."""
    return bool(library().fh_checked_build())


def check_selftest():
    """Checked build: the status of the index checks' self test (FH_ERR_INTERNAL
    with the self test named when the checks work); normal build:
    FH_ERR_UNSUPPORTED.  Returns (status, message)."""
    rc = library().fh_check_selftest()
    return rc, library().fh_last_error().decode()


def _check(rc, ok=(FH_OK,)):
    if rc not in ok:
        raise FhError(rc, library().fh_last_error().decode())
    return rc


def _ptr(a):
    """Address of a contiguous numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(a.ctypes.data)


def _buf(x, count, dtype, what, writable=False):
    """A buffer of exactly `count` elements of `dtype` for a C entry point.

    A torch tensor (host or CUDA) is checked and passed as it is.  A numpy
    array that the call writes (`writable`) is checked too; any other host
    input is converted to a contiguous `dtype` array.  A mismatch raises
    ValueError before the C call, which would otherwise read or write past
    the buffer."""
    dt = np.dtype(dtype)
    if hasattr(x, "data_ptr"):
        tdt = str(x.dtype).replace("torch.", "")
        if x.numel() != count or tdt != dt.name or not x.is_contiguous():
            raise ValueError(f"{what}: need a contiguous {dt.name} tensor of {count} elements, "
                             f"got {tdt} of shape {tuple(x.shape)}")
        return x
    if writable:
        if not isinstance(x, np.ndarray) or x.dtype != dt or x.size != count or not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{what}: need a C-contiguous {dt.name} array of {count} elements")
        return x
    a = np.ascontiguousarray(np.asarray(x, dtype=dt))
    if a.size != count:
        raise ValueError(f"{what}: need {count} elements, got shape {a.shape}")
    return a


def nv_of(d):
    return 3 if d == 2 else 6


# ---------------------------------------------------------------------------
# stiffness helpers (Mandel form, Sec. 3.1)
# ---------------------------------------------------------------------------

def lame(E, nu):
    """Lame constants lambda, mu of an isotropic solid (also used for plane strain)."""
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def isotropic_stiffness(lam, mu, d):
    """Mandel matrix of C = lam I(x)I + 2 mu Id: diagonal blocks lam + 2 mu / lam, shear 2 mu."""
    n = nv_of(d)
    Cm = np.zeros((n, n))
    Cm[:d, :d] = lam
    Cm[np.arange(d), np.arange(d)] = lam + 2 * mu
    Cm[np.arange(d, n), np.arange(d, n)] = 2 * mu
    return Cm


def generator(kind="dirichlet", alpha=None, xi=None, radius=0):
    """fh_generator for 'dirichlet', 'dlvp' (alpha = half ramp widths) or 'boxspline' (xi: d x s)."""
    g = fh_generator()
    if kind == "dirichlet":
        g.kind = FH_GEN_DIRICHLET
    elif kind == "dlvp":
        g.kind = FH_GEN_DLVP
        for i, a in enumerate(alpha):
            g.alpha[i] = float(a)
    elif kind == "boxspline":
        g.kind = FH_GEN_BOXSPLINE
        xi = np.asarray(xi, dtype=float)
        d, s = xi.shape
        g.n_xi = s
        for k in range(s):
            for i in range(d):
                g.xi[3 * k + i] = xi[i, k]
        g.alias_radius = int(radius)
    else:
        raise ValueError(kind)
    return g


def tensor_boxspline(d, order, radius):
    """Box spline with `order` copies of each unit vector (tensor-product B-spline)."""
    return generator("boxspline", xi=np.concatenate([np.eye(d)] * order, axis=1), radius=radius)


# ---------------------------------------------------------------------------
# pattern and solver objects (one method per C entry point)
# ---------------------------------------------------------------------------

class Pattern:
    """P(M) and G(M^T) of a regular integer matrix M (fh_pattern_*)."""

    def __init__(self, M):
        M = np.ascontiguousarray(np.asarray(M, dtype=np.int64))
        if M.ndim != 2 or M.shape[0] != M.shape[1] or M.shape[0] not in (2, 3):
            raise ValueError(f"M: need a square 2 x 2 or 3 x 3 integer matrix, got shape {M.shape}")
        self.d = M.shape[0]
        self.M = M
        h = C.c_void_p()
        _check(library().fh_pattern_create(self.d, _ptr(M), C.byref(h)))
        self._h = h
        m = C.c_int64()
        nd = C.c_int()
        dims = (C.c_int * 3)()
        _check(library().fh_pattern_info(h, C.byref(m), C.byref(nd), dims))
        self.m = m.value
        self.dims = [dims[k] for k in range(nd.value)]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fh_pattern_destroy(self._h)
            self._h = None

    def points(self):
        y = np.empty((self.m, self.d))
        _check(library().fh_pattern_points(self._h, _ptr(y)))
        return y

    def numerators(self):
        a = np.empty((self.m, self.d), dtype=np.int64)
        _check(library().fh_pattern_numerators(self._h, _ptr(a)))
        return a

    def half_freqs(self):
        nh = C.c_int64()
        _check(library().fh_pattern_half_freqs(self._h, None, C.byref(nh)))
        h = np.empty((nh.value, self.d), dtype=np.int64)
        _check(library().fh_pattern_half_freqs(self._h, _ptr(h), C.byref(nh)))
        return h


class Solver:
    """Basic-Scheme solver for one pattern and generator (fh_solver_*)."""

    def __init__(self, pattern, gen, nload_max, stream=0):
        self.pattern = pattern
        self.d = pattern.d
        self.nv = nv_of(self.d)
        self.m = pattern.m
        h = C.c_void_p()
        _check(library().fh_solver_create(pattern._h, C.byref(gen), int(nload_max), C.c_void_p(stream), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fh_solver_destroy(self._h)
            self._h = None

    __del__ = close

    def set_stiffness_phases(self, phase, Cp):
        """phase: m uint8 ids in storage order (numpy, or a host or CUDA tensor);
        Cp: (nphase, n_v, n_v) Mandel matrices."""
        Cp = np.ascontiguousarray(np.asarray(Cp, dtype=np.float64))
        if Cp.ndim != 3 or Cp.shape[1:] != (self.nv, self.nv):
            raise ValueError(f"Cp: need shape (nphase, {self.nv}, {self.nv}), got {Cp.shape}")
        if hasattr(phase, "data_ptr"):
            ph = _buf(phase, self.m, np.uint8, "phase")
        else:
            ph = np.asarray(phase)
            if ph.dtype != np.uint8 and ph.size and (ph.min() < 0 or ph.max() > 255):
                raise ValueError("phase: ids must lie in 0..255")
            ph = _buf(ph, self.m, np.uint8, "phase")
        _check(library().fh_set_stiffness_phases(self._h, _ptr(ph), int(Cp.shape[0]), _ptr(Cp)))

    def set_stiffness_field(self, C):
        """Point-by-point Mandel stiffness, shape (m, n_v, n_v) in storage order
        (numpy array or a CUDA tensor of float64)."""
        Cf = _buf(C, self.m * self.nv * self.nv, np.float64, "stiffness field")
        _check(library().fh_set_stiffness_field(self._h, _ptr(Cf)))

    def set_reference(self, C0=None):
        if C0 is None:
            _check(library().fh_set_reference(self._h, None))
        else:
            C0 = _buf(C0, self.nv * self.nv, np.float64, "C0")
            _check(library().fh_set_reference(self._h, _ptr(C0)))

    def solve(self, eps0, tol=1e-8, max_iter=1000, precision=FH_PREC_FP64, init=0, chunk=0, path=0, cluster=0,
              form=0, tune=0, method=0):
        """path: 0 automatic, 1 whole-GPU passes, 2 cluster-resident (2-axis grids);
        form: 0 Eq. (pde_coefficients), 1 the variational discretisation;
        tune: 1 picks path and cluster size by timing them (see fh_get_tuning);
        method: 0 the fixed point, 1 BiCGStab on the same equation."""
        eps0 = np.ascontiguousarray(np.atleast_2d(np.asarray(eps0, dtype=np.float64)))
        if eps0.ndim != 2 or eps0.shape[1] != self.nv:
            raise ValueError(f"eps0: need shape (n_L, {self.nv}), got {eps0.shape}")
        opts = fh_solve_opts(float(tol), int(max_iter), int(precision), int(init), int(chunk), int(path),
                             int(cluster), int(form), int(tune), int(method))
        res = fh_result()
        rc = library().fh_solve(self._h, eps0.shape[0], _ptr(eps0), C.byref(opts), C.byref(res))
        _check(rc, ok=(FH_OK, FH_NOT_CONVERGED, FH_DIVERGED, FH_NONFINITE))
        n = eps0.shape[0]
        return {
            "status": rc,
            "iterations": np.array(res.iterations[:n]),
            "residual": np.array(res.residual[:n]),
            "load_status": np.array(res.status[:n]),
            "mean_stress": np.array(res.mean_stress[: n * 6]).reshape(n, 6)[:, : self.nv],
            "elapsed_ms": res.elapsed_ms,
            "kernel_launches": res.kernel_launches,
            "path": res.path,
            "cluster": res.cluster,
        }

    def get_strain(self, load, out=None):
        """E of one load as (n_v, m) float64 (numpy, or into a given CUDA tensor)."""
        if out is None:
            out = np.empty((self.nv, self.m))
        out = _buf(out, self.nv * self.m, np.float64, "strain", writable=True)
        _check(library().fh_get_strain(self._h, int(load), _ptr(out)))
        return out

    def set_strain(self, load, E):
        E = _buf(E, self.nv * self.m, np.float64, "strain")
        _check(library().fh_set_strain(self._h, int(load), _ptr(E)))

    def get_ceff(self, voigt=False):
        out = np.empty((self.nv, self.nv))
        _check(library().fh_get_ceff(self._h, _ptr(out), int(bool(voigt))))
        return out

    def get_green(self):
        nh = len(self.pattern.half_freqs())
        out = np.empty((nh, self.nv, self.nv))
        _check(library().fh_get_green(self._h, _ptr(out)))
        return out

    def get_tuning(self, precision):
        path, cl, cand = C.c_int(), C.c_int(), C.c_int()
        us = (C.c_float * FH_TUNE_CANDIDATES)()
        _check(library().fh_get_tuning(self._h, int(precision), C.byref(path), C.byref(cl), C.byref(cand), us))
        return {"path": path.value, "cluster": cl.value, "candidate": cand.value, "us_per_iter": list(us)}

    def get_residuals(self, load):
        n = C.c_int()
        _check(library().fh_get_residuals(self._h, int(load), None, C.byref(n)))
        out = np.empty(n.value)
        if n.value:
            _check(library().fh_get_residuals(self._h, int(load), _ptr(out), C.byref(n)))
        return out

    def profile_passes(self, nload, precision=FH_PREC_FP64, reps=50):
        """Mean ms per launch of [row pass, axis-0 Green pass, mid forward, mid inverse]."""
        ms = np.zeros(4)
        _check(library().fh_profile_passes(self._h, int(nload), int(precision), int(reps), _ptr(ms)))
        return ms


def solve_batch(solvers, eps0s, tol=1e-6, max_iter=20000, precision=FH_PREC_MIXED, init=0, chunk=0, path=0,
                cluster=0, form=0, method=0):
    """fh_solve_batch over Solver objects; eps0s[i] is solver i's (n_L, n_v) strains.  With path and
    cluster automatic, solvers tuned before (Solver.solve(..., tune=1)) keep their tuned choice."""
    n = len(solvers)
    if len(eps0s) != n:
        raise ValueError("one eps0 array per solver")
    e0 = [np.ascontiguousarray(np.atleast_2d(np.asarray(e, dtype=np.float64))) for e in eps0s]
    for e, sv in zip(e0, solvers):
        if e.ndim != 2 or e.shape[1] != sv.nv:
            raise ValueError(f"eps0: need shape (n_L, {sv.nv}), got {e.shape}")
    hs = (C.c_void_p * n)(*[sv._h.value for sv in solvers])
    nl = (C.c_int * n)(*[e.shape[0] for e in e0])
    ptrs = (C.c_void_p * n)(*[e.ctypes.data for e in e0])
    opts = fh_solve_opts(float(tol), int(max_iter), int(precision), int(init), int(chunk), int(path), int(cluster),
                         int(form), 0, int(method))
    res = (fh_result * n)()
    rc = library().fh_solve_batch(hs, n, nl, ptrs, C.byref(opts), res)
    _check(rc, ok=(FH_OK, FH_NOT_CONVERGED, FH_DIVERGED, FH_NONFINITE))
    out = []
    for i, sv in enumerate(solvers):
        k = e0[i].shape[0]
        out.append({"iterations": np.array(res[i].iterations[:k]), "residual": np.array(res[i].residual[:k]),
                    "load_status": np.array(res[i].status[:k]),
                    "mean_stress": np.array(res[i].mean_stress[: k * 6]).reshape(k, 6)[:, : sv.nv],
                    "elapsed_ms": res[i].elapsed_ms, "kernel_launches": res[i].kernel_launches,
                    "path": res[i].path, "cluster": res[i].cluster})
    return rc, out


# ---------------------------------------------------------------------------
# learned start (fh_fno_*)
# ---------------------------------------------------------------------------

def _sig_fno():
    lib = library()
    P, I, V = C.c_void_p, C.c_int, None
    sig = {
        "fh_fno_create": (I, [I, I, I, I, I, I, I, P, C.POINTER(P)]),
        "fh_fno_destroy": (V, [P]),
        "fh_fno_param_count": (I, [P, P]),
        "fh_fno_set_params": (I, [P, P]),
        "fh_fno_get_params": (I, [P, P]),
        "fh_fno_get_grads": (I, [P, P]),
        "fh_fno_zero_grad": (I, [P]),
        "fh_fno_forward": (I, [P, I, P, P]),
        "fh_fno_set_tensor_cores": (I, [P, I]),
        "fh_fno_loss_grad": (I, [P, I, P, P, P]),
        "fh_fno_adam_step": (I, [P, C.c_float, C.c_float, C.c_float, C.c_float, I]),
        "fh_fno_make_input": (I, [P, P, I, P, P, P]),
        "fh_get_strain_f32": (I, [P, I, P]),
        "fh_set_strain_f32": (I, [P, I, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


FNO_SYMBOLS = ["fh_fno_create", "fh_fno_destroy", "fh_fno_param_count", "fh_fno_set_params", "fh_fno_get_params",
               "fh_fno_get_grads", "fh_fno_zero_grad", "fh_fno_forward", "fh_fno_loss_grad", "fh_fno_adam_step",
               "fh_fno_make_input", "fh_fno_set_tensor_cores", "fh_get_strain_f32", "fh_set_strain_f32"]


class FNO:
    """Fourier neural operator for the starting strain (fh_fno_*); device tensors in, out."""

    def __init__(self, n, cin=7, cout=6, width=32, modes=12, layers=4, max_batch=4, stream=0):
        lib = _sig_fno()
        h = C.c_void_p()
        _check(lib.fh_fno_create(n, cin, cout, width, modes, layers, max_batch, C.c_void_p(stream), C.byref(h)))
        self._h = h
        self.n, self.cin, self.cout, self.width, self.modes, self.layers = n, cin, cout, width, modes, layers
        cnt = C.c_longlong()
        _check(lib.fh_fno_param_count(h, C.byref(cnt)))
        self.nparam = cnt.value

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fh_fno_destroy(self._h)
            self._h = None

    __del__ = close

    def set_params(self, flat):
        flat = _buf(flat, self.nparam, np.float32, "params")
        _check(library().fh_fno_set_params(self._h, _ptr(flat)))

    def get_params(self):
        out = np.empty(self.nparam, dtype=np.float32)
        _check(library().fh_fno_get_params(self._h, _ptr(out)))
        return out

    def get_grads(self):
        out = np.empty(self.nparam, dtype=np.float32)
        _check(library().fh_fno_get_grads(self._h, _ptr(out)))
        return out

    def set_tensor_cores(self, enable):
        """Hidden 1 x 1 layers on the tensor cores (tcgen05) or as SIMT loops."""
        _check(library().fh_fno_set_tensor_cores(self._h, int(bool(enable))))

    def zero_grad(self):
        _check(library().fh_fno_zero_grad(self._h))

    def _io(self, x, other, ch, what):
        """Batch size of device input x (batch, cin, n^3) and the checked `other` (batch, ch, n^3)."""
        if not hasattr(x, "data_ptr") or not hasattr(other, "data_ptr"):
            raise ValueError("FNO inputs and outputs are device tensors")
        b = int(x.shape[0])
        _buf(x, b * self.cin * self.n ** 3, np.float32, "x")
        _buf(other, b * ch * self.n ** 3, np.float32, what)
        return b

    def forward(self, x, y):
        b = self._io(x, y, self.cout, "y")
        _check(library().fh_fno_forward(self._h, b, _ptr(x), _ptr(y)))
        return y

    def loss_grad(self, x, target):
        b = self._io(x, target, self.cout, "target")
        loss = C.c_double()
        _check(library().fh_fno_loss_grad(self._h, b, _ptr(x), _ptr(target), C.byref(loss)))
        return loss.value

    def adam_step(self, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(library().fh_fno_adam_step(self._h, float(lr), float(beta1), float(beta2), float(eps), int(step)))

    def make_input(self, phase, phase_logE, eps0, x):
        if not hasattr(phase, "data_ptr") or not hasattr(x, "data_ptr"):
            raise ValueError("phase and x are device tensors")
        _buf(phase, self.n ** 3, np.uint8, "phase")
        _buf(x, self.cin * self.n ** 3, np.float32, "x")
        plE = np.ascontiguousarray(np.asarray(phase_logE, dtype=np.float64)).ravel()
        e0 = _buf(eps0, 6, np.float64, "eps0")
        _check(library().fh_fno_make_input(self._h, _ptr(phase), len(plE), _ptr(plE), _ptr(e0), _ptr(x)))
        return x


def get_strain_f32(solver, load, out):
    out = _buf(out, solver.nv * solver.m, np.float32, "strain", writable=True)
    _check(_sig_fno().fh_get_strain_f32(solver._h, int(load), _ptr(out)))
    return out


def set_strain_f32(solver, load, E):
    E = _buf(E, solver.nv * solver.m, np.float32, "strain")
    _check(_sig_fno().fh_set_strain_f32(solver._h, int(load), _ptr(E)))
