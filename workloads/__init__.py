"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds geometry and material parameters only -- none of the
homogenisation method's arithmetic.  It draws random inclusion layouts
(disks in 2-D, spheres in 3-D) in the periodic unit cell [-1/2, 1/2)^d,
assigns a phase to each pattern point (collocation: a point belongs to an
inclusion iff its periodic distance to the centre is strictly less than the
radius) and states the workloads used for parity tests and timing:

* ``disk32``       M = diag(32,32), Dirichlet kernel, matrix E=1, one centred
                   disk of volume fraction 0.2 with E=10, nu=0.3, 3 loads,
                   Cauchy tolerance 1e-8.
* ``dlvp_sheared`` M = [[128,32],[0,128]] (m = 16384, grid 32 x 512), de la
                   Vallee Poussin trapezoid with plateau |u| <= 0.25 and ramp
                   to 0.75, 20 non-overlapping disks with radii U[0.03,0.08],
                   contrast 100, nu=0.3, 3 loads.
* ``box3d``        M = diag(128,128,128), tensor-product box spline of order 2
                   with alias radius 4, 50 non-overlapping spheres with radii
                   U[0.05,0.1], E_incl=50, E_mat=1, nu=0.3, 6 loads.
* ``batch2d``      512 two-phase 2-D microstructures with N drawn from
                   {64,96,128,192,256}, half diag(N,N), half [[N,s],[0,N]] with
                   s in {N/8,N/4,N/2}, 5..30 disks with radii U[0.03,0.1],
                   contrast log-uniform in [5,200], 3 loads each.
* ``fno3d``        M = diag(64,64,64), Dirichlet kernel, spheres with radii
                   U[0.06,0.12] added until a volume fraction drawn from
                   U[0.1,0.35], contrast U[10,100].

All randomness comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math

import numpy as np

NU = 0.3


def periodic_delta(y, c):
    """Nearest-image difference y - c in the unit cell, componentwise."""
    t = np.asarray(y, dtype=float) - np.asarray(c, dtype=float)
    return t - np.round(t)


def random_inclusions(rng, d, count, rmin, rmax, max_tries=200000):
    """``count`` non-overlapping periodic balls: centres in [-1/2,1/2)^d, radii U[rmin,rmax]."""
    centres, radii = [], []
    tries = 0
    while len(centres) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place the requested inclusions")
        c = rng.uniform(-0.5, 0.5, size=d)
        r = rng.uniform(rmin, rmax)
        ok = True
        for c2, r2 in zip(centres, radii):
            if np.linalg.norm(periodic_delta(c, c2)) <= r + r2:
                ok = False
                break
        if ok:
            centres.append(c)
            radii.append(r)
    return np.array(centres).reshape(-1, d), np.array(radii)


def inclusions_to_fraction(rng, d, target_vf, rmin, rmax, max_tries=200000):
    """Add non-overlapping periodic balls until their total volume reaches ``target_vf``."""
    unit = math.pi if d == 2 else 4.0 * math.pi / 3.0
    centres, radii = [], []
    vf, tries = 0.0, 0
    while vf < target_vf and tries < max_tries:
        tries += 1
        c = rng.uniform(-0.5, 0.5, size=d)
        r = rng.uniform(rmin, rmax)
        if all(np.linalg.norm(periodic_delta(c, c2)) > r + r2 for c2, r2 in zip(centres, radii)):
            centres.append(c)
            radii.append(r)
            vf += unit * r ** d
    return np.array(centres).reshape(-1, d), np.array(radii)


def phase_ids(points, centres, radii):
    """uint8 phase per point: 1 inside any ball (strict), else 0."""
    y = np.asarray(points, dtype=float)
    ph = np.zeros(len(y), dtype=np.uint8)
    for c, r in zip(centres, radii):
        dd = periodic_delta(y, c[None, :])
        ph[np.sum(dd * dd, axis=1) < r * r] = 1
    return ph


def laminate_ids(points, axis, fraction):
    """Layered phase field: phase 1 where y_axis lies in [-fraction/2, fraction/2)."""
    y = np.asarray(points, dtype=float)[:, axis]
    return ((y >= -fraction / 2) & (y < fraction / 2)).astype(np.uint8)


def mandel_units(nv):
    """The n_v macroscopic unit strains (Mandel basis vectors) used for C_eff."""
    return np.eye(nv)


# ---------------------------------------------------------------------------
# workload descriptions
# ---------------------------------------------------------------------------

def disk32():
    vf = 0.2
    return {
        "name": "disk32", "d": 2, "M": [[32, 0], [0, 32]],
        "generator": {"kind": "dirichlet"},
        "phases": [(1.0, NU), (10.0, NU)],
        "centres": np.zeros((1, 2)), "radii": np.array([math.sqrt(vf / math.pi)]),
        "nload": 3, "tol": 1e-8,
    }


def dlvp_sheared(seed=2):
    rng = np.random.default_rng(seed)
    c, r = random_inclusions(rng, 2, 20, 0.03, 0.08)
    return {
        "name": "dlvp_sheared", "d": 2, "M": [[128, 32], [0, 128]],
        "generator": {"kind": "dlvp", "alpha": [0.25, 0.25]},
        "phases": [(1.0, NU), (100.0, NU)],
        "centres": c, "radii": r, "nload": 3, "tol": 1e-6,
    }


def box3d(seed=3, n=128, count=50):
    rng = np.random.default_rng(seed)
    c, r = random_inclusions(rng, 3, count, 0.05, 0.1)
    return {
        "name": "box3d", "d": 3, "M": [[n, 0, 0], [0, n, 0], [0, 0, n]],
        "generator": {"kind": "boxspline", "order": 2, "radius": 4},
        "phases": [(1.0, NU), (50.0, NU)],
        "centres": c, "radii": r, "nload": 6, "tol": 1e-6,
    }


def batch2d_item(i):
    rng = np.random.default_rng(4000 + i)
    N = int(rng.choice([64, 96, 128, 192, 256]))
    if i % 2 == 0:
        M = [[N, 0], [0, N]]
    else:
        s = N // int(rng.choice([8, 4, 2]))
        M = [[N, s], [0, N]]
    count = int(rng.integers(5, 31))
    c, r = random_inclusions(rng, 2, count, 0.03, 0.1)
    contrast = float(math.exp(rng.uniform(math.log(5.0), math.log(200.0))))
    return {
        "name": f"batch2d[{i}]", "d": 2, "M": M,
        "generator": {"kind": "dirichlet"},
        "phases": [(1.0, NU), (contrast, NU)],
        "centres": c, "radii": r, "nload": 3, "tol": 1e-6,
    }


def fno3d_item(seed, n=64):
    rng = np.random.default_rng(seed)
    vf = rng.uniform(0.1, 0.35)
    c, r = inclusions_to_fraction(rng, 3, vf, 0.06, 0.12)
    contrast = float(rng.uniform(10.0, 100.0))
    return {
        "name": f"fno3d[{seed}]", "d": 3, "M": [[n, 0, 0], [0, n, 0], [0, 0, n]],
        "generator": {"kind": "dirichlet"},
        "phases": [(1.0, NU), (contrast, NU)],
        "centres": c, "radii": r, "nload": 6, "tol": 1e-6,
    }
