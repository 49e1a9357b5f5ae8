"""Shared set-up for the GPU parity tests: one workload built independently on the
oracle side and on the product side, plus the permutation between their point
orders (matched on the exact integer numerators of the pattern points)."""
import os
import sys

import numpy as np

import workloads as W
from oracle import generators as OG
from oracle import green as OGr
from oracle import lattice as OL
from oracle import material as OM
from oracle import scheme as OS


def oracle_generator(spec, d):
    k = spec["kind"]
    if k == "dirichlet":
        return OG.Generator("dirichlet")
    if k == "dlvp":
        return OG.Generator("dlvp", alpha=spec["alpha"])
    if k == "boxspline":
        xi = spec.get("xi")
        if xi is None:
            xi = OG.tensor_boxspline_xi(d, spec["order"])
        return OG.Generator("boxspline", xi=np.asarray(xi, float), radius=spec["radius"])
    raise ValueError(k)


def product_generator(fh, spec, d):
    k = spec["kind"]
    if k == "dirichlet":
        return fh.generator("dirichlet")
    if k == "dlvp":
        return fh.generator("dlvp", alpha=spec["alpha"])
    xi = spec.get("xi")
    if xi is None:
        xi = np.concatenate([np.eye(d)] * spec["order"], axis=1)
    return fh.generator("boxspline", xi=xi, radius=spec["radius"])


class Case:
    """A workload: M, generator spec, phases [(E, nu)], ball inclusions, load count."""

    def __init__(self, M, gen, phases, centres, radii, nload=None, brute=False):
        self.M = M
        self.d = len(M)
        self.nv = 3 if self.d == 2 else 6
        self.gen_spec = gen
        self.phases = phases
        self.centres = np.asarray(centres, float).reshape(-1, self.d)
        self.radii = np.asarray(radii, float)
        self.nload = self.nv if nload is None else nload
        self.eps0 = np.eye(self.nv)[: self.nload]
        T = OS.BruteTransform(M) if brute else OS.SNFTransform(M)
        self.T = T
        self.D = T.D
        self.ids = W.phase_ids(T.points / T.D, self.centres, self.radii)
        lm = [OM.lame(E, nu) for E, nu in phases]
        self.Cp_o = np.stack([OM.isotropic_mandel(l, m, self.d) for l, m in lm])
        l0, m0 = OM.reference_medium_ms([l for l, _ in lm], [m for _, m in lm])
        self.C0_o = OM.isotropic_mandel(l0, m0, self.d)
        self.gen_o = oracle_generator(gen, self.d)
        self._Gp = None

    @classmethod
    def from_workload(cls, w, nload=None):
        return cls(w["M"], w["generator"], w["phases"], w["centres"], w["radii"], nload=nload)

    @property
    def Gp(self):
        if self._Gp is None:
            self._Gp = OGr.gamma_p_table(self.M, self.gen_o, self.C0_o, self.T.freqs)
        return self._Gp

    def oracle_solve(self, tol=0.0, max_iter=10, eps0=None):
        e0 = self.eps0 if eps0 is None else eps0
        return OS.solve(self.T, self.Gp, self.Cp_o[self.ids], self.C0_o, e0, tol=tol, max_iter=max_iter)

    def product(self, fh, nload_max=None, stream=0, phase_tensor=None):
        p = fh.Pattern(self.M)
        A = p.numerators()
        idx = {tuple(a): i for i, a in enumerate(self.T.points.tolist())}
        perm = np.array([idx[tuple(a)] for a in A.tolist()])
        assert sorted(perm.tolist()) == list(range(self.D))
        ids_p = self.ids[perm]
        assert np.array_equal(ids_p, W.phase_ids(p.points(), self.centres, self.radii))
        Cp_p = np.stack([fh.isotropic_stiffness(*fh.lame(E, nu), self.d) for E, nu in self.phases])
        s = fh.Solver(p, product_generator(fh, self.gen_spec, self.d),
                      self.nload if nload_max is None else nload_max, stream)
        s.set_stiffness_phases(ids_p if phase_tensor is None else phase_tensor(ids_p), Cp_p)
        s.set_reference(None)
        self.perm = perm
        self.pattern = p
        return s

    def freq_perm(self, p):
        """Oracle index of every stored half-spectrum frequency of the product."""
        idx = {tuple(h): i for i, h in enumerate(self.T.freqs.tolist())}
        H = p.half_freqs()
        return np.array([idx[tuple(h)] for h in H.tolist()])

    def strain_error(self, s, oracle_E, loads=None):
        """max |E_gpu - E_oracle| / max |E_oracle + eps0| over the given loads."""
        worst = 0.0
        for L in range(self.nload) if loads is None else loads:
            Eg = s.get_strain(L)                       # (nv, m) product order
            Eo = oracle_E[L][self.perm].T              # (nv, m)
            scale = np.abs(Eo + self.eps0[L][:, None]).max()
            worst = max(worst, np.abs(Eg - Eo).max() / scale)
        return worst


def sampled_iteration_check(fh, w, loads, n_prev, nsample, seed, tol, precision=0):
    """One GPU iteration checked at sampled frequencies against the oracle.

    The GPU runs n_prev iterations (E_prev), then one more (E_next).  On the CPU,
    tau = (C - C0):(E_prev + eps0) is built with the oracle's own materials,
    transformed with numpy's FFT on the oracle's Smith grid, and the oracle's
    Gamma^p evaluated one frequency at a time at `nsample` random frequencies h
    predicts E^_next(h) = -Gamma^p_h tau^(h) (Eq. (pde_coefficients)), compared
    with the FFT of the GPU's E_next there.  `precision` selects the GPU's
    arithmetic (0: FP64, 1: FP32)."""
    case = Case.from_workload(w)   # oracle-side materials, generator, SNF grid (no table)
    s = case.product(fh)
    T = case.T
    rng = np.random.default_rng(seed)
    picks = rng.choice(T.m, size=nsample, replace=False)
    picks = picks[np.any(T.freqs[picks] != 0, axis=1)]
    Gp = np.stack([OGr.gamma_p(case.M, case.gen_o, case.C0_o, T.freqs[f]) for f in picks])
    dC = case.Cp_o[case.ids] - case.C0_o[None]
    inv = np.argsort(case.perm)            # oracle index -> product index
    worst = 0.0
    s.solve(case.eps0, tol=0.0, max_iter=n_prev, precision=precision)
    prev = {L: s.get_strain(L)[:, inv].T.copy() for L in loads}   # (m, nv) oracle order
    s.solve(case.eps0, tol=0.0, max_iter=1, init=1, precision=precision)
    for L in loads:
        nxt = s.get_strain(L)[:, inv].T
        tau = np.einsum("mab,mb->ma", dC, prev[L] + case.eps0[L][None])
        tau_h = T.fwd(tau.astype(complex))[picks]
        pred = -np.einsum("hab,hb->ha", Gp, tau_h)
        got = T.fwd(nxt.astype(complex))[picks]
        worst = max(worst, np.abs(pred - got).max() / np.abs(got).max())
    assert worst < tol, worst


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def det(M):
    return abs(OL.det_int(M))


def frob_rel(a, b):
    """Relative Frobenius distance ||a - b|| / ||b||."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
from golden_io import read_golden_blocks  # noqa: E402,F401
