"""Write the converged FP64 oracle C_eff of the benchmark workload (dlvp_sheared).

Calls only the oracle (and the seeded geometry of `workloads`).  The oracle is
iterated to a Cauchy residual of 1e-13 (Sec. 4's criterion, far below the 1e-6
used for timing), so the stored matrix is the discrete solution's C_eff to
within ~1e-12 relative.  Usage: python tests/golden/make_ceff_reference.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import generators as OG, green as OGr, material as OM, scheme as OS  # noqa: E402


def main():
    w = W.dlvp_sheared()
    T = OS.SNFTransform(w["M"])
    ids = W.phase_ids(T.points / T.D, w["centres"], w["radii"])
    lm = [OM.lame(E, nu) for E, nu in w["phases"]]
    Cp = np.stack([OM.isotropic_mandel(l, m, 2) for l, m in lm])
    l0, m0 = OM.reference_medium_ms([l for l, _ in lm], [m for _, m in lm])
    C0 = OM.isotropic_mandel(l0, m0, 2)
    Gp = OGr.gamma_p_table(w["M"], OG.Generator("dlvp", alpha=w["generator"]["alpha"]), C0, T.freqs)
    out = OS.solve(T, Gp, Cp[ids], C0, np.eye(3), tol=1e-13, max_iter=20000)
    Ce = OS.effective_stiffness(out["mean_stress"], np.eye(3))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ceff_dlvp_sheared.txt")
    with open(path, "w") as f:
        f.write("# C_eff (Mandel, 3x3) of workloads.dlvp_sheared from the FP64 oracle iterated to r <= 1e-13\n")
        f.write("# written by tests/golden/make_ceff_reference.py; iterations per load: "
                + " ".join(str(int(i)) for i in out["iters"]) + "\n")
        for row in Ce:
            f.write(" ".join(f"{v:.17e}" for v in row) + "\n")
    print(path)


if __name__ == "__main__":
    main()
