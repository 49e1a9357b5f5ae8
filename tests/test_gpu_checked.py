"""The checked build (-DFH_CHECKED): index checks in the solver's kernels.

The solver is compiled a second time with the checks (``build(checked=True)``)
and loaded in a child process (FH_CHECKED=1).  There the self test must
report the index it placed outside its extent, and small solves over every
kernel family -- the 2-D cluster solve and passes, 3-D block and warp passes
in FP64 and FP32 with both column-pass forms, BiCGStab, a batch, the
point-by-point stiffness -- must run without a violation (any would turn the
status into FH_ERR_INTERNAL and raise) and agree with the normal build: the
checks only skip accesses, so the results match to rounding (the compiler may
contract a few operations differently)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def fh():
    import torch
    assert torch.cuda.is_available()
    from paper_1701_04685_gb300 import build
    build.build()
    import paper_1701_04685_gb300 as fh
    return fh


def test_normal_build_has_no_checks(fh):
    assert not fh.checked_build()
    rc, msg = fh.check_selftest()
    assert rc == fh.FH_ERR_UNSUPPORTED and "checked build" in msg


def test_checked_build_runs_every_kernel_family_clean(fh, tmp_path):
    from paper_1701_04685_gb300 import build
    build.build(checked=True)
    out = tmp_path / "checked.npz"
    env = dict(os.environ, FH_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    got = dict(np.load(out))
    assert int(got.pop("checked")) == 1
    rc = int(got.pop("selftest_status"))
    msg = str(got.pop("selftest_message"))
    assert rc == fh.FH_ERR_INTERNAL, msg
    assert "self test" in msg and "index 5 outside [0, 4)" in msg and "(1 accesses)" in msg
    sys.path.insert(0, HERE)
    import checked_cases
    ref = checked_cases.run_cases(fh)
    assert set(ref) == set(got)
    for k in sorted(ref):
        a, b = got[k], ref[k]
        if k.endswith("/iters"):
            assert np.array_equal(a, b), k
            continue
        fp32 = "prec1" in k or "fp32" in k
        tol = 1e-5 if fp32 else 1e-11
        scale = max(np.abs(b).max(), 1e-300)
        assert np.abs(a - b).max() <= tol * scale, (k, np.abs(a - b).max() / scale)
