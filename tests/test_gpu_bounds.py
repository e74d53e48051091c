"""The bounds-checked build (libstokes_gb300_check.so, -DSTK_BOUNDS_CHECK):
every index the stencil, transfer and coarse-level kernels form is checked
against its array's length; an out-of-range index is counted and redirected
to element 0, so nothing faults.  A self-test kernel, which checks one index
out of range by one without touching memory, shows that the count works;
then small and odd-shaped grids with every boundary mix, both precisions and
the schedules that put the two-colour and coarse-level kernels on every
level run without a single out-of-range index."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECK_LIB = os.path.join(ROOT, "paper_1308_4605_gb300", "libstokes_gb300_check.so")


def test_bounds_checked_build_meets_no_out_of_range_index():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(CHECK_LIB):
        subprocess.run([sys.executable, "-m", "paper_1308_4605_gb300.build", "--bounds-check"],
                       cwd=ROOT, check=True, capture_output=True)
    env = dict(os.environ, STK_LIBRARY=CHECK_LIB)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_check_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["library"] == CHECK_LIB
    assert out["selftest"] == [1, 2, 7]            # counted: kind 2 (cell), index 7
    assert out["violations"][0] == 0, out["violations"]
    for rec in out["cases"]:
        for key, val in rec.items():
            if key.startswith("p"):
                its, res = val
                assert res <= 1e-10, (rec["n"], rec["bc"], key, its, res)


def test_release_build_reports_no_checks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_4605_gb300 import stokes as S
    if S.LIB_PATH.endswith("_check.so"):
        pytest.skip("running under the bounds-checked library")
    assert S.stk_bounds_violations()[0] == -1
    with pytest.raises(S.StokesError):
        S.stk_bounds_selftest()
