"""The bounds-check build (-DTF_BOUNDS_CHECK) on small, ragged and degenerate grids.

libtwofluid_bc.so checks the shared-memory and global indices of the tile,
strip and ensemble kernels against their extents; an index out of range is
redirected to 0 and reported as TF_ERR_BOUNDS by tf_sync, with no trap.  This
is the stand-in for a memory checker: the cases of bounds_check_cases.py must
run through it with no failed check, and give bitwise the same fields as the
normal library.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_check_build_reports_nothing_and_matches(tmp_path):
    from paper_2511_00445_gb300 import build
    build.build()
    import bounds_check_cases as C
    out = tmp_path / "bc.npz"
    env = dict(os.environ, TF_LIBRARY=build.BC_LIB_PATH)
    res = subprocess.run([sys.executable, os.path.join(HERE, "bounds_check_cases.py"), str(out)],
                         env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "libtwofluid_bc.so" in res.stdout
    checked = np.load(out)
    plain = C.run_cases()
    assert set(checked.files) == set(plain)
    for k, v in plain.items():
        assert np.array_equal(checked[k], v), k
