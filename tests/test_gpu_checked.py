"""The bounds-checked build (CFD_BOUNDS_CHECK): the same cases as the
normal build, run through the checked library in a process of its own, raise
no out-of-range index and give the same bits."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(lib, out):
    env = dict(os.environ, CFD_GB300_LIB=lib, PYTHONPATH=os.pathsep.join([os.path.dirname(HERE), HERE]))
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py"), out], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    return np.load(out)


def test_bounds_checked_build_runs_clean_and_identical(tmp_path):
    from paper_2209_15333_gb300 import build
    normal = build.build()
    checked = build.build(checked=True)
    a = _run(normal, str(tmp_path / "normal.npz"))
    b = _run(checked, str(tmp_path / "checked.npz"))
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
