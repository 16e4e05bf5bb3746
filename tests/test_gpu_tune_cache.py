"""The autotuner's choices persist across processes: the first process times
the kernel variants on its first step (extra launches), a second process
with the same cache file finds its choices there and launches on its first
step exactly what every later step launches, for a single-block context and
for an ensemble."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_15333_gb300 import build
    build.build()


def _run(cache):
    env = dict(os.environ, CFD_GB300_TUNE_CACHE=cache, PYTHONPATH=os.pathsep.join([os.path.dirname(HERE), HERE]))
    r = subprocess.run([sys.executable, os.path.join(HERE, "tune_cache_run.py")], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_second_process_skips_the_trial_launches(tmp_path):
    cache = str(tmp_path / "autotune.txt")
    a = _run(cache)
    b = _run(cache)
    for kind in ("single", "batch"):
        assert a[kind]["first"] > a[kind]["second"], kind      # trial launches on the first step
        assert b[kind]["first"] == b[kind]["second"], kind     # none: the choices came from the file
        assert b[kind]["variants"] == a[kind]["variants"], kind
    with open(cache) as f:
        assert len([ln for ln in f if "=" in ln]) == 2


def test_cache_off_keeps_tuning_in_the_process(tmp_path):
    a = _run("off")
    b = _run("off")
    assert a["single"]["first"] > a["single"]["second"]
    assert b["single"]["first"] > b["single"]["second"]
