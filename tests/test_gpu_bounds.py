"""The bounds-checked build (KK_DEBUG_BOUNDS) on odd shapes: every
staged-window read of the KK and DAS gathers is checked on the device; the
cases of tests/bounds_cases.py run in a child process that loads that build
and must report no violation and the oracle's images."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_checked_build_odd_shapes():
    env = dict(os.environ, KKBEAM_VARIANT="bounds")
    r = subprocess.run([sys.executable, "-m", "tests.bounds_cases"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    res = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert len(res) >= 14
    assert all(v["violations"] == 0 and v["rel_l2"] <= 1e-5 for v in res.values()), res
