"""NVTX ranges: the library names the stages each call enqueues
(kk_decompose and its spectrum / contraction / inverse, kk_beamform,
das_beamform and its two stages).  A child process loads a small NVTX
injection library (tests/nvtx_probe.c) that logs every push and pop; the
ranges must appear by name, in order, and balance."""
import os
import shutil
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1])
import torch
import kksynth
import paper_2603_22496_gb300 as kb
from tests import kkcases as kc
kb.load()
w = kksynth.workload_small()
ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 5)
plan = kc.kk_plan_for(w, rx, pairs, grp, J, kb.KK_COMPOUND_COHERENT)
ws, rt, B, I = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
d_rf = kc.to_dev(w.rf)
plan.decompose(d_rf, rt, ws)
plan.beamform(rt, B, I, ws)
dplan = kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), das=True)
dplan.das(d_rf, dplan.empty_image(), None, dplan.empty_workspace())
torch.cuda.synchronize()
print("child done")
"""


def test_nvtx_ranges_name_the_stages(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2603_22496_gb300 import build
    build.build()
    probe = tmp_path / "libnvtx_probe.so"
    subprocess.run([gcc, "-shared", "-fPIC", "-O1", "-o", str(probe), os.path.join(ROOT, "tests", "nvtx_probe.c")],
                   check=True)
    log = tmp_path / "nvtx.log"
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(probe), KK_NVTX_LOG=str(log))
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "child done" in r.stdout, (r.stdout[-2000:], r.stderr[-2000:])
    lines = log.read_text().splitlines()
    pushes = [ln[5:] for ln in lines if ln.startswith("push ")]
    ours = [p for p in pushes if p.startswith(("kk_", "das_"))]
    assert ours == ["kk_decompose", "kk_decompose/spectrum", "kk_decompose/contraction", "kk_decompose/inverse",
                    "kk_beamform", "das_beamform", "das_beamform/analytic", "das_beamform/gather"], ours
    # every push has its pop, and the depth never goes negative
    depth = 0
    for ln in lines:
        depth += 1 if ln.startswith("push ") else -1
        assert depth >= 0
    assert depth == 0
