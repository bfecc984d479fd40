"""Failure detection on the GPU without a fault: a bounded device wait is
made to run out (an mbarrier that nothing signals, a 2 ms limit), the status
word reports KK_ERR_TIMEOUT to the host, and the context stays usable: the
next plain KK and DAS frames still match the FP64 oracle."""
import time

import numpy as np
import pytest

import kksynth
import paper_2603_22496_gb300 as kb
from oracle import kk
from tests import kkcases as kc

pytestmark = pytest.mark.gpu

FS, C = kksynth.FS, kksynth.C_SOUND


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2603_22496_gb300 import build
    build.build()
    kb.load()


def test_bounded_wait_runs_out_reports_timeout_and_context_stays_usable():
    import torch
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("vernier", w.tx_angles, 11)
    plan = kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kb.KK_RF_F32, rx_angles=rx,
                   pairs=pairs, group_of_pair=grp, n_groups=J, compound=kb.KK_COMPOUND_COHERENT)
    assert plan.status() == kb.KK_OK
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    kb.kk_plan_check_wait_timeout(plan.handle, 2_000_000)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 >= 2e-3          # the wait ran to its limit
    assert plan.status() == kb.KK_ERR_TIMEOUT
    assert plan.status() == kb.KK_OK                 # read and reset
    # the context is still usable: a normal frame matches the oracle
    ws, rt, B, I = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
    plan.decompose(kc.to_dev(w.rf), rt, ws)
    plan.beamform(rt, B, I, ws)
    torch.cuda.synchronize()
    assert plan.status() == kb.KK_OK
    ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
    assert kc.rel_l2(kc.cplx(B), ref) <= 1e-5
    dplan = kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kb.KK_RF_F32, das=True)
    kb.kk_plan_check_wait_timeout(dplan.handle, 1000)
    torch.cuda.synchronize()
    assert dplan.status() == kb.KK_ERR_TIMEOUT
    dws, dB = dplan.empty_workspace(), dplan.empty_image()
    dplan.das(kc.to_dev(w.rf), dB, None, dws)
    torch.cuda.synchronize()
    assert kc.rel_l2(kc.cplx(dB)[0], kk.das_image(w.rf, w.tx_angles, w.elem_x, w.grid, FS, C)) <= 1e-5
