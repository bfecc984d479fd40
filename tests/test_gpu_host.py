"""kk_run_host: one call from host memory (upload, decomposition and image
formation, download) against the device calls on the same inputs, bit for
bit, for KK plans (compounded, trimmed records, no intensity), linear-array
DAS and volumetric DAS; and its argument checks."""
import numpy as np
import pytest

import kksynth
import paper_2603_22496_gb300 as kb
from tests import kkcases as kc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2603_22496_gb300 import build
    build.build()
    kb.load()


def _host_run(plan, rf, want_I=True):
    import torch
    h_rf = torch.from_numpy(np.ascontiguousarray(rf)).pin_memory()
    h_B = torch.empty(tuple(plan.empty_image().shape), dtype=torch.float32).pin_memory()
    h_I = torch.empty(tuple(plan.empty_intensity().shape), dtype=torch.float32).pin_memory() if want_I else None
    scratch = torch.empty(plan.scratch_bytes(), dtype=torch.uint8, device="cuda")
    plan.run_host(h_rf, h_B, h_I, scratch)
    torch.cuda.synchronize()
    return h_B, h_I


def _device_kk(plan, rf, want_I=True):
    import torch
    ws, rt, B = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image()
    I = plan.empty_intensity() if want_I else None
    plan.decompose(kc.to_dev(rf), rt, ws)
    plan.beamform(rt, B, I, ws)
    torch.cuda.synchronize()
    return B.cpu(), (I.cpu() if I is not None else None)


@pytest.mark.parametrize("trim", [False, True])
def test_run_host_kk_equals_device_calls(trim):
    import torch
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("hybrid", w.tx_angles, 7, js=[0, 2, 5])
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, kb.KK_COMPOUND_INCOHERENT)
    plan.set_trim(trim)
    hB, hI = _host_run(plan, w.rf)
    dB, dI = _device_kk(plan, w.rf)
    assert torch.equal(hB, dB) and torch.equal(hI, dI)
    assert plan.status() == kb.KK_OK


def test_run_host_kk_without_intensity_int16():
    import torch
    w = kksynth.workload_large()
    from oracle import schemes
    sub = schemes.strided_subset(75, 8)
    ops, (rx, pairs, grp, J) = kc.scheme_both("vernier", w.tx_angles, 16, tx_subset=sub)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J)
    hB, hI = _host_run(plan, w.rf, want_I=False)
    dB, _ = _device_kk(plan, w.rf, want_I=False)
    assert hI is None and torch.equal(hB, dB)


def test_run_host_das_linear_and_volume():
    import torch
    w = kksynth.workload_small()
    plan = kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), das=True)
    hB, hI = _host_run(plan, w.rf)
    ws, B, I = plan.empty_workspace(), plan.empty_image(), plan.empty_intensity()
    plan.das(kc.to_dev(w.rf), B, I, ws)
    torch.cuda.synchronize()
    assert torch.equal(hB, B.cpu()) and torch.equal(hI, I.cpu())
    wv = kksynth.volume_workload(lx=6, ly=5, nx=21, ny=5, nz=17, n_samples=512, speckle=40)
    vplan = kb.Plan(wv.elem_x, wv.tx_ax, wv.grid, wv.c, wv.fs, wv.n_samples, kb.KK_RF_F32, das=True,
                    elem_y=wv.elem_y, tx_angles_y=wv.tx_ay, grid_y=wv.grid_y)
    hB, hI = _host_run(vplan, wv.rf)
    ws, B, I = vplan.empty_workspace(), vplan.empty_image(), vplan.empty_intensity()
    vplan.das(kc.to_dev(wv.rf), B, I, ws)
    torch.cuda.synchronize()
    assert tuple(hB.shape) == (1, 5, 17, 21, 2)
    assert torch.equal(hB, B.cpu()) and torch.equal(hI, I.cpu())


def test_run_host_argument_checks():
    import torch
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 5)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, kb.KK_COMPOUND_COHERENT)
    h_rf = torch.from_numpy(np.ascontiguousarray(w.rf))
    h_B = torch.empty(tuple(plan.empty_image().shape), dtype=torch.float32)
    h_I = torch.empty(tuple(plan.empty_intensity().shape), dtype=torch.float32)
    scratch = torch.empty(plan.scratch_bytes() + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(kb.KKError) as e:              # scratch off its 256-byte alignment
        plan.run_host(h_rf, h_B, h_I, scratch[8:])
    assert e.value.status == kb.KK_ERR_INVALID_ARG
    with pytest.raises(kb.KKError):                   # a null host image
        kb.kk_run_host(plan.handle, h_rf, None, h_I, scratch)
