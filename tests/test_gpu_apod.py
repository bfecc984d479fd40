"""Apodization on the GPU against the FP64 oracle: per-pair weights in
Eq. (KK) (per-frame and batched forms), and the receive aperture of DAS
(boxcar and Hann) in both DAS kernels (staged windows and, on a coarse grid,
the synchronous wide-window kernel).  FP32 bound 1e-5 as for the plain path."""
import numpy as np
import pytest

import kksynth
import paper_2603_22496_gb300 as kb
from oracle import kk
from tests import kkcases as kc

pytestmark = pytest.mark.gpu
FS, C = kksynth.FS, kksynth.C_SOUND
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2603_22496_gb300 import build
    build.build()
    kb.load()


def _kk(w, rx, pairs, grp, J, weights, grid, precision=kb.KK_PREC_F32):
    import torch
    plan = kb.Plan(w.elem_x, w.tx_angles, grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), rx_angles=rx,
                   pairs=pairs, group_of_pair=grp, n_groups=J, compound=kb.KK_COMPOUND_COHERENT,
                   precision=precision, pair_weight=weights)
    ws, rt, B, I = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
    plan.decompose(kc.to_dev(w.rf), rt, ws)
    plan.beamform(rt, B, I, ws)
    torch.cuda.synchronize()
    return plan, kc.cplx(B), I.cpu().numpy()


@pytest.mark.parametrize("kind,M,kw", [("confocal", 11, {}), ("hybrid", 7, {"js": [0, 3, 5]})])
def test_pair_weights_match_oracle(kind, M, kw):
    w = kksynth.workload_small()
    grid = (70, 58, -5e-3, 0.11e-3, 6e-3, 0.09e-3)
    ops, (rx, pairs, grp, J) = kc.scheme_both(kind, w.tx_angles, M, **kw)
    wt = np.random.default_rng(3).uniform(0.0, 2.0, len(pairs))
    _, B, I = _kk(w, rx, pairs, grp, J, wt, grid)
    ref = kk.kk_image(w.rf, w.elem_x, ops, grid, FS, C, weights=wt)
    assert kc.rel_l2(B, ref) <= TOL
    assert kc.rel_l2(I, kk.compound(ref, "coherent")) <= 2 * TOL


def test_pair_weights_in_the_tensor_core_form():
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    wt = np.hanning(len(pairs) + 2)[1:-1]
    _, B, _ = _kk(w, rx, pairs, grp, J, wt, w.grid, kb.KK_PREC_BF16)
    ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C, weights=wt)
    assert kc.rel_l2(B, ref) <= 1e-2


def test_pair_weights_in_the_batched_form():
    import torch
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    wt = np.random.default_rng(5).uniform(0.5, 1.5, len(pairs))
    plan, B1, _ = _kk(w, rx, pairs, grp, J, wt, w.grid)
    fr = {"plan": plan, "rf": kc.to_dev(w.rf), "rf_theta": plan.empty_rf_theta(),
          "B": plan.empty_image().zero_(), "I": plan.empty_intensity().zero_(), "workspace": plan.empty_workspace()}
    batch = kb.Batch([fr], shape=408)
    batch.run()
    torch.cuda.synchronize()
    assert kc.rel_l2(kc.cplx(fr["B"]), B1) <= 1e-6


def _edge_clear_f_number(elem_x, grid, candidates):
    """An F-number with no (pixel, element) pair within 1e-4 of the boxcar
    edge (2 F |x - u| / z = 1), so that FP32 and FP64 take the same decision."""
    nx, nz, x0, dx, z0, dz = grid
    x = x0 + dx * np.arange(nx)
    z = z0 + dz * np.arange(nz)
    d = np.abs(x[None, :, None] - elem_x[None, None, :])
    for F in candidates:
        t = 2 * F * d / z[:, None, None]
        if np.min(np.abs(t - 1)) > 1e-4:
            return F
    raise AssertionError("no edge-clear F-number")


def _das(w, grid, f_number, aperture):
    import torch
    plan = kb.Plan(w.elem_x, w.tx_angles, grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), das=True,
                   f_number=f_number, aperture=aperture)
    ws, B = plan.empty_workspace(), plan.empty_image()
    plan.das(kc.to_dev(w.rf), B, None, ws)
    torch.cuda.synchronize()
    return plan, kc.cplx(B)[0]


@pytest.mark.parametrize("window", ["boxcar", "hann"])
def test_das_receive_aperture_matches_oracle(window):
    w = kksynth.workload_small()
    grid = (64, 48, -4.5e-3, 0.13e-3, 6e-3, 0.11e-3)
    F = _edge_clear_f_number(w.elem_x, grid, [1.1, 1.13, 1.17, 1.21])
    ap = kb.KK_APERTURE_BOXCAR if window == "boxcar" else kb.KK_APERTURE_HANN
    plan, B = _das(w, grid, F, ap)
    assert plan.info.is_das
    ref = kk.das_image(w.rf, w.tx_angles, w.elem_x, grid, FS, C, f_number=F, window=window)
    assert kc.rel_l2(B, ref) <= TOL
    full = kk.das_image(w.rf, w.tx_angles, w.elem_x, grid, FS, C)
    assert kc.rel_l2(ref, full) > 0.05          # the aperture changes the image


@pytest.mark.parametrize("F,window", [(0.0, "boxcar"), (1.6, "hann")])
def test_das_wide_window_kernel_matches_oracle(F, window):
    """1 mm pixels make the staged window wider than 256 entries, so the
    synchronous kernel forms the image."""
    w = kksynth.workload_small()
    grid = (16, 12, -7.5e-3, 1.0e-3, 6e-3, 1.0e-3)
    ap = kb.KK_APERTURE_BOXCAR if window == "boxcar" else kb.KK_APERTURE_HANN
    plan, B = _das(w, grid, F, ap)
    ref = kk.das_image(w.rf, w.tx_angles, w.elem_x, grid, FS, C, f_number=F, window=window)
    assert kc.rel_l2(B, ref) <= TOL


def test_bad_apodization_arguments_are_rejected():
    w = kksynth.workload_small()
    with pytest.raises(kb.KKError):
        kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), das=True,
                f_number=1.0, aperture=7)
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    bad = np.ones(len(pairs))
    bad[3] = np.nan
    with pytest.raises(kb.KKError):
        kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), rx_angles=rx,
                pairs=pairs, pair_weight=bad)
