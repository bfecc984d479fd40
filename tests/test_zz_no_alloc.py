"""kk_beamform_noalloc: KK image formation without any device allocation or
workspace, for callers that cannot call cudaMalloc (a host framework that
owns all device memory, a plugin inside one, a loop that must not allocate).

The entry point must give the same images as kk_beamform with a workspace,
call after call (its fixed scratch keeps the previous call's contents), and
refuse plans whose partial images exceed its fixed 8 MiB scratch.  This file
is collected last so that a stop-at-first-failure run has already run every
other test; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

import kksynth
import paper_2603_22496_gb300 as kb

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2603_22496_gb300 import build
    build.build()
    kb.load()


def _plan(w, compound, M=7, js=(0, 2, 5)):
    dth = (w.tx_angles.max() - w.tx_angles.min()) / (w.n_tx - 1)
    groups = [kb.kk_scheme_angles(kb.KK_SCHEME_SHIFTED, w.n_tx, dth, M, j) for j in js]
    rx = np.concatenate(groups)
    pairs, grp = [], []
    for g in range(len(groups)):
        for i in range(w.n_tx):
            for o in range(M):
                pairs.append((i, g * M + o))
                grp.append(g)
    return kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples,
                   kb.KK_RF_F32 if w.rf.dtype == np.float32 else kb.KK_RF_I16,
                   rx_angles=rx, pairs=np.array(pairs, np.int32), group_of_pair=np.array(grp, np.int32),
                   n_groups=len(groups), compound=compound)


def _rel(a, b):
    a = a.double().cpu().numpy().ravel()
    b = b.double().cpu().numpy().ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("compound", [kb.KK_COMPOUND_COHERENT, kb.KK_COMPOUND_INCOHERENT])
def test_noalloc_matches_workspace_path_twice_in_a_row(compound):
    import torch
    w = kksynth.workload_small()
    plan = _plan(w, compound)
    assert plan.info.launches_beamform == 2          # several pair slices: the scratch is used
    d_rf = torch.from_numpy(w.rf).cuda()
    ws, rt = plan.empty_workspace(), plan.empty_rf_theta()
    plan.decompose(d_rf, rt, ws)
    B_ref, I_ref = plan.empty_image(), plan.empty_intensity()
    kb.kk_beamform(plan.handle, rt, B_ref, I_ref, ws)
    for _ in range(2):
        B, I = plan.empty_image().fill_(float("nan")), plan.empty_intensity().fill_(float("nan"))
        kb.kk_beamform_noalloc(plan.handle, rt, B, I)
        torch.cuda.synchronize()
        assert _rel(B, B_ref) <= TOL
        assert _rel(I, I_ref) <= TOL


def test_noalloc_large_frame_and_back_to_back_plans():
    """The 9600-pair 512x512 frame (two slices, 4 MiB of partial images) and a
    second plan right after it: the shared scratch is fully rewritten."""
    import torch
    w = kksynth.workload_large()
    rx = np.deg2rad(np.linspace(-16, 16, 128))
    pairs = np.array([(i, o) for i in range(75) for o in range(128)], np.int32)
    plan = kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kb.KK_RF_I16,
                   rx_angles=rx, pairs=pairs, compound=kb.KK_COMPOUND_COHERENT)
    d_rf = torch.from_numpy(w.rf).cuda()
    ws, rt = plan.empty_workspace(), plan.empty_rf_theta()
    plan.decompose(d_rf, rt, ws)
    B_ref, I_ref = plan.empty_image(), plan.empty_intensity()
    kb.kk_beamform(plan.handle, rt, B_ref, I_ref, ws)
    B, I = plan.empty_image(), plan.empty_intensity()
    kb.kk_beamform_noalloc(plan.handle, rt, B, I)
    torch.cuda.synchronize()
    assert _rel(B, B_ref) <= TOL and _rel(I, I_ref) <= TOL
    # a different plan reuses the same scratch
    ws_small = kksynth.workload_small()
    p2 = _plan(ws_small, kb.KK_COMPOUND_INCOHERENT)
    rt2 = p2.empty_rf_theta()
    p2.decompose(torch.from_numpy(ws_small.rf).cuda(), rt2, p2.empty_workspace())
    B2r, I2r = p2.empty_image(), p2.empty_intensity()
    kb.kk_beamform(p2.handle, rt2, B2r, I2r, p2.empty_workspace())
    B2, I2 = p2.empty_image(), p2.empty_intensity()
    kb.kk_beamform_noalloc(p2.handle, rt2, B2, I2)
    torch.cuda.synchronize()
    assert _rel(B2, B2r) <= TOL and _rel(I2, I2r) <= TOL


def test_noalloc_rejects_plans_beyond_its_scratch():
    """Six groups on a 320x320 grid split over pair slices need at least
    2 x 6 x 320 x 320 x 8 bytes = 9.8 MB of partial images, more than the
    fixed 8 MiB: a clear error, nothing launched."""
    import torch
    w = kksynth.workload_small()
    grid = (320, 320, -9.5e-3, 19e-3 / 319, 5e-3, 19e-3 / 319)
    M, js = 15, (0, 1, 2, 3, 4, 5)
    dth = (w.tx_angles.max() - w.tx_angles.min()) / (w.n_tx - 1)
    rx = np.concatenate([kb.kk_scheme_angles(kb.KK_SCHEME_SHIFTED, w.n_tx, dth, M, j) for j in js])
    pairs = np.array([(i, g * M + o) for g in range(len(js)) for i in range(w.n_tx) for o in range(M)],
                     np.int32)
    grp = np.repeat(np.arange(len(js), dtype=np.int32), w.n_tx * M)
    plan = kb.Plan(w.elem_x, w.tx_angles, grid, w.c, w.fs, w.n_samples, kb.KK_RF_F32, rx_angles=rx,
                   pairs=pairs, group_of_pair=grp, n_groups=len(js), compound=kb.KK_COMPOUND_INCOHERENT)
    assert plan.info.launches_beamform == 2
    rt = torch.zeros((plan.info.n_pairs, w.n_samples, 2), device="cuda")
    B, I = plan.empty_image(), plan.empty_intensity()
    with pytest.raises(kb.KKError) as e:
        kb.kk_beamform_noalloc(plan.handle, rt, B, I)
    assert e.value.status == kb.KK_ERR_INVALID_ARG
    assert "scratch" in str(e.value)


def test_noalloc_volumetric_plan_with_pair_slices():
    """A 4-slice volume on a 32 x 32 x-z grid: few tiles, so the pair list is
    split and the scratch holds pair slices x groups x nx x nz x ny partial
    voxels (the y-slice factor of the size rule)."""
    import torch
    from oracle import schemes, volume as V
    w = kksynth.volume_workload(nx=32, ny=4, nz=32, speckle=200)
    rx1 = schemes.even_receive_set(np.deg2rad(12.0), 7)
    ps = V.product_set(w.tx_ax, w.tx_ay, [(np.tile(rx1, 7), np.repeat(rx1, 7))])
    pairs = np.stack([ps.tx_index, ps.rx_index], 1).astype(np.int32)
    plan = kb.Plan(w.elem_x, w.tx_ax, w.grid, w.c, w.fs, w.n_samples, kb.KK_RF_F32, rx_angles=ps.rx_ax,
                   pairs=pairs, group_of_pair=ps.group.astype(np.int32), n_groups=ps.n_groups,
                   compound=kb.KK_COMPOUND_COHERENT, elem_y=w.elem_y, tx_angles_y=w.tx_ay,
                   rx_angles_y=ps.rx_ay, grid_y=w.grid_y)
    assert plan.info.is_volume == 1 and plan.info.ny == 4
    assert plan.info.launches_beamform == 2          # pair slices: the scratch is used
    d_rf = torch.from_numpy(w.rf).cuda()
    ws, rt = plan.empty_workspace(), plan.empty_rf_theta()
    plan.decompose(d_rf, rt, ws)
    B_ref, I_ref = plan.empty_image(), plan.empty_intensity()
    kb.kk_beamform(plan.handle, rt, B_ref, I_ref, ws)
    for _ in range(2):
        B, I = plan.empty_image().fill_(float("nan")), plan.empty_intensity().fill_(float("nan"))
        kb.kk_beamform_noalloc(plan.handle, rt, B, I)
        torch.cuda.synchronize()
        assert _rel(B, B_ref) <= TOL and _rel(I, I_ref) <= TOL


def test_noalloc_single_slice_without_intensity():
    """Three transmits x 7 receive angles: too few pairs to split, so the
    scratch is never looked up; no compounding and no intensity buffer."""
    import torch
    w = kksynth.workload_small()
    sub = [3, 5, 7]
    dth = float(w.tx_angles[5] - w.tx_angles[3]) / 2
    rx = kb.kk_scheme_angles(kb.KK_SCHEME_VERNIER, 3, dth, 7)
    pairs = np.array([(i, o) for i in sub for o in range(7)], np.int32)
    plan = kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kb.KK_RF_F32, rx_angles=rx,
                   pairs=pairs, compound=kb.KK_COMPOUND_NONE)
    assert plan.info.launches_beamform == 1
    d_rf = torch.from_numpy(w.rf).cuda()
    ws, rt = plan.empty_workspace(), plan.empty_rf_theta()
    plan.decompose(d_rf, rt, ws)
    B_ref = plan.empty_image()
    kb.kk_beamform(plan.handle, rt, B_ref, None, ws)
    for _ in range(2):
        B = plan.empty_image().fill_(float("nan"))
        kb.kk_beamform_noalloc(plan.handle, rt, B, None)
        torch.cuda.synchronize()
        assert _rel(B, B_ref) <= TOL
