"""Batched form: frames of uneven size in one CUDA graph with a persistent
image-formation launch, against the per-frame calls and the FP64 oracle."""
import numpy as np
import pytest

import kksynth
import paper_2603_22496_gb300 as kb
from oracle import kk
from tests import kkcases as kc

pytestmark = pytest.mark.gpu

FS, C = kksynth.FS, kksynth.C_SOUND

# (elements, transmits over +-deg, T, grid (nx, nz, dx mm), scheme, M, extra, rf dtype)
FRAMES = [
    (64, 9, 10.0, 1024, (96, 80, 0.12), "confocal", 9, {}, "f32"),
    (48, 12, 12.0, 1536, (130, 70, 0.10), "vernier", 7, {}, "i16"),
    (32, 8, 8.0, 2048, (64, 64, 0.15), "hybrid", 5, {"js": [0, 2, 4]}, "f32"),
    (64, 6, 6.0, 3072, (200, 40, 0.08), "shifted", 5, {"j": 2}, "i16"),
    (96, 10, 9.0, 4096, (33, 140, 0.11), "same", 10, {}, "f32"),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2603_22496_gb300 import build
    build.build()
    kb.load()


def _make(idx, spec):
    L, N, th, T, (nx, nz, dmm), kind, M, kw, dt = spec
    d = dmm * 1e-3
    grid = (nx, nz, -d * (nx - 1) / 2, d, 6e-3, d)
    rng = np.random.default_rng(900 + idx)
    pts = [(0.0, 8.0), (-1.5, 10.0), (1.0, 12.0)]
    ph = kksynth.point_phantom(pts, amp=10.0)
    sx = rng.uniform(grid[2], -grid[2], 300)
    sz = rng.uniform(6e-3, 6e-3 + d * (nz - 1), 300)
    ph = kksynth.Phantom(np.concatenate([ph.x, sx]), np.concatenate([ph.z, sz]),
                         np.concatenate([ph.amp, rng.standard_normal(300)]), n_points=3)
    w = kksynth.workload_custom(f"batch{idx}", 900 + idx, L, 0.3e-3, N, th, T, grid, ph, rf_dtype=dt,
                                snr_db=30.0 if dt == "i16" else None)
    ops, (rx, pairs, grp, J) = kc.scheme_both(kind, w.tx_angles, M, **kw)
    comp = kb.KK_COMPOUND_INCOHERENT if J > 1 else kb.KK_COMPOUND_COHERENT
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, comp)
    return w, ops, plan


@pytest.fixture(scope="module")
def frames():
    return [_make(i, s) for i, s in enumerate(FRAMES)]


def _buffers(w, plan):
    return {"plan": plan, "rf": kc.to_dev(w.rf), "rf_theta": plan.empty_rf_theta(),
            "B": plan.empty_image().zero_(), "I": plan.empty_intensity().zero_(),
            "workspace": plan.empty_workspace()}


@pytest.mark.parametrize("shape", [0, 408, 804, 208])
def test_batch_matches_per_frame_and_oracle(frames, shape):
    import torch
    bufs = [_buffers(w, plan) for (w, ops, plan) in frames]
    batch = kb.Batch(bufs, shape=shape)
    info = batch.info
    assert info.n_frames == len(frames)
    if shape == 0:
        assert info.n_tuned >= 2
        assert info.rows * 100 + info.stage in list(info.tuned_shape)[:info.n_tuned]
    else:
        assert info.rows * 100 + info.stage == shape
    for _ in range(2):                         # the graph can be replayed
        batch.run()
        torch.cuda.synchronize()
    for (w, ops, plan), b in zip(frames, bufs):
        assert plan.status() == kb.KK_OK
        Bb = kc.cplx(b["B"])
        # per-frame path on the same inputs
        ws, rt, B1, I1 = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
        plan.decompose(b["rf"], rt, ws)
        plan.beamform(rt, B1, I1, ws)
        torch.cuda.synchronize()
        assert kc.rel_l2(Bb, kc.cplx(B1)) <= 1e-6
        assert kc.rel_l2(b["I"].cpu().numpy(), I1.cpu().numpy()) <= 2e-6
        ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
        assert kc.rel_l2(Bb, ref) <= 1e-5


def _volume_frame(seed, lx, ly, nx, ny, nz, M, i16):
    """A small matrix-array frame and its volumetric KK plan (M x M receive
    waves over +-10 deg, coherent)."""
    from oracle import volume as V
    w = kksynth.volume_workload(seed=seed, lx=lx, ly=ly, nx=nx, ny=ny, nz=nz, n_samples=1024, speckle=150,
                                rf_dtype="i16" if i16 else "f32", snr_db=30.0 if i16 else None)
    rx1 = np.deg2rad(np.linspace(-10.0, 10.0, M))
    ps = V.product_set(w.tx_ax, w.tx_ay, [(np.tile(rx1, M), np.repeat(rx1, M))])
    pairs = np.stack([ps.tx_index, ps.rx_index], 1).astype(np.int32)
    plan = kb.Plan(w.elem_x, w.tx_ax, w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), rx_angles=ps.rx_ax,
                   pairs=pairs, group_of_pair=ps.group.astype(np.int32), n_groups=ps.n_groups,
                   compound=kb.KK_COMPOUND_COHERENT, elem_y=w.elem_y, tx_angles_y=w.tx_ay, rx_angles_y=ps.rx_ay,
                   grid_y=w.grid_y)
    return w, ps, plan


@pytest.mark.parametrize("shape", [0, 408])
def test_batch_with_volumes_matches_per_frame_and_oracle(frames, shape):
    """Two linear-array frames and two volumes (8 x 8 and 6 x 5 arrays, ragged
    voxel grids, one int16) in one batch: the volumes form the second list,
    with its own persistent launch; every frame equals its per-frame path and
    the oracle."""
    import torch
    from oracle import volume as V
    vols = [_volume_frame(3300, 8, 8, 40, 9, 52, 5, False), _volume_frame(3301, 6, 5, 37, 7, 45, 3, True)]
    bufs = [_buffers(w, plan) for (w, ops, plan) in frames[:2]] + [_buffers(w, plan) for (w, ps, plan) in vols]
    batch = kb.Batch(bufs, shape=shape)
    info = batch.info
    assert info.n_frames == 4 and info.n_volume_frames == 2
    assert info.n_items > 0 and info.n_items_volume > 0
    if shape:
        assert info.rows_volume * 100 + info.stage_volume == shape
    assert info.pixel_pairs == sum(float(b["plan"].info.n_pairs) * b["plan"].info.nx * b["plan"].info.nz
                                   * b["plan"].info.ny for b in bufs)
    for _ in range(2):
        batch.run()
        torch.cuda.synchronize()
    for b in bufs:
        plan = b["plan"]
        assert plan.status() == kb.KK_OK
        ws, rt, B1, I1 = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
        plan.decompose(b["rf"], rt, ws)
        plan.beamform(rt, B1, I1, ws)
        torch.cuda.synchronize()
        assert kc.rel_l2(kc.cplx(b["B"]), kc.cplx(B1)) <= 1e-6
        assert kc.rel_l2(b["I"].cpu().numpy(), I1.cpu().numpy()) <= 2e-6
    for (w, ps, plan), b in zip(vols, bufs[2:]):
        ref = V.kk_volume(w.rf, w.elem_x, w.elem_y, ps, w.grid, w.grid_y, FS, C)
        assert kc.rel_l2(kc.cplx(b["B"]), ref) <= 1e-5


def test_batch_mixed_precision_forms(frames):
    """Frames in the BF16, FP16 and FP8 tensor-core forms beside an FP32 one
    in one graph (the persistent contraction of each form captured as a
    node): every frame equals its per-frame path, and the oracle within the
    forms' stated bound."""
    import torch
    forms = [kb.KK_PREC_BF16, kb.KK_PREC_F16, kb.KK_PREC_F8E4M3, kb.KK_PREC_F32]
    made = []
    for (w, ops, plan0), prec in zip(frames[:4], forms):
        i0 = plan0.info
        plan = kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w),
                       rx_angles=ops.rx_angles, pairs=np.stack([ops.tx_index, ops.rx_index], 1).astype(np.int32),
                       group_of_pair=ops.group.astype(np.int32), n_groups=i0.n_groups,
                       compound=kb.KK_COMPOUND_INCOHERENT if i0.n_groups > 1 else kb.KK_COMPOUND_COHERENT,
                       precision=prec)
        made.append((w, ops, plan, prec))
    bufs = [_buffers(w, plan) for (w, ops, plan, prec) in made]
    batch = kb.Batch(bufs, shape=0)
    batch.run()
    torch.cuda.synchronize()
    for (w, ops, plan, prec), b in zip(made, bufs):
        assert plan.status() == kb.KK_OK
        plan.set_gather(batch.info.rows, batch.info.stage)
        ws, rt, B1, I1 = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
        plan.decompose(b["rf"], rt, ws)
        plan.beamform(rt, B1, I1, ws)
        torch.cuda.synchronize()
        assert kc.rel_l2(kc.cplx(b["B"]), kc.cplx(B1)) <= 1e-6
        ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
        assert kc.rel_l2(kc.cplx(b["B"]), ref) <= (1e-5 if prec == kb.KK_PREC_F32 else 1e-2)


def test_batch_rejects_bad_frames(frames):
    w, ops, plan = frames[0]
    b = _buffers(w, plan)
    b["I"] = None                              # the plan compounds: I is required
    with pytest.raises(kb.KKError):
        kb.Batch([b], shape=408)
    b = _buffers(w, plan)
    with pytest.raises(kb.KKError):
        kb.Batch([b], shape=412)


def test_gpu_simulator_matches_cpu_forward_model():
    """The GPU input generator reproduces the CPU forward model (FP32 with
    fast intrinsics: rel-L2 below 1e-3)."""
    import torch
    w = kksynth.workload_small(speckle=400)
    sc = torch.tensor(np.stack([w.phantom.x, w.phantom.z, w.phantom.amp], 1), dtype=torch.float32).cuda()
    rf = kb.kk_simulate_rf(w.tx_angles, w.elem_x, w.n_samples, sc, w.fs, w.c)
    torch.cuda.synchronize()
    ref = kksynth.simulate_rf(w.phantom, w.elem_x, w.tx_angles, w.n_samples)
    assert kc.rel_l2(rf.cpu().numpy(), ref) <= 1e-3
    noisy = kb.kk_simulate_rf(w.tx_angles, w.elem_x, w.n_samples, sc, w.fs, w.c, noise_sigma=0.5, seed=7)
    d = (noisy - rf).cpu().numpy()
    assert abs(d.std() - 0.5) < 0.01 and abs(d.mean()) < 0.01


def test_batch_full_256_uneven_frames_match_per_frame():
    """The benchmark's batched workload at full size (256 frames of 64-256
    elements, 1024-4096 samples, 8-75 transmits, 32-512 pairs, 256^2-1024^2
    grids, autotuned launch shape): every frame of the graph equals the
    per-frame path.  Its inputs come from the GPU simulator, so the oracle
    checks the per-frame path on CPU-simulated inputs in the tests above
    instead."""
    import os
    import sys
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    frames = bench._batch_frames(kb, 256)
    batch = kb.Batch(frames, shape=0)
    batch.run()
    torch.cuda.synchronize()
    assert batch.info.n_frames == 256
    worst = 0.0
    for f in frames:
        plan = f["plan"]
        assert plan.status() == kb.KK_OK
        # the per-frame path at the batch's launch shape, so that both sum each
        # stage's pairs in the same order (the stage size sets the two-level sum)
        plan.set_gather(batch.info.rows, batch.info.stage)
        ws, rt, B1, I1 = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
        plan.decompose(f["rf"], rt, ws)
        plan.beamform(rt, B1, I1, ws)
        torch.cuda.synchronize()
        worst = max(worst, kc.rel_l2(kc.cplx(f["B"]), kc.cplx(B1)))
        del ws, rt, B1, I1
    assert worst <= 1e-6, worst
