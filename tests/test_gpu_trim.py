"""Records trimmed to the grid's reach (kk_plan_set_trim): the inverse stores
of each record y_p only the samples Eq. (KK)'s interpolation can read for
some pixel of the grid under any launch shape.  Records are pre-filled with
NaN, so a read of a sample the inverse left unwritten would show in the
image: images must equal the full-record path's bit for bit, at every launch
shape, through the streaming, batched and no-allocation paths too, and the
written samples must equal the full records'."""
import numpy as np
import pytest

import kksynth
import paper_2603_22496_gb300 as kb
from oracle import kk, schemes
from tests import kkcases as kc

pytestmark = pytest.mark.gpu

FS, C = kksynth.FS, kksynth.C_SOUND


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2603_22496_gb300 import build
    build.build()
    kb.load()


def _run(plan, d_rf, trim):
    import torch
    plan.set_trim(trim)
    assert plan.info.records_trimmed == int(trim)
    ws, rt, B, I = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
    rt.fill_(float("nan"))
    plan.decompose(d_rf, rt, ws)
    plan.beamform(rt, B, I, ws)
    torch.cuda.synchronize()
    return rt, B, I


def _both(plan, rf):
    """(written fraction, images full, images trimmed), after checking that
    the written samples of the trimmed records equal the full ones and form
    one range per record."""
    import torch
    d_rf = kc.to_dev(rf)
    rf_full, Bf, If = _run(plan, d_rf, False)
    rf_trim, Bt, It = _run(plan, d_rf, True)
    assert not bool(torch.isnan(rf_full).any())
    written = ~torch.isnan(rf_trim).any(dim=-1)
    assert bool((torch.isnan(rf_trim).any(dim=-1) == torch.isnan(rf_trim).all(dim=-1)).all())
    assert torch.equal(rf_trim[written], rf_full[written])
    w = written.cpu().numpy()
    for r in range(w.shape[0]):
        idx = np.flatnonzero(w[r])
        if idx.size:
            assert idx[-1] - idx[0] + 1 == idx.size, r
    return float(w.mean()), (Bf, If), (Bt, It)


def _same(a, b):
    import torch
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.mark.parametrize("kind,M,kw", [("confocal", 11, {}), ("shifted", 11, {"j": 5}),
                                       ("hybrid", 7, {"js": [0, 2, 5]})])
def test_trimmed_records_give_the_same_images(kind, M, kw):
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both(kind, w.tx_angles, M, **kw)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, kb.KK_COMPOUND_COHERENT)
    frac, full, trim = _both(plan, w.rf)
    _same(full, trim)
    assert 0.0 < frac <= 1.0
    ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
    assert kc.rel_l2(kc.cplx(trim[0]), ref) <= 1e-5


@pytest.mark.parametrize("nx,nz", [(1, 1), (33, 7), (97, 31)])
def test_trimmed_records_ragged_grids(nx, nz):
    w = kksynth.workload_small()
    grid = (nx, nz, -6e-3, 0.11e-3, 6e-3, 0.13e-3)
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 9)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, kb.KK_COMPOUND_COHERENT, grid)
    frac, full, trim = _both(plan, w.rf)
    _same(full, trim)
    assert frac < 0.5            # a small grid reads a short part of each record


@pytest.mark.parametrize("dx", [0.075e-3, 0.3e-3])
def test_trimmed_records_at_the_record_edges(dx):
    """Windows that start before sample 0 and run past T - 1."""
    w = kksynth.workload_small()
    nx = int(round(20e-3 / dx)) | 1
    grid = (nx, 160, -10e-3, dx, 0.5e-3, 0.15e-3)
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 13)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, kb.KK_COMPOUND_COHERENT, grid)
    frac, full, trim = _both(plan, w.rf)
    _same(full, trim)


def test_trimmed_records_pair_subset_without_column_identity():
    """A scattered pair subset with a repeated pair: the inverse without bulk
    copies of Y (rows read through a column table)."""
    grid = (50, 44, -4e-3, 0.12e-3, 5e-3, 0.14e-3)
    ph = kksynth.point_phantom([(0.5, 6.0), (-1.0, 8.0), (2.0, 9.5)])
    w = kksynth.workload_custom("odd", 77, 37, 0.25e-3, 9, 12.0, 1024, grid, ph, rf_dtype="i16")
    rx = np.deg2rad(np.array([-9.0, -2.5, 0.0, 3.0, 11.0]))
    pairs = np.array([[0, 1], [3, 4], [8, 0], [4, 2], [4, 2], [7, 3], [2, 2], [5, 0]], dtype=np.int32)
    grp = np.array([0, 1, 0, 1, 0, 1, 1, 0], dtype=np.int32)
    plan = kc.kk_plan_for(w, rx, pairs, grp, 2, kb.KK_COMPOUND_INCOHERENT)
    frac, full, trim = _both(plan, w.rf)
    _same(full, trim)


@pytest.mark.parametrize("rows,stage", [(2, 4), (2, 16), (4, 4), (4, 8), (8, 4), (8, 8)])
def test_trimmed_records_every_launch_shape(rows, stage):
    """The trimmed range covers every launch shape: records decomposed at the
    default shape image identically at each other shape."""
    import torch
    w = kksynth.workload_small()
    grid = (70, 58, -5e-3, 0.11e-3, 6e-3, 0.09e-3)
    ops, (rx, pairs, grp, J) = kc.scheme_both("hybrid", w.tx_angles, 7, js=[0, 3, 5])
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, kb.KK_COMPOUND_COHERENT, grid)
    d_rf = kc.to_dev(w.rf)
    rf_full, _, _ = _run(plan, d_rf, False)
    rf_trim, _, _ = _run(plan, d_rf, True)
    plan.set_gather(rows, stage)
    ws = plan.empty_workspace()
    out = []
    for rt in (rf_full, rf_trim):
        B, I = plan.empty_image(), plan.empty_intensity()
        plan.beamform(rt, B, I, ws)
        torch.cuda.synchronize()
        out.append((B, I))
    _same(out[0], out[1])


def test_trimmed_records_large_frame():
    """The 9600-pair frame: about half of each record is stored, the image is
    the full-record one bit for bit, also through the no-allocation call."""
    import torch
    w = kksynth.workload_large()
    rxa = schemes.even_receive_set(np.deg2rad(16.0), 128)
    rx, pairs, grp = kc.product_pairs(np.arange(75), [rxa])
    plan = kc.kk_plan_for(w, rx, pairs, grp, 1, kb.KK_COMPOUND_COHERENT)
    d_rf = kc.to_dev(w.rf)
    rf_full, Bf, If = _run(plan, d_rf, False)
    rf_trim, Bt, It = _run(plan, d_rf, True)
    _same((Bf, If), (Bt, It))
    frac = float((~torch.isnan(rf_trim).any(dim=-1)).float().mean())
    assert 0.3 < frac < 0.8, frac
    B, I = plan.empty_image(), plan.empty_intensity()
    kb.kk_beamform_noalloc(plan.handle, rf_trim, B, I)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(B).all()) and kc.rel_l2(kc.cplx(B), kc.cplx(Bf)) <= 1e-6


def test_trimmed_records_stream_and_batch():
    """The streaming decomposition and the batched form of a trimming plan
    give the full-record images (the stream bit for bit; the batch, whose
    gather sums in one slice, to FP32 order)."""
    import torch
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, compound=kb.KK_COMPOUND_COHERENT)
    _, Bf, If = _run(plan, kc.to_dev(w.rf), False)
    plan.set_trim(True)
    st = kb.Stream(plan, 4)
    B, I = plan.empty_image(), plan.empty_intensity()
    keep = []
    for i in range(w.rf.shape[0]):
        ev = torch.from_numpy(np.ascontiguousarray(w.rf[i])).pin_memory()
        st.push(i, h_event=ev)
        keep.append(ev)
    st.end_frame(B, I)
    st.sync()
    torch.cuda.synchronize()
    assert torch.equal(B, Bf) and torch.equal(I, If)
    rt = plan.empty_rf_theta().fill_(float("nan"))
    fr = {"plan": plan, "rf": kc.to_dev(w.rf), "rf_theta": rt, "B": plan.empty_image(),
          "I": plan.empty_intensity(), "workspace": plan.empty_workspace()}
    batch = kb.Batch([fr], shape=0)
    batch.run()
    torch.cuda.synchronize()
    assert bool(torch.isfinite(fr["B"]).all()) and kc.rel_l2(kc.cplx(fr["B"]), kc.cplx(Bf)) <= 1e-6


def test_trim_refusals():
    w = kksynth.workload_small()
    das = kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), das=True)
    with pytest.raises(kb.KKError):
        das.set_trim(True)
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 5)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J)
    with pytest.raises(kb.KKError):
        kb.kk_plan_set_trim(plan.handle, 2)
    from oracle import volume as V
    wv = kksynth.volume_workload(speckle=20, nx=9, ny=3, nz=11, lx=4, ly=3, n_samples=256)
    rx1 = schemes.even_receive_set(np.deg2rad(8.0), 3)
    ps = V.product_set(wv.tx_ax, wv.tx_ay, [(np.tile(rx1, 3), np.repeat(rx1, 3))])
    pv = np.stack([ps.tx_index, ps.rx_index], 1).astype(np.int32)
    vplan = kb.Plan(wv.elem_x, wv.tx_ax, wv.grid, wv.c, wv.fs, wv.n_samples, kb.KK_RF_F32, rx_angles=ps.rx_ax,
                    pairs=pv, group_of_pair=ps.group.astype(np.int32), n_groups=ps.n_groups,
                    elem_y=wv.elem_y, tx_angles_y=wv.tx_ay, rx_angles_y=ps.rx_ay, grid_y=wv.grid_y)
    with pytest.raises(kb.KKError) as e:
        vplan.set_trim(True)
    assert e.value.status == kb.KK_ERR_UNSUPPORTED
