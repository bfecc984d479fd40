"""Streaming decomposition (include/kkstream.h) on the GPU.

Transmit events are pushed one by one, in acquisition order, from pinned host
memory (or device memory); each full group of events is decomposed on its own
stream and the frame is imaged when it ends.  The result must equal the
whole-frame path (kk_decompose + kk_beamform) bit for bit in the FP32 form, since
Eq. (compression) is separable over transmits and the same kernels run per
group, and it must match the FP64 oracle at the FP32 bound.
"""
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


def _batch(plan, rf_dev):
    import torch
    ws, rt, B = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image()
    I = plan.empty_intensity()
    plan.decompose(rf_dev, rt, ws)
    plan.beamform(rt, B, I, ws)
    torch.cuda.synchronize()
    return B.cpu().numpy(), I.cpu().numpy()


def _stream_frames(st, plan, frames, device_src=False):
    """Push every row of each frame; returns the images of each frame."""
    import torch
    outs = []
    bufs = []
    for rf in frames:
        B, I = plan.empty_image(), plan.empty_intensity()
        for i in range(rf.shape[0]):
            if device_src:
                ev = torch.from_numpy(np.ascontiguousarray(rf[i])).cuda()
                st.push(i, d_event=ev)
            else:
                ev = torch.from_numpy(np.ascontiguousarray(rf[i])).pin_memory()
                st.push(i, h_event=ev)
            bufs.append(ev)                    # keep every source alive until sync
        st.end_frame(B, I)
        outs.append((B, I))
    st.sync()
    torch.cuda.synchronize()
    return [(B.cpu().numpy(), I.cpu().numpy()) for B, I in outs]


def _frames(w, n):
    out = [w.rf]
    for f in range(1, n):
        rng = np.random.default_rng(50 + f)
        out.append((w.rf * np.float32(0.5 + f) + rng.standard_normal(w.rf.shape).astype(np.float32)).astype(w.rf.dtype))
    return out


@pytest.mark.parametrize("group,ring", [(1, 2), (4, 2), (4, None), (11, 2), (3, 9)])
def test_stream_equals_whole_frame_f32(group, ring):
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, compound=kb.KK_COMPOUND_COHERENT)
    st = kb.Stream(plan, group, ring)
    assert st.info.ring_groups == (ring if ring else -(-11 // group) + 1)
    frames = _frames(w, 3)
    got = _stream_frames(st, plan, frames)
    for f, rf in enumerate(frames):
        B, I = _batch(plan, kc.to_dev(rf))
        assert np.array_equal(got[f][0], B), f
        assert np.array_equal(got[f][1], I), f
    info = st.info
    assert info.group == group and info.n_groups == -(-11 // group)
    assert info.events_pushed == 33 and info.events_dropped == 0
    assert info.groups_run == 3 * info.n_groups and info.frames_done == 3
    assert info.copies == 33                   # separate source buffers: one copy per event
    ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
    assert kc.rel_l2(got[0][0][..., 0] + 1j * got[0][0][..., 1], ref) <= 1e-5


def test_stream_drops_unused_transmits_and_uses_device_events():
    """Vernier 8 x 16 on the 75-transmit int16 frame: 67 of 75 events are dropped."""
    w = kksynth.workload_large()
    sub = schemes.strided_subset(75, 8)
    ops, (rx, pairs, grp, J) = kc.scheme_both("vernier", w.tx_angles, 16, tx_subset=sub)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, compound=kb.KK_COMPOUND_COHERENT)
    st = kb.Stream(plan, 3)                   # 8 = 3 + 3 + 2
    got = _stream_frames(st, plan, [w.rf, w.rf], device_src=True)
    B, I = _batch(plan, kc.to_dev(w.rf))
    for g in got:
        assert np.array_equal(g[0], B) and np.array_equal(g[1], I)
    assert st.info.events_dropped == 2 * 67 and st.info.groups_run == 2 * 3


def test_stream_pair_weights():
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("hybrid", w.tx_angles, 7, js=[0, 3, 5])
    wts = np.random.default_rng(3).uniform(0.2, 1.5, pairs.shape[0])
    plan = kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), rx_angles=rx,
                   pairs=pairs, group_of_pair=grp, n_groups=J, compound=kb.KK_COMPOUND_INCOHERENT,
                   pair_weight=wts)
    st = kb.Stream(plan, 5)
    got = _stream_frames(st, plan, [w.rf])
    B, I = _batch(plan, kc.to_dev(w.rf))
    assert np.array_equal(got[0][0], B) and np.array_equal(got[0][1], I)


def test_stream_bf16_full_frame():
    """The 75 x 128 BF16 form in groups of 15 transmits, four frames (both
    rf_theta buffers reused twice), against the whole-frame path."""
    w = kksynth.workload_large()
    rxa = schemes.even_receive_set(np.deg2rad(16.0), 128)
    rx, pairs, grp = kc.product_pairs(np.arange(75), [rxa])
    plan = kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kb.KK_RF_I16, rx_angles=rx,
                   pairs=pairs, group_of_pair=grp, n_groups=1, compound=kb.KK_COMPOUND_COHERENT,
                   precision=kb.KK_PREC_BF16)
    st = kb.Stream(plan, 15)
    frames = [w.rf, w.rf[::-1].copy(), w.rf, w.rf[::-1].copy()]
    got = _stream_frames(st, plan, frames)
    for f, rf in enumerate(frames):
        B, I = _batch(plan, kc.to_dev(rf))
        Bg = got[f][0][..., 0] + 1j * got[f][0][..., 1]
        Bb = B[..., 0] + 1j * B[..., 1]
        assert kc.rel_l2(Bg, Bb) <= 1e-6, f
    assert st.info.groups_run == 4 * 5


def test_stream_rejects_bad_order_and_incomplete_frames():
    import torch
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("vernier", w.tx_angles, 5, tx_subset=np.array([1, 4, 7]))
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, compound=kb.KK_COMPOUND_COHERENT)
    with pytest.raises(kb.KKError):
        kb.Stream(plan, 0)
    with pytest.raises(kb.KKError):
        kb.Stream(plan, 4)                     # only 3 transmits in use
    with pytest.raises(kb.KKError):
        kb.Stream(plan, 2, 1)                  # ring of fewer than two groups
    st = kb.Stream(plan, 2)
    ev = torch.from_numpy(np.ascontiguousarray(w.rf[0])).pin_memory()
    B, I = plan.empty_image(), plan.empty_intensity()
    st.push(0, h_event=ev)                     # unused: dropped
    with pytest.raises(kb.KKError):
        st.push(2, h_event=ev)                 # row 1 is in use and was skipped
    st.push(1, h_event=ev)
    with pytest.raises(kb.KKError):
        st.push(1, h_event=ev)                 # rows must increase
    with pytest.raises(kb.KKError):
        st.end_frame(B, I)                     # 1 of 3 transmits pushed
    st.push(4, h_event=ev)
    with pytest.raises(kb.KKError):
        st.push(5, h_event=None)               # unused rows need no data ...
        st.push(7, h_event=None)               # ... used rows do
    st.push(7, h_event=ev)
    st.push(9, h_event=None)                   # unused row after the frame is complete: dropped
    with pytest.raises(kb.KKError):
        st.end_frame(B, None)                  # compounding plan needs I
    st.end_frame(B, I)
    st.sync()
    assert st.info.frames_done == 1


def test_stream_push_many_coalesces_copies():
    """A frame pushed as blocks of consecutive rows from one pinned buffer:
    one host-to-device copy per group and block, same image as the
    whole-frame path."""
    import torch
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("shifted", w.tx_angles, 9, j=2)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, compound=kb.KK_COMPOUND_COHERENT)
    st = kb.Stream(plan, 4)                    # groups of 4, 4, 3
    h = torch.from_numpy(np.ascontiguousarray(w.rf)).pin_memory()
    B, I = plan.empty_image(), plan.empty_intensity()
    for f in range(2):
        st.push_many(0, h_events=h[0:5])       # block boundaries need not match groups
        st.push_many(5, h_events=h[5:11])
        st.end_frame(B, I)
    st.sync()
    Bb, Ib = _batch(plan, kc.to_dev(w.rf))
    assert np.array_equal(B.cpu().numpy(), Bb) and np.array_equal(I.cpu().numpy(), Ib)
    # groups {0..3}, {4..7}, {8..10}: the second straddles the two blocks
    assert st.info.copies == 2 * 4


def test_stream_after_protects_reused_output_buffers():
    """Pipelined end to end: frames pushed from pinned memory, imaged into two
    alternating device buffers, each downloaded on a caller stream; the image
    formation of frame f waits (kk_stream_after) for frame f - 2's download.
    Every downloaded frame equals the per-frame path."""
    import torch
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, compound=kb.KK_COMPOUND_COHERENT)
    st = kb.Stream(plan, 11)
    frames = _frames(w, 6)
    hs = [torch.from_numpy(np.ascontiguousarray(rf)).pin_memory() for rf in frames]
    dB = [plan.empty_image() for _ in range(2)]
    dI = [plan.empty_intensity() for _ in range(2)]
    hB = [torch.empty(dB[0].shape, dtype=torch.float32).pin_memory() for _ in frames]
    hI = [torch.empty(dI[0].shape, dtype=torch.float32).pin_memory() for _ in frames]
    cs = torch.cuda.Stream()
    for f in range(len(frames)):
        st.after(cs)
        st.push_many(0, h_events=hs[f])
        st.end_frame(dB[f % 2], dI[f % 2])
        st.wait(cs)
        with torch.cuda.stream(cs):
            hB[f].copy_(dB[f % 2], non_blocking=True)
            hI[f].copy_(dI[f % 2], non_blocking=True)
    st.sync()
    cs.synchronize()
    for f, rf in enumerate(frames):
        B, I = _batch(plan, kc.to_dev(rf))
        assert np.array_equal(hB[f].numpy(), B) and np.array_equal(hI[f].numpy(), I), f
