"""Odd-shape cases run on the bounds-checked build of the library (run as
``KKBEAM_VARIANT=bounds python -m tests.bounds_cases``; the GPU test
``test_gpu_bounds`` does that in a child process).

Every staged-window read of the KK gathers (the per-frame, volumetric and
batched forms) and of both DAS gathers is checked on
the device; each case must leave the violation counter at zero and match
the FP64 oracle.  Prints one JSON line."""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main() -> int:
    import torch

    import kksynth
    import paper_2603_22496_gb300 as kb
    from oracle import kk, schemes
    from oracle import volume as V
    from tests import kkcases as kc

    assert os.environ.get("KKBEAM_VARIANT") == "bounds", "run with KKBEAM_VARIANT=bounds"
    from paper_2603_22496_gb300 import build
    build.build(variant="bounds")
    kb.load()
    fs, c = kksynth.FS, kksynth.C_SOUND
    res = {}
    assert kb.kk_debug_bounds() == 0

    def check(name, got, ref, tol=1e-5):
        v = kb.kk_debug_bounds()
        e = kc.rel_l2(got, ref)
        res[name] = {"violations": v, "rel_l2": e}
        assert v == 0 and e <= tol, (name, v, e)

    # three elements, two transmits, T = 256, 7 x 5 grids: a coarse one (0.2 x
    # 0.25 mm pixels, long windows) and a fine one (0.05 mm), at every launch
    # shape whose window fits
    fine = (7, 5, -0.15e-3, 0.05e-3, 3e-3, 0.05e-3)
    grid = (7, 5, -0.6e-3, 0.2e-3, 3e-3, 0.25e-3)
    w = kksynth.workload_custom("odd3", 5, 3, 0.3e-3, 2, 6.0, 256, grid,
                                kksynth.point_phantom([(0.0, 3.5)]), snr_db=30.0)
    rx = np.deg2rad(np.array([-5.0, 1.0, 7.0]))
    pairs = np.array([(i, o) for i in range(2) for o in range(3)], np.int32)
    ops = schemes.PairSet(w.tx_angles, rx, pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64),
                          np.zeros(6, np.int64), 1)
    for gname, g, shapes in (("coarse", grid, [(4, 8), (4, 4), (2, 8), (2, 4)]),
                             ("fine", fine, [(8, 16), (8, 8), (4, 16), (2, 4)])):
        ref = kk.kk_image(w.rf, w.elem_x, ops, g, fs, c)
        for rows, stage in shapes:
            plan = kc.kk_plan_for(w, rx, pairs, np.zeros(6, np.int32), 1, kb.KK_COMPOUND_COHERENT, g)
            plan.set_gather(rows, stage)
            ws, rt, B, I = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
            plan.decompose(kc.to_dev(w.rf), rt, ws)
            plan.beamform(rt, B, I, ws)
            torch.cuda.synchronize()
            check(f"kk_L3_T256_7x5_{gname}_r{rows}_s{stage}", kc.cplx(B), ref)
    D, _, _ = kc.run_das(w, grid=grid)
    check("das_L3_T256_7x5", D, kk.das_image(w.rf, w.tx_angles, w.elem_x, grid, fs, c))

    # windows before the record start and past its end; a coarse x pitch
    ws_ = kksynth.workload_small()
    for dx in (0.075e-3, 0.3e-3):
        g2 = (int(round(20e-3 / dx)) | 1, 160, -10e-3, dx, 0.5e-3, 0.15e-3)
        ops2, (rx2, p2, gr2, J2) = kc.scheme_both("confocal", ws_.tx_angles, 13)
        B2, _, _, plan2 = kc.run_kk(ws_, rx2, p2, gr2, J2, grid=g2)
        check(f"kk_record_edges_dx{dx * 1e3:.3f}mm", B2, kk.kk_image(ws_.rf, ws_.elem_x, ops2, g2, fs, c))
        D2, _, _ = kc.run_das(ws_, grid=g2)
        check(f"das_dx{dx * 1e3:.3f}mm", D2, kk.das_image(ws_.rf, ws_.tx_angles, ws_.elem_x, g2, fs, c))

    # a coarse grid: the plain DAS kernel (windows wider than the staged one)
    g3 = (21, 17, -6e-3, 0.6e-3, 4e-3, 0.6e-3)
    D3, _, _ = kc.run_das(ws_, grid=g3)
    check("das_coarse_0.6mm", D3, kk.das_image(ws_.rf, ws_.tx_angles, ws_.elem_x, g3, fs, c))

    # volumetric gather: a 4 x 3 array, three y slices
    wv = kksynth.volume_workload(lx=4, ly=3, nx=9, ny=3, nz=11, n_samples=256, speckle=30)
    rx1 = schemes.even_receive_set(np.deg2rad(8.0), 3)
    ps = V.product_set(wv.tx_ax, wv.tx_ay, [(np.tile(rx1, 3), np.repeat(rx1, 3))])
    pv = np.stack([ps.tx_index, ps.rx_index], 1).astype(np.int32)
    plan = kb.Plan(wv.elem_x, wv.tx_ax, wv.grid, wv.c, wv.fs, wv.n_samples, kb.KK_RF_F32, rx_angles=ps.rx_ax,
                   pairs=pv, group_of_pair=ps.group.astype(np.int32), n_groups=ps.n_groups,
                   compound=kb.KK_COMPOUND_COHERENT, elem_y=wv.elem_y, tx_angles_y=wv.tx_ay,
                   rx_angles_y=ps.rx_ay, grid_y=wv.grid_y)
    ws3, rt3, B3, I3 = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
    plan.decompose(kc.to_dev(wv.rf), rt3, ws3)
    plan.beamform(rt3, B3, I3, ws3)
    torch.cuda.synchronize()
    y3 = V.decompose3(wv.rf, wv.elem_x, wv.elem_y, ps, fs, c)
    check("kk_volume_4x3_9x3x11", kc.cplx(B3),
          V.kk_beamform3(y3, wv.elem_x, wv.elem_y, ps, wv.grid, wv.grid_y, fs, c))

    # volumetric DAS on the same volume (slice terms in the staged DAS gather)
    dp = kb.Plan(wv.elem_x, wv.tx_ax, wv.grid, wv.c, wv.fs, wv.n_samples, kb.KK_RF_F32, das=True,
                 elem_y=wv.elem_y, tx_angles_y=wv.tx_ay, grid_y=wv.grid_y)
    dws, dB = dp.empty_workspace(), dp.empty_image()
    dp.das(kc.to_dev(wv.rf), dB, None, dws)
    torch.cuda.synchronize()
    check("das_volume_4x3_9x3x11", kc.cplx(dB)[0],
          V.das_volume(wv.rf, wv.tx_ax, wv.tx_ay, wv.elem_x, wv.elem_y, wv.grid, wv.grid_y, fs, c))

    # batched form: two uneven frames through the persistent gather
    frames, refs = [], []
    for seed, (M, gg) in enumerate([(5, (33, 20, -4e-3, 0.15e-3, 5e-3, 0.15e-3)),
                                    (9, (47, 38, -5e-3, 0.12e-3, 6e-3, 0.12e-3))]):
        opsb, (rxb, pb, gb, Jb) = kc.scheme_both("vernier", ws_.tx_angles, M)
        pl = kc.kk_plan_for(ws_, rxb, pb, gb, Jb, kb.KK_COMPOUND_COHERENT, gg)
        frames.append({"plan": pl, "rf": kc.to_dev(ws_.rf), "rf_theta": pl.empty_rf_theta(),
                       "B": pl.empty_image(), "I": pl.empty_intensity(), "workspace": pl.empty_workspace()})
        refs.append(kk.kk_image(ws_.rf, ws_.elem_x, opsb, gg, fs, c))
    # and the 4 x 3-array volume as the batch's volumetric list
    frames.append({"plan": plan, "rf": kc.to_dev(wv.rf), "rf_theta": plan.empty_rf_theta(),
                   "B": plan.empty_image(), "I": plan.empty_intensity(), "workspace": plan.empty_workspace()})
    refs.append(V.kk_beamform3(y3, wv.elem_x, wv.elem_y, ps, wv.grid, wv.grid_y, fs, c))
    batch = kb.Batch(frames, shape=408)
    batch.run()
    torch.cuda.synchronize()
    for n, f in enumerate(frames):
        check(f"kk_batch_frame{n}", kc.cplx(f["B"]), refs[n])
    print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
