"""Volumetric KK with a 2D array on the GPU against the FP64 oracle
(oracle.volume).  FP32 forms at the plain path's bound, rel-L2 <= 1e-5 over
the whole complex volume; a linear array described as a volume reproduces the
linear-array plan; groups, compounding, pair-range splits, the BF16 form and
the streaming decomposition run on volumes; the calls that do not support
volumes refuse them."""
import numpy as np
import pytest

import kksynth
import paper_2603_22496_gb300 as kb
from oracle import kk, schemes, volume as V
from tests import kkcases as kc

pytestmark = pytest.mark.gpu
FS, C = kksynth.FS, kksynth.C_SOUND
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2603_22496_gb300 import build
    build.build()
    kb.load()


def _plan(w, ps, compound=kb.KK_COMPOUND_COHERENT, precision=kb.KK_PREC_F32):
    pairs = np.stack([ps.tx_index, ps.rx_index], 1).astype(np.int32)
    return kb.Plan(w.elem_x, w.tx_ax, w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), rx_angles=ps.rx_ax,
                   pairs=pairs, group_of_pair=ps.group.astype(np.int32), n_groups=ps.n_groups,
                   compound=compound, precision=precision, elem_y=w.elem_y, tx_angles_y=w.tx_ay,
                   rx_angles_y=ps.rx_ay, grid_y=w.grid_y)


def _run(plan, rf):
    import torch
    ws, rt, B, I = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
    plan.decompose(kc.to_dev(rf), rt, ws)
    plan.beamform(rt, B, I, ws)
    torch.cuda.synchronize()
    return kc.cplx(B), I.cpu().numpy().astype(np.float64), kc.cplx(rt)


def _rx_product(theta_deg, m):
    rx1 = schemes.even_receive_set(np.deg2rad(theta_deg), m)
    return np.tile(rx1, m), np.repeat(rx1, m)


@pytest.fixture(scope="module")
def small():
    return kksynth.volume_workload(speckle=400)


def test_volume_full_matches_oracle(small):
    w = small
    ps = V.product_set(w.tx_ax, w.tx_ay, [_rx_product(12.0, 7)])
    plan = _plan(w, ps)
    info = plan.info
    assert info.is_volume == 1 and info.ny == 48 and info.n_pairs == 9 * 49
    assert (info.sep_lx, info.sep_ly, info.sep_mx, info.sep_my) == (16, 16, 7, 7)
    B, I, rt = _run(plan, w.rf)
    assert B.shape == (1, 48, 64, 48)
    y = V.decompose3(w.rf, w.elem_x, w.elem_y, ps, FS, C)
    assert kc.rel_l2(rt, y) <= 3e-6
    ref = V.kk_beamform3(y, w.elem_x, w.elem_y, ps, w.grid, w.grid_y, FS, C)
    assert kc.rel_l2(B, ref) <= TOL
    assert kc.rel_l2(I, np.abs(ref[0]) ** 2) <= 2 * TOL


@pytest.mark.parametrize("order", ["shuffled", "y_fastest"])
def test_separable_contraction_any_order_and_against_full_form(small, order):
    """The separable contraction (16 x 16 grid, 5 x 4 receive product) with
    elements listed in shuffled order (gathered into the grid) or y-fastest
    (bulk copies, the axes' roles swapped) and receive waves in shuffled
    order matches the oracle; one more receive wave off the product turns
    the plan to the full form, whose records of the shared pairs agree with
    the separable ones."""
    w = small
    rng = np.random.default_rng(11)
    rx1x = schemes.even_receive_set(np.deg2rad(12.0), 5)
    rx1y = schemes.even_receive_set(np.deg2rad(9.0), 4)
    rxx, rxy = np.tile(rx1x, 4), np.repeat(rx1y, 5)
    ro = rng.permutation(rxx.shape[0])
    L = w.elem_x.shape[0]
    eo = rng.permutation(L) if order == "shuffled" else np.arange(L).reshape(16, 16).T.ravel()
    ex, ey, rf = w.elem_x[eo], w.elem_y[eo], np.ascontiguousarray(w.rf[:, eo])
    ps = V.product_set(w.tx_ax, w.tx_ay, [(rxx[ro], rxy[ro])])
    pairs = np.stack([ps.tx_index, ps.rx_index], 1).astype(np.int32)

    def plan_of(bx, by, pr):
        return kb.Plan(ex, w.tx_ax, w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), rx_angles=bx, pairs=pr,
                       compound=kb.KK_COMPOUND_COHERENT, elem_y=ey, tx_angles_y=w.tx_ay, rx_angles_y=by,
                       grid_y=w.grid_y)

    sep = plan_of(ps.rx_ax, ps.rx_ay, pairs)
    assert (sep.info.sep_lx, sep.info.sep_ly, sep.info.sep_mx, sep.info.sep_my) == (16, 16, 5, 4)
    B, _, rt = _run(sep, rf)
    y = V.decompose3(rf, ex, ey, ps, FS, C)
    assert kc.rel_l2(rt, y) <= 3e-6
    assert kc.rel_l2(B, V.kk_beamform3(y, ex, ey, ps, w.grid, w.grid_y, FS, C)) <= TOL
    # one extra receive wave: not a product any more
    bx, by = np.append(ps.rx_ax, np.deg2rad(1.0)), np.append(ps.rx_ay, np.deg2rad(-2.0))
    extra = np.array([[i, bx.shape[0] - 1] for i in range(w.tx_ax.shape[0])], np.int32)
    full = plan_of(bx, by, np.concatenate([pairs, extra]))
    assert full.info.sep_lx == 0
    _, _, rt_full = _run(full, rf)
    assert kc.rel_l2(rt_full[:pairs.shape[0]], rt) <= 2e-6


def test_separable_contraction_odd_grid():
    """7 x 5 elements (odd L: the gathered form), 5 x 5 receive waves, 3 x 2
    tilts: the separable contraction against the oracle, and a batch of
    transmits that does not fill the last chunk."""
    w = kksynth.volume_workload(seed=3200, lx=7, ly=5, ntx=3, nty=2, n_samples=512, nx=24, ny=16, nz=32,
                                speckle=200)
    ps = V.product_set(w.tx_ax, w.tx_ay, [_rx_product(10.0, 5)])
    plan = _plan(w, ps)
    assert (plan.info.sep_lx, plan.info.sep_ly, plan.info.sep_mx, plan.info.sep_my) == (7, 5, 5, 5)
    B, _, rt = _run(plan, w.rf)
    y = V.decompose3(w.rf, w.elem_x, w.elem_y, ps, FS, C)
    assert kc.rel_l2(rt, y) <= 3e-6
    assert kc.rel_l2(B, V.kk_beamform3(y, w.elem_x, w.elem_y, ps, w.grid, w.grid_y, FS, C)) <= TOL


def test_volume_hybrid_groups_incoherent(small):
    """Three groups (x schemes shifted by j = 0, 1, 2) compounded incoherently:
    the multi-group kernel on volumes, with a pair-range split."""
    w = small
    tx1 = np.deg2rad(np.linspace(-8, 8, 3))
    groups = [V.separable_scheme("shifted", tx1, tx1, 5, 5, jx=j, jy=j) for j in (0, 1, 2)]
    ps = V.product_set(w.tx_ax, w.tx_ay, groups)
    plan = _plan(w, ps, compound=kb.KK_COMPOUND_INCOHERENT)
    B, I, _ = _run(plan, w.rf)
    ref = V.kk_volume(w.rf, w.elem_x, w.elem_y, ps, w.grid, w.grid_y, FS, C)
    assert kc.rel_l2(B, ref) <= TOL
    assert kc.rel_l2(I, np.sum(np.abs(ref) ** 2, axis=0)) <= 2 * TOL


def test_linear_array_as_a_volume():
    """A linear array, zero y tilts and one slice at y = 0 described as a volume
    gives the linear-array plan's image (the coefficients differ only by the
    rounding of sqrt(1 - sin^2) against cos)."""
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    B2, I2, _, _ = kc.run_kk(w, rx, pairs, grp, J, compound=kb.KK_COMPOUND_COHERENT)
    plan = kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), rx_angles=rx,
                   pairs=pairs, group_of_pair=grp, n_groups=J, compound=kb.KK_COMPOUND_COHERENT,
                   elem_y=np.zeros_like(w.elem_x), tx_angles_y=np.zeros_like(w.tx_angles),
                   rx_angles_y=np.zeros_like(rx), grid_y=(1, 0.0, 0.0))
    assert plan.info.is_volume == 1
    B3, I3, _ = _run(plan, w.rf)
    assert kc.rel_l2(B3[:, 0], B2) <= 1e-6
    assert kc.rel_l2(I3[0], I2) <= 2e-6


def test_volume_bf16_form_and_sampled_oracle():
    """8 x 16 array (128 elements: the tensor-core forms), int16 at 30 dB,
    5 x 3 tilts, 9 x 5 receive waves, 96 x 64 x 128 voxels; the oracle on
    sampled voxels."""
    w = kksynth.volume_workload(seed=3100, lx=16, ly=8, ntx=5, nty=3, theta_max_deg=10.0, n_samples=2048,
                                nx=96, ny=64, nz=128, dxyz=0.1e-3, z0=5e-3, speckle=3000, rf_dtype="i16")
    rx1x = schemes.even_receive_set(np.deg2rad(14.0), 9)
    rx1y = schemes.even_receive_set(np.deg2rad(10.0), 5)
    ps = V.product_set(w.tx_ax, w.tx_ay, [(np.tile(rx1x, 5), np.repeat(rx1y, 9))])
    rng = np.random.default_rng(7)
    vox = np.stack([rng.integers(0, 96, 1500), rng.integers(0, 64, 1500), rng.integers(0, 128, 1500)], 1)
    ref = V.kk_volume(w.rf, w.elem_x, w.elem_y, ps, w.grid, w.grid_y, FS, C, voxels=vox)[0]
    for prec, tol in ((kb.KK_PREC_F32, TOL), (kb.KK_PREC_BF16, 1e-2)):
        plan = _plan(w, ps, precision=prec)
        B, _, _ = _run(plan, w.rf)
        got = B[0][vox[:, 1], vox[:, 2], vox[:, 0]]
        assert kc.rel_l2(got, ref) <= tol, prec


def test_volume_streaming_equals_whole_frame(small):
    import torch
    w = small
    ps = V.product_set(w.tx_ax, w.tx_ay, [_rx_product(12.0, 5)])
    plan = _plan(w, ps)
    B0, I0, _ = _run(plan, w.rf)
    st = kb.Stream(plan, 4)
    h = torch.from_numpy(np.ascontiguousarray(w.rf)).pin_memory()
    B, I = plan.empty_image(), plan.empty_intensity()
    st.push_many(0, h_events=h)
    st.end_frame(B, I)
    st.sync()
    assert np.array_equal(kc.cplx(B), B0) and np.array_equal(I.cpu().numpy().astype(np.float64), I0)


def test_volume_rejections(small):
    import torch
    w = small
    ps = V.product_set(w.tx_ax, w.tx_ay, [_rx_product(12.0, 3)])
    pairs = np.stack([ps.tx_index, ps.rx_index], 1).astype(np.int32)
    bad = [dict(rx_angles_y=np.full(ps.rx_ay.shape, np.deg2rad(75.0))),        # tilts do not propagate
           dict(rx_angles_y=ps.rx_ay, grid_y=(4, 0.0, 0.0)),                     # ny > 1 needs dy > 0
           dict(rx_angles_y=ps.rx_ay, grid_y=(4, np.nan, 1e-4))]
    for kw in bad:
        args = dict(elem_y=w.elem_y, tx_angles_y=w.tx_ay, grid_y=w.grid_y)
        args.update(kw)
        with pytest.raises(kb.KKError) as e:
            kb.Plan(w.elem_x, w.tx_ax, w.grid, w.c, w.fs, w.n_samples, kb.KK_RF_F32, rx_angles=ps.rx_ax,
                    pairs=pairs, **args)
        assert e.value.status == kb.KK_ERR_INVALID_ARG
    torch.cuda.synchronize()


# --------------------------------------------------------------------------
# volumetric DAS (Eq. (DAS) with a 2D array): the staged DAS gather with the
# per-slice transmit term and the elements' y offsets
# --------------------------------------------------------------------------
def _das_plan(w, f_number=0.0, grid=None):
    return kb.Plan(w.elem_x, w.tx_ax, grid or w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w), das=True,
                   elem_y=w.elem_y, tx_angles_y=w.tx_ay, grid_y=w.grid_y, f_number=f_number)


def test_volume_das_matches_oracle(small):
    import torch
    w = small
    plan = _das_plan(w)
    info = plan.info
    assert info.is_das == 1 and info.is_volume == 1 and info.ny == 48
    assert info.launches_beamform == 4           # analytic signal (2), gather, slice reduce
    ws, B, I = plan.empty_workspace(), plan.empty_image(), plan.empty_intensity()
    assert B.shape == (1, 48, 64, 48, 2)
    plan.das(kc.to_dev(w.rf), B, I, ws)
    torch.cuda.synchronize()
    assert plan.status() == 0
    ref = V.das_volume(w.rf, w.tx_ax, w.tx_ay, w.elem_x, w.elem_y, w.grid, w.grid_y, FS, C)
    got = kc.cplx(B)[0]
    assert kc.rel_l2(got, ref) <= TOL
    assert kc.rel_l2(I.cpu().numpy().astype(np.float64), np.abs(ref) ** 2) <= 2 * TOL
    # each point target's peak sits on the oracle's voxel, within a voxel of
    # the target
    nx, nz, x0, dx, z0, dz = w.grid
    ny, y0, dy = w.grid_y
    for px, py, pz in w.points[:w.n_points, :3]:
        ix, iy, iz = (int(round((px - x0) / dx)), int(round((py - y0) / dy)), int(round((pz - z0) / dz)))
        win = np.s_[iy - 3:iy + 4, iz - 3:iz + 4, ix - 3:ix + 4]
        pg = np.unravel_index(int(np.argmax(np.abs(got[win]))), (7, 7, 7))
        pr = np.unravel_index(int(np.argmax(np.abs(ref[win]))), (7, 7, 7))
        assert pg == pr and max(abs(int(v) - 3) for v in pg) <= 1, (pg, pr)


def test_volume_das_ragged_and_int16():
    """A ragged volume (nx, nz off the tile grid, odd ny) from int16 RF with a
    3 x 4 array: more pair slices than tiles per SM, so the slice reduce runs."""
    import torch
    w = kksynth.volume_workload(seed=3100, lx=3, ly=4, nx=37, ny=5, nz=23, n_samples=512, speckle=60,
                                rf_dtype="i16", snr_db=30.0,
                                points=((0.0, 0.0, 7e-3), (1e-3, -0.3e-3, 8e-3)))
    plan = _das_plan(w)
    ws, B = plan.empty_workspace(), plan.empty_image()
    plan.das(kc.to_dev(w.rf), B, None, ws)
    torch.cuda.synchronize()
    ref = V.das_volume(w.rf, w.tx_ax, w.tx_ay, w.elem_x, w.elem_y, w.grid, w.grid_y, FS, C)
    assert kc.rel_l2(kc.cplx(B)[0], ref) <= TOL


def test_volume_das_refusals(small):
    w = small
    with pytest.raises(kb.KKError) as e:
        _das_plan(w, f_number=1.5)
    assert e.value.status == kb.KK_ERR_UNSUPPORTED
    nx, nz, x0, dx, z0, dz = w.grid
    with pytest.raises(kb.KKError) as e:               # 1 mm voxels: windows beyond 256 samples
        _das_plan(w, grid=(nx, nz, x0, 1e-3, z0, 1e-3))
    assert e.value.status == kb.KK_ERR_UNSUPPORTED
