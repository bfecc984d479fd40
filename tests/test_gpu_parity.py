"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  FP32 forms must reach rel-L2 <= 1e-5 over the whole
complex image (and over the compounded intensity)."""
import numpy as np
import pytest

import kksynth
import paper_2603_22496_gb300 as kb
from oracle import kk, schemes
from tests import kkcases as kc

pytestmark = pytest.mark.gpu

TOL = 1e-5       # FP32 end-to-end bound on rel-L2
FS, C = kksynth.FS, kksynth.C_SOUND


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2603_22496_gb300 import build
    build.build()
    kb.load()


# --------------------------------------------------------------------------
# stages, small workload (64 elements, 11 transmits, T = 512, 128x128)
# --------------------------------------------------------------------------
def test_stage_spectrum_matches_oracle():
    import torch
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("same", w.tx_angles, 11)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J)
    F = w.n_samples // 2
    X = torch.empty((F, plan.info.n_tx_used, w.n_elem, 2), device="cuda:0")
    plan.spectrum(kc.to_dev(w.rf), X)
    torch.cuda.synchronize()
    ref = np.transpose(kk.analytic_spectrum(w.rf), (2, 0, 1))       # [F][N][L]
    assert kc.rel_l2(kc.cplx(X), ref) <= 2e-6


@pytest.mark.parametrize("which", ["large_int16", "f32_odd_channels"])
def test_stage_spectrum_1024_bins_matches_oracle(which, request):
    """T = 2048 (F = 1024 bins, a 16 x 16 x 4 transform): every channel of the
    75 x 128 int16 frame, and a float32 record set whose channel count
    (5 x 37) is not a multiple of the records a CTA takes at a time."""
    import torch
    if which == "large_int16":
        w = request.getfixturevalue("large")
    else:
        grid = (40, 36, -3e-3, 0.15e-3, 4e-3, 0.15e-3)
        w = kksynth.workload_custom("spec1024", 77, 37, 0.3e-3, 5, 10.0, 2048, grid,
                                    kksynth.point_phantom([(0.0, 5.0), (1.5, 20.0)]), snr_db=25.0)
    ops, (rx, pairs, grp, J) = kc.scheme_both("same", w.tx_angles, 3)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J)
    F = w.n_samples // 2
    X = torch.empty((F, plan.info.n_tx_used, w.n_elem, 2), device="cuda:0")
    plan.spectrum(kc.to_dev(w.rf), X)
    torch.cuda.synchronize()
    ref = np.transpose(kk.analytic_spectrum(w.rf), (2, 0, 1))       # [F][N][L]
    assert kc.rel_l2(kc.cplx(X), ref) <= 2e-6


def test_stage_shear_matches_oracle():
    """Feed the oracle's spectra (rounded to FP32) and compare Y per bin."""
    import torch
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J)
    Xo = kk.analytic_spectrum(w.rf)                                   # [N][L][F]
    Xf = np.transpose(Xo, (2, 0, 1)).astype(np.complex64)             # [F][N][L]
    X = torch.from_numpy(np.ascontiguousarray(np.stack([Xf.real, Xf.imag], -1))).cuda()
    F = w.n_samples // 2
    Y = torch.empty((F, plan.info.n_tx_used, plan.info.n_rx_used, 2), device="cuda:0")
    plan.shear(X, Y)
    torch.cuda.synchronize()
    d = kk.shear_delays(w.elem_x, ops.rx_angles, C)
    k = np.arange(F)
    W = np.exp(2j * np.pi * k[None, None, :] * (FS * d)[:, :, None] / w.n_samples)
    ref = np.einsum("ilk,olk->kio", Xf.transpose(1, 2, 0).astype(np.complex128), W)
    assert kc.rel_l2(kc.cplx(Y), ref) <= 2e-6


@pytest.mark.parametrize("n_tx,M", [(5, 150), (11, 70), (24, 20), (40, 10), (12, 96), (33, 80)])
def test_stage_shear_few_transmits_matches_oracle(n_tx, M, request):
    """The few-transmit contraction (8 .. 64 transmits per CTA) on transmit
    subsets, against an FP64 einsum of the same FP32 spectra: one bin per CTA
    with the elements split over slices, on two angle tiles (5 x 150,
    11 x 70) and the 32- and 64-transmit tiles (24 x 20 and 40 x 10 on the
    128-element, T = 2048 frame); four bins per CTA with the phasor stepped
    bin to bin, the form of a lone frame with eight four-bin CTAs per SM
    (12 x 96 and 33 x 80 on that frame)."""
    import torch
    w = kksynth.workload_small() if n_tx <= 11 else request.getfixturevalue("large")
    sub = np.arange(n_tx)
    ops, (rx, pairs, grp, J) = kc.scheme_both("shifted", w.tx_angles[:n_tx], M, j=1, tx_subset=sub)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J)
    assert plan.info.n_tx_used == n_tx and plan.info.n_rx_used == M
    Xo = kk.analytic_spectrum(np.asarray(w.rf[:n_tx], dtype=np.float64))  # [n][L][F]
    Xf = np.transpose(Xo, (2, 0, 1)).astype(np.complex64)             # [F][n][L]
    X = torch.from_numpy(np.ascontiguousarray(np.stack([Xf.real, Xf.imag], -1))).cuda()
    F = w.n_samples // 2
    Y = torch.empty((F, n_tx, M, 2), device="cuda:0")
    plan.shear(X, Y)
    torch.cuda.synchronize()
    d = kk.shear_delays(w.elem_x, ops.rx_angles, C)
    k = np.arange(F)
    W = np.exp(2j * np.pi * k[None, None, :] * (FS * d)[:, :, None] / w.n_samples)
    ref = np.einsum("ilk,olk->kio", Xf.transpose(1, 2, 0).astype(np.complex128), W)
    assert kc.rel_l2(kc.cplx(Y), ref) <= 2e-6


@pytest.mark.parametrize("n_elem,n_tx,M", [(20, 9, 16), (64, 11, 11), (77, 9, 5), (128, 8, 16)])
def test_stage_shear_element_slices_matches_oracle(n_elem, n_tx, M):
    """The one-bin few-transmit contraction on 256-bin frames: the elements in
    one chunk (20) or split over two, three (77, the last chunk ragged) and
    four slices per CTA (128), against an FP64 einsum of the same FP32
    spectra; the first three transmits contracted alone equal their rows of
    the whole contraction bit for bit."""
    import torch
    grid = (32, 32, -3e-3, 0.2e-3, 5e-3, 0.2e-3)
    ph = kksynth.point_phantom([(0.0, 8.0), (1.5, 12.0), (-2.0, 16.0)])
    w = kksynth.workload_custom("slices", 31 + n_elem, n_elem, 0.3e-3, n_tx, 8.0, 512, grid, ph, snr_db=30.0)
    rxa = schemes.even_receive_set(np.deg2rad(10.0), M)
    Xo = kk.analytic_spectrum(np.asarray(w.rf, dtype=np.float64))       # [N][L][F]
    Xf = np.transpose(Xo, (2, 0, 1)).astype(np.complex64)             # [F][N][L]
    F = w.n_samples // 2
    out = []
    for n in (n_tx, 3):
        rx, pairs, grp = kc.product_pairs(np.arange(n), [rxa])
        plan = kc.kk_plan_for(w, rx, pairs, grp, 1)
        assert plan.info.n_tx_used == n and plan.info.n_rx_used == M and plan.info.n_bins == F
        Xn = np.ascontiguousarray(Xf[:, :n])
        X = torch.from_numpy(np.ascontiguousarray(np.stack([Xn.real, Xn.imag], -1))).cuda()
        Y = torch.full((F, n, M, 2), float("nan"), device="cuda:0")
        plan.shear(X, Y)
        torch.cuda.synchronize()
        out.append(Y.cpu())
    d = kk.shear_delays(w.elem_x, rxa, C)
    k = np.arange(F)
    W = np.exp(2j * np.pi * k[None, None, :] * (FS * d)[:, :, None] / w.n_samples)
    ref = np.einsum("ilk,olk->kio", Xf.transpose(1, 2, 0).astype(np.complex128), W)
    assert kc.rel_l2(kc.cplx(out[0]), ref) <= 2e-6
    assert torch.equal(out[1], out[0][:, :3])


def test_stage_inverse_matches_oracle():
    import torch
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("vernier", w.tx_angles, 5)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J)
    F = w.n_samples // 2
    rng = np.random.default_rng(4)
    Yh = (rng.standard_normal((F, plan.info.n_tx_used, plan.info.n_rx_used))
          + 1j * rng.standard_normal((F, plan.info.n_tx_used, plan.info.n_rx_used))).astype(np.complex64)
    Y = torch.from_numpy(np.ascontiguousarray(np.stack([Yh.real, Yh.imag], -1))).cuda()
    rt = plan.empty_rf_theta()
    plan.inverse(Y, rt)
    torch.cuda.synchronize()
    ref = kk.inverse_half_spectrum(
        np.stack([Yh[:, i, o] for i, o in zip(ops.tx_index, ops.rx_index)]).astype(np.complex128),
        w.n_samples)
    assert kc.rel_l2(kc.cplx(rt), ref) <= 2e-6


def test_decompose_matches_oracle():
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("shifted", w.tx_angles, 11, j=3)
    B, I, rt, plan = kc.run_kk(w, rx, pairs, grp, J)
    ref = kk.decompose(w.rf, w.elem_x, ops, FS, C)
    assert kc.rel_l2(rt, ref) <= 3e-6


# --------------------------------------------------------------------------
# end to end, small workload: every scheme, compounding, DAS
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind,M,kw", [("same", 11, {}), ("vernier", 11, {}), ("vernier", 6, {}),
                                       ("shifted", 11, {"j": 5}), ("confocal", 11, {}),
                                       ("confocal", 16, {})])
def test_kk_small_end_to_end(kind, M, kw):
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both(kind, w.tx_angles, M, **kw)
    B, I, rt, plan = kc.run_kk(w, rx, pairs, grp, J, compound=kb.KK_COMPOUND_COHERENT)
    ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
    err = kc.rel_l2(B, ref)
    assert err <= TOL, err
    assert kc.rel_l2(I, kk.compound(ref, "coherent")) <= 2 * TOL


@pytest.mark.parametrize("mode", [kb.KK_COMPOUND_COHERENT, kb.KK_COMPOUND_INCOHERENT])
def test_kk_hybrid_compounding(mode):
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("hybrid", w.tx_angles, 7, js=[0, 2, 5])
    B, I, rt, plan = kc.run_kk(w, rx, pairs, grp, J, compound=mode)
    ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
    assert B.shape == ref.shape == (3, 128, 128)
    assert kc.rel_l2(B, ref) <= TOL
    name = "coherent" if mode == kb.KK_COMPOUND_COHERENT else "incoherent"
    assert kc.rel_l2(I, kk.compound(ref, name)) <= 2 * TOL


def test_das_small_end_to_end():
    w = kksynth.workload_small()
    B, I, plan = kc.run_das(w, want_I=True)
    ref = kk.das_image(w.rf, w.tx_angles, w.elem_x, w.grid, FS, C)
    assert kc.rel_l2(B, ref) <= TOL
    assert kc.rel_l2(I, np.abs(ref) ** 2) <= 2 * TOL


def test_point_targets_focus_on_gpu():
    w = kksynth.workload_small(speckle=0)
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    B, I, rt, plan = kc.run_kk(w, rx, pairs, grp, J)
    ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
    A, Ar = np.abs(B[0]), np.abs(ref[0])
    nx, nz, x0, dx, z0, dz = w.grid
    for (x, z) in kksynth.phantom.SMALL_POINTS_MM:
        ix, iz = int(round((x * 1e-3 - x0) / dx)), int(round((z * 1e-3 - z0) / dz))
        sub, subr = A[iz - 6:iz + 7, ix - 6:ix + 7], Ar[iz - 6:iz + 7, ix - 6:ix + 7]
        assert np.argmax(sub) == np.argmax(subr)


# --------------------------------------------------------------------------
# edge cases: ragged grids, short and mixed-radix records, odd sizes, pair
# subsets with duplicates, reads past the record end
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nx,nz", [(1, 1), (33, 7), (45, 70), (97, 31)])
def test_ragged_grids(nx, nz):
    w = kksynth.workload_small()
    x0, z0 = -6e-3, 6e-3
    grid = (nx, nz, x0, 0.11e-3, z0, 0.13e-3)
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 9)
    B, I, rt, plan = kc.run_kk(w, rx, pairs, grp, J, grid=grid)
    ref = kk.kk_image(w.rf, w.elem_x, ops, grid, FS, C)
    assert kc.rel_l2(B, ref) <= TOL
    D, _, _ = kc.run_das(w, grid=grid)
    assert kc.rel_l2(D, kk.das_image(w.rf, w.tx_angles, w.elem_x, grid, FS, C)) <= TOL


@pytest.mark.parametrize("T", [256, 1536, 4096])
def test_record_lengths(T):
    """F = 128 (radix-2 pass), F = 768 (radix-3 pass), F = 2048."""
    grid = (40, 36, -3e-3, 0.15e-3, 4e-3, 0.15e-3)
    ph = kksynth.point_phantom([(0.0, 5.0), (1.5, 6.0)])
    w = kksynth.workload_custom(f"T{T}", 40 + T, 24, 0.3e-3, 5, 10.0, T, grid, ph, snr_db=25.0)
    ops, (rx, pairs, grp, J) = kc.scheme_both("shifted", w.tx_angles, 7, j=1)
    B, I, rt, plan = kc.run_kk(w, rx, pairs, grp, J)
    ref = kk.kk_image(w.rf, w.elem_x, ops, grid, FS, C)
    assert kc.rel_l2(B, ref) <= TOL
    D, _, _ = kc.run_das(w)
    assert kc.rel_l2(D, kk.das_image(w.rf, w.tx_angles, w.elem_x, grid, FS, C)) <= TOL


def test_int16_odd_element_count_and_pair_subset():
    grid = (50, 44, -4e-3, 0.12e-3, 5e-3, 0.14e-3)
    ph = kksynth.point_phantom([(0.5, 6.0), (-1.0, 8.0), (2.0, 9.5)])
    w = kksynth.workload_custom("odd", 77, 37, 0.25e-3, 9, 12.0, 1024, grid, ph, rf_dtype="i16")
    rx = np.deg2rad(np.array([-9.0, -2.5, 0.0, 3.0, 11.0]))
    # a scattered subset with a repeated pair, not a full product
    pairs = np.array([[0, 1], [3, 4], [8, 0], [4, 2], [4, 2], [7, 3], [2, 2], [5, 0]], dtype=np.int32)
    grp = np.array([0, 1, 0, 1, 0, 1, 1, 0], dtype=np.int32)
    ops = schemes.PairSet(w.tx_angles, rx, pairs[:, 0].astype(np.int64),
                          pairs[:, 1].astype(np.int64), grp.astype(np.int64), 2)
    B, I, rt, plan = kc.run_kk(w, rx, pairs, grp, 2, compound=kb.KK_COMPOUND_INCOHERENT)
    ref = kk.kk_image(w.rf, w.elem_x, ops, grid, FS, C)
    assert kc.rel_l2(rt, kk.decompose(w.rf, w.elem_x, ops, FS, C)) <= 3e-6
    assert kc.rel_l2(B, ref) <= TOL
    assert kc.rel_l2(I, kk.compound(ref, "incoherent")) <= 2 * TOL


def test_reads_past_the_record_end():
    """The small grid reaches 24 mm while 512 samples cover ~19.7 mm of depth:
    deep rows read beyond T-1 and must be exactly zero there."""
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("same", w.tx_angles, 11)
    B, I, rt, plan = kc.run_kk(w, rx, pairs, grp, J)
    ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
    assert np.abs(ref[0, -1]).max() == 0.0
    assert np.abs(B[0, -1]).max() == 0.0
    assert kc.rel_l2(B, ref) <= TOL


def test_gpu_linearity_and_determinism():
    import torch
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    rf2 = (1.5 * w.rf).astype(np.float32)
    B1, _, _, plan = kc.run_kk(w, rx, pairs, grp, J)
    B1b, _, _, _ = kc.run_kk(w, rx, pairs, grp, J)
    assert np.array_equal(B1, B1b)                 # run-to-run bitwise identical
    B2, _, _, _ = kc.run_kk(w, rx, pairs, grp, J, rf=rf2)
    assert kc.rel_l2(B2, 1.5 * B1) <= 1e-6


# --------------------------------------------------------------------------
# large workload: 128 elements, 75 transmits, T = 2048 int16, 512x512
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def large():
    return kksynth.workload_large()


def test_large_vernier_8x16_full_image(large):
    w = large
    sub = schemes.strided_subset(75, 8)
    ops, (rx, pairs, grp, J) = kc.scheme_both("vernier", w.tx_angles, 16, tx_subset=sub)
    B, I, rt, plan = kc.run_kk(w, rx, pairs, grp, J)
    assert plan.info.n_pairs == 128
    ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
    assert kc.rel_l2(B, ref) <= TOL


def _sample_pixels(grid, n, seed):
    rng = np.random.default_rng(seed)
    nx, nz = grid[0], grid[1]
    pix = np.stack([rng.integers(0, nx, n), rng.integers(0, nz, n)], 1)
    # always include the four corners and tile seams
    extra = np.array([[0, 0], [nx - 1, 0], [0, nz - 1], [nx - 1, nz - 1], [31, 32], [32, 31]])
    return np.concatenate([pix, extra])


def test_large_full_75x128_sampled_pixels(large):
    w = large
    rxa = schemes.even_receive_set(np.deg2rad(16.0), 128)
    rx, pairs, grp = kc.product_pairs(np.arange(75), [rxa])
    ops = schemes.full_product(w.tx_angles, np.arange(75), [rxa])
    B, I, rt, plan = kc.run_kk(w, rx, pairs, grp, 1, compound=kb.KK_COMPOUND_COHERENT)
    assert plan.info.n_pairs == 9600
    y = kk.decompose(w.rf, w.elem_x, ops, FS, C)
    assert kc.rel_l2(rt, y) <= 3e-6
    pix = _sample_pixels(w.grid, 3000, 1)
    ref = kk.kk_beamform(y, w.elem_x, ops, w.grid, FS, C, pixels=pix)[0]
    got = B[0][pix[:, 1], pix[:, 0]]
    assert kc.rel_l2(got, ref) <= TOL
    assert kc.rel_l2(I[pix[:, 1], pix[:, 0]], np.abs(ref) ** 2) <= 2 * TOL


def test_large_das_sampled_pixels(large):
    w = large
    B, I, plan = kc.run_das(w)
    pix = _sample_pixels(w.grid, 2000, 2)
    ref = kk.das_image(w.rf, w.tx_angles, w.elem_x, w.grid, FS, C, pixels=pix)
    assert kc.rel_l2(B[pix[:, 1], pix[:, 0]], ref) <= TOL


@pytest.mark.parametrize("rows,stage", [(2, 4), (2, 8), (4, 4), (4, 8), (8, 4)])
def test_every_gather_configuration(rows, stage):
    """Every launch shape of the KK gather gives the oracle's image (hybrid
    groups, coherent compounding, ragged grid)."""
    import torch
    w = kksynth.workload_small()
    grid = (70, 58, -5e-3, 0.11e-3, 6e-3, 0.09e-3)
    ops, (rx, pairs, grp, J) = kc.scheme_both("hybrid", w.tx_angles, 7, js=[0, 3, 5])
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, kb.KK_COMPOUND_COHERENT, grid)
    plan.set_gather(rows, stage)
    assert (plan.info.gather_rows, plan.info.gather_stage) == (rows, stage)
    ws, rt, B, I = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
    plan.decompose(kc.to_dev(w.rf), rt, ws)
    plan.beamform(rt, B, I, ws)
    torch.cuda.synchronize()
    ref = kk.kk_image(w.rf, w.elem_x, ops, grid, FS, C)
    assert kc.rel_l2(kc.cplx(B), ref) <= TOL
    assert kc.rel_l2(I.cpu().numpy(), kk.compound(ref, "coherent")) <= 2 * TOL


def test_gather_configuration_rejects_bad_shapes():
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("vernier", w.tx_angles, 5)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J)
    with pytest.raises(kb.KKError):
        plan.set_gather(6, 16)
    with pytest.raises(kb.KKError):
        plan.set_gather(8, 64)
    with pytest.raises(kb.KKError):      # small grid's window too long for 32 x 32 tiles x 16 pairs
        plan.set_gather(8, 16)
    plan.set_gather(4, 8)


def test_workspace_allocated_before_a_shape_change_stays_valid():
    """workspace_bytes covers every launch shape: a workspace allocated at the
    default shape serves every other shape (the grid is chosen so that the
    pair-slice split grows from 2 to 5 across shapes), with nothing written
    past its end (canary) and the same image from every shape."""
    import torch
    w = kksynth.workload_small()
    grid = (512, 256, -19e-3, 0.075e-3, 5e-3, 0.075e-3)
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, kb.KK_COMPOUND_COHERENT, grid)
    nbytes = plan.info.workspace_bytes
    canary = 1 << 20
    raw = torch.full((nbytes + canary,), 0x5A, dtype=torch.uint8, device="cuda")
    ws = raw[:nbytes]
    rt, I = plan.empty_rf_theta(), plan.empty_intensity()
    plan.decompose(kc.to_dev(w.rf), rt, ws)
    images = []
    splits = set()
    for rows, stage in [(4, 16), (8, 4), (8, 8), (2, 4), (4, 4)]:
        plan.set_gather(rows, stage)
        splits.add(plan.info.gather_split)
        assert plan.info.workspace_bytes == nbytes
        B = plan.empty_image()
        plan.beamform(rt, B, I, ws)
        torch.cuda.synchronize()
        images.append(kc.cplx(B))
    assert bool((raw[nbytes:] == 0x5A).all())
    assert len(splits) >= 3
    for img in images[1:]:
        assert kc.rel_l2(img, images[0]) <= 1e-6


@pytest.mark.parametrize("dx", [0.075e-3, 0.3e-3])
def test_windows_before_the_record_start_and_coarse_pitch(dx):
    """A grid from 0.5 mm below the array to past the record's end: the
    staged windows of some (tile, pair) start before sample 0 and others run
    past T - 1, and at the coarse pitch the delay step along x exceeds one
    sample; every pixel matches the oracle."""
    import torch
    w = kksynth.workload_small()
    nx = int(round(20e-3 / dx)) | 1
    grid = (nx, 160, -10e-3, dx, 0.5e-3, 0.15e-3)
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 13)
    plan = kc.kk_plan_for(w, rx, pairs, grp, J, kb.KK_COMPOUND_COHERENT, grid)
    ws, rt, B, I = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
    plan.decompose(kc.to_dev(w.rf), rt, ws)
    plan.beamform(rt, B, I, ws)
    torch.cuda.synchronize()
    ref = kk.kk_image(w.rf, w.elem_x, ops, grid, FS, C)
    assert kc.rel_l2(kc.cplx(B), ref) <= TOL
    assert kc.rel_l2(I.cpu().numpy(), kk.compound(ref, "coherent")) <= 2 * TOL
