"""Reduced-precision decomposition forms (BF16, FP16, FP8-e4m3 with
per-column scale) on the tensor cores, against the FP64 oracle.

Stated bound (rel-L2 of the complex image and of the decomposed records):
<= 1e-2 for every form -- BF16, FP16 and FP8 (each FP8 operand held as two
e4m3 terms); point-target peaks at exactly the oracle's pixels for every
form.
"""
import numpy as np
import pytest

import kksynth
import paper_2603_22496_gb300 as kb
from oracle import kk
from tests import kkcases as kc

pytestmark = pytest.mark.gpu

FS, C = kksynth.FS, kksynth.C_SOUND
FORMS = {"bf16": (kb.KK_PREC_BF16, 1e-2), "f16": (kb.KK_PREC_F16, 1e-2),
         "f8e4m3": (kb.KK_PREC_F8E4M3, 1e-2)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2603_22496_gb300 import build
    build.build()
    kb.load()


def _plan(w, rx, pairs, grp, J, prec, compound=kb.KK_COMPOUND_NONE, grid=None):
    return kb.Plan(w.elem_x, w.tx_angles, grid or w.grid, w.c, w.fs, w.n_samples, kc.rf_dtype_of(w),
                   rx_angles=rx, pairs=pairs, group_of_pair=grp, n_groups=J, compound=compound,
                   precision=prec)


def _run(plan, rf):
    import torch
    ws, rt, B = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image()
    plan.decompose(kc.to_dev(rf), rt, ws)
    plan.beamform(rt, B, None, ws)
    torch.cuda.synchronize()
    assert plan.status() == kb.KK_OK
    return kc.cplx(B)


@pytest.mark.parametrize("form", ["bf16", "f16", "f8e4m3"])
def test_tensor_core_contraction_stage(form):
    """kk_shear on given spectra against an FP64 einsum of the same (rounded)
    spectra: isolates the tensor-core contraction and its on-chip W."""
    import torch
    prec, _ = FORMS[form]
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    plan = _plan(w, rx, pairs, grp, J, prec)
    F, Nu, Mu, L = plan.info.n_bins, plan.info.n_tx_used, plan.info.n_rx_used, w.n_elem
    Xo = np.transpose(kk.analytic_spectrum(w.rf), (2, 0, 1))          # [F][N][L]
    Xo = Xo / np.abs(Xo).max()
    # float16 spectra are held times 2^-ceil(log2(2T)); kk_shear undoes it
    xs = 1.0 if form == "bf16" else 2.0 ** -int(np.ceil(np.log2(2 * w.n_samples)))
    if form == "bf16":
        t = torch.from_numpy(np.ascontiguousarray(np.stack([Xo.real, Xo.imag], -1))).float().to(torch.bfloat16)
    else:
        t = torch.from_numpy(np.ascontiguousarray(np.stack([Xo.real, Xo.imag], -1)) * xs).float().to(torch.float16)
    Xr = t.float().numpy() / xs
    Xr = Xr[..., 0] + 1j * Xr[..., 1]
    X = t.cuda().contiguous()
    Y = torch.empty((F, Nu, Mu, 2), device="cuda")
    plan.shear(X, Y)
    torch.cuda.synchronize()
    assert plan.status() == kb.KK_OK
    d = kk.shear_delays(w.elem_x, ops.rx_angles, C)
    k = np.arange(F)
    Wm = np.exp(2j * np.pi * k[None, None, :] * (FS * d)[:, :, None] / w.n_samples)
    ref = np.einsum("kil,olk->kio", Xr.astype(np.complex128), Wm)
    err = kc.rel_l2(kc.cplx(Y), ref)
    bound = {"bf16": 1e-2, "f16": 3e-3, "f8e4m3": 1e-2}[form]
    assert err <= bound, err


@pytest.mark.parametrize("form", ["bf16", "f16", "f8e4m3"])
def test_precision_forms_end_to_end_small(form):
    prec, bound = FORMS[form]
    w = kksynth.workload_small()
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    B = _run(_plan(w, rx, pairs, grp, J, prec), w.rf)
    ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
    err = kc.rel_l2(B, ref)
    assert err <= bound, err


@pytest.mark.parametrize("form", ["bf16", "f16", "f8e4m3"])
def test_precision_forms_point_peaks_exact(form):
    prec, _ = FORMS[form]
    w = kksynth.workload_small(speckle=0)
    ops, (rx, pairs, grp, J) = kc.scheme_both("confocal", w.tx_angles, 11)
    B = _run(_plan(w, rx, pairs, grp, J, prec), w.rf)
    ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
    A, Ar = np.abs(B[0]), np.abs(ref[0])
    nx, nz, x0, dx, z0, dz = w.grid
    for (x, z) in kksynth.phantom.SMALL_POINTS_MM:
        ix, iz = int(round((x * 1e-3 - x0) / dx)), int(round((z * 1e-3 - z0) / dz))
        sub, subr = A[iz - 6:iz + 7, ix - 6:ix + 7], Ar[iz - 6:iz + 7, ix - 6:ix + 7]
        assert np.argmax(sub) == np.argmax(subr), (form, x, z)


@pytest.mark.parametrize("form", ["bf16", "f16", "f8e4m3"])
def test_precision_forms_large_vernier(form):
    """128 elements, 75 transmits, T = 2048 int16, vernier 8 x 16 on 512 x 512."""
    from oracle import schemes
    prec, bound = FORMS[form]
    w = kksynth.workload_large()
    sub = schemes.strided_subset(75, 8)
    ops, (rx, pairs, grp, J) = kc.scheme_both("vernier", w.tx_angles, 16, tx_subset=sub)
    B = _run(_plan(w, rx, pairs, grp, J, prec), w.rf)
    ref = kk.kk_image(w.rf, w.elem_x, ops, w.grid, FS, C)
    assert kc.rel_l2(B, ref) <= bound


@pytest.mark.parametrize("form", ["bf16", "f16", "f8e4m3"])
def test_precision_forms_odd_shapes(form):
    """Odd element count (37: phases read one by one, a padded last K chunk),
    int16 records, 9 transmits, a scattered pair subset with a repeated pair
    (records through the inverse's column table) in two incoherently
    compounded groups, and a ragged grid: image, intensity and the point
    peaks against the oracle."""
    import torch
    from oracle import schemes
    prec, bound = FORMS[form]
    grid = (50, 44, -4e-3, 0.12e-3, 5e-3, 0.14e-3)
    pts = [(0.5, 6.0), (-1.0, 8.0), (2.0, 9.5)]
    w = kksynth.workload_custom("odd", 77, 37, 0.25e-3, 9, 12.0, 1024, grid, kksynth.point_phantom(pts),
                                rf_dtype="i16")
    rx = np.deg2rad(np.array([-9.0, -2.5, 0.0, 3.0, 11.0]))
    pairs = np.array([[0, 1], [3, 4], [8, 0], [4, 2], [4, 2], [7, 3], [2, 2], [5, 0], [1, 1], [6, 4]],
                     dtype=np.int32)
    grp = np.array([0, 1, 0, 1, 0, 1, 1, 0, 1, 0], dtype=np.int32)
    ops = schemes.PairSet(w.tx_angles, rx, pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64),
                          grp.astype(np.int64), 2)
    plan = _plan(w, rx, pairs, grp, 2, prec, kb.KK_COMPOUND_INCOHERENT)
    ws, rt, B, I = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
    plan.decompose(kc.to_dev(w.rf), rt, ws)
    plan.beamform(rt, B, I, ws)
    torch.cuda.synchronize()
    assert plan.status() == kb.KK_OK
    ref = kk.kk_image(w.rf, w.elem_x, ops, grid, FS, C)
    Bg = kc.cplx(B)
    assert kc.rel_l2(Bg, ref) <= bound
    assert kc.rel_l2(I.cpu().numpy().astype(np.float64), kk.compound(ref, "incoherent")) <= 2 * bound
    nx, nz, x0, dx, z0, dz = grid
    A, Ar = np.abs(Bg).sum(0), np.abs(ref).sum(0)
    for x, z in pts:
        ix, iz = int(round((x * 1e-3 - x0) / dx)), int(round((z * 1e-3 - z0) / dz))
        sub, subr = A[iz - 5:iz + 6, ix - 5:ix + 6], Ar[iz - 5:iz + 6, ix - 5:ix + 6]
        assert np.argmax(sub) == np.argmax(subr), (form, x, z)


def test_precision_plan_limits():
    w = kksynth.workload_custom("L160", 3, 160, 0.2e-3, 3, 8.0, 512, (8, 8, -1e-3, 0.2e-3, 5e-3, 0.2e-3),
                                kksynth.point_phantom([(0.0, 6.0)]))
    with pytest.raises(kb.KKError) as e:
        kb.Plan(w.elem_x, w.tx_angles, w.grid, w.c, w.fs, w.n_samples, kb.KK_RF_F32,
                rx_angles=np.zeros(1), pairs=np.array([[0, 0]], np.int32), precision=kb.KK_PREC_BF16)
    assert e.value.status == kb.KK_ERR_UNSUPPORTED


@pytest.fixture(scope="module")
def full_frame_oracle():
    """The 75 x 128 frame the benchmark times: oracle records and 3000 sampled pixels."""
    from oracle import schemes
    w = kksynth.workload_large()
    rxa = schemes.even_receive_set(np.deg2rad(16.0), 128)
    rx, pairs, grp = kc.product_pairs(np.arange(75), [rxa])
    ops = schemes.full_product(w.tx_angles, np.arange(75), [rxa])
    y = kk.decompose(w.rf, w.elem_x, ops, FS, C)
    rng = np.random.default_rng(11)
    pix = np.stack([rng.integers(0, 512, 3000), rng.integers(0, 512, 3000)], 1)
    ref = kk.kk_beamform(y, w.elem_x, ops, w.grid, FS, C, pixels=pix)[0]
    return w, rx, pairs, grp, y, pix, ref


@pytest.mark.parametrize("form", ["bf16", "f16", "f8e4m3"])
def test_precision_forms_full_75x128_sampled(form, full_frame_oracle):
    """The benchmark's frame and launch configuration (75 transmits x 128 receive
    angles, int16, 512 x 512) in each reduced-precision form: decomposed
    records and sampled pixels within the form's stated bound."""
    import torch
    w, rx, pairs, grp, y, pix, ref = full_frame_oracle
    prec, bound = FORMS[form]
    plan = _plan(w, rx, pairs, grp, 1, prec, compound=kb.KK_COMPOUND_COHERENT)
    ws, rt, B, I = plan.empty_workspace(), plan.empty_rf_theta(), plan.empty_image(), plan.empty_intensity()
    plan.decompose(kc.to_dev(w.rf), rt, ws)
    plan.beamform(rt, B, I, ws)
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert kc.rel_l2(kc.cplx(rt), y) <= bound
    got = kc.cplx(B)[0][pix[:, 1], pix[:, 0]]
    assert kc.rel_l2(got, ref) <= bound
