"""Image-quality kernels (gCNR, FWHM) on the GPU against the oracle.

Inputs are seeded synthetic speckle images (kksynth), never a beamformer's
output.  Every integer decision (region label, histogram bin, argmax,
crossing index) is taken with the same explicitly rounded operations on both
sides, and so is the final arithmetic, so the comparison is exact: gCNR
values, peak indices, peak envelopes and widths must be identical (NaN where
the oracle gives NaN).
"""
import numpy as np
import pytest

import kksynth
import paper_2603_22496_gb300 as kb
from oracle import quality as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2603_22496_gb300 import build
    build.build()
    kb.load()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _images(kind, imgs):
    """Device tensor for the kernel and host array for the oracle (same bytes)."""
    if kind == kb.KK_IMAGE_COMPLEX:
        return _dev(imgs.view(np.float32)), imgs
    re = imgs.real.astype(np.float32)
    im = imgs.imag.astype(np.float32)
    inten = np.add(np.multiply(re, re, dtype=np.float32), np.multiply(im, im, dtype=np.float32),
                   dtype=np.float32)
    return _dev(inten), inten


def _eq_nan(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape
    same = (a == b) | (np.isnan(a) & np.isnan(b))
    assert same.all(), (a[~same], b[~same])


GRID = (160, 128, -8e-3, 0.1e-3, 4e-3, 0.08e-3)   # x in [-8, 7.9] mm, z in [4, 14.16] mm
PAIRS = [
    # disk vs annulus (the usual lesion / background pair)
    ((Q.REGION_DISK, -3e-3, 8e-3, 1.2e-3, 0), (Q.REGION_ANNULUS, -3e-3, 8e-3, 1.6e-3, 2.5e-3)),
    # disk vs a rectangle beside it at the same depth (the paper's Fig. 5 layout)
    ((Q.REGION_DISK, 3e-3, 10e-3, 1.0e-3, 0), (Q.REGION_RECT, 4.5e-3, 7e-3, 9e-3, 11e-3)),
    # rectangle running off the grid vs an overlapping disk (pixels in both)
    ((Q.REGION_RECT, -9e-3, -6e-3, 3e-3, 6e-3), (Q.REGION_DISK, -6.5e-3, 5e-3, 1.5e-3, 0)),
    # region entirely outside the grid: NaN
    ((Q.REGION_DISK, 30e-3, 8e-3, 1e-3, 0), (Q.REGION_RECT, -1e-3, 1e-3, 5e-3, 6e-3)),
    # whole-grid background
    ((Q.REGION_DISK, 0.0, 12e-3, 0.5e-3, 0), (Q.REGION_RECT, -1, 1, -1, 1)),
]


def _grid_px(x, z, grid=GRID):
    nx, nz, x0, dx, z0, dz = grid
    return (x - x0) / dx, (z - z0) / dz


def _speckle(seed, n, grid=GRID, points=()):
    disks = []
    for inside, _ in PAIRS[:2]:
        cx, cz = _grid_px(inside[1], inside[2], grid)
        disks.append((cx, cz, inside[3] / min(grid[3], grid[5])))   # covers the disk region
    return kksynth.speckle_images(seed, n, grid[0], grid[1], disks_px=disks, points_px=points)


@pytest.mark.parametrize("kind", [kb.KK_IMAGE_COMPLEX, kb.KK_IMAGE_INTENSITY])
@pytest.mark.parametrize("n_bins", [1, 7, 256, 4096])
def test_gcnr_matches_oracle_exactly(kind, n_bins):
    import torch
    imgs = _speckle(11 + n_bins, 6)
    d_img, h_img = _images(kind, imgs)
    q = kb.Quality(GRID, [p[0] for p in PAIRS], [p[1] for p in PAIRS], n_bins=n_bins, image_kind=kind)
    got = q.gcnr(d_img)
    torch.cuda.synchronize()
    want = np.array([[Q.gcnr(h_img[n], GRID, a, b, n_bins, kind) for a, b in PAIRS]
                     for n in range(imgs.shape[0])])
    _eq_nan(got.cpu().numpy(), want)
    if n_bins >= 7:   # the dark disks give a clear separation; the overlap pair does not
        assert (want[:, 0] > 0.5).all() and (want[:, 1] > 0.5).all()
    assert np.isnan(want[:, 3]).all()


def test_gcnr_constant_and_disjoint_images():
    """A constant image gives 0 (hi == lo); two constant levels give 1."""
    import torch
    nx, nz = GRID[0], GRID[1]
    imgs = np.full((2, nz, nx), 2.0 + 0j, dtype=np.complex64)
    m = Q.region_mask(GRID, PAIRS[0][0])
    imgs[1][m] = 0.25j
    q = kb.Quality(GRID, [PAIRS[0][0]], [PAIRS[0][1]], n_bins=64)
    got = q.gcnr(_dev(imgs.view(np.float32)))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), [[0.0], [1.0]])


def test_gcnr_on_large_grid_sampled():
    """512 x 512 images at 0.075 mm with the three 2 mm cysts of the large
    phantom: the whole batch on the GPU, the oracle on three sampled images."""
    import torch
    nx = nz = 512
    dx = 0.075e-3
    grid = (nx, nz, -dx * (nx - 1) / 2, dx, 5e-3, dx)
    pairs = [((Q.REGION_DISK, cx * 1e-3, cz * 1e-3, 1.5e-3, 0),
              (Q.REGION_ANNULUS, cx * 1e-3, cz * 1e-3, 2.5e-3, 3.5e-3)) for cx, cz in kksynth.LARGE_CYSTS_MM]
    disks = [(((cx * 1e-3) - grid[2]) / dx, ((cz * 1e-3) - grid[4]) / dx, 2e-3 / dx)
             for cx, cz in kksynth.LARGE_CYSTS_MM]
    imgs = kksynth.speckle_images(5, 32, nx, nz, disks_px=disks)
    q = kb.Quality(grid, [p[0] for p in pairs], [p[1] for p in pairs], n_bins=256)
    got = q.gcnr(_dev(imgs.view(np.float32)))
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    for n in (0, 17, 31):
        want = [Q.gcnr(imgs[n], grid, a, b, 256) for a, b in pairs]
        _eq_nan(got[n], want)
    assert (got > 0.8).all()


def _targets():
    return [(40, 30, 6, 6), (100, 90, 5, 4), (0, 0, 3, 3), (159, 127, 2, 2),   # corner windows
            (400, 10, 3, 3),                                                  # outside: empty
            (80, 64, 0, 0), (120, 20, 20, 15)]


@pytest.mark.parametrize("kind", [kb.KK_IMAGE_COMPLEX, kb.KK_IMAGE_INTENSITY])
def test_fwhm_matches_oracle_exactly(kind):
    import torch
    pts = [(40.3, 30.0), (100.0, 89.6), (1.0, 2.0), (120.0, 20.0)]
    imgs = _speckle(23, 5, points=pts)
    d_img, h_img = _images(kind, imgs)
    tg = _targets()
    q = kb.Quality(GRID, targets=tg, image_kind=kind)
    raw = q.fwhm(d_img)
    torch.cuda.synchronize()
    got = kb.decode_fwhm(raw)
    assert got.shape == (imgs.shape[0], len(tg))
    for n in range(imgs.shape[0]):
        for t, target in enumerate(tg):
            w = Q.fwhm(h_img[n], GRID, target, kind)
            g = got[n, t]
            assert (int(g["ix"]), int(g["iz"])) == (w["ix"], w["iz"]), (n, t)
            _eq_nan([g["peak"], g["lateral"], g["axial"]], [w["peak"], w["lateral"], w["axial"]])
    # the bright points are resolved: finite widths of a few pixels
    lat = got["lateral"][:, 0]
    assert np.isfinite(lat).all() and (lat > 2 * GRID[3]).all() and (lat < 10 * GRID[3]).all()
    assert (got["ix"][:, 4] == -1).all()


def test_fwhm_ties_and_plateaus():
    """Equal maxima pick the first in row-major order; a plateau that reaches
    the edge gives NaN on that side."""
    import torch
    nx, nz = 64, 32
    grid = (nx, nz, 0.0, 1e-4, 0.0, 1e-4)
    img = np.zeros((1, nz, nx), dtype=np.complex64)
    img[0, 10, 30] = img[0, 10, 20] = img[0, 11, 5] = 3.0
    img[0, 20, :] = 1.0                     # row that never falls below half
    tg = [(20, 10, 15, 3), (40, 20, 2, 0)]
    q = kb.Quality(grid, targets=tg)
    got = kb.decode_fwhm(q.fwhm(_dev(img.view(np.float32))))
    torch.cuda.synchronize()
    for t, target in enumerate(tg):
        w = Q.fwhm(img[0], grid, target)
        g = got[0, t]
        assert (int(g["ix"]), int(g["iz"])) == (w["ix"], w["iz"])
        _eq_nan([g["peak"], g["lateral"], g["axial"]], [w["peak"], w["lateral"], w["axial"]])
    assert (int(got[0, 0]["ix"]), int(got[0, 0]["iz"])) == (20, 10)
    assert np.isnan(got[0, 1]["lateral"]) and np.isfinite(got[0, 1]["axial"])


def test_empty_batches_and_counts_are_no_ops():
    import torch
    q = kb.Quality(GRID, targets=[(1, 1, 1, 1)])
    x = torch.zeros(2 * GRID[0] * GRID[1], dtype=torch.float32, device="cuda")
    kb.kk_quality_gcnr(q.h, x, 0, None)           # no region pairs, no images: nothing to do
    kb.kk_quality_fwhm(q.h, x, 0, None)
    with pytest.raises(kb.KKError):
        kb.kk_quality_fwhm(q.h, x, -1, None)
    with pytest.raises(kb.KKError):
        kb.kk_quality_fwhm(q.h, x, 1, None)      # null output with work to do
    torch.cuda.synchronize()


def test_quality_study_runs_and_is_sane():
    """One realization of the gCNR / FWHM study of KK schemes against DAS
    (Table 1 acquisition, simulated on the GPU): every variant measured, values
    in range, DAS contrast clearly above chance."""
    from paper_2603_22496_gb300 import quality as H
    t = H.run(realizations=1, log=lambda *a: None)
    assert set(t) == {v[0] for v in H.variants()}
    for name, v in t.items():
        assert 0.0 < v["gcnr"] <= 1.0, name
        assert 0.05 < v["lateral_fwhm_mm"] < 2.0, name
        assert 0.05 < v["axial_fwhm_mm"] < 2.0, name
    assert t["DAS N=15"]["gcnr"] > 0.5
    assert t["KK j=0 M=7"]["compression"] > 27
