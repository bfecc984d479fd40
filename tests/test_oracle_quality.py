"""Pins of the image-quality oracle (gCNR and FWHM) against closed forms.

Each test names the mistake it would catch.  The gCNR definition is the
histogram overlap the paper cites for its contrast figures (Section III,
Fig. 5); FWHM is the half-amplitude width of a point response (Section III,
Fig. 4).
"""
import math

import numpy as np
import pytest

from oracle import quality as Q

GRID = (9, 7, -1.0, 0.25, 2.0, 0.25)  # nx, nz, x0, dx, z0, dz: every centre exact in binary


def _brute_mask(grid, region):
    nx, nz, x0, dx, z0, dz = grid
    kind, a, b, c, d = region
    m = np.zeros((nz, nx), dtype=bool)
    for iz in range(nz):
        for ix in range(nx):
            x = x0 + ix * dx
            z = z0 + iz * dz
            if kind == Q.REGION_RECT:
                m[iz, ix] = a <= x <= b and c <= z <= d
            else:
                r2 = (x - a) ** 2 + (z - b) ** 2
                m[iz, ix] = r2 <= c * c if kind == Q.REGION_DISK else (c * c < r2 <= d * d)
    return m


@pytest.mark.parametrize("region", [
    (Q.REGION_DISK, 0.0, 2.75, 0.5, 0.0),          # boundary pixels at exactly r are inside
    (Q.REGION_ANNULUS, 0.0, 2.75, 0.5, 0.75),      # ... and outside the annulus's inner edge
    (Q.REGION_RECT, -0.5, 0.25, 2.25, 3.0),        # closed box, edges on pixel centres
    (Q.REGION_DISK, 5.0, 5.0, 0.1, 0.0),           # empty
])
def test_region_masks_match_pointwise_definition(region):
    """Catches a half-open box, a strict disk test or a swapped x/z axis."""
    m = Q.region_mask(GRID, region)
    assert m.shape == (GRID[1], GRID[0])
    np.testing.assert_array_equal(m, _brute_mask(GRID, region))


def test_region_boundary_inclusion_exact():
    """A pixel centre at exactly distance r belongs to the disk, not to the annulus (r, R]."""
    disk = Q.region_mask(GRID, (Q.REGION_DISK, 0.0, 2.75, 0.5, 0.0))
    ann = Q.region_mask(GRID, (Q.REGION_ANNULUS, 0.0, 2.75, 0.5, 1.0))
    # centre (0, 2.75) is ix=4, iz=3; (0.5, 2.75) is ix=6
    assert disk[3, 6] and not ann[3, 6]
    assert not (disk & ann).any()


def test_envelope_exact_small_integers():
    """|3+4i| = 5 and sqrt(25) = 5 exactly; catches |B|^2 returned as the envelope."""
    e = Q.envelope_f32(np.array([3 + 4j, -5j, 0j], dtype=np.complex64))
    np.testing.assert_array_equal(e, np.array([5, 5, 0], dtype=np.float32))
    e = Q.envelope_f32(np.array([25.0, 0.0], dtype=np.float32), Q.IMG_INTENSITY)
    np.testing.assert_array_equal(e, np.array([5, 0], dtype=np.float32))


def test_gcnr_disjoint_supports_is_one():
    rng = np.random.default_rng(1)
    a = rng.uniform(0.0, 1.0, 500)
    b = rng.uniform(2.0, 3.0, 700)
    assert Q.gcnr_values(a, b, 256) == 1.0


def test_gcnr_identical_samples_is_zero():
    rng = np.random.default_rng(2)
    a = rng.rayleigh(1.0, 1000)
    assert Q.gcnr_values(a, a.copy(), 100) == 0.0
    assert Q.gcnr_values(a, a[::-1].copy(), 17) == 0.0


def test_gcnr_half_overlap_exact():
    """Integers 0..99 vs 50..149 with one integer per bin: OVL = 1/2 exactly."""
    a = np.arange(0, 100, dtype=np.float32)
    b = np.arange(50, 150, dtype=np.float32)
    assert Q.gcnr_values(a, b, 150) == 0.5


def test_gcnr_normalises_by_region_size():
    """0..99 vs 50..249: overlap sum_{50..99} min(1/100, 1/200) = 1/4, gCNR = 3/4.

    Raw counts (no division by region size) would give 1/2.
    """
    a = np.arange(0, 100, dtype=np.float32)
    b = np.arange(50, 250, dtype=np.float32)
    assert Q.gcnr_values(a, b, 250) == 0.75
    assert Q.gcnr_values(b, a, 250) == 0.75


def test_gcnr_bin_rule_edges():
    """lo goes to bin 0, hi to the last bin; a constant sample has gCNR 0."""
    v = np.array([1.0, 1.5, 2.0], dtype=np.float32)
    np.testing.assert_array_equal(Q.bin_index_f32(v, np.float32(1), np.float32(2), 4), [0, 2, 3])
    np.testing.assert_array_equal(Q.bin_index_f32(v, np.float32(1), np.float32(1), 4), [0, 0, 0])
    assert Q.gcnr_values(np.full(5, 2.0), np.full(3, 2.0), 64) == 0.0
    assert Q.gcnr_values(np.array([0.0, 1.0]), np.array([2.0, 3.0]), 1) == 0.0
    assert math.isnan(Q.gcnr_values(np.array([]), np.array([1.0]), 8))


def _rayleigh_quantiles(sigma, n):
    u = (np.arange(n) + 0.5) / n
    return sigma * np.sqrt(-2.0 * np.log1p(-u))


@pytest.mark.parametrize("s1,s2", [(1.0, 3.0), (1.0, 1.5), (0.2, 1.0)])
def test_gcnr_rayleigh_closed_form(s1, s2):
    """Two Rayleigh densities cross once at x*; gCNR = exp(-x*^2/2s2^2) - exp(-x*^2/2s1^2).

    Deterministic quantile samples (no sampling noise) and 400 bins leave only
    the histogram's discretisation error, well below 5e-3.  This is the
    speckle statistic of an anechoic-versus-background contrast measurement.
    """
    xs2 = 2.0 * math.log(s2 ** 2 / s1 ** 2) / (1.0 / s1 ** 2 - 1.0 / s2 ** 2)
    exact = math.exp(-xs2 / (2 * s2 ** 2)) - math.exp(-xs2 / (2 * s1 ** 2))
    est = Q.gcnr_values(_rayleigh_quantiles(s1, 200_000), _rayleigh_quantiles(s2, 300_000), 400)
    assert abs(est - exact) < 5e-3, (est, exact)


def test_gcnr_power_of_two_scale_invariance():
    """Scaling the image by 2^k scales lo, hi and every value exactly: identical bins."""
    rng = np.random.default_rng(3)
    a = rng.rayleigh(1.0, 3000).astype(np.float32)
    b = rng.rayleigh(2.0, 2000).astype(np.float32)
    g = Q.gcnr_values(a, b, 128)
    assert Q.gcnr_values(a * np.float32(8), b * np.float32(8), 128) == g
    assert 0.0 < g < 1.0


def test_gcnr_image_regions():
    """Dark disk of constant 1 inside an annulus of constant 3: gCNR 1; swap levels: still 1."""
    nx, nz = 33, 33
    grid = (nx, nz, -8e-3, 0.5e-3, 2e-3, 0.5e-3)
    inside = (Q.REGION_DISK, 0.0, 10e-3, 3e-3, 0.0)
    outside = (Q.REGION_ANNULUS, 0.0, 10e-3, 4e-3, 6e-3)
    img = np.full((nz, nx), 3.0, dtype=np.complex64)
    img[Q.region_mask(grid, inside)] = 1.0j
    assert Q.gcnr(img, grid, inside, outside, 64) == 1.0
    # pixels between the regions carry another value and must not enter either histogram
    ring = ~(Q.region_mask(grid, inside) | Q.region_mask(grid, outside))
    img[ring] = 100.0
    assert Q.gcnr(img, grid, inside, outside, 64) == 1.0
    # intensity input of the same envelope gives the same answer
    inten = (np.abs(img) ** 2).astype(np.float32)
    assert Q.gcnr(inten, grid, inside, outside, 64, kind=Q.IMG_INTENSITY) == 1.0


def _tri(n, c, a, dx):
    x = (np.arange(n) - c) * dx
    return np.maximum(0.0, 1.0 - np.abs(x) / a)


def test_fwhm_triangle_exact():
    """Separable triangle: linear interpolation is exact, widths a_x and a_z."""
    nx, nz, dx, dz = 64, 48, 0.1e-3, 0.05e-3
    grid = (nx, nz, -3.2e-3, dx, 1e-3, dz)
    ax_, az_ = 1.3e-3, 0.7e-3
    env = np.outer(_tri(nz, 20, az_, dz), _tri(nx, 30, ax_, dx)).astype(np.float32)
    r = Q.fwhm(env.astype(np.complex64), grid, (31, 21, 5, 5))
    assert (r["ix"], r["iz"]) == (30, 20)
    assert r["peak"] == 1.0
    assert abs(r["lateral"] - ax_) < 1e-9
    assert abs(r["axial"] - az_) < 1e-9


def test_fwhm_gaussian_closed_form():
    """Gaussian envelope of std s: FWHM = 2 s sqrt(2 ln 2) (interp error O((dx/s)^2))."""
    nx, nz, dx = 401, 3, 1e-5
    s = 25 * dx
    x = (np.arange(nx) - 200) * dx
    env = np.exp(-x ** 2 / (2 * s * s))
    img = np.tile(env, (nz, 1)).astype(np.complex64) * np.exp(0.7j).astype(np.complex64)
    img[0] *= 0.5
    img[2] *= 0.5
    r = Q.fwhm(img, (nx, nz, -200 * dx, dx, 0.0, dx), (200, 1, 10, 1))
    assert (r["ix"], r["iz"]) == (200, 1)
    assert abs(r["lateral"] / (2 * s * math.sqrt(2 * math.log(2))) - 1) < 1e-3
    assert math.isnan(r["axial"])   # the column never falls below half within the image


def test_fwhm_translation_and_ties():
    """Integer shift moves the peak, not the width; equal maxima pick the first row-major."""
    nx, nz, dx = 80, 40, 0.1e-3
    grid = (nx, nz, 0.0, dx, 0.0, dx)
    env = np.outer(_tri(nz, 12, 0.6e-3, dx), _tri(nx, 20, 0.9e-3, dx))
    r0 = Q.fwhm(env.astype(np.complex64), grid, (20, 12, 4, 4))
    env2 = np.roll(np.roll(env, 7, axis=1), 5, axis=0)
    r1 = Q.fwhm(env2.astype(np.complex64), grid, (27, 17, 4, 4))
    assert (r1["ix"], r1["iz"]) == (27, 17)
    assert abs(r1["lateral"] - r0["lateral"]) < 1e-12 and abs(r1["axial"] - r0["axial"]) < 1e-12
    flat = np.zeros((nz, nx), dtype=np.complex64)
    flat[10, 30] = flat[10, 20] = flat[11, 5] = 2.0
    r = Q.fwhm(flat, grid, (20, 10, 15, 3))
    assert (r["ix"], r["iz"]) == (20, 10)      # row 10 before row 11; x=20 before x=30


def test_fwhm_window_clipping_and_empty():
    nx, nz, dx = 16, 16, 1e-4
    grid = (nx, nz, 0.0, dx, 0.0, dx)
    env = np.outer(_tri(nz, 3, 4e-4, dx), _tri(nx, 0, 4e-4, dx))
    r = Q.fwhm(env.astype(np.complex64), grid, (0, 0, 3, 3))    # window clipped at the corner
    assert (r["ix"], r["iz"]) == (0, 3)
    assert math.isnan(r["lateral"])                             # left side runs off the image
    assert abs(r["axial"] - 4e-4) < 1e-12
    r = Q.fwhm(env.astype(np.complex64), grid, (40, 40, 2, 2))  # window outside the image
    assert r["ix"] == -1 and math.isnan(r["peak"])
