"""Pins of the oracle's apodization (the paper states Eqs. (DAS) and (KK)
without apodization factors and notes they fold in directly; Table 1 gives
the F-numbers of its acquisitions): per-pair weights in Eq. (KK), a receive
aperture of half-width z / (2 F) in Eq. (DAS), boxcar or Hann."""
import dataclasses

import numpy as np
import pytest

import kksynth
from oracle import kk, schemes

FS, C = kksynth.FS, kksynth.C_SOUND


@pytest.fixture(scope="module")
def small():
    w = kksynth.workload_small(speckle=200)
    ps = schemes.scheme("confocal", w.tx_angles, 7)
    grid = (20, 12, -2e-3, 0.2e-3, 8e-3, 0.25e-3)
    y = kk.decompose(w.rf, w.elem_x, ps, FS, C)
    return w, ps, grid, y


def test_unit_pair_weights_change_nothing(small):
    w, ps, grid, y = small
    a = kk.kk_beamform(y, w.elem_x, ps, grid, FS, C)
    b = kk.kk_beamform(y, w.elem_x, ps, grid, FS, C, weights=np.ones(ps.n_pairs))
    assert np.array_equal(a, b)


def test_pair_weights_are_linear(small):
    w, ps, grid, y = small
    r = np.random.default_rng(1)
    w1, w2 = r.standard_normal(ps.n_pairs), r.standard_normal(ps.n_pairs)
    B = lambda wt: kk.kk_beamform(y, w.elem_x, ps, grid, FS, C, weights=wt)
    assert np.allclose(B(w1 + w2), B(w1) + B(w2), rtol=1e-12, atol=1e-12 * np.abs(B(w1)).max())
    assert np.allclose(B(2.5 * w1), 2.5 * B(w1), rtol=1e-12, atol=0)


def test_zero_weights_remove_those_pairs(small):
    w, ps, grid, y = small
    keep = np.arange(ps.n_pairs) % 3 != 0
    wt = keep.astype(float)
    sub = dataclasses.replace(ps, tx_index=ps.tx_index[keep], rx_index=ps.rx_index[keep],
                              group=ps.group[keep])
    a = kk.kk_beamform(y, w.elem_x, ps, grid, FS, C, weights=wt)
    b = kk.kk_beamform(y[keep], w.elem_x, sub, grid, FS, C)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(b).max())


def test_full_aperture_is_plain_das(small):
    w = small[0]
    grid = small[2]
    a = kk.das_image(w.rf, w.tx_angles, w.elem_x, grid, FS, C)
    b = kk.das_image(w.rf, w.tx_angles, w.elem_x, grid, FS, C, f_number=0.0)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("F", [0.8, 1.7])
def test_boxcar_aperture_is_das_over_the_elements_inside(small, F):
    """At each pixel the boxcar aperture equals plain DAS over just the
    elements within z / (2F) of it."""
    w = small[0]
    ya = kk.analytic_signal(w.rf)
    pix = np.array([[3, 2], [10, 7], [17, 11], [0, 0]])
    nx, nz, x0, dx, z0, dz = small[2]
    B = kk.das_beamform_analytic(ya, w.tx_angles, w.elem_x, small[2], FS, C, pixels=pix, f_number=F)
    for q, (ix, iz) in enumerate(pix):
        x, z = x0 + dx * ix, z0 + dz * iz
        inside = np.abs(x - w.elem_x) <= z / (2 * F)
        assert 0 < inside.sum() < w.n_elem
        ref = kk.das_beamform_analytic(ya[:, inside], w.tx_angles, w.elem_x[inside], small[2], FS, C,
                                       pixels=pix[q:q + 1])
        assert np.allclose(B[q], ref[0], rtol=1e-12, atol=1e-12 * abs(ref[0]))


def test_hann_aperture_values_at_centre_half_width_and_edge():
    """With constant channel data every element contributes N x its weight:
    Hann gives 1 at the aperture centre, 1/2 at half the half-width, 0 at the
    edge and beyond."""
    F, z, N, T = 1.0, 4e-3, 3, 4096
    h = z / (2 * F)
    x = 0.0
    offsets = np.array([0.0, 0.5 * h, h, 1.25 * h])
    tx = np.deg2rad(np.array([-5.0, 0.0, 5.0]))
    y = np.ones((N, 1, T), complex)
    vals = []
    for d in offsets:
        B = kk.das_beamform_analytic(y, tx, np.array([x + d]), (1, 1, x, 1e-4, z, 1e-4), FS, C,
                                     pixels=np.array([[0, 0]]), f_number=F, window="hann")
        vals.append(B[0].real / N)
    assert np.allclose(vals, [1.0, 0.5, 0.0, 0.0], atol=1e-12)
    # boxcar: 1 up to and including the edge, 0 beyond
    vals = [kk.das_beamform_analytic(y, tx, np.array([x + d]), (1, 1, x, 1e-4, z, 1e-4), FS, C,
                                     pixels=np.array([[0, 0]]), f_number=F)[0].real / N for d in offsets]
    assert np.allclose(vals, [1.0, 1.0, 1.0, 0.0], atol=1e-12)
