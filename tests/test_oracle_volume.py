"""Pins of the volumetric (2D-array) KK oracle.

V1 ties the whole volumetric path to the pinned linear-array oracle: a
linear array, tilts without a y component and one y-slice at y = 0 must give
the linear-array result.  V2 ties the y axis to the x axis: transposing the
problem (array, tilts, phantom, grid) must transpose the volume.  V3 and V5
are physics (focus at the scatterers; full-pair KK close to DAS), V4 brute
force on a tiny case.  V6 pins the per-axis split of the shear on a grid
array with a product receive set, which the separable GPU contraction uses.
"""
import cmath
import math

import numpy as np
import pytest

import kksynth
from oracle import kk, schemes, volume as V

FS, C = kksynth.FS, kksynth.C_SOUND


def test_forward_model_reduces_to_linear_array():
    """Input check: the matrix-array simulator with v = 0, ay = 0, y = 0 is
    the linear-array simulator."""
    u = kksynth.element_positions(16, 0.3e-3)
    ax = np.deg2rad(np.array([-6.0, 0.0, 5.0]))
    pts = np.array([[1e-3, 0.0, 6e-3, 2.0], [-2e-3, 0.0, 9e-3, -1.0]])
    r3 = kksynth.simulate_rf3(pts, u, np.zeros_like(u), ax, np.zeros_like(ax), 512)
    r2 = kksynth.simulate_rf(kksynth.Phantom(pts[:, 0], pts[:, 2], pts[:, 3]), u, ax, 512)
    assert np.abs(r3 - r2).max() <= 1e-12 * np.abs(r2).max()


def test_v1_linear_array_reduction():
    """elem_y = 0, zero y tilts, one slice at y = 0: identical to oracle.kk
    (catches any x/z mix-up or dropped term of the volumetric path)."""
    w = kksynth.workload_small()
    ops = schemes.scheme("confocal", w.tx_angles, 11)
    zeros_t = np.zeros_like(w.tx_angles)
    ps3 = V.product_set(w.tx_angles, zeros_t, [(ops.rx_angles, np.zeros_like(ops.rx_angles))])
    assert np.array_equal(ps3.tx_index, ops.tx_index) and np.array_equal(ps3.rx_index, ops.rx_index)
    ey = np.zeros_like(w.elem_x)
    y3 = V.decompose3(w.rf, w.elem_x, ey, ps3, FS, C)
    y2 = kk.decompose(w.rf, w.elem_x, ops, FS, C)
    assert kk.rel_l2(y3, y2) <= 1e-12
    grid = (40, 36, -4e-3, 0.2e-3, 6e-3, 0.25e-3)
    B3 = V.kk_beamform3(y2, w.elem_x, ey, ps3, grid, (1, 0.0, 1e-4), FS, C)
    B2 = kk.kk_beamform(y2, w.elem_x, ops, grid, FS, C)
    assert B3.shape == (1, 1, 36, 40)
    assert kk.rel_l2(B3[:, 0], B2) <= 1e-12


def _small_matrix(lx, ly, px, py, tilts_x, tilts_y):
    u, v = kksynth.matrix_elements(lx, ly, px, py)
    ax = np.tile(tilts_x, len(tilts_y))
    ay = np.repeat(tilts_y, len(tilts_x))
    return u, v, ax, ay


def test_v2_transposition_symmetry():
    """Swapping the x and y axes of everything transposes the volume (pins the
    y path, including its shear reference, against the x path)."""
    tx_x = np.deg2rad([-4.0, 0.0, 4.0])
    tx_y = np.deg2rad([-3.0, 3.0])
    u, v, ax, ay = _small_matrix(6, 4, 0.3e-3, 0.25e-3, tx_x, tx_y)
    pts = np.array([[0.4e-3, -0.3e-3, 4e-3, 3.0], [-0.5e-3, 0.2e-3, 5e-3, -2.0]])
    T = 256
    rf = kksynth.simulate_rf3(pts, u, v, ax, ay, T)
    rxx, rxy = V.separable_scheme("shifted", tx_x, tx_y, 3, 2, jx=1, jy=0.5)
    ps = V.product_set(ax, ay, [(rxx, rxy)])
    grid, gy = (7, 6, -0.6e-3, 0.2e-3, 3.8e-3, 0.3e-3), (5, -0.4e-3, 0.2e-3)
    B = V.kk_volume(rf, u, v, ps, grid, gy, FS, C)[0]            # [ny][nz][nx]
    # transposed problem: element (x, y) -> (y, x), tilts swapped, phantom swapped
    rf_t = kksynth.simulate_rf3(pts[:, [1, 0, 2, 3]], v, u, ay, ax, T)
    ps_t = V.product_set(ay, ax, [(rxy, rxx)])
    grid_t, gy_t = (5, 6, -0.4e-3, 0.2e-3, 3.8e-3, 0.3e-3), (7, -0.6e-3, 0.2e-3)
    Bt = V.kk_volume(rf_t, v, u, ps_t, grid_t, gy_t, FS, C)[0]   # [nx][nz][ny]
    assert kk.rel_l2(np.transpose(Bt, (2, 1, 0)), B) <= 1e-11
    assert np.abs(B).max() > 0


def test_v3_point_focus():
    """Isolated points focus within one voxel of their positions."""
    tx1 = np.deg2rad(np.linspace(-6, 6, 3))
    u, v, ax, ay = _small_matrix(12, 12, 0.3e-3, 0.3e-3, tx1, tx1)
    targets = [(0.0, 0.0, 7e-3), (-1.2e-3, 0.9e-3, 8e-3)]
    pts = np.array([[x, y, z, 10.0] for x, y, z in targets])
    rf = kksynth.simulate_rf3(pts, u, v, ax, ay, 512)
    rx1 = schemes.even_receive_set(np.deg2rad(12.0), 7)
    rxx, rxy = np.tile(rx1, 7), np.repeat(rx1, 7)
    ps = V.product_set(ax, ay, [(rxx, rxy)])
    d = 0.15e-3
    grid, gy = (31, 31, -2.25e-3, d, 5.75e-3, d), (31, -2.25e-3, d)
    B = np.abs(V.kk_volume(rf, u, v, ps, grid, gy, FS, C)[0])
    for x, y, z in targets:
        ix, iy, iz = round((x + 2.25e-3) / d), round((y + 2.25e-3) / d), round((z - 5.75e-3) / d)
        win = B[max(iy - 4, 0):iy + 5, max(iz - 4, 0):iz + 5, max(ix - 4, 0):ix + 5]
        jy, jz, jx = np.unravel_index(np.argmax(win), win.shape)
        assert abs(jy + max(iy - 4, 0) - iy) <= 1 and abs(jz + max(iz - 4, 0) - iz) <= 1 \
            and abs(jx + max(ix - 4, 0) - ix) <= 1
        assert win.max() > 0.5 * B.max()


def _brute(rf, u, v, ax, ay, bx, by, pairs, vox, fs, c):
    """Pure-Python direct DFT and loops (no numpy FFT, no C)."""
    N, L, T = len(rf), len(rf[0]), len(rf[0][0])
    F = T // 2

    def dirv(a, b):
        sx, sy = math.sin(a), math.sin(b)
        return sx, sy, math.sqrt(1 - sx * sx - sy * sy)

    umax, umin, vmax, vmin = max(u), min(u), max(v), min(v)
    out = [0j] * len(vox)
    for (i, o) in pairs:
        sxo, syo, szo = dirv(bx[o], by[o])
        xr = umax if sxo > 0 else (umin if sxo < 0 else 0.0)
        yr = vmax if syo > 0 else (vmin if syo < 0 else 0.0)
        Y = [0j] * F
        for l in range(L):
            dl = ((xr - u[l]) * sxo + (yr - v[l]) * syo) / c
            for k in range(F):
                X = sum(rf[i][l][t] * cmath.exp(-2j * math.pi * k * t / T) for t in range(T))
                X *= 1.0 if k == 0 else 2.0
                Y[k] += X * cmath.exp(2j * math.pi * k * fs * dl / T)
        y = [sum(Y[k] * cmath.exp(2j * math.pi * k * t / T) for k in range(F)) / T for t in range(T)]
        sxi, syi, szi = dirv(ax[i], ay[i])
        for q, (x, yy, z) in enumerate(vox):
            s = fs * ((x * sxi + yy * syi + z * szi) + ((x - xr) * sxo + (yy - yr) * syo + z * szo)) / c
            k0 = math.floor(s)
            if 0 <= k0 and k0 + 1 <= T - 1:
                f = s - k0
                out[q] += (1 - f) * y[k0] + f * y[k0 + 1]
    return out


def test_v4_brute_force_tiny():
    rng = np.random.default_rng(4)
    u, v = kksynth.matrix_elements(2, 2, 0.3e-3, 0.3e-3)
    ax, ay = np.deg2rad([-5.0, 4.0]), np.deg2rad([3.0, -2.0])
    T = 32
    rf = rng.standard_normal((2, 4, T))
    bx, by = np.deg2rad([-7.0, 6.0]), np.deg2rad([2.0, -4.0])
    ps = V.product_set(ax, ay, [(bx, by)])
    grid, gy = (3, 3, -0.15e-3, 0.15e-3, 0.2e-3, 0.1e-3), (3, -0.1e-3, 0.1e-3)
    got = V.kk_volume(rf, u, v, ps, grid, gy, FS, C)[0].ravel()
    x, y, z = V.voxel_coords(grid, gy)
    pairs = list(zip(ps.tx_index.tolist(), ps.rx_index.tolist()))
    want = np.array(_brute(rf.tolist(), u.tolist(), v.tolist(), ax.tolist(), ay.tolist(), bx.tolist(),
                           by.tolist(), pairs, list(zip(x, y, z)), FS, C))
    assert np.abs(want).max() > 0
    assert kk.rel_l2(got, want) <= 1e-12


def test_v5_full_pairs_approximate_das():
    """Many receive waves spanning the aperture: the KK volume of a point is
    close to the DAS volume (the paper's KK ~ DAS statement, Section II-B)."""
    tx1 = np.deg2rad(np.linspace(-5, 5, 3))
    u, v, ax, ay = _small_matrix(16, 16, 0.3e-3, 0.3e-3, tx1, tx1)
    pts = np.array([[0.0, 0.0, 6e-3, 10.0]])
    rf = kksynth.simulate_rf3(pts, u, v, ax, ay, 512)
    rx1 = schemes.even_receive_set(np.deg2rad(22.0), 15)
    ps = V.product_set(ax, ay, [(np.tile(rx1, 15), np.repeat(rx1, 15))])
    d = 0.1e-3
    grid, gy = (21, 21, -1e-3, d, 5e-3, d), (21, -1e-3, d)
    Bk = np.abs(V.kk_volume(rf, u, v, ps, grid, gy, FS, C)[0])
    Bd = np.abs(V.das_volume(rf, ax, ay, u, v, grid, gy, FS, C))
    corr = float(np.sum(Bk * Bd) / np.sqrt(np.sum(Bk ** 2) * np.sum(Bd ** 2)))
    assert corr >= 0.9, corr
    assert np.unravel_index(np.argmax(Bk), Bk.shape) == np.unravel_index(np.argmax(Bd), Bd.shape)


def test_v6_shear_separates_per_axis_on_a_grid():
    """Reading R28 on the oracle's own definition: for elements on an x-y grid
    and receive waves on a product of x and y tilts, delta_l(o) is the sum of
    an x term (ox, lx) and a y term (oy, ly), so the per-bin phasor matrix is
    the Kronecker product of two per-axis matrices and the element sum can
    run as two per-axis contractions (the separable GPU form)."""
    lx, ly = 6, 4
    u, v = kksynth.matrix_elements(lx, ly, 0.3e-3, 0.25e-3)
    ax1 = np.deg2rad([-11.0, -3.0, 0.0, 7.0, 12.0])
    ay1 = np.deg2rad([-9.0, 0.0, 5.0])
    rxx, rxy = np.tile(ax1, ay1.shape[0]), np.repeat(ay1, ax1.shape[0])   # o = oy * Mx + ox
    d = V.shear_delays3(u, v, rxx, rxy, C)                                  # [M][L], l = ly * Lx + lx
    sx, sy = np.sin(ax1), np.sin(ay1)
    xr = np.where(sx > 0, u.max(), np.where(sx < 0, u.min(), 0.0))
    yr = np.where(sy > 0, v.max(), np.where(sy < 0, v.min(), 0.0))
    ux, vy = u[:lx], v[::lx]
    dx = (xr[:, None] - ux[None, :]) * sx[:, None] / C                     # [Mx][Lx]
    dy = (yr[:, None] - vy[None, :]) * sy[:, None] / C                     # [My][Ly]
    sep = dy[:, None, :, None] + dx[None, :, None, :]                      # [My][Mx][Ly][Lx]
    assert np.abs(sep.reshape(d.shape) - d).max() <= 1e-18
    # the two-step contraction equals the full one on random spectra
    rng = np.random.default_rng(6)
    T, k = 256, 37
    X = rng.standard_normal((3, ly * lx)) + 1j * rng.standard_normal((3, ly * lx))
    W = np.exp(2j * np.pi * k * FS * d / T)
    Wx = np.exp(2j * np.pi * k * FS * dx / T)
    Wy = np.exp(2j * np.pi * k * FS * dy / T)
    Z = np.einsum("iyx,ax->iya", X.reshape(3, ly, lx), Wx)                 # sum over lx
    Y2 = np.einsum("iya,by->iba", Z, Wy).reshape(3, -1)                    # sum over ly
    assert kk.rel_l2(Y2, X @ W.T) <= 1e-13


def test_v7_das_volume_focus_and_transposition():
    """The volumetric DAS oracle: isolated points off both axes focus within
    one voxel of their positions (a wrong sign or a dropped y term in either
    delay moves or smears them), and swapping x and y everywhere transposes
    the volume (pins its y path against its x path)."""
    tx1 = np.deg2rad(np.linspace(-6, 6, 3))
    u, v, ax, ay = _small_matrix(10, 8, 0.3e-3, 0.25e-3, tx1, tx1[:2])
    targets = [(0.9e-3, -0.6e-3, 6.5e-3), (-1.2e-3, 0.9e-3, 7.5e-3)]
    pts = np.array([[x, y, z, 10.0] for x, y, z in targets])
    rf = kksynth.simulate_rf3(pts, u, v, ax, ay, 512)
    d = 0.15e-3
    grid, gy = (25, 21, -1.8e-3, d, 5.5e-3, d), (21, -1.5e-3, d)
    B = np.abs(V.das_volume(rf, ax, ay, u, v, grid, gy, FS, C))       # [ny][nz][nx]
    for x, y, z in targets:
        ix, iy, iz = round((x + 1.8e-3) / d), round((y + 1.5e-3) / d), round((z - 5.5e-3) / d)
        win = B[iy - 3:iy + 4, iz - 3:iz + 4, ix - 3:ix + 4]
        jy, jz, jx = np.unravel_index(np.argmax(win), win.shape)
        assert max(abs(jy - 3), abs(jz - 3), abs(jx - 3)) <= 1, (jy, jz, jx)
    # transposition
    rf_t = kksynth.simulate_rf3(pts[:, [1, 0, 2, 3]], v, u, ay, ax, 512)
    grid_t, gy_t = (21, 21, -1.5e-3, d, 5.5e-3, d), (25, -1.8e-3, d)
    Bt = np.abs(V.das_volume(rf_t, ay, ax, v, u, grid_t, gy_t, FS, C))  # [nx][nz][ny]
    assert kk.rel_l2(np.transpose(Bt, (2, 1, 0)), B) <= 1e-11
