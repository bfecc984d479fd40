"""FP64 oracle of volumetric KK beamforming with a 2D (matrix) array.

TEST INFRASTRUCTURE -- not part of the product (see ``oracle/__init__``).

Section IV of the paper names 2D arrays and volumetric imaging as the setting
where the decomposition pays most; the method carries over unchanged with
plane waves in three dimensions.  Written out here:

* a plane wave with tilt angles (ax, ay) travels along the unit vector
  ``s = (sin ax, sin ay, sqrt(1 - sin^2 ax - sin^2 ay))`` and passes the origin
  at t = 0 (for ay = 0 this is the linear-array wave (sin ax, cos ax));
* Eq. (compression): receive wave o shears element l = (u_l, v_l) by
  ``delta_l(o) = ((xr_o - u_l) sx_o + (yr_o - v_l) sy_o) / c``, where
  ``xr_o`` (``yr_o``) is the array edge along x (y) that makes both terms
  non-negative advances (the linear-array rule applied per axis), applied by
  the Fourier shift theorem on the analytic spectrum as in ``oracle.kk``;
* Eq. (KK): ``B_j(r) = sum_{p in G_j} lerp(y_p, fs (tau_in + tau_out))`` with
  ``tau_in = s_i . r / c`` and
  ``tau_out = ((x - xr_o) sx_o + (y - yr_o) sy_o + z sz_o) / c``;
* Eq. (DAS): ``sum_{i,l} lerp(y_il, fs (s_i . r + |r - e_l|) / c)``.

Angle sets are products of the linear schemes (Section II-C/D) along x and y,
so the 2D coarray is the product of the two 1D coarrays.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import kk as _kk
from . import schemes as _schemes


def directions(ax, ay):
    """Unit propagation vectors (sx, sy, sz) of tilt angles (ax, ay)."""
    sx = np.sin(np.asarray(ax, dtype=np.float64))
    sy = np.sin(np.asarray(ay, dtype=np.float64))
    q = 1.0 - sx * sx - sy * sy
    if np.any(q <= 0):
        raise ValueError("tilt angles beyond the propagating range")
    return sx, sy, np.sqrt(q)


@dataclasses.dataclass
class PairSet3:
    """P pairs (transmit, receive) of a volumetric scheme in J groups."""
    tx_ax: np.ndarray
    tx_ay: np.ndarray
    rx_ax: np.ndarray
    rx_ay: np.ndarray
    tx_index: np.ndarray
    rx_index: np.ndarray
    group: np.ndarray
    n_groups: int

    @property
    def n_pairs(self) -> int:
        return int(self.tx_index.shape[0])


def product_set(tx_ax, tx_ay, rx_groups, tx_subset=None) -> PairSet3:
    """Every used transmit with every receive wave of each group.

    ``rx_groups``: list of (rx_ax, rx_ay) arrays, one per group."""
    tx_ax = np.asarray(tx_ax, dtype=np.float64)
    tx_ay = np.asarray(tx_ay, dtype=np.float64)
    sub = np.arange(tx_ax.shape[0]) if tx_subset is None else np.asarray(tx_subset)
    bx, by, ti, ri, gp = [], [], [], [], []
    base = 0
    for g, (rax, ray) in enumerate(rx_groups):
        rax = np.asarray(rax, dtype=np.float64)
        ray = np.asarray(ray, dtype=np.float64)
        for i in sub:
            for o in range(rax.shape[0]):
                ti.append(int(i))
                ri.append(base + o)
                gp.append(g)
        bx.append(rax)
        by.append(ray)
        base += rax.shape[0]
    return PairSet3(tx_ax, tx_ay, np.concatenate(bx), np.concatenate(by), np.array(ti, np.int64),
                    np.array(ri, np.int64), np.array(gp, np.int64), len(rx_groups))


def separable_scheme(kind: str, tx_x_1d, tx_y_1d, Mx: int, My: int, jx: float = 0, jy: float = 0):
    """Receive tilts of a 1D scheme along x times one along y (product grid,
    index o = oy * Mx + ox), from the linear schemes of ``oracle.schemes``."""
    def one(tx, M, j):
        tx = np.asarray(tx, dtype=np.float64)
        if tx.shape[0] == 1 or M == 1:
            return np.zeros(M)
        return _schemes.scheme(kind, tx, M, j=j).rx_angles
    rx = one(tx_x_1d, Mx, jx)
    ry = one(tx_y_1d, My, jy)
    return np.tile(rx, My), np.repeat(ry, Mx)


def shear_reference3(elem_x, elem_y, rx_ax, rx_ay):
    """(xr_o, yr_o): per axis the array edge that keeps the shear an advance."""
    u = np.asarray(elem_x, dtype=np.float64)
    v = np.asarray(elem_y, dtype=np.float64)
    sx, sy, _ = directions(rx_ax, rx_ay)
    xr = np.where(sx > 0, u.max(), np.where(sx < 0, u.min(), 0.0))
    yr = np.where(sy > 0, v.max(), np.where(sy < 0, v.min(), 0.0))
    return xr, yr


def shear_delays3(elem_x, elem_y, rx_ax, rx_ay, c: float) -> np.ndarray:
    """delta_l(o) in seconds, [M][L]."""
    u = np.asarray(elem_x, dtype=np.float64)
    v = np.asarray(elem_y, dtype=np.float64)
    sx, sy, _ = directions(rx_ax, rx_ay)
    xr, yr = shear_reference3(u, v, rx_ax, rx_ay)
    return ((xr[:, None] - u[None, :]) * sx[:, None] + (yr[:, None] - v[None, :]) * sy[:, None]) / c


def decompose3(rf, elem_x, elem_y, ps: PairSet3, fs: float, c: float) -> np.ndarray:
    """RF_theta of every pair, y[P][T] complex128 (Eq. (compression) per bin)."""
    T = rf.shape[-1]
    F = T // 2
    tx_used = np.unique(ps.tx_index)
    rx_used = np.unique(ps.rx_index)
    X = _kk.analytic_spectrum(np.asarray(rf, dtype=np.float64)[tx_used])        # [Nu][L][F]
    d = shear_delays3(elem_x, elem_y, ps.rx_ax[rx_used], ps.rx_ay[rx_used], c)  # [Mu][L]
    k = np.arange(F, dtype=np.float64)
    W = np.exp(2j * np.pi * k[None, None, :] * (fs * d)[:, :, None] / T)       # [Mu][L][F]
    Yk = np.matmul(np.transpose(X, (2, 0, 1)), np.transpose(W, (2, 1, 0)))      # [F][Nu][Mu]
    ti = np.searchsorted(tx_used, ps.tx_index)
    ri = np.searchsorted(rx_used, ps.rx_index)
    return _kk.inverse_half_spectrum(Yk[:, ti, ri].T, T)


def voxel_coords(grid, grid_y, voxels=None):
    """(x, y, z) of the whole volume in [y][z][x] order, or of listed (ix, iy, iz)."""
    nx, nz, x0, dx, z0, dz = grid
    ny, y0, dy = grid_y
    if voxels is None:
        iy, iz, ix = np.meshgrid(np.arange(ny), np.arange(nz), np.arange(nx), indexing="ij")
        ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    else:
        v = np.asarray(voxels, dtype=np.int64).reshape(-1, 3)
        ix, iy, iz = v[:, 0], v[:, 1], v[:, 2]
    return (x0 + dx * ix.astype(np.float64), y0 + dy * iy.astype(np.float64),
            z0 + dz * iz.astype(np.float64))


def kk_beamform3(y, elem_x, elem_y, ps: PairSet3, grid, grid_y, fs: float, c: float, voxels=None):
    """B[J][ny][nz][nx] (or B[J][n_vox] for a voxel list), complex128, Eq. (KK)."""
    lib = _kk._load()
    P, T = y.shape
    yc = np.ascontiguousarray(y, dtype=np.complex128)
    sxi, syi, szi = (np.ascontiguousarray(a) for a in directions(ps.tx_ax[ps.tx_index], ps.tx_ay[ps.tx_index]))
    sxo, syo, szo = (np.ascontiguousarray(a) for a in directions(ps.rx_ax[ps.rx_index], ps.rx_ay[ps.rx_index]))
    xr, yr = (np.ascontiguousarray(a) for a in
              shear_reference3(elem_x, elem_y, ps.rx_ax[ps.rx_index], ps.rx_ay[ps.rx_index]))
    grp = np.ascontiguousarray(ps.group, dtype=np.int32)
    px, py, pz = (np.ascontiguousarray(a) for a in voxel_coords(grid, grid_y, voxels))
    n = px.shape[0]
    B = np.zeros((ps.n_groups, n), dtype=np.complex128)
    d = _kk._d
    rc = lib.orc_kk_beamform_vol(P, T, d(yc.view(np.float64)), d(sxi), d(syi), d(szi), d(sxo), d(syo),
                                 d(szo), d(xr), d(yr), _kk._i(grp), ps.n_groups, n, d(px), d(py), d(pz),
                                 float(fs), float(c), d(B.view(np.float64)))
    if rc:
        raise RuntimeError(f"orc_kk_beamform_vol: {rc}")
    if voxels is None:
        nx, nz = grid[0], grid[1]
        return B.reshape(ps.n_groups, grid_y[0], nz, nx)
    return B


def kk_volume(rf, elem_x, elem_y, ps: PairSet3, grid, grid_y, fs, c, voxels=None):
    return kk_beamform3(decompose3(rf, elem_x, elem_y, ps, fs, c), elem_x, elem_y, ps, grid, grid_y,
                        fs, c, voxels)


def das_volume(rf, tx_ax, tx_ay, elem_x, elem_y, grid, grid_y, fs, c, voxels=None):
    """B[ny][nz][nx] (or [n_vox]) complex128, Eq. (DAS) with a 2D array."""
    lib = _kk._load()
    y = np.ascontiguousarray(_kk.analytic_signal(rf), dtype=np.complex128)
    N, L, T = y.shape
    sxi, syi, szi = (np.ascontiguousarray(a) for a in directions(tx_ax, tx_ay))
    ex = np.ascontiguousarray(elem_x, dtype=np.float64)
    ey = np.ascontiguousarray(elem_y, dtype=np.float64)
    px, py, pz = (np.ascontiguousarray(a) for a in voxel_coords(grid, grid_y, voxels))
    n = px.shape[0]
    B = np.zeros(n, dtype=np.complex128)
    d = _kk._d
    rc = lib.orc_das_beamform_vol(N, L, T, d(y.view(np.float64)), d(sxi), d(syi), d(szi), d(ex), d(ey),
                                  n, d(px), d(py), d(pz), float(fs), float(c), d(B.view(np.float64)))
    if rc:
        raise RuntimeError(f"orc_das_beamform_vol: {rc}")
    if voxels is None:
        nx, nz = grid[0], grid[1]
        return B.reshape(grid_y[0], nz, nx)
    return B
