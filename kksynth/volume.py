"""Matrix-array (2D) geometry, volumetric phantoms and their channel data
(input generation only).

Conventions, extending the linear-array ones of ``kksynth.phantom``:

* element (lx, ly) of an Lx x Ly array sits at
  ``u = (lx - (Lx-1)/2) * pitch_x``, ``v = (ly - (Ly-1)/2) * pitch_y``, z = 0,
  element index ``l = ly * Lx + lx``;
* a plane wave with tilt angles (ax, ay) travels along
  ``(sin ax, sin ay, sqrt(1 - sin^2 ax - sin^2 ay))`` and passes the origin
  at t = 0; transmit tilts form an even Nx x Ny product grid over
  ``[-theta_max, theta_max]^2``, index ``i = iy * Nx + ix``;
* voxel (ix, iy, iz) sits at ``(x0 + ix dx, y0 + iy dy, z0 + iz dz)``.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .phantom import (C_SOUND, FS, F0, BW, _dp, _load, pulse_alpha, pulse_half_window,
                      add_noise_and_quantise)


@dataclasses.dataclass
class Volume:
    """One frame of synthetic matrix-array channel data plus its voxel grid."""
    name: str
    seed: int
    elem_x: np.ndarray          # [L]
    elem_y: np.ndarray          # [L]
    tx_ax: np.ndarray           # [N] tilt about the y axis (x component)
    tx_ay: np.ndarray           # [N]
    n_samples: int
    fs: float
    c: float
    grid: tuple                 # (nx, nz, x0, dx, z0, dz)
    grid_y: tuple               # (ny, y0, dy)
    rf: np.ndarray              # [N][L][T]
    points: np.ndarray          # [n][4] scatterers (x, y, z, amp); bright targets first
    n_points: int = 0

    @property
    def n_elem(self) -> int:
        return int(self.elem_x.shape[0])

    @property
    def n_tx(self) -> int:
        return int(self.tx_ax.shape[0])


def matrix_elements(lx: int, ly: int, pitch_x: float, pitch_y: float):
    gx = (np.arange(lx) - (lx - 1) / 2.0) * pitch_x
    gy = (np.arange(ly) - (ly - 1) / 2.0) * pitch_y
    u = np.tile(gx, ly)
    v = np.repeat(gy, lx)
    return u, v


def tilt_grid(nx: int, ny: int, theta_max_deg: float):
    ax = np.deg2rad(np.linspace(-theta_max_deg, theta_max_deg, nx)) if nx > 1 else np.zeros(1)
    ay = np.deg2rad(np.linspace(-theta_max_deg, theta_max_deg, ny)) if ny > 1 else np.zeros(1)
    return np.tile(ax, ny), np.repeat(ay, nx)


def simulate_rf3(points: np.ndarray, elem_x, elem_y, tx_ax, tx_ay, n_samples: int, fs: float = FS,
                 c: float = C_SOUND, f0: float = F0, bw: float = BW) -> np.ndarray:
    """FP64 channel data ``rf[N][L][T]`` of point scatterers ``points[n][>=4]``."""
    lib = _load()
    ex = np.ascontiguousarray(elem_x, dtype=np.float64)
    ey = np.ascontiguousarray(elem_y, dtype=np.float64)
    ax = np.ascontiguousarray(tx_ax, dtype=np.float64)
    ay = np.ascontiguousarray(tx_ay, dtype=np.float64)
    pts = np.asarray(points, dtype=np.float64)
    px, py, pz, pa = (np.ascontiguousarray(pts[:, k]) for k in range(4))
    out = np.empty((ax.shape[0], ex.shape[0], n_samples), dtype=np.float64)
    rc = lib.kks_simulate3(int(ax.shape[0]), _dp(ax), _dp(ay), int(ex.shape[0]), _dp(ex), _dp(ey),
                           int(n_samples), float(fs), float(c), float(f0), pulse_alpha(f0, bw),
                           pulse_half_window(f0, bw), int(px.shape[0]), _dp(px), _dp(py), _dp(pz),
                           _dp(pa), _dp(out))
    if rc != 0:
        raise RuntimeError(f"kks_simulate3 failed with code {rc}")
    return out


def volume_workload(seed: int = 3000, lx: int = 16, ly: int = 16, pitch: float = 0.3e-3, ntx: int = 3,
                    nty: int = 3, theta_max_deg: float = 8.0, n_samples: int = 1024, nx: int = 48,
                    ny: int = 48, nz: int = 64, dxyz: float = 0.15e-3, z0: float = 6e-3,
                    points=((0.0, 0.0, 9e-3), (-2e-3, 1.5e-3, 8e-3), (1.5e-3, -2e-3, 10e-3)),
                    speckle: int = 0, snr_db=None, rf_dtype: str = "f32") -> Volume:
    """A matrix-array frame: ``points`` (x, y, z) of amplitude 10 plus
    ``speckle`` N(0,1) scatterers uniform in the voxel box."""
    rng = np.random.default_rng(seed)
    u, v = matrix_elements(lx, ly, pitch, pitch)
    ax, ay = tilt_grid(ntx, nty, theta_max_deg)
    x0 = -dxyz * (nx - 1) / 2.0
    y0 = -dxyz * (ny - 1) / 2.0
    pts = [np.array([[p[0], p[1], p[2], 10.0] for p in points])] if len(points) else []
    if speckle:
        sp = np.stack([rng.uniform(x0, -x0, speckle), rng.uniform(y0, -y0, speckle),
                       rng.uniform(z0, z0 + dxyz * (nz - 1), speckle), rng.standard_normal(speckle)], 1)
        pts.append(sp)
    allp = np.concatenate(pts) if pts else np.zeros((0, 4))
    rf64 = simulate_rf3(allp, u, v, ax, ay, n_samples)
    if rf_dtype == "i16":
        rf, _ = add_noise_and_quantise(rf64, 30.0 if snr_db is None else snr_db, seed)
    else:
        rf = rf64.astype(np.float32)
    return Volume(f"matrix{lx}x{ly}_N{ntx}x{nty}_T{n_samples}_vox{nx}x{ny}x{nz}", seed, u, v, ax, ay,
                  n_samples, FS, C_SOUND, (nx, nz, x0, dxyz, z0, dxyz), (ny, y0, dxyz), rf, allp,
                  len(points))
