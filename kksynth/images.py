"""Seeded synthetic complex images for the image-quality measures (input generation only).

Fully developed speckle (circular complex Gaussian pixels, Rayleigh envelope)
with darker disks standing in for anechoic inclusions and separable Gaussian
point responses standing in for wire targets, the structures the paper's
contrast and resolution figures measure (Section III, Figs. 4 and 5).
"""
from __future__ import annotations

import numpy as np


def speckle_images(seed: int, n_images: int, nx: int, nz: int, disks_px=(), disk_level: float = 0.1,
                   points_px=(), point_amp: float = 20.0, point_sigma_px=(2.0, 1.5)) -> np.ndarray:
    """complex64 ``[n_images][nz][nx]``.

    ``disks_px``: ``(cx, cz, r)`` in pixels, speckle scaled by ``disk_level``
    inside; ``points_px``: ``(px, pz)`` in pixels, each adds a Gaussian
    envelope of peak ``point_amp`` and widths ``point_sigma_px`` (x, z) with a
    random phase per image.
    """
    rng = np.random.default_rng(seed)
    shape = (int(n_images), int(nz), int(nx))
    b = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
    ix = np.arange(nx)[None, :]
    iz = np.arange(nz)[:, None]
    for cx, cz, r in disks_px:
        inside = (ix - cx) ** 2 + (iz - cz) ** 2 <= r * r
        b[:, inside] *= disk_level
    sx, sz = point_sigma_px
    for px, pz in points_px:
        g = np.exp(-((ix - px) ** 2) / (2 * sx * sx) - ((iz - pz) ** 2) / (2 * sz * sz))
        ph = np.exp(1j * rng.uniform(0, 2 * np.pi, int(n_images)))[:, None, None]
        b += point_amp * g[None] * ph
    return b.astype(np.complex64)
