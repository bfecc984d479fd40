"""Image-quality measures used to judge beamformed images: gCNR and FWHM.

TEST INFRASTRUCTURE -- not part of the product (see ``oracle/__init__``).

The paper judges its images by the generalized contrast-to-noise ratio of an
anechoic inclusion against a background region (Section III, Fig. 5 and the
Experimental Methods paragraph, which cite Rodriguez-Molares et al. 2020 and
Schlunk et al. 2023 for the definition), and by the width of the point-target
responses (Section III, Fig. 4: resolution and separability of wire targets).

Definitions written out here (plain numpy, one decision at a time):

* envelope -- ``|B|`` of the complex image, or ``sqrt(I)`` of an intensity
  image.  Formed in float32 with one rounding per operation (square, square,
  add, square root, no fused multiply-add), because every integer this module
  derives from it (a histogram bin, an argmax, a half-maximum crossing index)
  must be decided in the same precision by any implementation compared with
  it.
* regions -- pixel *centres* ``x = x0 + ix*dx``, ``z = z0 + iz*dz`` (FP64, one
  rounding per operation) tested against a disk ``d^2 <= r^2``, an annulus
  ``r1^2 < d^2 <= r2^2`` or a closed rectangle.
* gCNR -- ``1 - OVL`` where ``OVL = sum_b min(p_in[b], p_out[b])`` over a
  common set of ``n_bins`` equal-width bins spanning ``[lo, hi]``, the envelope
  range over the union of both regions; ``p = counts / region size``.  The
  bin of a value v is ``floor(((v - lo) * n_bins) / (hi - lo))`` in float32,
  clamped to ``n_bins - 1``; ``hi == lo`` puts everything in bin 0.  The sum
  is evaluated exactly as ``sum_b min(c_in[b]*n_out, c_out[b]*n_in)`` in
  integers, divided once by ``n_in*n_out``.  An empty region gives NaN.
* FWHM -- the peak of the envelope inside an integer search window (first
  maximum in row-major order), then along the peak's row (lateral) and column
  (axial) the nearest samples on each side that fall strictly below half the
  peak; each crossing is placed by linear interpolation between that sample
  and its inner neighbour; the width is the distance between the two
  crossings in metres.  A side that reaches the image edge without a sample
  below half the peak makes that width NaN.
"""
from __future__ import annotations

import numpy as np

REGION_DISK, REGION_ANNULUS, REGION_RECT = 0, 1, 2
IMG_COMPLEX, IMG_INTENSITY = 0, 1


def envelope_f32(img: np.ndarray, kind: int = IMG_COMPLEX) -> np.ndarray:
    """Envelope in float32, one rounding per operation.

    ``img``: complex64 array (``IMG_COMPLEX``) or float32 intensity
    (``IMG_INTENSITY``), any shape.
    """
    if kind == IMG_COMPLEX:
        a = np.ascontiguousarray(img, dtype=np.complex64)
        re = a.real.astype(np.float32)
        im = a.imag.astype(np.float32)
        s = np.add(np.multiply(re, re, dtype=np.float32), np.multiply(im, im, dtype=np.float32),
                   dtype=np.float32)
        return np.sqrt(s, dtype=np.float32)
    if kind == IMG_INTENSITY:
        return np.sqrt(np.ascontiguousarray(img, dtype=np.float32), dtype=np.float32)
    raise ValueError("kind must be IMG_COMPLEX or IMG_INTENSITY")


def pixel_centres(grid):
    """FP64 pixel-centre coordinates ``(x[nx], z[nz])`` of ``grid``."""
    nx, nz, x0, dx, z0, dz = grid
    ix = np.arange(int(nx), dtype=np.float64)
    iz = np.arange(int(nz), dtype=np.float64)
    return x0 + ix * dx, z0 + iz * dz


def region_mask(grid, region) -> np.ndarray:
    """Boolean ``[nz][nx]`` membership of each pixel centre in ``region``.

    ``region = (kind, a, b, c, d)``:
      * disk ``(REGION_DISK, cx, cz, r, _)``: ``(x-cx)^2 + (z-cz)^2 <= r^2``;
      * annulus ``(REGION_ANNULUS, cx, cz, r1, r2)``: ``r1^2 < d^2 <= r2^2``;
      * rectangle ``(REGION_RECT, x_lo, x_hi, z_lo, z_hi)``: closed box.
    """
    kind, a, b, c, d = region
    x, z = pixel_centres(grid)
    X = x[None, :]
    Z = z[:, None]
    if kind == REGION_RECT:
        return (X >= a) & (X <= b) & (Z >= c) & (Z <= d)
    ex = X - a
    ez = Z - b
    d2 = ex * ex + ez * ez
    if kind == REGION_DISK:
        return d2 <= c * c
    if kind == REGION_ANNULUS:
        return (d2 > c * c) & (d2 <= d * d)
    raise ValueError(f"unknown region kind {kind}")


def bin_index_f32(v: np.ndarray, lo: np.float32, hi: np.float32, n_bins: int) -> np.ndarray:
    """Equal-width bin of each float32 value over ``[lo, hi]`` (float32 decisions)."""
    v = np.asarray(v, dtype=np.float32)
    lo = np.float32(lo)
    hi = np.float32(hi)
    if hi == lo:
        return np.zeros(v.shape, dtype=np.int64)
    num = np.multiply(np.subtract(v, lo, dtype=np.float32), np.float32(n_bins), dtype=np.float32)
    q = np.divide(num, np.subtract(hi, lo, dtype=np.float32), dtype=np.float32)
    return np.minimum(np.floor(q).astype(np.int64), n_bins - 1)


def gcnr_values(v_in: np.ndarray, v_out: np.ndarray, n_bins: int) -> float:
    """gCNR of two float32 samples: ``1 - sum_b min(p_in[b], p_out[b])``."""
    if n_bins < 1:
        raise ValueError("n_bins must be >= 1")
    v_in = np.asarray(v_in, dtype=np.float32).ravel()
    v_out = np.asarray(v_out, dtype=np.float32).ravel()
    n_in, n_out = v_in.size, v_out.size
    if n_in == 0 or n_out == 0:
        return float("nan")
    both = np.concatenate([v_in, v_out])
    lo, hi = both.min(), both.max()
    c_in = np.bincount(bin_index_f32(v_in, lo, hi, n_bins), minlength=n_bins)
    c_out = np.bincount(bin_index_f32(v_out, lo, hi, n_bins), minlength=n_bins)
    s = 0
    for b in range(n_bins):  # exact integer overlap
        s += min(int(c_in[b]) * n_out, int(c_out[b]) * n_in)
    return 1.0 - float(s) / (float(n_in) * float(n_out))


def gcnr(img: np.ndarray, grid, inside, outside, n_bins: int = 256,
         kind: int = IMG_COMPLEX) -> float:
    """gCNR of one image ``[nz][nx]`` between two regions."""
    env = envelope_f32(img, kind)
    return gcnr_values(env[region_mask(grid, inside)], env[region_mask(grid, outside)], n_bins)


def _crossing(env_line: np.ndarray, coords: np.ndarray, k_pk: int, half: np.float32, step: int):
    """Half-maximum crossing walking from the peak in direction ``step``."""
    k = k_pk
    n = env_line.shape[0]
    while True:
        kn = k + step
        if kn < 0 or kn >= n:
            return float("nan")
        if env_line[kn] < half:
            e_in = float(env_line[k])      # >= half
            e_out = float(env_line[kn])    # < half
            t = (e_in - float(half)) / (e_in - e_out)
            return float(coords[k]) + t * (float(coords[kn]) - float(coords[k]))
        k = kn


def fwhm(img: np.ndarray, grid, target, kind: int = IMG_COMPLEX):
    """Peak and -6 dB (half-amplitude) widths of one point target.

    ``target = (ix, iz, wx, wz)``: search window ``[ix-wx, ix+wx] x
    [iz-wz, iz+wz]`` in pixel indices, clipped to the image.  Returns a dict
    with the peak indices, the peak envelope (float32) and the lateral and
    axial widths in metres (NaN where no crossing exists; all NaN/-1 for an
    empty window).
    """
    env = envelope_f32(img, kind)
    nz, nx = env.shape
    ix, iz, wx, wz = (int(t) for t in target)
    x_lo, x_hi = max(ix - wx, 0), min(ix + wx, nx - 1)
    z_lo, z_hi = max(iz - wz, 0), min(iz + wz, nz - 1)
    out = {"ix": -1, "iz": -1, "peak": float("nan"), "lateral": float("nan"),
           "axial": float("nan")}
    if x_lo > x_hi or z_lo > z_hi:
        return out
    best, bx, bz = None, -1, -1
    for zz in range(z_lo, z_hi + 1):          # first maximum in row-major order
        for xx in range(x_lo, x_hi + 1):
            v = env[zz, xx]
            if best is None or v > best:
                best, bx, bz = v, xx, zz
    half = np.float32(best) * np.float32(0.5)
    x, z = pixel_centres(grid)
    row = env[bz, :]
    col = env[:, bx]
    lat = _crossing(row, x, bx, half, +1) - _crossing(row, x, bx, half, -1)
    ax = _crossing(col, z, bz, half, +1) - _crossing(col, z, bz, half, -1)
    out.update(ix=bx, iz=bz, peak=float(best), lateral=lat, axial=ax)
    return out
