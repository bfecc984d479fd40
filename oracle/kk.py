"""FP64 oracle: analytic signal, far-field decomposition, KK and DAS images.

TEST INFRASTRUCTURE (see ``oracle/__init__``).  Plain, slow, FP64.  Library
primitives used as steps: numpy's FFT/IFFT and matmul.  Pixel loops are in
``kk_oracle.c`` (plain FP64 C, OpenMP over pixels only).

Readings of the paper taken here (the paper is silent or ambiguous on them):

* Analytic signal (Section II-F): FFT of length T (no zero padding), weights
  h_0 = 1, h_k = 2 for 1 <= k < T/2, the Nyquist bin and negative frequencies
  set to zero, IFFT with its 1/T.
* Shear of Eq. (compression) in image coordinates: the record of element l is
  advanced by delta_l(theta_o) = (x_ref(theta_o) - u_l) sin(theta_o) / c,
  x_ref = the largest u_l for theta_o > 0, the smallest for theta_o < 0, and 0
  for theta_o = 0, so every shift is a non-negative advance (reading later
  samples), as the paper's d_l makes it.  The matching receive delay of Eq.
  (KK) is then ((x - x_ref) sin theta_o + z cos theta_o) / c (stationary-phase
  arrival time of the sheared sum).
* The shear is applied by the Fourier shift theorem on the analytic spectrum
  (Section II-F), which makes it circular over the record.
* Interpolation (unspecified): linear, zero outside [0, T-1].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import schemes as _schemes

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libkkoracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``kk_oracle.c`` with plain gcc (FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "kk_oracle.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                           src, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            ci, cd = ctypes.c_int, ctypes.c_double
            lib.orc_kk_beamform.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp, ip, ci, ci, dp, dp,
                                            cd, cd, dp, dp]
            lib.orc_kk_beamform.restype = ci
            lib.orc_das_beamform.argtypes = [ci, ci, ci, dp, dp, dp, dp, ci, dp, dp, cd, cd, cd, ci, dp]
            lib.orc_das_beamform.restype = ci
            lib.orc_kk_beamform_vol.argtypes = [ci, ci, dp, dp, dp, dp, dp, dp, dp, dp, dp, ip, ci, ci,
                                                dp, dp, dp, cd, cd, dp]
            lib.orc_kk_beamform_vol.restype = ci
            lib.orc_das_beamform_vol.argtypes = [ci, ci, ci, dp, dp, dp, dp, dp, dp, ci, dp, dp, dp,
                                                 cd, cd, dp]
            lib.orc_das_beamform_vol.restype = ci
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


# --------------------------------------------------------------------------
# Steps 1-2 and 5: analytic signal (Section II-F)
# --------------------------------------------------------------------------
def hilbert_weights(T: int) -> np.ndarray:
    """h_k for k < T/2: 1 at DC, 2 for positive frequencies (Section II-F:
    negative frequencies set to zero; the Nyquist bin is dropped)."""
    if T % 2:
        raise ValueError("T must be even")
    h = np.full(T // 2, 2.0)
    h[0] = 1.0
    return h


def analytic_spectrum(rf: np.ndarray) -> np.ndarray:
    """X[..., k] = h_k sum_t rf[..., t] exp(-2 pi i k t / T), k < T/2."""
    T = rf.shape[-1]
    X = np.fft.fft(np.asarray(rf, dtype=np.float64), axis=-1)[..., : T // 2]
    return X * hilbert_weights(T)


def inverse_half_spectrum(Y: np.ndarray, T: int) -> np.ndarray:
    """y[..., t] = (1/T) sum_{k < T/2} Y[..., k] exp(+2 pi i k t / T)."""
    full = np.zeros(Y.shape[:-1] + (T,), dtype=np.complex128)
    full[..., : T // 2] = Y
    return np.fft.ifft(full, axis=-1)


def analytic_signal(rf: np.ndarray) -> np.ndarray:
    """Complex analytic record of every channel (Section II-F)."""
    return inverse_half_spectrum(analytic_spectrum(rf), rf.shape[-1])


# --------------------------------------------------------------------------
# Step 3-4: far-field decomposition, Eq. (compression)
# --------------------------------------------------------------------------
def shear_reference(elem_x, theta_o, rule: str = "advance") -> np.ndarray:
    """x_ref(theta_o): the array end that makes every shear a non-negative
    advance (rule 'advance', the reading of Eq. (compression)); 'retard' takes
    the opposite end and 'centre' takes 0 (used only by invariance tests)."""
    u = np.asarray(elem_x, dtype=np.float64)
    th = np.asarray(theta_o, dtype=np.float64)
    if rule == "advance":
        return np.where(th > 0, u.max(), np.where(th < 0, u.min(), 0.0))
    if rule == "retard":
        return np.where(th > 0, u.min(), np.where(th < 0, u.max(), 0.0))
    if rule == "centre":
        return np.zeros_like(th)
    raise ValueError(rule)


def shear_delays(elem_x, rx_angles, c: float, rule: str = "advance") -> np.ndarray:
    """delta_l(theta_o) = (x_ref(theta_o) - u_l) sin(theta_o) / c, seconds, [M][L]."""
    u = np.asarray(elem_x, dtype=np.float64)
    th = np.asarray(rx_angles, dtype=np.float64)
    xr = shear_reference(u, th, rule)
    return (xr[:, None] - u[None, :]) * np.sin(th)[:, None] / c


def decompose(rf: np.ndarray, elem_x, ps: "_schemes.PairSet", fs: float, c: float,
              rule: str = "advance") -> np.ndarray:
    """RF_theta for every pair, y[P][T] complex (Eq. (compression), Section II-F).

    Y[i][o][k] = h_k sum_l X[i][l][k] exp(+2 pi i k fs delta_l(theta_o) / T),
    then the inverse transform of the half spectrum.  Only the transmits and
    receive angles that appear in the pair set are transformed.
    """
    T = rf.shape[-1]
    F = T // 2
    tx_used = np.unique(ps.tx_index)
    rx_used = np.unique(ps.rx_index)
    X = analytic_spectrum(rf[tx_used])                         # [Nu][L][F]
    d = shear_delays(elem_x, ps.rx_angles[rx_used], c, rule)   # [Mu][L] seconds
    k = np.arange(F, dtype=np.float64)
    W = np.exp(2j * np.pi * k[None, None, :] * (fs * d)[:, :, None] / T)  # [Mu][L][F]
    # per bin: Y_k (Nu x Mu) = X_k (Nu x L) @ W_k (L x Mu)
    Yk = np.matmul(np.transpose(X, (2, 0, 1)), np.transpose(W, (2, 1, 0)))  # [F][Nu][Mu]
    ti = np.searchsorted(tx_used, ps.tx_index)
    ri = np.searchsorted(rx_used, ps.rx_index)
    Yp = Yk[:, ti, ri].T                                        # [P][F]
    return inverse_half_spectrum(Yp, T)


# --------------------------------------------------------------------------
# Step 6-7: KK image formation, Eq. (KK); compounding, Eqs. (coherent)/(incoherent)
# --------------------------------------------------------------------------
def grid_pixels(grid, pixels=None):
    """Pixel coordinates: the whole grid in [z][x] order, or the listed
    (ix, iz) pairs."""
    nx, nz, x0, dx, z0, dz = grid
    if pixels is None:
        iz, ix = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
        ix, iz = ix.ravel(), iz.ravel()
    else:
        pixels = np.asarray(pixels, dtype=np.int64).reshape(-1, 2)
        ix, iz = pixels[:, 0], pixels[:, 1]
    return (x0 + dx * ix.astype(np.float64)), (z0 + dz * iz.astype(np.float64))


def kk_beamform(y: np.ndarray, elem_x, ps: "_schemes.PairSet", grid, fs: float, c: float,
                pixels=None, rule: str = "advance", weights=None) -> np.ndarray:
    """B[J][nz][nx] (or B[J][n_pix] for a pixel list), complex128, Eq. (KK);
    with `weights` [P], pair p's term is multiplied by weights[p] (the
    apodization the paper leaves out of Eq. (KK) for simplicity)."""
    lib = _load()
    P, T = y.shape
    yc = np.ascontiguousarray(y, dtype=np.complex128)
    th_i = ps.theta_i().astype(np.float64)
    th_o = ps.theta_o().astype(np.float64)
    xref = shear_reference(elem_x, th_o, rule)
    si, ci_ = np.ascontiguousarray(np.sin(th_i)), np.ascontiguousarray(np.cos(th_i))
    so, co = np.ascontiguousarray(np.sin(th_o)), np.ascontiguousarray(np.cos(th_o))
    xref = np.ascontiguousarray(xref, dtype=np.float64)
    grp = np.ascontiguousarray(ps.group, dtype=np.int32)
    px, pz = grid_pixels(grid, pixels)
    px, pz = np.ascontiguousarray(px), np.ascontiguousarray(pz)
    npix = px.shape[0]
    B = np.zeros((ps.n_groups, npix), dtype=np.complex128)
    wv = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    if wv is not None and wv.shape != (P,):
        raise ValueError("weights must have one entry per pair")
    rc = lib.orc_kk_beamform(P, T, _d(yc.view(np.float64)), _d(si), _d(ci_), _d(so), _d(co),
                             _d(xref), _i(grp), ps.n_groups, npix, _d(px), _d(pz), float(fs),
                             float(c), _d(wv) if wv is not None else None, _d(B.view(np.float64)))
    if rc:
        raise RuntimeError(f"orc_kk_beamform: {rc}")
    if pixels is None:
        nx, nz = grid[0], grid[1]
        return B.reshape(ps.n_groups, nz, nx)
    return B


def compound(B: np.ndarray, mode: str) -> np.ndarray:
    """Eq. (coherent): |sum_j B_j|^2; Eq. (incoherent): sum_j |B_j|^2; for one
    group either is the confocal intensity |B|^2 (Section II-D)."""
    if mode == "coherent":
        return np.abs(B.sum(axis=0)) ** 2
    if mode == "incoherent":
        return (np.abs(B) ** 2).sum(axis=0)
    raise ValueError(mode)


def kk_image(rf, elem_x, ps, grid, fs, c, pixels=None, rule="advance", weights=None):
    """Decomposition then image formation: B[J][...] complex128."""
    y = decompose(rf, elem_x, ps, fs, c, rule)
    return kk_beamform(y, elem_x, ps, grid, fs, c, pixels, rule, weights)


# --------------------------------------------------------------------------
# Step 8: DAS, Eq. (DAS)
# --------------------------------------------------------------------------
APERTURE_WINDOWS = {"boxcar": 0, "hann": 1}


def das_beamform_analytic(y: np.ndarray, tx_angles, elem_x, grid, fs: float, c: float,
                          pixels=None, f_number: float = 0.0, window: str = "boxcar") -> np.ndarray:
    """B[nz][nx] (or [n_pix]) from analytic channel data y[N][L][T].  With
    f_number > 0 each element is weighted by the receive aperture of half-width
    z / (2 F) about the pixel (boxcar or Hann); 0 = full aperture."""
    lib = _load()
    N, L, T = y.shape
    yc = np.ascontiguousarray(y, dtype=np.complex128)
    th = np.asarray(tx_angles, dtype=np.float64)
    si, ci_ = np.ascontiguousarray(np.sin(th)), np.ascontiguousarray(np.cos(th))
    ex = np.ascontiguousarray(elem_x, dtype=np.float64)
    px, pz = grid_pixels(grid, pixels)
    px, pz = np.ascontiguousarray(px), np.ascontiguousarray(pz)
    npix = px.shape[0]
    B = np.zeros(npix, dtype=np.complex128)
    rc = lib.orc_das_beamform(N, L, T, _d(yc.view(np.float64)), _d(si), _d(ci_), _d(ex), npix,
                              _d(px), _d(pz), float(fs), float(c), float(f_number),
                              APERTURE_WINDOWS[window], _d(B.view(np.float64)))
    if rc:
        raise RuntimeError(f"orc_das_beamform: {rc}")
    if pixels is None:
        return B.reshape(grid[1], grid[0])
    return B


def das_image(rf, tx_angles, elem_x, grid, fs, c, pixels=None, f_number=0.0, window="boxcar"):
    """Hilbert transform of every channel, then Eq. (DAS)."""
    return das_beamform_analytic(analytic_signal(rf), tx_angles, elem_x, grid, fs, c, pixels,
                                 f_number, window)


def rel_l2(a, b) -> float:
    """||a - b||_2 / ||b||_2 over all (complex) entries."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = float(np.linalg.norm(b.ravel()))
    return float(np.linalg.norm((a - b).ravel())) / (nb if nb > 0 else 1.0)
