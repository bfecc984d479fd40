"""Phantoms, geometry and simulated RF (input generation only).

Conventions used throughout the repository:

* elements sit at ``u_l = (l - (L-1)/2) * pitch`` on the line z = 0; image x
  is measured from the array centre, z is depth (metres);
* sample n of a record is at time ``n / fs``; a transmit plane wave at angle
  theta passes the origin at t = 0;
* transmit angles are evenly spaced over ``[-theta_max, +theta_max]``
  (the paper's uniform transmit distribution, Section II-C).
"""
from __future__ import annotations

import ctypes
import dataclasses
import functools
import math
import os
import subprocess
import threading

import numpy as np

C_SOUND = 1540.0      # m/s
FS = 20e6             # Hz
F0 = 5e6              # Hz, pulse centre frequency
BW = 0.6              # fractional -6 dB bandwidth

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libkksim.so")
_lib = None
_lock = threading.Lock()


def build_sim(force: bool = False) -> str:
    """Compile the C forward model (plain gcc, FP64, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "sim.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                           "-shared", src, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_sim())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.kks_simulate.argtypes = [
                ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_double,
                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_int, dp, dp, dp, dp]
            lib.kks_simulate.restype = ctypes.c_int
            lib.kks_simulate3.argtypes = [
                ctypes.c_int, dp, dp, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_double,
                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_int, dp, dp, dp, dp, dp]
            lib.kks_simulate3.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def pulse_alpha(f0: float = F0, bw: float = BW) -> float:
    """Gaussian envelope rate so the spectrum is -6 dB at f0 (1 +- bw/2)."""
    return math.pi ** 2 * f0 ** 2 * bw ** 2 / (4.0 * math.log(10 ** (6 / 20)))


def pulse_half_window(f0: float = F0, bw: float = BW) -> float:
    """+-4 sigma of the Gaussian envelope, in seconds."""
    sigma = 1.0 / math.sqrt(2.0 * pulse_alpha(f0, bw))
    return 4.0 * sigma


def element_positions(n_elem: int, pitch: float) -> np.ndarray:
    return (np.arange(n_elem, dtype=np.float64) - (n_elem - 1) / 2.0) * pitch


def tx_angles_even(n_tx: int, theta_max_deg: float) -> np.ndarray:
    """Transmit angles evenly spaced over +-theta_max, endpoints included (rad)."""
    if n_tx == 1:
        return np.zeros(1)
    return np.deg2rad(np.linspace(-theta_max_deg, theta_max_deg, n_tx))


@dataclasses.dataclass
class Phantom:
    x: np.ndarray      # m
    z: np.ndarray      # m
    amp: np.ndarray    # reflectivity
    n_points: int = 0  # the first n_points entries are the bright point targets


@dataclasses.dataclass
class Workload:
    """One frame of synthetic CPWC channel data plus its imaging grid."""
    name: str
    seed: int
    elem_x: np.ndarray          # [L] m
    tx_angles: np.ndarray       # [N] rad (all acquired transmits)
    n_samples: int              # T
    fs: float
    c: float
    grid: tuple                 # (nx, nz, x0, dx, z0, dz), metres
    rf: np.ndarray              # [N][L][T] float32 or int16
    phantom: Phantom
    theta_max_deg: float
    pitch: float

    @property
    def n_elem(self) -> int:
        return int(self.elem_x.shape[0])

    @property
    def n_tx(self) -> int:
        return int(self.tx_angles.shape[0])

    def pixel_x(self) -> np.ndarray:
        nx, nz, x0, dx, z0, dz = self.grid
        return x0 + dx * np.arange(nx)

    def pixel_z(self) -> np.ndarray:
        nx, nz, x0, dx, z0, dz = self.grid
        return z0 + dz * np.arange(nz)


def simulate_rf(ph: Phantom, elem_x: np.ndarray, tx_angles: np.ndarray, n_samples: int,
                fs: float = FS, c: float = C_SOUND, f0: float = F0, bw: float = BW) -> np.ndarray:
    """FP64 channel data ``rf[N][L][T]`` for a point-scatterer phantom."""
    lib = _load()
    elem_x = np.ascontiguousarray(elem_x, dtype=np.float64)
    tx = np.ascontiguousarray(tx_angles, dtype=np.float64)
    sx = np.ascontiguousarray(ph.x, dtype=np.float64)
    sz = np.ascontiguousarray(ph.z, dtype=np.float64)
    sa = np.ascontiguousarray(ph.amp, dtype=np.float64)
    out = np.empty((tx.shape[0], elem_x.shape[0], n_samples), dtype=np.float64)
    rc = lib.kks_simulate(int(tx.shape[0]), _dp(tx), int(elem_x.shape[0]), _dp(elem_x),
                          int(n_samples), float(fs), float(c), float(f0), pulse_alpha(f0, bw),
                          pulse_half_window(f0, bw), int(sx.shape[0]), _dp(sx), _dp(sz), _dp(sa),
                          _dp(out))
    if rc != 0:
        raise RuntimeError(f"kks_simulate failed with code {rc}")
    return out


def add_noise_and_quantise(rf: np.ndarray, snr_db: float, seed: int):
    """White Gaussian noise at ``snr_db`` (rms over the frame), then int16.

    ``q = round_half_even(32767 * v / max|v|)``; returns ``(q, scale)`` with
    ``v ~= q * scale``.
    """
    rng = np.random.default_rng(seed + 7_000_000)
    rms = float(np.sqrt(np.mean(rf.astype(np.float64) ** 2)))
    v = rf + rng.standard_normal(rf.shape) * (rms * 10 ** (-snr_db / 20.0))
    peak = float(np.max(np.abs(v)))
    scale = peak / 32767.0 if peak > 0 else 1.0
    q = np.rint(v / scale)  # numpy rint rounds half to even
    return np.clip(q, -32767, 32767).astype(np.int16), scale


def _speckle(rng, n, xlo, xhi, zlo, zhi):
    return (rng.uniform(xlo, xhi, n), rng.uniform(zlo, zhi, n), rng.standard_normal(n))


def point_phantom(points_mm, amp=10.0) -> Phantom:
    pts = np.asarray(points_mm, dtype=np.float64) * 1e-3
    return Phantom(pts[:, 0].copy(), pts[:, 1].copy(), np.full(pts.shape[0], float(amp)),
                   n_points=pts.shape[0])


SMALL_POINTS_MM = [(-4.0, 8.0), (-2.0, 10.0), (0.0, 12.0), (2.0, 14.0), (4.0, 16.0)]
LARGE_WIRES_MM = [(x, z) for z in (10.0, 16.0, 22.0, 28.0, 34.0) for x in (-12.0, -4.0, 4.0, 12.0)]
LARGE_CYSTS_MM = [(-8.0, 20.0), (0.0, 30.0), (8.0, 38.0)]


@functools.lru_cache(maxsize=8)
def _small_cached(seed: int, speckle: int, points: bool):
    L, pitch, N, thmax, T = 64, 0.3e-3, 11, 8.0, 512
    elem_x = element_positions(L, pitch)
    tx = tx_angles_even(N, thmax)
    nx = nz = 128
    x0, z0 = -9.5e-3, 5e-3
    dx = 19e-3 / (nx - 1)
    dz = 19e-3 / (nz - 1)
    rng = np.random.default_rng(seed)
    xs, zs, amps = [], [], []
    npts = 0
    if points:
        ph0 = point_phantom(SMALL_POINTS_MM)
        xs.append(ph0.x); zs.append(ph0.z); amps.append(ph0.amp)
        npts = ph0.x.shape[0]
    if speckle:
        sx, sz, sa = _speckle(rng, speckle, x0, x0 + dx * (nx - 1), z0, z0 + dz * (nz - 1))
        xs.append(sx); zs.append(sz); amps.append(sa)
    ph = Phantom(np.concatenate(xs), np.concatenate(zs), np.concatenate(amps), n_points=npts)
    rf = simulate_rf(ph, elem_x, tx, T).astype(np.float32)
    return Workload("L64_N11_T512_f32_grid128", seed, elem_x, tx, T, FS, C_SOUND,
                    (nx, nz, x0, dx, z0, dz), rf, ph, thmax, pitch)


def workload_small(seed: int = 1000, speckle: int = 1000, points: bool = True) -> Workload:
    """64 elements (0.3 mm pitch), 11 transmits over +-8 deg, 512 fp32 samples,
    128x128 grid over x in [-9.5, 9.5] mm, z in [5, 24] mm; 5 point targets of
    amplitude 10 plus ``speckle`` N(0,1) scatterers uniform in the grid region."""
    return _small_cached(int(seed), int(speckle), bool(points))


@functools.lru_cache(maxsize=4)
def _large_cached(seed: int, speckle: int, nx: int, nz: int, n_samples: int, snr_db):
    L, pitch, N, thmax, T = 128, 0.3e-3, 75, 16.0, n_samples
    elem_x = element_positions(L, pitch)
    tx = tx_angles_even(N, thmax)
    dx = dz = pitch / 4.0
    x0 = -dx * (nx - 1) / 2.0
    z0 = 5e-3
    xmax, zmax = x0 + dx * (nx - 1), z0 + dz * (nz - 1)
    rng = np.random.default_rng(seed)
    ph0 = point_phantom([(x, z) for (x, z) in LARGE_WIRES_MM
                         if x0 * 1e3 <= x <= xmax * 1e3 and z0 * 1e3 <= z <= zmax * 1e3])
    sx, sz, sa = _speckle(rng, speckle, x0, xmax, z0, zmax)
    keep = np.ones(speckle, dtype=bool)
    for cx, cz in LARGE_CYSTS_MM:
        keep &= (sx - cx * 1e-3) ** 2 + (sz - cz * 1e-3) ** 2 > (2e-3) ** 2
    ph = Phantom(np.concatenate([ph0.x, sx[keep]]), np.concatenate([ph0.z, sz[keep]]),
                 np.concatenate([ph0.amp, sa[keep]]), n_points=ph0.x.shape[0])
    rf64 = simulate_rf(ph, elem_x, tx, T)
    if snr_db is None:
        rf = rf64.astype(np.float32)
        dt = "f32"
    else:
        rf, _ = add_noise_and_quantise(rf64, snr_db, seed)
        dt = "i16"
    return Workload(f"L128_N75_T{T}_{dt}_grid{nx}x{nz}", seed, elem_x, tx, T, FS, C_SOUND,
                    (nx, nz, x0, dx, z0, dz), rf, ph, thmax, pitch)


def workload_large(seed: int = 2000, speckle: int = 50_000, nx: int = 512, nz: int = 512,
                   n_samples: int = 2048, snr_db=30.0) -> Workload:
    """128 elements (0.3 mm pitch), 75 transmits over +-16 deg, 2048 samples as
    int16 quantised at 30 dB SNR, 512x512 grid at pitch/4 = 0.075 mm from 5 mm
    depth; 20 wire targets on a 4x5 lattice and 3 anechoic 4 mm cysts in
    ``speckle`` N(0,1) scatterers."""
    return _large_cached(int(seed), int(speckle), int(nx), int(nz), int(n_samples), snr_db)


def workload_tiny(seed: int = 7, n_elem: int = 4, n_tx: int = 2, n_samples: int = 32,
                  nx: int = 8, nz: int = 8, pitch: float = 0.3e-3, theta_max_deg: float = 8.0,
                  n_scat: int = 3) -> Workload:
    """Very small random frame for brute-force checks (float32 RF)."""
    rng = np.random.default_rng(seed)
    elem_x = element_positions(n_elem, pitch)
    tx = tx_angles_even(n_tx, theta_max_deg)
    dx = dz = pitch / 2
    x0 = -dx * (nx - 1) / 2
    z0 = 0.4e-3
    # scatterers placed so echoes land inside the short record
    ph = Phantom(rng.uniform(x0, -x0, n_scat), rng.uniform(z0, z0 + dz * (nz - 1), n_scat),
                 rng.standard_normal(n_scat))
    rf = simulate_rf(ph, elem_x, tx, n_samples).astype(np.float32)
    rf += rng.standard_normal(rf.shape).astype(np.float32) * np.float32(0.05)
    return Workload(f"tiny_L{n_elem}_N{n_tx}_T{n_samples}", seed, elem_x, tx, n_samples, FS,
                    C_SOUND, (nx, nz, x0, dx, z0, dz), rf, ph, theta_max_deg, pitch)


def workload_custom(name: str, seed: int, n_elem: int, pitch: float, n_tx: int,
                    theta_max_deg: float, n_samples: int, grid: tuple, phantom: Phantom,
                    rf_dtype: str = "f32", snr_db=None, fs: float = FS, c: float = C_SOUND) -> Workload:
    """Any geometry / phantom; ``rf_dtype`` 'f32' or 'i16' (int16 needs ``snr_db``)."""
    elem_x = element_positions(n_elem, pitch)
    tx = tx_angles_even(n_tx, theta_max_deg)
    rf64 = simulate_rf(phantom, elem_x, tx, n_samples, fs=fs, c=c)
    if rf_dtype == "i16":
        rf, _ = add_noise_and_quantise(rf64, 30.0 if snr_db is None else snr_db, seed)
    else:
        rf = rf64.astype(np.float32)
        if snr_db is not None:
            rng = np.random.default_rng(seed + 11)
            rms = float(np.sqrt(np.mean(rf64 ** 2)))
            rf = (rf64 + rng.standard_normal(rf64.shape) * rms * 10 ** (-snr_db / 20)).astype(np.float32)
    return Workload(name, seed, elem_x, tx, n_samples, fs, c, tuple(grid), rf, phantom,
                    theta_max_deg, pitch)
