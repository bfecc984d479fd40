"""KK beamforming on GB300: thin Python binding of the C ABI in include/kkbeam.h.

Every step of the path runs in the CUDA library ``_build/libkkbeam.so``;
this module only marshals arguments (torch tensors -> device pointers,
numpy arrays -> host pointers, torch streams -> cudaStream_t).  It fails
loudly when the library has not been built; there is no CPU fallback.

The functions carry the ABI's names (``kk_plan_create``, ``kk_decompose``,
``kk_beamform``, ``das_plan_create``, ``das_beamform``, ``kk_scheme_angles``,
...).  ``Plan`` is a small owner of a plan handle with the same calls as
methods.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

KK_OK, KK_ERR_INVALID_ARG, KK_ERR_UNSUPPORTED, KK_ERR_CUDA, KK_ERR_OOM, KK_ERR_TIMEOUT, KK_ERR_BOUNDS = range(7)
KK_RF_I16, KK_RF_F32 = 0, 1
KK_PREC_F32, KK_PREC_BF16, KK_PREC_F16, KK_PREC_F8E4M3 = 0, 1, 2, 3
KK_COMPOUND_NONE, KK_COMPOUND_COHERENT, KK_COMPOUND_INCOHERENT = 0, 1, 2
KK_SCHEME_SAME, KK_SCHEME_VERNIER, KK_SCHEME_SHIFTED, KK_SCHEME_CONFOCAL = 0, 1, 2, 3
KK_APERTURE_BOXCAR, KK_APERTURE_HANN = 0, 1
KK_REGION_DISK, KK_REGION_ANNULUS, KK_REGION_RECT = 0, 1, 2
KK_IMAGE_COMPLEX, KK_IMAGE_INTENSITY = 0, 1

_STATUS = {0: "KK_OK", 1: "KK_ERR_INVALID_ARG", 2: "KK_ERR_UNSUPPORTED", 3: "KK_ERR_CUDA",
           4: "KK_ERR_OOM", 5: "KK_ERR_TIMEOUT", 6: "KK_ERR_BOUNDS"}

# every symbol declared in include/kkbeam.h
EXPORTS = ["kk_plan_create", "das_plan_create", "kk_plan_destroy", "kk_plan_get_info",
           "kk_plan_set_gather", "kk_plan_set_trim", "kk_plan_status", "kk_plan_check_wait_timeout", "kk_debug_bounds",
           "kk_plan_workspace_size", "kk_decompose", "kk_spectrum", "kk_shear", "kk_inverse",
           "kk_beamform", "kk_beamform_noalloc", "das_beamform", "kk_run_host_scratch_size", "kk_run_host",
           "kk_scheme_angles", "kk_last_error", "kk_version",
           "kk_batch_create", "kk_batch_run", "kk_batch_get_info", "kk_batch_destroy",
           "kk_simulate_rf",
           # include/kknet.h
           "kk_net_create", "kk_net_destroy", "kk_net_info", "kk_net_status", "kk_nn_status", "kk_net_get_params", "kk_net_set_params",
           "kk_net_forward", "kk_net_loss_grad", "kk_net_adam", "kk_net_save", "kk_net_load",
           "kk_net_judge_filter", "kk_net_judge", "kk_net_image_scale",
           "kk_nn_conv3x3", "kk_nn_conv3x3_dgrad", "kk_nn_conv3x3_wgrad_workspace", "kk_nn_conv3x3_wgrad",
           # include/kkquality.h
           "kk_quality_create", "kk_quality_destroy", "kk_quality_gcnr", "kk_quality_fwhm",
           # include/kkstream.h
           "kk_stream_create", "kk_stream_push", "kk_stream_push_many", "kk_stream_end_frame", "kk_stream_wait", "kk_stream_after", "kk_stream_sync",
           "kk_stream_get_info", "kk_stream_destroy"]


class KKError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class kk_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("nz", ctypes.c_int32), ("x0", ctypes.c_double),
                ("dx", ctypes.c_double), ("z0", ctypes.c_double), ("dz", ctypes.c_double)]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


class kk_plan_desc(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int32), ("elem_x", _dp),
                ("n_tx", ctypes.c_int32), ("tx_angles", _dp),
                ("n_rx", ctypes.c_int32), ("rx_angles", _dp),
                ("n_pairs", ctypes.c_int32), ("pairs", _ip),
                ("group_of_pair", _ip), ("n_groups", ctypes.c_int32),
                ("compound", ctypes.c_int32), ("grid", kk_grid),
                ("c", ctypes.c_double), ("fs", ctypes.c_double),
                ("n_samples", ctypes.c_int32), ("rf_dtype", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
                ("pair_weight", _dp), ("f_number", ctypes.c_double), ("aperture", ctypes.c_int32),
                ("elem_y", _dp), ("tx_angles_y", _dp), ("rx_angles_y", _dp), ("ny", ctypes.c_int32),
                ("y0", ctypes.c_double), ("dy", ctypes.c_double)]


class kk_plan_info(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int32), ("n_tx", ctypes.c_int32),
                ("n_samples", ctypes.c_int32), ("n_bins", ctypes.c_int32),
                ("n_tx_used", ctypes.c_int32), ("n_rx_used", ctypes.c_int32),
                ("n_pairs", ctypes.c_int32), ("n_groups", ctypes.c_int32),
                ("nx", ctypes.c_int32), ("nz", ctypes.c_int32), ("is_das", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_size_t), ("rf_bytes", ctypes.c_size_t),
                ("rf_theta_bytes", ctypes.c_size_t), ("image_bytes", ctypes.c_size_t),
                ("intensity_bytes", ctypes.c_size_t), ("compression_factor", ctypes.c_double),
                ("launches_decompose", ctypes.c_int32), ("launches_beamform", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("is_volume", ctypes.c_int32),
                ("sep_lx", ctypes.c_int32), ("sep_ly", ctypes.c_int32), ("sep_mx", ctypes.c_int32),
                ("sep_my", ctypes.c_int32), ("gather_rows", ctypes.c_int32), ("gather_stage", ctypes.c_int32),
                ("gather_split", ctypes.c_int32), ("records_trimmed", ctypes.c_int32),
                ("rf_theta_stored_bytes", ctypes.c_size_t)]


class kk_batch_frame(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("d_rf", ctypes.c_void_p), ("d_rf_theta", ctypes.c_void_p),
                ("d_B", ctypes.c_void_p), ("d_I", ctypes.c_void_p), ("d_workspace", ctypes.c_void_p)]


class kk_batch_info(ctypes.Structure):
    _fields_ = [("n_frames", ctypes.c_int32), ("n_items", ctypes.c_int32), ("rows", ctypes.c_int32),
                ("stage", ctypes.c_int32), ("max_window", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("graph_nodes", ctypes.c_int32), ("n_tuned", ctypes.c_int32),
                ("pixel_pairs", ctypes.c_double), ("tuned_shape", ctypes.c_int32 * 16),
                ("tuned_ms", ctypes.c_float * 16), ("n_volume_frames", ctypes.c_int32),
                ("n_items_volume", ctypes.c_int32), ("rows_volume", ctypes.c_int32),
                ("stage_volume", ctypes.c_int32), ("max_window_volume", ctypes.c_int32)]


class kk_net_desc(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("base_channels", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class kk_region(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("c", ctypes.c_double), ("d", ctypes.c_double)]


class kk_target(ctypes.Structure):
    _fields_ = [("ix", ctypes.c_int32), ("iz", ctypes.c_int32), ("wx", ctypes.c_int32),
                ("wz", ctypes.c_int32)]


class kk_quality_desc(ctypes.Structure):
    _fields_ = [("grid", kk_grid), ("image_kind", ctypes.c_int32), ("n_contrast", ctypes.c_int32),
                ("inside", ctypes.POINTER(kk_region)), ("outside", ctypes.POINTER(kk_region)),
                ("n_bins", ctypes.c_int32), ("n_targets", ctypes.c_int32),
                ("targets", ctypes.POINTER(kk_target)), ("device", ctypes.c_int32)]


class kk_stream_info(ctypes.Structure):
    _fields_ = [("group", ctypes.c_int32), ("ring_groups", ctypes.c_int32), ("n_groups", ctypes.c_int32),
                ("events_pushed", ctypes.c_int64),
                ("events_dropped", ctypes.c_int64), ("groups_run", ctypes.c_int64),
                ("frames_done", ctypes.c_int64), ("device_bytes", ctypes.c_size_t), ("copies", ctypes.c_int64)]


# layout of kk_fwhm_result (32 bytes)
FWHM_DTYPE = np.dtype([("ix", "<i4"), ("iz", "<i4"), ("peak", "<f4"), ("reserved", "<i4"),
                       ("lateral", "<f8"), ("axial", "<f8")])

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the CUDA library; raise if it is missing (never falls back)."""
    global _lib
    if _lib is not None:
        return _lib
    # KKBEAM_VARIANT=bounds selects the bounds-checked build of the same
    # library (every gather index checked on the device; see kk_debug_bounds)
    variant = os.environ.get("KKBEAM_VARIANT", "")
    if variant not in _build.VARIANTS:
        raise RuntimeError(f"unknown KKBEAM_VARIANT {variant!r}")
    path = _build.VARIANTS[variant][1]
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"KK CUDA library not built ({path}); run "
                               "`python -m paper_2603_22496_gb300.build` or __graft_entry__.build()")
        _build.build(variant=variant)
    lib = ctypes.CDLL(path)
    vp, st = ctypes.c_void_p, ctypes.c_int
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "kk_plan_create": ([pp, ctypes.POINTER(kk_plan_desc)], st),
        "das_plan_create": ([pp, ctypes.POINTER(kk_plan_desc)], st),
        "kk_plan_destroy": ([vp], None),
        "kk_plan_get_info": ([vp, ctypes.POINTER(kk_plan_info)], st),
        "kk_plan_workspace_size": ([vp, ctypes.POINTER(ctypes.c_size_t)], st),
        "kk_plan_set_gather": ([vp, ctypes.c_int32, ctypes.c_int32], st),
        "kk_plan_set_trim": ([vp, ctypes.c_int32], st),
        "kk_plan_status": ([vp, ctypes.POINTER(ctypes.c_int32)], st),
        "kk_plan_check_wait_timeout": ([vp, ctypes.c_int64, vp], st),
        "kk_debug_bounds": ([ctypes.POINTER(ctypes.c_int64)], st),
        "kk_decompose": ([vp, vp, vp, vp, vp], st),
        "kk_spectrum": ([vp, vp, vp, vp], st),
        "kk_shear": ([vp, vp, vp, vp], st),
        "kk_inverse": ([vp, vp, vp, vp], st),
        "kk_beamform": ([vp, vp, vp, vp, vp, vp], st),
        "kk_beamform_noalloc": ([vp, vp, vp, vp, vp], st),
        "das_beamform": ([vp, vp, vp, vp, vp, vp], st),
        "kk_run_host_scratch_size": ([vp, ctypes.POINTER(ctypes.c_size_t)], st),
        "kk_run_host": ([vp, vp, vp, vp, vp, vp], st),
        "kk_scheme_angles": ([ctypes.c_int32, ctypes.c_int32, _dp, ctypes.c_double,
                              ctypes.c_int32, ctypes.c_double, _dp], st),
        "kk_batch_create": ([pp, ctypes.POINTER(kk_batch_frame), ctypes.c_int32, ctypes.c_int32, vp], st),
        "kk_batch_run": ([vp, vp], st),
        "kk_batch_get_info": ([vp, ctypes.POINTER(kk_batch_info)], st),
        "kk_batch_destroy": ([vp], None),
        "kk_simulate_rf": ([ctypes.c_int32, vp, ctypes.c_int32, vp, ctypes.c_int32, ctypes.c_double,
                            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32, vp,
                            ctypes.c_double, ctypes.c_uint64, vp, vp], st),
        "kk_last_error": ([], ctypes.c_char_p),
        "kk_version": ([], ctypes.c_char_p),
        "kk_net_create": ([pp, ctypes.POINTER(kk_net_desc)], st),
        "kk_net_destroy": ([vp], None),
        "kk_net_info": ([vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], st),
        "kk_net_get_params": ([vp, vp, vp], st),
        "kk_net_status": ([vp, ctypes.POINTER(ctypes.c_int32)], st),
        "kk_nn_status": ([ctypes.POINTER(ctypes.c_int32)], st),
        "kk_net_set_params": ([vp, vp, vp], st),
        "kk_net_forward": ([vp, ctypes.c_int32, vp, vp, vp, vp], st),
        "kk_net_loss_grad": ([vp, ctypes.c_int32, vp, vp, vp, vp, vp, vp, vp, vp], st),
        "kk_net_adam": ([vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                         ctypes.c_float, vp], st),
        "kk_net_save": ([vp, ctypes.c_char_p, vp], st),
        "kk_net_load": ([vp, ctypes.c_char_p, vp], st),
        "kk_net_judge_filter": ([vp, vp, vp, ctypes.c_float, vp], st),
        "kk_net_judge": ([vp, ctypes.c_int32, vp, vp, vp, vp], st),
        "kk_net_image_scale": ([vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, vp], st),
        "kk_nn_conv3x3": ([vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp,
                           ctypes.c_int32, vp, ctypes.c_int32, vp, vp, vp], st),
        "kk_nn_conv3x3_dgrad": ([vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp,
                                 ctypes.c_int32, vp, vp, vp], st),
        "kk_nn_conv3x3_wgrad_workspace": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)], st),
        "kk_nn_conv3x3_wgrad": ([vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp,
                                 ctypes.c_int32, vp, vp, vp, vp], st),
        "kk_quality_create": ([pp, ctypes.POINTER(kk_quality_desc)], st),
        "kk_quality_destroy": ([vp], None),
        "kk_quality_gcnr": ([vp, vp, ctypes.c_int32, vp, vp], st),
        "kk_quality_fwhm": ([vp, vp, ctypes.c_int32, vp, vp], st),
        "kk_stream_create": ([pp, vp, ctypes.c_int32, ctypes.c_int32], st),
        "kk_stream_push": ([vp, ctypes.c_int32, vp, vp], st),
        "kk_stream_push_many": ([vp, ctypes.c_int32, ctypes.c_int32, vp, vp], st),
        "kk_stream_end_frame": ([vp, vp, vp], st),
        "kk_stream_wait": ([vp, vp], st),
        "kk_stream_after": ([vp, vp], st),
        "kk_stream_sync": ([vp], st),
        "kk_stream_get_info": ([vp, ctypes.POINTER(kk_stream_info)], st),
        "kk_stream_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status: int):
    if status != KK_OK:
        raise KKError(status, load().kk_last_error().decode())


def _ptr(t) -> ctypes.c_void_p:
    """Device pointer of a contiguous CUDA torch tensor (None -> NULL)."""
    if t is None:
        return ctypes.c_void_p(0)
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous (the C ABI takes dense row-major buffers)")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous host tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def kk_version() -> str:
    return load().kk_version().decode()


def kk_scheme_angles(kind: int, n_tx: int, dtheta: float, M: int, j: float = 0.0, tx=None):
    """Receive angles of one scheme (host call into the library)."""
    out = np.empty(M, dtype=np.float64)
    txa = _f64(tx) if tx is not None else None
    _check(load().kk_scheme_angles(int(kind), int(n_tx),
                                   txa.ctypes.data_as(_dp) if txa is not None else None,
                                   float(dtheta), int(M), float(j), out.ctypes.data_as(_dp)))
    return out


def _desc(elem_x, tx_angles, grid, c, fs, n_samples, rf_dtype, rx_angles=None, pairs=None,
          group_of_pair=None, n_groups=1, compound=KK_COMPOUND_NONE, precision=KK_PREC_F32,
          device=0, pair_weight=None, f_number=0.0, aperture=KK_APERTURE_BOXCAR, elem_y=None,
          tx_angles_y=None, rx_angles_y=None, grid_y=None):
    keep = []
    ex = _f64(elem_x); keep.append(ex)
    tx = _f64(tx_angles); keep.append(tx)
    d = kk_plan_desc()
    d.n_elem = ex.shape[0]
    d.elem_x = ex.ctypes.data_as(_dp)
    d.n_tx = tx.shape[0]
    d.tx_angles = tx.ctypes.data_as(_dp)
    if rx_angles is not None:
        rx = _f64(rx_angles); keep.append(rx)
        d.n_rx = rx.shape[0]
        d.rx_angles = rx.ctypes.data_as(_dp)
    if pairs is not None:
        pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2); keep.append(pr)
        d.n_pairs = pr.shape[0]
        d.pairs = pr.ctypes.data_as(_ip)
    if group_of_pair is not None:
        gp = np.ascontiguousarray(group_of_pair, dtype=np.int32); keep.append(gp)
        d.group_of_pair = gp.ctypes.data_as(_ip)
    d.n_groups = int(n_groups)
    d.compound = int(compound)
    nx, nz, x0, dx, z0, dz = grid
    d.grid = kk_grid(int(nx), int(nz), float(x0), float(dx), float(z0), float(dz))
    d.c, d.fs = float(c), float(fs)
    d.n_samples = int(n_samples)
    d.rf_dtype = int(rf_dtype)
    d.precision = int(precision)
    d.device = int(device)
    if pair_weight is not None:
        pw = _f64(pair_weight); keep.append(pw)
        d.pair_weight = pw.ctypes.data_as(_dp)
    d.f_number = float(f_number)
    d.aperture = int(aperture)
    for name, arr in (("elem_y", elem_y), ("tx_angles_y", tx_angles_y), ("rx_angles_y", rx_angles_y)):
        if arr is not None:
            a = _f64(arr); keep.append(a)
            setattr(d, name, a.ctypes.data_as(_dp))
    if grid_y is not None:
        d.ny, d.y0, d.dy = int(grid_y[0]), float(grid_y[1]), float(grid_y[2])
    return d, keep


def kk_plan_create(desc: kk_plan_desc) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().kk_plan_create(ctypes.byref(h), ctypes.byref(desc)))
    return h


def das_plan_create(desc: kk_plan_desc) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().das_plan_create(ctypes.byref(h), ctypes.byref(desc)))
    return h


def kk_plan_destroy(h):
    if h:
        load().kk_plan_destroy(h)


def kk_plan_get_info(h) -> kk_plan_info:
    info = kk_plan_info()
    _check(load().kk_plan_get_info(h, ctypes.byref(info)))
    return info


def kk_plan_set_gather(h, rows: int, stage: int):
    _check(load().kk_plan_set_gather(h, int(rows), int(stage)))


def kk_plan_set_trim(h, on: bool):
    _check(load().kk_plan_set_trim(h, int(on)))



def kk_plan_status(h) -> int:
    """Device status word (KK_OK or KK_ERR_TIMEOUT); synchronises and resets it."""
    v = ctypes.c_int32()
    _check(load().kk_plan_status(h, ctypes.byref(v)))
    return int(v.value)


def kk_plan_check_wait_timeout(h, limit_ns: int, stream=None):
    """Run the bounded device wait on an mbarrier nothing signals (limit in
    ns): the plan's status word then reads KK_ERR_TIMEOUT."""
    _check(load().kk_plan_check_wait_timeout(h, int(limit_ns), _stream(stream)))


def kk_debug_bounds() -> int:
    """Failed gather-index checks since the last call (bounds-checked build;
    raises KKError(KK_ERR_UNSUPPORTED) in the product build)."""
    v = ctypes.c_int64()
    _check(load().kk_debug_bounds(ctypes.byref(v)))
    return int(v.value)


def kk_decompose(h, rf, rf_theta, workspace, stream=None):
    _check(load().kk_decompose(h, _ptr(rf), _ptr(rf_theta), _ptr(workspace), _stream(stream)))


def kk_spectrum(h, rf, X, stream=None):
    _check(load().kk_spectrum(h, _ptr(rf), _ptr(X), _stream(stream)))


def kk_shear(h, X, Y, stream=None):
    _check(load().kk_shear(h, _ptr(X), _ptr(Y), _stream(stream)))


def kk_inverse(h, Y, rf_theta, stream=None):
    _check(load().kk_inverse(h, _ptr(Y), _ptr(rf_theta), _stream(stream)))


def kk_beamform(h, rf_theta, B, I=None, workspace=None, stream=None):
    _check(load().kk_beamform(h, _ptr(rf_theta), _ptr(B), _ptr(I), _ptr(workspace),
                              _stream(stream)))


def kk_beamform_noalloc(h, rf_theta, B, I=None, stream=None):
    """kk_beamform without a workspace: the library's fixed device scratch is
    used instead (for callers that cannot allocate device memory)."""
    _check(load().kk_beamform_noalloc(h, _ptr(rf_theta), _ptr(B), _ptr(I), _stream(stream)))


def das_beamform(h, rf, B, I=None, workspace=None, stream=None):
    _check(load().das_beamform(h, _ptr(rf), _ptr(B), _ptr(I), _ptr(workspace), _stream(stream)))


def kk_run_host_scratch_size(h) -> int:
    n = ctypes.c_size_t()
    _check(load().kk_run_host_scratch_size(h, ctypes.byref(n)))
    return int(n.value)


def kk_run_host(h, h_rf, h_B, h_I, scratch, stream=None):
    """h_rf/h_B/h_I: CPU tensors (pinned for asynchronous copies)."""
    _check(load().kk_run_host(h, _host_ptr(h_rf), _host_ptr(h_B), _host_ptr(h_I),
                              _ptr(scratch), _stream(stream)))


class Plan:
    """Owner of a KK or DAS plan handle, with device buffers sized from it."""

    def __init__(self, elem_x, tx_angles, grid, c, fs, n_samples, rf_dtype=KK_RF_F32,
                 rx_angles=None, pairs=None, group_of_pair=None, n_groups=1,
                 compound=KK_COMPOUND_NONE, precision=KK_PREC_F32, device=0, das=False,
                 pair_weight=None, f_number=0.0, aperture=KK_APERTURE_BOXCAR, elem_y=None,
                 tx_angles_y=None, rx_angles_y=None, grid_y=None):
        """Volumetric plans (2D array, tilts about both axes, y slices): give
        elem_y, tx_angles_y, rx_angles_y and grid_y = (ny, y0, dy); images are
        then [J][ny][nz][nx] and intensities [ny][nz][nx]."""
        self.desc, self._keep = _desc(elem_x, tx_angles, grid, c, fs, n_samples, rf_dtype,
                                      rx_angles, pairs, group_of_pair, n_groups, compound,
                                      precision, device, pair_weight, f_number, aperture, elem_y,
                                      tx_angles_y, rx_angles_y, grid_y)
        self.handle = das_plan_create(self.desc) if das else kk_plan_create(self.desc)
        self.info = kk_plan_get_info(self.handle)
        self.is_das = das
        self.device = device

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                kk_plan_destroy(h)
            except Exception:
                pass
            self.handle = None

    # buffer helpers (torch allocations; torch is plumbing for device memory)
    def empty_workspace(self):
        import torch
        n = max(int(self.info.workspace_bytes), 256)
        return torch.empty(n, dtype=torch.uint8, device=f"cuda:{self.device}")

    def empty_rf_theta(self):
        import torch
        return torch.empty((self.info.n_pairs, self.info.n_samples, 2), dtype=torch.float32,
                           device=f"cuda:{self.device}")

    def empty_image(self):
        import torch
        J = 1 if self.is_das else self.info.n_groups
        shape = ((J, self.info.ny, self.info.nz, self.info.nx, 2) if self.info.is_volume
                 else (J, self.info.nz, self.info.nx, 2))
        return torch.empty(shape, dtype=torch.float32, device=f"cuda:{self.device}")

    def empty_intensity(self):
        import torch
        shape = ((self.info.ny, self.info.nz, self.info.nx) if self.info.is_volume
                 else (self.info.nz, self.info.nx))
        return torch.empty(shape, dtype=torch.float32, device=f"cuda:{self.device}")

    def set_gather(self, rows: int, stage: int):
        kk_plan_set_gather(self.handle, rows, stage)
        self.info = kk_plan_get_info(self.handle)

    def set_trim(self, on: bool = True):
        """Store only the record samples the grid's image formation can read."""
        kk_plan_set_trim(self.handle, on)
        self.info = kk_plan_get_info(self.handle)

    def status(self) -> int:
        return kk_plan_status(self.handle)

    def decompose(self, rf, rf_theta, workspace, stream=None):
        kk_decompose(self.handle, rf, rf_theta, workspace, stream)

    def beamform(self, rf_theta, B, I=None, workspace=None, stream=None):
        kk_beamform(self.handle, rf_theta, B, I, workspace, stream)

    def das(self, rf, B, I=None, workspace=None, stream=None):
        das_beamform(self.handle, rf, B, I, workspace, stream)

    def spectrum(self, rf, X, stream=None):
        kk_spectrum(self.handle, rf, X, stream)

    def shear(self, X, Y, stream=None):
        kk_shear(self.handle, X, Y, stream)

    def inverse(self, Y, rf_theta, stream=None):
        kk_inverse(self.handle, Y, rf_theta, stream)

    def run_host(self, h_rf, h_B, h_I, scratch, stream=None):
        kk_run_host(self.handle, h_rf, h_B, h_I, scratch, stream)

    def scratch_bytes(self) -> int:
        return kk_run_host_scratch_size(self.handle)


class Batch:
    """Owner of a kk_batch: many frames (each a Plan with its own buffers) in
    one CUDA graph with a persistent image-formation launch."""

    def __init__(self, frames, shape: int = 0, stream=None):
        """frames: list of dicts with keys plan, rf, rf_theta, B, I (or None),
        workspace (torch CUDA tensors).  shape 0 = autotune."""
        self._frames = frames          # keep the tensors alive
        arr = (kk_batch_frame * len(frames))()
        for k, f in enumerate(frames):
            arr[k] = kk_batch_frame(f["plan"].handle, _ptr(f["rf"]).value, _ptr(f["rf_theta"]).value,
                                    _ptr(f["B"]).value, _ptr(f.get("I")).value or None,
                                    _ptr(f["workspace"]).value)
        h = ctypes.c_void_p()
        _check(load().kk_batch_create(ctypes.byref(h), arr, len(frames), int(shape), _stream(stream)))
        self.handle = h
        self.info = kk_batch_info()
        _check(load().kk_batch_get_info(h, ctypes.byref(self.info)))

    def run(self, stream=None):
        _check(load().kk_batch_run(self.handle, _stream(stream)))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                load().kk_batch_destroy(h)
            except Exception:
                pass
            self.handle = None


def kk_simulate_rf(tx_angles, elem_x, n_samples, scatterers, fs, c, f0=5e6, bw=0.6,
                   noise_sigma=0.0, seed=0, out=None, stream=None):
    """GPU synthetic RF (input generation).  scatterers: CUDA float32 [n][4]
    (x, z, amplitude, unused) or [n][3]; returns / fills float32 [N][L][T]."""
    import torch
    dev = scatterers.device if hasattr(scatterers, "device") else torch.device("cuda")
    tx = torch.as_tensor(np.asarray(tx_angles, dtype=np.float64))
    sc = torch.stack([torch.sin(tx), torch.cos(tx)], -1).float().contiguous().to(dev)
    ex = torch.as_tensor(np.asarray(elem_x, dtype=np.float32)).contiguous().to(dev)
    sct = scatterers.float()
    if sct.shape[1] == 3:
        sct = torch.cat([sct, torch.zeros_like(sct[:, :1])], 1)
    sct = sct.contiguous()
    N, L = sc.shape[0], ex.shape[0]
    if out is None:
        out = torch.empty((N, L, int(n_samples)), dtype=torch.float32, device=dev)
    _check(load().kk_simulate_rf(N, _ptr(sc), L, _ptr(ex), int(n_samples), float(fs), float(c),
                                 float(f0), float(bw), int(sct.shape[0]), _ptr(sct),
                                 float(noise_sigma), int(seed) & (2**64 - 1), _ptr(out),
                                 _stream(stream)))
    return out


# --------------------------------------------------------------------------
# learned refiner (include/kknet.h)
# --------------------------------------------------------------------------
def kk_nn_conv3x3(x, w, bias=None, relu=False, y=None, yf=None, stream=None):
    """x [n][h][w][cin] bf16, w [cout][3][3][cin] bf16 (CUDA, contiguous)."""
    n, h, wd, cin = x.shape
    cout = w.shape[0]
    _check(load().kk_nn_conv3x3(_ptr(x), n, h, wd, cin, _ptr(w), cout, _ptr(bias), int(bool(relu)), _ptr(y),
                                _ptr(yf), _stream(stream)))


def kk_nn_status() -> int:
    """Status word of the layer calls' tensor-core kernels (read and reset)."""
    v = ctypes.c_int32()
    _check(load().kk_nn_status(ctypes.byref(v)))
    return v.value


def kk_nn_conv3x3_dgrad(dy, w, dx, stream=None):
    """dx [n][h][w][cin] = adjoint in x of conv3x3 applied to dy [n][h][w][cout]."""
    import torch
    n, h, wd, cout = dy.shape
    cin = w.shape[3]
    ws = torch.empty(cout * 9 * cin, dtype=torch.bfloat16, device=dy.device)
    _check(load().kk_nn_conv3x3_dgrad(_ptr(dy), n, h, wd, cout, _ptr(w), cin, _ptr(dx), _ptr(ws),
                                      _stream(stream)))


def kk_nn_conv3x3_wgrad(x, dy, dw, db=None, stream=None):
    import torch
    n, h, wd, cin = x.shape
    cout = dy.shape[3]
    nb = ctypes.c_size_t()
    _check(load().kk_nn_conv3x3_wgrad_workspace(n, h, wd, cin, cout, ctypes.byref(nb)))
    ws = torch.empty(max(nb.value // 4, 1), dtype=torch.float32, device=x.device)
    _check(load().kk_nn_conv3x3_wgrad(_ptr(x), n, h, wd, cin, _ptr(dy), cout, _ptr(dw), _ptr(db), _ptr(ws),
                                      _stream(stream)))


def kk_net_image_scale(img, out=None, stream=None):
    """img [nb][h][w][2] float32 (complex) -> [nb] float32 of 1 / rms."""
    import torch
    nb, h, w = img.shape[0], img.shape[1], img.shape[2]
    if out is None:
        out = torch.empty(nb, dtype=torch.float32, device=img.device)
    _check(load().kk_net_image_scale(_ptr(img), nb, h, w, _ptr(out), _stream(stream)))
    return out


class Net:
    """Owner of a kk_net handle (the refiner network) with the ABI's calls as
    methods.  Images are CUDA float32 tensors [nb][H][W][2] (complex)."""

    def __init__(self, max_batch: int, height: int, width: int, base_channels: int = 32, seed: int = 0):
        d = kk_net_desc(int(max_batch), int(height), int(width), int(base_channels), int(seed) & (2**64 - 1))
        h = ctypes.c_void_p()
        _check(load().kk_net_create(ctypes.byref(h), ctypes.byref(d)))
        self.handle = h
        self.max_batch, self.height, self.width, self.base_channels = max_batch, height, width, base_channels

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                load().kk_net_destroy(h)
            except Exception:
                pass
            self.handle = None

    def info(self):
        n, st = ctypes.c_int64(), ctypes.c_int64()
        _check(load().kk_net_info(self.handle, ctypes.byref(n), ctypes.byref(st)))
        return n.value, st.value

    def status(self) -> int:
        """Status word of the net's tensor-core kernels (read and reset)."""
        v = ctypes.c_int32()
        _check(load().kk_net_status(self.handle, ctypes.byref(v)))
        return v.value

    @property
    def n_params(self) -> int:
        return self.info()[0]

    @property
    def step(self) -> int:
        return self.info()[1]

    def get_params(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(load().kk_net_get_params(self.handle, _ptr(out), _stream(stream)))
        return out

    def set_params(self, params, stream=None):
        _check(load().kk_net_set_params(self.handle, _ptr(params), _stream(stream)))

    def forward(self, x, in_scale=None, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(x)
        _check(load().kk_net_forward(self.handle, x.shape[0], _ptr(x), _ptr(in_scale), _ptr(out),
                                     _stream(stream)))
        return out

    def loss_grad(self, x, target, in_scale=None, target_scale=None, loss=None, grad=None, out=None,
                  stream=None):
        import torch
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=x.device)
        _check(load().kk_net_loss_grad(self.handle, x.shape[0], _ptr(x), _ptr(in_scale), _ptr(target),
                                       _ptr(target_scale), _ptr(loss), _ptr(grad), _ptr(out),
                                       _stream(stream)))
        return loss

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
        _check(load().kk_net_adam(self.handle, float(lr), float(beta1), float(beta2), float(eps),
                                  float(weight_decay), _stream(stream)))

    def save(self, path, stream=None):
        _check(load().kk_net_save(self.handle, os.fsencode(path), _stream(stream)))

    def load(self, path, stream=None):
        _check(load().kk_net_load(self.handle, os.fsencode(path), _stream(stream)))

    def judge_filter(self, psf_c, psf_f, rho=0.1, stream=None):
        _check(load().kk_net_judge_filter(self.handle, _ptr(psf_c), _ptr(psf_f), float(rho), _stream(stream)))

    def judge(self, out, xc, stat=None, stream=None):
        """[nb][2] float32: (consistency residual, out-of-band fraction)."""
        import torch
        if stat is None:
            stat = torch.empty((out.shape[0], 2), dtype=torch.float32, device=out.device)
        _check(load().kk_net_judge(self.handle, out.shape[0], _ptr(out), _ptr(xc), _ptr(stat), _stream(stream)))
        return stat


def _region(r) -> kk_region:
    kind, a, b, c, d = r
    return kk_region(int(kind), float(a), float(b), float(c), float(d))


def kk_quality_create(desc: kk_quality_desc) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().kk_quality_create(ctypes.byref(h), ctypes.byref(desc)))
    return h


def kk_quality_destroy(h):
    if h:
        load().kk_quality_destroy(h)


def kk_quality_gcnr(h, images, n_images, out, stream=None):
    _check(load().kk_quality_gcnr(h, _ptr(images), int(n_images), _ptr(out), _stream(stream)))


def kk_quality_fwhm(h, images, n_images, out, stream=None):
    _check(load().kk_quality_fwhm(h, _ptr(images), int(n_images), _ptr(out), _stream(stream)))


class Quality:
    """Owner of a ``kk_quality`` handle: gCNR region pairs and FWHM targets on one grid.

    ``inside`` / ``outside``: sequences of ``(kind, a, b, c, d)`` regions
    (metres); ``targets``: sequences of ``(ix, iz, wx, wz)`` pixel windows.
    """

    def __init__(self, grid, inside=(), outside=(), targets=(), n_bins: int = 256,
                 image_kind: int = KK_IMAGE_COMPLEX, device: int = 0):
        if len(inside) != len(outside):
            raise ValueError("inside and outside need the same number of regions")
        nx, nz, x0, dx, z0, dz = grid
        self.grid = tuple(grid)
        self.n_contrast = len(inside)
        self.n_targets = len(targets)
        self.image_kind = int(image_kind)
        rin = (kk_region * max(1, self.n_contrast))(*[_region(r) for r in inside])
        rout = (kk_region * max(1, self.n_contrast))(*[_region(r) for r in outside])
        tg = (kk_target * max(1, self.n_targets))(*[kk_target(*(int(v) for v in t)) for t in targets])
        d = kk_quality_desc(kk_grid(int(nx), int(nz), float(x0), float(dx), float(z0), float(dz)),
                            self.image_kind, self.n_contrast, rin, rout, int(n_bins), self.n_targets,
                            tg, int(device))
        self.h = None
        self.h = kk_quality_create(d)

    def __del__(self):
        try:
            if self.h:
                kk_quality_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def _n_images(self, images):
        nx, nz = self.grid[0], self.grid[1]
        per = nx * nz * (2 if self.image_kind == KK_IMAGE_COMPLEX else 1)
        if images.dtype.itemsize != 4 or images.numel() % per:
            raise ValueError("images must be float32 / complex64 [n][nz][nx] on the plan's grid")
        return images.numel() // per

    def gcnr(self, images, out=None, stream=None):
        """float64 ``[n_images][n_contrast]`` gCNR (device tensor)."""
        import torch
        n = self._n_images(images)
        if out is None:
            out = torch.empty((n, self.n_contrast), dtype=torch.float64, device=images.device)
        kk_quality_gcnr(self.h, images, n, out, stream)
        return out

    def fwhm(self, images, out=None, stream=None):
        """Raw ``[n_images][n_targets][32]`` uint8 device tensor of kk_fwhm_result
        records; ``decode_fwhm`` turns it into a numpy structured array."""
        import torch
        n = self._n_images(images)
        if out is None:
            out = torch.empty((n, self.n_targets, FWHM_DTYPE.itemsize), dtype=torch.uint8,
                              device=images.device)
        kk_quality_fwhm(self.h, images, n, out, stream)
        return out


def decode_fwhm(raw) -> np.ndarray:
    """numpy structured array (``FWHM_DTYPE``) of a raw kk_fwhm_result tensor."""
    a = raw.detach().cpu().contiguous().numpy()
    return np.frombuffer(a.tobytes(), dtype=FWHM_DTYPE).reshape(a.shape[:-1])


# --------------------------------------------------------------------------
# streaming decomposition (include/kkstream.h)
# --------------------------------------------------------------------------
def kk_stream_create(plan_handle, group: int, ring_groups: int = 2) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().kk_stream_create(ctypes.byref(h), plan_handle, int(group), int(ring_groups)))
    return h


def kk_stream_push(h, tx_row: int, h_event=None, d_event=None):
    """h_event: pinned host tensor (or None); d_event: CUDA tensor (or None)."""
    _check(load().kk_stream_push(h, int(tx_row), _host_ptr(h_event), _ptr(d_event)))


def kk_stream_push_many(h, first_row: int, h_events=None, d_events=None):
    """Rows first_row.. from a [n][L][T] block (pinned host or CUDA tensor)."""
    n = (h_events if h_events is not None else d_events).shape[0]
    _check(load().kk_stream_push_many(h, int(first_row), int(n), _host_ptr(h_events), _ptr(d_events)))


def kk_stream_end_frame(h, B, I=None):
    _check(load().kk_stream_end_frame(h, _ptr(B), _ptr(I)))


def kk_stream_wait(h, stream=None):
    _check(load().kk_stream_wait(h, _stream(stream)))


def kk_stream_after(h, stream=None):
    _check(load().kk_stream_after(h, _stream(stream)))


def kk_stream_sync(h):
    _check(load().kk_stream_sync(h))


def kk_stream_get_info(h) -> kk_stream_info:
    info = kk_stream_info()
    _check(load().kk_stream_get_info(h, ctypes.byref(info)))
    return info


def kk_stream_destroy(h):
    if h:
        load().kk_stream_destroy(h)


class Stream:
    """Owner of a ``kk_stream`` handle on a KK ``Plan`` (kept alive by this object)."""

    def __init__(self, plan: "Plan", group: int, ring_groups: int | None = None):
        """ring_groups defaults to a frame's groups plus one."""
        self.plan = plan
        self.h = None
        if ring_groups is None:   # invalid group sizes are left to the library to reject
            ring_groups = min(64, max(2, -(-plan.info.n_tx_used // int(group)) + 1)) if group >= 1 else 2
        self.h = kk_stream_create(plan.handle, group, ring_groups)

    def __del__(self):
        try:
            if self.h:
                kk_stream_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def push(self, tx_row: int, h_event=None, d_event=None):
        kk_stream_push(self.h, tx_row, h_event, d_event)

    def push_many(self, first_row: int, h_events=None, d_events=None):
        kk_stream_push_many(self.h, first_row, h_events, d_events)

    def end_frame(self, B, I=None):
        kk_stream_end_frame(self.h, B, I)

    def wait(self, stream=None):
        kk_stream_wait(self.h, stream)

    def after(self, stream=None):
        kk_stream_after(self.h, stream)

    def sync(self):
        kk_stream_sync(self.h)

    @property
    def info(self) -> kk_stream_info:
        return kk_stream_get_info(self.h)
