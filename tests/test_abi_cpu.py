"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports
every symbol the header declares, and its host-only logic is right.  No
compute call is made (there may be no GPU here)."""
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2603_22496_gb300 as kb
from paper_2603_22496_gb300 import build as kbuild
from oracle import schemes

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")
HEADERS = sorted(os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h"))


@pytest.fixture(scope="module")
def lib():
    kbuild.build()
    return kb.load()


def _declared():
    txt = "".join(open(h).read() for h in HEADERS)
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(kk_\w+|das_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", kb.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(\S+)", out))
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    assert sorted(kb.EXPORTS) == declared
    for s in declared:
        assert hasattr(lib, s)


def test_build_targets_sm103a_only():
    assert kbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version_string(lib):
    assert "sm_103a" in kb.kk_version()


@pytest.mark.parametrize("kind,M,j", [("vernier", 11, 0), ("vernier", 16, 0), ("shifted", 15, 3),
                                      ("shifted", 7, 7), ("confocal", 15, 0), ("confocal", 21, 0),
                                      ("confocal", 16, 0)])
def test_scheme_angles_match_oracle(lib, kind, M, j):
    N = 15
    tx = np.deg2rad(np.linspace(-12, 12, N))
    dth = schemes.transmit_spacing(tx)
    ref = {"vernier": lambda: schemes.rx_vernier(dth, M),
           "shifted": lambda: schemes.rx_shifted(dth, M, j),
           "confocal": lambda: schemes.rx_confocal(dth, M, N)}[kind]()
    got = kb.kk_scheme_angles({"vernier": kb.KK_SCHEME_VERNIER, "shifted": kb.KK_SCHEME_SHIFTED,
                               "confocal": kb.KK_SCHEME_CONFOCAL}[kind], N, dth, M, j)
    assert np.abs(got - ref).max() <= 1e-15


def test_scheme_angles_rejects_bad_arguments(lib):
    with pytest.raises(kb.KKError) as e:
        kb.kk_scheme_angles(kb.KK_SCHEME_VERNIER, 5, 0.01, 0)
    assert e.value.status == kb.KK_ERR_INVALID_ARG
    with pytest.raises(kb.KKError):
        kb.kk_scheme_angles(kb.KK_SCHEME_CONFOCAL, 1, 0.01, 5)    # floor(N/2) = 0
    with pytest.raises(kb.KKError):
        kb.kk_scheme_angles(kb.KK_SCHEME_SAME, 3, 0.0, 4, tx=np.zeros(3))
    with pytest.raises(kb.KKError):
        kb.kk_scheme_angles(99, 5, 0.01, 5)


def test_plan_validation_is_host_side(lib):
    """Argument errors are reported before any device work."""
    d, keep = kb._desc(np.zeros(4), np.zeros(2), (8, 8, 0.0, 1e-4, 1e-3, 1e-4), 1540.0, 20e6,
                       100, kb.KK_RF_F32, rx_angles=np.zeros(1), pairs=[[0, 0]])
    with pytest.raises(kb.KKError) as e:          # T/2 = 50 is not a supported FFT length
        kb.kk_plan_create(d)
    assert e.value.status in (kb.KK_ERR_UNSUPPORTED, kb.KK_ERR_INVALID_ARG)
    d, keep = kb._desc(np.zeros(4), np.array([1.5]), (8, 8, 0.0, 1e-4, 1e-3, 1e-4), 1540.0, 20e6,
                       256, kb.KK_RF_F32, rx_angles=np.zeros(1), pairs=[[0, 0]])
    with pytest.raises(kb.KKError) as e:          # 86 degree transmit
        kb.kk_plan_create(d)
    assert e.value.status == kb.KK_ERR_INVALID_ARG
    assert kb.load().kk_last_error()


def test_quality_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the plan description / info and of kkquality.h and kkstream.h have the C
    compiler's sizes and offsets."""
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stddef.h>
#include <stdio.h>
#include "kkquality.h"
#include "kkstream.h"
#define P(T, f) printf(#T "." #f " %zu\\n", offsetof(T, f))
int main(void) {
  printf("kk_region %zu\\nkk_target %zu\\nkk_fwhm_result %zu\\nkk_quality_desc %zu\\n",
         sizeof(kk_region), sizeof(kk_target), sizeof(kk_fwhm_result), sizeof(kk_quality_desc));
  P(kk_region, a); P(kk_region, d); P(kk_fwhm_result, peak); P(kk_fwhm_result, lateral);
  P(kk_fwhm_result, axial); P(kk_quality_desc, image_kind); P(kk_quality_desc, inside);
  P(kk_quality_desc, n_bins); P(kk_quality_desc, targets); P(kk_quality_desc, device);
  printf("kk_stream_info %zu\\n", sizeof(kk_stream_info));
  printf("kk_plan_desc %zu\\nkk_plan_info %zu\\n", sizeof(kk_plan_desc), sizeof(kk_plan_info));
  P(kk_plan_desc, aperture); P(kk_plan_desc, elem_y); P(kk_plan_desc, rx_angles_y); P(kk_plan_desc, ny);
  P(kk_plan_desc, dy); P(kk_plan_info, ny); P(kk_plan_info, is_volume); P(kk_plan_info, sep_my);
  P(kk_plan_info, gather_rows); P(kk_plan_info, gather_split);
  P(kk_stream_info, n_groups); P(kk_stream_info, events_pushed); P(kk_stream_info, device_bytes);
  printf("kk_batch_info %zu\\n", sizeof(kk_batch_info));
  P(kk_batch_info, pixel_pairs); P(kk_batch_info, tuned_ms); P(kk_batch_info, n_volume_frames);
  P(kk_batch_info, max_window_volume);
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    import ctypes
    want = {"kk_region": ctypes.sizeof(kb.kk_region), "kk_target": ctypes.sizeof(kb.kk_target),
            "kk_fwhm_result": kb.FWHM_DTYPE.itemsize, "kk_quality_desc": ctypes.sizeof(kb.kk_quality_desc),
            "kk_region.a": kb.kk_region.a.offset, "kk_region.d": kb.kk_region.d.offset,
            "kk_fwhm_result.peak": kb.FWHM_DTYPE.fields["peak"][1],
            "kk_fwhm_result.lateral": kb.FWHM_DTYPE.fields["lateral"][1],
            "kk_fwhm_result.axial": kb.FWHM_DTYPE.fields["axial"][1],
            "kk_quality_desc.image_kind": kb.kk_quality_desc.image_kind.offset,
            "kk_quality_desc.inside": kb.kk_quality_desc.inside.offset,
            "kk_quality_desc.n_bins": kb.kk_quality_desc.n_bins.offset,
            "kk_quality_desc.targets": kb.kk_quality_desc.targets.offset,
            "kk_quality_desc.device": kb.kk_quality_desc.device.offset,
            "kk_stream_info": ctypes.sizeof(kb.kk_stream_info),
            "kk_stream_info.n_groups": kb.kk_stream_info.n_groups.offset,
            "kk_stream_info.events_pushed": kb.kk_stream_info.events_pushed.offset,
            "kk_stream_info.device_bytes": kb.kk_stream_info.device_bytes.offset,
            "kk_plan_desc": ctypes.sizeof(kb.kk_plan_desc), "kk_plan_info": ctypes.sizeof(kb.kk_plan_info),
            "kk_plan_desc.aperture": kb.kk_plan_desc.aperture.offset,
            "kk_plan_desc.elem_y": kb.kk_plan_desc.elem_y.offset,
            "kk_plan_desc.rx_angles_y": kb.kk_plan_desc.rx_angles_y.offset,
            "kk_plan_desc.ny": kb.kk_plan_desc.ny.offset, "kk_plan_desc.dy": kb.kk_plan_desc.dy.offset,
            "kk_plan_info.ny": kb.kk_plan_info.ny.offset, "kk_plan_info.is_volume": kb.kk_plan_info.is_volume.offset,
            "kk_plan_info.sep_my": kb.kk_plan_info.sep_my.offset,
            "kk_plan_info.gather_rows": kb.kk_plan_info.gather_rows.offset,
            "kk_plan_info.gather_split": kb.kk_plan_info.gather_split.offset,
            "kk_batch_info": ctypes.sizeof(kb.kk_batch_info),
            "kk_batch_info.pixel_pairs": kb.kk_batch_info.pixel_pairs.offset,
            "kk_batch_info.tuned_ms": kb.kk_batch_info.tuned_ms.offset,
            "kk_batch_info.n_volume_frames": kb.kk_batch_info.n_volume_frames.offset,
            "kk_batch_info.max_window_volume": kb.kk_batch_info.max_window_volume.offset}
    assert {k: int(v) for k, v in got.items()} == want


@pytest.mark.parametrize("kw", [
    dict(n_bins=0), dict(n_bins=4097), dict(image_kind=2),
    dict(inside=[(3, 0, 0, 1, 0)], outside=[(0, 0, 0, 1, 0)]),              # bad kind
    dict(inside=[(0, 0, 0, -1, 0)], outside=[(0, 0, 0, 1, 0)]),             # negative radius
    dict(inside=[(1, 0, 0, 2, 1)], outside=[(0, 0, 0, 1, 0)]),              # r1 > r2
    dict(inside=[(0, float("nan"), 0, 1, 0)], outside=[(0, 0, 0, 1, 0)]),   # non-finite
    dict(targets=[(1, 1, -1, 2)]),
    dict(grid=(0, 8, 0.0, 1e-4, 0.0, 1e-4)), dict(grid=(8, 8, 0.0, -1e-4, 0.0, 1e-4)),
])
def test_quality_validation_is_host_side(lib, kw):
    args = dict(grid=(8, 8, 0.0, 1e-4, 0.0, 1e-4), inside=(), outside=(), targets=(), n_bins=16,
                image_kind=kb.KK_IMAGE_COMPLEX)
    args.update(kw)
    with pytest.raises(kb.KKError) as e:
        kb.Quality(**args)
    assert e.value.status == kb.KK_ERR_INVALID_ARG


def test_bounds_checked_variant_builds_with_the_same_exports(lib):
    """The KK_DEBUG_BOUNDS variant compiles for sm_103a and exports the same
    symbols; the product build answers kk_debug_bounds with
    KK_ERR_UNSUPPORTED (no device call)."""
    path = kbuild.build(variant="bounds")
    sym = {}
    for p in (kb.library_path(), path):
        out = subprocess.run(["nm", "-D", "--defined-only", p], capture_output=True, text=True, check=True).stdout
        sym[p] = {s for s in re.findall(r"\s[TW]\s+(\S+)", out) if s.startswith(("kk_", "das_"))}
    assert sym[kb.library_path()] == sym[path]
    with pytest.raises(kb.KKError) as e:
        kb.kk_debug_bounds()
    assert e.value.status == kb.KK_ERR_UNSUPPORTED
