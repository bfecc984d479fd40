"""Image-quality study of KK beamforming against DAS: gCNR and FWHM.

The paper compares its receive-angle schemes with DAS by the contrast of an
anechoic inclusion (gCNR, Section III, Fig. 5), by the width and separability
of wire targets (Fig. 4) and by trading transmit angles for receive angles
(Fig. 6).  This module repeats those comparisons on synthetic phantoms
simulated on the GPU with the acquisition parameters of Table 1 (192
elements, 0.23 mm pitch, 5.2 MHz, 20.83 MHz sampling, 48 deg of transmit
range, 0.057 x 0.037 mm pixels), beamforms every variant with the library and
measures it with ``kk_quality_*``.  It reports what holds and what does not;
it asserts nothing.

Variants (N transmits evenly over +-24 deg, M receive angles, L/M the
compression factor):
  * DAS with all 192 elements (N = 15 and N = 7);
  * Eq. (uniform) with j = 0, 3, 6 at M = 7 and M = 19;
  * Eq. (confocal) at M = 21 and M = 57;
  * the j = 0, 3, 6 panels compounded coherently and incoherently (hybrid,
    Eqs. (coherent)/(incoherent)), M = 21 and 57 overall;
  * N = 7 with j = 0 at M = 19 and M = 57.

Phantom per realization: N(0,1) speckle at 100 per mm^2, three anechoic
cysts of 2 mm radius, eight bright wires, 30 dB white channel noise.

Run: ``python -m paper_2603_22496_gb300.quality [--realizations R (32)] [--json out.json]``.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import sys
import time

import numpy as np

from . import (KK_COMPOUND_COHERENT, KK_COMPOUND_INCOHERENT, KK_IMAGE_INTENSITY, KK_REGION_ANNULUS,
               KK_REGION_DISK, KK_RF_F32, KK_SCHEME_CONFOCAL, KK_SCHEME_SHIFTED, Plan, Quality,
               decode_fwhm, kk_scheme_angles, kk_simulate_rf, load)


@dataclasses.dataclass(frozen=True)
class Acquisition:
    """Table 1 parameters; the 48 deg angular range is read as +-24 deg."""
    n_elem: int = 192
    pitch: float = 0.23e-3
    f0: float = 5.2e6
    fs: float = 20.83e6
    c: float = 1540.0
    theta_max_deg: float = 24.0
    n_samples: int = 2048
    nx: int = 360
    dx: float = 0.057e-3
    nz: int = 800
    dz: float = 0.037e-3
    z0: float = 5e-3

    @property
    def grid(self):
        x0 = -self.dx * (self.nx - 1) / 2
        return (self.nx, self.nz, x0, self.dx, self.z0, self.dz)

    def elem_x(self):
        return (np.arange(self.n_elem) - (self.n_elem - 1) / 2.0) * self.pitch

    def tx(self, n_tx):
        return np.deg2rad(np.linspace(-self.theta_max_deg, self.theta_max_deg, n_tx))


CYSTS_MM = ((-4.0, 14.0), (4.0, 20.0), (0.0, 26.0))
CYST_RADIUS = 2e-3
WIRES_MM = tuple((x, z) for z in (8.0, 31.0) for x in (-6.0, -2.0, 2.0, 6.0))
SPECKLE_PER_MM2 = 100.0
WIRE_AMP = 50.0
SNR_DB = 30.0


def regions():
    """Inside disk (0.75 R) and background annulus (1.25 R .. 1.75 R) per cyst."""
    inside = [(KK_REGION_DISK, cx * 1e-3, cz * 1e-3, 0.75 * CYST_RADIUS, 0.0) for cx, cz in CYSTS_MM]
    outside = [(KK_REGION_ANNULUS, cx * 1e-3, cz * 1e-3, 1.25 * CYST_RADIUS, 1.75 * CYST_RADIUS)
               for cx, cz in CYSTS_MM]
    return inside, outside


def targets(acq: Acquisition):
    """Nearest pixel of each wire and a +-0.5 mm search window."""
    nx, nz, x0, dx, z0, dz = acq.grid
    wx, wz = int(round(0.5e-3 / dx)), int(round(0.5e-3 / dz))
    return [(int(round((x * 1e-3 - x0) / dx)), int(round((z * 1e-3 - z0) / dz)), wx, wz)
            for x, z in WIRES_MM]


def phantom(acq: Acquisition, seed: int):
    """float32 [n][4] (x, z, amplitude, 0) scatterers on the CPU."""
    rng = np.random.default_rng(seed)
    xmax = acq.dx * (acq.nx - 1) / 2 + 1e-3
    zlo, zhi = acq.z0 - 1e-3, acq.z0 + acq.dz * (acq.nz - 1) + 1e-3
    ns = int(SPECKLE_PER_MM2 * (2 * xmax * 1e3) * ((zhi - zlo) * 1e3))
    sx = rng.uniform(-xmax, xmax, ns)
    sz = rng.uniform(zlo, zhi, ns)
    keep = np.ones(ns, dtype=bool)
    for cx, cz in CYSTS_MM:
        keep &= (sx - cx * 1e-3) ** 2 + (sz - cz * 1e-3) ** 2 > CYST_RADIUS ** 2
    wx = np.array([w[0] for w in WIRES_MM]) * 1e-3
    wz = np.array([w[1] for w in WIRES_MM]) * 1e-3
    x = np.concatenate([sx[keep], wx])
    z = np.concatenate([sz[keep], wz])
    a = np.concatenate([rng.standard_normal(int(keep.sum())), np.full(wx.size, WIRE_AMP)])
    return np.stack([x, z, a, np.zeros_like(x)], 1).astype(np.float32)


def simulate(acq: Acquisition, n_tx: int, scat, seed: int):
    """GPU channel data [N][L][T] float32 with white noise at SNR_DB."""
    import torch
    rf = kk_simulate_rf(acq.tx(n_tx), acq.elem_x(), acq.n_samples, scat, acq.fs, acq.c, f0=acq.f0)
    rms = float(rf.pow(2).mean().sqrt())
    return kk_simulate_rf(acq.tx(n_tx), acq.elem_x(), acq.n_samples, scat, acq.fs, acq.c, f0=acq.f0,
                          noise_sigma=rms * 10 ** (-SNR_DB / 20), seed=seed, out=rf)


def variants():
    """(name, n_tx, kind, spec): kind 'das' or 'kk'; spec = list of (scheme, M, j) groups + compound."""
    v = [("DAS N=15", 15, "das", None)]
    for M in (7, 19):
        for j in (0, 3, 6):
            v.append((f"KK j={j} M={M}", 15, "kk", ([(KK_SCHEME_SHIFTED, M, j)], KK_COMPOUND_COHERENT)))
        grp = [(KK_SCHEME_SHIFTED, M, j) for j in (0, 3, 6)]
        v.append((f"KK confocal M={3 * M}", 15, "kk", ([(KK_SCHEME_CONFOCAL, 3 * M, 0)], KK_COMPOUND_COHERENT)))
        v.append((f"KK hybrid coherent M={3 * M}", 15, "kk", (grp, KK_COMPOUND_COHERENT)))
        v.append((f"KK hybrid incoherent M={3 * M}", 15, "kk", (grp, KK_COMPOUND_INCOHERENT)))
    v.append(("DAS N=7", 7, "das", None))
    for M in (19, 57):
        v.append((f"KK N=7 j=0 M={M}", 7, "kk", ([(KK_SCHEME_SHIFTED, M, 0)], KK_COMPOUND_COHERENT)))
    return v


def make_plan(acq: Acquisition, n_tx: int, kind: str, spec):
    tx = acq.tx(n_tx)
    if kind == "das":
        return Plan(acq.elem_x(), tx, acq.grid, acq.c, acq.fs, acq.n_samples, KK_RF_F32, das=True), acq.n_elem
    groups, compound = spec
    dth = float(tx[1] - tx[0])
    rx, pairs, grp = [], [], []
    for g, (scheme, M, j) in enumerate(groups):
        base = sum(len(r) for r in rx)
        rx.append(kk_scheme_angles(scheme, n_tx, dth, M, j))
        pairs += [(i, base + o) for i in range(n_tx) for o in range(M)]
        grp += [g] * (n_tx * M)
    rx = np.concatenate(rx)
    plan = Plan(acq.elem_x(), tx, acq.grid, acq.c, acq.fs, acq.n_samples, KK_RF_F32, rx_angles=rx,
                pairs=np.array(pairs, np.int32), group_of_pair=np.array(grp, np.int32),
                n_groups=len(groups), compound=compound)
    return plan, rx.shape[0]


def run(realizations: int = 32, seed0: int = 9000, acq: Acquisition = Acquisition(), log=print):
    """Per variant: mean gCNR over cysts and realizations, mean lateral and
    axial FWHM over wires and realizations (mm), and the compression factor."""
    import torch
    load()
    inside, outside = regions()
    q = Quality(acq.grid, inside, outside, targets(acq), n_bins=256, image_kind=KK_IMAGE_INTENSITY)
    vs = variants()
    plans = {}
    res = {name: {"gcnr": [], "lateral_mm": [], "axial_mm": []} for name, *_ in vs}
    t0 = time.time()
    for r in range(realizations):
        scat = torch.from_numpy(phantom(acq, seed0 + r)).cuda()
        rf = {n: simulate(acq, n, scat, seed0 + 100 * r + n) for n in (15, 7)}
        for name, n_tx, kind, spec in vs:
            if name not in plans:
                plans[name] = make_plan(acq, n_tx, kind, spec)
            plan, m_used = plans[name]
            ws, B, I = plan.empty_workspace(), plan.empty_image(), plan.empty_intensity()
            if kind == "das":
                plan.das(rf[n_tx], B, I, ws)
            else:
                rt = plan.empty_rf_theta()
                plan.decompose(rf[n_tx], rt, ws)
                plan.beamform(rt, B, I, ws)
            g = q.gcnr(I)
            f = decode_fwhm(q.fwhm(I))
            torch.cuda.synchronize()
            res[name]["gcnr"] += g.cpu().numpy().ravel().tolist()
            res[name]["lateral_mm"] += (f["lateral"].ravel() * 1e3).tolist()
            res[name]["axial_mm"] += (f["axial"].ravel() * 1e3).tolist()
            res[name]["M"] = int(m_used)
            res[name]["compression"] = acq.n_elem / m_used
    out = {}
    for name, d in res.items():
        out[name] = {"M": d["M"], "compression": round(d["compression"], 2),
                     "gcnr": float(np.nanmean(d["gcnr"])), "gcnr_sd": float(np.nanstd(d["gcnr"])),
                     "lateral_fwhm_mm": float(np.nanmean(d["lateral_mm"])),
                     "axial_fwhm_mm": float(np.nanmean(d["axial_mm"]))}
    log(f"# {realizations} realizations in {time.time() - t0:.1f} s")
    return out


def claims(t):
    """The paper's qualitative statements, evaluated on the table ``t``."""
    g = {k: v["gcnr"] for k, v in t.items()}
    w = {k: v["lateral_fwhm_mm"] for k, v in t.items()}
    c = []
    for M in (7, 19):
        c.append((f"Fig. 4: j=6 narrows the lateral response (M={M})", w[f"KK j=6 M={M}"] < w[f"KK j=0 M={M}"]))
        c.append((f"Fig. 5: larger j lowers gCNR (M={M})", g[f"KK j=6 M={M}"] < g[f"KK j=0 M={M}"]))
        kk = [k for k in g if k.startswith("KK") and "N=7" not in k and k.endswith(f"M={3 * M}")]
        c.append((f"Fig. 5: incoherent hybrid has the highest gCNR of the M={3 * M} variants",
                  max(kk, key=lambda k: g[k]) == f"KK hybrid incoherent M={3 * M}"))
    c.append(("Fig. 5: incoherent hybrid at M=57 (3.4x) matches or beats DAS",
              g["KK hybrid incoherent M=57"] >= g["DAS N=15"] - 0.02))
    c.append(("Fig. 5: gCNR falls with compression (M=7 below M=19, j=0)", g["KK j=0 M=7"] < g["KK j=0 M=19"]))
    c.append(("Fig. 6: fewer transmits lower gCNR (N=7 below N=15, j=0 M=19)",
              g["KK N=7 j=0 M=19"] < g["KK j=0 M=19"]))
    c.append(("Fig. 6: more receive angles compensate (N=7 M=57 recovers N=15 M=19 within 0.02)",
              g["KK N=7 j=0 M=57"] >= g["KK j=0 M=19"] - 0.02))
    return c


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--realizations", type=int, default=32)
    ap.add_argument("--seed", type=int, default=9000)
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    t = run(a.realizations, a.seed)
    print(f"{'variant':34s} {'M':>4s} {'L/M':>6s} {'gCNR':>7s} {'sd':>6s} {'lat mm':>7s} {'ax mm':>7s}")
    for k, v in t.items():
        print(f"{k:34s} {v['M']:4d} {v['compression']:6.1f} {v['gcnr']:7.3f} {v['gcnr_sd']:6.3f} "
              f"{v['lateral_fwhm_mm']:7.3f} {v['axial_fwhm_mm']:7.3f}")
    cl = claims(t)
    for text, ok in cl:
        print(f"{'holds' if ok else 'does not hold':14s} {text}")
    if a.json:
        with open(a.json, "w") as f:
            json.dump({"table": t, "claims": [{"claim": s, "holds": bool(ok)} for s, ok in cl]}, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
