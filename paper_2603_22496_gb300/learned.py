"""Learned refiner of compressed-pair-set KK images: training data made by
the method itself, the training loop, inference with the fallback judge.

The workload: a 128-element, 0.3 mm pitch array, 75 plane-wave transmits
over +-16 deg, 2048-sample records at 20 MHz; a 256 x 256 grid at 0.15 mm
from 5 mm depth.  The network's input is the KK image of a 6 x 12 vernier
pair subset (six transmits at a stride of 14 about the centre, twelve
vernier receive angles, Section II-D), its target the KK image of the full
75 x 128 pair set of the same channel data (128 receive angles evenly over
+-16 deg).  Phantoms (one seed each): speckle N(0, 1) at 10 scatterers per
mm^2, 1-8 bright point wires, 0-3 anechoic cysts of radius 1-5 mm, white
noise at an SNR drawn from 20-40 dB; simulated on the GPU
(``kk_simulate_rf``) and beamformed by the plain GPU path.

Every step of the refiner runs in the library (``Net``: forward, loss,
backward, Adam, judge); this module sequences the calls, draws phantoms
and batches, and keeps the training state.  Torch is used only to hold
buffers, to add the input noise and to gather batches.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import time

import numpy as np

from . import (KK_COMPOUND_NONE, KK_PREC_BF16, KK_PREC_F32, KK_RF_F32, KK_SCHEME_SHIFTED, KK_SCHEME_VERNIER, Net,
               Plan, kk_net_image_scale, kk_scheme_angles, kk_simulate_rf, load)

FS = 20e6
C_SOUND = 1540.0


@dataclasses.dataclass(frozen=True)
class Geometry:
    n_elem: int = 128
    pitch: float = 0.3e-3
    n_tx: int = 75
    theta_max_deg: float = 16.0
    n_samples: int = 2048
    nx: int = 256
    nz: int = 256
    d: float = 0.15e-3
    z0: float = 5e-3
    vernier_tx: int = 6
    vernier_rx: int = 12
    full_rx: int = 128
    speckle_per_mm2: float = 10.0

    @property
    def grid(self):
        return (self.nx, self.nz, -self.d * (self.nx - 1) / 2, self.d, self.z0, self.d)

    def elem_x(self):
        return (np.arange(self.n_elem) - (self.n_elem - 1) / 2.0) * self.pitch

    def tx_angles(self):
        return np.deg2rad(np.linspace(-self.theta_max_deg, self.theta_max_deg, self.n_tx))


def vernier_pairs(geo: Geometry):
    """Transmit subset of geo.vernier_tx angles at the widest even stride about
    the centre, vernier receive angles 2 o dtheta / M (Section II-D)."""
    a, N = geo.vernier_tx, geo.n_tx
    s = (N - 1) // (a - 1)
    s -= s % 2
    start = ((N - 1) - (a - 1) * s) // 2
    sub = start + s * np.arange(a)
    tx = geo.tx_angles()
    dth = float(tx[sub[-1]] - tx[sub[0]]) / (a - 1)
    rx = kk_scheme_angles(KK_SCHEME_VERNIER, a, dth, geo.vernier_rx)
    pairs = np.array([(int(i), o) for i in sub for o in range(geo.vernier_rx)], np.int32)
    return rx, pairs


def full_pairs(geo: Geometry):
    rx = np.deg2rad(np.linspace(-geo.theta_max_deg, geo.theta_max_deg, geo.full_rx))
    pairs = np.array([(i, o) for i in range(geo.n_tx) for o in range(geo.full_rx)], np.int32)
    return rx, pairs


def phantom(seed: int, geo: Geometry):
    """Scatterers [n][4] (x, z, amplitude, 0) and the SNR in dB of one seed."""
    sc, snr_db, _ = _phantom(seed, geo)
    return sc, snr_db


def wires(seed: int, geo: Geometry) -> np.ndarray:
    """(x, z) of the point wires of one seed's phantom, [nw][2] metres."""
    return _phantom(seed, geo)[2]


def _phantom(seed: int, geo: Geometry):
    rng = np.random.default_rng(seed)
    nx, nz, x0, dx, z0, dz = geo.grid
    m = 1e-3
    xl, xh, zl, zh = x0 - m, x0 + dx * (nx - 1) + m, z0 - m, z0 + dz * (nz - 1) + m
    ns = int(round(geo.speckle_per_mm2 * (xh - xl) * (zh - zl) * 1e6))
    sx, sz = rng.uniform(xl, xh, ns), rng.uniform(zl, zh, ns)
    amp = rng.standard_normal(ns)
    keep = np.ones(ns, bool)
    for _ in range(int(rng.integers(0, 4))):
        r = rng.uniform(1e-3, 5e-3)
        cx, cz = rng.uniform(x0, x0 + dx * (nx - 1)), rng.uniform(z0, z0 + dz * (nz - 1))
        keep &= (sx - cx) ** 2 + (sz - cz) ** 2 > r * r
    nw = int(rng.integers(1, 9))
    wx = rng.uniform(x0 + m, x0 + dx * (nx - 1) - m, nw)
    wz = rng.uniform(z0 + m, z0 + dz * (nz - 1) - m, nw)
    wa = 10.0 * rng.uniform(0.5, 2.0, nw)
    x = np.concatenate([sx[keep], wx])
    z = np.concatenate([sz[keep], wz])
    a = np.concatenate([amp[keep], wa])
    snr_db = float(rng.uniform(20.0, 40.0))
    return np.stack([x, z, a, np.zeros_like(x)], 1), snr_db, np.stack([wx, wz], 1)


class Synth:
    """Training pairs (compressed image, full image) from the plain GPU path."""

    def __init__(self, geo: Geometry = Geometry(), target_precision: int = KK_PREC_BF16,
                 input_precision: int = KK_PREC_F32):
        import torch
        load()
        self.geo = geo
        self.elem_x, self.tx = geo.elem_x(), geo.tx_angles()
        rc, pc = vernier_pairs(geo)
        rf_, pf = full_pairs(geo)
        self.plan_c = Plan(self.elem_x, self.tx, geo.grid, C_SOUND, FS, geo.n_samples, KK_RF_F32,
                           rx_angles=rc, pairs=pc, compound=KK_COMPOUND_NONE, precision=input_precision)
        self.plan_f = Plan(self.elem_x, self.tx, geo.grid, C_SOUND, FS, geo.n_samples, KK_RF_F32,
                           rx_angles=rf_, pairs=pf, compound=KK_COMPOUND_NONE, precision=target_precision)
        self.bufs = [(p, p.empty_workspace(), p.empty_rf_theta()) for p in (self.plan_c, self.plan_f)]
        self.rf = torch.empty((geo.n_tx, geo.n_elem, geo.n_samples), dtype=torch.float32, device="cuda")

    def images_of(self, rf, out_c, out_f):
        """KK images of one record set with both pair sets, [nz][nx][2] each."""
        for (p, ws, rt), out in zip(self.bufs, (out_c, out_f)):
            p.decompose(rf, rt, ws)
            p.beamform(rt, out, None, ws)

    def simulate(self, seed: int, noise: bool = True):
        import torch
        sc, snr = phantom(seed, self.geo)
        sct = torch.from_numpy(sc).float().cuda()
        kk_simulate_rf(self.tx, self.elem_x, self.geo.n_samples, sct, FS, C_SOUND, out=self.rf)
        if noise:
            rms = self.rf.pow(2).mean().sqrt()
            gen = torch.Generator(device="cuda").manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
            self.rf.add_(torch.randn(self.rf.shape, device="cuda", generator=gen) * (rms * 10 ** (-snr / 20)))
        return self.rf

    def dataset(self, seeds, progress=None):
        """(Xc, Yf): [n][nz][nx][2] float32 each, in HBM."""
        import torch
        g = self.geo
        X = torch.empty((len(seeds), g.nz, g.nx, 2), dtype=torch.float32, device="cuda")
        Y = torch.empty_like(X)
        for k, s in enumerate(seeds):
            self.images_of(self.simulate(int(s)), X[k], Y[k])
            if progress and (k + 1) % progress == 0:
                torch.cuda.synchronize()
                print(f"  simulated {k + 1}/{len(seeds)}", flush=True)
        return X, Y

    CORRUPTIONS = ("other_pair_set", "das", "noise", "wrong_sound_speed")

    def corrupted(self, seed: int, kind: str, out=None):
        """A wrong input for the judge, [nz][nx][2], from one seed's channel
        data: the KK image of another 72-pair set (shifted scheme, j = N/2),
        the DAS image, the compressed image plus white noise at 20 % of its
        rms, or the compressed image beamformed with c = 1480 m/s instead of
        1540 m/s."""
        import torch
        g = self.geo
        if out is None:
            out = torch.empty((g.nz, g.nx, 2), dtype=torch.float32, device="cuda")
        rf = self.simulate(int(seed))
        if kind == "other_pair_set":
            if not hasattr(self, "plan_o"):
                a = g.vernier_tx
                rc, pc = vernier_pairs(g)
                sub = np.unique(pc[:, 0])
                dth = float(self.tx[sub[-1]] - self.tx[sub[0]]) / (a - 1)
                ro = kk_scheme_angles(KK_SCHEME_SHIFTED, a, dth, g.vernier_rx, a // 2)
                self.plan_o = Plan(self.elem_x, self.tx, g.grid, C_SOUND, FS, g.n_samples, KK_RF_F32,
                                   rx_angles=ro, pairs=pc, compound=KK_COMPOUND_NONE)
                self.bufs_o = (self.plan_o.empty_workspace(), self.plan_o.empty_rf_theta())
            ws, rt = self.bufs_o
            self.plan_o.decompose(rf, rt, ws)
            self.plan_o.beamform(rt, out, None, ws)
        elif kind == "das":
            if not hasattr(self, "plan_d"):
                self.plan_d = Plan(self.elem_x, self.tx, g.grid, C_SOUND, FS, g.n_samples, KK_RF_F32, das=True)
                self.ws_d = self.plan_d.empty_workspace()
            self.plan_d.das(rf, out, None, self.ws_d)
        elif kind == "noise":
            p, ws, rt = self.bufs[0]
            p.decompose(rf, rt, ws)
            p.beamform(rt, out, None, ws)
            gen = torch.Generator(device="cuda").manual_seed(int(seed) + 17)
            rms = out.pow(2).sum(-1).mean().sqrt()
            out.add_(torch.randn(out.shape, device="cuda", generator=gen) * (0.2 * rms / np.sqrt(2.0)))
        elif kind == "wrong_sound_speed":
            if not hasattr(self, "plan_w"):
                rc, pc = vernier_pairs(g)
                self.plan_w = Plan(self.elem_x, self.tx, g.grid, 1480.0, FS, g.n_samples, KK_RF_F32,
                                   rx_angles=rc, pairs=pc, compound=KK_COMPOUND_NONE)
                self.bufs_w = (self.plan_w.empty_workspace(), self.plan_w.empty_rf_theta())
            ws, rt = self.bufs_w
            self.plan_w.decompose(rf, rt, ws)
            self.plan_w.beamform(rt, out, None, ws)
        else:
            raise ValueError(kind)
        return out

    def psf(self):
        """KK images of one point at the grid centre (no noise), both pair sets."""
        import torch
        nx, nz, x0, dx, z0, dz = self.geo.grid
        sc = torch.tensor([[x0 + dx * (nx // 2), z0 + dz * (nz // 2), 1.0, 0.0]], device="cuda")
        kk_simulate_rf(self.tx, self.elem_x, self.geo.n_samples, sc, FS, C_SOUND, out=self.rf)
        pc = torch.empty((nz, nx, 2), dtype=torch.float32, device="cuda")
        pf = torch.empty_like(pc)
        self.images_of(self.rf, pc, pf)
        return pc, pf


def ls_rel_err(a, y):
    """Evaluation metric (not part of the refiner): per image
    min over complex alpha of |alpha a - y| / |y| for [n][H][W][2] tensors."""
    import torch
    ac = torch.view_as_complex(a.reshape(a.shape[0], -1, 2).double())
    yc = torch.view_as_complex(y.reshape(y.shape[0], -1, 2).double())
    ip = (ac.conj() * yc).sum(1)
    aa = (ac.abs() ** 2).sum(1)
    yy = (yc.abs() ** 2).sum(1)
    return torch.sqrt(torch.clamp(1 - ip.abs() ** 2 / (aa * yy), min=0)).cpu().numpy()


def lr_at(step: int, total: int, lr: float, warmup: int = 50) -> float:
    if step < warmup:
        return lr * (step + 1) / warmup
    t = (step - warmup) / max(1, total - warmup)
    return lr * (0.1 + 0.9 * 0.5 * (1 + math.cos(math.pi * min(t, 1.0))))


def batch_indices(seed: int, step: int, n: int, batch: int) -> np.ndarray:
    """Deterministic batch of training indices for a step (epoch permutation
    seeded by (seed, epoch)): resuming at a step replays the same batches."""
    per = max(1, n // batch)
    ep, k = divmod(step, per)
    perm = np.random.default_rng([seed, ep]).permutation(n)
    return perm[k * batch:(k + 1) * batch]


class Refiner:
    """The network, its training loop and inference with the fallback judge."""

    def __init__(self, synth: Synth, max_batch: int = 16, base_channels: int = 32, seed: int = 0,
                 rho: float = 0.1):
        import torch
        self.synth = synth
        g = synth.geo
        self.net = Net(max_batch, g.nz, g.nx, base_channels, seed)
        pc, pf = synth.psf()
        self.net.judge_filter(pc, pf, rho)
        self.tau = (float("inf"), float("inf"))
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    # ---- training ---------------------------------------------------------
    def train(self, X, Y, steps: int, batch: int, lr: float = 3e-4, seed: int = 0, log_every: int = 0,
              ckpt: str | None = None, ckpt_every: int = 0, total_steps: int | None = None):
        """Adam steps from the net's current step count up to `steps` in all.
        Returns the host losses of the steps taken."""
        import torch
        total = total_steps or steps
        losses = []
        while self.net.step < steps:
            s = self.net.step
            idx = torch.from_numpy(batch_indices(seed, s, X.shape[0], batch)).cuda()
            xb, yb = X.index_select(0, idx), Y.index_select(0, idx)
            sx, sy = kk_net_image_scale(xb), kk_net_image_scale(yb)
            self.net.loss_grad(xb, yb, sx, sy, loss=self.loss)
            self.net.adam(lr_at(s, total, lr))
            losses.append(self.loss.clone())
            if log_every and (s + 1) % log_every == 0:
                print(f"  step {s + 1}: loss {float(self.loss):.5f}", flush=True)
            if ckpt and ckpt_every and (s + 1) % ckpt_every == 0:
                self.net.save(ckpt)
        return torch.cat(losses).cpu().numpy() if losses else np.zeros(0, np.float32)

    # ---- inference --------------------------------------------------------
    def forward(self, X, batch: int | None = None):
        """Refined images (in units of each input's 1/rms scale) and the judge
        statistics [n][2]."""
        import torch
        b = batch or self.net.max_batch
        out = torch.empty_like(X)
        stat = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        for i in range(0, X.shape[0], b):
            xb = X[i:i + b]
            s = kk_net_image_scale(xb)
            self.net.forward(xb, s, out=out[i:i + b])
            self.net.judge(out[i:i + b], xb, stat=stat[i:i + b])
        return out, stat

    def calibrate(self, X, margin: float = 1.25):
        """Tolerances of the judge fixed on training images: margin x the largest
        statistic seen."""
        _, st = self.forward(X)
        st = st.cpu().numpy()
        self.tau = (float(st[:, 0].max() * margin), float(st[:, 1].max() * margin))
        return self.tau

    def accept(self, stat):
        import torch
        return (stat[:, 0] <= self.tau[0]) & (stat[:, 1] <= self.tau[1])

    def refine(self, X, rf_list=None):
        """Refined images with the fallback: where the judge rejects image n,
        the plain full-pair KK image of rf_list[n] (when given) replaces it
        (scaled to unit rms).  Returns (images, accepted [n] bool, stat)."""
        out, stat = self.forward(X)
        ok = self.accept(stat)
        if rf_list is not None:
            bad = (~ok).nonzero().flatten().tolist()
            if bad:
                import torch
                tmp = torch.empty_like(X[0])
                for n in bad:
                    self.synth.images_of(rf_list[n], torch.empty_like(tmp), tmp)
                    sc = kk_net_image_scale(tmp[None])
                    out[n] = tmp * sc[0]
        return out, ok, stat

    def evaluate(self, X, Y):
        """Per image: (error of the compressed image, error of the refined
        image), both LS-scaled relative errors against the full-pair image."""
        out, stat = self.forward(X)
        return ls_rel_err(X, Y), ls_rel_err(out, Y), stat.cpu().numpy()


def main(argv=None):
    """Train on seeded phantoms and report the gain on held-out seeds (one
    JSON line)."""
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--train-frames", type=int, default=20000)
    ap.add_argument("--eval-frames", type=int, default=1000)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--ckpt", default=None)
    ap.add_argument("--ckpt-every", type=int, default=1000)
    ap.add_argument("--resume", action="store_true")
    a = ap.parse_args(argv)
    import torch
    t0 = time.time()
    syn = Synth()
    X, Y = syn.dataset(range(100_000, 100_000 + a.train_frames), progress=2000)
    Xe, Ye = syn.dataset(range(900_000, 900_000 + a.eval_frames))
    torch.cuda.synchronize()
    t_data = time.time() - t0
    ref = Refiner(syn, max_batch=a.batch, seed=a.seed)
    if a.resume and a.ckpt and os.path.exists(a.ckpt):
        ref.net.load(a.ckpt)
    t1 = time.time()
    losses = ref.train(X, Y, a.steps, a.batch, a.lr, a.seed, log_every=500, ckpt=a.ckpt, ckpt_every=a.ckpt_every)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    if a.ckpt:
        ref.net.save(a.ckpt)
    tau = ref.calibrate(X[:min(1000, X.shape[0])])
    e_in, e_net, st = ref.evaluate(Xe, Ye)
    acc = (st[:, 0] <= tau[0]) & (st[:, 1] <= tau[1])
    rejected = {}
    n_bad = min(a.eval_frames, 200)
    for kind in Synth.CORRUPTIONS:
        Xb = torch.stack([syn.corrupted(900_000 + i, kind).clone() for i in range(n_bad)])
        _, stb = ref.forward(Xb)
        rejected[kind] = float((~ref.accept(stb)).float().mean())
    print(json.dumps({
        "train_frames": a.train_frames, "eval_frames": a.eval_frames, "steps": a.steps, "batch": a.batch,
        "params": ref.net.n_params, "loss_first": float(losses[:50].mean()) if losses.size else None,
        "loss_last": float(losses[-50:].mean()) if losses.size else None,
        "err_compressed_mean": float(e_in.mean()), "err_refined_mean": float(e_net.mean()),
        "gain": float(e_in.mean() / e_net.mean()), "refined_better_frac": float((e_net < e_in).mean()),
        "judge_tau": tau, "accepted_frac": float(acc.mean()), "corrupted_rejected_frac": rejected,
        "data_s": round(t_data, 1), "train_s": round(t_train, 1),
        "train_images_per_s": round(len(losses) * a.batch / max(t_train, 1e-9), 1)}))


if __name__ == "__main__":
    main()
