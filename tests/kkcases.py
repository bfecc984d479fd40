"""Shared helpers for the GPU tests: run the CUDA path through the C ABI and
build matching pair sets on both sides.

The product side gets its receive angles from the library's own
``kk_scheme_angles``; the oracle side from ``oracle.schemes``.  Both sides
list the pairs in the same (group, transmit, receive) order, written out here
by plain loops.
"""
from __future__ import annotations

import numpy as np

import paper_2603_22496_gb300 as kb
from oracle import schemes

SCHEME_IDS = {"same": kb.KK_SCHEME_SAME, "vernier": kb.KK_SCHEME_VERNIER,
              "shifted": kb.KK_SCHEME_SHIFTED, "confocal": kb.KK_SCHEME_CONFOCAL}


def product_pairs(tx_subset, rx_groups):
    rx_all, pairs, grp = [], [], []
    base = 0
    for g, rx in enumerate(rx_groups):
        for i in tx_subset:
            for o in range(len(rx)):
                pairs.append((int(i), base + o))
                grp.append(g)
        rx_all.append(np.asarray(rx, dtype=np.float64))
        base += len(rx)
    return np.concatenate(rx_all), np.array(pairs, dtype=np.int32), np.array(grp, dtype=np.int32)


def scheme_both(kind, tx_angles, M, j=0, tx_subset=None, js=None):
    """(oracle PairSet, product (rx_all, pairs, groups, J)) for one scheme."""
    tx_angles = np.asarray(tx_angles, dtype=np.float64)
    if tx_subset is None:
        tx_subset = np.arange(tx_angles.shape[0])
    tx_subset = np.asarray(tx_subset)
    ops = schemes.scheme(kind, tx_angles, M, j=j, tx_subset=tx_subset, js=js)
    sub = tx_angles[tx_subset]
    n = sub.shape[0]
    dth = float((sub.max() - sub.min()) / (n - 1)) if n > 1 else 0.0
    if kind == "same":
        groups = [kb.kk_scheme_angles(kb.KK_SCHEME_SAME, n, 0.0, n, tx=sub)]
    elif kind == "hybrid":
        jl = list(js) if js is not None else [0, n // 4, n // 2]
        groups = [kb.kk_scheme_angles(kb.KK_SCHEME_SHIFTED, n, dth, M, jj) for jj in jl]
    else:
        groups = [kb.kk_scheme_angles(SCHEME_IDS[kind], n, dth, M, j)]
    rx_all, pairs, grp = product_pairs(tx_subset, groups)
    assert np.abs(rx_all - ops.rx_angles).max() <= 1e-15
    return ops, (rx_all, pairs, grp, len(groups))


def to_dev(a, device="cuda:0"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device).contiguous()


def cplx(t):
    """torch [..., 2] float32 -> numpy complex128"""
    a = t.detach().cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def rf_dtype_of(w):
    return kb.KK_RF_I16 if w.rf.dtype == np.int16 else kb.KK_RF_F32


def kk_plan_for(w, rx_all, pairs, grp, J, compound=kb.KK_COMPOUND_NONE, grid=None):
    return kb.Plan(w.elem_x, w.tx_angles, grid or w.grid, w.c, w.fs, w.n_samples,
                   rf_dtype_of(w), rx_angles=rx_all, pairs=pairs, group_of_pair=grp,
                   n_groups=J, compound=compound)


def run_kk(w, rx_all, pairs, grp, J, compound=kb.KK_COMPOUND_NONE, grid=None, rf=None):
    """Full CUDA path (decompose + beamform).  Returns (B [J][nz][nx] complex,
    I or None, rf_theta complex [P][T], plan)."""
    import torch
    plan = kk_plan_for(w, rx_all, pairs, grp, J, compound, grid)
    d_rf = to_dev(w.rf if rf is None else rf)
    ws = plan.empty_workspace()
    rt = plan.empty_rf_theta()
    B = plan.empty_image()
    I = plan.empty_intensity() if compound != kb.KK_COMPOUND_NONE else None
    plan.decompose(d_rf, rt, ws)
    plan.beamform(rt, B, I, ws)
    torch.cuda.synchronize()
    return cplx(B), (I.cpu().numpy().astype(np.float64) if I is not None else None), cplx(rt), plan


def run_das(w, grid=None, want_I=False):
    import torch
    plan = kb.Plan(w.elem_x, w.tx_angles, grid or w.grid, w.c, w.fs, w.n_samples,
                   rf_dtype_of(w), das=True)
    d_rf = to_dev(w.rf)
    ws = plan.empty_workspace()
    B = plan.empty_image()
    I = plan.empty_intensity() if want_I else None
    plan.das(d_rf, B, I, ws)
    torch.cuda.synchronize()
    return cplx(B)[0], (I.cpu().numpy().astype(np.float64) if I is not None else None), plan


def rel_l2(a, b):
    nb = float(np.linalg.norm(np.ravel(b)))
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b))) / (nb if nb > 0 else 1.0)


def nn_oracle_operands(theta, img, s_in, C):
    """What the refiner's GPU kernels compute with, for the FP64 network
    oracle: BF16-rounded weights, FP32 biases, the BF16-rounded scaled input
    (complex [n][H][W] times s_in[n])."""
    import torch
    from oracle import nn
    th = np.asarray(theta).astype(np.float64).copy()
    off = 0
    for ci, co, _ in nn.layer_shapes(C):
        nw = co * 9 * ci
        th[off:off + nw] = torch.from_numpy(np.asarray(theta[off:off + nw], np.float32)).to(
            torch.bfloat16).double().numpy()
        off += nw + co
    xs = (img * np.asarray(s_in, np.float64)[:, None, None]).astype(np.complex64)
    re = torch.from_numpy(xs.real.copy()).to(torch.bfloat16).double().numpy()
    im = torch.from_numpy(xs.imag.copy()).to(torch.bfloat16).double().numpy()
    return th, re + 1j * im
