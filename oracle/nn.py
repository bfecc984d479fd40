"""FP64 oracle of the learned refiner (test infrastructure only: used by
tests/, the smoke check and the benchmark's CPU baseline; the product never
imports it).

Plain NumPy definitions, NHWC layout, float64:

* 3x3 convolution (cross-correlation, zero padding 1, stride 1) with bias,
  its adjoint in the input (written as the transpose of the forward
  scatter, not via flipped weights) and its weight / bias gradients;
* ReLU, 2x2 average pooling, nearest 2x upsampling and their adjoints;
* the encoder-decoder topology of the refiner (5 levels, additive skips,
  residual output, a 16-channel head of which channels 0, 1 are used), its
  mean-squared-error loss and the full backward pass;
* one Adam step (Kingma & Ba, with bias correction);
* the fallback judge: k-space filter from two point-spread functions and
  the consistency statistic of a refined image with the compressed image.

The paper has no network (it motivates compressed pair sets, Sections II-D
and IV); these are textbook definitions, pinned in tests by central finite
differences, library routines (scipy correlate2d, numpy FFT) and closed
forms.
"""
from __future__ import annotations

import numpy as np

IN_CHANNELS = 16
HEAD_CHANNELS = 16


# --------------------------------------------------------------------------
# layers
# --------------------------------------------------------------------------
def conv3x3(x, w, b=None):
    """y[n,h,w,co] = b[co] + sum_{kh,kw,ci} xpad[n,h+kh,w+kw,ci] w[co,kh,kw,ci]."""
    n, H, W, cin = x.shape
    cout = w.shape[0]
    xp = np.zeros((n, H + 2, W + 2, cin))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    y = np.zeros((n, H, W, cout))
    for kh in range(3):
        for kw in range(3):
            y += xp[:, kh:kh + H, kw:kw + W, :] @ w[:, kh, kw, :].T
    if b is not None:
        y += b
    return y


def conv3x3_dx(dy, w):
    """Adjoint of conv3x3 in x: every output pixel scatters dy @ w back to the
    nine input pixels it read."""
    n, H, W, cout = dy.shape
    cin = w.shape[3]
    dxp = np.zeros((n, H + 2, W + 2, cin))
    for kh in range(3):
        for kw in range(3):
            dxp[:, kh:kh + H, kw:kw + W, :] += dy @ w[:, kh, kw, :]
    return dxp[:, 1:H + 1, 1:W + 1, :]


def conv3x3_dw(x, dy):
    """(dw[co,kh,kw,ci], db[co]) of sum(dy * conv3x3(x, w, b))."""
    n, H, W, cin = x.shape
    cout = dy.shape[3]
    xp = np.zeros((n, H + 2, W + 2, cin))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    dw = np.zeros((cout, 3, 3, cin))
    d2 = dy.reshape(-1, cout)
    for kh in range(3):
        for kw in range(3):
            dw[:, kh, kw, :] = d2.T @ xp[:, kh:kh + H, kw:kw + W, :].reshape(-1, cin)
    return dw, d2.sum(axis=0)


def relu(x):
    return np.maximum(x, 0.0)


def relu_bwd(dy, y):
    """derivative of max(0, s) taken as 0 at s = 0 (y is the ReLU output)."""
    return dy * (y > 0)


def pool2(x):
    n, H, W, c = x.shape
    return x.reshape(n, H // 2, 2, W // 2, 2, c).mean(axis=(2, 4))


def pool2_bwd(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_bwd(dy):
    n, H, W, c = dy.shape
    return dy.reshape(n, H // 2, 2, W // 2, 2, c).sum(axis=(2, 4))


# --------------------------------------------------------------------------
# network
# --------------------------------------------------------------------------
def layer_shapes(C: int):
    """(cin, cout, relu) per layer in parameter order: encoder e0a e0b e1a e1b
    e2a e2b e3 e4, decoder d3 d2 d1 d0, head."""
    return [(IN_CHANNELS, C, True), (C, C, True),
            (C, 2 * C, True), (2 * C, 2 * C, True),
            (2 * C, 4 * C, True), (4 * C, 4 * C, True),
            (4 * C, 8 * C, True),
            (8 * C, 8 * C, True),
            (8 * C, 4 * C, True), (4 * C, 2 * C, True),
            (2 * C, C, True), (C, C, True),
            (C, HEAD_CHANNELS, False)]


def n_params(C: int) -> int:
    return sum(co * 9 * ci + co for ci, co, _ in layer_shapes(C))


def unpack(theta, C: int):
    """flat vector -> list of (w [cout,3,3,cin], b [cout])."""
    out, off = [], 0
    for ci, co, _ in layer_shapes(C):
        nw = co * 9 * ci
        out.append((np.asarray(theta[off:off + nw], np.float64).reshape(co, 3, 3, ci),
                    np.asarray(theta[off + nw:off + nw + co], np.float64)))
        off += nw + co
    assert off == len(theta)
    return out


def pack(grads) -> np.ndarray:
    return np.concatenate([np.concatenate([dw.ravel(), db.ravel()]) for dw, db in grads])


def input_tensor(img, scale=None):
    """complex [n,H,W] -> [n,H,W,16]: (re, im) * scale, zeros."""
    img = np.asarray(img)
    s = np.ones(img.shape[0]) if scale is None else np.asarray(scale, np.float64)
    x = np.zeros(img.shape + (IN_CHANNELS,))
    x[..., 0] = img.real * s[:, None, None]
    x[..., 1] = img.imag * s[:, None, None]
    return x


def forward(theta, C, img, scale=None):
    """Returns (out complex [n,H,W], cache)."""
    P = unpack(theta, C)
    x = input_tensor(img, scale)
    a = [None] * 12

    def cv(i, t):
        w, b = P[i]
        y = conv3x3(t, w, b)
        return relu(y) if layer_shapes(C)[i][2] else y

    a[0] = cv(0, x)
    a[1] = cv(1, a[0])
    p0 = pool2(a[1])
    a[2] = cv(2, p0)
    a[3] = cv(3, a[2])
    p1 = pool2(a[3])
    a[4] = cv(4, p1)
    a[5] = cv(5, a[4])
    p2 = pool2(a[5])
    a[6] = cv(6, p2)
    p3 = pool2(a[6])
    a[7] = cv(7, p3)
    u3 = up2(a[7]) + a[6]
    a[8] = cv(8, u3)
    u2 = up2(a[8]) + a[5]
    a[9] = cv(9, u2)
    u1 = up2(a[9]) + a[3]
    a[10] = cv(10, u1)
    u0 = up2(a[10]) + a[1]
    a[11] = cv(11, u0)
    head = cv(12, a[11])
    out = (x[..., 0] + head[..., 0]) + 1j * (x[..., 1] + head[..., 1])
    cache = dict(P=P, x=x, a=a, p=[p0, p1, p2, p3], u=[u0, u1, u2, u3], head=head)
    return out, cache


def loss(out, target, tscale=None):
    """sum over images, pixels and (re, im) of (out - t s)^2 / (2 n H W)."""
    t = np.asarray(target)
    s = np.ones(t.shape[0]) if tscale is None else np.asarray(tscale, np.float64)
    e = out - t * s[:, None, None]
    return float((e.real ** 2 + e.imag ** 2).sum() / (2 * e.size))


def backward(theta, C, img, scale, target, tscale):
    """(loss, flat gradient) of loss(forward(theta, img, scale), target)."""
    out, c = forward(theta, C, img, scale)
    L = loss(out, target, tscale)
    t = np.asarray(target)
    s = np.ones(t.shape[0]) if tscale is None else np.asarray(tscale, np.float64)
    e = out - t * s[:, None, None]
    dhead = np.zeros(c["head"].shape)
    dhead[..., 0] = e.real / e.size
    dhead[..., 1] = e.imag / e.size
    P, a, p, u, x = c["P"], c["a"], c["p"], c["u"], c["x"]
    g = [None] * 13

    def back(i, inp, dy):
        """layer i: dy w.r.t. its (post-activation) output -> (dx)."""
        w, _ = P[i]
        g[i] = conv3x3_dw(inp, dy)
        return conv3x3_dx(dy, w)

    d = back(12, a[11], dhead)
    d = relu_bwd(d, a[11])
    du0 = back(11, u[0], d)
    d = relu_bwd(up2_bwd(du0), a[10])
    du1 = back(10, u[1], d)
    d = relu_bwd(up2_bwd(du1), a[9])
    du2 = back(9, u[2], d)
    d = relu_bwd(up2_bwd(du2), a[8])
    du3 = back(8, u[3], d)
    d = relu_bwd(up2_bwd(du3), a[7])
    dp3 = back(7, p[3], d)
    da6 = relu_bwd(du3 + pool2_bwd(dp3), a[6])
    dp2 = back(6, p[2], da6)
    da5 = relu_bwd(du2 + pool2_bwd(dp2), a[5])
    da4 = relu_bwd(back(5, a[4], da5), a[4])
    dp1 = back(4, p[1], da4)
    da3 = relu_bwd(du1 + pool2_bwd(dp1), a[3])
    da2 = relu_bwd(back(3, a[2], da3), a[2])
    dp0 = back(2, p[0], da2)
    da1 = relu_bwd(du0 + pool2_bwd(dp0), a[1])
    da0 = relu_bwd(back(1, a[0], da1), a[0])
    back(0, x, da0)
    return L, pack(g)


def init_like(C, seed):
    """A random parameter vector of the topology (for tests: not the
    library's initialisation)."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, co, _ in layer_shapes(C):
        out.append(rng.standard_normal(co * 9 * ci) * np.sqrt(2.0 / (9 * ci)))
        out.append(rng.standard_normal(co) * 0.1)
    return np.concatenate(out)


# --------------------------------------------------------------------------
# optimiser
# --------------------------------------------------------------------------
def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """Step t (1-based) of Adam with L2 term wd w added to the gradient.
    Returns new (w, m, v)."""
    g = g + wd * w
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


# --------------------------------------------------------------------------
# fallback judge
# --------------------------------------------------------------------------
def judge_filter(psf_c, psf_f, rho):
    """G = DFT(psf_c) / DFT(psf_f) where |DFT(psf_c)| >= rho max and
    |DFT(psf_f)| >= rho max, else 0 (numpy's forward DFT, e^{-i})."""
    Sc, Sf = np.fft.fft2(psf_c), np.fft.fft2(psf_f)
    m = (np.abs(Sc) >= rho * np.abs(Sc).max()) & (np.abs(Sf) >= rho * np.abs(Sf).max()) & (np.abs(Sf) > 0)
    G = np.zeros(Sc.shape, complex)
    G[m] = Sc[m] / Sf[m]
    return G


def judge_stat(out, xc, G):
    """Per image: (consistency, out-of-band).  consistency = 1 - |<G A, M C>|^2
    / (|G A|^2 |M C|^2) with A = DFT(out), C = DFT(xc), M = (G != 0): the
    normalised residual of the best complex-scaled fit of G A to M C.
    out-of-band = energy of C outside M / energy of C."""
    M = G != 0
    out, xc = np.asarray(out), np.asarray(xc)
    if out.ndim == 2:
        out, xc = out[None], xc[None]
    res = []
    for o, c in zip(out, xc):
        A, Cs = G * np.fft.fft2(o), np.fft.fft2(c)
        Cm = np.where(M, Cs, 0)
        den = np.vdot(A, A).real * np.vdot(Cm, Cm).real
        cons = 1.0 - abs(np.vdot(A, Cm)) ** 2 / den if den > 0 else 1.0
        tot = np.vdot(Cs, Cs).real
        oob = (tot - np.vdot(Cm, Cm).real) / tot if tot > 0 else 1.0
        res.append((max(cons, 0.0), oob))
    return np.array(res)


def image_scale(img):
    """1 / sqrt(mean |img|^2) per image."""
    img = np.asarray(img)
    return 1.0 / np.sqrt((np.abs(img) ** 2).reshape(img.shape[0], -1).mean(axis=1))
