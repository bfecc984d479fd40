"""Pins of the FP64 refiner oracle (CPU): every layer against a library
routine or an adjoint identity, every gradient against central finite
differences, Adam against its closed form under a constant gradient, the
judge statistic against its exact zero and bounds."""
import numpy as np
import pytest
from scipy import signal

from oracle import nn


def _rng(s):
    return np.random.default_rng(s)


def _dot(a, b):
    return float(np.vdot(a, b).real)


# ---- layers -----------------------------------------------------------------
@pytest.mark.parametrize("n,H,W,cin,cout", [(1, 5, 7, 3, 2), (2, 8, 6, 4, 5), (1, 1, 1, 2, 3)])
def test_conv3x3_matches_scipy_correlate2d(n, H, W, cin, cout):
    r = _rng(1)
    x = r.standard_normal((n, H, W, cin))
    w = r.standard_normal((cout, 3, 3, cin))
    b = r.standard_normal(cout)
    y = nn.conv3x3(x, w, b)
    ref = np.zeros_like(y)
    for i in range(n):
        for co in range(cout):
            ref[i, :, :, co] = b[co] + sum(
                signal.correlate2d(x[i, :, :, ci], w[co, :, :, ci], mode="same", boundary="fill")
                for ci in range(cin))
    assert np.allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_conv3x3_dx_is_the_adjoint():
    r = _rng(2)
    x = r.standard_normal((2, 6, 9, 4))
    w = r.standard_normal((3, 3, 3, 4))
    dy = r.standard_normal((2, 6, 9, 3))
    lhs = _dot(nn.conv3x3(x, w), dy)
    rhs = _dot(x, nn.conv3x3_dx(dy, w))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_conv3x3_dw_db_finite_differences():
    """conv is linear in (w, b): central differences are exact up to rounding."""
    r = _rng(3)
    x = r.standard_normal((2, 5, 4, 3))
    w = r.standard_normal((2, 3, 3, 3))
    b = r.standard_normal(2)
    R = r.standard_normal((2, 5, 4, 2))
    dw, db = nn.conv3x3_dw(x, R)
    h = 1e-3
    for idx in [(0, 0, 0, 0), (1, 2, 1, 2), (0, 1, 2, 1), (1, 0, 2, 0)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = (_dot(nn.conv3x3(x, wp, b), R) - _dot(nn.conv3x3(x, wm, b), R)) / (2 * h)
        assert abs(fd - dw[idx]) <= 1e-9 * max(1.0, abs(fd))
    for co in range(2):
        bp, bm = b.copy(), b.copy()
        bp[co] += h
        bm[co] -= h
        fd = (_dot(nn.conv3x3(x, w, bp), R) - _dot(nn.conv3x3(x, w, bm), R)) / (2 * h)
        assert abs(fd - db[co]) <= 1e-9 * max(1.0, abs(fd))


def test_pool_and_upsample_adjoints_and_values():
    r = _rng(4)
    x = r.standard_normal((2, 6, 8, 3))
    y = r.standard_normal((2, 3, 4, 3))
    assert abs(_dot(nn.pool2(x), y) - _dot(x, nn.pool2_bwd(y))) <= 1e-12 * np.abs(x).sum()
    assert abs(_dot(nn.up2(y), x) - _dot(y, nn.up2_bwd(x))) <= 1e-12 * np.abs(x).sum()
    assert np.allclose(nn.pool2(nn.up2(y)), y)
    a = np.arange(16.0).reshape(1, 4, 4, 1)
    assert np.array_equal(nn.pool2(a)[0, :, :, 0], [[2.5, 4.5], [10.5, 12.5]])
    assert np.array_equal(nn.up2(np.array([[[[1.0], [2.0]]]]))[0, :, :, 0], [[1, 1, 2, 2], [1, 1, 2, 2]])


def test_relu_backward_finite_differences():
    r = _rng(5)
    s = r.standard_normal(50)
    s = s[np.abs(s) > 1e-2]
    R = r.standard_normal(s.shape)
    g = nn.relu_bwd(R, nn.relu(s))
    h = 1e-6
    fd = (nn.relu(s + h) - nn.relu(s - h)) / (2 * h) * R
    assert np.allclose(g, fd, atol=1e-9)


# ---- network ----------------------------------------------------------------
def _tiny(seed=6, C=2, n=2, H=16, W=16):
    r = _rng(seed)
    theta = nn.init_like(C, seed)
    img = r.standard_normal((n, H, W)) + 1j * r.standard_normal((n, H, W))
    tgt = r.standard_normal((n, H, W)) + 1j * r.standard_normal((n, H, W))
    return theta, img, r.uniform(0.5, 2.0, n), tgt, r.uniform(0.5, 2.0, n)


def test_network_parameter_count():
    # C = 32, weights 9 cin cout: encoder 16*32 + 32*32 + 32*64 + 64*64 + 64*128 + 128*128
    # + 128*256 + 256*256 = 130560, decoder 256*128 + 128*64 + 64*32 + 32*32 + 32*16 = 44544;
    # 9 * 175104 = 1575936 weights + 1232 biases
    assert nn.n_params(32) == 1575936 + 1232
    assert nn.n_params(2) == sum(co * 9 * ci + co for ci, co, _ in nn.layer_shapes(2))


def test_network_gradient_finite_differences():
    """Whole-network gradient (every layer, skip, pool and upsample adjoint,
    loss normalisation) against central differences, <= 1e-6 relative."""
    C = 2
    theta, img, s_in, tgt, s_t = _tiny(C=C)
    L, g = nn.backward(theta, C, img, s_in, tgt, s_t)
    offs, off = [], 0
    for ci, co, _ in nn.layer_shapes(C):
        offs.append((off, co * 9 * ci, co))
        off += co * 9 * ci + co
    r = _rng(7)
    idx = []
    for o, nw, nb in offs:                    # two weights and one bias of every layer
        idx += list(o + r.choice(nw, 2, replace=False)) + [o + nw + int(r.integers(nb))]
    h = 1e-5
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (nn.loss(nn.forward(tp, C, img, s_in)[0], tgt, s_t) -
              nn.loss(nn.forward(tm, C, img, s_in)[0], tgt, s_t)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(fd), 1e-3), (k, fd, g[k])
    # head outputs 2..15 do not reach the loss: their gradients are exactly zero
    ci, co, _ = nn.layer_shapes(C)[-1]
    o, nw, _ = offs[-1]
    assert np.all(g[o:o + nw].reshape(co, -1)[2:] == 0) and np.all(g[o + nw + 2:o + nw + co] == 0)


def test_network_with_zero_head_is_identity():
    C = 2
    theta, img, s_in, _, _ = _tiny(C=C)
    ci, co, _ = nn.layer_shapes(C)[-1]
    theta[-(co * 9 * ci + co):] = 0.0
    out, _ = nn.forward(theta, C, img, s_in)
    assert np.allclose(out, img * s_in[:, None, None], rtol=0, atol=0)


def test_network_loss_definition():
    C = 2
    theta, img, s_in, tgt, s_t = _tiny(C=C)
    out, _ = nn.forward(theta, C, img, s_in)
    e = out - tgt * s_t[:, None, None]
    assert nn.loss(out, tgt, s_t) == pytest.approx(np.mean(np.abs(e) ** 2) / 2, rel=1e-14)


# ---- optimiser --------------------------------------------------------------
def test_adam_constant_gradient_closed_form():
    """With a constant gradient the bias-corrected moments are g and g^2 at
    every step, so each step moves by -lr g / (|g| + eps)."""
    r = _rng(8)
    w0 = r.standard_normal(10)
    g = r.standard_normal(10)
    w, m, v = w0.copy(), np.zeros(10), np.zeros(10)
    lr, eps = 1e-2, 1e-8
    for t in range(1, 6):
        w, m, v = nn.adam_step(w, g, m, v, t, lr, 0.9, 0.999, eps)
        assert np.allclose(w, w0 - t * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-14)


def test_adam_weight_decay_first_step():
    w0 = np.array([1.0, -2.0, 0.5])
    g = np.array([0.1, 0.0, -0.3])
    wd, lr = 0.1, 1e-3
    w, _, _ = nn.adam_step(w0, g, np.zeros(3), np.zeros(3), 1, lr, 0.9, 0.999, 1e-12, wd)
    ge = g + wd * w0
    assert np.allclose(w, w0 - lr * np.sign(ge), rtol=1e-9)


# ---- judge ------------------------------------------------------------------
def _psfs(H=32, W=32):
    """Two band-limited point responses: a narrow and a broad passband."""
    ky, kx = np.meshgrid(np.fft.fftfreq(H), np.fft.fftfreq(W), indexing="ij")
    band = lambda r: np.exp(-((ky - 0.2) ** 2 + kx ** 2) / (2 * r ** 2))
    return np.fft.ifft2(band(0.05)), np.fft.ifft2(band(0.1))


def test_judge_exact_zero_for_consistent_pair_and_scale_invariance():
    psf_c, psf_f = _psfs()
    G = nn.judge_filter(psf_c, psf_f, 0.1)
    r = _rng(9)
    y = r.standard_normal((32, 32)) + 1j * r.standard_normal((32, 32))
    xc = np.fft.ifft2(G * np.fft.fft2(y))          # exactly the compressed view of y
    st = nn.judge_stat(y, xc, G)[0]
    assert st[0] <= 1e-12 and st[1] <= 1e-12
    st2 = nn.judge_stat(y * (0.3 - 2j), xc * (1.5 + 0.5j), G)[0]
    assert st2[0] <= 1e-12


def test_judge_bounds_and_unrelated_images():
    psf_c, psf_f = _psfs()
    G = nn.judge_filter(psf_c, psf_f, 0.1)
    r = _rng(10)
    a = r.standard_normal((4, 32, 32)) + 1j * r.standard_normal((4, 32, 32))
    b = r.standard_normal((4, 32, 32)) + 1j * r.standard_normal((4, 32, 32))
    st = nn.judge_stat(a, b, G)
    assert np.all((st >= 0) & (st <= 1))
    assert np.all(st[:, 0] > 0.8)                  # unrelated: almost no fit
    frac_in = (G != 0).mean()
    assert np.allclose(st[:, 1], 1 - frac_in, atol=0.1)  # white input: energy spread evenly


def test_judge_filter_of_identical_psfs_is_the_mask():
    psf_c, _ = _psfs()
    G = nn.judge_filter(psf_c, psf_c, 0.2)
    S = np.abs(np.fft.fft2(psf_c))
    assert np.array_equal(G != 0, S >= 0.2 * S.max())
    assert np.allclose(G[G != 0], 1.0)


def test_image_scale():
    img = np.full((2, 4, 4), 3.0 + 4.0j)
    img[1] *= 2
    assert np.allclose(nn.image_scale(img), [0.2, 0.1])
