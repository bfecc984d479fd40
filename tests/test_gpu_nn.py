"""The refiner's kernels through the C ABI against the FP64 oracle: each
convolution kernel, the whole network's loss and gradient, Adam, the judge;
checkpoint / resume reproduces training bitwise.

Bounds (derived from the arithmetic):
* forward and weight-gradient convolutions write FP32 sums of exact BF16
  products: rel-L2 <= 1e-5 against FP64 on the same rounded operands;
* the backward-data convolution writes BF16: one rounding, unit roundoff
  2^-9, rms ~1.1e-3 -> rel-L2 <= 3e-3;
* whole-network gradients pass ~24 BF16-rounded tensors (activations and
  activation gradients): random-walk growth sqrt(24) x 1.1e-3 ~ 5.5e-3 ->
  rel-L2 <= 2e-2 over all parameters, <= 5e-2 per layer, loss <= 1e-2.
"""
import os

import numpy as np
import pytest

import paper_2603_22496_gb300 as kb
from oracle import nn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2603_22496_gb300 import build
    build.build()
    kb.load()


def _bf16(a):
    """(device bf16 tensor, float64 array of its exact values)"""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).cuda()
    return t, t.float().cpu().numpy().astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# shapes gathered with cp.async (tiles that cross rows or images) ...
SHAPES = [(2, 13, 21, 16, 16), (1, 32, 40, 32, 48), (3, 9, 70, 64, 32), (1, 1, 5, 16, 64)]
# ... and shapes fed by TMA (128-pixel tiles = row segments or whole rows; 64 for the weight gradient)
SHAPES += [(2, 16, 16, 256, 128), (1, 4, 256, 32, 32), (2, 8, 128, 64, 64), (1, 16, 32, 128, 256),
           (3, 32, 64, 16, 48), (2, 8, 64, 16, 16)]


@pytest.mark.parametrize("n,h,w,cin,cout", SHAPES)
def test_conv3x3_forward(n, h, w, cin, cout):
    import torch
    r = np.random.default_rng(n * 1000 + cin + cout)
    xt, x = _bf16(r.standard_normal((n, h, w, cin)))
    wt, wd = _bf16(r.standard_normal((cout, 3, 3, cin)) / np.sqrt(9 * cin))
    b = r.standard_normal(cout).astype(np.float32)
    bt = torch.from_numpy(b).cuda()
    yf = torch.empty((n, h, w, cout), dtype=torch.float32, device="cuda")
    yb = torch.empty((n, h, w, cout), dtype=torch.bfloat16, device="cuda")
    kb.kk_nn_conv3x3(xt, wt, bt, relu=True, y=yb, yf=yf)
    torch.cuda.synchronize()
    assert kb.kk_nn_status() == kb.KK_OK
    ref = nn.relu(nn.conv3x3(x, wd, b.astype(np.float64)))
    assert _rel(yf.cpu().numpy(), ref) <= 1e-5
    # the BF16 output is the FP32 result rounded once
    assert torch.equal(yb, yf.to(torch.bfloat16))


@pytest.mark.parametrize("n,h,w,cin,cout", SHAPES)
def test_conv3x3_backward_data(n, h, w, cin, cout):
    import torch
    r = np.random.default_rng(7 + n + cin)
    dyt, dy = _bf16(r.standard_normal((n, h, w, cout)))
    wt, wd = _bf16(r.standard_normal((cout, 3, 3, cin)) / np.sqrt(9 * cout))
    dx = torch.empty((n, h, w, cin), dtype=torch.bfloat16, device="cuda")
    kb.kk_nn_conv3x3_dgrad(dyt, wt, dx)
    torch.cuda.synchronize()
    assert kb.kk_nn_status() == kb.KK_OK
    assert _rel(dx.float().cpu().numpy(), nn.conv3x3_dx(dy, wd)) <= 3e-3


@pytest.mark.parametrize("n,h,w,cin,cout", SHAPES + [(8, 64, 64, 32, 32)])
def test_conv3x3_weight_gradient(n, h, w, cin, cout):
    import torch
    r = np.random.default_rng(11 + h + cout)
    xt, x = _bf16(r.standard_normal((n, h, w, cin)))
    dyt, dy = _bf16(r.standard_normal((n, h, w, cout)))
    dw = torch.empty((cout, 3, 3, cin), dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    kb.kk_nn_conv3x3_wgrad(xt, dyt, dw, db)
    torch.cuda.synchronize()
    rw, rb = nn.conv3x3_dw(x, dy)
    assert _rel(dw.cpu().numpy(), rw) <= 1e-5
    assert _rel(db.cpu().numpy(), rb) <= 1e-5


def test_layer_calls_reject_bad_shapes():
    import torch
    x = torch.zeros((1, 4, 4, 8), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros((16, 3, 3, 8), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((1, 4, 4, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(kb.KKError) as e:
        kb.kk_nn_conv3x3(x, w, yf=y)                  # cin = 8 is not a multiple of 16
    assert e.value.status == kb.KK_ERR_INVALID_ARG


# ---- whole network -----------------------------------------------------------
def _net_case(C=32, n=2, H=32, W=32, seed=5):
    import torch
    r = np.random.default_rng(seed)
    net = kb.Net(n, H, W, C, seed=1)
    theta = nn.init_like(C, seed).astype(np.float32)
    # head outputs 2..15 are unused: keep their weights at zero as the library does
    ci, co, _ = nn.layer_shapes(C)[-1]
    o = theta.size - (co * 9 * ci + co)
    hw = theta[o:o + co * 9 * ci].reshape(co, -1)
    hw[2:] = 0
    theta[o + co * 9 * ci + 2:] = 0
    net.set_params(torch.from_numpy(theta).cuda())
    img = (r.standard_normal((n, H, W)) + 1j * r.standard_normal((n, H, W))) * 3.0
    tgt = (r.standard_normal((n, H, W)) + 1j * r.standard_normal((n, H, W))) * 2.0
    return net, theta, img, tgt


def _c2t(z):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.stack([z.real, z.imag], -1), np.float32)).cuda()


def _oracle_operands(theta, img, s_in, C):
    """The oracle sees what the GPU computes with: BF16 weights, FP32 biases,
    the BF16-rounded scaled input."""
    import torch
    th = theta.astype(np.float64).copy()
    off = 0
    for ci, co, _ in nn.layer_shapes(C):
        nw = co * 9 * ci
        th[off:off + nw] = torch.from_numpy(theta[off:off + nw]).to(torch.bfloat16).double().numpy()
        off += nw + co
    xs = (img * s_in[:, None, None]).astype(np.complex64)
    re = torch.from_numpy(xs.real.copy()).to(torch.bfloat16).double().numpy()
    im = torch.from_numpy(xs.imag.copy()).to(torch.bfloat16).double().numpy()
    return th, re + 1j * im


def test_network_forward_loss_and_gradient_match_oracle():
    import torch
    C = 32
    net, theta, img, tgt = _net_case(C)
    s_in = np.array([0.5, 0.25], np.float32)
    s_t = np.array([0.3, 0.7], np.float32)
    g = torch.empty(net.n_params, dtype=torch.float32, device="cuda")
    out = torch.empty((2, 32, 32, 2), dtype=torch.float32, device="cuda")
    loss = net.loss_grad(_c2t(img), _c2t(tgt), torch.from_numpy(s_in).cuda(), torch.from_numpy(s_t).cuda(),
                         grad=g, out=out)
    torch.cuda.synchronize()
    th, xin = _oracle_operands(theta, img, s_in.astype(np.float64), C)
    ref_out, _ = nn.forward(th, C, xin, None)
    L, rg = nn.backward(th, C, xin, None, tgt, s_t.astype(np.float64))
    o = out.cpu().numpy()
    assert _rel(o[..., 0] + 1j * o[..., 1], ref_out) <= 1e-2
    assert abs(float(loss) - L) <= 1e-2 * L
    gg = g.cpu().numpy().astype(np.float64)
    assert _rel(gg, rg) <= 2e-2
    off = 0
    for i, (ci, co, _) in enumerate(nn.layer_shapes(C)):
        k = co * 9 * ci + co
        assert _rel(gg[off:off + k], rg[off:off + k]) <= 5e-2, i
        off += k
    # forward alone gives the same output as the loss pass
    out2 = net.forward(_c2t(img), torch.from_numpy(s_in).cuda())
    torch.cuda.synchronize()
    assert torch.equal(out2, out)
    assert net.status() == kb.KK_OK


def test_network_gradient_at_256_matches_oracle():
    """One 256 x 256 image: every layer runs on the TMA-fed kernels."""
    import torch
    C = 32
    net, theta, img, tgt = _net_case(C, n=1, H=256, W=256, seed=13)
    s_in = np.array([0.5], np.float32)
    g = torch.empty(net.n_params, dtype=torch.float32, device="cuda")
    loss = net.loss_grad(_c2t(img), _c2t(tgt), torch.from_numpy(s_in).cuda(), grad=g)
    torch.cuda.synchronize()
    assert net.status() == kb.KK_OK
    th, xin = _oracle_operands(theta, img, s_in.astype(np.float64), C)
    L, rg = nn.backward(th, C, xin, None, tgt, None)
    assert abs(float(loss) - L) <= 1e-2 * L
    gg = g.cpu().numpy().astype(np.float64)
    assert _rel(gg, rg) <= 2e-2
    off = 0
    for i, (ci, co, _) in enumerate(nn.layer_shapes(C)):
        k = co * 9 * ci + co
        assert _rel(gg[off:off + k], rg[off:off + k]) <= 5e-2, i
        off += k


def test_adam_steps_match_oracle():
    import torch
    C = 16
    net, theta, img, tgt = _net_case(C, seed=9)
    w = theta.astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    g = torch.empty(net.n_params, dtype=torch.float32, device="cuda")
    for t in (1, 2, 3):
        net.loss_grad(_c2t(img), _c2t(tgt), grad=g)
        gi = g.cpu().numpy().astype(np.float64)
        net.adam(1e-3, 0.9, 0.999, 1e-8, 1e-4)
        w, m, v = nn.adam_step(w, gi, m, v, t, 1e-3, 0.9, 0.999, 1e-8, 1e-4)
        p = net.get_params()
        torch.cuda.synchronize()
        assert np.max(np.abs(p.cpu().numpy() - w)) <= 1e-6 * max(1.0, np.abs(w).max())
        # continue the oracle from the GPU's FP32 weights
        w = p.cpu().numpy().astype(np.float64)
    assert net.step == 3


def _train_steps(net, X, Y, steps, batch=2, seed=4):
    import torch
    from paper_2603_22496_gb300.learned import batch_indices
    losses = []
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    while net.step < steps:
        idx = torch.from_numpy(batch_indices(seed, net.step, X.shape[0], batch)).cuda()
        xb, yb = X.index_select(0, idx), Y.index_select(0, idx)
        net.loss_grad(xb, yb, kb.kk_net_image_scale(xb), kb.kk_net_image_scale(yb), loss=loss)
        net.adam(1e-3)
        losses.append(float(loss))
    return losses


def test_checkpoint_resume_is_bitwise(tmp_path):
    import torch
    r = np.random.default_rng(3)
    X = torch.from_numpy(r.standard_normal((8, 32, 32, 2)).astype(np.float32)).cuda()
    Y = torch.from_numpy(r.standard_normal((8, 32, 32, 2)).astype(np.float32)).cuda()
    a = kb.Net(2, 32, 32, 32, seed=11)
    la = _train_steps(a, X, Y, 3)
    path = str(tmp_path / "net.ckpt")
    a.save(path)
    la += _train_steps(a, X, Y, 6)
    pa = a.get_params()
    b = kb.Net(2, 32, 32, 32, seed=99)             # different init: load must overwrite it
    b.load(path)
    assert b.step == 3
    lb = _train_steps(b, X, Y, 6)
    pb = b.get_params()
    torch.cuda.synchronize()
    assert la[3:] == lb
    assert torch.equal(pa, pb)
    # an uninterrupted run from the same seed gives the same curve
    c = kb.Net(2, 32, 32, 32, seed=11)
    assert _train_steps(c, X, Y, 6) == la
    # a checkpoint of another topology is refused
    d = kb.Net(2, 32, 32, 16, seed=1)
    with pytest.raises(kb.KKError):
        d.load(path)


@pytest.mark.parametrize("H,W", [(32, 32), (48, 32), (64, 48)])
def test_judge_and_image_scale_match_oracle(H, W):
    """Power-of-two axes run the Stockham FFT, others the direct DFT."""
    import torch
    ky, kx = np.meshgrid(np.fft.fftfreq(H), np.fft.fftfreq(W), indexing="ij")
    band = lambda r: np.exp(-((ky - 0.2) ** 2 + kx ** 2) / (2 * r ** 2))
    psf_c, psf_f = np.fft.ifft2(band(0.05)), np.fft.ifft2(band(0.1))
    rho = next(r for r in np.arange(0.1, 0.3, 0.005)          # a threshold >= 2e-3 from every bin
               if min(np.min(np.abs(S / S.max() - r)) for S in
                      (np.abs(np.fft.fft2(psf_c)), np.abs(np.fft.fft2(psf_f)))) > 2e-3)
    net = kb.Net(4, H, W, 16, seed=0)
    net.judge_filter(_c2t(psf_c), _c2t(psf_f), rho)
    G = nn.judge_filter(psf_c, psf_f, rho)
    r = np.random.default_rng(2)
    y = r.standard_normal((4, H, W)) + 1j * r.standard_normal((4, H, W))
    xc = np.fft.ifft2(G * np.fft.fft2(y))
    xc[2] = r.standard_normal((H, W)) + 1j * r.standard_normal((H, W))   # unrelated
    xc[3] = xc[3] * (2 - 1j)
    st = net.judge(_c2t(y), _c2t(xc)).cpu().numpy()
    ref = nn.judge_stat(y, xc, G)
    assert np.allclose(st, ref, atol=2e-4)
    sc = kb.kk_net_image_scale(_c2t(y)).cpu().numpy()
    assert np.allclose(sc, nn.image_scale(y), rtol=1e-5)


def test_net_rejects_bad_calls():
    import torch
    net = kb.Net(2, 32, 32, 16, seed=0)
    x = torch.zeros((3, 32, 32, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(kb.KKError):
        net.forward(x)                               # nb > max_batch
    with pytest.raises(kb.KKError) as e:
        net.judge(x[:2], x[:2])                      # no judge filter yet
    assert e.value.status == kb.KK_ERR_INVALID_ARG
    with pytest.raises(kb.KKError):
        kb.Net(2, 30, 32, 32)                        # H not a multiple of 16
    with pytest.raises(kb.KKError):
        net.adam(-1.0)
