"""The learned refiner end to end on the GPU: phantoms beamformed by the
plain path (6 x 12 vernier input, full 75 x 128 target, 256 x 256 at
0.15 mm), a short training run with the library's kernels, and on held-out
seeds: what the network gains over the compressed image, the judge's
acceptance, its rejection of inputs that are not KK images, and the
fallback to the plain full-pair image.

The network output has no exact oracle; the gain is measured against the
plain full-pair KK image (LS-scaled relative error, the complex scale fitted
per image).  Stated bars for this short run (384 phantoms, 400 steps of 8):
mean error at most 0.97 x that of the compressed image and lower on at
least 90 % of held-out frames."""
import numpy as np
import pytest

import paper_2603_22496_gb300 as kb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    import torch
    from paper_2603_22496_gb300 import build
    from paper_2603_22496_gb300 import learned as L
    build.build()
    kb.load()
    syn = L.Synth()
    X, Y = syn.dataset(range(100_000, 100_384))
    Xe, Ye = syn.dataset(range(900_000, 900_032))
    ref = L.Refiner(syn, max_batch=8, seed=0)
    losses = ref.train(X, Y, 400, 8, 3e-4, seed=0)
    ref.calibrate(X[:128])
    torch.cuda.synchronize()
    return syn, ref, X, Y, Xe, Ye, losses


def test_training_reduces_the_loss(trained):
    losses = trained[-1]
    assert np.all(np.isfinite(losses))
    assert losses[-40:].mean() < 0.8 * losses[:40].mean()


def test_refined_images_gain_on_held_out_seeds(trained):
    syn, ref, X, Y, Xe, Ye, _ = trained
    e_in, e_net, st = ref.evaluate(Xe, Ye)
    assert e_net.mean() <= 0.97 * e_in.mean(), (e_in.mean(), e_net.mean())
    assert (e_net < e_in).mean() >= 0.9


def test_judge_accepts_held_out_and_rejects_noise(trained):
    import torch
    syn, ref, X, Y, Xe, Ye, _ = trained
    _, st = ref.forward(Xe)
    assert ref.accept(st).float().mean().item() >= 0.9
    g = torch.Generator(device="cuda").manual_seed(1)
    noise = torch.randn((8, 256, 256, 2), device="cuda", generator=g)
    _, stn = ref.forward(noise)
    assert not ref.accept(stn).any()


def test_fallback_returns_the_plain_full_pair_image(trained):
    import torch
    syn, ref, X, Y, Xe, Ye, _ = trained
    g = torch.Generator(device="cuda").manual_seed(2)
    noise = torch.randn((2, 256, 256, 2), device="cuda", generator=g)
    rfs = [syn.simulate(900_000).clone(), syn.simulate(900_001).clone()]
    out, ok, _ = ref.refine(noise, rf_list=rfs)
    assert not ok.any()
    for n in range(2):
        # the fallback is the full-pair image of that record set, unit rms
        assert torch.allclose(out[n] / out[n].pow(2).sum(-1).mean().sqrt(),
                              Ye[n] / Ye[n].pow(2).sum(-1).mean().sqrt(), rtol=1e-4, atol=1e-4)
