"""Pins for the FP64 CNN reference: library cross-checks (scipy correlation,
torch pixel shuffle and Adam) and central finite differences."""
import numpy as np
import pytest
import torch

from oracle import cnn as N


def test_conv3x3_matches_scipy_correlation():
    from scipy.signal import correlate2d
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 9, 3))
    w = rng.standard_normal((4, 9, 3))
    b = rng.standard_normal(4)
    y = N.conv3x3(x, w, b)
    for bb in range(2):
        for o in range(4):
            ref = np.full((7, 9), b[o])
            for c in range(3):
                k = w[o, :, c].reshape(3, 3)    # tap (dy, dx) at [dy + 1, dx + 1]
                ref += correlate2d(x[bb, :, :, c], k, mode="same", boundary="fill")
            assert np.allclose(y[bb, :, :, o], ref, atol=1e-12)


def test_pixel_shuffle_matches_torch():
    rng = np.random.default_rng(1)
    z = rng.standard_normal((2, 3, 5, 16))
    ref = torch.nn.functional.pixel_shuffle(torch.from_numpy(z).permute(0, 3, 1, 2), 4)[:, 0].numpy()
    assert np.array_equal(N.pixel_shuffle(z), ref)
    assert np.array_equal(N.pixel_unshuffle(N.pixel_shuffle(z)), z)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    params = N.init_params(C=4, seed=3)
    params = [p + 0.05 * rng.standard_normal(p.shape) for p in params]   # non-zero biases too
    x = rng.random((1, 12, 12))
    t = rng.random((1, 48, 48))
    loss, grads = N.loss_and_grads(params, x, t)
    h = 1e-6
    for q, p in enumerate(params):
        flat = p.ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = N.loss_and_grads(params, x, t)
            flat[idx] = old - h
            lm, _ = N.loss_and_grads(params, x, t)
            flat[idx] = old
            num = (lp - lm) / (2 * h)
            ana = grads[q].ravel()[idx]
            assert abs(num - ana) <= 1e-6 * max(1e-3, abs(ana)) + 1e-9, (q, idx, num, ana)


def test_adam_matches_torch():
    rng = np.random.default_rng(4)
    params = [rng.standard_normal((3, 4)), rng.standard_normal(5)]
    tp = [torch.tensor(p.copy(), requires_grad=True) for p in params]
    opt = torch.optim.Adam(tp, lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    ad = N.Adam(params)
    for step in range(5):
        grads = [rng.standard_normal(p.shape) for p in params]
        for p, g in zip(tp, grads):
            p.grad = torch.tensor(g)
        opt.step()
        params = ad.step(params, grads)
    for p, q in zip(params, tp):
        assert np.allclose(p, q.detach().numpy(), rtol=0, atol=1e-12)


def test_target_heatmap_peak_and_sum():
    t = N.target_heatmap(10, 8, [(17.0, 13.0)])
    assert t[17, 13] == 1.0 and np.unravel_index(np.argmax(t), t.shape) == (17, 13)
    assert t.sum() == pytest.approx(2 * np.pi, rel=1e-6)    # integral of a unit Gaussian, sigma 1
