"""Pins of the learned denoiser (forward/backward/Adam) and the quality measures."""
import math

import numpy as np
import pytest
import scipy.signal

import oracle as O


def test_conv3x3_matches_library_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 9, 11))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    out = O.conv3x3(x, w, b)
    for co in range(4):
        ref = b[co] + sum(scipy.signal.correlate2d(x[ci], w[co, ci], mode="same", boundary="fill")
                          for ci in range(3))
        assert np.max(np.abs(out[co] - ref)) < 1e-12


def test_zero_last_layer_is_identity():
    params = O.cnn_init(c_in=4, width=8, depth=4, seed=1)
    w, b = params[-1]
    params[-1] = (np.zeros_like(w), np.zeros_like(b))
    r = np.random.default_rng(2).standard_normal((12, 10)) * 50 + 100
    assert np.max(np.abs(O.cnn_denoise(params, r, 7.0) - r)) < 1e-12


def test_density_map_blocks():
    """Each pixel carries m_i / B^2 of its own block (raster order, cropped)."""
    d = O.density_map([0, 4, 16, 8, 2, 1], 8, 12, 4)
    assert d.shape == (8, 12)
    assert d[0, 0] == 0.0 and d[3, 5] == 4 / 16 and d[0, 11] == 1.0
    assert d[4, 0] == 0.5 and d[7, 7] == 2 / 16 and d[5, 9] == 1 / 16


def test_iteration_input():
    """tau_t = min(t, 8) / 8: 0 for the first denoising of A^T y, 1 from t = 8."""
    assert [O.cnn_iter_input(t) for t in (0, 1, 2, 4, 8, 9, 30)] == [0.0, 0.125, 0.25, 0.5, 1.0, 1.0, 1.0]
    x = O.cnn_input(np.ones((3, 4)), 51.0, None, 0.375)
    assert x.shape == (4, 3, 4)
    assert np.all(x[0] == 1 / 255) and np.all(x[1] == 0.2) and np.all(x[2] == 0) and np.all(x[3] == 0.375)


def test_iteration_channel_enters_the_first_layer():
    """Only the first layer's channel-3 weights see tau."""
    params = O.cnn_init(c_in=4, width=4, depth=3, seed=19)
    r = np.random.default_rng(15).standard_normal((6, 7)) * 30 + 100
    assert np.max(np.abs(O.cnn_denoise(params, r, 5.0, None, 0.5) - O.cnn_denoise(params, r, 5.0))) > 0
    w0, b0 = params[0]
    w0 = w0.copy()
    w0[:, 3] = 0.0
    p2 = [(w0, b0)] + params[1:]
    assert np.max(np.abs(O.cnn_denoise(p2, r, 5.0, None, 0.5) - O.cnn_denoise(p2, r, 5.0))) < 1e-12


def test_oracle_ida_passes_the_iteration():
    """With with_iteration the denoiser is called with t = 0, 1, 2, ... in order."""
    img = np.arange(256, dtype=np.float64).reshape(16, 16) % 97
    out = O.sense(img.astype(np.uint8), 8, 0.5, O.ZZ)
    seen = []
    O.ida(out["y"], out["counts"], 16, 16, 8, 3, denoiser=lambda r, s, t: (seen.append(t), r)[1],
          with_iteration=True)
    assert seen == [0, 1, 2]


def test_density_channel_enters_the_first_layer():
    """Only the first layer's channel-2 weights see the density map."""
    params = O.cnn_init(c_in=4, width=4, depth=3, seed=9)
    r = np.random.default_rng(5).standard_normal((6, 7)) * 30 + 100
    d = np.random.default_rng(6).random((6, 7))
    assert np.max(np.abs(O.cnn_denoise(params, r, 5.0, d) - O.cnn_denoise(params, r, 5.0))) > 0
    w0, b0 = params[0]
    w0 = w0.copy()
    w0[:, 2] = 0.0
    p2 = [(w0, b0)] + params[1:]
    assert np.max(np.abs(O.cnn_denoise(p2, r, 5.0, d) - O.cnn_denoise(p2, r, 5.0))) < 1e-12


def test_cnn_gradients_central_differences():
    rng = np.random.default_rng(3)
    params = O.cnn_init(c_in=4, width=4, depth=3, seed=4)
    params = [(w + 0.05 * rng.standard_normal(w.shape), b + 0.05 * rng.standard_normal(b.shape))
              for w, b in params]
    r = rng.standard_normal((8, 8)) * 40 + 120
    clean = r + rng.standard_normal((8, 8)) * 5
    dens = rng.random((8, 8))
    sigma, tau = 11.0, 0.625
    loss, grads = O.cnn_loss_and_grads(params, r, sigma, clean, dens, tau)
    h = 1e-6
    for l, (w, b) in enumerate(params):
        for arr, g in ((w, grads[l][0]), (b, grads[l][1])):
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp, _ = O.cnn_loss_and_grads(params, r, sigma, clean, dens, tau)
                flat[idx] = old - h
                lm, _ = O.cnn_loss_and_grads(params, r, sigma, clean, dens, tau)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g.reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)) + 1e-9, (l, idx)


def test_adam_first_step_closed_form():
    """Step 1: m_hat = g and v_hat = g^2, so the update is lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    p = np.zeros(3)
    p1, m, v = O.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_psnr_known_values():
    ref = np.full((8, 8), 100.0)
    assert O.psnr(ref, ref) == math.inf
    assert abs(O.psnr(ref + 5.0, ref) - 10 * math.log10(255 ** 2 / 25.0)) < 1e-12
    # clipping to [0, 255] happens before the error is taken
    assert abs(O.psnr(np.full((8, 8), 300.0), np.full((8, 8), 250.0)) - 10 * math.log10(255 ** 2 / 25.0)) < 1e-12


def test_ssim_closed_forms():
    rng = np.random.default_rng(0)
    x = rng.integers(0, 256, size=(32, 32)).astype(float)
    assert abs(O.ssim(x, x) - 1.0) < 1e-12
    a, b = 60.0, 90.0
    C1 = (0.01 * 255) ** 2
    got = O.ssim(np.full((20, 20), a), np.full((20, 20), b))
    assert abs(got - (2 * a * b + C1) / (a * a + b * b + C1)) < 1e-12
