"""Pins of the IDA loop (Eqs. 13, 15, 25, 28) and of the plain denoiser."""
import itertools
import math

import numpy as np
import pytest
import scipy.fft
import scipy.ndimage

import oracle as O
from paper_2001_09632_gb300 import synth


def _setup(H=64, W=48, B=16, r=0.3, variant=O.BBV, seed=2):
    img = synth.gen_image(H, W, seed)
    out = O.sense(img, B, r, variant)
    return img, out


def test_A_At_adjoint_and_AAt_identity():
    img, out = _setup()
    counts, B = out["counts"], 16
    rng = np.random.default_rng(0)
    x = rng.standard_normal((64, 48))
    z = rng.standard_normal(len(out["y"]))
    assert abs(np.dot(O.A(x, counts, B), z) - np.sum(x * O.At(z, counts, B, 64, 48))) < 1e-9
    # rows of A are orthonormal: A A^T = I on the packed space
    assert np.max(np.abs(O.A(O.At(z, counts, B, 64, 48), counts, B) - z)) < 1e-12


def _c_sequence(T, DF):
    c = [1.0, 1.0 / DF]
    while len(c) < T:
        c.append((c[-1] - c[-2]) / DF)
    return c[:T]


@pytest.mark.parametrize("DF", [1.0, 1.5, 2.0, 3.0])
def test_ida_identity_denoiser_closed_form(DF):
    """With D = identity the kept coefficients a^t = A x^t obey
    e^t = y - a^t, z^t = e^t + z^{t-1}/D_F, a^{t+1} = a^t + z^t, which gives
    z^t = c_t y with c_0 = 1, c_1 = 1/D_F, c_t = (c_{t-1} - c_{t-2}) / D_F and
    x^T = (sum_{s<T} c_s) A^T y.  (D_F = 1 oscillates with period 6.)"""
    img, out = _setup()
    y, counts = out["y"], out["counts"]
    T = 12
    x, sig, rs, zs = O.ida(y, counts, 64, 48, 16, T, DF=DF, denoiser=None, trace=True)
    c = _c_sequence(T, DF)
    At_y = O.reconstruct(counts, y, 64, 48, 16)
    assert np.max(np.abs(x - sum(c) * At_y)) < 1e-8 * np.max(np.abs(At_y))
    ny = np.linalg.norm(y)
    for t in range(T):
        assert abs(sig[t] - abs(c[t]) * ny / math.sqrt(len(y))) < 1e-9 * ny
        assert np.max(np.abs(zs[t] - c[t] * y)) < 1e-8 * np.max(np.abs(y))
    if DF == 1.0:
        assert np.allclose(c[:7], [1, 1, 0, -1, -1, 0, 1])


def test_ida_first_iterate_is_denoised_idct():
    img, out = _setup()
    y, counts = out["y"], out["counts"]
    seen = []

    def den(r, s):
        seen.append((r.copy(), s))
        return 0.5 * r
    O.ida(y, counts, 64, 48, 16, 2, DF=2.0, denoiser=den)
    assert np.allclose(seen[0][0], O.reconstruct(counts, y, 64, 48, 16))
    assert abs(seen[0][1] - np.linalg.norm(y) / math.sqrt(len(y))) < 1e-9
    # second iterate: x1 = 0.5 A^T y -> z1 = y - 0.5 y + y/2 = y
    assert abs(seen[1][1] - np.linalg.norm(y) / math.sqrt(len(y))) < 1e-9


def test_tidct_lambda_zero_is_identity():
    rng = np.random.default_rng(3)
    r = rng.standard_normal((20, 28)) * 30 + 100
    assert np.max(np.abs(O.tidct_denoise(r, 5.0, 0.0) - r)) < 1e-10


def test_tidct_infinite_threshold_is_triangle_filter():
    """Only the DC survives: every window is replaced by its mean, and the
    average over the 64 windows covering a pixel is a separable triangle
    filter (8 - |k|)/64, k = -7..7, on the symmetric extension."""
    rng = np.random.default_rng(4)
    r = rng.standard_normal((24, 40)) * 20 + 80
    tri = (8.0 - np.abs(np.arange(-7, 8))) / 64.0
    ref = scipy.ndimage.correlate(r, np.outer(tri, tri), mode="reflect")
    assert np.max(np.abs(O.tidct_denoise(r, 1e12, 1.0) - ref)) < 1e-9


def test_tidct_brute_force_per_pixel():
    """Pixel-centric restatement: average, over the 64 windows containing the
    pixel, of the hard-thresholded window (scipy DCT)."""
    rng = np.random.default_rng(5)
    H, W = 10, 12
    r = rng.standard_normal((H, W)) * 40 + 120
    sigma, lam = 9.0, 2.5

    def refl(i, n):
        i = i % (2 * n)
        return i if i < n else 2 * n - 1 - i

    ref = np.zeros((H, W))
    for py, px in itertools.product(range(H), range(W)):
        acc = 0.0
        for y0 in range(py - 7, py + 1):
            for x0 in range(px - 7, px + 1):
                win = np.array([[r[refl(y0 + a, H), refl(x0 + b, W)] for b in range(8)] for a in range(8)])
                C = scipy.fft.dctn(win, norm="ortho")
                keep = np.abs(C) > lam * sigma
                keep[0, 0] = True
                acc += scipy.fft.idctn(C * keep, norm="ortho")[py - y0, px - x0]
        ref[py, px] = acc / 64
    assert np.max(np.abs(O.tidct_denoise(r, sigma, lam) - ref)) < 1e-9


def test_tidct_constant_image_unchanged():
    r = np.full((16, 24), 42.0)
    assert np.max(np.abs(O.tidct_denoise(r, 3.0, 2.7) - r)) < 1e-10
