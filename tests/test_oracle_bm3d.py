"""Pins of the oracle's BM3D hard-thresholding step against properties of
the algorithm that do not re-use its code."""
import math

import numpy as np
import pytest

import oracle as O


def test_haar_is_orthonormal_and_row0_is_the_mean():
    for n in (1, 2, 4, 8, 16):
        H = O.haar_matrix(n)
        assert np.allclose(H @ H.T, np.eye(n), atol=1e-14)
        assert np.allclose(H[0], 1.0 / math.sqrt(n), atol=1e-15)
    assert np.allclose(O.haar_matrix(2), np.array([[1, 1], [1, -1]]) / math.sqrt(2), atol=1e-15)


def test_zero_threshold_is_the_identity():
    """lam3d = 0 keeps every coefficient: each patch estimate is the patch
    itself, so the weighted average of overlapping copies is the image."""
    rng = np.random.default_rng(0)
    r = rng.normal(100, 20, (32, 40))
    out = O.bm3d_ht(r, 10.0, lam3d=0.0)
    assert np.max(np.abs(out - r)) < 1e-9


def test_constant_image_is_unchanged():
    r = np.full((24, 32), 77.0)
    for s in (5.0, 50.0):
        assert np.max(np.abs(O.bm3d_ht(r, s) - 77.0)) < 1e-9


def test_infinite_threshold_gives_group_means():
    """A threshold above every coefficient keeps only each group's 3D DC:
    every patch estimate is the mean pixel of its group.  With a very large
    sigma (tau 5000, far above these distances) every candidate matches, so
    on an image whose 8x8 window means are all equal (a checkerboard of
    period 2) the output is that mean everywhere."""
    yy, xx = np.mgrid[0:24, 0:24]
    r = 100.0 + 20.0 * ((yy + xx) % 2)
    out = O.bm3d_ht(r, 1e6, lam3d=1.0)
    assert np.max(np.abs(out - 110.0)) < 1e-9


def test_denoises_a_noisy_step():
    """Noise at sigma 20 on a two-level image: the estimate is closer to
    the clean image than the input (MSE at least halved)."""
    rng = np.random.default_rng(1)
    clean = np.where(np.arange(40)[None, :] < 20, 60.0, 180.0) * np.ones((40, 1))
    noisy = clean + rng.normal(0, 20, clean.shape)
    out = O.bm3d_ht(noisy, 20.0)
    assert np.mean((out - clean) ** 2) < 0.5 * np.mean((noisy - clean) ** 2)
