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


def _scene(seed=0, H=80, W=80):
    """iid uniform noise: two unrelated 8x8 patches differ by d ~ 2 * 255^2 / 12
    ~ 10800 on average, far above both thresholds, so only planted patches match."""
    return np.random.default_rng(seed).uniform(0, 255, (H, W))


def _plant(r, y, x, P):
    r[y:y + 8, x:x + 8] = P


def test_block_matching_window_threshold_ties_and_power_of_two():
    """Hand-built group for the reference at (30, 30): copies of its patch
    planted at known offsets and known distances d = ||P_ref - P||^2 / 64.
      B (11, 49): +1 everywhere, d = 1, offset (-19, +19), inside the window
      A (49, 30): +1 everywhere, d = 1, offset (+19, 0), inside, ties with B
      C (30, 50): exact copy, d = 0, offset (0, +20), outside the window
      E (40, 12): d = 2501 (one pixel carries the extra 64), offset (+10, -18)
    sigma <= 40 (tau 2500): matches B, A -> 3 candidates -> a group of 2, and
    of the tie the lower row (B) comes first; sigma > 40 (tau 5000): B, A, E
    -> 4 -> the reference, B, A, E."""
    r = _scene(0)
    P = r[30:38, 30:38].copy()
    _plant(r, 11, 49, P + 1.0)
    _plant(r, 49, 30, P + 1.0)
    _plant(r, 30, 50, P)
    Q = P + 50.0
    Q[3, 4] = P[3, 4] + math.sqrt(2564.0)       # 63 * 2500 + 2564 = 64 * 2501
    _plant(r, 40, 12, Q)
    for s in (5.0, 40.0):
        g = O.bm3d_group(r, 30, 30, s)
        assert [(yy, xx) for _, yy, xx in g] == [(30, 30), (11, 49)], s
        assert g[1][0] == pytest.approx(1.0, abs=1e-9)
    g = O.bm3d_group(r, 30, 30, 40.5)
    assert [(yy, xx) for _, yy, xx in g] == [(30, 30), (11, 49), (49, 30), (40, 12)]
    assert [d for d, _, _ in g] == pytest.approx([0.0, 1.0, 1.0, 2501.0], abs=1e-9)


def test_block_matching_threshold_is_inclusive():
    """d = 2500 exactly joins at sigma = 40 (tau 2500, d <= tau)."""
    r = _scene(1)
    P = r[30:38, 30:38].copy()
    _plant(r, 12, 14, P + 50.0)                  # d = 50^2, offset (-18, -16)
    _plant(r, 45, 44, P + 2.0)                   # d = 4, offset (+15, +14)
    g = O.bm3d_group(r, 30, 30, 40.0)
    assert [(yy, xx) for _, yy, xx in g] == [(30, 30), (45, 44)]       # 3 candidates -> 2
    assert O.bm3d_group(r, 30, 30, 40.0, N2=16)[1][0] == pytest.approx(4.0, abs=1e-9)
    _plant(r, 45, 44, _scene(9)[0:8, 0:8])       # remove the close match: the reference and d = 2500 remain
    g = O.bm3d_group(r, 30, 30, 40.0)
    assert [(yy, xx) for _, yy, xx in g] == [(30, 30), (12, 14)]
    assert g[1][0] == pytest.approx(2500.0, abs=1e-9)


def test_block_matching_keeps_the_sixteen_closest():
    """24 planted copies on a 9-pixel grid around the reference at (40, 40),
    at distances d = delta^2 for distinct delta: the group is the reference and
    the 15 closest (N2 = 16), in order of distance."""
    r = _scene(2, 96, 96)
    P = r[40:48, 40:48].copy()
    deltas = np.random.default_rng(5).permutation(np.arange(1, 25)).astype(float)
    pos = [(40 + 9 * i - 18, 40 + 9 * j - 18) for i in range(5) for j in range(5) if (i, j) != (2, 2)]
    for (yy, xx), dl in zip(pos, deltas):
        _plant(r, yy, xx, P + dl)
    g = O.bm3d_group(r, 40, 40, 20.0)
    assert len(g) == 16
    order = np.argsort(deltas)[:15]
    assert [(yy, xx) for _, yy, xx in g[1:]] == [pos[i] for i in order]
    assert [d for d, _, _ in g[1:]] == pytest.approx(list(np.sort(deltas)[:15] ** 2), abs=1e-9)


def test_block_matching_clips_the_window_at_the_border():
    """Reference at (0, 0): the window covers rows and columns 0..19 only; a
    copy at (19, 19) (inside) matches, one at (0, 20) does not."""
    r = _scene(3, 48, 48)
    P = r[0:8, 0:8].copy()
    _plant(r, 19, 19, P + 3.0)
    _plant(r, 0, 20, P)
    g = O.bm3d_group(r, 0, 0, 10.0)
    assert [(yy, xx) for _, yy, xx in g] == [(0, 0), (19, 19)]

