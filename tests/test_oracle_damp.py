"""Pins of the oracle's D-AMP / DAMP-D (Eqs. 24, 27) and of its Monte-Carlo
divergence, against closed forms."""
import numpy as np
import pytest

import oracle as O
from paper_2001_09632_gb300 import synth


def _rademacher(shape, seed):
    return np.where(np.random.default_rng(seed).random(shape) < 0.5, -1.0, 1.0)


def test_divergence_of_linear_and_soft_threshold_denoisers():
    rng = np.random.default_rng(0)
    r = rng.normal(0, 30, (16, 24))
    b = _rademacher(r.shape, 1)
    # linear shrink D(r) = c r: div = c N exactly
    for c in (1.0, 0.5, 0.125):
        d = O.mc_divergence(lambda v, s: c * v, r, 1.0, c * r, b)
        assert d == pytest.approx(c * r.size, rel=1e-9)
    # soft threshold at tau: derivative 1 where |r| > tau, else 0 (no r within eps of tau)
    tau = 20.0
    near = np.abs(np.abs(r) - tau) < 1.0                          # keep every |r| away from tau
    r[near] = np.sign(r[near]) * (tau + 2.0)
    soft = lambda v, s: np.sign(v) * np.maximum(np.abs(v) - tau, 0.0)
    eps = 1e-3 * np.max(np.abs(r))
    assert np.all(np.abs(np.abs(r) - tau) > eps)
    d = O.mc_divergence(soft, r, 1.0, soft(r, 1.0), b)
    assert d == pytest.approx(float(np.sum(np.abs(r) > tau)), rel=1e-9)


def test_identity_denoiser_alpha_closed_form():
    """With D = identity, div = b^T b = N for a +-1 probe, so every
    alpha^t (t >= 1) is N / (M D_F)."""
    img = synth.gen_image(48, 64, 3)
    out = O.sense(img, 16, 0.3, O.BBV)
    b = _rademacher((48, 64), 2)
    M = len(out["y"])
    for DF in (1.0, 2.0):
        _, _, alphas = O.damp(out["y"], out["counts"], 48, 64, 16, 4, b, DF=DF)
        assert alphas[0] == 0.0
        for a in alphas[1:]:
            assert a == pytest.approx(48 * 64 / (M * DF), rel=1e-12)


def test_first_iteration_equals_ida():
    """alpha^0 multiplies z^{-1} = 0: the first iterate of D-AMP is IDA's."""
    img = synth.gen_image(32, 48, 4)
    out = O.sense(img, 16, 0.3, O.DD)
    b = _rademacher((32, 48), 5)
    den = lambda r, s: O.tidct_denoise(r, s, 2.3)
    x1, s1, _ = O.damp(out["y"], out["counts"], 32, 48, 16, 1, b, DF=1.0, denoiser=den)
    xi, si = O.ida(out["y"], out["counts"], 32, 48, 16, 1, DF=2.0, denoiser=den)
    assert np.array_equal(x1, xi) and s1 == si
