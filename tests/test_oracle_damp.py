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


def test_alpha_uses_the_divergence_at_the_previous_input():
    """Eqs. 24 / 27: alpha^t = div D_{sigma^{t-1}}(r^{t-1}) / (M D_F).  With a
    soft threshold at tau = sigma / 2 the divergence is #{|r_i| > tau}, which
    changes from iterate to iterate; the denoiser logs its inputs, so the
    expected alpha^t is counted by hand on r^{t-1}.  The Monte-Carlo
    estimate differs from the exact count only for entries within eps of
    tau (slack).  The counts of neighbouring iterates differ by more than
    the slacks, so taking the divergence at r^t or at r^{t-2} fails."""
    img = synth.gen_image(48, 64, 12)
    out = O.sense(img, 16, 0.3, O.BBV)
    b = _rademacher((48, 64), 13)
    M = len(out["y"])
    log = []

    def soft(v, s):
        log.append((np.array(v, copy=True), s))
        return np.sign(v) * np.maximum(np.abs(v) - 0.5 * s, 0.0)

    iters, DF = 6, 2.0
    _, sigmas, alphas = O.damp(out["y"], out["counts"], 48, 64, 16, iters, b, DF=DF, denoiser=soft)
    assert len(log) == 2 * iters - 1                       # D(r^t), then D(r^t + eps b) except at the end
    r = [log[2 * t][0] for t in range(iters)]
    for t in range(iters):
        assert log[2 * t][1] == sigmas[t]
        if t + 1 < iters:                                  # the probe call: same sigma, r^t + eps b
            eps = 1e-3 * np.max(np.abs(r[t]))
            assert log[2 * t + 1][1] == sigmas[t]
            assert np.allclose(log[2 * t + 1][0], r[t] + eps * b, rtol=0, atol=1e-12 * np.max(np.abs(r[t])))

    def count(t):
        return int(np.sum(np.abs(r[t]) > 0.5 * sigmas[t]))

    def slack(t):
        eps = 1e-3 * np.max(np.abs(r[t]))
        return int(np.sum(np.abs(np.abs(r[t]) - 0.5 * sigmas[t]) <= eps))

    assert alphas[0] == 0.0
    discriminating = 0
    for t in range(1, iters):
        assert abs(alphas[t] * M * DF - count(t - 1)) <= slack(t - 1) + 1e-6, t
        if abs(count(t) - count(t - 1)) > slack(t) + slack(t - 1):
            discriminating += 1
    assert discriminating >= 3
