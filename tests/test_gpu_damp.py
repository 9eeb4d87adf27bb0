"""GPU parity of D-AMP / DAMP-D (Eqs. 24, 27; abcs_damp) against the FP64
oracle, with the same +-1 probe on both sides.

With the identity denoiser the divergence is b^T b = N exactly, so alpha^t
has the closed form N / (M D_F) and the iteration is linear; the bar is
1e-4 of the trajectory's largest sigma (alpha's FP32 estimate has a
relative error near 6e-5, and the recursion cancels: alpha > 1 here).  With
the TI-DCT denoiser the Monte-Carlo divergence also sees the threshold
decisions of D(r + eps b); a decision that flips between FP32 and FP64 moves
alpha by about 0.3% of its value, so the first iterations are compared
within 2% (alpha) and 1e-3 (images).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2001_09632_gb300 import abcs, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def _probe(n, H, W, seed):
    rng = np.random.default_rng(seed)
    return np.where(rng.random((n, H, W)) < 0.5, -1.0, 1.0).astype(np.float32)


def _run(handle, got, n, H, W, B, iters, DF, den, probe, lam=2.3):
    Hc, Wc = (H // B) * B, (W // B) * B
    x = torch.full((n, Hc, Wc), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.zeros((n, iters), dtype=torch.float32, device="cuda")
    at = torch.full((n, iters), float("nan"), dtype=torch.float32, device="cuda")
    pb = torch.tensor(probe, device="cuda")
    abcs.abcs_damp(handle, *got["d"], n, H, W, B, iters, DF, den, lam, None, pb, x, st, at)
    assert abcs.abcs_sync_status(handle) == 0
    return x.cpu().numpy(), st.cpu().numpy(), at.cpu().numpy()


@pytest.mark.parametrize("DF", [1.0, 2.0])
def test_identity_denoiser_alpha_closed_form_and_iterates(handle, DF):
    n, H, W, B = 2, 64, 96, 16
    imgs = np.stack([synth.gen_image(H, W, 70 + k) for k in range(n)])
    got = G.sense(handle, imgs, B, 0.3, O.BBV)
    probe = _probe(n, H, W, 1)
    iters = 4
    x, st, at = _run(handle, got, n, H, W, B, iters, DF, abcs.DEN_NONE, probe)
    nB = got["plan"]["n_blocks"]
    for k in range(n):
        out = O.sense(imgs[k], B, 0.3, O.BBV)
        M = len(out["y"])
        assert at[k, 0] == 0.0
        assert np.allclose(at[k, 1:], H * W / (M * DF), rtol=1e-4)
        xr, sr, ar = O.damp(out["y"], out["counts"], H, W, B, iters, probe[k].astype(float), DF=DF)
        # alpha's FP32 estimate forms (r + eps b) - r with eps = max|r| / 1000: a
        # relative error of about 2^-24 * 1000 ~ 6e-5 per element, multiplied into
        # z^{t-1}; the recursion cancels (alpha > 1 here), so the bar is 1e-4 of the
        # trajectory's largest sigma, and for x scaled by how far it shrinks
        amp = max(sr) / sr[-1]
        assert np.all(np.abs(st[k] - sr) <= 1e-4 * max(sr)), (st[k], sr)
        assert G.rel_l2(x[k], xr) <= 1e-4 * amp


@pytest.mark.parametrize("DF", [1.0, 2.0])
def test_tidct_damp_first_iterations(handle, DF):
    n, H, W, B = 2, 64, 96, 16
    imgs = np.stack([synth.gen_image(H, W, 80 + k) for k in range(n)])
    got = G.sense(handle, imgs, B, 0.3, O.DD)
    probe = _probe(n, H, W, 2)
    iters = 3
    x, st, at = _run(handle, got, n, H, W, B, iters, DF, abcs.DEN_TIDCT, probe)
    for k in range(n):
        out = O.sense(imgs[k], B, 0.3, O.DD)
        den = lambda r, s: O.tidct_denoise(r, s, 2.3)
        xr, sr, ar = O.damp(out["y"], out["counts"], H, W, B, iters, probe[k].astype(float), DF=DF, denoiser=den)
        assert at[k, 0] == 0.0
        assert np.allclose(at[k, 1:], ar[1:], rtol=2e-2), (at[k], ar)
        assert np.allclose(st[k], sr, rtol=1e-3), (st[k], sr)
        assert G.rel_l2(x[k], xr) <= 1e-3


def test_damp_needs_a_probe(handle):
    got = G.sense(handle, synth.gen_image(32, 32, 1)[None], 16, 0.3, O.BBV)
    x = torch.empty((1, 32, 32), dtype=torch.float32, device="cuda")
    with pytest.raises(abcs.AbcsError):
        abcs.abcs_damp(handle, *got["d"], 1, 32, 32, 16, 2, 1.0, abcs.DEN_NONE, 0.0, None, None, x)
