"""abcs_psnr_ssim (the paper's PSNR and SSIM, Tables 3, 6, 7) against the
oracle's definitions: x clipped to [0, 255], SSIM of Wang et al. with an
11 x 11 Gaussian window (sigma 1.5) over the valid region."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2001_09632_gb300 import abcs, synth

pytestmark = pytest.mark.gpu


def _run(h, x, ref, pitch=None):
    """x: (n, H, W) float; ref: (n, H, W) uint8 (optionally padded to `pitch`)."""
    n, H, W = x.shape
    if pitch is None:
        pitch = W
    buf = np.full((n, H, pitch), 77, np.uint8)
    buf[:, :, :W] = ref
    d_x = torch.tensor(x, dtype=torch.float32, device="cuda")
    d_r = torch.from_numpy(buf).cuda()
    ps = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    ss = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    abcs.abcs_psnr_ssim(h, d_x, d_r, n, H, W, pitch, H * pitch, ps, ss)
    assert abcs.abcs_sync_status(h) == 0
    return ps.cpu().numpy(), ss.cpu().numpy(), d_x.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n,H,W,pitch", [(3, 64, 80, None), (2, 11, 11, None), (2, 37, 100, 112), (1, 90, 45, 48)])
def test_psnr_ssim_match_oracle(handle, n, H, W, pitch):
    """Reconstructions with noise, blur and values outside [0, 255] (the
    clipping), ragged tiles of the SSIM map, a padded reference."""
    rng = np.random.default_rng(H * W)
    ref = np.stack([synth.gen_image(max(H, 16), max(W, 16), 40 + k)[:H, :W] for k in range(n)])
    x = ref.astype(np.float64) + rng.normal(0, 12, ref.shape) + rng.normal(0, 30) * (rng.random(ref.shape) < 0.02)
    ps, ss, x32 = _run(handle, x, ref, pitch)
    for k in range(n):
        assert abs(ps[k] - O.psnr(x32[k], ref[k])) <= 1e-6 * abs(ps[k]), k
        assert abs(ss[k] - O.ssim(x32[k], ref[k])) <= 1e-5, k


def test_identical_images(handle):
    """Identical images: PSNR +infinity, SSIM 1."""
    ref = synth.gen_batch(2, 40, 56, 9)
    ps, ss, _ = _run(handle, ref.astype(np.float64), ref)
    assert np.all(np.isinf(ps)) and np.all(ps > 0)
    np.testing.assert_allclose(ss, 1.0, atol=1e-7)


def test_full_size(handle):
    """2 x 512x512 and one 1088 x 1920 frame (the benches' image sizes)."""
    for n, H, W in ((2, 512, 512), (1, 1088, 1920)):
        ref = synth.gen_batch(n, H, W, 71) if H == 512 else synth.gen_video(1, H, W, 72)
        rng = np.random.default_rng(n + H)
        x = ref + rng.normal(0, 6, ref.shape)
        ps, ss, x32 = _run(handle, x, ref)
        for k in range(n):
            assert abs(ps[k] - O.psnr(x32[k], ref[k])) <= 1e-6 * ps[k]
            assert abs(ss[k] - O.ssim(x32[k], ref[k])) <= 1e-5


def test_rejects_small_images(handle):
    x = torch.zeros((1, 10, 40), device="cuda")
    r = torch.zeros((1, 10, 40), dtype=torch.uint8, device="cuda")
    o = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(abcs.AbcsError) as e:
        abcs.abcs_psnr_ssim(handle, x, r, 1, 10, 40, 40, 400, o, o)
    assert e.value.status == 1
