"""GPU parity of IDA and the plain denoiser against the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2001_09632_gb300 import abcs, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def _ambiguous_mask(r, thr, band=2e-4):
    """Pixels covered by an 8x8 window (of the 64 shifts) holding an AC
    coefficient within `band` of the threshold: there FP32 and FP64 may
    legitimately take different keep/zero decisions.  The band is ~20x the
    typical FP32 error of an 8x8 DCT coefficient of [0, 255] data (~1e-5);
    a flip outside it fails the test."""
    H, W = r.shape
    D = O.dct_matrix(8)
    mask = np.zeros((H, W), bool)
    for sy in range(8):
        ny = -(-(H + sy) // 8)
        rows = np.arange(-sy, -sy + 8 * ny)
        for sx in range(8):
            nx = -(-(W + sx) // 8)
            cols = np.arange(-sx, -sx + 8 * nx)
            ext = r[O.reflect_index(rows, H)][:, O.reflect_index(cols, W)]
            C = D @ ext.reshape(ny, 8, nx, 8).transpose(0, 2, 1, 3) @ D.T
            amb = np.abs(np.abs(C) - thr) <= band
            amb[:, :, 0, 0] = False
            win = amb.any(axis=(2, 3))
            full = np.repeat(np.repeat(win, 8, 0), 8, 1)
            mask |= full[sy:sy + H, sx:sx + W]
    return mask


@pytest.mark.parametrize("H,W", [(64, 64), (100, 250), (200, 520), (13, 300), (3, 5), (1, 17), (7, 30)])
@pytest.mark.parametrize("sigma,lam", [(8.0, 2.7), (25.0, 2.7), (3.0, 0.0)])
def test_tidct_parity(handle, H, W, sigma, lam):
    """Images narrower than a window (3 x 5, 1 x 17, 7 x 30) reflect each
    window several times over."""
    rng = np.random.default_rng(H * W)
    clean = synth.gen_image(max(H, 8), max(W, 8), 5)[:H, :W].astype(float)
    r = clean + rng.standard_normal((H, W)) * sigma
    ref = O.tidct_denoise(r, sigma, lam)
    d_in = torch.tensor(r[None], dtype=torch.float32, device="cuda")
    d_out = torch.full_like(d_in, float("nan"))
    d_sig = torch.tensor([sigma], dtype=torch.float32, device="cuda")
    abcs.abcs_denoise_tidct(handle, d_in, 1, H, W, d_sig, lam, d_out)
    got = d_out.cpu().numpy()[0]
    # the FP32 input itself is rounded: use that exact input for the masks
    r32 = d_in.cpu().numpy()[0].astype(float)
    ref = O.tidct_denoise(r32, float(np.float32(sigma)), lam)
    mask = _ambiguous_mask(r32, lam * float(np.float32(sigma))) if lam > 0 else np.zeros_like(r, bool)
    # measured on these inputs: at most 3.5% of the pixels (100 x 250, sigma 8)
    assert mask.mean() < 0.05, mask.mean()
    err = np.abs(got - ref)[~mask]
    assert err.max() <= 1e-5 * np.abs(ref).max()
    assert G.rel_l2(got[~mask], ref[~mask]) <= 1e-6


def _setup(H, W, B, r, variant, seed):
    img = synth.gen_image(H, W, seed)
    out = O.sense(img, B, r, variant)
    return img, out


@pytest.mark.parametrize("B", [8, 16, 32])
@pytest.mark.parametrize("DF", [1.0, 2.0])
def test_ida_identity_denoiser_parity(handle, B, DF):
    """Linear part of IDA: with D = identity every iterate is linear in y,
    so FP32 must track FP64 to 1e-5 relative L2 at every iteration count."""
    H, W = 96, 320
    img, out = _setup(H, W, B, 0.3, O.BBV, 21)
    got = G.sense(handle, img[None], B, 0.3, O.BBV)
    for iters in (1, 2, 5, 12):
        x, tr, bits = G.ida(handle, *got["d"], 1, H, W, B, iters, DF, abcs.DEN_NONE)
        assert bits == 0
        Hc, Wc = out["plan"]["nbh"] * B, out["plan"]["nbw"] * B
        xr, sig = O.ida(out["y"], out["counts"], Hc, Wc, B, iters, DF=DF, denoiser=None)
        # error relative to ||A^T y||: with D_F = 1 some iterates are exactly 0
        scale = np.linalg.norm(O.reconstruct(out["counts"], out["y"], Hc, Wc, B))
        assert np.linalg.norm(x[0] - xr) <= 1e-5 * scale, iters
        assert np.max(np.abs(x[0] - xr)) <= 1e-4 * 255, iters       # every pixel
        np.testing.assert_allclose(tr[0, :iters], sig, rtol=1e-5, atol=1e-4 * max(sig))


@pytest.mark.parametrize("variant", [O.BBV, O.DD])
def test_ida_linear_step_full_size(handle, variant):
    """The linear part of IDA (Eqs. 25, 28: residual, Onsager term, A^T z) on
    2 x 512x512 images at B = 16, r = 0.3, in the launch configuration of the
    batched workload: with D = identity every iterate is linear in y; every
    pixel and sigma^t of iterations 1, 3 and 6 against the FP64 oracle."""
    n, H, W, B, r = 2, 512, 512, 16, 0.3
    imgs = synth.gen_batch(n, H, W, 611)
    got = G.sense(handle, imgs, B, r, variant)
    outs = [O.sense(im, B, r, variant) for im in imgs]
    for iters in (1, 3, 6):
        x, tr, bits = G.ida(handle, *got["d"], n, H, W, B, iters, 2.0, abcs.DEN_NONE)
        assert bits == 0
        for k in range(n):
            xr, sig = O.ida(outs[k]["y"], outs[k]["counts"], H, W, B, iters, DF=2.0, denoiser=None)
            G.check_pixels(x[k], xr, 1e-5, (iters, k))
            np.testing.assert_allclose(tr[k, :iters], sig, rtol=1e-5)


def test_ida_tidct_end_to_end(handle):
    """256x256 image, BBV r = 0.3, 10 IDA iterations with the TI-DCT
    denoiser.  The hard threshold makes the loop discontinuous, so the bar is:
    sigma^0 to 1e-6, and the final PSNR within 0.05 dB of the FP64 oracle's."""
    H = W = 256
    B, lam = 16, 2.7
    img, out = _setup(H, W, B, 0.3, O.BBV, 1)
    got = G.sense(handle, img[None], B, 0.3, O.BBV)
    x, tr, bits = G.ida(handle, *got["d"], 1, H, W, B, 10, 2.0, abcs.DEN_TIDCT, lam)
    assert bits == 0
    xr, sig = O.ida(out["y"], out["counts"], H, W, B, 10, DF=2.0,
                    denoiser=lambda rr, s: O.tidct_denoise(rr, s, lam))
    assert abs(tr[0, 0] - sig[0]) <= 1e-6 * sig[0]
    p_gpu, p_ref = O.psnr(x[0], img), O.psnr(xr, img)
    p_idct = O.psnr(O.reconstruct(out["counts"], out["y"], H, W, B), img)
    assert abs(p_gpu - p_ref) <= 0.05, (p_gpu, p_ref)
    assert G.rel_l2(x[0], xr) <= 1e-3
    print(f"IDCT {p_idct:.3f} dB, IDA oracle {p_ref:.3f} dB, IDA GPU {p_gpu:.3f} dB")


def test_ida_batch_matches_single(handle):
    H, W, B = 64, 272, 16
    imgs = np.stack([synth.gen_image(H, W, 50 + k) for k in range(3)])
    got = G.sense(handle, imgs, B, 0.2, O.DD)
    xb, trb, _ = G.ida(handle, *got["d"], 3, H, W, B, 4, 2.0, abcs.DEN_TIDCT, 2.7)
    for k in range(3):
        g1 = G.sense(handle, imgs[k:k + 1], B, 0.2, O.DD)
        x1, tr1, _ = G.ida(handle, *g1["d"], 1, H, W, B, 4, 2.0, abcs.DEN_TIDCT, 2.7)
        assert np.array_equal(x1[0], xb[k]) and np.array_equal(tr1[0], trb[k])


def test_ida_capture_matches_oracle_trace(handle):
    """r^t and sigma^t of iteration t (the learned denoiser's training input)."""
    H, W, B = 64, 96, 16
    img, out = _setup(H, W, B, 0.3, O.BBV, 8)
    got = G.sense(handle, img[None], B, 0.3, O.BBV)
    _, sig, rs, _ = O.ida(out["y"], out["counts"], H, W, B, 3, DF=2.0, denoiser=None, trace=True)
    for t in (0, 2):
        r_out = torch.empty((1, H, W), dtype=torch.float32, device="cuda")
        s_out = torch.empty(1, dtype=torch.float32, device="cuda")
        abcs.abcs_ida_capture(handle, *got["d"], 1, H, W, B, t, 2.0, abcs.DEN_NONE, 0.0, None, r_out, s_out)
        assert abcs.abcs_sync_status(handle) == 0
        assert G.rel_l2(r_out.cpu().numpy()[0], rs[t]) <= 1e-5
        assert abs(s_out.item() - sig[t]) <= 1e-5 * sig[t]
