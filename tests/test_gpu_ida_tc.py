"""The IDA linear step (Eqs. 25, 28: z = y - A x + z_prev / D_F and
r = x + A^T z) on the tensor cores (B = 16, abcs_set_ida_precision) against
the FP64 oracle.  With D = identity every iterate is linear in y, so the
transform error is all there is: FP16x2 must meet the FP32 bar (1e-5),
BF16x2 and BF16 the sensing bounds of their precision."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2001_09632_gb300 import abcs, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
BOUND = {abcs.TC_FP16X2: 1e-5, abcs.TC_BF16X2: 1e-4, abcs.TC_BF16: 1e-2}


@pytest.fixture
def tc(handle):
    """The handle with a tensor-core precision set by the test; FP32 again after it."""
    def set_precision(p):
        abcs.abcs_set_ida_precision(handle, p)
        return handle
    yield set_precision
    abcs.abcs_set_ida_precision(handle, abcs.FP32)


@pytest.mark.parametrize("precision", list(BOUND))
@pytest.mark.parametrize("DF", [1.0, 2.0])
def test_ida_tc_identity_denoiser_parity(tc, precision, DF):
    """96 x 330 (cropped to 96 x 320: a full 16-block tile and a ragged
    4-block one per block row), BBV r = 0.3, iterations 1, 2, 5 and 12."""
    h = tc(precision)
    H, W, B = 96, 330, 16
    img = synth.gen_image(H, W, 21)
    out = O.sense(img, B, 0.3, O.BBV)
    got = G.sense(h, img[None], B, 0.3, O.BBV)
    tol = BOUND[precision]
    Hc, Wc = out["plan"]["nbh"] * B, out["plan"]["nbw"] * B
    scale = np.linalg.norm(O.reconstruct(out["counts"], out["y"], Hc, Wc, B))
    for iters in (1, 2, 5, 12):
        x, tr, bits = G.ida(h, *got["d"], 1, H, W, B, iters, DF, abcs.DEN_NONE)
        assert bits == 0
        xr, sig = O.ida(out["y"], out["counts"], Hc, Wc, B, iters, DF=DF, denoiser=None)
        # error relative to ||A^T y||: with D_F = 1 some iterates are exactly 0
        assert np.linalg.norm(x[0] - xr) <= tol * scale, iters
        assert np.max(np.abs(x[0] - xr)) <= 10 * tol * 255, iters
        np.testing.assert_allclose(tr[0, :iters], sig, rtol=tol, atol=10 * tol * max(sig))


@pytest.mark.parametrize("variant", [O.BBV, O.DD])
def test_ida_tc_linear_step_full_size(tc, variant):
    """2 x 512x512 at r = 0.3, FP16x2, iterations 1, 3 and 6: every pixel and
    sigma^t against the FP64 oracle at the FP32 bar."""
    h = tc(abcs.TC_FP16X2)
    n, H, W, B, r = 2, 512, 512, 16, 0.3
    imgs = synth.gen_batch(n, H, W, 611)
    got = G.sense(h, imgs, B, r, variant)
    outs = [O.sense(im, B, r, variant) for im in imgs]
    for iters in (1, 3, 6):
        x, tr, bits = G.ida(h, *got["d"], n, H, W, B, iters, 2.0, abcs.DEN_NONE)
        assert bits == 0
        for k in range(n):
            xr, sig = O.ida(outs[k]["y"], outs[k]["counts"], H, W, B, iters, DF=2.0, denoiser=None)
            G.check_pixels(x[k], xr, 1e-5, (iters, k))
            np.testing.assert_allclose(tr[k, :iters], sig, rtol=1e-5)


@pytest.mark.parametrize("r", [0.01, 1.0])
def test_ida_tc_extreme_subrates(tc, r):
    """L-DCT-ZZ with every coefficient measured (r = 1: A^T A = I, so
    r^0 = A^T y is the image itself; the full 16-block tiles hold 4096
    coefficients, more than the kernel stages, so they read y and z_prev
    from global memory, and the 2-block ragged tiles are staged) and with
    2 coefficients per block (r = 0.01)."""
    h = tc(abcs.TC_FP16X2)
    H, W, B = 64, 288, 16
    img = synth.gen_image(H, W, 77)
    out = O.sense(img, B, r, O.ZZ)
    got = G.sense(h, img[None], B, r, O.ZZ)
    for iters in (1, 4):
        x, tr, bits = G.ida(h, *got["d"], 1, H, W, B, iters, 2.0, abcs.DEN_NONE)
        assert bits == 0
        xr, sig = O.ida(out["y"], out["counts"], H, W, B, iters, DF=2.0, denoiser=None)
        G.check_pixels(x[0], xr, 1e-5, iters)
        np.testing.assert_allclose(tr[0, :iters], sig, rtol=1e-5)


def test_ida_tc_tidct_end_to_end(tc):
    """256x256, BBV r = 0.3, 10 iterations with the TI-DCT denoiser on the
    FP16x2 linear step: sigma^0 to 1e-6 and the final PSNR within 0.05 dB of
    the FP64 oracle's (the hard threshold makes the loop discontinuous)."""
    h = tc(abcs.TC_FP16X2)
    H = W = 256
    B, lam = 16, 2.7
    img = synth.gen_image(H, W, 1)
    out = O.sense(img, B, 0.3, O.BBV)
    got = G.sense(h, img[None], B, 0.3, O.BBV)
    x, tr, bits = G.ida(h, *got["d"], 1, H, W, B, 10, 2.0, abcs.DEN_TIDCT, lam)
    assert bits == 0
    xr, sig = O.ida(out["y"], out["counts"], H, W, B, 10, DF=2.0,
                    denoiser=lambda rr, s: O.tidct_denoise(rr, s, lam))
    assert abs(tr[0, 0] - sig[0]) <= 1e-6 * sig[0]
    assert abs(O.psnr(x[0], img) - O.psnr(xr, img)) <= 0.05


def test_ida_tc_capture(tc):
    """abcs_ida_capture runs the same tensor-core step: r^2 and sigma^2
    (identity denoiser) against the oracle's trace."""
    h = tc(abcs.TC_FP16X2)
    H, W, B = 64, 96, 16
    img = synth.gen_image(H, W, 8)
    out = O.sense(img, B, 0.3, O.BBV)
    got = G.sense(h, img[None], B, 0.3, O.BBV)
    _, sig, rs, _ = O.ida(out["y"], out["counts"], H, W, B, 3, DF=2.0, denoiser=None, trace=True)
    r_out = torch.empty((1, H, W), dtype=torch.float32, device="cuda")
    s_out = torch.empty(1, dtype=torch.float32, device="cuda")
    abcs.abcs_ida_capture(h, *got["d"], 1, H, W, B, 2, 2.0, abcs.DEN_NONE, 0.0, None, r_out, s_out)
    assert abcs.abcs_sync_status(h) == 0
    assert G.rel_l2(r_out.cpu().numpy()[0], rs[2]) <= 1e-5
    assert abs(s_out.item() - sig[2]) <= 1e-5 * sig[2]


def test_ida_tc_matches_fp32_path(tc, handle):
    """The two linear-step kernels on the same 3-image DD batch: iterates
    agree to the FP32 bar (they differ only in rounding)."""
    H, W, B = 64, 272, 16
    imgs = np.stack([synth.gen_image(H, W, 50 + k) for k in range(3)])
    got = G.sense(handle, imgs, B, 0.2, O.DD)
    x32, tr32, _ = G.ida(handle, *got["d"], 3, H, W, B, 6, 2.0, abcs.DEN_NONE)
    h = tc(abcs.TC_FP16X2)
    x16, tr16, bits = G.ida(h, *got["d"], 3, H, W, B, 6, 2.0, abcs.DEN_NONE)
    assert bits == 0
    for k in range(3):
        assert G.rel_l2(x16[k], x32[k]) <= 1e-5
    np.testing.assert_allclose(tr16, tr32, rtol=1e-5)


def test_set_ida_precision_rejects_unknown(handle):
    with pytest.raises(abcs.AbcsError) as e:
        abcs.abcs_set_ida_precision(handle, 7)
    assert e.value.status == 1


def test_ida_tc_blocks_with_no_measurement(tc):
    """A flat half gives blocks with m_i = 0 beside textured blocks near the
    cap: their residual is empty (no z, no correction) in every iteration."""
    h = tc(abcs.TC_FP16X2)
    H, W, B = 96, 192, 16
    img = synth.gen_image(H, W, 933)
    img[:, : W // 2] = 117
    out = O.sense(img, B, 0.3, O.BBV)
    assert (out["counts"] == 0).sum() > 0
    got = G.sense(h, img[None], B, 0.3, O.BBV)
    for iters in (1, 4):
        x, tr, bits = G.ida(h, *got["d"], 1, H, W, B, iters, 2.0, abcs.DEN_NONE)
        assert bits == 0
        xr, sig = O.ida(out["y"], out["counts"], H, W, B, iters, DF=2.0, denoiser=None)
        G.check_pixels(x[0], xr, 1e-5, iters)
        np.testing.assert_allclose(tr[0, :iters], sig, rtol=1e-5)
