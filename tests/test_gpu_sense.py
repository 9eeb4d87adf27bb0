"""GPU parity of sensing and reconstruction against the FP64 oracle.

Counts, offsets and pilot values must be bit-exact.  Coefficients and
pixels must be within 1e-5 relative L2 (FP32).  Sizes span several CTA
tiles (256 pixel columns each) with ragged tails and cropped edges.
"""
import numpy as np
import pytest

import oracle as O
from paper_2001_09632_gb300 import abcs, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _oracle_batch(imgs, B, r, variant):
    outs = [O.sense(im, B, r, variant) for im in imgs]
    counts = np.concatenate([o["counts"] for o in outs])
    offsets = np.concatenate([[0], np.cumsum(counts)])
    y = np.concatenate([o["y"] for o in outs])
    pilot = np.concatenate([o["pilot"] for o in outs])
    return counts, offsets, y, pilot, outs


CASES = [
    # (n, H, W, B)  -- widths cover 1, 2 and 3 tiles plus ragged tails and crops
    (1, 64, 64, 16),
    (3, 96, 336, 16),
    (2, 100, 337, 16),
    (2, 72, 520, 8),
    (1, 64, 300, 32),
    (2, 40, 1030, 4),
]


@pytest.mark.parametrize("variant", [O.ZZ, O.BBV, O.DD])
@pytest.mark.parametrize("r", [0.1, 0.3, 0.5])
@pytest.mark.parametrize("case", CASES)
def test_sense_parity(handle, case, r, variant):
    n, H, W, B = case
    imgs = np.stack([synth.gen_image(H, W, 100 + k) for k in range(n)])
    c_ref, o_ref, y_ref, p_ref, _ = _oracle_batch(imgs, B, r, variant)
    got = G.sense(handle, imgs, B, r, variant)
    assert got["bits"] == 0
    assert np.array_equal(got["counts"], c_ref)
    assert np.array_equal(got["offsets"], o_ref)
    if variant != O.ZZ:
        assert np.array_equal(got["pilot"], p_ref)
    assert len(got["y"]) == len(y_ref)
    G.check_coeffs(got["y"], y_ref, c_ref, o_ref, TOL)
    # reconstruction of the same measurements
    rec, rec8, bits = G.reconstruct(handle, *got["d"], n, H, W, B, u8=True)
    assert bits == 0
    Hc, Wc = (H // B) * B, (W // B) * B
    for k in range(n):
        ref = O.reconstruct(c_ref[k * (Hc // B) * (Wc // B):(k + 1) * (Hc // B) * (Wc // B)],
                            y_ref[o_ref[k * (Hc // B) * (Wc // B)]:o_ref[(k + 1) * (Hc // B) * (Wc // B)]],
                            Hc, Wc, B)
        G.check_pixels(rec[k], ref, TOL, k)
        ref8 = np.clip(np.round(ref), 0, 255)
        assert np.max(np.abs(rec8[k].astype(float) - ref8)) <= 1    # rounding ties may differ


def test_sense_pitched_rows(handle):
    imgs = np.stack([synth.gen_image(48, 200, 7)])
    ref = _oracle_batch(imgs, 16, 0.3, O.BBV)
    got = G.sense(handle, imgs, 16, 0.3, O.BBV, pitch=272)
    assert np.array_equal(got["counts"], ref[0])
    G.check_coeffs(got["y"], ref[2], ref[0], ref[1], TOL)


@pytest.mark.parametrize("B", [4, 8, 16, 32])
def test_full_measurement_recovers_image(handle, B):
    imgs = np.stack([synth.gen_image(2 * B + 64, 3 * B + 256, 9)])
    got = G.sense(handle, imgs, B, 1.0, O.ZZ)
    assert np.all(got["counts"] == B * B)
    rec, rec8, _ = G.reconstruct(handle, *got["d"], 1, imgs.shape[1], imgs.shape[2], B, u8=True)
    Hc, Wc = rec.shape[1:]
    assert np.max(np.abs(rec[0] - imgs[0, :Hc, :Wc])) < 2e-3
    assert np.array_equal(rec8[0], imgs[0, :Hc, :Wc])


def test_dd_exact_ties(handle):
    """DC = T exactly is not counted; DC = T + 1/8 is (Sec. V-B 'exceeds')."""
    x = np.full((8, 8), 2, np.uint8)
    x[0, :] = 1                               # sum 120 -> DC = 15 = T at C_F = 2
    y = x.copy(); y[7, 7] = 3                 # sum 121
    imgs = np.stack([np.tile(x, (1, 40)), np.tile(y, (1, 40))])   # 8 x 320, two tiles
    got = G.sense(handle, imgs, 8, 0.5, O.DD)
    assert got["plan"]["T"] == 15
    assert np.all(got["pilot"][:40] == 0) and np.all(got["pilot"][40:] == 1)
    ref = _oracle_batch(imgs, 8, 0.5, O.DD)
    assert np.array_equal(got["counts"], ref[0])


def test_dd_exact_rational_coefficient(handle):
    s4 = np.sign(np.cos(np.pi * (2 * np.arange(8) + 1) / 4)).astype(int)
    x = np.full((8, 8), 2, np.int64)
    x[:6, s4 > 0] += 10                       # c(0,4) = 30 exactly
    x2 = x.copy(); x2[7, 0] += 1
    imgs = np.stack([np.tile(x, (1, 33)), np.tile(x2, (1, 33))]).astype(np.uint8)
    r = 1.0 / 2.1
    ref = _oracle_batch(imgs, 8, r, O.DD)
    got = G.sense(handle, imgs, 8, r, O.DD)
    assert np.array_equal(got["pilot"], ref[3]) and np.array_equal(got["counts"], ref[0])


def test_constant_image_bbv_falls_back(handle):
    imgs = np.full((1, 64, 64), 131, np.uint8)
    got = G.sense(handle, imgs, 16, 0.3, O.BBV)
    assert np.all(got["counts"] == int(256 * 0.3)) and np.all(got["pilot"] == 0)


def test_argument_errors(handle):
    import torch
    d = torch.zeros(64 * 64, dtype=torch.uint8, device="cuda")
    c = torch.zeros(16, dtype=torch.int32, device="cuda")
    o = torch.zeros(17, dtype=torch.int64, device="cuda")
    y = torch.zeros(4096, dtype=torch.float32, device="cuda")
    with pytest.raises(abcs.AbcsError) as e:       # capacity below n * M
        abcs.abcs_sense(handle, d, 1, 64, 64, 64, 4096, 16, 0.3, O.BBV, 0, c, o, y, 100)
    assert e.value.status == 3
    with pytest.raises(abcs.AbcsError) as e:       # L = 1 for BBV
        abcs.abcs_sense(handle, d, 1, 64, 64, 64, 4096, 16, 0.6, O.BBV, 0, c, o, y, 4096)
    assert e.value.status == 2
    with pytest.raises(abcs.AbcsError) as e:       # image smaller than a block
        abcs.abcs_sense(handle, d, 1, 8, 64, 64, 4096, 16, 0.3, O.BBV, 0, c, o, y, 4096)
    assert e.value.status == 1
    with pytest.raises(abcs.AbcsError) as e:
        abcs.abcs_sense(handle, None, 1, 64, 64, 64, 4096, 16, 0.3, O.BBV, 0, c, o, y, 4096)
    assert e.value.status == 1
    assert abcs.abcs_sync_status(handle) == 0


@pytest.mark.parametrize("variant", [O.BBV, O.DD])
def test_full_size_batch_counts(handle, variant):
    """64 x 512^2, B = 16, r = 0.3 (the batched benchmark workload): counts,
    offsets and pilot bit-exact for every image; coefficients of a sample of
    images within tolerance."""
    n, H, W = 64, 512, 512
    imgs = synth.gen_batch(n, H, W, 1000)
    got = G.sense(handle, imgs, 16, 0.3, variant)
    assert got["bits"] == 0
    c_ref, o_ref, y_ref, p_ref, _ = _oracle_batch(imgs, 16, 0.3, variant)
    assert np.array_equal(got["counts"], c_ref)
    assert np.array_equal(got["offsets"], o_ref)
    assert np.array_equal(got["pilot"], p_ref)
    G.check_coeffs(got["y"], y_ref, c_ref, o_ref, TOL)
