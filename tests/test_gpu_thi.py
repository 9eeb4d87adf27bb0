"""GPU parity of THI (full sensing, the M coefficients of largest magnitude
per image; Sec. IV, Sec. V-B, Table 2) against the FP64 oracle.

The GPU ranks the FP32 coefficients abcs_sense writes; the oracle ranks its
FP64 ones.  The two rankings can differ only between coefficients within
FP32 rounding of the threshold, so counts are compared bit-exactly when the
M-th coefficient is the only one in that band, and otherwise checked to
differ by at most the coefficients in the band (both keep exactly M).
Whatever the band, the GPU's selection is checked in full on the FP32
values it ranked (exactly M kept, nothing dropped above a kept magnitude,
ties in index order, counts and masked values consistent), and rho and the
THI image are compared with the oracle's on the GPU's kept set.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2001_09632_gb300 import abcs, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def _full(handle, imgs, B):
    """Every coefficient of every block (ZZ at subrate 1), zigzag order per block."""
    n, H, W = imgs.shape
    got = G.sense(handle, imgs, B, 1.0, O.ZZ)
    assert got["bits"] == 0
    nB = got["plan"]["n_blocks"]
    assert np.all(got["counts"] == B * B)
    return got["d"][2][: n * nB * B * B], nB


def _thi(handle, coeffs, n, H, W, B, M, adaptive=None, masked=True):
    nB = (H // B) * (W // B)
    counts = torch.full((n * nB,), -1, dtype=torch.int32, device="cuda")
    rho = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") if adaptive is not None else None
    mk = torch.full_like(coeffs, float("nan")) if masked else None
    abcs.abcs_thi(handle, coeffs, n, H, W, B, M, adaptive, counts, rho, mk)
    assert abcs.abcs_sync_status(handle) == 0
    return counts.cpu().numpy(), (rho.cpu().numpy() if rho is not None else None), mk


def _band(img, B, M):
    """Coefficients within FP32 rounding of the FP64 threshold."""
    mag = np.sort(np.abs(O.full_coefficients(img, B)).reshape(-1))[::-1]
    t = mag[M - 1]
    return int(np.sum(np.abs(mag - t) <= 2e-6 * t + 2e-3))


def _check_kept_set(Z, mk, counts, M, tag=""):
    """Full validity of one image's selection, on the FP32 coefficients the
    GPU ranked: exactly M kept; the masked output holds the kept
    coefficients bit for bit and zeros elsewhere; every kept |c| >= every
    dropped |c|; among magnitudes equal to the threshold the lowest
    (block, zigzag rank) indices are kept; the counts are the per-block
    numbers kept.  Returns the kept mask (n_B, B*B)."""
    Z = np.asarray(Z, dtype=np.float32)
    mk = np.asarray(mk, dtype=np.float32)
    kept = mk != 0
    assert np.all((mk == 0) | (mk == Z)), tag                    # kept values are the inputs, bit for bit
    a = np.abs(Z).reshape(-1)
    k = kept.reshape(-1)
    t = a[k].min()
    assert t > 0, tag                                            # no zero coefficient needs keeping here
    assert int(k.sum()) == M, (tag, int(k.sum()), M)
    assert np.all(a[~k] <= t), tag                               # nothing dropped above the threshold
    tied = np.flatnonzero(a == t)
    n_tied_kept = M - int(np.sum(a > t))
    assert np.array_equal(np.flatnonzero(k & (a == t)), tied[:n_tied_kept]), tag   # ties in index order
    assert np.array_equal(np.asarray(counts), kept.sum(axis=1)), tag
    return kept


def _check_counts(got, ref, amb):
    assert got.sum() == ref.sum()
    if amb <= 1:
        assert np.array_equal(got, ref)
    else:
        assert np.abs(got - ref).sum() <= 2 * (amb - 1)


@pytest.mark.parametrize("shape,B", [((1, 64, 64), 16), ((3, 96, 336), 16), ((2, 100, 337), 8),
                                     ((1, 64, 300), 32), ((2, 40, 104), 4)])
@pytest.mark.parametrize("variant", [O.BBV, O.DD])
def test_thi_counts_rho_and_image(handle, shape, B, variant):
    n, H, W = shape
    r = 0.3
    imgs = np.stack([synth.gen_image(H, W, 40 + k) for k in range(n)])
    coeffs, nB = _full(handle, imgs, B)
    ad = G.sense(handle, imgs, B, r, variant)
    M = O.plan(H, W, B, r, variant)["M"]
    counts, rho, mk = _thi(handle, coeffs, n, H, W, B, M, adaptive=ad["d"][0])
    Hc, Wc = (H // B) * B, (W // B) * B
    offs = torch.arange(0, n * nB + 1, dtype=torch.int64, device="cuda") * (B * B)
    full = torch.full((n * nB,), B * B, dtype=torch.int32, device="cuda")
    rec, _, bits = G.reconstruct(handle, full, offs, mk, n, H, W, B)
    assert bits == 0
    Zg = coeffs.cpu().numpy().reshape(n, nB, B * B)
    Mk = mk.cpu().numpy().reshape(n, nB, B * B)
    zr = O.zigzag_rank(B).reshape(-1)
    for k in range(n):
        ref = O.thi_counts(imgs[k], B, M)
        amb = _band(imgs[k], B, M)
        got = counts[k * nB:(k + 1) * nB]
        _check_counts(got, ref, amb)
        kept = _check_kept_set(Zg[k], Mk[k], got, M, k)
        # rho of the GPU's counts, and the image of the GPU's kept set with
        # the oracle's FP64 coefficients
        assert rho[k] == pytest.approx(O.pearson(got, ad["counts"][k * nB:(k + 1) * nB]), abs=1e-12)
        Zo = np.where(kept, O.full_coefficients(imgs[k], B), 0.0)
        img_kept = O.idct2_blocks(Zo[:, zr].reshape(Hc // B, Wc // B, B, B))
        G.check_pixels(rec[k], img_kept, 1e-5, k)
        if amb <= 1:
            assert rho[k] == pytest.approx(O.pearson(ref, ad["counts"][k * nB:(k + 1) * nB]), abs=1e-12)
            G.check_pixels(rec[k], O.thi_reconstruct(imgs[k], B, M)[:Hc, :Wc], 1e-5, k)


def test_thi_ties_follow_block_order(handle):
    """Identical blocks: the one coefficient beyond the DCs goes to block 0,
    and three beyond two per block go to blocks 0, 1, 2."""
    B = 16
    rng = np.random.default_rng(3)
    tile = rng.integers(0, 256, (B, B)).astype(np.uint8)
    img = np.tile(tile, (3, 5))[None]
    coeffs, nB = _full(handle, img, B)
    H, W = img.shape[1:]
    c1, _, _ = _thi(handle, coeffs, 1, H, W, B, nB + 1)
    assert np.array_equal(c1, O.thi_counts(img[0], B, nB + 1))
    assert c1[0] == 2 and np.all(c1[1:] == 1)
    c2, _, _ = _thi(handle, coeffs, 1, H, W, B, 2 * nB + 3)
    assert np.array_equal(c2, O.thi_counts(img[0], B, 2 * nB + 3))


def test_thi_edges(handle):
    B = 8
    img = synth.gen_image(48, 64, 9)[None]
    coeffs, nB = _full(handle, img, B)
    N = nB * B * B
    c, _, mk = _thi(handle, coeffs, 1, 48, 64, B, N)                 # everything kept
    assert np.all(c == B * B)
    assert torch.equal(mk, coeffs)
    c, _, mk = _thi(handle, coeffs, 1, 48, 64, B, 1)                 # the single largest
    assert c.sum() == 1 and np.array_equal(c, O.thi_counts(img[0], B, 1))
    assert int((mk != 0).sum()) == 1
    cnt = torch.zeros(nB, dtype=torch.int32, device="cuda")
    for bad in (0, N + 1):
        with pytest.raises(abcs.AbcsError):
            abcs.abcs_thi(handle, coeffs, 1, 48, 64, B, bad, None, cnt, None, None)
    with pytest.raises(abcs.AbcsError):
        abcs.abcs_thi(handle, coeffs, 1, 48, 64, B, 5, None, cnt,
                      torch.zeros(1, dtype=torch.float64, device="cuda"), None)


def test_thi_full_batch(handle):
    """The 64 x 512x512 batch (B = 16, BBV r = 0.3): every image keeps
    exactly M; counts and rho of three sampled images against the oracle."""
    B, r, n = 16, 0.3, 64
    imgs = synth.gen_batch(n, 512, 512, 1234)
    coeffs, nB = _full(handle, imgs, B)
    ad = G.sense(handle, imgs, B, r, O.BBV, precision=abcs.TC_FP16X2)
    M = O.plan(512, 512, B, r, O.BBV)["M"]
    counts, rho, mk = _thi(handle, coeffs, n, 512, 512, B, M, adaptive=ad["d"][0], masked=True)
    assert np.all(counts.reshape(n, nB).sum(axis=1) == M)
    assert np.all((rho > 0.0) & (rho <= 1.0))
    Zg = coeffs.cpu().numpy().reshape(n, nB, B * B)
    Mk = mk.cpu().numpy().reshape(n, nB, B * B)
    for k in range(n):                                   # every image: a valid selection of exactly M
        _check_kept_set(Zg[k], Mk[k], counts[k * nB:(k + 1) * nB], M, k)
        assert rho[k] == pytest.approx(O.pearson(counts[k * nB:(k + 1) * nB], ad["counts"][k * nB:(k + 1) * nB]),
                                       abs=1e-12)
    for k in (0, 31, 63):
        ref = O.thi_counts(imgs[k], B, M)
        amb = _band(imgs[k], B, M)
        _check_counts(counts[k * nB:(k + 1) * nB], ref, amb)
        if amb <= 1:
            assert rho[k] == pytest.approx(O.pearson(ref, ad["counts"][k * nB:(k + 1) * nB]), abs=1e-12)
