"""Tensor-core block DCT (B = 16): FP16 hi+lo and BF16 hi+lo split products,
and the single BF16 product, against the FP64 oracle.

Counts never depend on the precision (the pilot decisions are exact), so
they must be bit-exact for every precision.  Coefficients and pixels:
FP16x2 must meet the FP32 bar (1e-5 relative L2); BF16x2 and BF16 are
reported with the bounds their arithmetic gives (16 and 8 significant bits).
"""
import numpy as np
import pytest

import oracle as O
from paper_2001_09632_gb300 import abcs, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

BOUND = {abcs.FP32: 1e-5, abcs.TC_FP16X2: 1e-5, abcs.TC_BF16X2: 1e-4, abcs.TC_BF16: 1e-2}
NAMES = {abcs.FP32: "fp32", abcs.TC_FP16X2: "fp16x2", abcs.TC_BF16X2: "bf16x2", abcs.TC_BF16: "bf16"}


def _oracle(imgs, B, r, variant):
    outs = [O.sense(im, B, r, variant) for im in imgs]
    counts = np.concatenate([o["counts"] for o in outs])
    y = np.concatenate([o["y"] for o in outs])
    return outs, counts, y


@pytest.mark.parametrize("kernel", ["umma", "mma"])
@pytest.mark.parametrize("prec", [abcs.TC_FP16X2, abcs.TC_BF16X2, abcs.TC_BF16])
@pytest.mark.parametrize("variant", [O.ZZ, O.BBV, O.DD])
@pytest.mark.parametrize("shape", [(2, 96, 336), (1, 64, 1040), (3, 48, 48), (5, 160, 208), (2, 80, 337)])
def test_tc_sense_and_reconstruct(handle, monkeypatch, kernel, prec, variant, shape):
    """Both sensing kernels: the per-block mma.sync one (the default) and the
    tcgen05 one (ABCS_SENSE_TC=umma; 16-byte aligned rows only, a row of 337
    bytes falls back to the other)."""
    if kernel == "umma":
        monkeypatch.setenv("ABCS_SENSE_TC", "umma")
    n, H, W = shape
    B, r = 16, 0.3
    imgs = np.stack([synth.gen_image(H, W, 300 + k) for k in range(n)])
    outs, c_ref, y_ref = _oracle(imgs, B, r, variant)
    got = G.sense(handle, imgs, B, r, variant, precision=prec)
    assert got["bits"] == 0
    if variant != O.ZZ:
        assert np.array_equal(got["pilot"], np.concatenate([o["pilot"] for o in outs]))
    assert np.array_equal(got["counts"], c_ref)
    o_ref = np.concatenate([[0], np.cumsum(c_ref)])
    assert np.array_equal(got["offsets"], o_ref)
    G.check_coeffs(got["y"], y_ref, c_ref, o_ref, BOUND[prec])
    rec, _, bits = G.reconstruct(handle, *got["d"], n, H, W, B, precision=prec)
    assert bits == 0
    Hc, Wc = (H // B) * B, (W // B) * B
    for k in range(n):
        ref = O.reconstruct(outs[k]["counts"], outs[k]["y"], Hc, Wc, B)
        G.check_pixels(rec[k], ref, BOUND[prec], k)


@pytest.mark.parametrize("prec", [abcs.TC_FP16X2, abcs.TC_BF16X2, abcs.TC_BF16])
@pytest.mark.parametrize("variant,shape", [(O.BBV, (2, 96, 336)), (O.DD, (5, 160, 208)), (O.ZZ, (3, 48, 48)),
                                           (O.BBV, (9, 512, 512))])
def test_tc_reconstruct_tensor_memory_kernel(handle, monkeypatch, prec, variant, shape):
    """The tcgen05 reconstruct kernel (ABCS_RECON_TC=umma: basis images in
    tensor memory, 128-block tiles) against the oracle; the shapes leave a
    partial last tile, and 9 x 512^2 spans several tiles per CTA."""
    n, H, W = shape
    B, r = 16, 0.3
    imgs = np.stack([synth.gen_image(H, W, 500 + k) for k in range(n)])
    outs, c_ref, _ = _oracle(imgs, B, r, variant)
    got = G.sense(handle, imgs, B, r, variant, precision=prec)
    assert np.array_equal(got["counts"], c_ref)
    monkeypatch.setenv("ABCS_RECON_TC", "umma")
    rec, rec8, bits = G.reconstruct(handle, *got["d"], n, H, W, B, precision=prec, u8=True)
    monkeypatch.delenv("ABCS_RECON_TC")
    assert bits == 0
    # uint8 output: the rounded, clamped FP32 pixels (a value within rounding of .5 may go either way)
    assert np.max(np.abs(rec8.astype(int) - np.clip(np.rint(rec), 0, 255))) <= 1
    rec_mma, _, _ = G.reconstruct(handle, *got["d"], n, H, W, B, precision=prec)
    Hc, Wc = (H // B) * B, (W // B) * B
    for k in range(n):
        ref = O.reconstruct(outs[k]["counts"], outs[k]["y"], Hc, Wc, B)
        G.check_pixels(rec[k], ref, BOUND[prec], k)
        assert G.rel_l2(rec[k], rec_mma[k]) <= BOUND[prec]


def test_precision_table(handle, capsys):
    """Relative L2 error vs FP64, and the PSNR and SSIM of the reconstruction
    against the FP64 reconstruction's, for each precision on 8 images of
    512x512, BBV, r = 0.3 (printed; asserted bounds).  PSNR and SSIM are the
    oracle's definitions (Sec. VII; SSIM of Wang et al.) applied to the
    GPU's output and to the oracle's."""
    B, r = 16, 0.3
    imgs = synth.gen_batch(8, 512, 512, 77)
    outs, c_ref, y_ref = _oracle(imgs, B, r, O.BBV)
    o_ref = np.concatenate([[0], np.cumsum(c_ref)])
    recs_ref = [O.reconstruct(o["counts"], o["y"], 512, 512, B) for o in outs]
    ssim_ref = [O.ssim(recs_ref[k], imgs[k]) for k in range(8)]
    lines = []
    for prec in (abcs.FP32, abcs.TC_FP16X2, abcs.TC_BF16X2, abcs.TC_BF16):
        got = G.sense(handle, imgs, B, r, O.BBV, precision=prec)
        rec, _, _ = G.reconstruct(handle, *got["d"], 8, 512, 512, B, precision=prec)
        assert np.array_equal(got["counts"], c_ref)
        ey = G.check_coeffs(got["y"], y_ref, c_ref, o_ref, BOUND[prec])
        ex = G.check_pixels(rec, np.stack(recs_ref), BOUND[prec])
        dpsnr = np.mean([O.psnr(rec[k], imgs[k]) - O.psnr(recs_ref[k], imgs[k]) for k in range(8)])
        dssim = np.mean([O.ssim(rec[k], imgs[k]) - ssim_ref[k] for k in range(8)])
        lines.append(f"{NAMES[prec]:7s} coeff relL2 {ey:.3e}  pixel relL2 {ex:.3e}  dPSNR {dpsnr:+.5f} dB"
                     f"  dSSIM {dssim:+.2e}")
        if prec in (abcs.FP32, abcs.TC_FP16X2):
            assert abs(dpsnr) <= 1e-3 and abs(dssim) <= 1e-5
    with capsys.disabled():
        print("\n" + "\n".join(lines))


@pytest.mark.parametrize("variant,r", [(O.BBV, 0.3), (O.DD, 0.3), (O.BBV, 0.5), (O.DD, 0.1)])
def test_sense_kernels_agree_on_the_full_batch(handle, monkeypatch, variant, r):
    """64 x 512x512 (the batched workload): the tcgen05 sensing kernel and
    the per-block mma.sync kernel give the same counts and offsets, and
    coefficients within the FP32 bar of each other and of the oracle on
    sampled images (r = 0.5 BBV puts ranks >= 128 in every tile)."""
    B, n = 16, 64
    imgs = synth.gen_batch(n, 512, 512, 4242)
    got_m = G.sense(handle, imgs, B, r, variant, precision=abcs.TC_FP16X2)
    monkeypatch.setenv("ABCS_SENSE_TC", "umma")
    got_u = G.sense(handle, imgs, B, r, variant, precision=abcs.TC_FP16X2)
    monkeypatch.delenv("ABCS_SENSE_TC")
    assert got_u["bits"] == 0 and got_m["bits"] == 0
    assert np.array_equal(got_u["counts"], got_m["counts"])
    assert np.array_equal(got_u["offsets"], got_m["offsets"])
    G.check_coeffs(got_u["y"], got_m["y"], got_m["counts"], got_m["offsets"], 1e-5)
    nB = got_u["plan"]["n_blocks"]
    off = got_u["offsets"]
    for k in (0, 33, 63):
        ref = O.sense(imgs[k], B, r, variant)
        assert np.array_equal(got_u["counts"][k * nB:(k + 1) * nB], ref["counts"])
        G.check_coeffs(got_u["y"][off[k * nB]:off[(k + 1) * nB]], ref["y"], ref["counts"], ref["offsets"], 1e-5, k)


def test_sense_full_batch_counts_and_samples(handle):
    """The bench workload (64 x 512x512, BBV r = 0.3, FP16x2) in the launch
    configuration the bench times: pilot values and counts of every image
    bit-exact against the oracle's BBV and allocation of the same images,
    offsets their exclusive prefix, coefficients of 4 sampled images within
    the FP32 bar."""
    B, r, n = 16, 0.3, 64
    imgs = synth.gen_batch(n, 512, 512, 1234)
    got = G.sense(handle, imgs, B, r, O.BBV, precision=abcs.TC_FP16X2)
    assert got["bits"] == 0
    nB = got["plan"]["n_blocks"]
    p = O.plan(512, 512, B, r, O.BBV)
    for k in range(n):
        Xc = imgs[k].astype(np.int64)
        pilot = O.bbv(Xc, B, p["L"], p["X0"], p["nS"]).reshape(-1)
        assert np.array_equal(got["pilot"][k * nB:(k + 1) * nB], pilot), k
        assert np.array_equal(got["counts"][k * nB:(k + 1) * nB], O.allocate(pilot, p["R"], p["cap"])), k
    assert np.array_equal(got["offsets"], np.concatenate([[0], np.cumsum(got["counts"])]))
    off = got["offsets"]
    for k in (0, 17, 40, 63):
        ref = O.sense(imgs[k], B, r, O.BBV)
        y = got["y"][off[k * nB] - off[0]: off[(k + 1) * nB] - off[0]]
        G.check_coeffs(y, ref["y"], ref["counts"], ref["offsets"], 1e-5, k)


def test_tc_rejects_other_block_sizes(handle):
    import torch
    d = torch.zeros(64 * 64, dtype=torch.uint8, device="cuda")
    c = torch.zeros(64, dtype=torch.int32, device="cuda")
    o = torch.zeros(65, dtype=torch.int64, device="cuda")
    y = torch.zeros(4096, dtype=torch.float32, device="cuda")
    with pytest.raises(abcs.AbcsError) as e:
        abcs.abcs_sense(handle, d, 1, 64, 64, 64, 4096, 8, 0.3, O.ZZ, abcs.TC_FP16X2, c, o, y, 4096)
    assert e.value.status == 2


@pytest.mark.parametrize("kernel", ["umma", "mma"])
@pytest.mark.parametrize("prec", [abcs.TC_FP16X2, abcs.TC_BF16X2, abcs.TC_BF16])
@pytest.mark.parametrize("variant,r", [(O.ZZ, 1.0), (O.DD, 1.0), (O.ZZ, 0.01), (O.DD, 0.01), (O.BBV, 0.01)])
def test_tc_extreme_subrates(handle, monkeypatch, kernel, prec, variant, r):
    """Every coefficient measured (r = 1: full staging buffers in sense and
    reconstruct; for the tensor-memory kernel a worst-case span per tile and,
    on 10 x 512^2 = 80 tiles, two tiles per CTA through its ring) and almost
    none (r = 0.01: m1 = 1 for DD, the L-DCT-ZZ fallback for BBV since
    n_S = 0).  Counts bit-exact; coefficients and both reconstruct kernels
    within the precision's bound."""
    n, H, W, B = 10, 512, 512, 16
    imgs = synth.gen_batch(n, H, W, 2024)
    outs, c_ref, y_ref = _oracle(imgs, B, r, variant)
    if kernel == "umma":
        monkeypatch.setenv("ABCS_SENSE_TC", "umma")
    got = G.sense(handle, imgs, B, r, variant, precision=prec)
    monkeypatch.delenv("ABCS_SENSE_TC", raising=False)
    assert got["bits"] == 0
    assert np.array_equal(got["counts"], c_ref)
    G.check_coeffs(got["y"], y_ref, c_ref, np.concatenate([[0], np.cumsum(c_ref)]), BOUND[prec])
    refs = [O.reconstruct(o["counts"], o["y"], H, W, B) for o in outs]
    rec, _, bits = G.reconstruct(handle, *got["d"], n, H, W, B, precision=prec)
    assert bits == 0
    monkeypatch.setenv("ABCS_RECON_TC", "umma")
    rec_u, _, bits_u = G.reconstruct(handle, *got["d"], n, H, W, B, precision=prec)
    monkeypatch.delenv("ABCS_RECON_TC")
    assert bits_u == 0
    for k in (0, 5, 9):
        G.check_pixels(rec[k], refs[k], BOUND[prec], k)
        G.check_pixels(rec_u[k], refs[k], BOUND[prec], k)


def test_empty_batch_is_rejected(handle):
    import torch
    d = torch.zeros(64 * 64, dtype=torch.uint8, device="cuda")
    c = torch.zeros(16, dtype=torch.int32, device="cuda")
    o = torch.zeros(17, dtype=torch.int64, device="cuda")
    y = torch.zeros(4096, dtype=torch.float32, device="cuda")
    x = torch.zeros(4096, dtype=torch.float32, device="cuda")
    for prec in (abcs.FP32, abcs.TC_FP16X2):
        with pytest.raises(abcs.AbcsError) as e:
            abcs.abcs_sense(handle, d, 0, 64, 64, 64, 4096, 16, 0.3, O.BBV, prec, c, o, y, 4096)
        assert e.value.status == 1
        with pytest.raises(abcs.AbcsError) as e:
            abcs.abcs_reconstruct(handle, c, o, y, 0, 64, 64, 16, prec, x)
        assert e.value.status == 1
    with pytest.raises(abcs.AbcsError) as e:
        abcs.abcs_ida(handle, c, o, y, 0, 64, 64, 16, 2, 2.0, abcs.DEN_TIDCT, 2.3, None, x)
    assert e.value.status == 1
    assert abcs.abcs_sync_status(handle) == 0


@pytest.mark.parametrize("prec", [abcs.FP32, abcs.TC_FP16X2])
def test_blocks_with_no_measurement(handle, prec):
    """Images whose left part is flat: BBV is 0 there, so those blocks get
    m_i = 0 (Eq. 22) and the scatter / gather of every transform must leave
    them out (no store, zero coefficients in the reconstruction), beside
    textured blocks near the cap."""
    n, H, W, B, r = 3, 96, 192, 16, 0.3
    imgs = np.stack([synth.gen_image(H, W, 900 + k) for k in range(n)])
    imgs[:, :, : W // 2] = 117                     # flat half: zero boundary variation
    outs, c_ref, y_ref = _oracle(imgs, B, r, O.BBV)
    assert (c_ref == 0).sum() > 0 and c_ref.max() > 100
    got = G.sense(handle, imgs, B, r, O.BBV, precision=prec)
    assert got["bits"] == 0
    assert np.array_equal(got["counts"], c_ref)
    o_ref = np.concatenate([[0], np.cumsum(c_ref)])
    assert np.array_equal(got["offsets"], o_ref)
    G.check_coeffs(got["y"], y_ref, c_ref, o_ref, BOUND[prec])
    rec, _, bits = G.reconstruct(handle, *got["d"], n, H, W, B, precision=prec)
    assert bits == 0
    for k in range(n):
        ref = O.reconstruct(outs[k]["counts"], outs[k]["y"], H, W, B)
        G.check_pixels(rec[k], ref, BOUND[prec], k)
