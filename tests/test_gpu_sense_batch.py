"""abcs_sense_batch: images of different sizes, block sizes, variants and
subrates sensed in two launches (Alg. 1 / Alg. 2 per image), against the
FP64 oracle image by image: counts, pilot values and offsets bit-exact,
measurements within the FP32 bar; the layout is the batch's global one."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2001_09632_gb300 import abcs, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
TOL = 1e-5

# (H, W, B, variant, subrate, extra pitch bytes): every block size and
# variant, cropped sizes, ragged tile columns, padded rows, L-DCT-ZZ and BBV
# with n_S = 0 (B = 4 at subrate 0.2) among them
MIXED = [(64, 80, 16, O.BBV, 0.3, 0), (96, 336, 16, O.DD, 0.3, 16), (100, 337, 8, O.BBV, 0.1, 3),
         (48, 48, 32, O.ZZ, 0.25, 0), (72, 520, 8, O.DD, 0.5, 0), (64, 300, 32, O.BBV, 0.4, 20),
         (40, 104, 4, O.BBV, 0.2, 0), (33, 530, 16, O.DD, 0.1, 7), (256, 256, 16, O.BBV, 0.3, 0)]


def _layout(imgs, specs, align=1):
    """One uint8 buffer; image k at an offset with its own pitch."""
    descs, off = [], 0
    for img, (H, W, B, v, r, extra) in zip(imgs, specs):
        pitch = W + extra
        descs.append((H, W, B, v, r, off, pitch))
        off += (H * pitch + align - 1) // align * align + 5       # odd gaps between images
    buf = np.full(off + 16, 0xA5, np.uint8)
    for img, d in zip(imgs, descs):
        H, W, pitch, o = d[0], d[1], d[6], d[5]
        view = buf[o:o + H * pitch].reshape(H, pitch)
        view[:, :W] = img
    return torch.from_numpy(buf).cuda(), descs


def _run(handle, buf, descs, pilot=True):
    plans = [abcs.abcs_plan(H, W, B, r, v) for (H, W, B, v, r, _, _) in descs]
    nb = sum(p["n_blocks"] for p in plans)
    cap = sum(p["M"] for p in plans)
    c = torch.full((nb,), -7, dtype=torch.int32, device="cuda")
    o = torch.full((nb + 1,), -7, dtype=torch.int64, device="cuda")
    y = torch.full((max(cap, 1),), float("nan"), dtype=torch.float32, device="cuda")
    p = torch.full((nb,), -7, dtype=torch.int32, device="cuda") if pilot else None
    abcs.abcs_sense_batch(handle, buf, descs, abcs.FP32, c, o, y, cap, p)
    assert abcs.abcs_sync_status(handle) == 0
    off = o.cpu().numpy()
    return plans, c.cpu().numpy(), off, y[:int(off[-1])].cpu().numpy(), (p.cpu().numpy() if pilot else None)


def _check_against_oracle(imgs, descs, plans, counts, off, y, pilot, sample=None):
    b0 = 0
    assert off[0] == 0
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(counts)]))
    for k, (img, d, p) in enumerate(zip(imgs, descs, plans)):
        H, W, B, v, r = d[:5]
        nB = p["n_blocks"]
        if sample is None or k in sample:
            ref = O.sense(img, B, r, v)
            assert np.array_equal(counts[b0:b0 + nB], ref["counts"]), k
            if pilot is not None:       # zero for L-DCT-ZZ and BBV with n_S = 0
                assert np.array_equal(pilot[b0:b0 + nB], ref["pilot"]), k
            yk = y[off[b0]:off[b0 + nB]]
            G.check_coeffs(yk, ref["y"], ref["counts"], ref["offsets"], TOL, k)
        b0 += nB


@pytest.mark.parametrize("pilot", [True, False])
def test_sense_batch_mixed_matches_oracle(handle, pilot):
    imgs = [synth.gen_image(H, W, 900 + k) for k, (H, W, *_) in enumerate(MIXED)]
    buf, descs = _layout(imgs, MIXED)
    plans, counts, off, y, pl = _run(handle, buf, descs, pilot)
    _check_against_oracle(imgs, descs, plans, counts, off, y, pl)


def test_sense_batch_equals_per_image_sense(handle):
    """Each image of the batch sensed alone by abcs_sense: the same counts and
    bit-identical measurements (the batch runs the same FP32 tile code)."""
    imgs = [synth.gen_image(H, W, 950 + k) for k, (H, W, *_) in enumerate(MIXED)]
    buf, descs = _layout(imgs, MIXED, align=16)
    plans, counts, off, y, _ = _run(handle, buf, descs)
    b0 = 0
    for img, d, p in zip(imgs, descs, plans):
        H, W, B, v, r = d[:5]
        nB = p["n_blocks"]
        one = G.sense(handle, img[None], B, r, v)
        assert np.array_equal(one["counts"], counts[b0:b0 + nB])
        assert np.array_equal(one["y"], y[off[b0]:off[b0 + nB]])
        b0 += nB


def test_sense_batch_uneven_full_size(handle):
    """The uneven batch of the persistent-IDA configuration (256 images:
    40% 256x256, 40% 512x512, 20% 1024x1024; B cycling 8, 16, 32; BBV at
    subrate 0.2) in one call: BBV values and counts of every image bit-exact
    against the oracle's Eq. 19 and allocation, offsets the batch prefix,
    measurements of one image per (size, B) against the oracle."""
    items = synth.gen_uneven_batch(256, 5000)
    imgs = [im for im, _ in items]
    specs = [(im.shape[0], im.shape[1], B, O.BBV, 0.2, 0) for im, B in items]
    buf, descs = _layout(imgs, specs, align=16)
    plans, counts, off, y, pl = _run(handle, buf, descs)
    b0 = 0
    seen = {}
    for k, ((img, B), p) in enumerate(zip(items, plans)):
        nB = p["n_blocks"]
        ref_w = O.bbv(img.astype(np.int64), B, p["L"], p["X0"], p["nS"]).reshape(-1)
        assert np.array_equal(pl[b0:b0 + nB], ref_w), k
        assert np.array_equal(counts[b0:b0 + nB], O.allocate(ref_w, p["R"], p["cap"])), k
        seen.setdefault((img.shape, B), k)
        b0 += nB
    _check_against_oracle(imgs, descs, plans, counts, off, y, pl, sample=set(seen.values()))


def test_sense_batch_errors(handle):
    d = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    c = torch.zeros(1024, dtype=torch.int32, device="cuda")
    o = torch.zeros(1025, dtype=torch.int64, device="cuda")
    y = torch.zeros(1 << 16, dtype=torch.float32, device="cuda")
    ok = [(64, 64, 16, O.BBV, 0.3, 0, 64)]
    with pytest.raises(abcs.AbcsError) as e:                     # capacity below the images' M
        abcs.abcs_sense_batch(handle, d, ok, abcs.FP32, c, o, y, 10)
    assert e.value.status == 3
    with pytest.raises(abcs.AbcsError) as e:                     # BBV with L = 1
        abcs.abcs_sense_batch(handle, d, ok + [(64, 64, 16, O.BBV, 0.7, 4096, 64)], abcs.FP32, c, o, y, 1 << 16)
    assert e.value.status == 2 and "descriptor 1" in abcs.abcs_last_error()
    with pytest.raises(abcs.AbcsError) as e:                     # pitch below W
        abcs.abcs_sense_batch(handle, d, [(64, 64, 16, O.BBV, 0.3, 0, 32)], abcs.FP32, c, o, y, 1 << 16)
    assert e.value.status == 1
    with pytest.raises(abcs.AbcsError) as e:                     # tensor-core precision
        abcs.abcs_sense_batch(handle, d, ok, abcs.TC_FP16X2, c, o, y, 1 << 16)
    assert e.value.status == 2
    assert abcs.abcs_sync_status(handle) == 0
