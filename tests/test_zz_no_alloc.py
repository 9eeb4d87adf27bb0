"""abcs_sense_noalloc: sensing for callers that cannot allocate device memory
while running (a fixed memory budget reserved at start-up, or a real-time
loop that cannot take cudaMalloc's implicit synchronisation).  Its results
must equal abcs_sense's, call after call, although its scratch is one
static device array shared by every call.

Collected last on purpose (file name), so a stop-at-first-failure run has
already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2001_09632_gb300 import abcs, synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _buffers(n, plan):
    nB = plan["n_blocks"]
    cap = n * plan["M"]
    return (torch.full((n * nB,), -1, dtype=torch.int32, device="cuda"),
            torch.full((n * nB + 1,), -1, dtype=torch.int64, device="cuda"),
            torch.full((cap,), float("nan"), dtype=torch.float32, device="cuda"),
            torch.full((n * nB,), -1, dtype=torch.int32, device="cuda"), cap)


def _run(fn, imgs, B, r, variant, use_pilot):
    n, H, W = imgs.shape
    plan = abcs.abcs_plan(H, W, B, r, variant)
    counts, offsets, coeffs, pilot, cap = _buffers(n, plan)
    d_img = torch.from_numpy(imgs).cuda()
    fn(d_img, counts, offsets, coeffs, cap, pilot if use_pilot else None)
    torch.cuda.synchronize()
    total = int(offsets[-1].item())
    return counts.cpu().numpy(), offsets.cpu().numpy(), coeffs[:total].cpu().numpy(), \
        (pilot.cpu().numpy() if use_pilot else None)


@pytest.mark.parametrize("variant,use_pilot", [(abcs.BBV, False), (abcs.DD, True)])
def test_noalloc_matches_sense_on_two_calls_in_a_row(variant, use_pilot):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B, r = 16, 0.3
    h = abcs.abcs_create()
    try:
        for call, (n, H, W, seed) in enumerate([(3, 96, 336, 7), (2, 128, 520, 11)]):
            imgs = np.stack([synth.gen_image(H, W, seed + k) for k in range(n)])

            def ref_fn(d_img, counts, offsets, coeffs, cap, pilot):
                abcs.abcs_sense(h, d_img, n, H, W, W, H * W, B, r, variant, abcs.FP32,
                                counts, offsets, coeffs, cap, pilot)

            def na_fn(d_img, counts, offsets, coeffs, cap, pilot):
                abcs.abcs_sense_noalloc(d_img, n, H, W, W, H * W, B, r, variant, abcs.FP32,
                                        counts, offsets, coeffs, cap, pilot)

            c0, o0, y0, p0 = _run(ref_fn, imgs, B, r, variant, use_pilot)
            c1, o1, y1, p1 = _run(na_fn, imgs, B, r, variant, use_pilot)
            assert np.array_equal(c1, c0), call
            assert np.array_equal(o1, o0), call
            if use_pilot:
                assert np.array_equal(p1, p0), call
            assert np.linalg.norm(y1 - y0) <= TOL * np.linalg.norm(y0), call
        assert abcs.abcs_sync_status(h) == 0
    finally:
        abcs.abcs_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(abcs.AbcsError) as e:        # 4097 images > 4096
        abcs.abcs_sense_noalloc(d, 4097, 16, 16, 16, 256, 16, 0.3, abcs.BBV, abcs.FP32,
                                d, d, d, 10 ** 9, None)
    assert e.value.status == 1
    with pytest.raises(abcs.AbcsError) as e:        # 4096 x 1024 blocks > 2^20 without a pilot buffer
        abcs.abcs_sense_noalloc(d, 4096, 512, 512, 512, 512 * 512, 16, 0.3, abcs.BBV, abcs.FP32,
                                d, d, d, 10 ** 12, None)
    assert e.value.status == 3
    assert "static scratch" in abcs.abcs_last_error()
