"""abcs_sense_noalloc: sensing for callers that cannot allocate device memory
while running (a fixed memory budget reserved at start-up, or a real-time
loop that cannot take cudaMalloc's implicit synchronisation).  Its results
must equal abcs_sense's, call after call, although its scratch is one
static device array shared by every call, and it must allocate nothing.

Collected last on purpose (file name), so a stop-at-first-failure run has
already run every other test.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2001_09632_gb300 import abcs, synth

pytestmark = pytest.mark.gpu
TOL = 1e-5
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def _compare(h, imgs, B, r, variant, use_pilot, tag):
    n, H, W = imgs.shape

    def ref_fn(d_img, counts, offsets, coeffs, cap, pilot):
        abcs.abcs_sense(h, d_img, n, H, W, W, H * W, B, r, variant, abcs.FP32,
                        counts, offsets, coeffs, cap, pilot)

    def na_fn(d_img, counts, offsets, coeffs, cap, pilot):
        abcs.abcs_sense_noalloc(d_img, n, H, W, W, H * W, B, r, variant, abcs.FP32,
                                counts, offsets, coeffs, cap, pilot)

    c1, o1, y1, p1 = _run(na_fn, imgs, B, r, variant, use_pilot)
    c0, o0, y0, p0 = _run(ref_fn, imgs, B, r, variant, use_pilot)
    assert np.array_equal(c1, c0), tag
    assert np.array_equal(o1, o0), tag
    if use_pilot:
        assert np.array_equal(p1, p0), tag
    assert np.linalg.norm(y1 - y0) <= TOL * np.linalg.norm(y0), tag
    assert np.max(np.abs(y1 - y0)) <= 1e-4 * max(1.0, float(np.max(np.abs(y0)))), tag


# (variant, B, subrate, pilot buffer): BBV and DD through their pilots, the
# L-DCT-ZZ allocation, and BBV with n_S = floor(B / L) = 0 (B = 4, L = 5),
# which falls back to L-DCT-ZZ counts and clears a given pilot buffer
CASES = [(abcs.BBV, 16, 0.3, False), (abcs.DD, 16, 0.3, True), (abcs.ZZ, 8, 0.25, True),
         (abcs.BBV, 4, 0.2, True)]


@pytest.mark.parametrize("variant,B,r,use_pilot", CASES)
def test_noalloc_matches_sense_on_two_calls_in_a_row(variant, B, r, use_pilot):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = abcs.abcs_create()
    try:
        for call, (n, H, W, seed) in enumerate([(3, 96, 336, 7), (2, 128, 520, 11)]):
            imgs = np.stack([synth.gen_image(H, W, seed + k) for k in range(n)])
            _compare(h, imgs, B, r, variant, use_pilot, (variant, B, call))
        assert abcs.abcs_sync_status(h) == 0
        assert abcs.abcs_sense_noalloc_status() == 0
    finally:
        abcs.abcs_destroy(h)


_FRESH = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2001_09632_gb300 import abcs, synth
out = {}
# the first call of the process, before any handle exists: the set-up of
# the allocation-free path (its own table uploads) is all that has run
for variant, B, r, use_pilot in [(1, 16, 0.3, False), (2, 16, 0.3, True), (0, 8, 0.25, True), (1, 4, 0.2, True)]:
    n, H, W = 2, 112, 208
    imgs = np.stack([synth.gen_image(H, W, 31 + k) for k in range(n)])
    plan = abcs.abcs_plan(H, W, B, r, variant)
    nB, cap = plan["n_blocks"], n * plan["M"]
    d = torch.from_numpy(imgs).cuda()
    res = []
    frees = []
    bufs = [(torch.empty(n * nB, dtype=torch.int32, device="cuda"),
             torch.empty(n * nB + 1, dtype=torch.int64, device="cuda"),
             torch.empty(cap, dtype=torch.float32, device="cuda"),
             torch.empty(n * nB, dtype=torch.int32, device="cuda")) for _ in range(3)]
    torch.cuda.synchronize()
    for c, o, y, p in bufs:
        frees.append(torch.cuda.mem_get_info()[0])
        abcs.abcs_sense_noalloc(d, n, H, W, W, H * W, B, r, variant, abcs.FP32, c, o, y, cap,
                                p if use_pilot else None)
        torch.cuda.synchronize()
    frees.append(torch.cuda.mem_get_info()[0])
    res = [(c.cpu().numpy(), o.cpu().numpy(), y[:int(o[-1])].cpu().numpy()) for c, o, y, p in bufs]
    bits = abcs.abcs_sense_noalloc_status()
    # the handle path afterwards, on the same images
    h = abcs.abcs_create()
    c, o, y, p = (torch.empty_like(t) for t in bufs[0])
    abcs.abcs_sense(h, d, n, H, W, W, H * W, B, r, variant, abcs.FP32, c, o, y, cap, p if use_pilot else None)
    torch.cuda.synchronize()
    ref = (c.cpu().numpy(), o.cpu().numpy(), y[:int(o[-1])].cpu().numpy())
    abcs.abcs_destroy(h)
    ok = all(np.array_equal(a[0], ref[0]) and np.array_equal(a[1], ref[1]) and
             np.linalg.norm(a[2] - ref[2]) <= 1e-5 * np.linalg.norm(ref[2]) for a in res)
    out[f"{variant}-{B}"] = {"ok": bool(ok), "frees": frees, "bits": bits}
print(json.dumps(out))
"""


def test_noalloc_first_call_in_a_fresh_process_allocates_nothing():
    """The allocation-free path set up by its own first call (no handle in
    the process yet), compared with abcs_sense afterwards; the device's free
    memory does not change across the calls that follow the first."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    for key, v in out.items():
        assert v["ok"], key
        assert v["bits"] == 0, key
        # frees[1] is after the first call (set-up); the later calls leave it unchanged
        assert v["frees"][1] == v["frees"][2] == v["frees"][3], (key, v["frees"])


def test_noalloc_status_bits_are_reported_and_cleared():
    """Device status bits of the allocation-free calls collect in the static
    array's status word until abcs_sense_noalloc_status reads and clears
    them (the host-side hook stands in for a device condition)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n, H, W, B, r = 1, 64, 64, 16, 0.3
    img = torch.from_numpy(synth.gen_image(H, W, 3)[None]).cuda()
    plan = abcs.abcs_plan(H, W, B, r, abcs.DD)
    c, o, y, p, cap = _buffers(n, plan)
    args = (img, n, H, W, W, H * W, B, r, abcs.DD, abcs.FP32, c, o, y, cap, p)
    abcs.abcs_sense_noalloc(*args)
    assert abcs.abcs_sense_noalloc_status() == 0
    os.environ["ABCS_FAULT_NOALLOC_BITS"] = str(abcs.DEV_AMBIGUOUS)
    try:
        abcs.abcs_sense_noalloc(*args)
    finally:
        del os.environ["ABCS_FAULT_NOALLOC_BITS"]
    abcs.abcs_sense_noalloc(*args)                  # a clean call keeps the earlier bit
    assert abcs.abcs_sense_noalloc_status() == abcs.DEV_AMBIGUOUS
    assert abcs.abcs_sense_noalloc_status() == 0    # read and cleared


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
    with pytest.raises(abcs.AbcsError) as e:        # 4096 x 2^20 blocks >= 2^31, even with a pilot buffer
        abcs.abcs_sense_noalloc(d, 4096, 16384, 16384, 16384, 16384 * 16384, 16, 0.3, abcs.BBV, abcs.FP32,
                                d, d, d, 10 ** 15, d)
    assert e.value.status == 1
    with pytest.raises(abcs.AbcsError) as e:        # tensor-core precision: not built here
        abcs.abcs_sense_noalloc(d, 1, 16, 16, 16, 256, 16, 0.3, abcs.BBV, abcs.TC_FP16X2,
                                d, d, d, 10 ** 9, None)
    assert e.value.status == 2
    with pytest.raises(abcs.AbcsError) as e:        # not a precision at all
        abcs.abcs_sense_noalloc(d, 1, 16, 16, 16, 256, 16, 0.3, abcs.BBV, 7,
                                d, d, d, 10 ** 9, None)
    assert e.value.status == 1
