"""Failure detection without a GPU fault: errors made on the host (an
allocation refused through ABCS_FAULT_WS_LIMIT, a buffer that is too small,
a NaN written into an input) must come back as status codes or device
status bits, and the handle must stay usable.  Guard words after each
output buffer must be untouched by every call (no write past the end)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2001_09632_gb300 import abcs, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
GUARD = 12345.0


def test_workspace_allocation_failure_is_reported(handle, monkeypatch):
    h = abcs.abcs_create()                     # a fresh handle: empty workspace
    try:
        img = synth.gen_image(96, 128, 1)[None]
        got = G.sense(handle, img, 16, 0.3, O.BBV)
        x = torch.empty((1, 96, 128), dtype=torch.float32, device="cuda")
        monkeypatch.setenv("ABCS_FAULT_WS_LIMIT", "1024")
        with pytest.raises(abcs.AbcsError) as e:
            abcs.abcs_ida(h, *got["d"], 1, 96, 128, 16, 3, 2.0, abcs.DEN_TIDCT, 2.3, None, x)
        assert e.value.status == 4                                     # ABCS_ERR_OOM
        monkeypatch.delenv("ABCS_FAULT_WS_LIMIT")
        abcs.abcs_ida(h, *got["d"], 1, 96, 128, 16, 3, 2.0, abcs.DEN_TIDCT, 2.3, None, x)
        assert abcs.abcs_sync_status(h) == 0
        assert torch.isfinite(x).all()
    finally:
        abcs.abcs_destroy(h)


def test_too_small_coefficient_buffer(handle):
    img = torch.from_numpy(synth.gen_image(64, 64, 2)[None]).cuda()
    plan = abcs.abcs_plan(64, 64, 16, 0.3, abcs.BBV)
    c = torch.empty(16, dtype=torch.int32, device="cuda")
    o = torch.empty(17, dtype=torch.int64, device="cuda")
    y = torch.empty(plan["M"], dtype=torch.float32, device="cuda")
    with pytest.raises(abcs.AbcsError) as e:
        abcs.abcs_sense(handle, img, 1, 64, 64, 64, 64 * 64, 16, 0.3, abcs.BBV, abcs.FP32, c, o, y, plan["M"] - 1)
    assert e.value.status == 3                                         # ABCS_ERR_CAPACITY
    abcs.abcs_sense(handle, img, 1, 64, 64, 64, 64 * 64, 16, 0.3, abcs.BBV, abcs.FP32, c, o, y, plan["M"])
    assert abcs.abcs_sync_status(handle) == 0


def test_nan_in_the_measurements_is_flagged(handle):
    imgs = np.stack([synth.gen_image(64, 96, 3 + k) for k in range(2)])
    got = G.sense(handle, imgs, 16, 0.3, O.DD)
    y = got["d"][2]
    y[5] = float("nan")                                                # image 0 only
    x = torch.empty((2, 64, 96), dtype=torch.float32, device="cuda")
    tr = torch.zeros((2, 3), dtype=torch.float32, device="cuda")
    abcs.abcs_ida(handle, *got["d"], 2, 64, 96, 16, 3, 2.0, abcs.DEN_TIDCT, 2.3, None, x, tr)
    bits = abcs.abcs_sync_status(handle)
    assert bits & abcs.DEV_NONFINITE
    t = tr.cpu().numpy()
    assert not np.isfinite(t[0, 0]) and np.all(np.isfinite(t[1]))    # the other image is unaffected
    assert torch.isfinite(x[1]).all()
    # the handle keeps working
    good = G.sense(handle, imgs, 16, 0.3, O.DD)
    abcs.abcs_ida(handle, *good["d"], 2, 64, 96, 16, 3, 2.0, abcs.DEN_TIDCT, 2.3, None, x)
    assert abcs.abcs_sync_status(handle) == 0


def test_nan_coefficient_in_thi_is_flagged(handle):
    img = synth.gen_image(32, 32, 4)[None]
    full = G.sense(handle, img, 8, 1.0, O.ZZ)["d"][2][: 32 * 32].clone()
    full[100] = float("nan")
    cnt = torch.empty(16, dtype=torch.int32, device="cuda")
    abcs.abcs_thi(handle, full, 1, 32, 32, 8, 50, None, cnt, None, None)
    assert abcs.abcs_sync_status(handle) & abcs.DEV_NONFINITE


def _guarded(n, dtype, fill):
    t = torch.full((n + 64,), fill, dtype=dtype, device="cuda")
    t[n:] = GUARD
    return t


def test_outputs_leave_guard_words_untouched(handle):
    """Ragged sizes (a partial last tile, a cropped edge) through sense,
    reconstruct, IDA (plain, learned-free), THI and BM3D: the 64 elements
    after every output stay as written before the call."""
    n, H, W, B, r = 2, 100, 337, 16, 0.3
    imgs = np.stack([synth.gen_image(H, W, 20 + k) for k in range(n)])
    plan = abcs.abcs_plan(H, W, B, r, abcs.BBV)
    nB, M = plan["n_blocks"], plan["M"]
    Hc, Wc = plan["nbh"] * B, plan["nbw"] * B
    d_img = torch.from_numpy(imgs).cuda()
    c = _guarded(n * nB, torch.int32, -1)
    o = _guarded(n * nB + 1, torch.int64, -1)
    y = _guarded(n * M, torch.float32, float("nan"))
    pil = _guarded(n * nB, torch.int32, -1)
    for prec in (abcs.FP32, abcs.TC_FP16X2):
        abcs.abcs_sense(handle, d_img, n, H, W, W, H * W, B, r, abcs.BBV, prec, c, o, y, n * M, pil)
        rec = _guarded(n * Hc * Wc, torch.float32, float("nan"))
        abcs.abcs_reconstruct(handle, c, o, y, n, H, W, B, prec, rec)
        assert abcs.abcs_sync_status(handle) == 0
        for t in (c, o, y, pil, rec):
            assert torch.all(t[-64:] == GUARD)
    x = _guarded(n * Hc * Wc, torch.float32, float("nan"))
    tr = _guarded(n * 3, torch.float32, float("nan"))
    abcs.abcs_ida(handle, c, o, y, n, H, W, B, 3, 2.0, abcs.DEN_TIDCT, 2.3, None, x, tr)
    xb = _guarded(n * Hc * Wc, torch.float32, float("nan"))
    sig = torch.full((n,), 15.0, device="cuda")
    abcs.abcs_denoise_bm3d(handle, x, n, Hc, Wc, sig, 2.7, xb)
    full = G.sense(handle, imgs, B, 1.0, O.ZZ)["d"][2][: n * Hc * Wc]
    cnt = _guarded(n * nB, torch.int32, -1)
    rho = _guarded(n, torch.float64, float("nan"))
    mk = _guarded(n * Hc * Wc, torch.float32, float("nan"))
    abcs.abcs_thi(handle, full, n, H, W, B, M, c, cnt, rho, mk)
    assert abcs.abcs_sync_status(handle) == 0
    for t in (x, tr, xb, cnt, rho, mk):
        assert torch.all(t[-64:] == GUARD)
