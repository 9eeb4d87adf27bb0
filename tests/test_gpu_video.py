"""The streaming video pipeline (paper_2001_09632_gb300.video): copy, sense
and IDA of consecutive frame batches on three streams give exactly the
images of the same calls run one after another, and those of per-batch
abcs_sense / abcs_ida calls; a ragged last batch included.  With the
identity denoiser, every streamed frame is also compared with the FP64
oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2001_09632_gb300 import abcs, synth
from tests import gpu_util as G
from paper_2001_09632_gb300.video import VideoPipeline

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("den", [abcs.DEN_TIDCT, abcs.DEN_NONE])
def test_overlapped_equals_sequential(den):
    H, W, B, F, fpb = 96, 160, 16, 7, 3
    frames = torch.from_numpy(synth.gen_video(F, H, W, 5)).pin_memory()
    vp = VideoPipeline(H, W, B, 0.25, abcs.DD, fpb, 4, den)
    try:
        a = torch.full((F, vp.Hc, vp.Wc), float("nan"), device="cuda")
        b = torch.full_like(a, float("nan"))
        vp.run(frames, a, overlap=True)
        vp.run(frames, b, overlap=False)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        # per-batch calls on a fresh handle
        h = abcs.abcs_create()
        plan = abcs.abcs_plan(H, W, B, 0.25, abcs.DD)
        for f0 in range(0, F, fpb):
            n = min(fpb, F - f0)
            d = frames[f0:f0 + n].cuda()
            c = torch.empty(n * plan["n_blocks"], dtype=torch.int32, device="cuda")
            o = torch.empty(n * plan["n_blocks"] + 1, dtype=torch.int64, device="cuda")
            y = torch.empty(n * plan["M"], dtype=torch.float32, device="cuda")
            abcs.abcs_sense(h, d, n, H, W, W, H * W, B, 0.25, abcs.DD, abcs.FP32, c, o, y, n * plan["M"])
            x = torch.empty((n, vp.Hc, vp.Wc), device="cuda")
            abcs.abcs_ida(h, c, o, y, n, H, W, B, 4, 2.0, den, 2.3, None, x)
            assert abcs.abcs_sync_status(h) == 0
            assert torch.equal(x, a[f0:f0 + n])
        abcs.abcs_destroy(h)
        if den == abcs.DEN_NONE:
            # with the identity denoiser every streamed frame is linear in its
            # measurements: each against the FP64 oracle's sensing and IDA
            for f in range(F):
                ref = O.sense(frames[f].numpy(), B, 0.25, O.DD)
                xr, _ = O.ida(ref["y"], ref["counts"], vp.Hc, vp.Wc, B, 4, DF=2.0, denoiser=None)
                G.check_pixels(a[f].cpu().numpy(), xr, 1e-5, f)
    finally:
        vp.close()
