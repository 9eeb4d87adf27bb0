"""SenseReconPipeline (copy-in, sense + reconstruct, copy-out of consecutive
batches overlapped on three streams): its host outputs equal the plain
per-batch sequence bit for bit (the same kernels on the same inputs), and
match the FP64 oracle within the FP32 bar."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2001_09632_gb300 import abcs, synth
from paper_2001_09632_gb300.pipeline import SenseReconPipeline
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [abcs.FP32, abcs.TC_FP16X2])
def test_pipeline_equals_sequence(handle, prec):
    n, H, W, B, r = 3, 96, 144, 16, 0.3
    nb = 5
    batches = [np.stack([synth.gen_image(H, W, 40 * j + k) for k in range(n)]) for j in range(nb)]
    pipe = SenseReconPipeline(n, H, W, B, r, O.BBV, prec)
    try:
        h_in = [torch.from_numpy(b).pin_memory() for b in batches]
        h_out = [torch.full((n, H, W), float("nan")).pin_memory() for _ in range(nb)]
        pipe.run(h_in, h_out)
        torch.cuda.synchronize()
    finally:
        pipe.close()
    for j in range(nb):
        got = G.sense(handle, batches[j], B, r, O.BBV, precision=prec)
        rec, _, bits = G.reconstruct(handle, *got["d"], n, H, W, B, precision=prec)
        assert bits == 0
        assert np.array_equal(h_out[j].numpy(), rec), j
        for k in range(n):
            out = O.sense(batches[j][k], B, r, O.BBV)
            ref = O.reconstruct(out["counts"], out["y"], H, W, B)
            assert G.rel_l2(rec[k], ref) <= 1e-5


def test_pipeline_reuses_host_buffers(handle):
    """Two host output buffers alternating over six batches: each holds the
    last batch written to it."""
    n, H, W, B, r = 2, 64, 64, 16, 0.3
    batches = [np.stack([synth.gen_image(H, W, 7 * j + k) for k in range(n)]) for j in range(6)]
    pipe = SenseReconPipeline(n, H, W, B, r, O.DD, abcs.FP32)
    try:
        h_in = [torch.from_numpy(b).pin_memory() for b in batches]
        h_out = [torch.empty((n, H, W)).pin_memory() for _ in range(2)]
        pipe.run(h_in, [h_out[j % 2] for j in range(6)])
        torch.cuda.synchronize()
    finally:
        pipe.close()
    for j, slot in ((4, 0), (5, 1)):
        got = G.sense(handle, batches[j], B, r, O.DD)
        rec, _, _ = G.reconstruct(handle, *got["d"], n, H, W, B)
        assert np.array_equal(h_out[slot].numpy(), rec)


def test_pipeline_uint8_output(handle):
    """out_u8: the pipeline copies back the rounded uint8 reconstruction,
    equal to abcs_reconstruct's out_u8 of the same batch."""
    n, H, W, B, r = 3, 80, 112, 16, 0.3
    batches = [np.stack([synth.gen_image(H, W, 11 * j + k) for k in range(n)]) for j in range(3)]
    pipe = SenseReconPipeline(n, H, W, B, r, O.BBV, abcs.TC_FP16X2, out_u8=True)
    try:
        h_in = [torch.from_numpy(b).pin_memory() for b in batches]
        h_out = [torch.zeros((n, H, W), dtype=torch.uint8).pin_memory() for _ in range(3)]
        pipe.run(h_in, h_out)
        torch.cuda.synchronize()
    finally:
        pipe.close()
    for j in range(3):
        got = G.sense(handle, batches[j], B, r, O.BBV, precision=abcs.TC_FP16X2)
        _, rec8, bits = G.reconstruct(handle, *got["d"], n, H, W, B, precision=abcs.TC_FP16X2, u8=True)
        assert bits == 0
        assert np.array_equal(h_out[j].numpy(), rec8)
