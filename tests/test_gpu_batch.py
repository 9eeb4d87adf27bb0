"""Uneven batch IDA (images of different sizes and block sizes) in one
persistent launch: identical to per-image abcs_ida (same tile arithmetic,
same fixed-order reductions), graph replay stable, bounded barrier waits."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2001_09632_gb300 import abcs, synth
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

SHAPES = [(64, 96, 8), (96, 64, 16), (128, 128, 32), (48, 80, 4), (64, 64, 16), (100, 300, 16), (72, 40, 8)]


def _build(handle, shapes, r=0.3, seed=400):
    counts, offsets, ys, descs = [], [], [], []
    blk = coeff = pix = 0
    singles = []
    for k, (H, W, B) in enumerate(shapes):
        img = synth.gen_image(H, W, seed + k)
        got = G.sense(handle, img[None], B, r, O.BBV)
        singles.append((img, got))
        nB = len(got["counts"])
        counts.append(got["counts"])
        offsets.append(got["offsets"][:-1])        # image-relative offsets
        ys.append(got["y"])
        descs.append((H, W, B, blk, coeff, pix))
        blk += nB
        coeff += len(got["y"])
        pix += (H // B) * B * (W // B) * B
    d = lambda a, t: torch.tensor(np.concatenate(a), dtype=t, device="cuda")
    return singles, descs, d(counts, torch.int32), d(offsets, torch.int64), d(ys, torch.float32), pix


@pytest.mark.parametrize("denoiser", [abcs.DEN_NONE, abcs.DEN_TIDCT])
def test_batch_equals_single_image_ida(handle, denoiser):
    iters = 6
    singles, descs, c, o, y, npx = _build(handle, SHAPES)
    x = torch.full((npx,), float("nan"), dtype=torch.float32, device="cuda")
    tr = torch.zeros((len(SHAPES), iters), dtype=torch.float32, device="cuda")
    for _ in range(2):      # the second call replays the captured graph
        abcs.abcs_ida_batch(handle, descs, c, o, y, y.numel(), iters, 2.0, denoiser, 2.3, x, tr)
        assert abcs.abcs_sync_status(handle) == 0
        xb, tb = x.cpu().numpy(), tr.cpu().numpy()
        for k, ((H, W, B), (img, got)) in enumerate(zip(SHAPES, singles)):
            xs, ts, _ = G.ida(handle, *got["d"], 1, H, W, B, iters, 2.0, denoiser, 2.3)
            p0 = descs[k][5]
            n = xs[0].size
            assert np.array_equal(xb[p0:p0 + n].reshape(xs[0].shape), xs[0]), k
            assert np.array_equal(tb[k], ts[0]), k


def test_batch_tidct_matches_oracle_psnr(handle):
    shapes = [(128, 128, 8), (96, 160, 16), (128, 96, 32)]
    singles, descs, c, o, y, npx = _build(handle, shapes, seed=500)
    x = torch.empty((npx,), dtype=torch.float32, device="cuda")
    abcs.abcs_ida_batch(handle, descs, c, o, y, y.numel(), 8, 2.0, abcs.DEN_TIDCT, 2.3, x)
    assert abcs.abcs_sync_status(handle) == 0
    xb = x.cpu().numpy()
    for k, ((H, W, B), (img, _)) in enumerate(zip(shapes, singles)):
        out = O.sense(img, B, 0.3, O.BBV)
        xr, _ = O.ida(out["y"], out["counts"], H, W, B, 8, DF=2.0,
                      denoiser=lambda rr, s: O.tidct_denoise(rr, s, 2.3))
        p0 = descs[k][5]
        xg = xb[p0:p0 + xr.size].reshape(xr.shape)
        assert abs(O.psnr(xg, img) - O.psnr(xr, img)) <= 0.05


def test_batch_barrier_timeout_is_reported(handle):
    """A CTA that never arrives makes the others' bounded waits expire: the
    launch ends, ABCS_DEV_TIMEOUT is reported, the context stays usable."""
    singles, descs, c, o, y, npx = _build(handle, SHAPES[:3], seed=600)
    x = torch.empty((npx,), dtype=torch.float32, device="cuda")
    abcs.abcs_ida_batch(handle, descs, c, o, y, y.numel(), 2, 2.0, abcs.DEN_TIDCT, 2.3, x)   # tune first
    assert abcs.abcs_sync_status(handle) == 0
    os.environ["ABCS_FAULT_SKIP_ARRIVE"] = "0"
    try:
        abcs.abcs_ida_batch(handle, descs, c, o, y, y.numel(), 2, 2.0, abcs.DEN_TIDCT, 2.3, x)
        bits = abcs.abcs_sync_status(handle)
    finally:
        del os.environ["ABCS_FAULT_SKIP_ARRIVE"]
    assert bits & abcs.DEV_TIMEOUT
    abcs.abcs_ida_batch(handle, descs, c, o, y, y.numel(), 2, 2.0, abcs.DEN_TIDCT, 2.3, x)
    assert abcs.abcs_sync_status(handle) == 0


def test_uneven_batch_module_equals_per_group_ida(handle):
    """paper_2001_09632_gb300.uneven: the whole batch sensed by one
    abcs_sense_batch call and reconstructed by one abcs_ida_batch call gives
    the same counts, measurements and images as one abcs_sense and one
    abcs_ida call per (size, B) group."""
    from paper_2001_09632_gb300.uneven import UnevenBatch
    items = synth.gen_uneven_batch(10, 700, sizes=((64, 64), (96, 128), (128, 192)))
    ub = UnevenBatch(handle, items, 0.2)
    ub.ida(handle, 5, abcs.DEN_TIDCT, 2.3)
    assert abcs.abcs_sync_status(handle) == 0
    off = ub.offsets.cpu().numpy()
    for (H, W, B, ks, c, o, y) in ub.per_group_sensing(handle, items):
        ni, nB = len(ks), (H // B) * (W // B)
        cg, og = c.cpu().numpy(), o.cpu().numpy()
        for j, k in enumerate(ks):
            b0 = ub.block0[k]
            assert np.array_equal(ub.counts[b0:b0 + nB].cpu().numpy(), cg[j * nB:(j + 1) * nB]), k
            yb = ub.y[off[b0]:off[b0 + nB]].cpu().numpy()
            assert np.array_equal(yb, y[og[j * nB]:og[(j + 1) * nB]].cpu().numpy()), k
        xo = torch.empty((ni, (H // B) * B, (W // B) * B), dtype=torch.float32, device="cuda")
        abcs.abcs_ida(handle, c, o, y, ni, H, W, B, 5, 2.0, abcs.DEN_TIDCT, 2.3, None, xo, None)
        for j, k in enumerate(ks):
            assert torch.equal(ub.image(k), xo[j]), (H, W, B, k)
    assert min(ub.psnr()) > 15.0
