"""Fixed workloads for timing and profiling single kernels of the library
(each with its inputs seeded, run a few times, timed with CUDA events):

  python -m paper_2001_09632_gb300.profile_cases bm3d   # abcs_denoise_bm3d, 16 x 512x512, sigma 20
  python -m paper_2001_09632_gb300.profile_cases thi    # abcs_thi, 64 x 512x512, M = floor(0.3 N)
  python -m paper_2001_09632_gb300.profile_cases damp   # abcs_damp, 16 x 512x512, DD r 0.1, 3 iterations
  python -m paper_2001_09632_gb300.profile_cases recon  # abcs_reconstruct FP16x2, 64 x 512x512, BBV r 0.3
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import abcs, synth


def _timed(fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def bm3d(h):
    n, H, W = 16, 512, 512
    imgs = synth.gen_batch(n, H, W, 5).astype(np.float32)
    rng = np.random.default_rng(0)
    r = torch.tensor(imgs + rng.normal(0, 20, imgs.shape).astype(np.float32), device="cuda")
    out = torch.empty_like(r)
    sig = torch.full((n,), 20.0, device="cuda")
    run = lambda: abcs.abcs_denoise_bm3d(h, r, n, H, W, sig, 2.7, out)
    for _ in range(2):
        run()
    return {"case": "bm3d", "ms": _timed(run)}


def thi(h):
    n, H, W, B = 64, 512, 512, 16
    d = torch.from_numpy(synth.gen_batch(n, H, W, 4321)).cuda()
    plan = abcs.abcs_plan(H, W, B, 1.0, abcs.ZZ)
    nB = plan["n_blocks"]
    c = torch.empty(n * nB, dtype=torch.int32, device="cuda")
    o = torch.empty(n * nB + 1, dtype=torch.int64, device="cuda")
    y = torch.empty(n * plan["M"], dtype=torch.float32, device="cuda")
    abcs.abcs_sense(h, d, n, H, W, W, H * W, B, 1.0, abcs.ZZ, abcs.FP32, c, o, y, n * plan["M"])
    M = abcs.abcs_plan(H, W, B, 0.3, abcs.BBV)["M"]
    cnt = torch.empty(n * nB, dtype=torch.int32, device="cuda")
    run = lambda: abcs.abcs_thi(h, y, n, H, W, B, M, None, cnt, None, None)
    for _ in range(2):
        run()
    return {"case": "thi", "ms": _timed(run)}


def damp(h):
    n, H, W, B = 16, 512, 512, 16
    d = torch.from_numpy(synth.gen_batch(n, H, W, 8765)).cuda()
    plan = abcs.abcs_plan(H, W, B, 0.1, abcs.DD)
    nB = plan["n_blocks"]
    c = torch.empty(n * nB, dtype=torch.int32, device="cuda")
    o = torch.empty(n * nB + 1, dtype=torch.int64, device="cuda")
    y = torch.empty(n * plan["M"], dtype=torch.float32, device="cuda")
    abcs.abcs_sense(h, d, n, H, W, W, H * W, B, 0.1, abcs.DD, abcs.FP32, c, o, y, n * plan["M"])
    gen = torch.Generator(device="cuda").manual_seed(3)
    probe = torch.where(torch.rand((n, H, W), device="cuda", generator=gen) < 0.5, -1.0, 1.0)
    x = torch.empty((n, H, W), device="cuda")
    run = lambda: abcs.abcs_damp(h, c, o, y, n, H, W, B, 3, 2.0, abcs.DEN_TIDCT, 2.3, None, probe, x)
    run()
    return {"case": "damp", "ms": _timed(run)}


def recon(h):
    n, H, W, B, r = 64, 512, 512, 16, 0.3
    d = torch.from_numpy(synth.gen_batch(n, H, W, 1234)).cuda()
    plan = abcs.abcs_plan(H, W, B, r, abcs.BBV)
    nB = plan["n_blocks"]
    c = torch.empty(n * nB, dtype=torch.int32, device="cuda")
    o = torch.empty(n * nB + 1, dtype=torch.int64, device="cuda")
    y = torch.empty(n * plan["M"], dtype=torch.float32, device="cuda")
    abcs.abcs_sense(h, d, n, H, W, W, H * W, B, r, abcs.BBV, abcs.TC_FP16X2, c, o, y, n * plan["M"])
    x = torch.empty((n, H, W), device="cuda")
    run = lambda: abcs.abcs_reconstruct(h, c, o, y, n, H, W, B, abcs.TC_FP16X2, x)
    for _ in range(3):
        run()
    return {"case": "recon", "ms": _timed(run)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["bm3d", "thi", "damp", "recon"])
    a = ap.parse_args()
    h = abcs.abcs_create()
    res = {"bm3d": bm3d, "thi": thi, "damp": damp, "recon": recon}[a.case](h)
    res["status"] = abcs.abcs_sync_status(h)
    print(json.dumps(res))
    abcs.abcs_destroy(h)


if __name__ == "__main__":
    main()
