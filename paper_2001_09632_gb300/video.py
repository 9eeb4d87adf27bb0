"""Streaming intra-frame video: frames arrive in host memory in batches; each
batch is copied to the device, sensed (abcs_sense) and reconstructed with
IDA (abcs_ida), every frame on its own.  With `overlap`, the three stages of
consecutive batches run on three streams, so batch j + 1 is copied and
sensed while batch j is reconstructed.

Each stage owns its buffers twice (batch j uses slot j % 2) and waits on
events for the stage before it and for the slot's previous user.  Sensing
and IDA run on two library handles, since a handle's workspace serves one
call at a time.  The results do not depend on `overlap`: the same kernels
run on the same inputs.  Nothing here computes.
"""
from __future__ import annotations

import torch

from . import abcs


class VideoPipeline:
    def __init__(self, H, W, B, subrate, variant, frames_per_batch, iters, denoiser=abcs.DEN_TIDCT,
                 lam=2.3, damping=2.0, cnn_packed=None):
        self.H, self.W, self.B, self.subrate, self.variant = H, W, B, subrate, variant
        self.fpb, self.iters, self.denoiser, self.lam, self.damping = frames_per_batch, iters, denoiser, lam, damping
        self.packed = cnn_packed
        plan = abcs.abcs_plan(H, W, B, subrate, variant)
        self.nB, self.M = plan["n_blocks"], plan["M"]
        self.Hc, self.Wc = plan["nbh"] * B, plan["nbw"] * B
        self.h_sense = abcs.abcs_create()
        self.h_ida = abcs.abcs_create()
        n = frames_per_batch
        self.d_img = [torch.empty((n, H, W), dtype=torch.uint8, device="cuda") for _ in range(2)]
        self.counts = [torch.empty(n * self.nB, dtype=torch.int32, device="cuda") for _ in range(2)]
        self.offsets = [torch.empty(n * self.nB + 1, dtype=torch.int64, device="cuda") for _ in range(2)]
        self.y = [torch.empty(n * self.M, dtype=torch.float32, device="cuda") for _ in range(2)]
        self.streams = [torch.cuda.Stream() for _ in range(3)]          # copy, sense, ida

    def close(self):
        torch.cuda.synchronize()
        abcs.abcs_destroy(self.h_sense)
        abcs.abcs_destroy(self.h_ida)

    def run(self, frames, out, overlap=True):
        """frames: pinned host uint8 (F, H, W); out: device float (F, Hc, Wc).
        Returns out; raises if either handle reports device status bits."""
        F = frames.shape[0]
        nb = (F + self.fpb - 1) // self.fpb
        cs, ss, ids = self.streams if overlap else [torch.cuda.current_stream()] * 3
        ev = {k: [torch.cuda.Event() for _ in range(nb)] for k in ("copy", "sense", "ida")}
        for j in range(nb):
            f0, f1 = j * self.fpb, min(F, (j + 1) * self.fpb)
            n, sl = f1 - f0, j % 2
            # copy: the slot's frames were read by sense of batch j - 2
            with torch.cuda.stream(cs):
                if j >= 2:
                    cs.wait_event(ev["sense"][j - 2])
                self.d_img[sl][:n].copy_(frames[f0:f1], non_blocking=True)
                ev["copy"][j].record(cs)
            # sense: counts / offsets / y of the slot were read by ida of batch j - 2
            with torch.cuda.stream(ss):
                ss.wait_event(ev["copy"][j])
                if j >= 2:
                    ss.wait_event(ev["ida"][j - 2])
                abcs.abcs_sense(self.h_sense, self.d_img[sl], n, self.H, self.W, self.W, self.H * self.W, self.B,
                                self.subrate, self.variant, abcs.FP32, self.counts[sl],
                                self.offsets[sl][:n * self.nB + 1], self.y[sl], n * self.M, None, ss)
                ev["sense"][j].record(ss)
            with torch.cuda.stream(ids):
                ids.wait_event(ev["sense"][j])
                abcs.abcs_ida(self.h_ida, self.counts[sl], self.offsets[sl], self.y[sl], n, self.H, self.W,
                              self.B, self.iters, self.damping, self.denoiser, self.lam, self.packed, out[f0:f1],
                              None, ids)
                ev["ida"][j].record(ids)
        torch.cuda.current_stream().wait_event(ev["ida"][nb - 1])
        bits = 0
        for h, s in ((self.h_sense, ss), (self.h_ida, ids)):
            bits |= abcs.abcs_sync_status(h, s)
        if bits:
            raise RuntimeError(f"device status bits 0x{bits:x}")
        return out
