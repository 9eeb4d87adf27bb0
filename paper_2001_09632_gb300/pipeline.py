"""Batches of images in host memory -> reconstructions in host memory, with
the transfers overlapped: the copy-in of batch j + 1, the sensing and
reconstruction of batch j (abcs_sense, abcs_reconstruct) and the copy-out of
batch j - 1 run on three streams, so in steady state a batch costs the
slowest of the three instead of their sum.

Every device buffer exists twice (batch j uses slot j % 2); each stage waits
on events for the stage before it and for the slot's previous user.  Each
copy may be split by images into `copy_chunks` pieces on as many streams, so
that several copy engines share the host link (on one GB300 the
copy-out of 64 x 512^2 FP32 runs at 183-185 GB/s with 1 or 2 pieces, near
the 192 GB/s of a plain device-to-host copy, and slower with 4 or 8).  With
`out_u8` the reconstructions are rounded to uint8 on the device (the
abcs_reconstruct out_u8 output), a quarter of the bytes to copy back.  The
results do not depend on
the overlap: the same kernels run on the same inputs as in a plain
sense -> reconstruct sequence.  Nothing here computes.
"""
from __future__ import annotations

import torch

from . import abcs


class SenseReconPipeline:
    def __init__(self, n_img, H, W, B, subrate, variant, precision=abcs.FP32, copy_chunks=1, out_u8=False):
        self.n, self.H, self.W, self.B = n_img, H, W, B
        self.subrate, self.variant, self.precision = subrate, variant, precision
        plan = abcs.abcs_plan(H, W, B, subrate, variant)
        self.nB, self.M = plan["n_blocks"], plan["M"]
        self.Hc, self.Wc = plan["nbh"] * B, plan["nbw"] * B
        self.h = abcs.abcs_create()
        n = n_img
        self.d_img = [torch.empty((n, H, W), dtype=torch.uint8, device="cuda") for _ in range(2)]
        self.counts = [torch.empty(n * self.nB, dtype=torch.int32, device="cuda") for _ in range(2)]
        self.offsets = [torch.empty(n * self.nB + 1, dtype=torch.int64, device="cuda") for _ in range(2)]
        self.y = [torch.empty(n * self.M, dtype=torch.float32, device="cuda") for _ in range(2)]
        self.out_u8 = out_u8
        self.rec = [torch.empty((n, self.Hc, self.Wc), dtype=torch.uint8 if out_u8 else torch.float32,
                                device="cuda") for _ in range(2)]
        self.chunks = max(1, min(copy_chunks, n_img))
        bounds = [n_img * c // self.chunks for c in range(self.chunks + 1)]
        self.parts = [(bounds[c], bounds[c + 1]) for c in range(self.chunks)]
        self.cin = [torch.cuda.Stream() for _ in range(self.chunks)]     # copy-in, one stream per piece
        self.comp = torch.cuda.Stream()
        self.cout = [torch.cuda.Stream() for _ in range(self.chunks)]    # copy-out

    def close(self):
        torch.cuda.synchronize()
        abcs.abcs_destroy(self.h)

    def run(self, inputs, outputs):
        """inputs[j]: pinned host uint8 (n, H, W); outputs[j]: pinned host
        float (n, Hc, Wc), or uint8 with out_u8; the same tensor may appear
        several times.  The
        copies and launches are queued after the work already on the current
        stream, which waits for the last copy-out.  Raises if the handle
        reports device status bits."""
        nb = len(inputs)
        cur = torch.cuda.current_stream()
        comp = self.comp
        ev = {k: [[torch.cuda.Event() for _ in self.parts] for _ in range(nb)] for k in ("in", "out")}
        ev["comp"] = [torch.cuda.Event() for _ in range(nb)]
        start = torch.cuda.Event()
        start.record(cur)
        for j in range(nb):
            sl = j % 2
            for c, (a, b) in enumerate(self.parts):
                s = self.cin[c]
                with torch.cuda.stream(s):
                    s.wait_event(start)
                    if j >= 2:
                        s.wait_event(ev["comp"][j - 2])      # the slot's images were read by batch j - 2
                    self.d_img[sl][a:b].copy_(inputs[j][a:b], non_blocking=True)
                    ev["in"][j][c].record(s)
            with torch.cuda.stream(comp):
                for c in range(self.chunks):
                    comp.wait_event(ev["in"][j][c])
                    if j >= 2:
                        comp.wait_event(ev["out"][j - 2][c])  # the slot's reconstruction was copied out
                abcs.abcs_sense(self.h, self.d_img[sl], self.n, self.H, self.W, self.W, self.H * self.W, self.B,
                                self.subrate, self.variant, self.precision, self.counts[sl], self.offsets[sl],
                                self.y[sl], self.n * self.M, None, comp)
                f32, u8 = (None, self.rec[sl]) if self.out_u8 else (self.rec[sl], None)
                abcs.abcs_reconstruct(self.h, self.counts[sl], self.offsets[sl], self.y[sl], self.n, self.H,
                                      self.W, self.B, self.precision, f32, u8, comp)
                ev["comp"][j].record(comp)
            for c, (a, b) in enumerate(self.parts):
                s = self.cout[c]
                with torch.cuda.stream(s):
                    s.wait_event(ev["comp"][j])
                    outputs[j][a:b].copy_(self.rec[sl][a:b], non_blocking=True)
                    ev["out"][j][c].record(s)
        for c in range(self.chunks):
            cur.wait_event(ev["out"][nb - 1][c])
        bits = abcs.abcs_sync_status(self.h, comp)
        if bits:
            raise RuntimeError(f"device status bits 0x{bits:x}")
        return outputs
