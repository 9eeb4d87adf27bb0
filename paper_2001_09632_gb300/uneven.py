"""Uneven-size batches: images of different sizes and block sizes sensed on
the device and reconstructed by one abcs_ida_batch call (one persistent
launch under a captured CUDA graph).

Layout of the batch (all device arrays, built by `UnevenBatch`):
  counts / offsets  one entry per block, images in groups of equal
                    (H, W, B), each group followed by one spare entry (its
                    offsets total); `offsets` of a group count from the
                    group's first coefficient, `coeff_base` of its images
                    points there
  y                 the groups' packed measurement vectors, each group at a
                    capacity-sized slot
  x                 image k at pixel_offset k, Hc x Wc row-major
Sensing is one abcs_sense call per group (Alg. 1: pilot BBV, allocation
Eqs. 22-23, zigzag DCT coefficients); nothing here computes.
"""
from __future__ import annotations

from collections import OrderedDict

import numpy as np
import torch

from . import abcs


class UnevenBatch:
    def __init__(self, h, items, subrate, variant=abcs.BBV, device="cuda", stream=None):
        """items: list of (uint8 image (H, W), B) in batch order."""
        self.n = len(items)
        groups = OrderedDict()
        for k, (img, B) in enumerate(items):
            groups.setdefault((img.shape[0], img.shape[1], B), []).append(k)
        n_blocks = cap = 0
        plans = {}
        for key, ks in groups.items():
            H, W, B = key
            p = abcs.abcs_plan(H, W, B, subrate, variant)
            plans[key] = p
            n_blocks += len(ks) * p["n_blocks"]
            cap += len(ks) * p["M"]
        # one spare entry per group keeps each group's offsets[n_blocks] total intact
        self.counts = torch.zeros(n_blocks + len(groups), dtype=torch.int32, device=device)
        self.offsets = torch.empty(n_blocks + len(groups), dtype=torch.int64, device=device)
        self.y = torch.empty(max(cap, 1), dtype=torch.float32, device=device)
        self.y_len = cap
        desc = [None] * self.n
        self.shapes = [None] * self.n
        blk = coeff = 0
        self.measurements = 0
        self.groups = []          # (H, W, B, images, first block, first coefficient, capacity)
        self.members = []         # batch indices of each group's images
        for key, ks in groups.items():
            H, W, B = key
            p = plans[key]
            nB, gcap = p["n_blocks"], len(ks) * p["M"]
            imgs = torch.from_numpy(np.stack([items[k][0] for k in ks])).to(device)
            nb = len(ks) * nB
            abcs.abcs_sense(h, imgs, len(ks), H, W, W, H * W, B, subrate, variant, abcs.FP32,
                            self.counts[blk:blk + nb], self.offsets[blk:blk + nb + 1],
                            self.y[coeff:coeff + gcap], gcap, None, stream)
            self.measurements += int(self.offsets[blk + nb].item())
            for j, k in enumerate(ks):
                desc[k] = (H, W, B, blk + j * nB, coeff)
                self.shapes[k] = (p["nbh"] * B, p["nbw"] * B)
            self.groups.append((H, W, B, len(ks), blk, coeff, gcap))
            self.members.append(list(ks))
            blk += nb + 1
            coeff += gcap
        self.pixels = 0
        self.descs = []
        for k in range(self.n):
            H, W, B, bo, cb = desc[k]
            self.descs.append((H, W, B, bo, cb, self.pixels))
            self.pixels += self.shapes[k][0] * self.shapes[k][1]
        self.clean = [torch.from_numpy(np.ascontiguousarray(img[:hc, :wc])).to(device)
                      for (img, _), (hc, wc) in zip(items, self.shapes)]
        self.x = torch.empty(self.pixels, dtype=torch.float32, device=device)

    def ida(self, h, iters, denoiser=abcs.DEN_TIDCT, lam=2.3, damping=2.0, sigma_trace=None, stream=None):
        abcs.abcs_ida_batch(h, self.descs, self.counts, self.offsets, self.y, self.y_len, iters, damping,
                            denoiser, lam, self.x, sigma_trace, stream)
        return self.x

    def image(self, k):
        hc, wc = self.shapes[k]
        p0 = self.descs[k][5]
        return self.x[p0:p0 + hc * wc].view(hc, wc)

    def psnr(self):
        """Per image PSNR of the current x (clipped to [0, 255]) against the clean image."""
        out = []
        for k in range(self.n):
            d = self.image(k).clamp(0, 255) - self.clean[k].float()
            out.append(float(10.0 * torch.log10(255.0 ** 2 / (d * d).mean())))
        return out
