"""Uneven-size batches: images of different sizes and block sizes sensed on
the device by one abcs_sense_batch call and reconstructed by one
abcs_ida_batch call (one persistent launch under a captured CUDA graph).

Layout of the batch (all device arrays, built by `UnevenBatch`):
  pixels            every image row-major in one uint8 buffer, image k at
                    its own byte offset
  counts / offsets  one entry per block, images in batch order, offsets the
                    exclusive prefix over the whole batch (one extra entry:
                    the total)
  y                 the packed measurements of the whole batch
  x                 image k at pixel_offset k, Hc x Wc row-major
Sensing is Alg. 1 / Alg. 2 per image (pilot, allocation Eqs. 22-23, zigzag
DCT coefficients) in two launches for the batch; nothing here computes.
"""
from __future__ import annotations

import numpy as np
import torch

from . import abcs


class UnevenBatch:
    def __init__(self, h, items, subrate, variant=abcs.BBV, device="cuda", stream=None):
        """items: list of (uint8 image (H, W), B) in batch order."""
        self.n = len(items)
        descs, plans = [], []
        off = 0
        for img, B in items:
            H, W = img.shape
            descs.append((H, W, B, variant, subrate, off, W))
            plans.append(abcs.abcs_plan(H, W, B, subrate, variant))
            off += (H * W + 15) // 16 * 16
        buf = np.zeros(max(off, 16), np.uint8)
        for (img, _), d in zip(items, descs):
            buf[d[5]:d[5] + img.size] = img.reshape(-1)
        self.pixels_u8 = torch.from_numpy(buf).to(device)
        n_blocks = sum(p["n_blocks"] for p in plans)
        cap = sum(p["M"] for p in plans)
        self.counts = torch.zeros(n_blocks, dtype=torch.int32, device=device)
        self.offsets = torch.empty(n_blocks + 1, dtype=torch.int64, device=device)
        self.y = torch.empty(max(cap, 1), dtype=torch.float32, device=device)
        self.y_len = max(cap, 1)
        self.sense_descs = descs
        self.subrate, self.variant = subrate, variant
        self.sense(h, stream)
        self.measurements = int(self.offsets[n_blocks].item())
        self.shapes = [(p["nbh"] * B, p["nbw"] * B) for p, (_, B) in zip(plans, items)]
        self.block0 = np.concatenate([[0], np.cumsum([p["n_blocks"] for p in plans])])[:-1].tolist()
        self.pixels = 0
        self.descs = []
        for k, ((img, B), (hc, wc)) in enumerate(zip(items, self.shapes)):
            H, W = img.shape
            self.descs.append((H, W, B, self.block0[k], 0, self.pixels))
            self.pixels += hc * wc
        self.clean = [torch.from_numpy(np.ascontiguousarray(img[:hc, :wc])).to(device)
                      for (img, _), (hc, wc) in zip(items, self.shapes)]
        self.x = torch.empty(self.pixels, dtype=torch.float32, device=device)

    def sense(self, h, stream=None):
        """The whole batch's measurements: one abcs_sense_batch call."""
        abcs.abcs_sense_batch(h, self.pixels_u8, self.sense_descs, abcs.FP32, self.counts, self.offsets, self.y,
                              self.y_len, None, stream)

    def per_group_sensing(self, h, items, stream=None):
        """The same images sensed by one abcs_sense call per (H, W, B) group
        (for comparisons): list of (H, W, B, member indices, counts,
        offsets, y), the group's own arrays."""
        groups = {}
        for k, (img, B) in enumerate(items):
            groups.setdefault((img.shape[0], img.shape[1], B), []).append(k)
        out = []
        for (H, W, B), ks in groups.items():
            p = abcs.abcs_plan(H, W, B, self.subrate, self.variant)
            n, nB = len(ks), p["n_blocks"]
            imgs = torch.from_numpy(np.stack([items[k][0] for k in ks])).to(self.x.device)
            c = torch.empty(n * nB, dtype=torch.int32, device=self.x.device)
            o = torch.empty(n * nB + 1, dtype=torch.int64, device=self.x.device)
            y = torch.empty(max(n * p["M"], 1), dtype=torch.float32, device=self.x.device)
            abcs.abcs_sense(h, imgs, n, H, W, W, H * W, B, self.subrate, self.variant, abcs.FP32, c, o, y,
                            n * p["M"], None, stream)
            out.append((H, W, B, ks, c, o, y))
        return out

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
