"""Helpers for the GPU tests: allocate device buffers with torch and call
the C ABI through the binding (argument marshalling only)."""
import numpy as np
import torch

from paper_2001_09632_gb300 import abcs


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def sense(h, imgs, B, r, variant, precision=abcs.FP32, pitch=None):
    """imgs: (n, H, W) uint8 numpy.  Returns numpy counts, offsets, y, pilot, status bits."""
    imgs = np.ascontiguousarray(imgs)
    n, H, W = imgs.shape
    plan = abcs.abcs_plan(H, W, B, r, variant)
    nB = plan["n_blocks"]
    if pitch is None:
        d_img = torch.from_numpy(imgs).cuda()
        pitch, stride = W, H * W
    else:
        buf = np.zeros((n, H, pitch), np.uint8)
        buf[:, :, :W] = imgs
        d_img = torch.from_numpy(buf).cuda()
        stride = H * pitch
    counts = torch.full((n * nB,), -7, dtype=torch.int32, device="cuda")
    offsets = torch.full((n * nB + 1,), -7, dtype=torch.int64, device="cuda")
    cap = n * plan["M"]
    coeffs = torch.full((max(cap, 1),), float("nan"), dtype=torch.float32, device="cuda")
    pilot = torch.full((n * nB,), -7, dtype=torch.int32, device="cuda")
    abcs.abcs_sense(h, d_img, n, H, W, pitch, stride, B, r, variant, precision,
                    counts, offsets, coeffs, cap, pilot)
    bits = abcs.abcs_sync_status(h)
    off = offsets.cpu().numpy()
    return dict(plan=plan, counts=counts.cpu().numpy(), offsets=off,
                y=coeffs[: int(off[-1])].cpu().numpy(), pilot=pilot.cpu().numpy(), bits=bits,
                d=(counts, offsets, coeffs))


def reconstruct(h, d_counts, d_offsets, d_coeffs, n, H, W, B, precision=abcs.FP32, u8=False):
    Hc, Wc = (H // B) * B, (W // B) * B
    out = torch.full((n, Hc, Wc), float("nan"), dtype=torch.float32, device="cuda")
    out8 = torch.zeros((n, Hc, Wc), dtype=torch.uint8, device="cuda") if u8 else None
    abcs.abcs_reconstruct(h, d_counts, d_offsets, d_coeffs, n, H, W, B, precision, out, out8)
    bits = abcs.abcs_sync_status(h)
    return out.cpu().numpy(), (out8.cpu().numpy() if u8 else None), bits


def ida(h, d_counts, d_offsets, d_coeffs, n, H, W, B, iters, DF, denoiser, lam=2.7):
    Hc, Wc = (H // B) * B, (W // B) * B
    x = torch.full((n, Hc, Wc), float("nan"), dtype=torch.float32, device="cuda")
    tr = torch.zeros((n, max(iters, 1)), dtype=torch.float32, device="cuda")
    abcs.abcs_ida(h, d_counts, d_offsets, d_coeffs, n, H, W, B, iters, DF, denoiser, lam, None, x, tr)
    bits = abcs.abcs_sync_status(h)
    return x.cpu().numpy(), tr.cpu().numpy(), bits
