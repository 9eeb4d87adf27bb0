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


def block_scale(y_ref, counts, offsets):
    """Per coefficient: max(1, the largest |coefficient| of its block in y_ref)
    (the block's DC for every block with m_i >= 1).  A coefficient's FP32
    error is bounded relative to its block's energy, not to its own size."""
    y_ref = np.abs(np.asarray(y_ref, dtype=np.float64))
    counts = np.asarray(counts, dtype=np.int64)
    starts = np.asarray(offsets, dtype=np.int64)[:-1] - int(offsets[0])
    scale = np.ones(len(y_ref))
    nz = counts > 0
    if len(y_ref):
        mx = np.maximum.reduceat(y_ref, starts[nz]) if nz.any() else np.zeros(0)
        scale = np.repeat(np.maximum(1.0, mx), counts[nz])
    return scale


def check_coeffs(y, y_ref, counts, offsets, tol, tag=""):
    """Packed measurements against the oracle's: relative L2 over all of them
    <= tol, and every single coefficient within 10 tol of its block's scale
    (a coefficient off by 1, or one block off by a few units, fails)."""
    y = np.asarray(y, dtype=np.float64)
    y_ref = np.asarray(y_ref, dtype=np.float64)
    assert y.shape == y_ref.shape, (tag, y.shape, y_ref.shape)
    e = rel_l2(y, y_ref)
    assert e <= tol, (tag, "relL2", e)
    if len(y):
        worst = float(np.max(np.abs(y - y_ref) / block_scale(y_ref, counts, offsets)))
        assert worst <= 10 * tol, (tag, "max per-coefficient error / block scale", worst)
    return e


def check_pixels(x, x_ref, tol, tag="", scale=255.0):
    """Pixels against the oracle's: relative L2 <= tol and every pixel within
    10 tol of the pixel range (one pixel off by 1 fails)."""
    x = np.asarray(x, dtype=np.float64)
    x_ref = np.asarray(x_ref, dtype=np.float64)
    e = rel_l2(x, x_ref)
    assert e <= tol, (tag, "relL2", e)
    worst = float(np.max(np.abs(x - x_ref))) / scale
    assert worst <= 10 * tol, (tag, "max per-pixel error / range", worst)
    return e


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
