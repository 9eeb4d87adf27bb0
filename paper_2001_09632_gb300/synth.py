"""Seeded synthetic inputs for the ABCS hot path.

The paper evaluates on its Set256 / Set512 greyscale photographs (Sec. VII,
Figs. 4-5).  Those images are not distributed with this library, so every
test, the benchmark and the training driver use procedurally generated
stand-ins with the same shapes (256x256, 512x512, plus 1024x1024 and
1920x1088 frames), the same uint8 [0, 255] range and natural-image-like
structure: piecewise-constant shapes (edges, flat regions) over a 1/f^2
Gaussian random-field texture.

This module holds the input recipe only.  It computes none of the method's
arithmetic (no DCT, no allocation, no reconstruction), so both the CUDA path
and the FP64 oracle can consume its outputs without sharing any code.

Recipe (seed -> image), numpy PCG64:
  * background: one uniform integer grey level in [0, 255];
  * 12 shapes painted in order, each an ellipse or a rectangle with
    probability 1/2, centre uniform over the image, semi-axes uniform in
    [0.03, 0.3] * min(H, W), rotation uniform in [0, pi), grey level a
    uniform integer in [0, 255];
  * texture: white Gaussian noise shaped by 1/|f| in amplitude (power
    ~ 1/f^2, DC removed), scaled to standard deviation 20;
  * sum rounded half-to-even and clipped to [0, 255].
Video frames reuse the recipe with every shape moving `drift` pixels per
frame along its own random direction over a static texture.
"""
from __future__ import annotations

import numpy as np

N_SHAPES = 12
TEXTURE_STD = 20.0
_AXIS_RANGE = (0.03, 0.3)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _draw_shapes(rng: np.random.Generator, H: int, W: int, n_shapes: int):
    shapes = []
    lo, hi = _AXIS_RANGE
    s = min(H, W)
    for _ in range(n_shapes):
        kind = int(rng.integers(0, 2))          # 0 = ellipse, 1 = rectangle
        cy = float(rng.uniform(0.0, H))
        cx = float(rng.uniform(0.0, W))
        a = float(rng.uniform(lo, hi)) * s      # semi-axis along the rotated x
        b = float(rng.uniform(lo, hi)) * s      # semi-axis along the rotated y
        th = float(rng.uniform(0.0, np.pi))
        grey = int(rng.integers(0, 256))
        phi = float(rng.uniform(0.0, 2.0 * np.pi))  # drift direction (video)
        shapes.append((kind, cy, cx, a, b, th, grey, phi))
    return shapes


def _texture(rng: np.random.Generator, H: int, W: int, std: float) -> np.ndarray:
    noise = rng.standard_normal((H, W))
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    f = np.sqrt(fy * fy + fx * fx)
    amp = np.zeros_like(f)
    nz = f > 0
    amp[nz] = 1.0 / f[nz]                       # DC stays 0
    field = np.fft.ifft2(np.fft.fft2(noise) * amp).real
    sd = field.std()
    if sd > 0:
        field *= std / sd
    return field


def _render(H: int, W: int, bg: int, shapes, texture: np.ndarray, t: float, drift: float) -> np.ndarray:
    img = np.full((H, W), float(bg))
    for kind, cy, cx, a, b, th, grey, phi in shapes:
        cy = cy + t * drift * np.sin(phi)
        cx = cx + t * drift * np.cos(phi)
        r = max(a, b)
        y0, y1 = max(0, int(np.floor(cy - r)) - 1), min(H, int(np.ceil(cy + r)) + 2)
        x0, x1 = max(0, int(np.floor(cx - r)) - 1), min(W, int(np.ceil(cx + r)) + 2)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = np.arange(y0, y1, dtype=np.float64)[:, None] + 0.5 - cy
        xx = np.arange(x0, x1, dtype=np.float64)[None, :] + 0.5 - cx
        c, s = np.cos(th), np.sin(th)
        u = xx * c + yy * s
        v = -xx * s + yy * c
        if kind == 0:
            mask = (u / a) ** 2 + (v / b) ** 2 <= 1.0
        else:
            mask = (np.abs(u) <= a) & (np.abs(v) <= b)
        img[y0:y1, x0:x1][mask] = grey
    img += texture
    return np.clip(np.round(img), 0, 255).astype(np.uint8)


def gen_image(H: int, W: int, seed: int, n_shapes: int = N_SHAPES,
              texture_std: float = TEXTURE_STD) -> np.ndarray:
    """One H x W uint8 greyscale image, deterministic in `seed`."""
    rng = _rng(seed)
    bg = int(rng.integers(0, 256))
    shapes = _draw_shapes(rng, H, W, n_shapes)
    tex = _texture(rng, H, W, texture_std)
    return _render(H, W, bg, shapes, tex, 0.0, 0.0)


def gen_batch(n: int, H: int, W: int, base_seed: int) -> np.ndarray:
    """n images of one size; image k uses seed base_seed + k.  Shape (n, H, W)."""
    return np.stack([gen_image(H, W, base_seed + k) for k in range(n)])


def gen_video(n_frames: int, H: int, W: int, seed: int, drift: float = 2.0,
              first_frame: int = 0) -> np.ndarray:
    """Frames first_frame .. first_frame + n_frames - 1 of one synthetic clip.

    The texture is static; every shape moves `drift` pixels per frame along
    its own random direction.  Shape (n_frames, H, W), uint8.
    """
    rng = _rng(seed)
    bg = int(rng.integers(0, 256))
    shapes = _draw_shapes(rng, H, W, N_SHAPES)
    tex = _texture(rng, H, W, TEXTURE_STD)
    return np.stack([_render(H, W, bg, shapes, tex, float(first_frame + k), drift)
                     for k in range(n_frames)])


def gen_uneven_batch(n: int, base_seed: int, sizes=((256, 256), (512, 512), (1024, 1024)),
                     mix=(0.4, 0.4, 0.2), blocks=(8, 16, 32)):
    """A list of (image, B) pairs of mixed sizes and block sizes.

    Sizes follow `mix` exactly (rounded, remainder to the last size); the block
    size of image k cycles through `blocks`.  Image k uses seed base_seed + k.
    """
    counts = [int(round(n * p)) for p in mix[:-1]]
    counts.append(n - sum(counts))
    out = []
    k = 0
    for (H, W), c in zip(sizes, counts):
        for _ in range(c):
            out.append((gen_image(H, W, base_seed + k), blocks[k % len(blocks)]))
            k += 1
    return out


def gen_noise(shape, seed: int, std: float = 1.0) -> np.ndarray:
    """Seeded Gaussian noise (float64), e.g. for denoiser training pairs."""
    return _rng(seed).standard_normal(shape) * std
