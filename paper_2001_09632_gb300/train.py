"""Training and evaluation driver of the learned IDA denoiser.

Everything numeric runs in libabcs.so through the C ABI; this module only
moves tensors (torch is used for device memory, random crop indices and the
PSNR bookkeeping of the evaluation).

  python -m paper_2001_09632_gb300.train tune-lambda   # plain TI-DCT threshold factor
  python -m paper_2001_09632_gb300.train train --out weights.f32
  python -m paper_2001_09632_gb300.train eval --weights weights.f32
  python -m paper_2001_09632_gb300.train video --weights weights.f32  # 1920x1088 DD clip
  python -m paper_2001_09632_gb300.train time --iters 2               # learned IDA throughput

Training pairs follow the method itself: synthetic images are sensed
(AL-DCT-BBV or AL-DCT-DD, subrate drawn from {0.1, ..., 0.5}), plain IDA
runs on them, and the denoiser input r^t of iteration t (with its sigma^t)
is captured for several t; random 64x64 crops of (r^t, clean image) form the
training set.  Seeds of training, tuning and evaluation images are disjoint.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import abcs, synth

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "cnn_ida_b16.f32")
DEFAULT_LAMBDA = 2.3   # tuned: tune_lambda() over 2.0..3.5 on held-out synthetic images
TRAIN_SEED, TUNE_SEED, EVAL_SEED = 10_000_000, 20_000_000, 30_000_000


def iter_input(t: int) -> float:
    """The learned denoiser's iteration input in IDA iteration t, as abcs_ida
    passes it: min(t, 8) / 8."""
    return min(int(t), 8) / 8.0


def load_weights(path: str = WEIGHTS) -> np.ndarray:
    w = np.fromfile(path, dtype="<f4")
    if w.size != abcs.abcs_cnn_param_count():
        raise ValueError(f"{path}: {w.size} values, expected {abcs.abcs_cnn_param_count()}")
    return w


def init_params(seed: int) -> np.ndarray:
    """He-normal weights (last layer x 0.1), zero biases, in the ABI's layout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    chans = [4] + [32] * 7 + [1]
    out = []
    for l in range(8):
        ci, co = chans[l], chans[l + 1]
        w = rng.standard_normal((co, ci, 3, 3)) * math.sqrt(2.0 / (9 * ci))
        if l == 7:
            w *= 0.1
        out += [w.reshape(-1), np.zeros(co)]
    return np.concatenate(out).astype(np.float32)


class Sensed:
    """One batch of equally sized images sensed on the device."""

    def __init__(self, h, imgs: np.ndarray, B: int, subrate: float, variant: int):
        n, H, W = imgs.shape
        plan = abcs.abcs_plan(H, W, B, subrate, variant)
        nB = plan["n_blocks"]
        self.n, self.H, self.W, self.B = n, H, W, B
        self.Hc, self.Wc = plan["nbh"] * B, plan["nbw"] * B
        self.d_img = torch.from_numpy(imgs).cuda()
        self.clean = self.d_img[:, : self.Hc, : self.Wc].float()
        self.counts = torch.empty(n * nB, dtype=torch.int32, device="cuda")
        self.offsets = torch.empty(n * nB + 1, dtype=torch.int64, device="cuda")
        cap = n * plan["M"]
        self.y = torch.empty(cap, dtype=torch.float32, device="cuda")
        abcs.abcs_sense(h, self.d_img, n, H, W, W, H * W, B, subrate, variant, abcs.FP32,
                        self.counts, self.offsets, self.y, cap)
        # the learned denoiser's third input: measured fraction of each pixel's block
        self.density = torch.empty((n, self.Hc, self.Wc), dtype=torch.float32, device="cuda")
        abcs.abcs_density_map(h, self.counts, n, H, W, B, self.density)

    def ida(self, h, iters, denoiser, lam=DEFAULT_LAMBDA, packed=None, x=None):
        x = torch.empty((self.n, self.Hc, self.Wc), dtype=torch.float32, device="cuda") if x is None else x
        abcs.abcs_ida(h, self.counts, self.offsets, self.y, self.n, self.H, self.W, self.B, iters, 2.0,
                      denoiser, lam, packed, x)
        return x

    def capture(self, h, t, lam=DEFAULT_LAMBDA, packed=None):
        r = torch.empty((self.n, self.Hc, self.Wc), dtype=torch.float32, device="cuda")
        s = torch.empty(self.n, dtype=torch.float32, device="cuda")
        den = abcs.DEN_TIDCT if packed is None else abcs.DEN_CNN
        abcs.abcs_ida_capture(h, self.counts, self.offsets, self.y, self.n, self.H, self.W, self.B, t, 2.0,
                              den, lam, packed, r, s)
        return r, s


def quality(h, x: torch.Tensor, sd: "Sensed"):
    """Per-image PSNR and SSIM of x against the batch's clean images, from
    the library (abcs_psnr_ssim): two float lists."""
    ps = torch.empty(sd.n, dtype=torch.float64, device="cuda")
    ss = torch.empty_like(ps)
    abcs.abcs_psnr_ssim(h, x, sd.d_img, sd.n, sd.Hc, sd.Wc, sd.W, sd.H * sd.W, ps, ss)
    return ps.tolist(), ss.tolist()


def psnr(x: torch.Tensor, ref: torch.Tensor) -> torch.Tensor:
    """Per image 10 log10(255^2 / MSE) of x clipped to [0, 255]."""
    d = x.clamp(0, 255) - ref
    mse = (d * d).flatten(1).mean(1)
    return 10.0 * torch.log10(255.0 ** 2 / mse)


def make_pairs(h, n_images=512, H=512, W=512, captures=(0, 1, 2, 4, 8, 16, 29), crops=56, crop=64,
               batch=32, seed=TRAIN_SEED, lam=DEFAULT_LAMBDA, packed=None, large_every=0,
               large_size=(1024, 1024), log=print):
    """(r^t, clean, sigma^t, density, tau_t) crops; r^t from plain IDA, or
    from learned IDA when `packed` weights are given (its own trajectories);
    tau_t = min(t, 8) / 8 is the network's iteration input.  A capture index
    listed twice contributes twice the crops.  With large_every = n, every
    n-th batch uses 8 images of large_size instead."""
    subrates = (0.1, 0.2, 0.3, 0.4, 0.5)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    R, C, S, D, T = [], [], [], [], []
    t0 = time.time()
    for i0 in range(0, n_images, batch):
        j = i0 // batch
        if large_every and j % large_every == large_every - 1:
            imgs = synth.gen_batch(8, large_size[0], large_size[1], seed + i0)
        else:
            imgs = synth.gen_batch(min(batch, n_images - i0), H, W, seed + i0)
        variant = abcs.BBV if j % 2 == 0 else abcs.DD
        sd = Sensed(h, imgs, 16, subrates[j % len(subrates)], variant)
        for t in captures:
            r, s = sd.capture(h, t, lam, packed)
            n = r.shape[0]
            ys = torch.randint(0, sd.Hc - crop + 1, (n, crops), device="cuda", generator=gen)
            xs = torch.randint(0, sd.Wc - crop + 1, (n, crops), device="cuda", generator=gen)
            ar = torch.arange(crop, device="cuda")
            rows = (ys[..., None] + ar)[..., :, None]          # n, crops, crop, 1
            cols = (xs[..., None] + ar)[..., None, :]          # n, crops, 1, crop
            kk = torch.arange(n, device="cuda")[:, None, None, None]
            R.append(r[kk, rows, cols].reshape(-1, crop, crop))
            C.append(sd.clean[kk, rows, cols].reshape(-1, crop, crop))
            D.append(sd.density[kk, rows, cols].reshape(-1, crop, crop))
            S.append(s[:, None].expand(n, crops).reshape(-1))
            T.append(torch.full((n * crops,), iter_input(t), dtype=torch.float32, device="cuda"))
        if j % 8 == 0:
            log(f"pairs: {i0 + batch}/{n_images} images, {sum(x.shape[0] for x in R)} crops, {time.time() - t0:.1f}s")
    assert abcs.abcs_sync_status(h) == 0
    return torch.cat(R), torch.cat(C), torch.cat(S), torch.cat(D), torch.cat(T)


def save_checkpoint(path: str, state: dict) -> None:
    """Write `state` (numpy arrays and scalars) to path atomically: into
    path + '.tmp', flushed to disk, then renamed over path, so a process
    killed while writing leaves the previous checkpoint intact."""
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        np.savez(f, **state)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def load_checkpoint(path: str):
    """The state written by save_checkpoint, or None if there is none."""
    if not path or not os.path.exists(path):
        return None
    with np.load(path, allow_pickle=False) as z:
        return {k: z[k] for k in z.files}


def train(h, R, C, S, D, steps=4000, batch=128, lr=1e-3, seed=1, params=None, log=print, ckpt=None,
          ckpt_every=500, until=None, T=None):
    """Adam on the crops (R, C, S, D) with a cosine learning-rate decay over
    `steps`.  With `ckpt`, the FP32 parameters, Adam's moments, the step and
    the state of the crop sampler are saved every `ckpt_every` steps and
    where the run stops, and a run finding that file resumes after its
    step.  `until` stops after that step of the same schedule (a job cut
    into pieces)."""
    n, crop = R.shape[0], R.shape[1]
    p = torch.tensor(init_params(seed) if params is None else params, device="cuda")
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    packed = torch.empty(abcs.abcs_cnn_packed_bytes(), dtype=torch.uint8, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(seed)
    hist = []
    t0 = time.time()
    first = 1
    st = load_checkpoint(ckpt)
    if st is not None:
        p.copy_(torch.from_numpy(st["params"]))
        m.copy_(torch.from_numpy(st["m"]))
        v.copy_(torch.from_numpy(st["v"]))
        gen.set_state(torch.from_numpy(st["gen"]))
        first = int(st["step"]) + 1
        hist = [tuple(x) for x in st["hist"].tolist()]
        log(f"resumed after step {first - 1}")

    def save(step):
        save_checkpoint(ckpt, {"params": p.cpu().numpy(), "m": m.cpu().numpy(), "v": v.cpu().numpy(),
                               "gen": gen.get_state().numpy(), "step": np.int64(step),
                               "hist": np.asarray(hist, dtype=np.float64).reshape(-1, 2)})

    last = steps if until is None else min(until, steps)
    for step in range(first, last + 1):
        idx = torch.randint(0, n, (batch,), device="cuda", generator=gen)
        rb, cb, sb, db = R[idx].contiguous(), C[idx].contiguous(), S[idx].contiguous(), D[idx].contiguous()
        tb = T[idx].contiguous() if T is not None else None
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * (step - 1) / steps))     # cosine decay
        abcs.abcs_cnn_train_step(h, p, m, v, step, lr_t, packed, rb, cb, sb, db, batch, crop, crop, loss, tau=tb)
        if step % 200 == 0 or step == 1:
            l = loss.item()
            hist.append((step, l))
            log(f"step {step:5d}  loss {l:.6f}  (rmse {255 * math.sqrt(l):.2f})  {time.time() - t0:.1f}s")
        if ckpt and (step % ckpt_every == 0 or step == last):
            save(step)
    torch.cuda.synchronize()
    assert abcs.abcs_sync_status(h) == 0
    return p.cpu().numpy(), hist, time.time() - t0


def trajectory_psnr(h, weights, n=16, H=512, W=512, subrates=(0.1, 0.3), iters=(1, 2, 3, 4, 6),
                    seed=TUNE_SEED + 500, log=print):
    """Mean PSNR of learned IDA after each iteration count on n tuning images
    (disjoint from the training and evaluation seeds): the check that the
    network stays useful along its own trajectory."""
    p = torch.tensor(weights, device="cuda")
    packed = torch.empty(abcs.abcs_cnn_packed_bytes(), dtype=torch.uint8, device="cuda")
    abcs.abcs_cnn_pack(h, p, packed)
    imgs = synth.gen_batch(n, H, W, seed)
    out = {}
    for r in subrates:
        sd = Sensed(h, imgs, 16, r, abcs.BBV)
        out[str(r)] = {str(t): float(psnr(sd.ida(h, t, abcs.DEN_CNN, DEFAULT_LAMBDA, packed), sd.clean).mean())
                       for t in iters}
    log("trajectory psnr " + json.dumps(out))
    return out


def tune_lambda(h, n=16, H=512, W=512, iters=30, grid=None, log=print):
    grid = grid or [round(2.0 + 0.1 * i, 1) for i in range(16)]
    imgs = synth.gen_batch(n, H, W, TUNE_SEED)
    res = {}
    for r in (0.1, 0.3, 0.5):
        sd = Sensed(h, imgs, 16, r, abcs.BBV)
        for lam in grid:
            x = sd.ida(h, iters, abcs.DEN_TIDCT, lam)
            res.setdefault(lam, []).append(float(psnr(x, sd.clean).mean()))
    mean = {lam: float(np.mean(v)) for lam, v in res.items()}
    best = max(mean, key=mean.get)
    log(json.dumps({"lambda_psnr": mean, "best": best}))
    return best, mean


def timed_ida(h, sd: Sensed, iters, denoiser, lam, packed, reps=3):
    x = sd.ida(h, iters, denoiser, lam, packed)
    torch.cuda.synchronize()
    ev = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sd.ida(h, iters, denoiser, lam, packed, x)
        e1.record()
        ev.append((e0, e1))
    torch.cuda.synchronize()
    ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
    return x, ms


def evaluate(h, weights, n=128, H=512, W=512, subrates=(0.1, 0.2, 0.3, 0.4, 0.5), variant=abcs.BBV,
             plain_iters=(1, 3, 5, 10, 20, 30), learned_iters=(1, 2, 3, 4, 6, 10), lam=DEFAULT_LAMBDA,
             batch=32, seed=EVAL_SEED, log=print):
    """Plain IDA (TI-DCT) and learned IDA (CNN) on held-out images: mean PSNR
    and SSIM after each iteration count, and Mpixel/s of a full
    reconstruction with that many iterations.  `equal` compares the fewest
    learned iterations whose PSNR reaches the plain reference (its last
    iteration count) minus 0.1 dB with that reference."""
    p = torch.tensor(weights, device="cuda")
    packed = torch.empty(abcs.abcs_cnn_packed_bytes(), dtype=torch.uint8, device="cuda")
    abcs.abcs_cnn_pack(h, p, packed)
    out = {}
    for r in subrates:
        ps, ss = {("idct", 0): []}, {("idct", 0): []}
        ms = {}
        px = 0
        for i0 in range(0, n, batch):
            imgs = synth.gen_batch(min(batch, n - i0), H, W, seed + i0)
            sd = Sensed(h, imgs, 16, r, variant)
            x0 = sd.ida(h, 1, abcs.DEN_NONE)      # one identity iteration = A^T y, the IDCT image
            p_, s_ = quality(h, x0, sd)
            ps[("idct", 0)] += p_
            ss[("idct", 0)] += s_
            for kind, its, den, pk in (("plain", plain_iters, abcs.DEN_TIDCT, None),
                                       ("learned", learned_iters, abcs.DEN_CNN, packed)):
                for it in its:
                    x, t_ms = timed_ida(h, sd, it, den, lam, pk, reps=2)
                    p_, s_ = quality(h, x, sd)
                    ps.setdefault((kind, it), []).extend(p_)
                    ss.setdefault((kind, it), []).extend(s_)
                    ms[(kind, it)] = ms.get((kind, it), 0.0) + t_ms
            px += sd.n * sd.Hc * sd.Wc
        res = {"psnr_idct": float(np.mean(ps[("idct", 0)])), "ssim_idct": float(np.mean(ss[("idct", 0)]))}
        for kind, its in (("plain", plain_iters), ("learned", learned_iters)):
            res[kind] = {str(it): {"psnr": float(np.mean(ps[(kind, it)])), "ssim": float(np.mean(ss[(kind, it)])),
                                   "Mpx_per_s": px / (ms[(kind, it)] * 1e-3) / 1e6} for it in its}
        ref_it = str(plain_iters[-1])
        ref = res["plain"][ref_it]
        eq = None
        for it in learned_iters:
            e = res["learned"][str(it)]
            if e["psnr"] >= ref["psnr"] - 0.1:
                eq = {"learned_iters": it, "plain_iters": plain_iters[-1], "psnr_learned": e["psnr"],
                      "psnr_plain": ref["psnr"], "speedup": e["Mpx_per_s"] / ref["Mpx_per_s"]}
                break
        res["equal"] = eq
        out[str(r)] = res
        log(f"r={r}: idct {res['psnr_idct']:.2f}  plain " +
            " ".join(f"{k}:{v['psnr']:.2f}" for k, v in res["plain"].items()) + "  learned " +
            " ".join(f"{k}:{v['psnr']:.2f}" for k, v in res["learned"].items()) + f"  equal {eq}")
    assert abcs.abcs_sync_status(h) == 0
    return out


def video_eval(h, weights, n_frames=120, H=1088, W=1920, batch=30, subrate=0.25, variant=abcs.DD, B=16,
               plain_iters=(10, 20, 30), learned_iters=(1, 2, 3, 4, 6, 10), lam=DEFAULT_LAMBDA, seed=EVAL_SEED + 7,
               reps=2, log=print):
    """Intra-frame video: every frame of a synthetic clip (shapes drifting 2
    px/frame over a static texture) sensed on its own with AL-DCT-DD, batches
    of `batch` frames per call.  Mean PSNR and Mpixel/s of the IDCT image,
    plain IDA (TI-DCT) and learned IDA (CNN) after each iteration count; the
    headline pair is learned-10 vs plain-30, and `equal` names the fewest
    learned iterations within 0.1 dB of plain-30."""
    p = torch.tensor(weights, device="cuda")
    packed = torch.empty(abcs.abcs_cnn_packed_bytes(), dtype=torch.uint8, device="cuda")
    abcs.abcs_cnn_pack(h, p, packed)
    ps, ms = {}, {}
    px = 0
    sense_ms = 0.0
    for f0 in range(0, n_frames, batch):
        frames = synth.gen_video(min(batch, n_frames - f0), H, W, seed, first_frame=f0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sd = Sensed(h, frames, B, subrate, variant)
        e1.record()
        torch.cuda.synchronize()
        sense_ms += e0.elapsed_time(e1)
        x0 = sd.ida(h, 1, abcs.DEN_NONE)
        ps.setdefault(("idct", 0), []).extend(psnr(x0, sd.clean).tolist())
        for kind, its, den, pk in (("plain", plain_iters, abcs.DEN_TIDCT, None),
                                   ("learned", learned_iters, abcs.DEN_CNN, packed)):
            for it in its:
                x, t_ms = timed_ida(h, sd, it, den, lam, pk, reps=reps)
                ps.setdefault((kind, it), []).extend(psnr(x, sd.clean).tolist())
                ms[(kind, it)] = ms.get((kind, it), 0.0) + t_ms
        px += sd.n * sd.Hc * sd.Wc
        del sd, x, x0
    res = {"frames": n_frames, "size": [H, W], "B": B, "subrate": subrate,
           "variant": "DD" if variant == abcs.DD else "BBV", "frames_per_call": batch,
           "sense_Mpx_per_s": px / (sense_ms * 1e-3) / 1e6,
           "psnr_idct": float(np.mean(ps[("idct", 0)]))}
    for kind, its in (("plain", plain_iters), ("learned", learned_iters)):
        res[kind] = {str(it): {"psnr": float(np.mean(ps[(kind, it)])),
                               "Mpx_per_s": px / (ms[(kind, it)] * 1e-3) / 1e6} for it in its}
    ref = res["plain"][str(plain_iters[-1])]
    head = res["learned"][str(learned_iters[-1])]
    res["learned_vs_plain"] = {"learned_iters": learned_iters[-1], "plain_iters": plain_iters[-1],
                               "psnr_learned": head["psnr"], "psnr_plain": ref["psnr"],
                               "dpsnr": head["psnr"] - ref["psnr"],
                               "speedup": head["Mpx_per_s"] / ref["Mpx_per_s"]}
    res["equal"] = None
    for it in learned_iters:
        e = res["learned"][str(it)]
        if e["psnr"] >= ref["psnr"] - 0.1:
            res["equal"] = {"learned_iters": it, "plain_iters": plain_iters[-1], "psnr_learned": e["psnr"],
                            "psnr_plain": ref["psnr"], "speedup": e["Mpx_per_s"] / ref["Mpx_per_s"]}
            break
    log(f"video: idct {res['psnr_idct']:.2f}  plain " +
        " ".join(f"{k}:{v['psnr']:.2f}" for k, v in res["plain"].items()) + "  learned " +
        " ".join(f"{k}:{v['psnr']:.2f}" for k, v in res["learned"].items()) + f"  equal {res['equal']}")
    assert abcs.abcs_sync_status(h) == 0
    return res


def time_learned(h, weights, iters=2, n=16, H=512, W=512, subrate=0.3, seed=77, log=print):
    """Learned IDA on n seeded images: one warm-up call, one timed call.
    Returns Gpixel * iteration / s."""
    p = torch.tensor(weights, device="cuda")
    packed = torch.empty(abcs.abcs_cnn_packed_bytes(), dtype=torch.uint8, device="cuda")
    abcs.abcs_cnn_pack(h, p, packed)
    sd = Sensed(h, synth.gen_batch(n, H, W, seed), 16, subrate, abcs.BBV)
    x = sd.ida(h, iters, abcs.DEN_CNN, DEFAULT_LAMBDA, packed)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sd.ida(h, iters, abcs.DEN_CNN, DEFAULT_LAMBDA, packed, x)
    e1.record()
    torch.cuda.synchronize()
    assert abcs.abcs_sync_status(h) == 0
    ms = e0.elapsed_time(e1)
    v = n * sd.Hc * sd.Wc * iters / (ms * 1e-3) / 1e9
    log(json.dumps({"learned_ida_iters": iters, "images": n, "ms": ms, "Gpx_iter_per_s": v}))
    return v


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["tune-lambda", "train", "eval", "video", "time", "all"])
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--images", type=int, default=512)
    ap.add_argument("--steps", type=int, default=12000)
    ap.add_argument("--lam", type=float, default=DEFAULT_LAMBDA)
    ap.add_argument("--eval-images", type=int, default=128)
    ap.add_argument("--report", default=None, help="write a JSON report here")
    ap.add_argument("--captures-a", default="0,0,0,1,2,3,4,6,8",
                    help="IDA iterations whose denoiser inputs form the phase-A crops (repeat to weight)")
    ap.add_argument("--captures-b", default="0,0,1,2,2,3,3,4,4,5,6,8",
                    help="iterations captured along the network's own trajectories (phase B)")
    ap.add_argument("--rounds", type=int, default=8, help="phase B rounds (own trajectories, fine-tuning)")
    ap.add_argument("--init", default=None, help="train: start phase B from these weights (no phase A)")
    ap.add_argument("--round-steps", type=int, default=4000, help="Adam steps per phase B round")
    ap.add_argument("--large-every", type=int, default=3,
                    help="every n-th training batch of large images (0: none)")
    ap.add_argument("--large-size", default="1088,1920", help="H,W of the large training images")
    ap.add_argument("--iters", type=int, default=2, help="time: learned IDA iterations")
    a = ap.parse_args()
    h = abcs.abcs_create()
    report = {}
    if a.cmd in ("tune-lambda", "all"):
        best, mean = tune_lambda(h)
        report["tune_lambda"] = {"best": best, "mean_psnr": mean}
    if a.cmd in ("train", "all"):
        # phase A: denoiser inputs along plain-IDA trajectories
        caps_a = tuple(int(x) for x in a.captures_a.split(","))
        caps_b = tuple(int(x) for x in a.captures_b.split(","))
        large = tuple(int(x) for x in a.large_size.split(","))
        if a.init:
            # continue from trained weights: phase B rounds only
            w, hist_a, secs_a = load_weights(a.init), [], 0.0
            R = C = D = torch.empty((0, 64, 64), dtype=torch.float32, device="cuda")
            S = T = torch.empty(0, dtype=torch.float32, device="cuda")
        else:
            R, C, S, D, T = make_pairs(h, n_images=a.images, lam=a.lam, captures=caps_a, crops=48,
                                       large_every=a.large_every, large_size=large)
            print(f"phase A: {R.shape[0]} training crops")
            w, hist_a, secs_a = train(h, R, C, S, D, steps=a.steps, T=T)
        report["train"] = {"phase_a_crops": int(R.shape[0]), "steps": [a.steps], "seconds": secs_a,
                           "loss": {"A": hist_a}, "rounds": []}
        report["train"]["rounds"].append({"round": 0, "trajectory_psnr": trajectory_psnr(h, w)})
        # phase B, in rounds: inputs along the network's own IDA trajectories
        # (Eq. 13 with the Onsager term of Eq. 28), captured with the current
        # weights on fresh images, join the training set, and the network is
        # fine-tuned; each round sees the trajectories its predecessor made
        pk = torch.empty(abcs.abcs_cnn_packed_bytes(), dtype=torch.uint8, device="cuda")
        for rnd in range(1, a.rounds + 1):
            abcs.abcs_cnn_pack(h, torch.tensor(w, device="cuda"), pk)
            R2, C2, S2, D2, T2 = make_pairs(h, n_images=a.images // 2, lam=a.lam, captures=caps_b, crops=64,
                                            seed=TRAIN_SEED + 5_000_000 * rnd, packed=pk,
                                            large_every=a.large_every, large_size=large)
            R, C, S, D, T = (torch.cat([R, R2]), torch.cat([C, C2]), torch.cat([S, S2]), torch.cat([D, D2]),
                             torch.cat([T, T2]))
            del R2, C2, S2, D2, T2
            print(f"phase B round {rnd}: {R.shape[0]} training crops")
            w, hist_b, secs_b = train(h, R, C, S, D, steps=a.round_steps, lr=3e-4, params=w, seed=1 + rnd, T=T)
            report["train"]["rounds"].append({"round": rnd, "crops": int(R.shape[0]), "seconds": secs_b,
                                              "loss": hist_b, "trajectory_psnr": trajectory_psnr(h, w)})
            report["train"]["seconds"] += secs_b
            os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
            w.astype("<f4").tofile(a.out)
            if a.report:
                with open(a.report, "w") as f:
                    json.dump(report, f, indent=1)
        del R, C, S, D, T
        torch.cuda.empty_cache()
    if a.cmd in ("eval", "all"):
        w = load_weights(a.out if a.cmd == "all" else a.weights)
        report["eval"] = evaluate(h, w, n=a.eval_images, lam=a.lam)
        report["lambda"] = a.lam
    if a.cmd == "time":
        time_learned(h, load_weights(a.weights), iters=a.iters)
    if a.cmd in ("video", "all"):
        w = load_weights(a.out if a.cmd == "all" else a.weights)
        report["video"] = video_eval(h, w, lam=a.lam)
    if a.report:
        with open(a.report, "w") as f:
            json.dump(report, f, indent=1)
    abcs.abcs_destroy(h)


if __name__ == "__main__":
    main()
