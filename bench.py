#!/usr/bin/env python3
"""Benchmark of the ABCS hot path on GB300.

Workload (the batched sensing/reconstruction configuration): 64 synthetic
512x512 uint8 greyscale images (seeded generator, paper_2001_09632_gb300.synth),
B = 16, AL-DCT-BBV, subrate 0.3, FP32.  One step = abcs_sense +
abcs_reconstruct over the whole batch (pilot BBV, exact allocation, packed
zigzag DCT measurements, block inverse DCT).  `value` is whole-job
Mpixel/s with the inputs resident in HBM; L2 (129 MB) is flushed between
timed steps by writing a 512 MB buffer.  A second timed region measures IDA
(plain TI-DCT denoiser, D_F = 2) in Mpixel*iteration/s on the same batch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl abcs|reference]

With torchrun (N > 1) every rank senses its own 64-image batch (replicas,
no data-path collective); the time is the max over ranks.
`--impl reference` times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload, on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel/s ABCS sense+recon and IDA/iter; learned vs plain IDA at equal PSNR"
N_IMG, H, W, B, SUBRATE, SEED = 64, 512, 512, 16, 0.3, 1000
IDA_ITERS, LAMBDA, DF = 10, 2.3, 2.0
FLUSH_BYTES = 512 << 20
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the kernels of
# one step on this workload, from an ncu capture of the current kernels
# (None where none was taken); must be re-measured whenever a kernel
# changes.  Taken with
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
#       --clock-control none -k regex:"bbv_image|sense_tc_kernel|recon_tc_kernel" -s 3 -c 3
#       python bench.py --case step
# (64 x 512x512, BBV r 0.3, FP16x2; ncu flushes the caches before each launch)
# (sense = bbv_image_kernel 10,559,232 + 0 and sense_tc_kernel 17,604,608 + 0 bytes;
# reconstruct = recon_tc_kernel 18,111,744 + 7,710,208 bytes)
TRAFFIC = {"recon_fp16x2": 25821952, "sense_fp16x2": 28163840}


# ---------------------------------------------------------------------------
# Fixed single-kernel workloads (`--case NAME`): each seeds its inputs, runs
# the call a few times and times the last run with CUDA events.  They are
# the programs the ncu summaries under profiles/ capture.
# ---------------------------------------------------------------------------
def _timed(fn, reps=10):
    """Mean ms per call of `reps` calls queued back to back (the host runs
    ahead of the device, so launch overheads between calls are hidden)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def case_bm3d(h):
    """abcs_denoise_bm3d, 16 x 512x512, sigma 20."""
    import numpy as np
    import torch
    from paper_2001_09632_gb300 import abcs, synth
    n, H, W = 16, 512, 512
    imgs = synth.gen_batch(n, H, W, 5).astype(np.float32)
    rng = np.random.default_rng(0)
    r = torch.tensor(imgs + rng.normal(0, 20, imgs.shape).astype(np.float32), device="cuda")
    out = torch.empty_like(r)
    sig = torch.full((n,), 20.0, device="cuda")
    run = lambda: abcs.abcs_denoise_bm3d(h, r, n, H, W, sig, 2.7, out)
    for _ in range(2):
        run()
    return _timed(run, 1)


def case_thi(h):
    """abcs_thi, 64 x 512x512, M = floor(0.3 N)."""
    import torch
    from paper_2001_09632_gb300 import abcs, synth
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
    return _timed(run)


def case_damp(h):
    """abcs_damp, 16 x 512x512, DD r 0.1, 3 iterations, TI-DCT."""
    import torch
    from paper_2001_09632_gb300 import abcs, synth
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
    return _timed(run, 1)


def case_tidct(h):
    """abcs_denoise_tidct (the plain denoiser alone), 64 x 512x512, sigma 20 per image."""
    import torch
    from paper_2001_09632_gb300 import abcs, synth
    n, H, W = 64, 512, 512
    gen = torch.Generator(device="cuda").manual_seed(11)
    r = torch.from_numpy(synth.gen_batch(n, H, W, 4321)).cuda().float()
    r += 20.0 * torch.randn((n, H, W), device="cuda", generator=gen)
    sig = torch.full((n,), 20.0, device="cuda")
    x = torch.empty_like(r)
    run = lambda: abcs.abcs_denoise_tidct(h, r, n, H, W, sig, 2.3, x)
    for _ in range(3):
        run()
    return _timed(run)


def _sense_case(h, variant, r, prec, seed=1234):
    import torch
    from paper_2001_09632_gb300 import abcs, synth
    n, H, W, B = 64, 512, 512, 16
    d = torch.from_numpy(synth.gen_batch(n, H, W, seed)).cuda()
    plan = abcs.abcs_plan(H, W, B, r, variant)
    nB = plan["n_blocks"]
    c = torch.empty(n * nB, dtype=torch.int32, device="cuda")
    o = torch.empty(n * nB + 1, dtype=torch.int64, device="cuda")
    y = torch.empty(n * plan["M"], dtype=torch.float32, device="cuda")
    sense = lambda: abcs.abcs_sense(h, d, n, H, W, W, H * W, B, r, variant, prec, c, o, y, n * plan["M"])
    return sense, (c, o, y, n, H, W, B)


def case_recon(h):
    """abcs_reconstruct FP16x2, 64 x 512x512, BBV r 0.3."""
    import torch
    from paper_2001_09632_gb300 import abcs
    sense, (c, o, y, n, H, W, B) = _sense_case(h, abcs.BBV, 0.3, abcs.TC_FP16X2)
    sense()
    x = torch.empty((n, H, W), device="cuda")
    run = lambda: abcs.abcs_reconstruct(h, c, o, y, n, H, W, B, abcs.TC_FP16X2, x)
    for _ in range(3):
        run()
    return _timed(run)


def case_sense(h):
    """abcs_sense FP16x2, 64 x 512x512, BBV r 0.3 (pilot + allocation + sensing)."""
    from paper_2001_09632_gb300 import abcs
    sense, _ = _sense_case(h, abcs.BBV, 0.3, abcs.TC_FP16X2)
    for _ in range(3):
        sense()
    return _timed(sense)


def case_step(h):
    """One step of the bench: abcs_sense + abcs_reconstruct FP16x2, 64 x 512x512, BBV r 0.3."""
    import torch
    from paper_2001_09632_gb300 import abcs
    sense, (c, o, y, n, H, W, B) = _sense_case(h, abcs.BBV, 0.3, abcs.TC_FP16X2)
    x = torch.empty((n, H, W), device="cuda")

    def step():
        sense()
        abcs.abcs_reconstruct(h, c, o, y, n, H, W, B, abcs.TC_FP16X2, x)
    for _ in range(3):
        step()
    return _timed(step)


def case_sense_dd(h):
    """abcs_sense FP16x2, 64 x 512x512, DD r 0.3 (DD pilot + allocation + sensing)."""
    from paper_2001_09632_gb300 import abcs
    sense, _ = _sense_case(h, abcs.DD, 0.3, abcs.TC_FP16X2)
    for _ in range(3):
        sense()
    return _timed(sense)


def ida_linear_step(h, s, counts, offsets, coeffs, x, total_coeffs, iters=10, reps=5):
    """The IDA linear step (Eqs. 25, 28) plus sigma (Eq. 15) per iteration on
    the bench workload: abcs_ida with the identity denoiser, FP32 and the
    tensor-core FP16x2 step.  Algorithmic bytes of an iteration with x and
    z_prev: x read, r written (8 B/px), y and z_prev read, z written
    (12 B per measurement)."""
    import torch
    from paper_2001_09632_gb300 import abcs
    n, H, W = x.shape
    px = n * H * W
    out = {}
    for name, prec in (("fp32", abcs.FP32), ("fp16x2", abcs.TC_FP16X2)):
        abcs.abcs_set_ida_precision(h, prec)
        run = lambda: abcs.abcs_ida(h, counts, offsets, coeffs, n, H, W, 16, iters, 2.0, abcs.DEN_NONE, 0.0,
                                    None, x, None, s)
        run()
        ev = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(torch.cuda.current_stream())     # s is the current stream's handle
            run()
            e1.record(torch.cuda.current_stream())
            ev.append((e0, e1))
        torch.cuda.synchronize()
        out[name + "_us_per_iteration"] = 1e3 * statistics.median(a.elapsed_time(b) for a, b in ev) / iters
    abcs.abcs_set_ida_precision(h, abcs.FP32)
    assert abcs.abcs_sync_status(h, s) == 0
    bytes_it = 8 * px + 12 * total_coeffs
    out["bytes_per_iteration"] = bytes_it
    out["hbm_floor_us"] = None
    out["how"] = ("abcs_ida, identity denoiser, 10 iterations per call, median of 5 calls / 10; each iteration "
                  "is the linear kernel and the sigma kernel; iteration 0 reads no x or z_prev")
    return out


def _ida_linear_setup(h, seed=2468):
    """64 x 512x512 sensed with BBV r 0.3 and an abcs_ida call with the
    identity denoiser: each iteration is the linear step (Eqs. 25, 28) and
    sigma (Eq. 15) alone."""
    import torch
    from paper_2001_09632_gb300 import abcs
    sense, (c, o, y, n, H, W, B) = _sense_case(h, abcs.BBV, 0.3, abcs.TC_FP16X2, seed)
    sense()
    x = torch.empty((n, H, W), device="cuda")
    iters = 10
    run = lambda: abcs.abcs_ida(h, c, o, y, n, H, W, B, iters, 2.0, abcs.DEN_NONE, 0.0, None, x)
    return run, iters, (c, o, y, n, H, W, B)


def case_ida_linear(h):
    """abcs_ida with the identity denoiser (10 iterations: linear step +
    sigma), 64 x 512x512, BBV r 0.3, tensor-core FP16x2 linear step."""
    from paper_2001_09632_gb300 import abcs
    abcs.abcs_set_ida_precision(h, abcs.TC_FP16X2)
    run, iters, _ = _ida_linear_setup(h)
    for _ in range(2):
        run()
    return _timed(run, 3)


def case_ida_linear_fp32(h):
    """The same with the FP32 CUDA-core linear step."""
    run, iters, _ = _ida_linear_setup(h)
    for _ in range(2):
        run()
    return _timed(run, 3)


CASES = {"bm3d": case_bm3d, "thi": case_thi, "damp": case_damp, "recon": case_recon, "sense": case_sense,
         "sense_dd": case_sense_dd, "step": case_step, "ida_linear": case_ida_linear,
         "ida_linear_fp32": case_ida_linear_fp32, "tidct": case_tidct}


def run_case(name):
    from paper_2001_09632_gb300 import abcs
    h = abcs.abcs_create()
    ms = CASES[name](h)
    print(json.dumps({"case": name, "ms": ms, "status": abcs.abcs_sync_status(h)}), flush=True)
    abcs.abcs_destroy(h)


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="abcs", choices=["abcs", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the uneven-batch IDA and the learned-vs-plain video measurements")
    ap.add_argument("--case", default=None, choices=sorted(CASES),
                    help="time one fixed single-kernel workload (for ncu) instead of the bench")
    ap.add_argument("--precision", default="fp16x2", choices=["fp32", "fp16x2", "bf16x2", "bf16"],
                    help="block-DCT arithmetic of the timed path (fp16x2 and bf16x2 meet the "
                         "1e-5 relative-L2 bar against the FP64 oracle; bf16 does not)")
    return ap.parse_args()


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling in the background (every 100 ms)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        self.t0 = time.time()

    def mark(self):
        return time.time()

    def stop(self, t_start, t_end):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        # rows are sampled at ~100 ms; keep the ones inside [t_start, t_end]
        n = len(rows)
        dt = (time.time() - self.t0) / max(n, 1)
        sel = [r for i, r in enumerate(rows) if t_start - dt <= self.t0 + i * dt <= t_end + dt] or rows
        sm = [float(r[1]) for r in sel if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in sel if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in sel:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip() == "Active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sel)}


def _oracle_sense_recon(imgs):
    import oracle as O
    for im in imgs:
        out = O.sense(im, B, SUBRATE, O.BBV)
        O.reconstruct(out["counts"], out["y"], im.shape[0], im.shape[1], B)


def cpu_baseline(imgs, budget_s=6.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample:
    images of the batch in order (wrapping around) until budget_s elapses."""
    t0, c0 = time.perf_counter(), time.process_time()
    done = 0
    while time.perf_counter() - t0 < budget_s and done < 20 * len(imgs):
        _oracle_sense_recon(imgs[done % len(imgs):done % len(imgs) + 1])
        done += 1
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    px = done * imgs.shape[1] * imgs.shape[2]
    return {"value": px / wall / 1e6, "unit": "Mpixel/s", "cores": max(1, round(cpu / wall)),
            "kind": "oracle",
            "sample": f"{done} images of 512x512 (the batch, in order), sense (BBV r=0.3 B=16) + "
                      f"IDCT, FP64 numpy, {wall:.1f} s"}


def _oracle_repeat(args):
    img, reps = args
    for _ in range(reps):
        _oracle_sense_recon(img[None])
    return reps


def cpu_baseline_all_cores(imgs, per_img_s, budget_s=6.0):
    """The same oracle on every host core the process may use: one spawned
    worker per core (numpy single-threaded in each), each repeating one image
    of the batch for about budget_s."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    reps = max(1, int(budget_s / max(per_img_s, 1e-4)))
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_repeat, [(imgs[0][:64], 1)] * cores)          # workers up and imported
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_repeat, [(imgs[k % len(imgs)], reps) for k in range(cores)]))
        wall = time.perf_counter() - t0
    px = done * imgs.shape[1] * imgs.shape[2]
    return {"value": px / wall / 1e6, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} images of 512x512 on {cores} spawned processes ({reps} repeats of one batch "
                      f"image each), sense (BBV r=0.3 B=16) + IDCT, FP64 numpy, {wall:.1f} s"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    from paper_2001_09632_gb300 import synth
    img = synth.gen_image(H, W, SEED)
    t = time.perf_counter()
    _oracle_sense_recon(img[None])
    per_img = time.perf_counter() - t
    # a step is a crop of `rows` rows of one image, sized so K + W steps take <~ 120 s
    rows = H
    while rows > B and (a.steps + a.warmup) * per_img * rows / H > 120.0:
        rows //= 2
    sample = img[:rows]
    for _ in range(a.warmup):
        _oracle_sense_recon(sample[None])
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(a.steps):
        _oracle_sense_recon(sample[None])
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    v = a.steps * rows * W / wall / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpixel/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": wall / a.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "64 x 512x512 uint8, B=16, BBV, subrate 0.3: sense + IDCT",
                       "sample_per_step": f"{rows}x{W} crop of one image"},
            "cpu_baseline": {"value": v, "unit": "Mpixel/s", "cores": max(1, round(cpu / wall)),
                             "kind": "oracle", "sample": f"{rows}x{W} crop per step"},
            "e2e": {"value": v, "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def uneven_batch_ida(h, world, max_over_ranks, barrier, n=256, subrate=0.2, iters=30, seed=5000):
    """256 images, 40% 256^2 / 40% 512^2 / 20% 1024^2, B cycling 8/16/32,
    AL-DCT-BBV at subrate 0.2, 30 plain IDA iterations in ONE abcs_ida_batch
    call (persistent kernel, graph replay).  Also the same work as one
    abcs_ida call per (size, B) group, for comparison."""
    import torch
    from paper_2001_09632_gb300 import abcs, synth
    from paper_2001_09632_gb300.uneven import UnevenBatch
    items = synth.gen_uneven_batch(n, seed)
    ub = UnevenBatch(h, items, subrate)
    stream = torch.cuda.current_stream()
    for _ in range(2):                     # first call: autotune + capture
        ub.ida(h, iters, abcs.DEN_TIDCT, LAMBDA, DF)
    torch.cuda.synchronize()
    ev = []
    barrier()
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ub.ida(h, iters, abcs.DEN_TIDCT, LAMBDA, DF)
        e1.record(stream)
        ev.append((e0, e1))
    barrier()
    ms = max_over_ranks(statistics.median(a.elapsed_time(b) for a, b in ev))
    assert abcs.abcs_sync_status(h) == 0
    psnr = ub.psnr()
    # the same images, one abcs_sense and one abcs_ida call per (size, B) group
    groups = ub.per_group_sensing(h, items)
    outs = [torch.empty((len(ks), (H // B) * B, (W // B) * B), dtype=torch.float32, device="cuda")
            for (H, W, B, ks, c, o, y) in groups]

    def per_group():
        for (H, W, B, ks, c, o, y), xo in zip(groups, outs):
            abcs.abcs_ida(h, c, o, y, len(ks), H, W, B, iters, DF, abcs.DEN_TIDCT, LAMBDA, None, xo, None)
    per_group()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    per_group()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_groups = max_over_ranks(e0.elapsed_time(e1))
    same = all(torch.equal(ub.image(k), xo[j]) for (H, W, B, ks, c, o, y), xo in zip(groups, outs)
               for j, k in enumerate(ks))
    # sensing the whole batch: one abcs_sense_batch call (two launches)
    for _ in range(3):
        ub.sense(h)
    ev = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ub.sense(h)
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    sense_ms = max_over_ranks(statistics.median(a.elapsed_time(b) for a, b in ev))
    assert abcs.abcs_sync_status(h) == 0
    return {"value": world * ub.pixels * iters / (ms * 1e-3) / 1e6, "unit": "Mpixel*iter/s",
            "images": n, "mix": "40% 256x256, 40% 512x512, 20% 1024x1024; B cycles 8, 16, 32",
            "subrate": subrate, "variant": "BBV", "iters": iters, "denoiser": "tidct", "lambda": LAMBDA,
            "pixels": ub.pixels, "measurements": ub.measurements, "ms_per_call": ms,
            "launch": "one persistent cooperative kernel per call, CUDA graph replay",
            "sensing": {"ms_per_call": sense_ms, "Mpixel_per_s": world * ub.pixels / (sense_ms * 1e-3) / 1e6,
                        "how": "one abcs_sense_batch call over the 256 images (pilot + allocation launch, "
                               "sensing launch), FP32"},
            "per_group_calls": {"calls": len(groups), "ms": ms_groups,
                                "value": world * ub.pixels * iters / (ms_groups * 1e-3) / 1e6,
                                "identical_output": same},
            "mean_psnr": sum(psnr) / len(psnr),
            "l2": "working set (x, r, z, y: ~1.2 GB) larger than L2"}


def video_learned_vs_plain(h):
    """The 120-frame 1920x1088 clip, AL-DCT-DD at subrate 0.25, 30 frames
    per call: learned IDA (10 iterations) vs plain IDA (30 iterations)."""
    from paper_2001_09632_gb300 import train
    return train.video_eval(h, train.load_weights(), reps=1, log=lambda *_: None)


def images_learned_vs_plain(h, n=128):
    """128 held-out 512x512 images (seeds disjoint from training),
    AL-DCT-BBV at subrates 0.1..0.5: mean PSNR of plain IDA after 30
    iterations and of learned IDA after 1, 2, 3, 4, 6, 10, and the Mpixel/s
    speedup of the fewest learned iterations within 0.1 dB of plain-30."""
    from paper_2001_09632_gb300 import train
    out = train.evaluate(h, train.load_weights(), n=n, plain_iters=(10, 30), learned_iters=(1, 2, 3, 4, 6, 10),
                         log=lambda *_: None)
    return {"images": n, "size": [512, 512], "variant": "BBV", "quality": "abcs_psnr_ssim",
            "per_subrate": {r: {"psnr_idct": v["psnr_idct"], "ssim_idct": v["ssim_idct"],
                                "psnr_plain30": v["plain"]["30"]["psnr"],
                                "ssim_plain30": v["plain"]["30"]["ssim"],
                                "Mpx_per_s_plain30": v["plain"]["30"]["Mpx_per_s"],
                                "learned": {it: {"psnr": e["psnr"], "ssim": e["ssim"], "Mpx_per_s": e["Mpx_per_s"]}
                                            for it, e in v["learned"].items()},
                                "equal": v["equal"]} for r, v in out.items()}}


def video_stream(h, n_frames=120, H=1088, W=1920, fpb=30):
    """The video clip as a stream: 120 frames of 1920x1088 in pinned
    host memory, 30 per batch, each batch copied to the device, sensed with
    AL-DCT-DD at r = 0.25 and reconstructed by IDA; Mpixel/s from the first
    copy to the last image, with the stages of consecutive batches run one
    after another or overlapped on three streams (paper_2001_09632_gb300.video;
    identical images either way).  Learned IDA (1 iteration) and plain IDA
    (30 iterations)."""
    import numpy as np
    import torch
    from paper_2001_09632_gb300 import abcs, synth, train
    from paper_2001_09632_gb300.video import VideoPipeline
    seed = train.EVAL_SEED + 7
    frames = torch.from_numpy(np.concatenate([synth.gen_video(min(fpb, n_frames - f0), H, W, seed, first_frame=f0)
                                              for f0 in range(0, n_frames, fpb)])).pin_memory()
    p = torch.tensor(train.load_weights(), device="cuda")
    packed = torch.empty(abcs.abcs_cnn_packed_bytes(), dtype=torch.uint8, device="cuda")
    abcs.abcs_cnn_pack(h, p, packed)
    out = {"frames": n_frames, "size": [H, W], "frames_per_batch": fpb, "variant": "DD", "subrate": 0.25,
           "from": "pinned host frames (H2D copy inside the timed region)"}
    for name, iters, den in (("learned_1", 1, abcs.DEN_CNN), ("plain_30", 30, abcs.DEN_TIDCT)):
        vp = VideoPipeline(H, W, 16, 0.25, abcs.DD, fpb, iters, den, cnn_packed=packed)
        x = torch.empty((n_frames, vp.Hc, vp.Wc), dtype=torch.float32, device="cuda")
        vp.run(frames, x, overlap=True)                          # warm-up
        row = {}
        for mode, ov in (("sequential", False), ("overlapped", True)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            vp.run(frames, x, overlap=ov)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            row[mode] = {"ms": ms, "Mpx_per_s": n_frames * vp.Hc * vp.Wc / (ms * 1e-3) / 1e6}
        clean = frames[:, :vp.Hc, :vp.Wc].cuda().float()
        d = x.clamp(0, 255) - clean
        row["psnr"] = float((10.0 * torch.log10(255.0 ** 2 / (d * d).flatten(1).mean(1))).mean())
        row["overlap_gain"] = row["sequential"]["ms"] / row["overlapped"]["ms"]
        out[name] = row
        vp.close()
        del x, clean, d
    return out


def bm3d_comparison(h, n=16, H=512, W=512, B=16, iters=(10, 30)):
    """BM3D (hard-thresholding step) as IDA's plain denoiser, the one the
    paper pairs with IDA (Sec. VII, Fig. 7a), beside TI-DCT and the learned
    CNN: mean PSNR on n held-out 512x512 images (DD and BBV at r = 0.1 and
    0.3) and Mpixel/s of each; learned IDA (1 iteration) against plain IDA
    with BM3D (30 iterations)."""
    import torch
    from paper_2001_09632_gb300 import abcs, synth, train
    imgs = synth.gen_batch(n, H, W, 8765)
    d_img = torch.from_numpy(imgs).cuda()
    clean = d_img.float()
    nB = (H // B) * (W // B)
    x = torch.empty((n, H, W), dtype=torch.float32, device="cuda")
    p = torch.tensor(train.load_weights(), device="cuda")
    packed = torch.empty(abcs.abcs_cnn_packed_bytes(), dtype=torch.uint8, device="cuda")
    abcs.abcs_cnn_pack(h, p, packed)

    def psnr():
        d = x.clamp(0, 255) - clean
        return float((10.0 * torch.log10(255.0 ** 2 / (d * d).flatten(1).mean(1))).mean())

    def run(c, o, y, it, den, lam, pk):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        abcs.abcs_ida(h, c, o, y, n, H, W, B, it, 2.0, den, lam, pk, x)
        e1.record()
        torch.cuda.synchronize()
        return psnr(), n * H * W / (e0.elapsed_time(e1) * 1e-3) / 1e6

    out = {"images": n, "size": [H, W], "B": B, "lambda_tidct": 2.3, "lambda_bm3d": 2.7, "cases": {}}
    for vname, variant in (("dd", abcs.DD), ("bbv", abcs.BBV)):
        for r in (0.1, 0.3):
            plan = abcs.abcs_plan(H, W, B, r, variant)
            c = torch.empty(n * nB, dtype=torch.int32, device="cuda")
            o = torch.empty(n * nB + 1, dtype=torch.int64, device="cuda")
            y = torch.empty(n * plan["M"], dtype=torch.float32, device="cuda")
            abcs.abcs_sense(h, d_img, n, H, W, W, H * W, B, r, variant, abcs.FP32, c, o, y, n * plan["M"])
            row = {}
            run(c, o, y, 1, abcs.DEN_BM3D, 2.7, None)                   # warm-up
            for it in iters:
                for name, den, lam, pk in (("tidct", abcs.DEN_TIDCT, 2.3, None), ("bm3d", abcs.DEN_BM3D, 2.7, None)):
                    ps, mpx = run(c, o, y, it, den, lam, pk)
                    row[f"{name}_{it}"] = {"psnr": ps, "Mpx_per_s": mpx}
            ps, mpx = run(c, o, y, 1, abcs.DEN_CNN, 0.0, packed)
            row["learned_1"] = {"psnr": ps, "Mpx_per_s": mpx}
            ref = row[f"bm3d_{iters[-1]}"]
            row["learned_1_vs_bm3d"] = {"dpsnr": ps - ref["psnr"], "speedup": mpx / ref["Mpx_per_s"]}
            out["cases"][f"{vname}_r{r}"] = row
    assert abcs.abcs_sync_status(h) == 0
    return out


def damp_vs_ida(h, n=16, H=512, W=512, B=16, iters=(10, 30)):
    """Sec. VI-1/2, Figs. 7-8: D-AMP (Eq. 24, D_F = 1), DAMP-D (Eq. 27,
    D_F = 2) and IDA (Eq. 28, D_F = 2), all with the TI-DCT denoiser, on n
    held-out 512x512 images sensed with AL-DCT-DD and AL-DCT-BBV at
    r = 0.1 and 0.3: mean PSNR after each iteration count, and the time per
    iteration of each (D-AMP runs the denoiser twice per iteration)."""
    import torch
    from paper_2001_09632_gb300 import abcs, synth
    imgs = synth.gen_batch(n, H, W, 8765)
    d_img = torch.from_numpy(imgs).cuda()
    clean = d_img.float()
    gen = torch.Generator(device="cuda").manual_seed(11)
    probe = torch.where(torch.rand((n, H, W), device="cuda", generator=gen) < 0.5, -1.0, 1.0)
    nB = (H // B) * (W // B)
    x = torch.empty((n, H, W), dtype=torch.float32, device="cuda")
    lam = 2.3

    def psnr():
        d = x.clamp(0, 255) - clean
        mse = (d * d).flatten(1).mean(1)
        return float((10.0 * torch.log10(255.0 ** 2 / mse)).mean())

    out = {"images": n, "size": [H, W], "B": B, "denoiser": "tidct", "lambda": lam, "psnr": {}, "ms_per_iter": {}}
    for vname, variant in (("dd", abcs.DD), ("bbv", abcs.BBV)):
        for r in (0.1, 0.3):
            plan = abcs.abcs_plan(H, W, B, r, variant)
            c = torch.empty(n * nB, dtype=torch.int32, device="cuda")
            o = torch.empty(n * nB + 1, dtype=torch.int64, device="cuda")
            y = torch.empty(n * plan["M"], dtype=torch.float32, device="cuda")
            abcs.abcs_sense(h, d_img, n, H, W, W, H * W, B, r, variant, abcs.FP32, c, o, y, n * plan["M"])
            row = {}
            for name in ("ida", "damp_d", "d_amp"):
                for it in iters:
                    if name == "ida":
                        abcs.abcs_ida(h, c, o, y, n, H, W, B, it, 2.0, abcs.DEN_TIDCT, lam, None, x)
                    else:
                        abcs.abcs_damp(h, c, o, y, n, H, W, B, it, 2.0 if name == "damp_d" else 1.0,
                                       abcs.DEN_TIDCT, lam, None, probe, x)
                    row[f"{name}_{it}"] = psnr()
            out["psnr"][f"{vname}_r{r}"] = row
    assert abcs.abcs_sync_status(h) == 0
    # time per iteration at DD r = 0.1
    for name in ("ida", "damp_d", "d_amp"):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        if name == "ida":
            abcs.abcs_ida(h, c, o, y, n, H, W, B, 10, 2.0, abcs.DEN_TIDCT, lam, None, x)
        else:
            abcs.abcs_damp(h, c, o, y, n, H, W, B, 10, 2.0 if name == "damp_d" else 1.0, abcs.DEN_TIDCT, lam,
                           None, probe, x)
        e1.record()
        torch.cuda.synchronize()
        out["ms_per_iter"][name] = e0.elapsed_time(e1) / 10
    assert abcs.abcs_sync_status(h) == 0
    return out


def thi_correlation(h, n=64, H=512, W=512, B=16, reps=5):
    """THI (Sec. IV, Sec. V-B): the correlation coefficient rho between the
    per-block counts BBV / DD allocate and the counts THI keeps at the same
    M, mean over n held-out images per subrate (the analogue of Table 2 on
    synthetic images; the paper's own values, on its image set, are quoted
    as context), the PSNR of THI's image against the adaptive IDCT images
    at r = 0.3, and the time of one abcs_thi call over the batch."""
    import torch
    from paper_2001_09632_gb300 import abcs, synth
    imgs = synth.gen_batch(n, H, W, 4321)
    d_img = torch.from_numpy(imgs).cuda()
    nB = (H // B) * (W // B)
    N = nB * B * B

    def sense(r, variant):
        plan = abcs.abcs_plan(H, W, B, r, variant)
        c = torch.empty(n * nB, dtype=torch.int32, device="cuda")
        o = torch.empty(n * nB + 1, dtype=torch.int64, device="cuda")
        y = torch.empty(max(n * plan["M"], 1), dtype=torch.float32, device="cuda")
        abcs.abcs_sense(h, d_img, n, H, W, W, H * W, B, r, variant, abcs.FP32, c, o, y, n * plan["M"])
        return plan, c, o, y

    def psnr_of(rec):
        d = rec.clamp(0, 255) - d_img.float()
        mse = (d * d).flatten(1).mean(1)
        return float((10.0 * torch.log10(255.0 ** 2 / mse)).mean())

    _, _, _, full = sense(1.0, abcs.ZZ)                      # every coefficient, zigzag order
    cnt = torch.empty(n * nB, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    out = {"images": n, "size": [H, W], "B": B, "rho": {"bbv": {}, "dd": {}}}
    rec = torch.empty((n, H, W), dtype=torch.float32, device="cuda")
    for name, variant in (("bbv", abcs.BBV), ("dd", abcs.DD)):
        for r in (0.1, 0.2, 0.3, 0.4, 0.5):
            plan, c, o, y = sense(r, variant)
            abcs.abcs_thi(h, full, n, H, W, B, plan["M"], c, cnt, rho, None)
            out["rho"][name][str(r)] = float(rho.mean())
            if r == 0.3:
                abcs.abcs_reconstruct(h, c, o, y, n, H, W, B, abcs.FP32, rec)
                out.setdefault("psnr_r03", {})[name + "_idct"] = psnr_of(rec)
    assert abcs.abcs_sync_status(h) == 0
    M = abcs.abcs_plan(H, W, B, 0.3, abcs.BBV)["M"]
    masked = torch.empty_like(full[: n * N])
    allc = torch.full((n * nB,), B * B, dtype=torch.int32, device="cuda")
    offs = torch.arange(0, n * nB + 1, dtype=torch.int64, device="cuda") * (B * B)
    abcs.abcs_thi(h, full, n, H, W, B, M, None, cnt, None, masked)
    abcs.abcs_reconstruct(h, allc, offs, masked, n, H, W, B, abcs.FP32, rec)
    out["psnr_r03"]["thi"] = psnr_of(rec)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    abcs.abcs_thi(h, full, n, H, W, B, M, None, cnt, None, None)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        abcs.abcs_thi(h, full, n, H, W, B, M, None, cnt, None, None)
    e1.record()
    torch.cuda.synchronize()
    assert abcs.abcs_sync_status(h) == 0
    ms = e0.elapsed_time(e1) / reps
    out["thi_ms"] = ms
    out["thi_Mpx_per_s"] = n * H * W / (ms * 1e-3) / 1e6
    out["paper_table2_512_context"] = {"dd": [0.741, 0.818, 0.818, 0.807, 0.852],
                                       "bbv": [0.719, 0.784, 0.795, 0.786, 0.802]}
    return out


def subrate_sweep(h, prec, d_img, flush, hbm_peak, steps=30):
    """The batched workload at every subrate and both adaptive variants
    (64 x 512x512, B = 16, BBV and DD, r = 0.1 .. 0.5; the bench default
    precision): abcs_sense and abcs_reconstruct timed with CUDA events on
    the launching stream, L2 flushed before each step; Mpixel/s and the
    step's HBM fraction against the algorithmic bytes 5 + 8 M/N per pixel
    (uint8 image read, packed coefficients written and read back, counts
    and offsets, FP32 image written)."""
    import torch
    from paper_2001_09632_gb300 import abcs
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream
    n = N_IMG
    nB = (H // B) * (W // B)
    cap = n * abcs.abcs_plan(H, W, B, 0.5, abcs.DD)["M"]
    counts = torch.empty(n * nB, dtype=torch.int32, device="cuda")
    offsets = torch.empty(n * nB + 1, dtype=torch.int64, device="cuda")
    coeffs = torch.empty(cap, dtype=torch.float32, device="cuda")
    rec = torch.empty((n, H, W), dtype=torch.float32, device="cuda")
    out = {}
    for name, variant in (("bbv", abcs.BBV), ("dd", abcs.DD)):
        for r in (0.1, 0.2, 0.3, 0.4, 0.5):
            def sense():
                abcs.abcs_sense(h, d_img, n, H, W, W, H * W, B, r, variant, prec, counts, offsets, coeffs, cap,
                                None, s)

            def recon():
                abcs.abcs_reconstruct(h, counts, offsets, coeffs, n, H, W, B, prec, rec, None, s)
            for _ in range(3):
                sense()
                recon()
            ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
            for e0, e1, e2 in ev:
                flush.fill_(1)
                e0.record(stream)
                sense()
                e1.record(stream)
                recon()
                e2.record(stream)
            torch.cuda.synchronize()
            assert abcs.abcs_sync_status(h, s) == 0
            sm = statistics.median(e0.elapsed_time(e1) for e0, e1, _ in ev)
            rm = statistics.median(e1.elapsed_time(e2) for _, e1, e2 in ev)
            total = int(offsets[-1].item())
            px = n * nB * B * B
            step_bytes = 2 * px + 8 * total + 24 * n * nB + 4 * px   # image, y twice, counts+offsets twice, FP32 out
            out[f"{name}_r{r}"] = {"sense_ms": sm, "reconstruct_ms": rm,
                                   "Mpixel_per_s": px / ((sm + rm) * 1e-3) / 1e6,
                                   "measured_fraction": total / px,
                                   "step_frac_hbm": step_bytes / ((sm + rm) * 1e-3) / 1e9 / hbm_peak}
    return out


def single_image_latency(h, iters=10):
    """One 256x256 image (the single-image configuration: B = 16, BBV,
    r = 0.3): abcs_sense + abcs_reconstruct + abcs_ida (10 plain TI-DCT
    iterations) captured once into a CUDA graph and replayed; the median
    latency of a replay (image already on the device)."""
    import torch
    from paper_2001_09632_gb300 import abcs, synth
    H1 = W1 = 256
    plan = abcs.abcs_plan(H1, W1, B, SUBRATE, abcs.BBV)
    nB = plan["n_blocks"]
    d_img = torch.from_numpy(synth.gen_image(H1, W1, 77)[None]).cuda()
    counts = torch.empty(nB, dtype=torch.int32, device="cuda")
    offsets = torch.empty(nB + 1, dtype=torch.int64, device="cuda")
    coeffs = torch.empty(plan["M"], dtype=torch.float32, device="cuda")
    rec = torch.empty((1, H1, W1), dtype=torch.float32, device="cuda")
    x = torch.empty((1, H1, W1), dtype=torch.float32, device="cuda")
    out = {}
    for prec_name, prec in (("fp32", abcs.FP32), ("fp16x2", abcs.TC_FP16X2)):
        side = torch.cuda.Stream()

        def run(st):
            abcs.abcs_sense(h, d_img, 1, H1, W1, W1, H1 * W1, B, SUBRATE, abcs.BBV, prec, counts, offsets, coeffs,
                            plan["M"], None, st)
            abcs.abcs_reconstruct(h, counts, offsets, coeffs, 1, H1, W1, B, prec, rec, None, st)
            abcs.abcs_ida(h, counts, offsets, coeffs, 1, H1, W1, B, iters, DF, abcs.DEN_TIDCT, LAMBDA, None, x,
                          None, st)
        with torch.cuda.stream(side):
            for _ in range(3):                   # workspace grown, kernels loaded, before the capture
                run(side.cuda_stream)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            run(side.cuda_stream)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        ts = []
        for _ in range(20):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        assert abcs.abcs_sync_status(h) == 0
        out[prec_name] = {"ms_median": statistics.median(ts), "ms_min": min(ts)}
    out["workload"] = "1 x 256x256, B=16, BBV r 0.3: sense + IDCT + 10 plain IDA iterations (TI-DCT), CUDA graph replay"
    return out


def main():
    a = _args()
    if a.case:
        return run_case(a.case)
    if a.impl == "reference":
        return run_reference(a)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2001_09632_gb300 import abcs, synth
    from paper_2001_09632_gb300.pipeline import SenseReconPipeline

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    imgs = synth.gen_batch(N_IMG, H, W, SEED + rank * N_IMG)
    plan = abcs.abcs_plan(H, W, B, SUBRATE, abcs.BBV)
    nB = plan["n_blocks"]
    cap = N_IMG * plan["M"]
    h = abcs.abcs_create()
    d_img = torch.from_numpy(imgs).to(dev)
    counts = torch.empty(N_IMG * nB, dtype=torch.int32, device=dev)
    offsets = torch.empty(N_IMG * nB + 1, dtype=torch.int64, device=dev)
    coeffs = torch.empty(cap, dtype=torch.float32, device=dev)
    rec = torch.empty((N_IMG, H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream

    prec = abcs.PRECISIONS[a.precision]

    def step(p=None):
        p = prec if p is None else p
        abcs.abcs_sense(h, d_img, N_IMG, H, W, W, H * W, B, SUBRATE, abcs.BBV, p,
                        counts, offsets, coeffs, cap, None, s)
        abcs.abcs_reconstruct(h, counts, offsets, coeffs, N_IMG, H, W, B, p, rec, None, s)

    def timed_steps(K, p):
        """K steps of precision p, L2 flushed before each; per-call event times (ms)."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for i in range(K):
            flush.fill_(i & 0xFF)                  # evict L2 between timed steps
            e0, e1, e2 = ev[i]
            e0.record(stream)
            abcs.abcs_sense(h, d_img, N_IMG, H, W, W, H * W, B, SUBRATE, abcs.BBV, p,
                            counts, offsets, coeffs, cap, None, s)
            e1.record(stream)
            abcs.abcs_reconstruct(h, counts, offsets, coeffs, N_IMG, H, W, B, p, rec, None, s)
            e2.record(stream)
        torch.cuda.synchronize()
        return ([e0.elapsed_time(e1) for e0, e1, _ in ev], [e1.elapsed_time(e2) for _, e1, e2 in ev])

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    for _ in range(max(3, a.warmup)):
        step()
    assert abcs.abcs_sync_status(h, s) == 0
    total_coeffs = int(offsets[-1].item())

    clk = Clocks(local)
    time.sleep(0.3)
    K = a.steps
    barrier()
    t_start = time.time()
    sense_ms, recon_ms = timed_steps(K, prec)
    barrier()
    t_end = time.time()
    step_ms = sum(sense_ms) / K + sum(recon_ms) / K
    step_ms = max_over_ranks(step_ms)
    px = N_IMG * plan["N"]
    value = world * px / (step_ms * 1e-3) / 1e6

    # ---- the other precisions of the block DCT (same workload) ------------
    # with the mean PSNR / SSIM of the reconstructions (abcs_psnr_ssim) and
    # their difference from the FP32 path's
    qp = torch.empty(N_IMG, dtype=torch.float64, device=dev)
    qs = torch.empty_like(qp)

    def quality():
        abcs.abcs_psnr_ssim(h, rec, d_img, N_IMG, H, W, W, H * W, qp, qs, s)
        torch.cuda.synchronize()
        return float(qp.mean()), float(qs.mean())

    sweep = {}
    for name, p in abcs.PRECISIONS.items():
        for _ in range(3):
            step(p)
        sm, rm = timed_steps(min(K, 200), p)
        q_psnr, q_ssim = quality()
        sweep[name] = {"sense_ms": statistics.median(sm), "reconstruct_ms": statistics.median(rm),
                       "Mpixel_per_s": world * N_IMG * plan["N"] / ((statistics.median(sm) +
                                                                    statistics.median(rm)) * 1e-3) / 1e6,
                       "psnr": q_psnr, "ssim": q_ssim}
    for name in abcs.PRECISIONS:
        sweep[name]["dpsnr_vs_fp32"] = sweep[name]["psnr"] - sweep["fp32"]["psnr"]
        sweep[name]["dssim_vs_fp32"] = sweep[name]["ssim"] - sweep["fp32"]["ssim"]
    # the tcgen05 sensing kernel (basis in tensor memory), same workload
    os.environ["ABCS_SENSE_TC"] = "umma"
    for _ in range(3):
        step(prec)
    sm, rm = timed_steps(min(K, 200), prec)
    del os.environ["ABCS_SENSE_TC"]
    assert abcs.abcs_sync_status(h, s) == 0
    sweep["tensor_memory_sense"] = {
        "precision": a.precision, "sense_ms": statistics.median(sm),
        "kernel": "sense_umma_kernel (ABCS_SENSE_TC=umma; not the default)"}
    # the tcgen05 reconstruct kernel (basis images in tensor memory), same workload
    os.environ["ABCS_RECON_TC"] = "umma"
    for _ in range(3):
        step(prec)
    sm, rm = timed_steps(min(K, 200), prec)
    del os.environ["ABCS_RECON_TC"]
    assert abcs.abcs_sync_status(h, s) == 0
    sweep["tensor_memory_reconstruct"] = {
        "precision": a.precision, "reconstruct_ms": statistics.median(rm),
        "kernel": "recon_umma_kernel (ABCS_RECON_TC=umma; not the default)"}
    step(prec)
    torch.cuda.synchronize()

    # ---- IDA, plain TI-DCT denoiser --------------------------------------
    # the linear step in the step's precision (tensor cores unless FP32)
    x = torch.empty((N_IMG, H, W), dtype=torch.float32, device=dev)
    abcs.abcs_set_ida_precision(h, prec)
    for _ in range(2):
        abcs.abcs_ida(h, counts, offsets, coeffs, N_IMG, H, W, B, IDA_ITERS, DF, abcs.DEN_TIDCT,
                      LAMBDA, None, x, None, s)
    reps = 5
    ida_ms = []
    barrier()
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        abcs.abcs_ida(h, counts, offsets, coeffs, N_IMG, H, W, B, IDA_ITERS, DF, abcs.DEN_TIDCT,
                      LAMBDA, None, x, None, s)
        e1.record(stream)
        ida_ms.append((e0, e1))
    barrier()
    t_end2 = time.time()
    ida_ms = max_over_ranks(statistics.median(e0.elapsed_time(e1) for e0, e1 in ida_ms))
    abcs.abcs_set_ida_precision(h, abcs.FP32)
    assert abcs.abcs_sync_status(h, s) == 0
    lin = ida_linear_step(h, s, counts, offsets, coeffs, x, total_coeffs)

    # ---- end to end through the C ABI with host buffers -------------------
    h_img = torch.from_numpy(imgs).pin_memory()
    h_rec = torch.empty((N_IMG, H, W), dtype=torch.float32).pin_memory()
    Ke = K
    eve = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(Ke)]
    barrier()
    for i in range(Ke):
        flush.fill_(i & 0xFF)
        e0, e1 = eve[i]
        e0.record(stream)
        d_img.copy_(h_img, non_blocking=True)
        step()
        h_rec.copy_(rec, non_blocking=True)
        e1.record(stream)
    barrier()
    e2e_seq_ms = max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in eve) / Ke)
    # the same steps through SenseReconPipeline: copy-in of step j + 1, sense
    # + reconstruct of step j and copy-out of step j - 1 overlapped on three
    # streams (two device slots: a 200 MB working set, larger than L2)
    pipe = SenseReconPipeline(N_IMG, H, W, B, SUBRATE, abcs.BBV, prec)
    h_out = [torch.empty((N_IMG, H, W), dtype=torch.float32).pin_memory() for _ in range(2)]
    pipe.run([h_img] * 4, [h_out[j % 2] for j in range(4)])
    torch.cuda.synchronize()
    barrier()
    ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ep0.record(stream)
    pipe.run([h_img] * Ke, [h_out[j % 2] for j in range(Ke)])
    ep1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(ep0.elapsed_time(ep1) / Ke)
    assert torch.equal(h_out[(Ke - 1) % 2], rec.cpu()), "pipelined output differs from the plain sequence"
    pipe.close()
    # the same with the uint8 decoder output (a quarter of the bytes back)
    pipe8 = SenseReconPipeline(N_IMG, H, W, B, SUBRATE, abcs.BBV, prec, out_u8=True)
    h_out8 = [torch.empty((N_IMG, H, W), dtype=torch.uint8).pin_memory() for _ in range(2)]
    pipe8.run([h_img] * 4, [h_out8[j % 2] for j in range(4)])
    barrier()
    ep0.record(stream)
    pipe8.run([h_img] * Ke, [h_out8[j % 2] for j in range(Ke)])
    ep1.record(stream)
    barrier()
    e2e_u8_ms = max_over_ranks(ep0.elapsed_time(ep1) / Ke)
    pipe8.close()
    hbm_peak, peak_kind = _peaks()
    sweep_sub = subrate_sweep(h, prec, d_img, flush, hbm_peak)
    latency = single_image_latency(h)
    t_end3 = time.time()
    clocks = clk.stop(t_start, t_end3)
    extras = {}
    if not a.no_extras:
        del x
        extras["ida_batch"] = uneven_batch_ida(h, world, max_over_ranks, barrier)
        if rank == 0:
            extras["learned_vs_plain"] = {"video_1920x1088_dd_r025": video_learned_vs_plain(h),
                                          "images_512": images_learned_vs_plain(h)}
            extras["thi"] = thi_correlation(h)
            extras["damp_vs_ida"] = damp_vs_ida(h)
            extras["video_stream"] = video_stream(h)
            extras["bm3d_comparison"] = bm3d_comparison(h)

    if rank != 0:
        abcs.abcs_destroy(h)
        if world > 1:
            dist.destroy_process_group()
        return

    recon_bytes = 4 * total_coeffs + 12 * N_IMG * nB + 4 * px
    sense_bytes = px + 4 * total_coeffs + 12 * N_IMG * nB
    recon_avg = sum(recon_ms) / K
    sense_avg = sum(sense_ms) / K
    # the roofline object describes the longer of the step's two calls: the
    # sensing call (pilot + allocation kernel, then the sensing kernel) or
    # the reconstruct kernel; both are in `kernels`
    sense_frac = sense_bytes / (sense_avg * 1e-3) / 1e9 / hbm_peak
    recon_frac = recon_bytes / (recon_avg * 1e-3) / 1e9 / hbm_peak
    if sense_avg >= recon_avg:
        dom = {"kernel": "abcs_sense: bbv_image_kernel (pilot + allocation) then "
                         + ("sense_tc_kernel" if prec != abcs.FP32 else "sense_pack_kernel<16>"),
               "bytes": sense_bytes, "ms": sense_avg, "traffic": TRAFFIC.get("sense_" + a.precision),
               "bytes_are": "uint8 image read once + packed FP32 coefficients written + counts and offsets "
                            "(the pilot's reads of the same pixels are L2 hits and not counted)"}
    else:
        dom = {"kernel": "recon_tc_kernel" if prec != abcs.FP32 else "recon_kernel<16>",
               "bytes": recon_bytes, "ms": recon_avg, "traffic": TRAFFIC.get("recon_" + a.precision),
               "bytes_are": "packed FP32 coefficients + counts and offsets read, FP32 image written"}
    achieved = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world, "steps": K,
        "warmup": a.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp16x2": "f16x2 (hi+lo split, FP32 accumulate)", "bf16x2": "bf16x2 (hi+lo split, FP32 accumulate)", "bf16": "bf16 (FP32 accumulate)"}[a.precision], "data": "synthetic",
        "config": {"workload": "64 x 512x512 uint8 greyscale (seeded shapes + 1/f^2 texture), "
                               "B=16, AL-DCT-BBV, subrate 0.3: sense + IDCT reconstruct",
                   "precision": a.precision,
                   "value_is": "sense+reconstruct Mpixel/s", "l2": "flushed between timed steps (512 MB write)",
                   "measurements_per_step": total_coeffs, "parallelism": f"replicas x{world}"},
        "roofline": {"kernel": dom["kernel"], "bound": "hbm", "achieved": achieved,
                     "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "peak_kind": peak_kind, "traffic": dom["traffic"],
                     "traffic_source": "DRAM read + write bytes per call of these kernels on this workload "
                                       "in an ncu capture (cold caches; the step's outputs are still in "
                                       "L2 when a kernel ends, so they can read below the algorithmic bytes)",
                     "algorithmic_bytes_per_launch": dom["bytes"], "algorithmic_bytes_are": dom["bytes_are"],
                     "ms_per_launch": dom["ms"]},
        "kernels": {"sense_ms": sense_avg, "reconstruct_ms": recon_avg,
                    "sense_GBps_algorithmic": sense_bytes / (sense_avg * 1e-3) / 1e9,
                    "sense_frac_hbm": sense_frac, "reconstruct_frac_hbm": recon_frac,
                    "sense_plus_recon_frac_hbm": (sense_bytes + recon_bytes) / (step_ms * 1e-3) / 1e9 / hbm_peak,
                    "step_bytes_per_pixel": (sense_bytes + recon_bytes) / px},
        "subrate_sweep": sweep_sub,
        "single_image_latency": latency,
        "precision_sweep": sweep,
        "ida": {"value": world * px * IDA_ITERS / (ida_ms * 1e-3) / 1e6, "unit": "Mpixel*iter/s",
                "iters": IDA_ITERS, "denoiser": "tidct", "lambda": LAMBDA, "damping": DF,
                "linear_step": a.precision, "ms_per_call": ida_ms},
        "ida_linear": dict(lin, hbm_floor_us=lin["bytes_per_iteration"] / hbm_peak / 1e3,
                           fp16x2_frac_hbm=lin["bytes_per_iteration"] / (lin["fp16x2_us_per_iteration"] * 1e-6)
                           / 1e9 / hbm_peak),
        "e2e": {"value": world * px / (e2e_ms * 1e-3) / 1e6, "unit": "Mpixel/s",
                "h2d_bytes_per_step": int(h_img.numel()), "d2h_bytes_per_step": int(h_rec.numel() * 4),
                "ms_per_step": e2e_ms,
                "how": "SenseReconPipeline: pinned host images -> device -> abcs_sense + abcs_reconstruct -> "
                       "pinned host FP32 reconstructions, copy-in / compute / copy-out of consecutive steps "
                       "overlapped on three streams; K steps between two events, no L2 flush (two device "
                       "slots, 200 MB working set)",
                "sequential": {"value": world * px / (e2e_seq_ms * 1e-3) / 1e6, "ms_per_step": e2e_seq_ms,
                               "how": "one stream, L2 flushed before each step (outside the timed region)"},
                "uint8_output": {"value": world * px / (e2e_u8_ms * 1e-3) / 1e6, "ms_per_step": e2e_u8_ms,
                                 "d2h_bytes_per_step": int(h_img.numel()),
                                 "how": "the same pipeline, reconstruction rounded to uint8 on the device"}},
        **extras,
        # per timed step: the BBV pilot with its fused allocation, the sensing
        # kernel and the reconstruct kernel (the L2 flush runs before the step)
        "gpu_launches": 3 * K,
        "clocks": clocks,
    }
    if world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(imgs)
        per_img = H * W / (line["cpu_baseline"]["value"] * 1e6)
        line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(imgs, per_img)
    abcs.abcs_destroy(h)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
