#!/usr/bin/env python
"""Benchmark of the Batch-FPM mini-batch step on one or more GB300s.

Workload: the paper-scale multi-parameter reconstruction (1024^2 object
spectrum, 256^2 low-res images, 15x15 = 225 LEDs, batch 16, object, Zernike
pupil, defocus, LED intensities and LED offsets all learned), on synthetic
data shaped like the paper's simulation (Section 3.1).

A step is one pass of the whole hot path over one batch: the fused per-LED
forward model + adjoint kernel, then the batch-ordered gradient gather with
Adam. The metric is LED forward+backward updates per second (batch size /
step time), summed over ranks (one independent job per GPU, weak scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl engine|reference]

Prints one JSON line on rank 0.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LED fwd+bwd updates/s at 1024² ROI, 225 LEDs; %HBM roofline; serve p50/p99 TTC"
UNIT = "LED-updates/s"
WORKLOAD = ("c2_multiparam_1024: 1024x1024 object spectrum, 256x256 images, 15x15=225 LEDs "
            "(pitch 12 px, +-0.5 px jitter), pupil r=50 px + Noll 2..15 aberrations, z=15 um, "
            "gamma U(0.8,1.2), Poisson 2000/20 photons + read noise 2; batch 16; all parameters learned")
FLUSH_BYTES = 256 << 20        # > 129 MB L2: cleared before every timed step
L2_NOTE = "L2 flushed (256 MB device memset) before every timed step"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _peak_bf16():
    """Measured dense BF16 tensor throughput (burst: a kernel timed on its own)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


# --------------------------------------------------------------------------
# workload
# --------------------------------------------------------------------------

def workload(seed_shift: int = 0):
    from synth import recipes as S
    c = S.config("c2")
    if seed_shift:
        c = c.with_(seed=c.seed + 1000 * seed_shift)
    nominal, truth = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)
    return c, nominal, truth


def support_pixels(R: float) -> int:
    """Lattice points of the anti-aliased pupil support |p| < R + 1/2."""
    r = int(math.ceil(R + 1))
    p = np.arange(-r, r + 1)
    return int(np.sum(np.hypot(p[:, None], p[None, :]) < R + 0.5))


def union_pixels(nominal, R: float, N: int) -> int:
    """|union of LED supports| on the spectrum grid (the region where Adam acts)."""
    mask = np.zeros((N, N), bool)
    r = int(math.ceil(R + 1))
    p = np.arange(-r, r + 1)
    disk = np.hypot(p[:, None], p[None, :]) < R + 0.5
    for n in np.rint(nominal).astype(int):
        y0, x0 = N // 2 + n[0] - r, N // 2 + n[1] - r
        mask[y0:y0 + 2 * r + 1, x0:x0 + 2 * r + 1] |= disk
    return int(mask.sum())


def led_flops_per_led(m: int, W: int, D: int) -> float:
    """Algorithmic FP32 flops of one LED in the per-LED kernel: 2 (W + m) m-point
    transforms at 5 m log2 m, the residual (15 per image pixel) and the per-pixel
    pupil (40) and box-gradient (95) work on the support D."""
    return 2 * (W + m) * 5 * m * math.log2(m) + 15 * m * m + 135 * D


def make_stack_gpu(c, truth):
    """Clean intensities from the engine's forward model at the truth, plus the camera noise."""
    from paper_2408_13782_gb300 import Engine
    from synth import recipes as S
    eng = Engine(c.m, c.s, truth, c.R, c.lambda_um, c.dk_per_um, c.edge)
    eng.set_object_field(S.make_object(c.N, c.seed))
    eng.set(zernike=S.zernike_coeffs(c.zernike_sigma, c.seed), defocus=c.z_um,
            gamma=S.led_gamma(c.n_leds, *c.gamma_range, c.seed), offset=truth - np.rint(truth))
    I = np.concatenate([eng.forward(np.arange(k, min(k + 32, c.n_leds))) for k in range(0, c.n_leds, 32)])
    eng.close()
    nominal = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)[0]
    bright = S.brightfield_mask(nominal, c.R)
    nz = c.noise
    return S.add_noise(I, bright, nz["bf_mean"], nz["df_mean"], nz["read_sigma"], c.seed).astype(np.float32)


def full_batches(n: int, B: int, n_steps: int, seed: int, first_epoch: int = 0) -> np.ndarray:
    """n_steps consecutive full batches of the random schedule (Eq. 13-14): each pass
    is a fresh permutation; its short tail batch is left out of the timed steps."""
    from synth import recipes as S
    out, e = [], first_epoch
    while len(out) < n_steps:
        perm = S.epoch_permutation(n, seed, e)
        out.extend(perm[k:k + B] for k in range(0, n - B + 1, B))
        e += 1
    return np.stack(out[:n_steps]).astype(np.int32)


def kernel_source_hash() -> str:
    import hashlib
    m = hashlib.sha256()
    for f in ("led.cu", "device.cuh", "pixel.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_2408_13782_gb300", "csrc", f), "rb") as fh:
            m.update(fh.read())
    return m.hexdigest()[:16]


def led_traffic_from_profile():
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged since
    (led.cu and the headers it includes hash to the recorded value)."""
    path = os.path.join(ROOT, "profiles", "led_kernel_c2_1024_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    if kv.get("source_hash") != kernel_source_hash():
        return None
    return float(kv["bytes_per_launch"])


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi polled every 20 ms with timestamps; summary() reports the samples
    that fall in a given host-time window (the timed region) and in the whole run."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _parse(ln):
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 8:
            return None
        try:
            sm, smax = float(parts[1]), float(parts[2])
        except ValueError:
            return None
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        return sm, smax, {nm for nm, v in zip(names, parts[4:8]) if v.lower().startswith("active")}

    def summary(self, t0=None, t1=None, margin=0.025):
        rows = [(t, self._parse(ln)) for t, ln in self.lines]
        rows = [(t, r) for t, r in rows if r is not None]
        inside = [r for t, r in rows if t0 is not None and t0 - margin <= t <= t1 + margin]
        use = inside if inside else [r for _, r in rows]
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"], "samples": 0}
        reasons = set()
        for r in use:
            reasons |= r[2]
        return {"sm_mhz": statistics.median(r[0] for r in use), "sm_max_mhz": use[-1][1],
                "reasons": sorted(reasons), "samples": len(use), "samples_in_timed_region": len(inside),
                "samples_in_run": len(rows),
                "window": "the timed steps" if inside else
                          "the run (identical flushed steps before and after the timed ones; none of the 20 ms samples "
                          "fell inside the timed region)"}


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, single thread
# --------------------------------------------------------------------------

def cpu_worker(stack_path: str, sample_s: float, leds_per_step: int, max_steps: int, threads: int = 1):
    """Runs oracle steps on the workload in a child process: one thread, or (threads > 1)
    the oracle's 2-D FFTs through scipy.fft with that many workers and numpy's BLAS
    threads left at that count (the oracle's arithmetic is unchanged)."""
    if threads > 1:
        import scipy.fft as sfft
        np.fft.fft2 = lambda x, *a, **k: sfft.fft2(x, *a, workers=threads, **k)
        np.fft.ifft2 = lambda x, *a, **k: sfft.ifft2(x, *a, workers=threads, **k)
    import oracle as orc
    c, nominal, truth = workload()
    I = np.load(stack_path)
    g = orc.Geometry(c.N, c.m, nominal, c.R, c.edge, c.lambda_um, c.dk_per_um)
    rec = orc.Reconstruction(g, I, orc.Hparams(lr=dict(c.lr), learn=c.learn))
    sched = full_batches(c.n_leds, c.B, max_steps, c.seed)
    t0 = time.perf_counter()
    n_led, steps = 0, 0
    while steps < max_steps:
        b = sched[steps][:leds_per_step]
        rec.step(b)
        n_led += len(b)
        steps += 1
        if time.perf_counter() - t0 >= sample_s:
            break
    dt = time.perf_counter() - t0
    print(json.dumps({"updates": n_led, "seconds": dt, "steps": steps}))


def run_cpu_child(stack, sample_s: float, leds_per_step: int, max_steps: int, threads: int = 1):
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "stack.npy")
        np.save(path, stack)
        t = str(threads)
        env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t,
                   CUDA_VISIBLE_DEVICES="")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", path,
                            "--cpu-sample-s", str(sample_s), "--cpu-leds", str(leds_per_step),
                            "--cpu-max-steps", str(max_steps), "--cpu-threads", t],
                           capture_output=True, text=True, env=env, timeout=1800)
        if r.returncode != 0:
            raise RuntimeError("CPU baseline worker failed:\n" + r.stderr[-2000:])
        return json.loads(r.stdout.strip().splitlines()[-1])


# --------------------------------------------------------------------------
# serving: continuous batching of uneven reconstructions vs the same jobs serially
# --------------------------------------------------------------------------

def serving_jobs(n_jobs: int, rate_hz: float, seed: int, shape=None):
    """Seeded Poisson arrivals; ROI from {256, 512, 1024, 2048}^2 at upsample 4, grids
    {7, 11, 15}^2, the 64-px recipe (hard pupil, aberration-free, noise-free) per job.
    shape=(N, grid): every job of that shape instead (a homogeneous request stream)."""
    from paper_2408_13782_gb300 import Engine
    from paper_2408_13782_gb300 import serve as sv
    from synth import recipes as S
    rng = np.random.default_rng([seed, 40])
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_jobs))
    jobs = []
    for k in range(n_jobs):
        N = int(rng.choice([256, 512, 1024, 2048]))
        grid = int(rng.choice([7, 11, 15]))
        if shape is not None:
            N, grid = shape
        c = S.serving_job_config(N, grid, seed * 1000 + k)
        nominal, truth = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)
        eng = Engine(c.m, c.s, truth, c.R, c.lambda_um, c.dk_per_um, c.edge)
        eng.set_object_field(S.make_object(c.N, c.seed))
        stack = np.concatenate([eng.forward(np.arange(i, min(i + 64, c.n_leds))) for i in range(0, c.n_leds, 64)])
        eng.close()
        desc = sv.job_desc(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge, batch=c.B,
                           max_epochs=c.epochs, rel_tol=1e-4, seed=c.seed, lr=dict(c.lr))
        jobs.append((desc, stack, float(t[k]), N, grid))
    return jobs


def serving_run(jobs, budget: int, max_active: int, admission: str = "arrival", grouping: str = "config"):
    from paper_2408_13782_gb300 import serve as sv
    srv = sv.Server(budget, max_active, admission, grouping)
    ids, st, wall = sv.run_arrivals(srv, [(d, s, t) for d, s, t, _, _ in jobs])
    stats = srv.stats()
    srv.close()
    ttc = np.array([x["t_done"] - x["t_submit"] for x in st])
    upd = sum(x["led_updates"] for x in st)
    span = max(x["t_done"] for x in st) - min(x["t_submit"] for x in st)
    return {"p50_ttc_s": float(np.percentile(ttc, 50)), "p99_ttc_s": float(np.percentile(ttc, 99)),
            "mean_ttc_s": float(ttc.mean()), "led_updates_per_s": upd / span, "grouping": grouping,
            "jobs_done": int(sum(x["state"] == sv.JOB_DONE for x in st)),
            "epochs_median": float(np.median([x["epochs"] for x in st])), "makespan_s": span,
            "admission": admission, "max_active": max_active, "server": stats}


def rgb_section(budget: int, N=512, grid=11, seed=17):
    """Section 3.3's colour workflow: three wavelengths of one field of view as three
    jobs submitted together (co-scheduled) against the three run one after another."""
    from paper_2408_13782_gb300 import Engine
    from paper_2408_13782_gb300 import serve as sv
    from synth import recipes as S
    jobs = []
    for c in S.rgb_job_configs(N, grid, seed):
        nominal, truth = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)
        eng = Engine(c.m, c.s, truth, c.R, c.lambda_um, c.dk_per_um, c.edge)
        eng.set_object_field(S.make_object(c.N, c.seed))
        stack = np.concatenate([eng.forward(np.arange(i, min(i + 64, c.n_leds))) for i in range(0, c.n_leds, 64)])
        eng.close()
        desc = sv.job_desc(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge, batch=c.B,
                           max_epochs=c.epochs, rel_tol=1e-4, seed=c.seed, lr=dict(c.lr))
        jobs.append((desc, stack, 0.0, N, grid))
    out = {"what": f"three channels (470/523/623 nm) of one {N}^2 field, {grid}x{grid} LEDs, submitted together; "
                   "time until all three are done", "wavelengths_um": list(S.RGB_WAVELENGTHS_UM)}
    for name, act in (("co_scheduled", 3), ("serial", 1)):
        r = serving_run(jobs, budget, max_active=act)
        out[name] = {"all_done_s": r["makespan_s"], "led_updates_per_s": r["led_updates_per_s"],
                     "epochs_median": r["epochs_median"]}
    return out


def serving_section(n_jobs=100, rate_hz=40.0, seed=5):
    import torch
    jobs = serving_jobs(n_jobs, rate_hz, seed)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.6 * free)
    runs = {"continuous": serving_run(jobs, budget, max_active=64),
            "continuous_smallest_first": serving_run(jobs, budget, max_active=64, admission="smallest"),
            "continuous_8_active": serving_run(jobs, budget, max_active=8),
            "continuous_group_by_size": serving_run(jobs, budget, max_active=64, grouping="size"),
            "continuous_sizes_mixed": serving_run(jobs, budget, max_active=64, grouping="mixed"),
            "serial": serving_run(jobs, budget, max_active=1)}
    same = serving_jobs(16, 1000.0, seed + 1, shape=(512, 11))
    same_serving = serving_run(same, budget, max_active=64)
    same_serial = serving_run(same, budget, max_active=1)
    mix = {}
    for _, _, _, N, g in jobs:
        mix[f"{N}^2/{g}x{g}"] = mix.get(f"{N}^2/{g}x{g}", 0) + 1
    return {"what": f"{n_jobs} jobs, Poisson arrivals {rate_hz:g}/s, ROI from {{256,512,1024,2048}}^2 at "
                    "upsample 4, LED grids {7,11,15}^2, stop at relative epoch-loss change < 1e-4 or 40 epochs; "
                    "continuous batching (jobs admitted by device-memory footprint, overlapping; jobs with "
                    "the same steps per epoch stepped together in one launch per step, grouped by kernel "
                    "configuration (default), by low-res size, or with sizes 64/128/256 mixed in one launch; admission "
                    "in arrival order or smallest expected work first; at most 64 or 8 resident) vs the same "
                    "jobs one at a time (FCFS) on the same GPU",
            "mix_counts": mix, "hbm_budget_bytes": budget, **runs,
            "same_shape": {"what": "16 jobs of 512^2 / 11x11 arriving in a burst (Poisson 1000/s)",
                           "continuous": same_serving, "serial": same_serial},
            "rgb": rgb_section(budget)}


# --------------------------------------------------------------------------
# distributed helpers (torchrun: one rank per GPU, independent jobs)
# --------------------------------------------------------------------------

def gemm_mma_flops(m: int, W: int, split: bool) -> float:
    """Tensor-core FLOPs of one LED in the DFT-as-contraction form (padded shapes
    as issued: box W padded to a multiple of 16, row tiles and column chunks of
    at most 128, complex contractions as real ones of twice the depth)."""
    Wp = -(-W // 16) * 16
    YT = X = min(m, 128)
    ntile, nchunk = m // YT, m // X
    macs = ntile * (2 * 128 * Wp * 2 * Wp                      # step 1, real and imaginary blocks
                    + nchunk * (128 * 2 * X * 2 * Wp)          # step 2
                    + nchunk * (2 * 128 * YT * 2 * X)          # step 3
                    + 128 * 2 * Wp * 2 * YT)                   # step 4
    return 2.0 * macs * (3 if split else 1)


def measure_tf32_peak(dev, n=8192, reps=5):
    """Dense TF32 tensor throughput of this GPU: cuBLAS FP32 GEMM with TF32 allowed
    (torch.matmul, n^3), best of reps, CUDA events; TFLOP/s."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        a = torch.randn(n, n, device=dev)
        b = torch.randn(n, n, device=dev)
        torch.matmul(a, b)
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        del a, b
        return 2.0 * n ** 3 / best / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def tensor_forms_section(c, nominal, stack, flush, n_steps=40):
    """The per-LED kernel in each tensor-core DFT form on the same workload and
    schedule (L2 flushed before every step): kernel time and tensor throughput
    against the measured BF16 peak (BF16 forms) and the TF32 peak measured here
    (TF32 forms)."""
    import torch
    from paper_2408_13782_gb300 import Engine
    peak_bf16, kind = _peak_bf16()
    peak_tf32 = measure_tf32_peak(torch.device("cuda"))
    box = 2 * (int(np.floor(c.R + 0.5 + np.sqrt(2.0))) + 1) + 1
    out = {}
    sched = full_batches(c.n_leds, c.B, n_steps + 3, c.seed, first_epoch=500)
    for form in ("bf16", "bf16x3", "tf32", "tf32x3"):
        eng = Engine(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge)
        eng.set_hparams(lr=dict(c.lr), learn=c.learn, precision=form)
        eng.load(stack, init=True)
        eng.run(sched[:3], losses=False)
        led_ms, upd_ms, step_ms = eng.profile_run(sched[3:], flush=flush)
        eng.close()
        flops = c.B * gemm_mma_flops(c.m, box, form.endswith("x3"))
        t = float(np.mean(led_ms)) / 1e3
        peak = peak_bf16 if form.startswith("bf16") else peak_tf32
        out[form] = {"led_kernel_ms": t * 1e3, "update_kernel_ms": float(np.mean(upd_ms)),
                     "led_updates_per_s": c.B / (float(np.mean(step_ms)) / 1e3),
                     "tensor_tflops": flops / t / 1e12, "peak_tflops": peak,
                     "frac": flops / t / 1e12 / peak, "mma_flops_per_launch": flops}
    out["peak_source"] = {"bf16": f"{kind} (MEASURED_PEAKS.json)", "tf32": "measured in this run (cuBLAS TF32 GEMM 8192^3)"}
    out["peak_tf32_tflops"] = peak_tf32
    return out


def amplitude_psnr(O, o_true, s: int) -> float:
    """PSNR (dB, peak 1) of the reconstructed amplitude against the true one, after the best
    complex scale (the reconstruction is defined up to a global phase, and the intensity
    factors can trade a global scale with the object). O: centred spectrum, 1/s^2 scaled."""
    o = np.fft.ifft2(np.fft.ifftshift(np.asarray(O, np.complex128))) * (s * s)
    a = np.vdot(o, o_true) / np.vdot(o, o)
    err = np.abs(a * o) - np.abs(o_true)
    return float(10.0 * np.log10(1.0 / np.mean(err * err)))


def batch_sweep_section(c, nominal, stack, epochs=20, every=4, batches=(1, 4, 16, 64, 225)):
    """Reconstruction quality against time for several batch sizes on the same noisy stack
    (Fig. 4-style): B = 1 is the sequential mode (Eq. 7), B = n_leds the global one (Eq. 6).
    Each epoch is one pass in a fresh random order (Eq. 14), its full batches as one CUDA
    graph and the short tail batch on its own; wall-clock time with the device synchronised."""
    import torch

    from paper_2408_13782_gb300 import Engine
    from synth import recipes as S
    o_true = S.make_object(c.N, c.seed)
    out = {"what": f"{epochs} epochs per batch size, Adam as in the headline workload, amplitude PSNR "
                   "(peak 1) of the reconstructed object against the synthetic truth after the best "
                   "complex scale, every " + str(every) + " epochs; wall-clock seconds of the epochs",
           "runs": {}}
    for B in batches:
        eng = Engine(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge)
        eng.set_hparams(lr=dict(c.lr), learn=c.learn)
        eng.load(stack, init=True)
        sched = S.schedule(c.n_leds, B, epochs, c.seed)
        nb = -(-c.n_leds // B)
        t_run, curve = 0.0, [(0, 0.0, amplitude_psnr(eng.get()["object"], o_true, c.s))]
        for e in range(epochs):
            ep = sched[e * nb:(e + 1) * nb]
            full = [b for b in ep if len(b) == B]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if full:
                eng.run(np.stack(full), losses=False)
            for b in ep:
                if len(b) != B:
                    eng.step(b, loss=False)
            torch.cuda.synchronize()
            t_run += time.perf_counter() - t0
            if (e + 1) % every == 0:
                curve.append((e + 1, t_run, amplitude_psnr(eng.get()["object"], o_true, c.s)))
        eng.close()
        out["runs"][str(B)] = {"epoch_s_psnr_db": [[k, round(t, 6), round(p, 3)] for k, t, p in curve],
                               "steps_per_epoch": nb, "final_psnr_db": round(curve[-1][2], 3),
                               "seconds": round(t_run, 6)}
    return out


def autograd_section(dev, reps=3):
    """Recompute-in-backward vs stored fields through the torch.autograd.Function
    on the 2048^2 / 512^2, 15 x 15-LED instance at batch 64: device memory held
    by torch across forward + backward and the time of the pair."""
    import torch
    from paper_2408_13782_gb300 import Engine
    from paper_2408_13782_gb300.autograd import fpm_intensities
    from synth import recipes as S
    c = S.config("c3_mem")
    nominal, truth = S.led_grid(c.grid, c.pitch, c.jitter, c.seed)
    eng = Engine(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge)
    rng = np.random.default_rng(c.seed)
    O = torch.tensor((S.make_object(c.N, c.seed)).astype(np.complex64), device=dev)
    leaves = [O, torch.tensor(S.zernike_coeffs(c.zernike_sigma, c.seed), dtype=torch.float32, device=dev),
              torch.tensor([c.z_um], dtype=torch.float32, device=dev),
              torch.ones(c.n_leds, dtype=torch.float32, device=dev),
              torch.zeros((c.n_leds, 2), dtype=torch.float32, device=dev)]
    leaves = [x.requires_grad_(True) for x in leaves]
    idx = rng.permutation(c.n_leds)[:c.B].astype(np.int32)
    w = torch.tensor(rng.normal(size=(c.B, c.m, c.m)).astype(np.float32), device=dev)
    res = {"workload": f"{c.N}^2 object, {c.m}^2 images, {c.n_leds} LEDs, batch {c.B}",
           "field_bytes": c.B * c.m * c.m * 8}
    for store in (False, True):
        for x in leaves:
            x.grad = None
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats(dev)
        base = torch.cuda.memory_allocated(dev)
        times = []
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            I = fpm_intensities(eng, idx, *leaves, store_fields=store)
            (I * w).sum().backward()
            e1.record()
            torch.cuda.synchronize()
            if r:
                times.append(e0.elapsed_time(e1))
            del I
            for x in leaves:
                x.grad = None
        res["store" if store else "recompute"] = {
            "peak_torch_bytes": int(torch.cuda.max_memory_allocated(dev) - base),
            "fwd_bwd_ms": float(np.median(times))}
    eng.close()
    return res


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("FPM_BENCH_BACKEND", "nccl")
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg, device=None):
    if pg is not None:
        if device is not None:
            pg.barrier(device_ids=[device])
        else:
            pg.barrier()


def allreduce_max(pg, x: float, device) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------
# engine arm
# --------------------------------------------------------------------------

def engine_arm(args):
    import torch

    import __graft_entry__
    from paper_2408_13782_gb300 import Engine

    world, rank, local, pg = dist_setup()
    assert torch.cuda.is_available(), "the engine arm needs a CUDA GPU"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()

    c, nominal, truth = workload(seed_shift=rank)
    stack = make_stack_gpu(c, truth)
    eng = Engine(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge)
    eng.set_hparams(lr=dict(c.lr), learn=c.learn)
    eng.load(stack, init=True)
    K, W, B = args.steps, args.warmup, c.B
    sched = full_batches(c.n_leds, B, W + 2 * K, c.seed)
    eng.run(sched[:W], losses=False)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    barrier(pg, local)
    # the timed region: K steps, each bracketed by events on the engine's stream,
    # the update kernel launched early by programmatic dependent launch as in run().
    # The clock sampler polls every 20 ms; identical flushed steps run untimed for
    # about 0.3 s before the timed ones so that a short timed region still has
    # samples of the same load around it
    pre = full_batches(c.n_leds, B, 2000, c.seed, first_epoch=2000)
    with ClockSampler(local) as clk:
        t_pre, k_pre = time.time(), 0
        while time.time() - t_pre < 0.3 and k_pre + 200 <= len(pre):
            eng.profile_run(pre[k_pre:k_pre + 200], flush=flush, per_kernel=False)
            k_pre += 200
        torch.cuda.synchronize()
        t_timed0 = time.time()
        _, _, step_ms = eng.profile_run(sched[W:W + K], flush=flush, per_kernel=False)
        torch.cuda.synchronize()
        t_timed1 = time.time()
        time.sleep(0.05)
    clocks = clk.summary(t_timed0, t_timed1)
    clocks["pre_roll_steps"] = k_pre
    barrier(pg, local)
    # the per-kernel split (kernels back to back, events between them) on the next K steps
    led_ms, upd_ms, split_ms = eng.profile_run(sched[W + K:], flush=flush)
    # context only: the production path (one CUDA graph of K steps, no flush, L2 warm)
    sched2 = full_batches(c.n_leds, B, K, c.seed, first_epoch=1000)
    eng.run(sched2, losses=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    eng.run(sched2, losses=False)
    e1.record()
    torch.cuda.synchronize()
    warm_ms = e0.elapsed_time(e1)
    total_ms = float(np.sum(step_ms))
    total_ms_max = allreduce_max(pg, total_ms, dev)
    value = world * K * B / (total_ms_max / 1e3)

    # roofline of the dominant kernel (the fused per-LED kernel): algorithmic bytes
    # against the measured copy bandwidth, and algorithmic FP32 flops against the
    # measured FMA throughput of this GPU
    D = support_pixels(c.R)
    A = union_pixels(nominal, c.R, c.N)
    led_bytes = B * (4 * c.m * c.m + 16 * D)            # image read + O on support + gradient box
    step_bytes = B * (4 * c.m * c.m + 24 * D) + 48 * A  # + gradient read and the Adam state of O
    led_avg_s = float(np.mean(led_ms)) / 1e3
    peak, peak_kind = _peaks()
    achieved = led_bytes / led_avg_s / 1e9
    traffic = led_traffic_from_profile()
    box = 2 * (int(np.floor(c.R + 0.5 + np.sqrt(2.0))) + 1) + 1
    led_flops = B * led_flops_per_led(c.m, box, D)
    from paper_2408_13782_gb300.engine import probe_fp32_fma
    fp32_peak, _ = probe_fp32_fma()
    alu_achieved = led_flops / led_avg_s / 1e12
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": total_ms_max / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": B * world, "l2": L2_NOTE,
                   "parallelism": f"independent job per GPU x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "led_kernel (fused per-LED forward + adjoint, m=256)",
                     "peak_source": peak_kind, "algorithmic_bytes_per_launch": led_bytes,
                     "avg_launch_ms": led_avg_s * 1e3,
                     "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                             "peak_source": peak_kind},
                     "alu": {"achieved": alu_achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                             "frac": alu_achieved / fp32_peak, "peak_source": "measured (fpm_probe_fp32_fma, this run)",
                             "algorithmic_flops_per_launch": led_flops,
                             "flops": "per LED 2 (W + m) transforms x 5 m log2 m + 15 m^2 (residual) + "
                                      "135 |D| (pupil 40, box gradient 95 per support pixel)"}},
        "step_hbm_roofline": {"algorithmic_bytes_per_step": step_bytes,
                              "achieved_gbs": step_bytes / (total_ms / K / 1e3) / 1e9,
                              "frac": step_bytes / (total_ms / K / 1e3) / 1e9 / peak},
        "kernel_ms": {"led_kernel": float(np.mean(led_ms)), "update_kernel": float(np.mean(upd_ms)),
                      "step_back_to_back": float(np.mean(split_ms)),
                      "what": "a second pass of K steps with events between the two kernels (no overlap)"},
        "graph_l2_warm": {"value": K * B / (warm_ms / 1e3), "ms_per_step": warm_ms / K,
                          "what": "context: fpm_run of K steps as one CUDA graph, no flush, timed with "
                                  "CUDA events on the caller's stream"},
        "gpu_launches": 2 * K,
        "clocks": clocks,
    }

    # end to end through the C ABI with host buffers: a whole job (load, 20 passes, read back)
    eng.close()   # the timed engine and its K-step graph are no longer needed
    e2e_steps = full_batches(c.n_leds, B, 14 * c.epochs, c.seed)
    pinned = torch.from_numpy(stack).pin_memory()
    # the job's result lands in pinned host buffers that a serving process would reuse
    res_host = {"object": torch.empty((c.N, c.N, 2), dtype=torch.float32).pin_memory(),
                "zernike": torch.empty(14, dtype=torch.float32).pin_memory(),
                "defocus": torch.empty(1, dtype=torch.float32).pin_memory(),
                "gamma": torch.empty(c.n_leds, dtype=torch.float32).pin_memory(),
                "offset": torch.empty((c.n_leds, 2), dtype=torch.float32).pin_memory()}
    eng2 = Engine(c.m, c.s, nominal, c.R, c.lambda_um, c.dk_per_um, c.edge)
    eng2.set_hparams(lr=dict(c.lr), learn=c.learn)
    eng2.load(pinned, init=True)
    eng2.run(e2e_steps, losses=True)          # warm: graphs built, caches populated
    torch.cuda.synchronize()
    barrier(pg, local)
    t0 = time.perf_counter()
    eng2.load(pinned, init=True)
    losses = eng2.run(e2e_steps, losses=True)
    out = eng2.get(out=res_host)
    t1 = time.perf_counter()
    barrier(pg, local)
    e2e_s = allreduce_max(pg, t1 - t0, dev)
    n_e2e = len(e2e_steps)
    result["e2e"] = {"value": world * n_e2e * B / e2e_s, "unit": UNIT,
                     "h2d_bytes_per_step": (stack.nbytes + e2e_steps.nbytes + 8) / n_e2e,
                     "d2h_bytes_per_step": (losses.nbytes + c.N * c.N * 8 + 4 * (15 + 3 * c.n_leds)) / n_e2e,
                     "what": f"one job of {n_e2e} steps: stack upload from pinned host memory, object "
                             "initialisation, the steps, per-step losses and the final state read back"}
    assert np.all(np.isfinite(losses)) and bool(torch.isfinite(out["object"]).all())

    if rank == 0 and world == 1 and not args.no_serving:
        result["serving"] = serving_section()
    if rank == 0 and world == 1 and not args.no_variants:
        result["tensor_core_forms"] = tensor_forms_section(c, nominal, stack, flush)
        result["autograd_memory"] = autograd_section(dev)
    if rank == 0 and world == 1 and not args.no_sweep:
        result["batch_sweep"] = batch_sweep_section(c, nominal, stack)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = run_cpu_child(stack, args.cpu_sample_s, B, 10_000)
        result["cpu_baseline"] = {"value": r["updates"] / r["seconds"], "unit": UNIT, "cores": 1,
                                  "kind": "oracle",
                                  "sample": f"{r['steps']} oracle steps of 16 LEDs on this workload "
                                            f"({r['seconds']:.1f} s, FP64 numpy, 1 thread)"}
        ncpu = os.cpu_count() or 1
        r = run_cpu_child(stack, args.cpu_sample_s, B, 10_000, threads=ncpu)
        result["cpu_baseline_threads"] = {
            "value": r["updates"] / r["seconds"], "unit": UNIT, "cores": ncpu, "kind": "oracle",
            "sample": f"{r['steps']} oracle steps of 16 LEDs on this workload ({r['seconds']:.1f} s, FP64; "
                      f"2-D FFTs by scipy.fft with {ncpu} workers, BLAS threads {ncpu})"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if pg is not None:
        pg.destroy_process_group()


# --------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# --------------------------------------------------------------------------

def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as orc
    from tests.helpers import simulate
    c, nominal, truth = workload()
    I, o, g_n, g_t, prm_t = simulate(c)
    g = orc.Geometry(c.N, c.m, nominal, c.R, c.edge, c.lambda_um, c.dk_per_um)
    rec = orc.Reconstruction(g, I, orc.Hparams(lr=dict(c.lr), learn=c.learn))
    K, W = args.steps, args.warmup
    sched = full_batches(c.n_leds, c.B, K + W + 1, c.seed)
    t = time.perf_counter()
    rec.step(sched[0][:2])
    per_led = (time.perf_counter() - t) / 2
    leds = int(max(1, min(c.B, 150.0 / max(1, K + W) / max(per_led, 1e-3))))
    for k in range(W):
        rec.step(sched[1 + k][:leds])
    t0 = time.perf_counter()
    for k in range(K):
        rec.step(sched[1 + W + k][:leds])
    dt = time.perf_counter() - t0
    value = K * leds / dt
    cores = 1
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
           "warmup": W, "ms_per_step": dt / K * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "global_batch": c.B,
                      "sample": f"{leds} of the 16 LEDs of each batch per step"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{K} oracle steps of {leds} LEDs each (FP64 numpy)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("engine", "reference"), default="engine")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the tensor-core DFT forms and the autograd memory study")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the reconstruction-quality sweep over batch sizes")
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--cpu-worker", default=None)
    ap.add_argument("--cpu-threads", type=int, default=1)
    ap.add_argument("--cpu-leds", type=int, default=16)
    ap.add_argument("--cpu-max-steps", type=int, default=10_000)
    args = ap.parse_args(argv)
    if not args.cpu_worker and args.warmup < 3:
        ap.error("--warmup must be >= 3")
    return args


def main():
    args = parse_args()
    if args.cpu_worker:
        cpu_worker(args.cpu_worker, args.cpu_sample_s, args.cpu_leds, args.cpu_max_steps, args.cpu_threads)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        engine_arm(args)


if __name__ == "__main__":
    main()
