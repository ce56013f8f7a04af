#!/usr/bin/env python
"""Throughput benchmark of the B300 PIV image-pair renderer.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step renders one batch of the workload the paper's throughput study uses
(Section 3.1: 512x512 pairs; batch 64 as in the ablation defaults of
Section 3.3) with every stage of the method: 64 pairs 512x512, ppp 0.05,
d ~ U[1, 4], a distinct Fourier-mode flow per pair (rms 3 px/frame),
illumination 0.7-1.0, noise 0.02, blur 0.7, 8-bit output.  Inputs are
synthetic and seeded; the timed region starts with them resident in HBM.

Timing: W untimed warm-up steps, then K steps, each preceded by an L2 flush
(a 256 MiB write) outside its events; per-step device time from CUDA events
recorded by the library on its stream at the start and end of the launch
sequence.  One JSON line is printed by rank 0.

`--impl reference` times the FP64 CPU oracle (the correctness reference) on
the host cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PIV image pairs/s at 512², ppp 0.05 (batched/FP16 vs plain FP32); % roofline"
UNIT = "pairs/s"
N_PAIRS = 64
HBM_PEAK_FALLBACK = 6400.0  # GB/s, used only when MEASURED_PEAKS.json is absent
FP32_LANES_PER_SM = 128

# ncu DRAM traffic of k_splat per launch (bytes), with the sha256 of the
# kernel sources (splat.cuh, phi.cuh, then kernels.cuh) it was taken on; reported only
# while they are unchanged.
SPLAT_TRAFFIC = {"sha256": "709f5b93270a098f8bf97d7902416b248fac8057dbcb4138b46dcd4f6995aaaa",
                 "bytes_per_launch": 47457280 + 8827648,
                 "capture": "profiles/k_splat_batch64_512_u8.md"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--tile", type=int, default=0, help="0: autotune")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--pairs", type=int, default=N_PAIRS, help="pairs per step (profiling a smaller case)")
    ap.add_argument("--workload", default="batch64_512_u8",
                    choices=("batch64_512_u8", "single256", "uneven256", "diff32_256", "large_mixed",
                             "shapes64_512", "ablations", "stream512"),
                    help="the headline workload (default) or one of the other workloads, measured on their own")
    ap.add_argument("--advect", choices=("seed", "tiled", "gather"), default="seed",
                    help="headline workload: advect per particle while seeding (default), tile by tile "
                         "from on-chip flow windows, or per particle with a counting sort")
    ap.add_argument("--quick", action="store_true",
                    help="timed steps only (no autotune, graph, FP16, e2e, per-pair or CPU legs): for profilers")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# replicas over ranks: each rank renders its own pairs (disjoint pair ids, so
# the outputs are those of one large batch); the step time is the maximum
# over ranks and the value counts the pairs of every rank
# ----------------------------------------------------------------------------

def rank_pair_ids(rank: int, n_pairs: int):
    """Pair ids rank `rank` renders: [rank * n_pairs, (rank + 1) * n_pairs)."""
    return [rank * n_pairs + b for b in range(n_pairs)]


def max_over_ranks(x: float, dist, device="cpu") -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_pairs_per_s(world: int, pairs_per_rank: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: the pairs of all ranks over the slowest rank's time."""
    return world * pairs_per_rank * steps / (total_ms / 1e3)


def workload(rank: int = 0, n_pairs: int = N_PAIRS):
    from paper_2512_09664_b300 import workloads as W
    wl = W.batch_512_u8(n_pairs=n_pairs, seed=1)
    if rank:  # weak scaling: every rank renders its own pairs
        for p, pid in zip(wl.pairs, rank_pair_ids(rank, n_pairs)):
            p.pair_id = pid
    return wl


def workload_config(wl, extra=None):
    cfg = {"workload": "batch64_512_u8: 64 pairs 512x512, ppp 0.05 (13107 particles/frame), d~U[1,4] px, "
                       "I~U[0.8,1], z~U[-1,1] sheet 0.5, Fourier flow rms 3 px/frame (one grid per pair), "
                       "RK4 x4 dt 1, illum 0.7-1.0, noise 0.02, blur 0.7, 8-bit",
           "pairs_per_step": wl.n_pairs, "height": 512, "width": 512, "ppp": 0.05,
           "l2": "flushed between steps (256 MiB write outside the timed events)"}
    if extra:
        cfg.update(extra)
    return cfg


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": HBM_PEAK_FALLBACK, "sm_max_mhz": 2032.0}, "fallback"


# ----------------------------------------------------------------------------
# algorithmic work of the method (per pair), the roofline numerators
# ----------------------------------------------------------------------------

def algorithmic(wl):
    """Bytes and FP32 lane-operations the method needs, summed over the batch.

    bytes: both output frames written once + the FP32 flow grid read once.
    lane-ops (minimum arithmetic of the method, an FMA counted once):
      per particle and frame: (6 E[d] + 4) window edges x 12 (one Phi value:
      a cubic piece of the tabulated normal tail, its index and scaling) +
      E[(3d + 1)^2] pixels x 2 (product and accumulation);
      per output pixel: illumination 1, noise 13 (a quarter of a 10-round
      Philox call at 4 ops per round plus half a Box-Muller pair),
      blur 2 (2R + 1), quantisation 2.
    """
    nbytes, ops = 0, 0.0
    osize = {"u8": 1, "u16": 2, "f16": 2, "bf16": 2, "f32": 4}[wl.out_dtype]
    for p in wl.pairs:
        g = wl.flows[p.flow_index]
        nbytes += 2 * p.height * p.width * osize
        lo, hi = float(p.d_min), float(p.d_max)
        ed, ed2 = (lo + hi) / 2, (lo * lo + lo * hi + hi * hi) / 3
        edges = 6 * ed + 4
        pixels = 9 * ed2 + 6 * ed + 1
        ops += 2 * p.n_particles * (12 * edges + 2 * pixels)
        R = math.ceil(3 * float(p.blur_sigma)) if p.blur_sigma > 0 else 0
        per_px = 1 + (13 if p.noise_sigma > 0 else 0) + (2 * (2 * R + 1) if R else 0) + 2
        ops += 2 * p.height * p.width * per_px
    flow_bytes = sum(f.size * 4 for f in wl.flows)
    return nbytes + flow_bytes, ops


def shapes_algorithmic(wl, samples: int = 200000, seed: int = 0):
    """Lane-operations of the general-shape splat plus the epilogue (batch sum).

    Per visible particle and frame (expectations over the drawn d, d_y, rho):
      rho = 0: (n_x + 1 + n_y + 1) edge values x 12 + n_x n_y pixels x 2;
      rho != 0: per window column 4 m Gauss-Legendre nodes (m sub-intervals
      of the pixel no wider than min(sigma_x, sigma_x sqrt(1-rho^2)/|rho|)),
      each with its density weight (6) and n_y + 1 conditional edge values
      (x 12) and n_y weighted differences (x 2); + n_x n_y accumulations.
    with n_x = 3 d + 1, n_y = 3 d_y + 1.  Epilogue per output pixel as in
    algorithmic().  Frame-2 variation is small and not modelled.
    """
    import numpy as np
    rng = np.random.default_rng(seed)
    ops = 0.0
    for p in wl.pairs:
        d = rng.uniform(float(p.d_min), float(p.d_max), samples)
        same = float(p.dy_min) == 0.0 and float(p.dy_max) == 0.0
        dy = d if same else rng.uniform(float(p.dy_min), float(p.dy_max), samples)
        rho = rng.uniform(float(p.rho_min), float(p.rho_max), samples)
        nx, ny = 3 * d + 1, 3 * dy + 1
        c = np.sqrt(1 - rho * rho)
        sx = d / 4
        ell = np.where(np.abs(rho) > c, sx * c / np.maximum(np.abs(rho), 1e-30), sx)
        m = np.clip(np.ceil(1.0 / ell), 1, 256)
        sep = (nx + 1 + ny + 1) * 12 + nx * ny * 2
        quad = nx * 4 * m * (6 + (ny + 1) * 12 + ny * 2) + nx * ny
        per = np.where(rho == 0.0, sep, quad).mean()
        ops += 2 * p.n_particles * (1.0 - float(wl.hide_prob)) * per
        R = math.ceil(3 * float(p.blur_sigma)) if p.blur_sigma > 0 else 0
        per_px = 1 + (13 if p.noise_sigma > 0 else 0) + (2 * (2 * R + 1) if R else 0) + 2
        ops += 2 * p.height * p.width * per_px
    return ops


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        load = [s for s in sm if s > 0.5 * mx] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("", "[N/A]"))}


# ----------------------------------------------------------------------------
# CPU arms (oracle)
# ----------------------------------------------------------------------------

def oracle_sample(wl, n_pairs: int, start: int, threads: int):
    import oracle
    idx = [(start + k) % wl.n_pairs for k in range(n_pairs)]
    t0 = time.perf_counter()
    oracle.render_workload(wl, pairs=idx, threads=threads)
    return time.perf_counter() - t0


def cpu_baseline(wl, seconds: float):
    cores = os.cpu_count() or 1
    threads = min(cores, wl.n_pairs)
    done, elapsed, start = 0, 0.0, 0
    while elapsed < seconds:
        elapsed += oracle_sample(wl, threads, start, threads)
        done += threads
        start += threads
    return {"value": done / elapsed, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{done} pairs of the same workload (FP64 C oracle, {threads} host threads, "
                      f"{elapsed:.1f} s)"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = workload()
    cores = os.cpu_count() or 1
    threads = min(cores, wl.n_pairs)
    for w in range(args.warmup):
        oracle_sample(wl, threads, w * threads, threads)
    total = 0.0
    for k in range(args.steps):
        total += oracle_sample(wl, threads, k * threads, threads)
    value = args.steps * threads / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(wl, {"step": f"{threads} pairs of the workload per step"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{threads} pairs per step, {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def splat_source_hash():
    data = b""
    for name in ("splat.cuh", "phi.cuh", "kernels.cuh"):
        with open(os.path.join(ROOT, "paper_2512_09664_b300", "csrc", name), "rb") as f:
            data += f.read()
    return hashlib.sha256(data).hexdigest()


def device_alu_peak(dev, peaks):
    """FP32 lane-op peak (T/s) of the device: SMs (queried) x 128 lanes x the max SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2032.0))
    return sms * FP32_LANES_PER_SM * mhz * 1e6 / 1e12, f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {mhz:.0f} MHz"


def step_roofline(wl, ms, peaks, alu_peak):
    """The method's step roofline: t_roof = max(algorithmic bytes / HBM peak,
    algorithmic lane-ops / FP32 peak); frac = t_roof / measured step time."""
    alg_bytes, alg_ops = algorithmic(wl)
    t_hbm = alg_bytes / (float(peaks["hbm_gbs"]) * 1e9) * 1e6
    t_alu = alg_ops / (alu_peak * 1e12) * 1e6
    t_roof = max(t_hbm, t_alu)
    return {"t_hbm_us": t_hbm, "t_alu_us": t_alu, "t_roof_us": t_roof, "t_step_us": ms * 1e3,
            "frac": t_roof / (ms * 1e3), "bound": "hbm" if t_hbm >= t_alu else "alu",
            "algorithmic_bytes": alg_bytes, "algorithmic_lane_ops": alg_ops}


def _events(n):
    import torch
    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]


def _timed(fn, steps, flush, stream, flush_l2=True):
    """Per-call device times (ms) of fn on stream, CUDA events around each call."""
    import torch
    ev = _events(steps)
    torch.cuda.synchronize()
    for k in range(steps):
        if flush_l2:
            flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def leg_single_pair(flush, stream, peaks, alu_peak, steps):
    """Config 1: one 256^2 pair (Lamb-Oseen, FP32 output): a latency-bound render."""
    import statistics

    from paper_2512_09664_b300 import workloads as W
    from paper_2512_09664_b300.binding import Renderer
    wl = W.single_pair_256(seed=0)
    r = Renderer(wl)
    for _ in range(3):
        r.render()
    eager = statistics.median(_timed(r.render, steps, flush, stream))
    r.capture()
    for _ in range(3):
        r.replay()
    graph = statistics.median(_timed(r.replay, steps, flush, stream))
    return {"config": wl.description, "eager_ms": eager, "graph_ms": graph, "value": 1.0 / (graph / 1e3),
            "unit": UNIT, "mpx_per_s": 2 * 256 * 256 / (graph / 1e3) / 1e6,
            "step_roofline": step_roofline(wl, graph, peaks, alu_peak),
            "note": "median over the timed renders; one pair is bound by launch and dependency latency"}


def leg_uneven(flush, stream, peaks, alu_peak, steps):
    """Config 3: 256 pairs of uneven sizes in one persistent, graph-captured
    launch sequence with autotuned per-size-class parameters, against one
    autotuned edge for the whole batch and against per-pair launches."""
    import statistics

    import torch

    from paper_2512_09664_b300 import workloads as W
    from paper_2512_09664_b300.binding import Renderer
    wl = W.uneven_batch(n_pairs=256, seed=2)
    r = Renderer(wl)
    tuned = r.tune(reps=2)
    r.capture()
    for _ in range(2):
        r.replay()
    g_ms = statistics.median(_timed(r.replay, steps, flush, stream))
    one = Renderer(wl)
    edge, _ = one.autotune(reps=2)
    one.capture()
    for _ in range(2):
        one.replay()
    one_ms = statistics.median(_timed(one.replay, steps, flush, stream))
    del one
    per = [Renderer(wl.subset([b])) for b in range(wl.n_pairs)]  # tile 0: the tuned table
    for p in per:
        p.render()

    def per_pair():
        for p in per:
            p.render()
    p_ms = statistics.median(_timed(per_pair, max(3, steps // 5), flush, stream))
    del per
    torch.cuda.empty_cache()
    return {"config": wl.description, "tuned": tuned, "graph_persistent_ms": g_ms,
            "value": wl.n_pairs / (g_ms / 1e3), "unit": UNIT, "mpx_per_s": wl.image_elems() / (g_ms / 1e3) / 1e6,
            "single_edge": {"tile": edge, "graph_ms": one_ms, "value": wl.n_pairs / (one_ms / 1e3)},
            "per_pair_launches": {"ms": p_ms, "value": wl.n_pairs / (p_ms / 1e3)},
            "speedup_over_per_pair": p_ms / g_ms, "speedup_over_single_edge": one_ms / g_ms,
            "particles": sum(p.n_particles for p in wl.pairs),
            "step_roofline": step_roofline(wl, g_ms, peaks, alu_peak)}


def leg_differentiable(flush, stream, peaks, alu_peak, steps):
    """Config 4: 32 pairs 256^2 from a 32^2 control grid: forward render from
    the seeded particles and the adjoint (gradients w.r.t. flow, x0, y0, d)."""
    import statistics

    import numpy as np
    import torch

    from paper_2512_09664_b300 import workloads as W
    from paper_2512_09664_b300.binding import Renderer
    wl = W.differentiable_batch(n_pairs=32)
    ctrl = torch.tensor(np.stack(wl.meta["control"]), dtype=torch.float32)
    up = torch.nn.functional.interpolate(ctrl.permute(0, 3, 1, 2), size=(256, 256), mode="bilinear",
                                         align_corners=False).permute(0, 2, 3, 1).contiguous()
    wl.flows = [f.numpy() for f in up]
    r = Renderer(wl)
    G = torch.randn(r.images.shape, device=r.images.device)
    gf = torch.zeros_like(r.flows)
    gp = torch.empty((sum(p.n_particles for p in wl.pairs), 3), device=r.images.device)
    for _ in range(3):
        r.render_from()
        r.backward(G, grad_flows=gf, grad_particles=gp)
    f_ms = statistics.median(_timed(r.render_from, steps, flush, stream))
    b_ms = statistics.median(_timed(lambda: r.backward(G, grad_flows=gf, grad_particles=gp), steps, flush, stream))
    n_part = sum(p.n_particles for p in wl.pairs)
    # backward bytes: dL/dimages read once (FP32), flows read, flow gradients written, particle gradients written
    b_bytes = r.images.numel() * 4 + 2 * r.flows.numel() * 4 + n_part * 12
    hbm = float(peaks["hbm_gbs"]) * 1e9
    return {"config": wl.description, "forward_ms": f_ms, "backward_ms": b_ms,
            "value": wl.n_pairs / ((f_ms + b_ms) / 1e3), "unit": UNIT,
            "forward_value": wl.n_pairs / (f_ms / 1e3),
            "forward_step_roofline": step_roofline(wl, f_ms, peaks, alu_peak),
            "backward_roofline_hbm": {"algorithmic_bytes": b_bytes, "t_hbm_us": b_bytes / hbm * 1e6,
                                      "frac": (b_bytes / hbm * 1e3) / b_ms}}


def leg_large_mixed(flush, stream, peaks, alu_peak, steps):
    """Config 5: 16 x 2048^2 + 16 x 1920x1080, 16-bit output; FP32 (fused, on
    chip) vs FP16 and BF16 intermediate frames in HBM, each autotuned."""
    import statistics

    import torch

    from paper_2512_09664_b300 import workloads as W
    from paper_2512_09664_b300.binding import Renderer
    wl = W.large_mixed_batch()
    res = {}
    for inter in ("f32", "f16", "bf16"):
        r = Renderer(wl, inter_dtype=inter)
        tuned = r.tune(reps=1)
        for _ in range(2):
            r.render()
        ms = statistics.median(_timed(r.render, steps, flush, stream))
        res[inter] = {"ms_per_step": ms, "value": wl.n_pairs / (ms / 1e3), "tuned": tuned,
                      "mpx_per_s": wl.image_elems() / (ms / 1e3) / 1e6,
                      "step_roofline": step_roofline(wl, ms, peaks, alu_peak)}
        del r
        torch.cuda.empty_cache()
    return {"config": wl.description, "paths": res, "value": res["f16"]["value"], "unit": UNIT,
            "f16_speedup_over_f32": res["f32"]["ms_per_step"] / res["f16"]["ms_per_step"]}


def run_ours(args, rank, world, dist):
    import statistics

    import torch

    from paper_2512_09664_b300.binding import Renderer
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = workload(rank, args.pairs)
    from paper_2512_09664_b300.binding import FLAG_GATHER_ADVECT, FLAG_TILED_ADVECT
    adv_flags = {"seed": 0, "tiled": FLAG_TILED_ADVECT, "gather": FLAG_GATHER_ADVECT}[args.advect]
    # tile 0: per-size-class edges (defaults, then autotuned)
    r = Renderer(wl, device=dev, tile=args.tile, flags=adv_flags)
    stream = torch.cuda.current_stream()
    tuned = None
    if args.tile == 0 and not args.quick:
        tuned = r.tune(reps=2)

    def barrier():
        if dist is not None:
            dist.barrier()

    def new_events():
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        for e in evs:
            e.record(stream)  # creates the CUDA event
        return evs

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        flush.fill_(1)
        r.render()
    torch.cuda.synchronize()
    # timed steps: one event pair around each render (nothing between its launches)
    events = _events(args.steps)
    from paper_2512_09664_b300.binding import launch_count
    with ClockSampler(dev.index) as clk:
        barrier()
        torch.cuda.synchronize()
        launches0 = launch_count()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            events[k][0].record(stream)
            r.render()
            events[k][1].record(stream)
        launches = launch_count() - launches0  # the library's kernels of the timed steps
        torch.cuda.synchronize()
        barrier()
    clocks = clk.summary()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in events]
    total_ms = sum(step_ms)
    # per-stage breakdown: a separate pass with events recorded by the library between its launches
    n_staged = min(args.steps, 50)
    staged = [new_events() for _ in range(n_staged)]
    torch.cuda.synchronize()
    for k in range(n_staged):
        flush.fill_(k & 0xFF)
        r.render_staged(staged[k])
    torch.cuda.synchronize()
    stage_ms = _stage_medians(staged)
    total_ms = max_over_ranks(total_ms, dist, dev)
    value = aggregate_pairs_per_s(world, wl.n_pairs, args.steps, total_ms)
    ms_per_step = total_ms / args.steps
    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms_per_step,
                              "stage_ms": stage_ms, "quick": True, "pairs_per_step": wl.n_pairs}), flush=True)
        return

    # the same step replayed from a captured CUDA graph (no host launch cost)
    r.capture()
    for _ in range(2):
        r.replay()
    graph_ms = statistics.mean(_timed(r.replay, min(args.steps, 50), flush, stream))

    # the batched path with FP16 intermediate frames (splat, then a separate
    # finishing kernel reading the 16-bit frames)
    r16 = Renderer(wl, device=dev, tile=args.tile, inter_dtype="f16", flags=adv_flags)
    if args.tile == 0:
        r16.tune(reps=2)
    for _ in range(3):
        r16.render()
    f16_ms = statistics.mean(_timed(r16.render, min(args.steps, 50), flush, stream))
    f16_tuning = r16.tuning()
    del r16

    # end to end through the same C ABI: every step copies its flows in from
    # pinned host memory and its images out to pinned host memory; the
    # pipeline overlaps step k's render with the copies of its neighbours
    from paper_2512_09664_b300.binding import HostPipeline
    flows_host = torch.from_numpy(r.pk.flows_host).pin_memory()
    img_host = [torch.empty(r.images.shape, dtype=r.images.dtype).pin_memory() for _ in range(2)]
    pipe = HostPipeline(r, depth=2)
    e2e_steps = max(3, min(args.steps, 30))
    for k in range(2):
        pipe.submit(flows_host, img_host[k % 2], stream)
    pipe.synchronize(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for k in range(e2e_steps):
        pipe.submit(flows_host, img_host[k % 2], stream)
    pipe.synchronize(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    h2d = flows_host.numel() * flows_host.element_size()
    d2h = img_host[0].numel() * img_host[0].element_size()
    e2e_serial_ms = _e2e_serial_ms(r, flows_host, img_host[0], stream, e2e_steps)

    # plain per-pair path at the same accuracy: one launch sequence per pair,
    # the same u8 output and epilogue, FP32 throughout
    plain = [Renderer(wl.subset([b]), device=dev, tile=args.tile, flags=adv_flags) for b in range(wl.n_pairs)]
    for p in plain:
        p.render()
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    p0.record(stream)
    for _ in range(reps):
        for p in plain:
            p.render()
    p1.record(stream)
    torch.cuda.synchronize()
    plain_pairs_s = reps * wl.n_pairs / (p0.elapsed_time(p1) / 1e3)
    plain_tuning = plain[0].tuning()
    del plain

    peaks, peak_kind = measured_peaks()
    alu_peak, alu_src = device_alu_peak(dev, peaks)
    alg_bytes, alg_ops = algorithmic(wl)
    splat_ms = stage_ms["splat_epilogue"]
    # the epilogue and splat work run in the splat kernel; seeding/advection
    # arithmetic is not counted there
    achieved = alg_ops / (splat_ms / 1e3) / 1e12
    traffic = None
    if SPLAT_TRAFFIC["sha256"] == splat_source_hash():
        traffic = SPLAT_TRAFFIC["bytes_per_launch"]
    hbm_peak = float(peaks["hbm_gbs"])
    step_gbs = alg_bytes / (ms_per_step / 1e3) / 1e9
    probes = alu_probes(stream)
    legs = {}
    if rank == 0 and world == 1:  # the other configurations, on one GPU
        legs["single_pair_256"] = leg_single_pair(flush, stream, peaks, alu_peak, max(args.steps, 20))
        legs["uneven256"] = leg_uneven(flush, stream, peaks, alu_peak, min(args.steps, 20))
        legs["diff32_256"] = leg_differentiable(flush, stream, peaks, alu_peak, min(args.steps, 20))
        legs["large_mixed"] = leg_large_mixed(flush, stream, peaks, alu_peak, min(args.steps, 10))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(wl, {"tuning": r.tuning(), "tuning_choice": "autotuned" if args.tile == 0
                                       else "fixed", "path": "fused FP32 splat + epilogue (on-chip intermediate)",
                                       "advection": {"seed": "per particle while seeding, fixed bins",
                                                     "tiled": "tile by tile from on-chip flow windows, fixed bins",
                                                     "gather": "per particle, counting-sort bins"}[args.advect],
                                       "parallelism": f"replicas x{world}"}),
        "mpx_per_s": value * 2 * 512 * 512 / 1e6,
        "stage_ms": stage_ms,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tlane-op/s",
                     "frac": achieved / alu_peak, "traffic": traffic, "kernel": "k_splat",
                     "peak_source": alu_src,
                     "measured_fma_peak": probes["fma"], "frac_of_measured_fma": achieved / probes["fma"]},
        "alu_probes": {"unit": "T op/s", **probes,
                       "source": "synthpix_alu_probe (measurement library), best of 3 launches of one full wave "
                                 "after the timed steps"},
        "step_roofline": step_roofline(wl, ms_per_step, peaks, alu_peak),
        "step_roofline_hbm": {"achieved_gbs": step_gbs, "peak_gbs": hbm_peak, "frac": step_gbs / hbm_peak,
                              "peak_source": peak_kind, "algorithmic_bytes_per_step": alg_bytes},
        "plain_fp32_per_pair": {"value": plain_pairs_s, "unit": UNIT, "speedup": value / world / plain_pairs_s,
                                "output": "u8 with the same illumination, noise, blur and quantisation",
                                "tuning": plain_tuning},
        "batched_f16_intermediate": {
            "value": wl.n_pairs / (f16_ms / 1e3), "unit": UNIT, "ms_per_step": f16_ms, "tuning": f16_tuning,
            "speedup_over_fused_f32": (ms_per_step / world) / f16_ms,
            "why": "at 512x512 the fused FP32 path keeps the splatted frame on chip and writes each output "
                   "pixel once, so 16-bit intermediate frames only add an HBM round trip and a second kernel; "
                   "they pay where a frame's tile cannot be finished on chip (see large_mixed)"},
        "graph_replay": {"ms_per_step": graph_ms, "value": world * wl.n_pairs / (graph_ms / 1e3), "unit": UNIT},
        "e2e": {"value": world * wl.n_pairs / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "path": "HostPipeline: pinned flows in, render, pinned images out; two device buffer sets, "
                        "copies of neighbouring steps overlap the render",
                "serial_value": world * wl.n_pairs / (e2e_serial_ms / 1e3)},
        "workloads": legs,
        "gpu_launches": launches,  # counted by the library (synthpix_launch_count) around the timed steps
        "clocks": clocks,
    }
    if tuned is not None:
        line["config"]["autotune"] = tuned
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# the other workloads (not the headline): measured with their own comparisons
# ----------------------------------------------------------------------------

def _time_device(fn, steps, flush, stream):
    import torch
    tot = 0.0
    for k in range(steps):
        flush.fill_(k & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / steps


def alu_probes(stream):
    """Measured throughput (T op/s) of FP32 FMA, erfcf, ex2 and the Philox high multiply."""
    from paper_2512_09664_b300 import binding as B
    iters = {"fma": 4096, "erfc": 256, "ex2": 2048, "umulhi": 2048}
    from paper_2512_09664_b300 import measure
    return {k: measure.alu_probe(k, iters=n, reps=3, stream=stream) / 1e12 for k, n in iters.items()}


def _e2e_serial_ms(r, flows_host, img_host, stream, steps):
    """The same end-to-end step with nothing overlapped: copy in, render, copy out."""
    import torch
    for _ in range(2):
        r.flows.copy_(flows_host, non_blocking=True)
        r.render(stream)
        img_host.copy_(r.images, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        r.flows.copy_(flows_host, non_blocking=True)
        r.render(stream)
        img_host.copy_(r.images, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _stage_ms(r, n, flush, stream):
    """Median per-stage times over n renders with the library's stage events."""
    import torch

    staged = []
    for k in range(n):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        for e in evs:
            e.record(stream)
        staged.append(evs)
    torch.cuda.synchronize()
    for k in range(n):
        flush.fill_(k & 0xFF)
        r.render_staged(staged[k])
    torch.cuda.synchronize()
    return _stage_medians(staged)


def _stage_medians(staged):
    """Per-stage median over renders of the times between the library's stage events.

    The median, not the mean: a render whose launches the host enqueued late
    (the GPU idle between two stage events) would otherwise inflate a stage.
    """
    import numpy as np

    from paper_2512_09664_b300.binding import STAGES
    return {name: float(np.median([ev[i].elapsed_time(ev[i + 1]) for ev in staged]))
            for i, name in enumerate(STAGES)}


def _step_stats(ms):
    """pairs/s statistics over per-step times (ms) of n_pairs-pair steps: filled in by the caller."""
    import numpy as np
    a = np.asarray(ms)
    return {"ms_mean": float(a.mean()), "ms_min": float(a.min()), "ms_max": float(a.max()),
            "ms_q1": float(np.percentile(a, 25)), "ms_q3": float(np.percentile(a, 75)), "ms_std": float(a.std())}


def run_ablations(args, flush, stream):
    """The throughput ablations of Section 3.3 on synthetic inputs: one axis at
    a time around the paper's fixed point (512^2, ppp 0.06, d~U[0.8,1.2], B 64,
    F 1).  Each point: per-step device times over args.steps renders (L2
    flushed before each), as pairs/s mean and spread.  The flow-reuse axis
    times the end-to-end loop: flows copied from pinned host memory once
    every R batches, images copied back every batch."""
    import torch

    from paper_2512_09664_b300 import workloads as W
    from paper_2512_09664_b300.binding import Renderer

    def point(axis, value, wl, reuse=None):
        r = Renderer(wl)
        for _ in range(2):
            r.render()
        torch.cuda.synchronize()
        ms = []
        if reuse is None:
            for k in range(args.steps):
                flush.fill_(k & 0xFF)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r.render()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
        else:
            fh = torch.from_numpy(r.pk.flows_host).pin_memory()
            ih = torch.empty(r.images.shape, dtype=r.images.dtype).pin_memory()
            for k in range(args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if reuse == 0 or k % reuse == 0:
                    r.flows.copy_(fh, non_blocking=True)
                r.render()
                ih.copy_(r.images, non_blocking=True)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
        st = _step_stats(ms)
        n = wl.n_pairs
        out = {"axis": axis, "value": value, "pairs_s": n / (st["ms_mean"] / 1e3),
               "pairs_s_min": n / (st["ms_max"] / 1e3), "pairs_s_max": n / (st["ms_min"] / 1e3),
               "pairs_s_q1": n / (st["ms_q3"] / 1e3), "pairs_s_q3": n / (st["ms_q1"] / 1e3),
               "tile": r.pk.batch.tile, **st}
        del r
        torch.cuda.empty_cache()
        return out

    pts = []
    for size in (128, 256, 512, 1024, 2048):
        pts.append(point("image_size", size, W.ablation_batch(size=size)))
    for ppp in (0.01, 0.02, 0.04, 0.06, 0.08, 0.1):
        pts.append(point("ppp", ppp, W.ablation_batch(ppp=ppp)))
    for dmax in (1.2, 2.0, 3.0, 4.0, 6.0, 8.0):
        pts.append(point("d_max", dmax, W.ablation_batch(d_max=dmax)))
    for pmin in (0.01, 0.02, 0.04, 0.06):
        pts.append(point("ppp_min", pmin, W.ablation_batch(ppp=0.06, ppp_min=pmin)))
    for B in (1, 4, 16, 64, 256, 1024):
        pts.append(point("batch", B, W.ablation_batch(n_pairs=B)))
    for F in (1, 4, 16, 64):
        pts.append(point("flows_per_batch", F, W.ablation_batch(n_flows=F)))
    for R in (1, 2, 4, 16):
        pts.append(point("batches_per_flow", R, W.ablation_batch(), reuse=R))
    return {"config": "Section 3.3 ablations around 512^2, ppp 0.06, d~U[0.8,1.2], B 64, F 1 (synthetic "
                      "Fourier flows, RK4 x4, f32 output, no epilogue)", "points": pts,
            "value": next(p["pairs_s"] for p in pts if p["axis"] == "batch" and p["value"] == 64)}


def run_other(args):
    import numpy as np
    import torch

    from paper_2512_09664_b300 import workloads as W
    from paper_2512_09664_b300.binding import Renderer
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    line = {"workload": args.workload, "steps": args.steps, "warmup": args.warmup, "unit": UNIT}
    peaks, peak_kind = measured_peaks()
    alu_peak, alu_src = device_alu_peak(torch.device("cuda", 0), peaks)
    if args.workload == "uneven256":
        line.update(leg_uneven(flush, stream, peaks, alu_peak, args.steps))
    elif args.workload == "diff32_256":
        line.update(leg_differentiable(flush, stream, peaks, alu_peak, args.steps))
    elif args.workload == "single256":
        line.update(leg_single_pair(flush, stream, peaks, alu_peak, args.steps))
    elif args.workload == "shapes64_512":
        # Eq. 1 shape options: elliptical axis-misaligned particles with frame-2
        # variation and hiding (general-shape splat), and round particles with
        # variation and hiding (round splat, per-particle advection)
        res = {}
        for kind in ("general", "round", "focus"):
            # focus: round particles, the Remark's out-of-focus intensity and a w grid per pair
            wl = W.focus_batch(n_pairs=64) if kind == "focus" else W.shapes_batch(n_pairs=64,
                                                                                 general=kind == "general")
            r = Renderer(wl)
            tuned = r.tune(reps=1)
            for _ in range(args.warmup):
                flush.fill_(1)
                r.render()
            with ClockSampler(0) as clk:
                ms = _time_device(r.render, args.steps, flush, stream)
            st = _stage_ms(r, min(args.steps, 20), flush, stream)
            res[kind] = {"ms_per_step": ms, "value": wl.n_pairs / (ms / 1e3), "tuning": tuned, "stage_ms": st,
                         "config": wl.description, "clocks": clk.summary()}
            if kind == "general":
                achieved = shapes_algorithmic(wl) / (st["splat_epilogue"] / 1e3) / 1e12
                alg_bytes, _ = algorithmic(wl)
                step_gbs = alg_bytes / (ms / 1e3) / 1e9
                res[kind]["roofline"] = {
                    "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tlane-op/s",
                    "frac": achieved / alu_peak, "traffic": None, "kernel": "k_splat (general shapes)",
                    "peak_source": alu_src}
                res[kind]["step_roofline_hbm"] = {"achieved_gbs": step_gbs, "peak_gbs": float(peaks["hbm_gbs"]),
                                                  "frac": step_gbs / float(peaks["hbm_gbs"]),
                                                  "peak_source": peak_kind}
                if not args.no_cpu_baseline:
                    res[kind]["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
            del r
            torch.cuda.empty_cache()
        line.update({"paths": res, "value": res["general"]["value"],
                     "general_over_round_ms": res["general"]["ms_per_step"] / res["round"]["ms_per_step"]})
    elif args.workload == "ablations":
        line.update(run_ablations(args, flush, stream))
    elif args.workload == "stream512":
        # the streaming sampler on the headline configuration: a new set of
        # procedural flows every batch (generated on a side stream, one set
        # ahead) or one set reused; device time per batch on the render stream
        from paper_2512_09664_b300 import sampler as S
        res = {}
        import numpy as np
        hist = ((np.exp(-np.arange(256) / 40.0) * 1e5).astype(np.int64) + 1).tolist()
        for name, F, R, th in (("F64_R1", 64, 1, None), ("F1_R1", 1, 1, None), ("F64_reused", 64, 10 ** 9, None),
                               ("F1_R1_histogram_matched", 1, 1, hist)):
            cfg = {"image_shape": [512, 512], "batch_size": 64, "flows_per_batch": F, "batches_per_flow": R,
                   "seed": 1, "seeding_density": 0.05, "diameter": [1.0, 4.0], "illumination": [0.7, 1.0],
                   "noise_sigma": 0.02, "blur_sigma": 0.7, "output": "u8", "bits": 8,
                   "flow": {"kind": "fourier", "rms": 3.0}, "target_histogram": th}
            smp = S.make(cfg)
            for _ in range(args.warmup):
                next(smp)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                next(smp)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            res[name] = {"ms_per_batch": ms, "value": 64 / (ms / 1e3), "flows_per_batch": F,
                         "batches_per_flow": R if R < 10 ** 9 else "all"}
            del smp
            torch.cuda.empty_cache()
        # the two kernels the sampler adds, timed alone: histogram matching of a
        # rendered 64 x 512^2 u8 batch (HBM: codes read twice, written once) and
        # 64 Fourier fields of 512^2 with 64 modes (FP32: a product and three FMAs,
        # 7 flops, per node and mode)
        from paper_2512_09664_b300 import binding as Bn
        wlh = W.batch_512_u8(n_pairs=64, seed=1)
        r = Renderer(wlh)
        r.render()
        tgt = torch.tensor(hist, dtype=torch.int64, device="cuda")
        ws = Bn.match_histogram(r.pk, r.images, tgt)
        n = max(args.steps, 10)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            Bn.match_histogram(r.pk, r.images, tgt, ws)
        e1.record(stream)
        torch.cuda.synchronize()
        h_ms = e0.elapsed_time(e1) / n
        h_bytes = 3 * r.images.numel()
        modes = torch.from_numpy(np.stack([W.fourier_modes(9000 + f, 512, 512) for f in range(64)])).cuda()
        fl = torch.empty((64, 512, 512, 2), dtype=torch.float32, device="cuda")
        fws = torch.empty(Bn.fourier_flows_workspace_bytes(64, 64, 512, 512), dtype=torch.uint8, device="cuda")
        Bn.fourier_flows(modes, 512, 512, 512, 512, 3.0, fl, fws)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            Bn.fourier_flows(modes, 512, 512, 512, 512, 3.0, fl, fws)
        e1.record(stream)
        torch.cuda.synchronize()
        f_ms = e0.elapsed_time(e1) / n
        f_flop = 64 * 512 * 512 * 64 * 7.0
        fp32_peak = 2 * alu_peak
        line.update({"config": "streaming sampler, 64 pairs 512x512 u8 per batch (the headline recipe), "
                               "Fourier flows rms 3 generated on the device", "paths": res,
                     "value": res["F64_R1"]["value"],
                     "histogram_matching": {"ms_per_batch": h_ms, "roofline": {
                         "bound": "hbm", "achieved": h_bytes / (h_ms / 1e3) / 1e9, "peak": float(peaks["hbm_gbs"]),
                         "unit": "GB/s", "frac": h_bytes / (h_ms / 1e3) / 1e9 / float(peaks["hbm_gbs"]),
                         "algorithmic_bytes": h_bytes, "peak_source": peak_kind}},
                     "flow_generation_64x512": {"ms": f_ms, "roofline": {
                         "bound": "alu", "achieved": f_flop / (f_ms / 1e3) / 1e12, "peak": fp32_peak,
                         "unit": "TFLOP/s (FP32)", "frac": f_flop / (f_ms / 1e3) / 1e12 / fp32_peak,
                         "peak_source": alu_src + " x 2 flops"}}})
    else:  # large_mixed
        line.update(leg_large_mixed(flush, stream, peaks, alu_peak, args.steps))
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload != "batch64_512_u8":
        run_other(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    run_ours(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
