#!/usr/bin/env python
"""Benchmark of the sequential phase-linking hot path on one GB300 per rank.

A step is one mini-stack through the whole path (amplitude statistics, GLRT SHP
selection, coherence, EMI phase linking with reference and temporal coherence,
compressed SLC), i.e. one plk_ministack_step on the burst-shaped workload:
N = 15 complex64 SLCs of 4096 x 16384 pixels, 11 x 5 window, output strides
6 x 3 (1365 x 2730 output pixels), synthetic exponential-decay coherence with
tau ~ U(12, 120) days and 5% persistent scatterers.  The stack (8.05 GB) is far
larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(the baseline this build has; the paper's system is a CPU cloud pipeline with no
GPU path) on a bounded crop of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "phase-linked pixels/s (N=15, 11×5 window) and % of HBM/FP32 roofline"
UNIT = "output px/s"
WINDOW = (5, 11, 3, 6)  # wy, wx, sy, sx  ("11 x 5", strides 6 x 3)
N_DATES = 15
PS_DA_MAX = 0.2  # production PS threshold on the amplitude dispersion (Sec. IV)
GS_RADIUS = 7    # gamma_s window radius in output pixels: ~200 m at the 30 m posting (Sec. III-C)
ADMM_ITERS = 50  # L1 network inversion: fixed ADMM iterations (rho = 1), exact on 2%-error synthetic stacks
H_FULL, W_FULL = 4096, 16384
WORKLOAD = "burst-shaped mini-stack: N=15 complex64 SLCs x 4096x16384 px, 11x5 window, output strides 6x3"


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except Exception:
            pass
    return {}


# FP32 SIMT peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop
# (FMA) x 2.070 GHz maximum SM clock.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


# DRAM bytes per output pixel of a launch, from the ncu capture summarised in
# profiles/k_emi32_k_cov_async_1024x4096.md (1024x4096 case; traffic grows with
# the pixel count).  Valid for the kernel versions profiled there: a kernel
# changed since its capture must drop out of this table (traffic null).
NCU_DRAM_BYTES_PER_OUTPUT_PX = {
    "covariance": (515.460096e6 + 203.568128e6) / 232562,
    "phase_link_fp32": (223.616256e6 + 11.620864e6) / 232562,
}


def flops_covariance(N: int, looks_total: float) -> float:
    """Algorithmic flops of the Hermitian sample covariance: 4 N^2 per look."""
    return 4.0 * N * N * looks_total


def flops_emi(N: int, npx: int) -> float:
    """Algorithmic flops of EMI per pixel: inverse of |C| and a factorisation of
    the shifted Hadamard product ((8/3) N^3 each), ten inverse-iteration steps
    (8 N^2 each) and gamma_t (~10 N^2)."""
    return npx * ((16.0 / 3.0) * N ** 3 + 90.0 * N * N)


def flops_admm_iteration(n_ifg: int, nx: int) -> float:
    """Algorithmic flops of one ADMM iteration for one pixel: A x, the residual,
    the clamp of u, the next v and A^T v (10 per interferogram), and the banded
    forward and back substitutions with A^T A's Cholesky factor (14 per date)."""
    return 10.0 * n_ifg + 14.0 * nx


def flops_similarity_pair(M: int) -> float:
    """Algorithmic flops of one (pixel, neighbour) similarity over the nearest-3
    network: per date the phasor product v_p conj(v_x) (6 flop) and three
    network terms Re(w_b conj w_a) (4 flop each)."""
    return 18.0 * M


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.idx)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_crop_run(z_np, window, alpha=1e-3):
    """One pass of the FP64 oracle over a crop (test infrastructure: the CPU baseline)."""
    import oracle
    N, H, W = z_np.shape
    ch = oracle.OracleChain(H, W, window, K_max=6, alpha=alpha)
    t = time.perf_counter()
    ch.step(z_np)
    return time.perf_counter() - t, (H // window[2]) * (W // window[3])


def cpu_crop(z_dev, rows: int, cols: int):
    import numpy as np
    c = z_dev[:, :rows, :cols].contiguous().cpu().numpy()
    return np.ascontiguousarray(c)


def size_cpu_sample(z_dev, target_s: float):
    """Pick a crop of the workload whose oracle run takes about target_s."""
    cols = 4096
    pilot_rows = 24
    dt, npx = oracle_crop_run(cpu_crop(z_dev, pilot_rows, cols), WINDOW)
    rate = npx / max(dt, 1e-6)
    want_px = rate * target_s
    rows = int(want_px / (cols // WINDOW[3])) * WINDOW[2]
    rows = max(WINDOW[2] * 4, min(H_FULL, rows))
    return rows, cols, rate


def run_reference(args, rank: int):
    """FP64 CPU oracle on the machine's host cores, bounded crop per step."""
    import oracle
    import torch
    from paper_2511_12051_gb300 import synth
    if rank != 0:
        return 0
    spec = synth.config_spec(1)
    # Only the crop is drawn: the generator draws row chunks in order, so the
    # first rows of a smaller image equal the full image's first rows.
    spec.H = 512
    z = synth.generate(spec, device="cpu")
    per_step_target = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    if args.ref_step_seconds is not None:
        per_step_target = args.ref_step_seconds
    rows, cols, _ = size_cpu_sample(z, per_step_target)
    rows = min(rows, spec.H - spec.H % WINDOW[2])
    crop = cpu_crop(z, rows, cols)
    for _ in range(args.warmup):
        oracle_crop_run(crop, WINDOW)
    ts = []
    npx = 0
    for _ in range(args.steps):
        dt, npx = oracle_crop_run(crop, WINDOW)
        ts.append(dt)
    mean = sum(ts) / len(ts)
    value = npx / mean
    sample = f"{rows}x{cols} px crop of the workload ({npx} output px) per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


BATCH_STACKS, BATCH_H, BATCH_W = 64, 1024, 2048


def run_batch(args, rank: int, world: int, local: int):
    """Uneven-stack batch: 64 stacks of 1024x2048 (N drawn from 5..30, gamma0
    from 0.3..0.9, 1% of the pixels in 32x32 near-singular patches), 11x5
    window, strides 6x3; one recorded CUDA graph per run, timed against the
    same stacks through one single-stack step each (the plain form)."""
    import numpy as np
    import torch
    from paper_2511_12051_gb300 import build, synth, plk
    from paper_2511_12051_gb300 import dist as pdist
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(pdist.unit_seed(2, rank))
    Ns = rng.integers(5, 31, BATCH_STACKS)
    g0 = rng.uniform(0.3, 0.9, BATCH_STACKS)
    zs = []
    for i in range(BATCH_STACKS):
        spec = synth.config_spec(2, N=int(Ns[i]), rho0=float(g0[i]), seed=int(rng.integers(1 << 30)),
                                 H=BATCH_H, W=BATCH_W)
        zs.append(synth.generate(spec, device=dev))
    stream = torch.cuda.Stream(dev)
    ctx = plk.Context(dev, stream)
    with torch.cuda.stream(stream):
        b = plk.Batch(ctx, zs, WINDOW)
        b.run()  # tunes and records
    torch.cuda.synchronize(dev)
    npx = sum(o["status"].numel() for o in b.out)

    def timed(fn, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    ms_graph = timed(b.run, args.steps)
    st = plk.State(ctx, BATCH_H, BATCH_W, WINDOW, K_max=1, M_max=30)
    with torch.cuda.stream(stream):
        outs = []
        for z in zs:  # output tensors allocated once
            st.reset()
            outs.append(st.step(z))

    def per_stack():
        for z, o in zip(zs, outs):
            st.reset()
            st.step(z, out=o)

    ms_plain = timed(per_stack, max(1, args.steps // 2))
    hist = np.zeros(5, np.int64)
    for o in b.out:
        hist += np.bincount(o["status"].view(-1).cpu().numpy(), minlength=5)[:5]
    info = b.info()
    if rank == 0:
        line = {
            "metric": METRIC, "value": npx * world / (ms_graph / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{BATCH_STACKS} uneven stacks of {BATCH_H}x{BATCH_W} px, N drawn from 5..30, "
                                   "gamma0 from 0.3..0.9, 1% near-singular 32x32 patches, 11x5 window, strides 6x3",
                       "N_per_stack": [int(n) for n in Ns], "output_px_per_gpu": npx,
                       "graph": info},
            "plain_per_stack_steps": {"value": npx * world / (ms_plain / 1e3), "unit": UNIT, "ms_per_step": ms_plain},
            "pixel_status_hist": hist.tolist(),
        }
        print(json.dumps(line), flush=True)
    b.close()
    st.close()
    return 0


def run_adjoint(args, rank: int, world: int, local: int):
    """Adjoint workload: N=20 x 1024x1024 (the 128x128 stack's coherence and ramp), 11x5
    window, stride 1, masks frozen; forward = coherence + EMI (single-precision
    solve), backward = plk_phase_link_backward of sum(w * phase), w ~ U(-1, 1);
    beside it, plk_phase_uncertainty (one adjoint solve per date and pixel) and
    plk_shp_weight_gradient (dL/dw over every window sample)."""
    import torch
    from paper_2511_12051_gb300 import build, synth, plk
    from paper_2511_12051_gb300 import dist as pdist
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    win = (5, 11, 1, 1)
    spec = synth.config_spec(4, seed=pdist.unit_seed(4, rank))
    z = synth.generate(spec, device=dev)
    N = z.shape[0]
    stream = torch.cuda.Stream(dev)
    ctx = plk.Context(dev, stream)
    with torch.cuda.stream(stream):
        P, _ = ctx.amp_stats(z)
        mask, _ = ctx.shp_select(P, N, win, 1e-3)
        prm = plk.default_params(fp64_resolve=0)
        C = ctx.estimate_covariance(z, win, mask)
        out = ctx.phase_link(C, N, 0, prm)
        g = torch.Generator(device=dev).manual_seed(4)
        w = torch.rand(out["phase"].shape, device=dev, generator=g) * 2 - 1
        dz = ctx.phase_link_backward(z, win, mask, 0, w, prm)
        sd = ctx.phase_uncertainty(z, win, mask, 0, 0.01, prm)
        dwt = ctx.shp_weight_gradient(z, win, mask, 0, w, prm)
    torch.cuda.synchronize(dev)

    def fwd():
        ctx.estimate_covariance(z, win, mask, C=C)
        ctx.phase_link(C, N, 0, prm)

    def bwd():
        ctx.phase_link_backward(z, win, mask, 0, w, prm, dslc=dz)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            e0.record(stream)
            for _ in range(args.steps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / args.steps

    def unc():
        ctx.phase_uncertainty(z, win, mask, 0, 0.01, prm, out=sd)

    def wgrad():
        ctx.shp_weight_gradient(z, win, mask, 0, w, prm, out=dwt)

    ms_f, ms_b, ms_u, ms_w = timed(fwd), timed(bwd), timed(unc), timed(wgrad)
    ctx.profile(True)
    with torch.cuda.stream(stream):
        for _ in range(2):
            bwd()
    torch.cuda.synchronize(dev)
    stages = {kk: v[0] / 2 for kk, v in ctx.profile_collect().items()}
    ctx.profile(False)
    npx = out["status"].numel()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": npx * world / (ms_b / 1e3), "unit": "output px/s (backward)", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "adjoint: N=20 x 1024x1024, 11x5 window, stride 1, masks frozen, "
                                   "L = sum(w * phase), w ~ U(-1, 1)", "output_px_per_gpu": npx},
            "forward_ms": ms_f, "backward_ms": ms_b, "backward_over_forward": ms_b / ms_f,
            "backward_stages_ms": stages,
            "forward_px_per_s": npx * world / (ms_f / 1e3),
            "uncertainty_ms": ms_u, "uncertainty_px_per_s": npx * world / (ms_u / 1e3),
            "weight_gradient_ms": ms_w}), flush=True)
    return 0


def run_chain(args, rank: int, world: int, local: int):
    """Sequential chain: 60 dates of 2048x4096 (the +2 rad patch from date 31)
    through four mini-stacks of 15 new SLCs, stride 1, keeping 3 compressed
    SLCs (N = 15, 16, 17, 18 per step).  Each timed pass runs the whole chain
    from a reset state; reported per step and for the chain."""
    import torch
    from paper_2511_12051_gb300 import build, synth, plk
    from paper_2511_12051_gb300 import dist as pdist
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    spec = synth.config_spec(3, seed=pdist.unit_seed(3, rank))
    z = synth.generate(spec, device=dev)
    win, K_max, M = (5, 11, 1, 1), 3, 15
    slices = synth.ministack_slices(spec.N, M)
    parts = [z[sl].contiguous() for sl in slices]
    stream = torch.cuda.Stream(dev)
    ctx = plk.Context(dev, stream)
    st = plk.State(ctx, spec.H, spec.W, win, K_max=K_max, M_max=M)
    with torch.cuda.stream(stream):
        outs = []
        for zz in parts:
            outs.append(st.step(zz))
    torch.cuda.synchronize(dev)
    npx = st.Ho * st.Wo

    def chain():
        st.reset()
        for zz, o in zip(parts, outs):
            st.step(zz, out=o)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            chain()
    torch.cuda.synchronize(dev)
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pdist.barrier()
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            chain()
        e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_chain = pdist.max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    stages = {kk: v[0] / args.steps for kk, v in ctx.profile_collect().items()}
    ctx.profile(False)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": len(slices) * npx * world / (ms_chain / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_chain,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sequential chain: 60 dates of 2048x4096 (+2 rad patch from date 31), 4 mini-stacks "
                                   "of 15, K_max 3 (N = 15..18 per step), 11x5 window, stride 1",
                       "output_px_per_step": npx, "steps_per_chain": len(slices)},
            "ms_per_chain": ms_chain, "ms_per_ministack_step": ms_chain / len(slices),
            "stages_ms_per_chain": stages}), flush=True)
    st.close()
    return 0


def run_small(args, rank: int, world: int, local: int):
    """The 128x128 stack (N = 10, 11x5 window, stride 1): launch- and
    latency-bound; one step reported in microseconds and pixels/s."""
    import torch
    from paper_2511_12051_gb300 import build, synth, plk
    from paper_2511_12051_gb300 import dist as pdist
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    z = synth.generate(synth.config_spec(0, seed=pdist.unit_seed(0, rank)), device=dev)
    stream = torch.cuda.Stream(dev)
    ctx = plk.Context(dev, stream)
    st = plk.State(ctx, 128, 128, (5, 11, 1, 1), K_max=6, M_max=10)
    with torch.cuda.stream(stream):
        out = st.step(z)
    torch.cuda.synchronize(dev)

    def one():
        st.reset()
        st.step(z, out=out)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(args.steps, 100)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            one()
        e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = pdist.max_over_ranks(e0.elapsed_time(e1) / reps, dev)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": 128 * 128 * world / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": reps, "warmup": args.warmup, "ms_per_step": ms, "us_per_step": ms * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "N=10 x 128x128, 11x5 window, stride 1 (launch- and latency-bound)",
                       "output_px_per_gpu": 128 * 128}}), flush=True)
    st.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="plk", choices=["plk", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-e2e-ci16", action="store_true",
                    help="leave out the host-buffer step with complex 16-bit input")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=None,
                    help="CPU seconds of oracle work per step of the reference arm (default: 2-20 s, "
                         "so that the whole run takes a few minutes)")
    ap.add_argument("--rows", type=int, default=H_FULL, help="image rows (smaller cases for profiling only)")
    ap.add_argument("--cols", type=int, default=W_FULL, help="image columns (smaller cases for profiling only)")
    ap.add_argument("--cov-precision", default="fp32", choices=["fp32", "bf16", "fp16"],
                    help="coherence arithmetic of the timed step (fp32: the plain path)")
    ap.add_argument("--no-modes", action="store_true",
                    help="skip timing the reduced-precision, PS, gamma_s and L1-inversion modes beside it")
    ap.add_argument("--ps-da-max", type=float, default=0.0,
                    help="PS threshold on the amplitude dispersion in the timed step (0: no PS regridding)")
    ap.add_argument("--workload", default="burst", choices=["burst", "batch", "adjoint", "chain", "small"],
                    help="burst: the headline mini-stack step; batch: 64 uneven stacks in one recorded graph; "
                         "adjoint: forward and backward of the phase linking on N=20 x 1024x1024; chain: 60 dates "
                         "of 2048x4096 in four mini-stacks; small: N=10 x 128x128")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    from paper_2511_12051_gb300 import dist as pdist
    rank, world, local = pdist.rank_info()

    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == "batch":
        return run_batch(args, rank, world, local)
    if args.workload == "adjoint":
        return run_adjoint(args, rank, world, local)
    if args.workload == "chain":
        return run_chain(args, rank, world, local)
    if args.workload == "small":
        return run_small(args, rank, world, local)

    import torch
    import torch.distributed as dist
    from paper_2511_12051_gb300 import build, synth
    build.build()
    from paper_2511_12051_gb300 import plk

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    # Each rank processes its own burst (weak scaling; no data-path collective).
    spec = synth.config_spec(1, seed=pdist.unit_seed(1, rank), H=args.rows, W=args.cols)
    z = synth.generate(spec, device=dev)
    stream = torch.cuda.Stream(dev)
    ctx = plk.Context(dev, stream)
    st = plk.State(ctx, spec.H, spec.W, WINDOW, K_max=6, M_max=N_DATES)
    prec = {"fp32": plk.COV_FP32, "bf16": plk.COV_BF16, "fp16": plk.COV_FP16}[args.cov_precision]
    params = plk.default_params(cov_precision=prec, ps_da_max=args.ps_da_max)
    with torch.cuda.stream(stream):
        out = st.step(z, params)  # allocates the output tensors once
    torch.cuda.synchronize(dev)
    Ho, Wo = st.Ho, st.Wo
    npx = Ho * Wo

    def one_step():
        st.reset()
        st.step(z, params, out=out)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
    torch.cuda.synchronize(dev)
    looks_total = float(out["count"].view(torch.int16).to(torch.int32).sum().item())  # SHP looks, all pixels
    status_hist = torch.bincount(out["status"].view(-1).to(torch.int64), minlength=5).tolist()

    # ---------------------------------------------------------- timed region
    clocks = ClockSampler(local)
    ctx.profile(True)
    pdist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            one_step()
        e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    kernels = ctx.profile_collect()
    ctx.profile(False)
    ms_total = pdist.max_over_ranks(ms_total, dev)
    ms_step = ms_total / args.steps
    value = npx * world * args.steps / (ms_total / 1e3)
    launches = sum(c for _, c in kernels.values())

    # ------------------------------------------------------------- roofline
    peaks = measured_peaks()
    dom = max(kernels.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n) = dom
    dom_avg_s = dom_ms / dom_n / 1e3
    if dom_name == "covariance":
        work = flops_covariance(N_DATES, looks_total)
        roof = {"bound": "alu", "achieved": work / dom_avg_s / 1e12, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2.070 GHz"}
    elif dom_name.startswith("phase_link"):
        work = flops_emi(N_DATES, npx)
        roof = {"bound": "alu", "achieved": work / dom_avg_s / 1e12, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2.070 GHz"}
    else:
        nbytes = {"amp_stats": N_DATES * spec.H * spec.W * 8 + spec.H * spec.W * 8,
                  "compress": N_DATES * spec.H * spec.W * 8 + spec.H * spec.W * 8,
                  "shp_select": spec.H * spec.W * 4 + npx * 10}.get(dom_name, 0)
        hbm = peaks.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": nbytes / dom_avg_s / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"}
    roof["kernel"] = dom_name
    roof["frac"] = roof["achieved"] / roof["peak"]
    per_px = NCU_DRAM_BYTES_PER_OUTPUT_PX.get(dom_name)
    roof["traffic"] = per_px * npx if (per_px and args.rows == H_FULL and args.cols == W_FULL) else None
    roof["avg_launch_ms"] = dom_ms / dom_n

    # Whole step against its roofline: a kernel's ideal time is the larger of its
    # algorithmic flops at the FP32 peak and its algorithmic bytes at the HBM
    # peak; the fraction is the sum of the ideal times over the measured step.
    hbm_bs = peaks.get("hbm_gbs", 6800.0) * 1e9
    plane = spec.H * spec.W
    ntri = N_DATES * (N_DATES + 1) // 2
    ideal = {
        "amp_stats": (0.0, N_DATES * plane * 8 + plane * 8),
        "shp_select": (0.0, plane * 4 + npx * 10),
        "covariance": (flops_covariance(N_DATES, looks_total), N_DATES * plane * 8 + npx * 8 + npx * ntri * 8),
        "phase_link_fp32": (flops_emi(N_DATES, npx), npx * ntri * 8 + npx * (4 * N_DATES + 5)),
        "phase_link_fp64": (0.0, npx),
        "compress": (0.0, N_DATES * plane * 8 + plane * 8),
    }
    t_ideal = {kk: max(f / (FP32_PEAK_TFLOPS * 1e12), b / hbm_bs) * 1e3 for kk, (f, b) in ideal.items()}
    step_roof = {"ideal_ms": sum(t_ideal.values()), "step_ms": ms_step,
                 "frac": sum(t_ideal.values()) / ms_step,
                 "ideal_ms_by_kernel": t_ideal,
                 "model": "per kernel max(algorithmic flops / FP32 peak, algorithmic bytes / HBM peak), summed"}

    # ------------------------------------------------------------------ e2e
    # Through the C ABI with host buffers (plk_ministack_step_host): every step
    # copies its 15 SLCs from pinned host memory and writes phases, gamma_t and
    # status back to pinned host memory; a step's copy overlaps the previous
    # step's compute inside the library.
    e2e = None
    e2e_ci16 = None
    if not args.no_e2e:
        zh = torch.empty(z.shape, dtype=z.dtype, pin_memory=True)
        zh.copy_(z)
        oh = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items() if k != "count"}
        oh["count"] = None
        bi = zh.numel() * zh.element_size()
        bo = sum(v.numel() * v.element_size() for v in oh.values() if v is not None)

        st.enable_host_io()

        def e2e_step():
            st.reset()
            st.step_host(zh, params, out=oh)

        e2e_step()
        ctx.sync()
        torch.cuda.synchronize(dev)
        # The host link's rate at this moment (it is shared with the other GPUs
        # of the node): one plain pinned-host -> device copy of the same bytes.
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            l0.record(stream)
            z.copy_(zh, non_blocking=True)
            l1.record(stream)
        torch.cuda.synchronize(dev)
        link_gbs = bi / (l0.elapsed_time(l1) / 1e3) / 1e9
        pdist.barrier()
        # An event on the compute stream after each call marks when that step's
        # outputs are back in host memory: the first interval holds the first
        # copy and the first step back to back (nothing to overlap yet), the
        # later ones the steady state, where the copy of step i+1 runs under
        # the compute of step i.
        ne = max(2, min(2 * args.steps, 20))
        fe = [torch.cuda.Event(enable_timing=True) for _ in range(ne + 1)]
        fe[0].record(stream)
        for i in range(ne):
            e2e_step()
            fe[i + 1].record(stream)
        ctx.sync()
        torch.cuda.synchronize(dev)
        ms_e2e = pdist.max_over_ranks(fe[0].elapsed_time(fe[ne]), dev)
        iv = [fe[i].elapsed_time(fe[i + 1]) for i in range(ne)]
        steady = sorted(iv[1:])[len(iv[1:]) // 2] if ne > 1 else iv[0]
        e2e = {"value": npx * world * ne / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "steps": ne, "ms_per_step": ms_e2e / ne,
               "first_step_ms": iv[0], "steady_median_ms": steady, "compute_alone_ms": ms_step,
               "intervals_ms": [round(v, 1) for v in iv],
               "h2d_link_gbs": link_gbs, "input_copy_bound_ms": bi / (link_gbs * 1e9) * 1e3}
        del zh

        # The same through plk_ministack_step_host_ci16: the SLCs as complex
        # 16-bit integers (Sentinel-1's sample format), half the bytes over
        # the host link, widened on the device.  The workload quantised once,
        # outside the timed region: round(2048 z) (|z| stays below 16 here).
        e2e_ci16 = None
        if not args.no_e2e_ci16:
            with torch.cuda.stream(stream):
                qd = torch.stack([torch.round(z.real * 2048.0), torch.round(z.imag * 2048.0)], dim=-1)
                qd = qd.clamp_(-32768, 32767).to(torch.int16)
            torch.cuda.synchronize(dev)
            qh = torch.empty(qd.shape, dtype=torch.int16, pin_memory=True)
            qh.copy_(qd)
            del qd
            bq = qh.numel() * qh.element_size()
            st.enable_host_io_ci16()

            def e2e_step16():
                st.reset()
                st.step_host_ci16(qh, params, out=oh)

            e2e_step16()
            ctx.sync()
            torch.cuda.synchronize(dev)
            pdist.barrier()
            fq = [torch.cuda.Event(enable_timing=True) for _ in range(ne + 1)]
            fq[0].record(stream)
            for i in range(ne):
                e2e_step16()
                fq[i + 1].record(stream)
            ctx.sync()
            torch.cuda.synchronize(dev)
            ms_q = pdist.max_over_ranks(fq[0].elapsed_time(fq[ne]), dev)
            ivq = [fq[i].elapsed_time(fq[i + 1]) for i in range(ne)]
            e2e_ci16 = {"value": npx * world * ne / (ms_q / 1e3), "unit": UNIT, "h2d_bytes_per_step": bq,
                        "d2h_bytes_per_step": bo, "steps": ne, "ms_per_step": ms_q / ne,
                        "first_step_ms": ivq[0],
                        "steady_median_ms": sorted(ivq[1:])[len(ivq[1:]) // 2] if ne > 1 else ivq[0],
                        "intervals_ms": [round(v, 1) for v in ivq],
                        "input": "complex int16 samples round(2048 z) of the same workload, widened exactly on "
                                 "the device (plk_ministack_step_host_ci16)"}
            del qh
        del oh

    # ------------------------- other modes of the same step, timed beside it
    def time_mode(alt):
        def alt_step():
            st.reset()
            st.step(z, alt, out=out)

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                alt_step()
        torch.cuda.synchronize(dev)
        ctx.profile(True)
        pdist.barrier()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            g0.record(stream)
            for _ in range(args.steps):
                alt_step()
            g1.record(stream)
        torch.cuda.synchronize(dev)
        kalt = ctx.profile_collect()
        ctx.profile(False)
        ms_alt = pdist.max_over_ranks(g0.elapsed_time(g1), dev)
        return {"value": npx * world * args.steps / (ms_alt / 1e3), "unit": UNIT, "ms_per_step": ms_alt / args.steps,
                "kernels_ms_per_step": {kk: v[0] / args.steps for kk, v in kalt.items()}}

    def time_similarity():
        # gamma_s of the step's linked phases over the ~200 m window (radius 7 at the 30 m posting)
        one_step()
        ph = out["phase"]
        gs = torch.empty((Ho, Wo), dtype=torch.float32, device=dev)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                ctx.phase_similarity(ph, GS_RADIUS, gs)
        torch.cuda.synchronize(dev)
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            h0.record(stream)
            for _ in range(args.steps):
                ctx.phase_similarity(ph, GS_RADIUS, gs)
            h1.record(stream)
        torch.cuda.synchronize(dev)
        ms = h0.elapsed_time(h1) / args.steps
        n_nb = len([1 for dy in range(-GS_RADIUS, GS_RADIUS + 1) for dx in range(-GS_RADIUS, GS_RADIUS + 1)
                    if 0 < dy * dy + dx * dx <= GS_RADIUS ** 2])
        flop = npx * n_nb * flops_similarity_pair(N_DATES)
        return {"value": npx * world / (ms / 1e3), "unit": UNIT, "ms_per_call": ms, "radius": GS_RADIUS,
                "neighbours": n_nb, "median_gamma_s": float(torch.nanmedian(gs).item()),
                "roofline": {"bound": "alu", "achieved": flop / (ms / 1e3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                             "unit": "TFLOP/s", "frac": flop / (ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                             "work": "18 flop per date and neighbour (phasor product, three network terms)"}}

    def time_inversion():
        # L1 ADMM inversion of the nearest-3 network of the 15 real dates at every
        # output pixel: synthetic unwrapped phases A x + 2 pi k (2% wrong
        # interferograms) + noise, drawn on the device from a seeded generator.
        pairs = [(a, a + d) for d in (1, 2, 3) for a in range(N_DATES - d)]
        nx = N_DATES - 1
        g = torch.Generator(device=dev)
        g.manual_seed(pdist.unit_seed(7, rank))
        xt = torch.cumsum(1.5 * torch.randn((nx, npx), generator=g, device=dev), dim=0)
        xt = torch.cat([torch.zeros((1, npx), device=dev), xt])
        ia = torch.tensor([p[0] for p in pairs], device=dev)
        ib = torch.tensor([p[1] for p in pairs], device=dev)
        wrong = (torch.rand((len(pairs), npx), generator=g, device=dev) < 0.02).float()
        sign = torch.where(torch.rand((len(pairs), npx), generator=g, device=dev) < 0.5, -1.0, 1.0)
        unw = (xt[ib] - xt[ia] + 2 * math.pi * wrong * sign
               + 0.3 * torch.randn((len(pairs), npx), generator=g, device=dev)).contiguous()
        del xt, wrong, sign
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                ctx.invert_l1(unw, N_DATES, pairs, rho=1.0, iters=ADMM_ITERS)
        torch.cuda.synchronize(dev)
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            h0.record(stream)
            for _ in range(args.steps):
                ctx.invert_l1(unw, N_DATES, pairs, rho=1.0, iters=ADMM_ITERS)
            h1.record(stream)
        torch.cuda.synchronize(dev)
        ms = h0.elapsed_time(h1) / args.steps
        flop = npx * ADMM_ITERS * flops_admm_iteration(len(pairs), nx)
        del unw
        return {"value": npx * world / (ms / 1e3), "unit": UNIT, "ms_per_call": ms, "n_ifg": len(pairs),
                "iters": ADMM_ITERS, "rho": 1.0,
                "roofline": {"bound": "alu", "achieved": flop / (ms / 1e3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                             "unit": "TFLOP/s", "frac": flop / (ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                             "work": "10 flop per interferogram and 14 per date, per pixel and iteration"}}

    modes = None
    if not args.no_modes and prec == plk.COV_FP32 and args.ps_da_max == 0:
        modes = {}
        modes["bf16_covariance"] = time_mode(plk.default_params(cov_precision=plk.COV_BF16))
        modes["bf16_covariance"]["accuracy"] = ("measured against the FP64 oracle by tests/test_gpu_bf16.py "
                                                "(linked-phase p50/p99/max)")
        modes["fp16_covariance"] = time_mode(plk.default_params(cov_precision=plk.COV_FP16))
        modes["fp16_covariance"]["accuracy"] = ("measured against the FP64 oracle by tests/test_gpu_fp16.py "
                                                "(linked-phase p50/p99/max)")
        modes["ps_regrid"] = time_mode(plk.default_params(ps_da_max=PS_DA_MAX))
        modes["ps_regrid"]["ps_da_max"] = PS_DA_MAX
        modes["ps_regrid"]["ps_cells"] = int((out["status"] == plk.PX_PS).sum().item())
        modes["ps_regrid"]["output_cells"] = npx
        modes["gamma_s"] = time_similarity()
        modes["l1_inversion"] = time_inversion()

    # ---------------------------------------------------------- CPU baseline
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        rows, cols, _ = size_cpu_sample(z, args.cpu_seconds)
        crop = cpu_crop(z, rows, cols)
        dt, cnpx = oracle_crop_run(crop, WINDOW)
        cpu = {"value": cnpx / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{rows}x{cols} px crop of the workload ({cnpx} output px), {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if (spec.H, spec.W) == (H_FULL, W_FULL) else
                       f"profiling case {spec.H}x{spec.W} (not the headline workload)", "N": N_DATES,
                       "H": spec.H, "W": spec.W,
                       "window_wy_wx_sy_sx": list(WINDOW), "output_px_per_gpu": npx,
                       "l2": "inputs (8.05 GB per step) larger than L2; no flush",
                       "parallelism": f"{world} independent bursts, one per GPU"},
            "roofline": roof,
            "step_roofline": step_roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "e2e_ci16": e2e_ci16,
            "gpu_launches": launches,
            "clocks": clk,
            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in kernels.items()},
            "pixel_status_hist": status_hist,
            "cov_precision": args.cov_precision,
            "ps_da_max": args.ps_da_max,
            "modes": modes,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        pdist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
