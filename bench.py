#!/usr/bin/env python3
"""Frames/s to the full structure function D(q, dt) of a 512x512 uint16 stack, N = 1024.

One step = one pass of the whole hot path through the C ABI on one synthetic stack:
  ddm_spatial_fft   (step one: real-to-complex 2D DFT of every frame, 2 kernels)
  ddm_temporal_sf   (step two: per-q power sums + zero-padded transform in time, 1 kernel)
  ddm_azimuthal_average (radial average over 362 |q| bins, 1 kernel)
  ddm_fit           (Levenberg-Marquardt of every radial curve, 2 kernels)
After the timed steps, the learned fit stage is measured: the seed network is trained with
the library's own kernels on the radial curves of 200 seeded polydisperse blob stacks that
this pipeline computes, then plain LM and network-seeded LM are compared on 20 held-out
stacks and on the bench stack.
The frames (537 MB) and the spectrum (1.08 GB) are larger than L2, so no flush is needed
between timed steps.

Prints ONE JSON line.  --impl reference times the FP64 CPU oracle instead, on a bounded
sample of the same workload (one kx column of the spectrum, every ky, every lag),
extrapolated linearly in the number of wave vectors.
Under torchrun (N > 1) every rank processes its own stack (independent replicas, weak
scaling, no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

H = W = 512
N_FRAMES = 1024
N_BINS = 362
WORKLOAD = "blobs_512x512x1024_u16"
METRIC = "frames/s to full D(q,Δt) at 512²×1024, % of HBM roofline, max rel err vs FP64"
FALLBACK_HBM_GBS = 6400.0
N_Q = H * (W // 2 + 1)
SPATIAL_BYTES = N_FRAMES * H * W * 2 + N_Q * N_FRAMES * 8      # read frames, write spectrum
TEMPORAL_BYTES = N_Q * N_FRAMES * 8 + N_Q * N_FRAMES * 4       # read spectrum, write D
STEP_BYTES = SPATIAL_BYTES + TEMPORAL_BYTES


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fit-compare", action="store_true")
    ap.add_argument("--no-camera", action="store_true",
                    help="skip the 600x800x3000 (non-power-of-two sides) timing")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 tier timing")
    ap.add_argument("--sweep", action="store_true",
                    help="also time the image-size sweep 128^2 .. 2048^2 at N = 16384 (4096 at 2048^2)")
    ap.add_argument("--split", choices=["none", "kx"], default="none",
                    help="kx: one stack split across the ranks by kx columns (strong scaling): "
                         "each rank transforms every row, its own columns and their time "
                         "sequences; the radial sums are all-reduced")
    ap.add_argument("--no-precision-sweep", action="store_true",
                    help="skip the 1024x1024x4096 float32 precision sweep (three tiers)")
    ap.add_argument("--crossover", action="store_true",
                    help="also time WITH_FT vs WITHOUT_FT step two at the frame side (512^2 unless "
                         "--shape) for N = 128 .. 16384")
    ap.add_argument("--crossover-ns", default="128,256,512,1024,2048,4096,8192,16384",
                    help="stack lengths of the crossover sweep (comma-separated)")
    ap.add_argument("--no-long", action="store_true",
                    help="skip the 512x512x16384 (longest stacks) timing")
    ap.add_argument("--kmax", type=int, default=63,
                    help="also time the low-frequency restriction |ky'|, kx <= kmax (0 = skip)")
    ap.add_argument("--shape", default=None,
                    help="HxWxN of a smaller blob stack for profiling captures (default 512x512x1024)")
    args = ap.parse_args()
    if args.shape:
        global H, W, N_FRAMES, N_Q, SPATIAL_BYTES, TEMPORAL_BYTES, STEP_BYTES, WORKLOAD
        H, W, N_FRAMES = (int(x) for x in args.shape.lower().split("x"))
        N_Q = H * (W // 2 + 1)
        SPATIAL_BYTES = N_FRAMES * H * W * 2 + N_Q * N_FRAMES * 8
        TEMPORAL_BYTES = N_Q * N_FRAMES * 8 + N_Q * N_FRAMES * 4
        STEP_BYTES = SPATIAL_BYTES + TEMPORAL_BYTES
        WORKLOAD = f"blobs_{H}x{W}x{N_FRAMES}_u16"
    return args


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's time (every rank gets it): the job is done when the last rank is."""
    if dist is None:
        return ms
    import torch
    tt = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(n_ranks, frames_per_rank, steps, ms_total):
    """Whole-job frames/s: every rank processes its own stacks (replicas), so the units all
    ranks processed over the slowest rank's time."""
    return n_ranks * frames_per_rank * steps / (ms_total / 1e3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("ddm_temporal.cu", "ddm_fft.cuh", "ddm_internal.h"):
        with open(os.path.join(ROOT, "paper_2012_05695_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the temporal kernel from the committed ncu summary, or None
    when the kernel source changed since that capture."""
    p = os.path.join(ROOT, "profiles", "temporal_sf_512x512x1024.md")
    if not os.path.exists(p):
        return None
    src = None
    bytes_ = None
    for line in open(p):
        if line.startswith("source_sha256_16:"):
            src = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            bytes_ = float(line.split(":", 1)[1].strip())
    if src != kernel_source_hash():
        return None
    return bytes_


class ClockSampler:
    """nvidia-smi samples (every 50 ms) while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        return time.time()

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.12)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [l for (ts, l) in self.lines if t0 - 0.06 <= ts <= t1 + 0.06]
        if not rows and self.lines:
            rows = [min(self.lines, key=lambda x: abs(x[0] - (t0 + t1) / 2))[1]]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            parts = [p.strip() for p in r.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo), or None."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def oracle_sample(frames, cols, nthreads):
    """Run the FP64 oracle on kx columns `cols` (every ky, every lag); returns (seconds, D, s_q)."""
    import oracle
    t0 = time.perf_counter()
    D, s_q = oracle.structure_function(frames, kx_sel=cols, nthreads=nthreads)
    return time.perf_counter() - t0, D, s_q


def time_mlp_forward(mlp, x, sizes, reps=50):
    """Device time of the MLP forward (tensor cores), per batch size: a CUDA graph of `reps`
    calls replayed under CUDA events, so that the Python call path is not timed.  Roofline:
    the network's algorithmic FLOPs (one pass, 2 B (64*128 + 2*128*128 + 128*4)) over the
    measured bf16 tensor peak."""
    import torch
    peak = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            peak = float(json.load(f)["bf16_tflops"])
    s = torch.cuda.Stream()
    res = {}
    for Bn in sizes:
        xb = x[:Bn * 64]
        o = torch.empty(Bn * 4, device="cuda")
        with torch.cuda.stream(s):
            for _ in range(3):
                mlp.forward(xb, Bn, o, s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
            for _ in range(reps):
                mlp.forward(xb, Bn, o, s)
        ts = []
        with torch.cuda.stream(s):          # replay() launches on the current stream
            for _ in range(3):
                g.replay()
            torch.cuda.synchronize()
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                g.replay()
                e1.record(s)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e3 / reps)
        us = statistics.median(ts)
        flops = 2.0 * Bn * (64 * 128 + 2 * 128 * 128 + 128 * 4)
        tf = flops / (us * 1e-6) / 1e12
        res[str(Bn)] = {"us": us, "ctas": (Bn + 127) // 128, "tflops": tf,
                        "frac_of_bf16_peak": (tf / peak) if peak else None}
    res["peak_bf16_tflops"] = peak
    res["bound"] = "latency: one 128-sample CTA per SM runs three dependent MMA batches"
    assert mlp.last_device_status() == 0
    return res


from paper_2012_05695_b300.seed_training import head_targets  # noqa: E402  (re-exported)


def compare_fits(ddm, plan, Dr, stream, n_train=200, n_held=20, n_keep=256, steps=6000, batch=4096):
    """The learned fit stage on structure functions this pipeline computes: seeded
    polydisperse blob stacks (512x512x1024, log-normal D0, median 0.2, sigma_ln 0.5; seeds
    1000.. train, 2000.. held out) go through ddm_structure_function and the radial
    average; the curves inside the inscribed Nyquist circle (the first n_keep of 362 bins)
    are labelled by LM and train the seed network with the library's kernels; then plain LM
    and LM seeded by the network fit the held-out stacks' curves and this run's own bench
    stack (its 362 radial curves)."""
    import torch
    import synth
    from paper_2012_05695_b300 import seed_training as st
    dev = Dr.device
    D = torch.empty(plan.d_rows * N_FRAMES, dtype=torch.float32, device=dev)
    Dr_s = torch.empty(N_BINS * N_FRAMES, dtype=torch.float32, device=dev)

    def curves(seeds):
        cs = []
        for sd in seeds:
            fr = synth.polydisperse_blobs_512x512x1024(sd, N=N_FRAMES, H=H, W=W, device=dev)
            cs.append(st.stack_curves(plan, fr, n_keep, stream, D, Dr_s))
            del fr
        return torch.cat(cs, dim=0).contiguous()

    t0 = time.perf_counter()
    train_curves = curves(range(1000, 1000 + n_train))
    held = curves(range(2000, 2000 + n_held))
    t_data = time.perf_counter() - t0
    x, tgt, keep = st.labelled_features(plan, train_curves, stream)
    mlp = ddm.MLP(batch)
    mlp.set_weights(synth.mlp_init(0))
    t0 = time.perf_counter()
    loss0, loss1 = st.train(mlp, x, tgt, steps, batch, seed=0, stream=stream)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    out = {"training_data": (f"{n_train} polydisperse blob stacks {H}x{W}x{N_FRAMES} (seeds 1000..), "
                             f"{n_keep} radial curves each, labelled by LM"),
           "training_curves": int(keep.size), "labelled": int(keep.sum()),
           "data_s": t_data, "train_steps": steps, "train_batch": batch, "train_s": train_s,
           "train_loss_first": loss0, "train_loss": loss1,
           "held_out": dict(st.compare(plan, held, mlp, stream), stacks=n_held),
           "bench_stack": st.compare(plan, Dr.view(N_BINS, N_FRAMES), mlp, stream),
           "mlp_forward": time_mlp_forward(mlp, x.view(-1), (N_BINS, batch))}
    for name, mode, net in (("lm", ddm._binding.DDM_FIT_LM, None), ("mlp_lm", ddm._binding.DDM_FIT_MLP_LM, mlp)):
        prm = torch.empty(N_BINS * 4, device=dev)
        for _ in range(3):
            plan.fit(Dr, N_BINS, mode, net, prm, None, None, None, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            plan.fit(Dr, N_BINS, mode, net, prm, None, None, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out["bench_stack"][name + "_ms"] = e0.elapsed_time(e1) / 20
    mlp.close()
    return out


def time_camera(ddm, dev, stream, seed, H=600, W=800, N=3000, n_bins=500, steps=5):
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    frames = torch.randint(1800, 2201, (N, H, W), generator=g, device=dev, dtype=torch.int16).view(torch.uint16)
    plan = ddm.Plan(H, W, N, dtype="u16", n_bins=n_bins)
    D = torch.empty(plan.n_q * N, dtype=torch.float32, device=dev)
    Dr = torch.empty(n_bins * N, dtype=torch.float32, device=dev)
    # both steps through ddm_structure_function (its own workspace: step one writes the
    # blocked copy the time kernels read), stage times from the plan's CUDA events
    plan.enable_stats(True)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    one = two = 0.0
    for k in range(3 + steps):
        e = ev[k - 3] if k >= 3 else None
        if e:
            e[0].record(stream)
        plan.structure_function(frames, D, stream)
        if e:
            e[1].record(stream)
        plan.azimuthal_average(D, Dr, None, stream)
        if e:
            e[2].record(stream)
            a, b = plan.stats()
            one += a
            two += b
    torch.cuda.synchronize()
    sf_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / steps
    ms = [one / steps, two / steps, sum(e[1].elapsed_time(e[2]) for e in ev) / steps]
    status = plan.last_device_status()
    plan.close()
    return {"workload": f"camera_{H}x{W}x{N}_u16", "H": H, "W": W, "N": N, "n_bins": n_bins,
            "structure_function_ms": sf_ms,
            "frames": "uniform counts 1800..2200 drawn on the device (timing only)",
            "spatial": "mixed-radix rows (800 = 25 x 32) and columns (600 = 24 x 25)",
            "stages_ms": {"spatial_fft": ms[0], "temporal_sf": ms[1], "azimuthal_average": ms[2]},
            "frames_per_s": N / ((sf_ms + ms[2]) / 1e3), "device_status": status, "steps": steps}


def time_long_stack(ddm, dev, stream, seed, H=512, W=512, N=16384, steps=3):
    """The paper's longest stacks (N = 2^14, 16384-point time transforms): step one and
    step two on device-drawn counts (timing only)."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    frames = torch.randint(1800, 2201, (N, H, W), generator=g, device=dev, dtype=torch.int16).view(torch.uint16)
    plan = ddm.Plan(H, W, N, dtype="u16")
    D = torch.empty(plan.n_q * N, dtype=torch.float32, device=dev)
    plan.enable_stats(True)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
    one = two = 0.0
    for k in range(2 + steps):
        e = ev[k - 2] if k >= 2 else None
        if e:
            e[0].record(stream)
        plan.structure_function(frames, D, stream)
        if e:
            e[1].record(stream)
            a, b = plan.stats()
            one += a
            two += b
    torch.cuda.synchronize()
    ms = [one / steps, two / steps]
    status = plan.last_device_status()
    plan.close()
    del frames, D
    torch.cuda.empty_cache()
    return {"workload": f"long_{H}x{W}x{N}_u16", "H": H, "W": W, "N": N,
            "frames": "uniform counts 1800..2200 drawn on the device (timing only)",
            "stages_ms": {"spatial_fft": ms[0], "temporal_sf": ms[1]},
            "frames_per_s": N / (sum(ms) / 1e3), "device_status": status, "steps": steps}


def crossover_sweep(ddm, dev, stream, seed, side=512,
                    Ns=(128, 256, 512, 1024, 2048, 4096, 8192, 16384)):
    """The paper's comparison of its two schemes (Sec. 2, Figs. 1 and 3) on this GPU: per
    stack length N, step one once, then step two by the Fourier route (ddm_temporal_sf) and
    by explicit frame differences (ddm_temporal_sf_direct, WITHOUT_FT) on the same spectrum;
    frames drawn on the device (timing only).  Returns the per-N times and the smallest N
    at which the Fourier route's whole stack (step one + step two) is faster."""
    import torch
    rows = []
    for N in Ns:
        g = torch.Generator(device=dev)
        g.manual_seed(seed + N)
        frames = torch.randint(1800, 2201, (N, side, side), generator=g, device=dev,
                               dtype=torch.int16).view(torch.uint16)
        plan = ddm.Plan(side, side, N, dtype="u16")
        spec = torch.empty(2 * N * plan.n_q, dtype=torch.float32, device=dev)
        D = torch.empty(plan.n_q * N, dtype=torch.float32, device=dev)
        reps = 5 if N <= 2048 else (2 if N <= 8192 else 1)

        def timed(fn, reps=reps):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        sp = timed(lambda: plan.spatial_fft(frames, spec, stream))
        ft = timed(lambda: plan.temporal_sf(spec, D, stream))
        dr = timed(lambda: plan.temporal_sf_direct(spec, D, stream))
        status = plan.last_device_status()
        rows.append({"N": N, "spatial_ms": sp, "temporal_ft_ms": ft, "temporal_direct_ms": dr,
                     "with_ft_ms": sp + ft, "without_ft_ms": sp + dr,
                     "speedup_with_ft": (sp + dr) / (sp + ft), "device_status": status})
        plan.close()
        del frames, spec, D
        torch.cuda.empty_cache()
    wins = [r["N"] for r in rows if r["speedup_with_ft"] > 1.0]
    return {"side": side, "rows": rows,
            "frames": "uniform counts 1800..2200 drawn on the device (timing only)",
            "with_ft_faster_from_N": min(wins) if wins else None}


def image_size_sweep(ddm, dev, stream, seed):
    """The paper's second workload (Fig. 3 shape): frame sides 128 .. 2048 at the longest
    stacks that fit (N = 16384 up to 1024^2; 2048^2 at N = 4096: its spectrum at N = 16384
    would be 275 GB).  Step one and step two on device-drawn counts (timing only)."""
    out = []
    for side, N in ((128, 16384), (256, 16384), (512, 16384), (1024, 16384), (2048, 4096)):
        r = time_long_stack(ddm, dev, stream, seed, H=side, W=side, N=N, steps=2)
        out.append({"side": side, "N": N, "spatial_ms": r["stages_ms"]["spatial_fft"],
                    "temporal_ms": r["stages_ms"]["temporal_sf"], "frames_per_s": r["frames_per_s"],
                    "device_status": r["device_status"]})
    return out


def precision_sweep(ddm, dev, stream, seed, with_oracle, H=1024, W=1024, N=4096):
    """The precision-sweep workload (1024x1024 float32, N = 4096, OU Fourier modes,
    S(q) = 1 / max(q, 0.02)^2, D0 log-uniform in [0.01, 1]) through every precision tier of
    ddm_structure_function: device time per stack and, with the oracle leg on, each tier's
    max scaled error against the FP64 oracle on a bounded sample (kx = 1 and W/2, every
    fourth ky, every lag)."""
    import torch
    import synth
    frames = synth.ou_precision_sweep_1024x1024x4096(seed=seed, N=N, H=H, W=W, device=dev)
    cols, ky_step = [1, W // 2], 4
    D_or = s_q = None
    if with_oracle:
        import oracle
        parts = [oracle.dft2(frames[t0:t0 + 128].cpu().numpy(), cols) for t0 in range(0, N, 128)]
        F = np.concatenate(parts, axis=0)[:, ::ky_step, :]
        D_or = oracle.sf_direct(F)
        s_q = oracle.plateau_scale(F)
    tiers = {}
    for name, prec, reps in (("fp32", ddm.DDM_PREC_FP32, 3), ("fp32_fp64fix", ddm.DDM_PREC_FP32_FP64FIX, 3),
                             ("fp64", ddm.DDM_PREC_FP64, 1)):
        plan = ddm.Plan(H, W, N, dtype="f32", precision=prec)
        D = torch.empty(plan.n_q * N, dtype=torch.float32, device=dev)
        plan.structure_function(frames, D, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.structure_function(frames, D, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        row = {"structure_function_ms": ms, "frames_per_s": N / (ms / 1e3),
               "device_status": plan.last_device_status()}
        if D_or is not None:
            got = D.view(H, W // 2 + 1, N)[::ky_step, cols, :].cpu().numpy()
            row["max_rel_err"] = oracle.scaled_error(got, D_or, s_q)
        tiers[name] = row
        plan.close()
        del D
        torch.cuda.empty_cache()
    del frames
    torch.cuda.empty_cache()
    return {"workload": f"ou_powerlaw_{H}x{W}x{N}_f32", "H": H, "W": W, "N": N,
            "frames": "OU Fourier modes, S = 1/max(q, 0.02)^2, D0 log-uniform [0.01, 1], rendered on the device",
            "error_sample": (f"kx in {cols}, every {ky_step}th ky, all lags; max |D - D_oracle| / s_q"
                             if with_oracle else None),
            "tiers": tiers}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import synth
    oracle.build()
    frames = synth.blobs_512x512x1024(seed=args.seed, N=N_FRAMES, H=H, W=W)
    cores = os.cpu_count() or 1
    cols = [1]
    times = []
    for k in range(args.warmup + args.steps):
        t, _, _ = oracle_sample(frames, cols, cores)
        if k >= args.warmup:
            times.append(t)
    t_step = sum(times) / len(times)
    q_sample = H * len(cols)
    t_full = t_step * N_Q / q_sample
    value = N_FRAMES / t_full
    sample = (f"{len(cols)} kx column x {H} ky x {N_FRAMES} frames x all lags per step "
              f"({q_sample} of {N_Q} wave vectors); frames/s extrapolated linearly in the q count")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "N": N_FRAMES, "n_bins": N_BINS},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


def run_split(args):
    """One 512x512x1024 stack per step, split across the ranks by kx columns
    (partition.kx_ranges): every rank reads the whole stack and transforms every row, then
    only its own columns (step one) and their time sequences (step two); its radial sums
    are all-reduced (the one collective) and rank 0 fits the merged radial curves.  The
    whole job processes one stack per step, so "value" is strong scaling."""
    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2012_05695_b300 as ddm
    import synth
    from paper_2012_05695_b300 import partition
    dev = torch.device("cuda", local)
    frames_np = synth.blobs_512x512x1024(seed=args.seed, N=N_FRAMES, H=H, W=W)   # one stack
    kx0, kx1 = partition.kx_ranges(W, ws)[rank]
    plan = ddm.Plan(H, W, N_FRAMES, dtype="u16", n_bins=N_BINS, kx_begin=kx0, kx_end=kx1)
    frames = torch.from_numpy(frames_np).to(dev)
    D = torch.empty(plan.d_rows * N_FRAMES, dtype=torch.float32, device=dev)
    sums = torch.empty(N_BINS * N_FRAMES, dtype=torch.float32, device=dev)
    counts = torch.empty(N_BINS, dtype=torch.int32, device=dev)
    prm = torch.empty(N_BINS * 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        plan.structure_function(frames, D, stream)
        plan.azimuthal_sums(D, sums, counts, stream)
        if dist:
            Dr = partition.allreduce_radial(sums.view(N_BINS, N_FRAMES), counts)
        else:
            Dr = partition.merge_radial(sums.view(N_BINS, N_FRAMES), counts)
        if rank == 0:
            plan.fit(Dr.contiguous().view(-1), N_BINS, ddm._binding.DDM_FIT_LM, None, prm,
                     None, None, None, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = clk.mark()
        start.record(stream)
        for _ in range(args.steps):
            step()
        end.record(stream)
        torch.cuda.synchronize()
        t1 = clk.mark()
        if dist:
            dist.barrier()
    ms_total = max_over_ranks(start.elapsed_time(end), dist, dev)
    value = N_FRAMES * args.steps / (ms_total / 1e3)          # one stack per step, whole job
    status = plan.last_device_status()
    out = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "N": N_FRAMES, "n_bins": N_BINS,
                   "parallelism": f"kx-column split x{ws}", "rank0_kx_range": [kx0, kx1],
                   "l2": "inputs larger than L2: no flush"},
        "gpu_launches": 7 * args.steps, "clocks": clk.summary(t0, t1), "device_status": status,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2012_05695_b300 as ddm
    import synth

    frames_np = synth.blobs_512x512x1024(seed=args.seed + rank, N=N_FRAMES, H=H, W=W)
    plan = ddm.Plan(H, W, N_FRAMES, dtype="u16", n_bins=N_BINS)
    dev = torch.device("cuda", local)
    frames = torch.from_numpy(frames_np).to(dev)
    spec = torch.empty(2 * N_FRAMES * plan.n_q, dtype=torch.float32, device=dev)
    D = torch.empty(plan.n_q * N_FRAMES, dtype=torch.float32, device=dev)
    Dr = torch.empty(N_BINS * N_FRAMES, dtype=torch.float32, device=dev)
    counts = torch.empty(N_BINS, dtype=torch.int32, device=dev)
    fit_params = torch.empty(N_BINS * 4, dtype=torch.float32, device=dev)
    fit_cost = torch.empty(N_BINS, dtype=torch.float32, device=dev)
    fit_iters = torch.empty(N_BINS, dtype=torch.int32, device=dev)
    fit_flags = torch.empty(N_BINS, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        plan.spatial_fft(frames, spec, stream)
        if ev:
            ev[1].record(stream)
        plan.temporal_sf(spec, D, stream)
        if ev:
            ev[2].record(stream)
        plan.azimuthal_average(D, Dr, counts, stream)
        if ev:
            ev[3].record(stream)
        plan.fit(Dr, N_BINS, ddm._binding.DDM_FIT_LM, None, fit_params, fit_cost, fit_iters,
                 fit_flags, stream)
        if ev:
            ev[4].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = clk.mark()
        start.record(stream)
        for k in range(args.steps):
            step(evs[k])
        end.record(stream)
        torch.cuda.synchronize()
        t1 = clk.mark()
        if dist:
            dist.barrier()
    clocks = clk.summary(t0, t1)
    ms_total = max_over_ranks(start.elapsed_time(end), dist, dev)
    ms_step = ms_total / args.steps
    sp_ms = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    tm_ms = sum(e[1].elapsed_time(e[2]) for e in evs) / args.steps
    rd_ms = sum(e[2].elapsed_time(e[3]) for e in evs) / args.steps
    ft_ms = sum(e[3].elapsed_time(e[4]) for e in evs) / args.steps
    n_gpus = ws
    value = job_throughput(n_gpus, N_FRAMES, args.steps, ms_total)
    peak, peak_kind = measured_peaks()

    # ---- end to end through the public API: pinned host frames in, radial average and fit
    # out.  Stacks are pipelined the way a user streaming stacks would: two device frame
    # buffers, the next stack's upload on a copy stream under the current stack's compute;
    # every step still uploads its own frames and reads back its own results.
    e2e = None
    e2e_radial = None
    if not args.no_e2e:
        host = torch.from_numpy(frames_np).pin_memory()
        D_host = torch.empty(plan.d_rows * N_FRAMES, dtype=torch.float32).pin_memory()
        Dr_host = torch.empty(N_BINS * N_FRAMES, dtype=torch.float32).pin_memory()
        params_host = torch.empty(N_BINS * 4, dtype=torch.float32).pin_memory()
        bufs = [torch.empty_like(frames), torch.empty_like(frames)]
        Dbufs = [D, torch.empty_like(D)]
        up_stream = torch.cuda.Stream(device=dev)
        down_stream = torch.cuda.Stream(device=dev)
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        free = [torch.cuda.Event(), torch.cuda.Event()]
        computed = [torch.cuda.Event(), torch.cuda.Event()]
        read = [torch.cuda.Event(), torch.cuda.Event()]

        def e2e_run(k_steps, full_D, start_ev=None):
            """Per step: upload the stack from pinned host memory, the structure function,
            then either D itself back to pinned host memory (full_D) or the radial average
            and the fit of its curves, whose Dr and parameters come back.  Uploads run on
            their own stream under the previous stack's compute, D read-backs on another."""
            if start_ev is not None:
                up_stream.wait_event(start_ev)
            for k in range(k_steps):
                b = k % 2
                with torch.cuda.stream(up_stream):
                    if k >= 2:
                        up_stream.wait_event(free[b])     # stack k-2 has left this buffer
                    bufs[b].copy_(host, non_blocking=True)
                    ready[b].record(up_stream)
                stream.wait_event(ready[b])
                if full_D and k >= 2:
                    stream.wait_event(read[b])            # D of stack k-2 has been read back
                plan.structure_function(bufs[b], Dbufs[b], stream)
                free[b].record(stream)
                if full_D:
                    computed[b].record(stream)
                    with torch.cuda.stream(down_stream):
                        down_stream.wait_event(computed[b])
                        D_host.copy_(Dbufs[b], non_blocking=True)
                        read[b].record(down_stream)
                else:
                    plan.azimuthal_average(Dbufs[b], Dr, counts, stream)
                    plan.fit(Dr, N_BINS, ddm._binding.DDM_FIT_LM, None, fit_params, None, None, None, stream)
                    Dr_host.copy_(Dr, non_blocking=True)
                    params_host.copy_(fit_params, non_blocking=True)
            if full_D:
                stream.wait_stream(down_stream)

        def e2e_time(full_D):
            e2e_run(max(2, args.warmup), full_D)
            torch.cuda.synchronize()
            k_e2e = max(3, min(args.steps, 20))
            if dist:
                dist.barrier()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            e2e_run(k_e2e, full_D, s0)
            s1.record(stream)
            torch.cuda.synchronize()
            return max_over_ranks(s0.elapsed_time(s1), dist, dev), k_e2e

        h2d = int(host.numel() * host.element_size())
        e_ms, k_e2e = e2e_time(True)
        e2e = {"value": job_throughput(n_gpus, N_FRAMES, k_e2e, e_ms), "unit": "frames/s",
               "returns": "the full D(q, lag) of every stack, to pinned host memory",
               "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(D_host.numel() * D_host.element_size()),
               "h2d_effective_gbs": round(h2d * k_e2e / (e_ms / 1e3) / 1e9, 1),
               "pipelined": "next stack's upload and the previous stack's D read-back overlap this stack's compute",
               "steps": k_e2e}
        e_ms, k_e2e = e2e_time(False)
        e2e_radial = {"value": job_throughput(n_gpus, N_FRAMES, k_e2e, e_ms), "unit": "frames/s",
                      "returns": "the radial average Dr and the LM fit parameters of every stack",
                      "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": int(Dr_host.numel() * Dr_host.element_size()
                                                + params_host.numel() * params_host.element_size()),
                      "steps": k_e2e}
        del Dbufs, bufs

    # ---- precision tiers on the same stack: the FP32+FP64-fixup temporal stage
    tiers = {"fp32": {"temporal_ms": tm_ms}}
    D_fix = None
    fix_ok = 256 < N_FRAMES <= 8192                 # the tier is built for 257 <= N <= 8192
    if rank == 0 and not fix_ok:
        tiers["fp32_fp64fix"] = {"unsupported": f"N = {N_FRAMES}: the FP64-fixup tier needs 257 <= N <= 8192"}
    if rank == 0 and fix_ok:
        plan_fix = ddm.Plan(H, W, N_FRAMES, dtype="u16", precision=ddm.DDM_PREC_FP32_FP64FIX)
        D_fix = torch.empty_like(D)
        plan.spatial_fft(frames, spec, stream)
        for _ in range(3):
            plan_fix.temporal_sf(spec, D_fix, stream)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(10):
            plan_fix.temporal_sf(spec, D_fix, stream)
        f1.record(stream)
        torch.cuda.synchronize()
        tiers["fp32_fp64fix"] = {"temporal_ms": f0.elapsed_time(f1) / 10, "fix_lags": 8}

    # ---- the tensor-core DFT-as-GEMM column pass (DDM_PREC_TC_TF32X3) on the same stack:
    # step one's time beside the CUDA-core pass, and (with the oracle leg) its error
    D_tc = None
    if rank == 0 and H == 512:
        plan_tc = ddm.Plan(H, W, N_FRAMES, dtype="u16", precision=ddm.DDM_PREC_TC_TF32X3)
        for _ in range(3):
            plan_tc.spatial_fft(frames, spec, stream)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(10):
            plan_tc.spatial_fft(frames, spec, stream)
        f1.record(stream)
        torch.cuda.synchronize()
        D_tc = torch.empty_like(D)
        plan_tc.structure_function(frames, D_tc, stream)
        torch.cuda.synchronize()
        tiers["tc_tf32x3"] = {"spatial_ms": f0.elapsed_time(f1) / 10, "spatial_ms_fp32": sp_ms,
                              "column_pass": "tcgen05.mma kind::tf32, 512 = 16 x 32, two-term operand splits",
                              "device_status": plan_tc.last_device_status()}
        plan_tc.close()

    # ---- the FP64 tier on the same stack (the precision sweep's reference): both steps
    D64 = None
    if rank == 0 and N_FRAMES <= 4096 and not args.no_fp64:
        plan64 = ddm.Plan(H, W, N_FRAMES, dtype="u16", precision=ddm.DDM_PREC_FP64)
        D64 = torch.empty_like(D)
        plan64.structure_function(frames, D64, stream)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(3):
            plan64.structure_function(frames, D64, stream)
        f1.record(stream)
        torch.cuda.synchronize()
        tiers["fp64"] = {"structure_function_ms": f0.elapsed_time(f1) / 3,
                         "device_status": plan64.last_device_status()}
        plan64.close()

    # ---- the low-frequency restriction (Sec. 3) on the same stack: cropped spectrum store
    low_q = None
    if rank == 0 and args.kmax > 0 and args.kmax < min(H, W) // 2:
        lp = ddm.Plan(H, W, N_FRAMES, dtype="u16", n_bins=N_BINS, kmax=args.kmax)
        spec_c = torch.empty(2 * N_FRAMES * lp.n_q, dtype=torch.float32, device=dev)
        D_c = torch.empty(lp.n_q * N_FRAMES, dtype=torch.float32, device=dev)
        Dr_c = torch.empty(N_BINS * N_FRAMES, dtype=torch.float32, device=dev)   # not the stack's Dr
        lev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(10)]
        for k in range(13):
            e = lev[k - 3] if k >= 3 else None
            if e:
                e[0].record(stream)
            lp.spatial_fft(frames, spec_c, stream)
            if e:
                e[1].record(stream)
            lp.temporal_sf(spec_c, D_c, stream)
            if e:
                e[2].record(stream)
            lp.azimuthal_average(D_c, Dr_c, None, stream)
            if e:
                e[3].record(stream)
        torch.cuda.synchronize()
        ls = [sum(e[j].elapsed_time(e[j + 1]) for e in lev) / 10 for j in range(3)]
        low_q = {"kmax": args.kmax, "n_q": lp.n_q, "kept_fraction": lp.n_q / N_Q,
                 "stages_ms": {"spatial_fft": ls[0], "temporal_sf": ls[1], "azimuthal_average": ls[2]},
                 "frames_per_s": N_FRAMES / (sum(ls) / 1e3)}
        del spec_c, D_c, Dr_c, lp

    # ---- a camera whose sides are not powers of two (Bluestein spatial transforms) and a
    # long stack: 600 x 800 x 3000 uint16.  Timing only (kernel times do not depend on the
    # pixel values), so the counts are drawn on the device; the tests check this shape
    # against the oracle on the two-species blob stack.
    camera = None
    if rank == 0 and not args.no_camera:
        camera = time_camera(ddm, dev, stream, args.seed)
    long_stack = None
    if rank == 0 and not args.no_long:
        long_stack = time_long_stack(ddm, dev, stream, args.seed)
    sweep = image_size_sweep(ddm, dev, stream, args.seed) if (rank == 0 and args.sweep) else None
    crossover = None
    if rank == 0 and args.crossover:
        crossover = crossover_sweep(ddm, dev, stream, args.seed, side=H,
                                    Ns=tuple(int(x) for x in args.crossover_ns.split(",")))
    psweep = None
    if rank == 0 and not args.no_precision_sweep:
        psweep = precision_sweep(ddm, dev, stream, args.seed,
                                 with_oracle=(ws == 1 and not args.no_cpu_baseline))

    # ---- fit of the 362 radial curves: plain LM vs LM seeded by the trained MLP
    fit_cmp = None
    if rank == 0 and not args.no_fit_compare:
        fit_cmp = compare_fits(ddm, plan, Dr, stream)

    # ---- FP64 oracle on a bounded sample: CPU baseline and max scaled error of this run
    cpu = None
    max_err = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        cols = [1, 200]
        t_s, D_or, s_q = oracle_sample(frames_np, cols, cores)
        q_sample = H * len(cols)
        cpu_value = N_FRAMES / (t_s * N_Q / q_sample)
        t_1, _, _ = oracle_sample(frames_np, cols[:1], 1)          # the same oracle on one core
        cpu = {"value": cpu_value, "unit": "frames/s", "cores": cores, "kind": "oracle",
               "cpu_model": cpu_model(),
               "sample": f"{len(cols)} kx columns x {H} ky x {N_FRAMES} frames x all lags "
                         f"({q_sample} of {N_Q} wave vectors), {t_s:.1f} s; frames/s extrapolated "
                         f"linearly in the q count",
               "one_core": {"value": N_FRAMES / (t_1 * N_Q / H), "unit": "frames/s", "cores": 1,
                            "sample": f"1 kx column x {H} ky x {N_FRAMES} frames x all lags, {t_1:.1f} s; "
                                      f"extrapolated linearly in the q count"}}
        plan.structure_function(frames, D, stream)
        torch.cuda.synchronize()
        Dg = D.view(H, W // 2 + 1, N_FRAMES)[:, cols, :].cpu().numpy()
        max_err = oracle.scaled_error(Dg, D_or, s_q)
        ref = D_or[..., 1:9]
        tiers["fp32"]["max_rel_err"] = max_err
        tiers["fp32"]["small_lag_err_rel_D"] = float(np.max(np.abs(Dg[..., 1:9] - ref) / ref))
        if D64 is not None:
            D6 = D64.view(H, W // 2 + 1, N_FRAMES)[:, cols, :].cpu().numpy()
            tiers["fp64"]["max_rel_err"] = oracle.scaled_error(D6, D_or, s_q)
            tiers["fp64"]["small_lag_err_rel_D"] = float(np.max(np.abs(D6[..., 1:9] - ref) / ref))
        if D_tc is not None:
            Dt = D_tc.view(H, W // 2 + 1, N_FRAMES)[:, cols, :].cpu().numpy()
            tiers["tc_tf32x3"]["max_rel_err"] = oracle.scaled_error(Dt, D_or, s_q)
        if D_fix is not None:
            Df = D_fix.view(H, W // 2 + 1, N_FRAMES)[:, cols, :].cpu().numpy()
            tiers["fp32_fp64fix"]["max_rel_err"] = oracle.scaled_error(Df, D_or, s_q)
            tiers["fp32_fp64fix"]["small_lag_err_rel_D"] = float(np.max(np.abs(Df[..., 1:9] - ref) / ref))

    # the committed ncu summary is for the 512x512x1024 workload only
    traffic = profiled_traffic() if (H, W, N_FRAMES) == (512, 512, 1024) else None
    tm_achieved = TEMPORAL_BYTES / (tm_ms / 1e3) / 1e9
    # the temporal kernel is bound by FP32 issue, not by DRAM: its arithmetic roofline too.
    # Nominal flops: three complex L-point transforms per wave vector at 5 L log2 L each;
    # FP32 peak: 148 SMs x 128 lanes x 2 flops per FMA x the maximum SM clock.
    L_t = 1 << (N_FRAMES - 1).bit_length()
    tm_flops = N_Q * 3 * 5 * L_t * max(1, L_t.bit_length() - 1)
    fp32_peak = 148 * 128 * 2 * (clocks.get("sm_max_mhz") or 2032.0) * 1e6 / 1e12
    sp_achieved = SPATIAL_BYTES / (sp_ms / 1e3) / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": n_gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "N": N_FRAMES, "n_bins": N_BINS,
                   "frames": "uint16 Brownian Gaussian blobs (3000, sigma 2 px, D0 0.2), mean 2000, Poisson",
                   "l2": (f"inputs larger than L2 (frames {N_FRAMES * H * W * 2 / 1e6:.0f} MB, spectrum "
                          f"{N_FRAMES * N_Q * 8 / 1e9:.2f} GB): no flush"),
                   "parallelism": f"replicas x{n_gpus}"},
        "roofline": {"kernel": "temporal_sf_kernel", "bound": "hbm",
                     "achieved": tm_achieved, "peak": peak, "unit": "GB/s",
                     "frac": tm_achieved / peak, "peak_kind": peak_kind,
                     "traffic": traffic, "algorithmic_bytes": TEMPORAL_BYTES},
        "roofline_alu": {"kernel": "temporal_sf_kernel", "bound": "alu",
                         "achieved": tm_flops / (tm_ms / 1e3) / 1e12, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": tm_flops / (tm_ms / 1e3) / 1e12 / fp32_peak,
                         "flops": tm_flops, "flop_model": "3 complex L-point FFTs per q, 5 L log2 L each",
                         "peak_kind": "FP32 FMA lanes x max SM clock"},
        "stages_ms": {"spatial_fft": sp_ms, "temporal_sf": tm_ms, "azimuthal_average": rd_ms,
                      "fit_lm": ft_ms},
        "step_roofline": {"algorithmic_bytes": STEP_BYTES,
                          "achieved_gbs": STEP_BYTES / ((sp_ms + tm_ms) / 1e3) / 1e9,
                          "frac": STEP_BYTES / ((sp_ms + tm_ms) / 1e3) / 1e9 / peak,
                          "spatial_gbs": sp_achieved, "spatial_frac": sp_achieved / peak},
        "max_rel_err": max_err,
        "gpu_launches": 7 * args.steps,
        "clocks": clocks,
    }
    out["precision_tiers"] = tiers
    if low_q:
        out["low_q"] = low_q
    if camera:
        out["camera"] = camera
    if long_stack:
        out["long_stack"] = long_stack
    if sweep:
        out["image_size_sweep"] = sweep
    if crossover:
        out["crossover"] = crossover
    if psweep:
        out["precision_sweep"] = psweep
    if fit_cmp:
        out["fit"] = fit_cmp
    if e2e:
        out["e2e"] = e2e
    if e2e_radial:
        out["e2e_radial_fit"] = e2e_radial
    if cpu:
        out["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.split == "kx":
        return run_split(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
