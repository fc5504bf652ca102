#!/usr/bin/env python
"""Benchmark of the Pointing SelfCal hot path on GB300 (one JSON line).

Headline workload (default): "drift197_l128ch", the full-scale case -- 197
antennas (19,306 baselines) of 15 m uniform-disk apertures in a centrally
concentrated disk of 8 km radius, 128 channels over 0.95-1.76 GHz, 1800 x 1 s
in 30 solution intervals of 60 s, a 4096^2 model image (1") with 10^4
power-law sources padded to an 8192^2 grid; 4,448,102,400 visibilities
(35.6 GB of complex64, resident in HBM), weights one scalar 1/sigma^2 per
interval.  Observed data are simulated by the GPU predictor at the seeded
drifting true offsets plus 1 mJy noise from a seeded device generator.

One step = one Levenberg-Marquardt iteration over all 30 intervals as one
batch: a solver restart to the zero start (one small kernel), one persistent
fused launch over all intervals (degrid with the pointing-modified kernel,
the four pointing derivatives, residuals, per-baseline chi^2 / gradient /
normal sums), the deterministic per-antenna reductions and the LM updates
(damped full solve), replayed from a CUDA graph.  value = visibilities
evaluated with derivatives per second (Gvis/s).  Every step is the first
iteration of a solve from zero offsets, so no step can be skipped by a
stopped solver.  The model-grid DFT and the aperture tables are pre-computes
outside the iteration loop (Algorithm 1); their time is "precompute_ms".

Secondary keys: the precision-study workload "vla27_l64ch" measured the same
way; solves/s of the small plain-method workload "vla27_l1ch"; the learned
initial estimate against plain LM ("learned_init"); and the further sections
(mixed batch, two polarisations, exact kernel, W-snapshots, residual-w stack).

``--impl reference`` times the FP64 CPU oracle on the host cores instead
(rank 0 only), on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gvis/s predict+∂/∂pointing; solves/s to 1″ RMS offset, learned vs plain LM"
# workloads whose weights are one scalar per interval (w = NULL): the 35.6 GB
# of visibilities stay the only per-visibility input
SCALAR_WEIGHTS = ("drift197_l128ch",)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="drift197_l128ch")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    p.add_argument("--no-secondary", action="store_true", help="skip every section after the headline")
    p.add_argument("--no-learned", action="store_true", help="skip the learned-initialiser comparison")
    p.add_argument("--no-exact", action="store_true", help="skip the exact-disk-kernel section")
    p.add_argument("--no-wsnap", action="store_true", help="skip the W-snapshot section")
    p.add_argument("--no-wstack", action="store_true", help="skip the residual-w stack section")
    p.add_argument("--no-squint", action="store_true", help="skip the two-polarisation section")
    p.add_argument("--mixed-intervals", type=int, default=256,
                   help="intervals of the mixed-array batched-solve section (0 skips it)")
    p.add_argument("--learned-train", type=int, default=100_000, help="training intervals of the learned initialiser")
    p.add_argument("--learned-eval", type=int, default=10_000, help="held-out intervals of the comparison")
    p.add_argument("--learned-steps", type=int, default=20_000, help="AdamW steps of the network's training")
    return p.parse_args()


def dist_env():
    from paper_1709_08681_gb300 import dist as D
    return D.rank_info()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                self.samples.append((time.time(), float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                pass

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        win = [s for s in self.samples if t0 <= s[0] <= t1]
        if not win:
            mid = 0.5 * (t0 + t1)
            win = sorted(self.samples, key=lambda s: abs(s[0] - mid))[:3]
        reasons = set()
        for s in win:
            for name, v in zip(self.NAMES, s[3]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median([s[1] for s in win])), "sm_max_mhz": float(win[0][2]),
                "reasons": sorted(reasons), "samples": len(win)}


# ---------------------------------------------------------------- shared helpers

def config_for(wl) -> dict:
    """The workload description both arms print (identical dictionaries)."""
    scalar_w = wl.name in SCALAR_WEIGHTS
    vis_gb = wl.n_vis * 8 / 1e9
    w_gb = 0.0 if scalar_w else wl.n_vis * 4 / 1e9
    return {"workload": wl.name, "n_ant": wl.n_ant, "n_bl": wl.n_bl, "n_time": wl.n_time, "n_chan": wl.n_chan,
            "n_interval": len(wl.intervals), "n_vis": int(wl.n_vis), "image": int(wl.image.shape[0]),
            "grid": int(wl.n_grid), "support": wl.support, "oversample": wl.oversample, "aperture": wl.ap_kind,
            "weights": "scalar 1/sigma^2 per interval" if scalar_w else "per visibility",
            "l2": "inputs larger than L2 (vis %.1f GB + weights %.1f GB + grid %.2f GB per step)"
                  % (vis_gb, w_gb, wl.n_grid ** 2 * 8 / 1e9),
            "step": "one LM iteration of all intervals (one persistent fused launch, graph replay)"}


def oracle_model(wl, grid, t0, n_t, chans):
    from oracle import psc
    return psc.Model(uvw_m=wl.uvw_m[t0:t0 + n_t], freq_hz=wl.freq_hz[chans], n_ant=wl.n_ant, grid=grid,
                     cell_rad=wl.cell_rad, support=wl.support, oversample=wl.oversample, ap_kind=wl.ap_kind,
                     diam_m=wl.diam_m, alpha_per_dlambda=wl.alpha_per_dlambda, decorrelation=wl.decorrelation)


def sample_channels(wl, n=8):
    """n channels spread over the band (all of them when there are fewer)."""
    if wl.n_chan <= n:
        return np.arange(wl.n_chan)
    return np.unique(np.round(np.linspace(0, wl.n_chan - 1, n)).astype(int))


def oracle_sample(wl, target_s, seed=0):
    """Times the FP64 oracle (predict + derivatives + chi^2/gradient/normal
    sums, at zero offsets) on the first time steps of interval 0 over a few
    channels spread across the band, enough for about ``target_s`` seconds.
    The oracle's cost per visibility does not depend on the values, so the
    observed data are seeded noise of the sample's shape."""
    from oracle import model_grid, psc
    from paper_1709_08681_gb300 import inputs as I
    grid = model_grid.grid_from_image(wl.image, wl.n_grid)
    chans = sample_channels(wl)
    t_max = wl.intervals[0][1]

    def run(n_t):
        m = oracle_model(wl, grid, 0, n_t, chans)
        vis = I.complex_noise((n_t, wl.n_bl, len(chans)), 1.0, seed, 77)
        w = np.full(vis.shape, 1.0 / wl.sigma_noise ** 2)
        t = time.perf_counter()
        psc.chi2_grad_normal(m, np.zeros((wl.n_ant, 2)), vis, w)
        return time.perf_counter() - t

    dt1 = run(1)
    n_t = int(max(1, min(t_max, round(target_s / max(dt1, 1e-3)))))
    dt = run(n_t) if n_t != 1 else dt1
    n_vis = n_t * wl.n_bl * len(chans)
    return n_vis, dt, n_t, len(chans)


def profiled_traffic(wl_name):
    """DRAM bytes per fused launch of ``wl_name`` from its committed ncu
    summary (profiles/*.md naming the workload), or None when the kernel
    source changed since the counters were taken (sha256 prefix)."""
    pdir = os.path.join(ROOT, "profiles")
    try:
        names = sorted(os.listdir(pdir))
    except OSError:
        return None
    for fn in names:
        if not fn.endswith(".md"):
            continue
        text = open(os.path.join(pdir, fn)).read()
        m = re.search(r"headline traffic for: (\S+)", text)
        if not m or m.group(1) != wl_name:
            continue
        try:
            src, want = re.search(r"source sha256 prefix: (\S+) ([0-9a-f]+)", text).groups()
            have = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()[:len(want)]
            if have != want:
                return None
            return float(re.search(r"traffic per launch \(read \+ write, full workload\) \| ([0-9.e+]+) B", text)
                         .group(1))
        except (OSError, AttributeError, ValueError):
            return None
    return None


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this machine type (GB/s), else the
    profiling fallback of 6800 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


def host_mem_available():
    """Bytes of host memory available (Linux /proc/meminfo), or 0."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except (OSError, ValueError, IndexError):
        pass
    return 0


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1709_08681_gb300 import inputs as I
    from oracle import model_grid, psc
    wl = I.make_workload(args.workload, seed=args.seed)
    grid = model_grid.grid_from_image(wl.image, wl.n_grid)
    chans = sample_channels(wl)
    m = oracle_model(wl, grid, 0, 1, chans)
    # the oracle's own observed data for the sample: its prediction at the true offsets plus noise
    V, _ = psc.predict(m, wl.lm_true[0], False)
    vis = V + I.complex_noise(V.shape, wl.sigma_noise, wl.seed, 5)
    w = np.full(vis.shape, 1.0 / wl.sigma_noise ** 2)
    lm = np.zeros((wl.n_ant, 2))
    for _ in range(args.warmup):
        psc.chi2_grad_normal(m, lm, vis, w)
    t = time.perf_counter()
    for _ in range(args.steps):
        psc.chi2_grad_normal(m, lm, vis, w)
    dt = time.perf_counter() - t
    n_vis = vis.size
    value = n_vis * args.steps / dt / 1e9
    sample = ("interval 0, time step 0 x %d baselines x %d channels spread over the band (%d visibilities) per "
              "step; FP64 predict + derivatives + chi^2/gradient/normal sums" % (wl.n_bl, len(chans), n_vis))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gvis/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_for(wl),
        "cpu_baseline": {"value": value, "unit": "Gvis/s", "cores": omp_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Gvis/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm

def gpu_index_of(local):
    vis_dev = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis_dev:
        try:
            return int(vis_dev.split(",")[local])
        except (ValueError, IndexError):
            return local
    return local


def measure_iteration(wl, sess, vis, w, stream, steps, warmup, ws=1, sample_clocks=None):
    """Times `steps` batched LM iterations (restart + one iteration, graph
    replay) over all intervals, then the fused launch alone with CUDA events.
    Returns a dict with value, ms, roofline and the batch (kept open)."""
    import torch
    from paper_1709_08681_gb300 import _abi, dist as D, roofline as RL
    n_ctx = len(sess.ctxs)
    lm0 = np.zeros((wl.n_ant, 2))
    w_scale = [1.0 if w is not None else 1.0 / wl.sigma_noise ** 2] * n_ctx
    vk = [sess.vis_slice(vis, k) for k in range(n_ctx)]
    wk = [sess.vis_slice(w, k) for k in range(n_ctx)] if w is not None else None
    batch = _abi.Batch(sess.ctxs, vk, wk, w_scale=w_scale, stream=stream)
    tiles = batch.psc_batch_autotune()
    batch.psc_batch_begin([lm0] * n_ctx, _abi.psc_solve_opts_default())

    def step():
        batch.psc_batch_restart()
        batch.psc_batch_iterate(1)

    for _ in range(max(3, warmup)):
        step()
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = sample_clocks() if sample_clocks else None
    if sampler:
        time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    if ws > 1:
        torch.distributed.barrier()
    ms = D.max_over_ranks(e0.elapsed_time(e1), device="cuda")
    # the fused kernel's own launch time: the same steps again, launched
    # directly with CUDA events around each persistent fused launch
    batch.psc_batch_profile(True)
    for _ in range(max(3, min(steps, 20))):
        step()
    batch.psc_batch_profile(False)
    kern_ms, kern_n = batch.psc_batch_profile_read()
    clocks = None
    if sampler:
        time.sleep(0.2)
        sampler.stop()
        clocks = sampler.summary(t_wall0, t_wall1)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peak = RL.fp32_peak_tflops(props.multi_processor_count)
    flops = RL.flops_per_eval(wl, wl.intervals, wl.n_bl)
    flops_impl = RL.flops_per_eval(wl, wl.intervals, wl.n_bl, RL.FLOPS_PER_TAP_IMPL)
    avg = kern_ms / max(kern_n, 1)
    achieved = flops / (avg * 1e-3) / 1e12
    kern = batch.psc_batch_kernel()
    return {
        "value": ws * wl.n_vis * steps / (ms * 1e-3) / 1e9, "ms_per_step": ms / steps, "tiling": tiles,
        "clocks": clocks, "batch": batch, "vk": vk, "wk": wk, "w_scale": w_scale,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": profiled_traffic(wl.name),
                     "kernel": kern + ", persistent over all intervals (fused degrid + derivatives + residual + sums)",
                     "avg_launch_ms": avg, "flops_per_launch": flops, "flops_per_tap": RL.FLOPS_PER_TAP,
                     "frac_at_implemented_flops": flops_impl / (avg * 1e-3) / 1e12 / peak,
                     "implemented_flops_per_tap": RL.FLOPS_PER_TAP_IMPL,
                     "peak_basis": "%d SMs x 128 FP32 lanes x 2 x 2070 MHz" % props.multi_processor_count},
    }


def measure_e2e(wl, sess, vis, w, w_scale, stream, k_steps):
    """The same step through the public batch API with its inputs copied from
    pinned host memory every step and the offsets plus chi^2 read back (a
    synchronising call).  The copy precedes the iteration on the same stream:
    on this machine a host-to-device copy makes little progress while the
    fused kernel streams the grid and the visibilities through L2 (it runs at
    the full rate only beside compute-only work), so overlapping the next
    step's copy with this step's evaluation only lengthens the step."""
    import torch
    from paper_1709_08681_gb300 import _abi, dist as D
    n_ctx = len(sess.ctxs)
    lm0 = np.zeros((wl.n_ant, 2))
    vis_h = torch.empty(vis.shape, dtype=vis.dtype, pin_memory=True)
    vis_h.copy_(vis)
    w_h = None
    if w is not None:
        w_h = torch.empty(w.shape, dtype=w.dtype, pin_memory=True)
        w_h.copy_(w)
    batch = _abi.Batch(sess.ctxs, [sess.vis_slice(vis, k) for k in range(n_ctx)],
                       [sess.vis_slice(w, k) for k in range(n_ctx)] if w is not None else None,
                       w_scale=w_scale, stream=stream)
    batch.psc_batch_begin([lm0] * n_ctx, _abi.psc_solve_opts_default())
    batch.psc_batch_restart()                                  # untimed: graph capture
    batch.psc_batch_iterate(1)
    batch.psc_batch_end()
    d2h = 0
    # events on the stream split each step into its copy and its iteration
    # (recording them adds no synchronisation)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(k_steps)]
    torch.cuda.synchronize()
    t = time.perf_counter()
    for k in range(k_steps):
        ev[k][0].record(stream)
        with torch.cuda.stream(stream):
            vis.copy_(vis_h, non_blocking=True)
            if w_h is not None:
                w.copy_(w_h, non_blocking=True)
        ev[k][1].record(stream)
        batch.psc_batch_restart()
        batch.psc_batch_iterate(1)
        ev[k][2].record(stream)
        lm_out, reps = batch.psc_batch_end()                   # synchronises; offsets + chi^2 to the host
        d2h = sum(x.nbytes for x in lm_out) + 8 * 5 * len(reps)
    dt = D.max_over_ranks(time.perf_counter() - t, device="cuda")
    copy_ms = float(np.median([a.elapsed_time(b) for a, b, _ in ev]))
    iter_ms = float(np.median([b.elapsed_time(c) for _, b, c in ev]))
    batch.close()
    h2d = vis.numel() * 8 + (w.numel() * 4 if w is not None else 0)
    return {"value": wl.n_vis * k_steps / dt / 1e9, "unit": "Gvis/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": k_steps, "h2d_gb_per_s": h2d * k_steps / dt / 1e9,
            "copy_ms_per_step": copy_ms, "copy_gb_per_s": h2d / copy_ms / 1e6, "iterate_ms_per_step": iter_ms}


def setup_workload(wl, stream):
    import torch
    from paper_1709_08681_gb300.session import Session
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sess = Session(wl, stream=stream)
    e1.record(stream)
    stream.synchronize()
    precompute_ms = e0.elapsed_time(e1)
    vis = sess.simulate()
    w = None
    if wl.name not in SCALAR_WEIGHTS:
        w = torch.full(vis.shape, 1.0 / wl.sigma_noise ** 2, dtype=torch.float32, device=vis.device)
    stream.synchronize()
    return sess, vis, w, precompute_ms


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the CUDA library is the only implementation)")
    torch.cuda.set_device(local)
    from paper_1709_08681_gb300 import _abi, dist as D, inputs as I
    from paper_1709_08681_gb300 import roofline as RL

    # weak scaling: every rank solves its own copy of the workload (own seed)
    wl = I.make_workload(args.workload, seed=D.rank_seed(args.seed, rank))
    stream = torch.cuda.Stream()
    gpu_index = gpu_index_of(local)
    with torch.cuda.stream(stream):
        sess, vis, w, precompute_ms = setup_workload(wl, stream)
        head = measure_iteration(wl, sess, vis, w, stream, args.steps, args.warmup, ws,
                                 sample_clocks=lambda: ClockSampler(gpu_index))
        # full batched solves (plain LM from zero) of every interval
        solve = None
        if rank == 0:
            vk, wk = head["vk"], head["wk"]
            _abi.psc_solve_batch(sess.ctxs, vk, wk, w_scale=head["w_scale"])       # warm
            torch.cuda.synchronize()
            t = time.perf_counter()
            sols, reps = _abi.psc_solve_batch(sess.ctxs, vk, wk, w_scale=head["w_scale"])
            dt = time.perf_counter() - t
            errs = [np.sqrt(np.mean((sols[k] - wl.lm_true[k]) ** 2)) / I.ARCSEC for k in range(len(sess.ctxs))]
            solve = {"intervals_per_s": len(sess.ctxs) / dt, "solve_s": dt,
                     "mean_lm_iters": float(np.mean([r.n_iter for r in reps])),
                     "rms_err_arcsec_median": float(np.median(errs)), "init": "zero (plain LM)", "batched": True}
        head["batch"].close()
        e2e = None
        if not args.no_e2e:
            need = wl.n_vis * 8 * 1.3 + (wl.n_vis * 4 if w is not None else 0) + (16 << 30)
            if host_mem_available() >= need:
                e2e = measure_e2e(wl, sess, vis, w, head["w_scale"], stream, max(3, min(args.steps, 10)))
            else:
                e2e = {"value": None, "unit": "Gvis/s", "skipped": "host memory below %.0f GB" % (need / 1e9)}
        if rank == 0 and ws == 1 and not args.no_cpu_baseline:
            n_s, dt, n_t, n_c = oracle_sample(wl, args.cpu_seconds, args.seed)
            rate = n_s / dt
            cpu = {"value": rate / 1e9, "unit": "Gvis/s", "cores": omp_threads(), "kind": "oracle",
                   "sample": "interval 0, first %d time steps x %d baselines x %d channels spread over the band "
                             "(%d visibilities, %.1f s): FP64 predict + derivatives + chi^2/gradient/normal sums "
                             "at zero offsets" % (n_t, wl.n_bl, n_c, n_s, dt),
                   "extrapolated": True,
                   "step_s_extrapolated": wl.n_vis / rate,
                   "extrapolation": "linear in visibilities (the oracle's cost per visibility is fixed: the full "
                                    "S x S window)"}
        else:
            cpu = None
        sess.close()
        del vis, w
        torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": head["value"], "unit": "Gvis/s", "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_for(wl),
        "roofline": head["roofline"],
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": head["clocks"],
        # restart, persistent fused launch, per-baseline reduce, per-antenna
        # assembly, LM update per step (the queue reset is a memset)
        "gpu_launches": 5 * args.steps,
        "tiling": [list(t) for t in head["tiling"][:1]],
        "precompute_ms": precompute_ms,
    }
    if line["cpu_baseline"] is None:
        del line["cpu_baseline"]
    if solve:
        line["solve"] = solve
    if rank == 0 and not args.no_secondary:
        secondary(args, line, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def secondary(args, line, local):
    import torch
    from paper_1709_08681_gb300 import inputs as I, roofline as RL
    stream = torch.cuda.Stream()
    props = torch.cuda.get_device_properties(local)
    peak = RL.fp32_peak_tflops(props.multi_processor_count)
    with torch.cuda.stream(stream):
        # the precision-study workload, measured the same way as the headline
        if args.workload != "vla27_l64ch":
            wl = I.make_workload("vla27_l64ch", seed=args.seed)
            sess, vis, w, pre = setup_workload(wl, stream)
            r = measure_iteration(wl, sess, vis, w, stream, 50, 5)
            r["batch"].close()
            line["vla27_l64ch"] = {"value": r["value"], "unit": "Gvis/s", "ms_per_step": r["ms_per_step"],
                                   "n_vis": int(wl.n_vis), "roofline": r["roofline"],
                                   "tiling": [list(t) for t in r["tiling"][:1]]}
            sess.close()
            del vis, w
        # solves/s of the small plain-method workload: 64 draws of offsets and
        # noise on its geometry and sky, batched and one at a time
        from paper_1709_08681_gb300 import solves as SV
        line["vla27_l1ch"] = SV.run("vla27_l1ch", n_draws=64, seed=args.seed, stream=stream)
    if not args.no_learned:
        # solves/s to 1 arcsec RMS, learned initial estimate vs plain LM, on the
        # 64-antenna 16-channel workload (network trained here on GPU-simulated
        # intervals with the library's kernels)
        from paper_1709_08681_gb300 import learned_init as LI
        rep = LI.run_at_scale(n_train=args.learned_train, n_eval=args.learned_eval, steps=args.learned_steps,
                              seed=args.seed)
        line["learned_init"] = {"workload": "disk64_l16ch", **rep}
    if args.mixed_intervals > 0:
        from paper_1709_08681_gb300 import mixed as MX
        mrep, _ = MX.run(n_intervals=args.mixed_intervals, seed=args.seed)
        mrep.pop("tiling", None)
        mrep["roofline"] = {"bound": "alu", "achieved": mrep["fused_tflops"], "peak": peak, "unit": "TFLOP/s",
                            "frac": mrep["fused_tflops"] / peak}
        line["mixed_batch"] = {"workload": "mixed_batch%d" % args.mixed_intervals, **mrep}
    if not args.no_squint:
        from paper_1709_08681_gb300 import squint as SQ
        srep, _, _ = SQ.run("vla27_l64ch", seed=args.seed)
        line["squint"] = {"workload": "vla27_l64ch, R and L", **srep}
    if not args.no_exact:
        from paper_1709_08681_gb300 import exact_kernel as EK
        line["exact_kernel"] = {"workload": "vla27_l64ch, offsets sigma 60\"", **EK.run("vla27_l64ch", seed=args.seed)}
    if not args.no_wsnap:
        from paper_1709_08681_gb300 import wsnap as WS
        line["wsnap"] = {"workload": "vla27_l64ch, W-snapshot grid per interval", **WS.run("vla27_l64ch", seed=args.seed)}
    if not args.no_wstack:
        from paper_1709_08681_gb300 import wstack as WK
        line["wstack"] = {"workload": "vla27_l64ch, 600 time steps as one interval", **WK.run("vla27_l64ch", seed=args.seed)}
    # drifting pointing: cold batched solves against warm-started solves in time order
    from paper_1709_08681_gb300 import drift as DR
    drep = DR.run(seed=args.seed)
    drep["roofline"] = {"bound": "alu", "achieved": drep["fused_tflops"], "peak": peak, "unit": "TFLOP/s",
                        "frac": drep["fused_tflops"] / peak}
    drep["warm_latency_ms_per_interval"] = 1e3 * drep["warm_sequential_s"] / drep["n_intervals"]
    line["drift_full"] = {"workload": "drift197_l128ch", **drep}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
