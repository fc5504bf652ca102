#!/usr/bin/env python
"""Benchmark of the Pointing SelfCal hot path on GB300 (one JSON line).

Workload: "vla27_l64ch" -- 27 antennas (351 baselines) in a Y layout with
1 km arms, 25 m uniform-disk apertures, 64 channels over 1-2 GHz, 600 x 2 s
split into 4 solution intervals, a 2048^2 model image (8") with 2000
power-law sources; 13,478,400 visibilities, observed data simulated by the
GPU predictor at seeded true offsets (sigma 20") plus 1 mJy noise.

One step = one Levenberg-Marquardt iteration over all four intervals as one
batch: a solver restart to the zero start (one small kernel), one persistent
fused launch over the bricks of all intervals (degrid with the
pointing-modified kernel, the four pointing derivatives, residuals,
per-baseline chi^2 / gradient / normal sums), the deterministic per-antenna
reductions and the LM updates (damped full solve), replayed from a CUDA graph.  value = visibilities evaluated with derivatives per second
(Gvis/s).  Every step is the first iteration of a solve from zero offsets,
so no step can be skipped by a stopped solver.  The model-grid DFT and the aperture tables are
pre-computes outside the iteration loop (Algorithm 1); their time is reported
under "precompute_ms".

``--impl reference`` times the FP64 CPU oracle on the host cores instead
(rank 0 only), on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gvis/s predict+∂/∂pointing; solves/s to 1″ RMS offset, learned vs plain LM"
SMS_GB300 = 152


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="vla27_l64ch")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    p.add_argument("--no-learned", action="store_true", help="skip the learned-initialiser comparison")
    p.add_argument("--no-drift", action="store_true", help="skip the full-scale drifting-pointing section")
    p.add_argument("--no-exact", action="store_true", help="skip the exact-disk-kernel section")
    p.add_argument("--no-wsnap", action="store_true", help="skip the W-snapshot section")
    p.add_argument("--no-wstack", action="store_true", help="skip the residual-w stack section")
    p.add_argument("--mixed-intervals", type=int, default=256,
                   help="intervals of the mixed-array batched-solve section (0 skips it)")
    p.add_argument("--learned-train", type=int, default=3000, help="training intervals of the learned initialiser")
    p.add_argument("--learned-eval", type=int, default=20, help="held-out intervals of the comparison")
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


# ---------------------------------------------------------------- workload helpers

def cpu_sample_oracle(wl, vis_host, w_host, target_s, interval=0, min_t=1):
    """Times the FP64 oracle (predict + derivatives + reductions) on the first
    timesteps of one interval, enough to take about ``target_s`` seconds."""
    from oracle import model_grid, psc
    grid = model_grid.grid_from_image(wl.image, wl.n_grid)
    t0, nt = 0, wl.n_time          # the sample may run over every interval's time steps

    def run(n_t):
        m = psc.Model(uvw_m=wl.uvw_m[t0:t0 + n_t], freq_hz=wl.freq_hz, n_ant=wl.n_ant, grid=grid,
                      cell_rad=wl.cell_rad, support=wl.support, oversample=wl.oversample, ap_kind=wl.ap_kind,
                      diam_m=wl.diam_m, alpha_per_dlambda=wl.alpha_per_dlambda, decorrelation=wl.decorrelation)
        lm = np.zeros((wl.n_ant, 2))
        t = time.perf_counter()
        psc.chi2_grad_normal(m, lm, vis_host[t0:t0 + n_t], w_host[t0:t0 + n_t])
        return time.perf_counter() - t

    dt1 = run(min_t)
    n_t = int(max(min_t, min(nt, round(min_t * target_s / max(dt1, 1e-3)))))
    dt = run(n_t) if n_t != min_t else dt1
    n_vis = n_t * wl.n_bl * wl.n_chan
    return n_vis, dt, n_t, grid


def profiled_traffic():
    """DRAM bytes per fused launch from the committed ncu summary, or None
    when eval.cu changed since the counters were taken (sha256 prefix)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "eval_kernel_vla27_l64ch.md")
    src = os.path.join(ROOT, "paper_1709_08681_gb300", "csrc", "eval.cu")
    try:
        text = open(path).read()
        want = re.search(r"eval.cu sha256 prefix: ([0-9a-f]+)", text).group(1)
        have = hashlib.sha256(open(src, "rb").read()).hexdigest()[:len(want)]
        if want != have:
            return None
        return float(re.search(r"traffic per launch \(read \+ write\) \| ([0-9.]+) MB", text).group(1)) * 1e6
    except (OSError, AttributeError, ValueError):
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


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1709_08681_gb300 import inputs as I
    from oracle import model_grid, psc
    wl = I.make_workload(args.workload, seed=args.seed)
    # observed data for the sample: the oracle's own prediction at the true offsets plus noise
    grid = model_grid.grid_from_image(wl.image, wl.n_grid)
    t0, nt = wl.intervals[0]
    n_t = 1
    m = psc.Model(uvw_m=wl.uvw_m[t0:t0 + n_t], freq_hz=wl.freq_hz, n_ant=wl.n_ant, grid=grid, cell_rad=wl.cell_rad,
                  support=wl.support, oversample=wl.oversample, ap_kind=wl.ap_kind, diam_m=wl.diam_m,
                  alpha_per_dlambda=wl.alpha_per_dlambda, decorrelation=wl.decorrelation)
    V, _ = psc.predict(m, wl.lm_true[0], False)
    vis = V + wl.noise()[t0:t0 + n_t]
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
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gvis/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": "interval 0, first timestep: %d visibilities per step" % n_vis},
        "cpu_baseline": {"value": value, "unit": "Gvis/s", "cores": omp_threads(), "kind": "oracle",
                         "sample": "interval 0, 1 timestep x 351 baselines x 64 channels per step"},
        "e2e": {"value": value, "unit": "Gvis/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the CUDA library is the only implementation)")
    torch.cuda.set_device(local)
    from paper_1709_08681_gb300 import _abi, inputs as I
    from paper_1709_08681_gb300 import roofline as RL
    from paper_1709_08681_gb300.session import Session

    # weak scaling: every rank solves its own batch of four intervals (own seed)
    from paper_1709_08681_gb300 import dist as D
    wl = I.make_workload(args.workload, seed=D.rank_seed(args.seed, rank))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sess = Session(wl, stream=stream)
        e1.record(stream)
        stream.synchronize()
        precompute_ms = e0.elapsed_time(e1)
        vis = sess.simulate()
        w = torch.full(vis.shape, 1.0 / wl.sigma_noise ** 2, dtype=torch.float32, device=vis.device)
        stream.synchronize()

        lm0 = np.zeros((wl.n_ant, 2))
        opts = _abi.psc_solve_opts_default()
        vk = [sess.vis_slice(vis, k) for k in range(len(sess.ctxs))]
        wk = [sess.vis_slice(w, k) for k in range(len(sess.ctxs))]
        # all intervals in one batch: one persistent fused launch per iteration
        batch = _abi.Batch(sess.ctxs, vk, wk, stream=stream)
        tiles = batch.psc_batch_autotune()
        batch.psc_batch_begin([lm0] * len(sess.ctxs), opts)

        def step():
            batch.psc_batch_restart()
            batch.psc_batch_iterate(1)

        for _ in range(max(3, args.warmup)):
            step()
        stream.synchronize()

        gpu_index = local
        vis_dev = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis_dev:
            try:
                gpu_index = int(vis_dev.split(",")[local])
            except ValueError:
                gpu_index = local
        sampler = ClockSampler(gpu_index)
        time.sleep(0.3)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t_wall0 = time.time()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        t_wall1 = time.time()
        if ws > 1:
            torch.distributed.barrier()
        ms = e0.elapsed_time(e1)
        # the fused kernel's own launch time: the same steps again, launched
        # directly with CUDA events around each persistent fused launch
        batch.psc_batch_profile(True)
        k_prof = max(3, min(args.steps, 50))
        for _ in range(k_prof):
            step()
        batch.psc_batch_profile(False)
        kern_ms, kern_n = batch.psc_batch_profile_read()
        time.sleep(0.2)
        sampler.stop()
        clocks = sampler.summary(t_wall0, t_wall1)
        ms = D.max_over_ranks(ms, device="cuda")

        n_vis = wl.n_vis
        value = ws * n_vis * args.steps / (ms * 1e-3) / 1e9
        # restart, persistent fused launch, per-baseline reduce, per-antenna
        # assembly, LM update (the queue reset is a memset, not a kernel)
        launches_per_step = 5

        # roofline of the fused kernel (FP32 ALU bound); one launch = all intervals
        taps = RL.taps_per_channel(wl)
        flops_per_launch = 0.0
        for (t0, nt) in wl.intervals:
            flops_per_launch += nt * wl.n_bl * float(np.sum(taps)) * RL.FLOPS_PER_TAP
        avg_launch_ms = kern_ms / max(kern_n, 1)
        achieved = flops_per_launch / (avg_launch_ms * 1e-3) / 1e12
        props = torch.cuda.get_device_properties(local)
        n_sm = props.multi_processor_count
        peak = RL.fp32_peak_tflops(n_sm)
        fma_measured = _abi.psc_fp32_fma_rate(stream)

        # materialised predict (V and the four derivative planes written to HBM):
        # HBM-bound, 40 bytes written per visibility
        vo = torch.empty((max(nt for _, nt in wl.intervals), wl.n_bl, wl.n_chan), dtype=torch.complex64,
                         device=vis.device)
        do = torch.empty((4,) + tuple(vo.shape), dtype=torch.complex64, device=vis.device)
        pm_ms = 0.0
        for k, ctx in enumerate(sess.ctxs):
            nt_k = wl.intervals[k][1]
            vv, dd = vo[:nt_k], do[:, :nt_k]
            lm_k = 0.5 * wl.lm_true[k]
            ctx.psc_predict(lm_k, vv, dd)                    # warm
            e0.record(stream)
            ctx.psc_predict(lm_k, vv, dd)
            e1.record(stream)
            torch.cuda.synchronize()
            pm_ms += e0.elapsed_time(e1)
        del vo, do
        hbm_peak = hbm_peak_gbs()
        pm_gbs = 40.0 * wl.n_vis / (pm_ms * 1e-3) / 1e9
        # same taps as the fused evaluation, so the FP32 ALU still binds; the
        # HBM share of its 40 written bytes per visibility is reported beside it
        pm_tflops = flops_per_launch / (pm_ms * 1e-3) / 1e12
        predict_mat = {"gvis_per_s": wl.n_vis / (pm_ms * 1e-3) / 1e9, "ms": pm_ms,
                       "roofline": {"bound": "alu", "achieved": pm_tflops, "peak": peak, "unit": "TFLOP/s",
                                    "frac": pm_tflops / peak},
                       "hbm": {"achieved_gbs": pm_gbs, "peak_gbs": hbm_peak, "frac": pm_gbs / hbm_peak,
                               "bytes_per_vis": 40, "peak_source": "measured copy bandwidth"}}

        # end to end: pinned host buffers; every step copies its inputs host->device
        # and reads its offsets and chi^2 back (a synchronising call).  The copies
        # run on a second stream into two alternating device buffers (one batch
        # per buffer over the same contexts), so that step k+1's copy overlaps
        # step k's evaluation; an event keeps a buffer from being overwritten
        # before the step that reads it has finished.
        vis_h = vis.cpu().pin_memory()
        w_h = w.cpu().pin_memory()
        n_ctx = len(sess.ctxs)
        bufs = [(torch.empty_like(vis), torch.empty_like(w)) for _ in range(2)]
        batches_e2e = [_abi.Batch(sess.ctxs, [sess.vis_slice(vd, k) for k in range(n_ctx)],
                                  [sess.vis_slice(wd, k) for k in range(n_ctx)], stream=stream) for vd, wd in bufs]
        for b_ in batches_e2e:
            b_.psc_batch_begin([lm0] * n_ctx, opts)
        copy_stream = torch.cuda.Stream(device=vis.device)
        ev_copied = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]

        def issue_copy(slot):
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(ev_done[slot])          # the step that last read this buffer is done
                bufs[slot][0].copy_(vis_h, non_blocking=True)
                bufs[slot][1].copy_(w_h, non_blocking=True)
                ev_copied[slot].record(copy_stream)

        for slot, b_ in enumerate(batches_e2e):                # untimed: graph capture of both batches
            bufs[slot][0].copy_(vis)
            bufs[slot][1].copy_(w)
            b_.psc_batch_restart()
            b_.psc_batch_iterate(1)
            b_.psc_batch_end()
        k_e2e = max(3, min(args.steps, 50))
        d2h = 0
        torch.cuda.synchronize()
        t = time.perf_counter()
        issue_copy(0)
        for step_i in range(k_e2e):
            slot = step_i % 2
            stream.wait_event(ev_copied[slot])
            batches_e2e[slot].psc_batch_restart()
            batches_e2e[slot].psc_batch_iterate(1)
            ev_done[slot].record(stream)
            if step_i + 1 < k_e2e:
                issue_copy(1 - slot)
            lm_out, reps = batches_e2e[slot].psc_batch_end()   # synchronises; offsets + chi^2 to the host
            d2h = sum(x.nbytes for x in lm_out) + 8 * 5 * len(reps)
        e2e_s = D.max_over_ranks(time.perf_counter() - t, device="cuda")
        e2e_value = ws * n_vis * k_e2e / e2e_s / 1e9
        h2d = vis.numel() * 8 + w.numel() * 4
        for b_ in batches_e2e:
            b_.close()
        del bufs

        # full solves (plain LM from zero) of the four intervals, batched
        solve = None
        if rank == 0:
            iters, errs = [], []
            n_rep = 3
            _abi.psc_solve_batch(sess.ctxs, vk, wk)              # warm
            torch.cuda.synchronize()
            t = time.perf_counter()
            for _ in range(n_rep):
                sols, reps = _abi.psc_solve_batch(sess.ctxs, vk, wk)
                for k in range(len(sess.ctxs)):
                    iters.append(reps[k].n_iter)
                    errs.append(np.sqrt(np.mean((sols[k] - wl.lm_true[k]) ** 2)) / I.ARCSEC)
            dt = time.perf_counter() - t
            solve = {"intervals_per_s": n_rep * len(sess.ctxs) / dt, "mean_lm_iters": float(np.mean(iters)),
                     "rms_err_arcsec": float(np.mean(errs)), "init": "zero (plain LM)", "batched": True}
        batch.close()

    line = {
        "metric": METRIC, "value": value, "unit": "Gvis/s", "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "n_ant": wl.n_ant, "n_bl": wl.n_bl, "n_time": wl.n_time,
                   "n_chan": wl.n_chan, "n_interval": len(wl.intervals), "n_vis": n_vis,
                   "image": wl.image.shape[0], "grid": wl.n_grid, "support": wl.support,
                   "oversample": wl.oversample, "aperture": wl.ap_kind,
                   "l2": "inputs larger than L2 (vis 108 MB + weights 54 MB + grid 32 MB per step)",
                   "step": "one LM iteration of all intervals (one persistent fused launch, graph replay)",
                   "tiling": [list(t) for t in tiles], "precompute_ms": precompute_ms},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": profiled_traffic() if args.workload == "vla27_l64ch" else None,
                     "kernel": "eval_kernel<false>, persistent over all intervals (fused degrid + derivatives + residual + sums)",
                     "avg_launch_ms": avg_launch_ms, "flops_per_launch": flops_per_launch,
                     "peak_basis": "%d SMs x 128 FP32 lanes x 2 x 2070 MHz" % n_sm,
                     "fp32_fma_measured_tflops": fma_measured, "frac_of_measured_fma": achieved / fma_measured},
        "predict_materialised": predict_mat,
        "e2e": {"value": e2e_value, "unit": "Gvis/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "clocks": clocks,
        "gpu_launches": launches_per_step * args.steps,
    }
    if solve:
        line["solve"] = solve
    if rank == 0 and not args.no_learned:
        # solves/s to 1 arcsec RMS, learned initial estimate vs plain LM, on the
        # 64-antenna 16-channel workload (network trained here on GPU-simulated
        # intervals with the library's kernels; sizes reduced to fit the bench)
        from paper_1709_08681_gb300 import learned_init as LI
        rep, _ = LI.run(n_train=args.learned_train, n_eval=args.learned_eval, steps=3000, batch=1024, n_geom=8,
                        seed=args.seed, log=None, n_eval_batched=64)
        line["learned_init"] = {"workload": "disk64_l16ch", **rep}
    if rank == 0 and args.mixed_intervals > 0:
        # batched solves over mixed intervals: 27/64/197-antenna arrays,
        # 30-600 time steps, offsets 10-60" with 2' outliers (one persistent
        # launch per LM iteration over all intervals, graph-replayed)
        from paper_1709_08681_gb300 import mixed as MX
        mrep, _ = MX.run(n_intervals=args.mixed_intervals, seed=args.seed)
        mrep.pop("tiling", None)
        props = torch.cuda.get_device_properties(local)
        mrep["roofline"] = {"bound": "alu", "achieved": mrep["fused_tflops"],
                            "peak": RL.fp32_peak_tflops(props.multi_processor_count), "unit": "TFLOP/s"}
        mrep["roofline"]["frac"] = mrep["roofline"]["achieved"] / mrep["roofline"]["peak"]
        line["mixed_batch"] = {"workload": "mixed_batch%d" % args.mixed_intervals, **mrep}
    if rank == 0:
        # two parallel-hand polarisations solved separately: squint and
        # mechanical offsets of every antenna (4 intervals x 2 polarisations, one batch)
        from paper_1709_08681_gb300 import squint as SQ
        srep, _, _ = SQ.run("vla27_l64ch", seed=args.seed)
        line["squint"] = {"workload": "vla27_l64ch, R and L", **srep}
    if rank == 0 and not args.no_exact:
        # the exact disk kernel (two shifted disk patterns' product) in place of
        # the Gaussian decorrelation model: throughput of its fused evaluation
        # and its solutions against the Gaussian model's, on data it simulates
        from paper_1709_08681_gb300 import exact_kernel as EK
        line["exact_kernel"] = {"workload": "vla27_l64ch, offsets sigma 60\"", **EK.run("vla27_l64ch", seed=args.seed)}
    if rank == 0 and not args.no_wsnap:
        # W-snapshots: per-interval uvw plane, model components moved to the
        # snapshot frame, their grid on the tensor cores, then the usual batch
        from paper_1709_08681_gb300 import wsnap as WS
        line["wsnap"] = {"workload": "vla27_l64ch, W-snapshot grid per interval", **WS.run("vla27_l64ch", seed=args.seed)}
    if rank == 0 and not args.no_wstack:
        # residual-w stack: all 600 time steps as one interval, the model grid
        # stacked in the w left after the plane fit, two planes read per tap
        from paper_1709_08681_gb300 import wstack as WK
        line["wstack"] = {"workload": "vla27_l64ch, 600 time steps as one interval", **WK.run("vla27_l64ch", seed=args.seed)}
    if rank == 0 and not args.no_drift:
        # full scale: 197 antennas, 128 channels, 1800 x 1 s (4.45e9 visibilities),
        # pointing drifting as a random walk, solved every 60 s (30 intervals):
        # cold batched solves vs warm-started solves in time order
        from paper_1709_08681_gb300 import drift as DR
        drep = DR.run(seed=args.seed)
        props = torch.cuda.get_device_properties(local)
        drep["roofline"] = {"bound": "alu", "achieved": drep["fused_tflops"],
                            "peak": RL.fp32_peak_tflops(props.multi_processor_count), "unit": "TFLOP/s"}
        drep["roofline"]["frac"] = drep["roofline"]["achieved"] / drep["roofline"]["peak"]
        drep["warm_latency_ms_per_interval"] = 1e3 * drep["warm_sequential_s"] / drep["n_intervals"]
        line["drift_full"] = {"workload": "drift197_l128ch", **drep}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        vis_host = vis.cpu().numpy()
        w_host = w.cpu().numpy()
        n_s, dt, n_t, _ = cpu_sample_oracle(wl, vis_host, w_host, args.cpu_seconds)
        line["cpu_baseline"] = {"value": n_s / dt / 1e9, "unit": "Gvis/s", "cores": omp_threads(), "kind": "oracle",
                                "sample": "first %d timesteps x %d baselines x %d channels (%d vis, %.1f s): FP64 "
                                          "predict + derivatives + chi^2/gradient/normal sums at zero offsets"
                                          % (n_t, wl.n_bl, wl.n_chan, n_s, dt)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sess.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
