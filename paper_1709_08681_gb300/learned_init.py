"""Learned initial estimate of the pointing offsets: simulation, training and
the comparison with plain Levenberg-Marquardt from zero.

An addition to the paper's method (which starts the minimiser from zero or
from earlier solutions).  Everything numerical runs in the CUDA library:
observed data are simulated by ``psc_predict`` at seeded offsets plus seeded
thermal noise (as the paper simulates its test data, Sec. 4.1), features
come from ``psc_features``, the network trains with ``psc_mlp_train_step``
and infers with ``psc_learned_init``; torch only holds device memory,
streams and the noise draws.

Data: a pool of observation geometries (hour-angle windows of one array and
sky, one shared model grid); each training or evaluation interval draws a
geometry, Gaussian offsets (sigma_pt per antenna per axis) and noise.
Targets are the true offsets over sigma_prior.

Comparison (per interval): the number of LM iterations and the time until
the solver's current solution is within 1 arcsec RMS of the truth, from zero
(plain) and from the network's estimate (learned); the learned time includes
the features and the network.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import _abi
from . import inputs as I
from .session import Session

SIGMA_PRIOR = 30.0 * I.ARCSEC
N_FEAT = 52


class Simulator:
    def __init__(self, name="disk64_l16ch", n_geom=8, seed=0, stream=None, ha_span_h=6.0):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.sessions = []
        grid = None
        for k in range(n_geom):
            ha = -ha_span_h / 2 + ha_span_h * (k + 0.5) / n_geom
            wl = I.make_workload(name, seed=seed, ha_centre_h=ha)
            s = Session(wl, stream=self.stream, grid=grid)
            grid = s.grid
            self.sessions.append(s)
        self.wl = self.sessions[0].wl
        self.n_ant = self.wl.n_ant
        self.gen = torch.Generator(device=self.sessions[0].device)
        self.gen.manual_seed(int(seed) * 7919 + 17)
        self.rng = np.random.default_rng([int(seed), 4242])
        self.w_scale = 1.0 / self.wl.sigma_noise ** 2

    def draw(self):
        """(geometry index, observed visibilities on the device, true offsets)."""
        k = int(self.rng.integers(len(self.sessions)))
        s = self.sessions[k]
        lm = self.rng.normal(0.0, self.wl.sigma_pt, (self.n_ant, 2))
        vis = s.empty_vis()
        s.ctxs[0].psc_predict(lm, vis)
        noise = torch.randn(vis.shape + (2,), generator=self.gen, device=vis.device) * self.wl.sigma_noise
        vis += torch.view_as_complex(noise)
        return k, vis, lm

    def features(self, k, vis, time_stride):
        return self.sessions[k].ctxs[0].psc_features(vis, None, self.w_scale, SIGMA_PRIOR, time_stride)

    def close(self):
        for s in self.sessions:
            s.close()


def make_dataset(sim: Simulator, n_intervals: int, time_stride: int = 15):
    X = torch.empty((n_intervals * sim.n_ant, N_FEAT), dtype=torch.float32, device="cuda")
    T = torch.empty((n_intervals * sim.n_ant, 2), dtype=torch.float32, device="cuda")
    for i in range(n_intervals):
        k, vis, lm = sim.draw()
        X[i * sim.n_ant:(i + 1) * sim.n_ant] = sim.features(k, vis, time_stride)
        T[i * sim.n_ant:(i + 1) * sim.n_ant] = torch.from_numpy(lm / SIGMA_PRIOR).to(torch.float32)
    return X, T


def init_params(X: torch.Tensor, seed: int) -> np.ndarray:
    """He-initialised weights, zero biases, input standardisation from X."""
    rng = np.random.default_rng([int(seed), 99])
    shapes = [(52, 256), (256,), (256, 256), (256,), (256, 256), (256,), (256, 2), (2,)]
    parts = []
    for shp in shapes:
        if len(shp) == 2:
            parts.append(rng.normal(0.0, math.sqrt(2.0 / shp[0]), shp).reshape(-1))
        else:
            parts.append(np.zeros(shp))
    xs = X.double().cpu().numpy()
    mu = xs.mean(axis=0)
    sd = xs.std(axis=0)
    sd = np.where(sd > 1e-12, sd, 1.0)
    parts += [mu, sd]
    return np.concatenate(parts).astype(np.float32)


def train(net: "_abi.Mlp", X, T, steps=2000, batch=1024, lr=1e-3, seed=0, log_every=0):
    """AdamW with a cosine learning-rate decay over shuffled minibatches."""
    n = X.shape[0]
    g = torch.Generator(device=X.device)
    g.manual_seed(int(seed) + 5)
    perm = torch.randperm(n, generator=g, device=X.device)
    Xs, Ts = X[perm].contiguous(), T[perm].contiguous()
    losses = []
    pos = 0
    for it in range(steps):
        if pos + batch > n:
            perm = torch.randperm(n, generator=g, device=X.device)
            Xs, Ts = X[perm].contiguous(), T[perm].contiguous()
            pos = 0
        rate = lr * 0.5 * (1.0 + math.cos(math.pi * it / steps))
        want = log_every and (it % log_every == 0 or it == steps - 1)
        l = net.psc_mlp_train_step(Xs[pos:pos + batch], Ts[pos:pos + batch], max(rate, 1e-6), want_loss=bool(want))
        if want:
            losses.append((it, l))
        pos += batch
    return losses


def _rms_arcsec(a, b):
    return float(np.sqrt(np.mean((np.asarray(a) - np.asarray(b)) ** 2)) / I.ARCSEC)


def _iterations_to(ctx, vis, w_scale, lm0, truth, target_arcsec, max_iter):
    """LM iterations until the solver's accepted offsets are within target RMS
    of the truth (0 if the start already is); None if never."""
    if _rms_arcsec(lm0, truth) <= target_arcsec:
        return 0
    opts = _abi.psc_solve_opts_default()
    ctx.psc_lm_begin(lm0, opts)
    ctx.psc_lm_iterate(vis, None, w_scale, 1)          # evaluation at the start, first step proposed
    for k in range(1, max_iter + 1):
        ctx.psc_lm_iterate(vis, None, w_scale, 1)      # evaluates the trial, accepts or rejects
        lm, rep = ctx.psc_lm_end()
        if _rms_arcsec(lm, truth) <= target_arcsec:
            return k
        if rep.reason != 0:
            return None
    return None


def evaluate(sim: Simulator, net: "_abi.Mlp", n_eval: int, time_stride=15, target_arcsec=1.0, max_iter=20):
    """Per-interval iterations to the target from zero and from the network,
    and the measured times of one LM iteration and of the learned estimate."""
    plain_it, learned_it, init_rms = [], [], []
    stream = sim.stream
    for _ in range(n_eval):
        k, vis, lm = sim.draw()
        ctx = sim.sessions[k].ctxs[0]
        lm_init = ctx.psc_learned_init(net, vis, None, sim.w_scale, SIGMA_PRIOR, time_stride)
        init_rms.append(_rms_arcsec(lm_init, lm))
        plain_it.append(_iterations_to(ctx, vis, sim.w_scale, np.zeros_like(lm), lm, target_arcsec, max_iter))
        learned_it.append(_iterations_to(ctx, vis, sim.w_scale, lm_init, lm, target_arcsec, max_iter))
    # device times (CUDA events on the stream): one LM iteration (fused
    # evaluation + reductions + update) and the learned estimate (features +
    # network)
    k, vis, lm = sim.draw()
    ctx = sim.sessions[k].ctxs[0]
    opts = _abi.psc_solve_opts_default()
    ctx.psc_lm_begin(np.zeros_like(lm), opts)
    ctx.psc_lm_iterate(vis, None, sim.w_scale, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(stream)
    for _ in range(reps):
        ctx.psc_lm_restart()
        ctx.psc_lm_iterate(vis, None, sim.w_scale, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    t_iter = e0.elapsed_time(e1) / reps / 1e3
    feat = sim.features(k, vis, time_stride)
    net.psc_mlp_forward(feat)
    e0.record(stream)
    for _ in range(reps):
        sim.features(k, vis, time_stride)
        net.psc_mlp_forward(feat)
    e1.record(stream)
    torch.cuda.synchronize()
    t_init = [e0.elapsed_time(e1) / reps / 1e3] * n_eval
    ok_p = [x for x in plain_it if x is not None]
    ok_l = [x for x in learned_it if x is not None]
    # time to the target: every iteration after the first costs one evaluation
    # and update; the first also pays the evaluation at the start point
    tp = [(x + 1) * t_iter for x in ok_p]
    tl = [ti + (x + 1) * t_iter if x > 0 else ti for x, ti in zip(learned_it, t_init) if x is not None]
    return {
        "n_eval": n_eval,
        "plain_mean_iters": float(np.mean(ok_p)) if ok_p else None,
        "learned_mean_iters": float(np.mean(ok_l)) if ok_l else None,
        "plain_reached": len(ok_p), "learned_reached": len(ok_l),
        "learned_init_rms_arcsec": float(np.median(init_rms)),
        "t_lm_iter_ms": 1e3 * t_iter, "t_learned_init_ms": 1e3 * float(np.median(t_init)),
        "plain_intervals_per_s": len(tp) / sum(tp) if tp else None,
        "learned_intervals_per_s": len(tl) / sum(tl) if tl else None,
        "target_arcsec": target_arcsec,
    }


def _batch_rms_trace(batch, lm0, truth, max_iter):
    """Per-interval RMS error (arcsec) after 0..max_iter batched LM
    iterations from lm0; [max_iter + 1][n]."""
    opts = _abi.psc_solve_opts_default()
    batch.psc_batch_begin(lm0, opts)
    trace = [[_rms_arcsec(a, b) for a, b in zip(lm0, truth)]]
    batch.psc_batch_iterate(1)                       # evaluation at the start, first step proposed
    for _ in range(max_iter):
        batch.psc_batch_iterate(1)                   # evaluates the trial, accepts or rejects
        lm, _ = batch.psc_batch_end()
        trace.append([_rms_arcsec(a, b) for a, b in zip(lm, truth)])
    return np.asarray(trace)


def evaluate_batched(sim: Simulator, net: "_abi.Mlp", n_eval: int, time_stride=15, target_arcsec=1.0,
                     max_iter=10, reps=5):
    """The held-out intervals solved as one batch (one persistent launch per
    LM iteration over all of them), from zero and from the network's
    estimate.  Iterations to the target: the first batched iteration after
    which every interval is within target_arcsec RMS of its truth.  Times
    (CUDA events on the stream): a batched iteration, and the learned
    estimate of all intervals (features of each, then one network forward
    over all their antennas)."""
    stream = sim.stream
    draws = [sim.draw() for _ in range(n_eval)]
    # one context per interval (a batch holds each context once); they borrow
    # the geometry's uvw and the shared grid
    ctxs = []
    for k, vis, lm in draws:
        s = sim.sessions[k]
        wl = s.wl
        g = s.grid_args
        ctxs.append(_abi.Context(wl.n_ant, wl.n_time, wl.n_chan, s.uvw, wl.freq_hz, wl.ap_kind, wl.diam_m,
                                 wl.alpha_per_dlambda, wl.decorrelation, g["n_img"], g["n_grid"], g["cell_rad"],
                                 g["support"], g["oversample"], s.grid, stream))
    vis = [d[1] for d in draws]
    truth = [d[2] for d in draws]
    n_ant = sim.n_ant
    feats = torch.empty((n_eval * n_ant, N_FEAT), dtype=torch.float32, device=vis[0].device)
    y = torch.empty((n_eval * n_ant, 2), dtype=torch.float32, device=vis[0].device)

    def learned_estimate():
        for j, c in enumerate(ctxs):
            c.psc_features(vis[j], None, sim.w_scale, SIGMA_PRIOR, time_stride, out=feats[j * n_ant:(j + 1) * n_ant])
        net.psc_mlp_forward(feats, out=y)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    learned_estimate()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        learned_estimate()
    e1.record(stream)
    torch.cuda.synchronize()
    t_init = e0.elapsed_time(e1) / reps / 1e3
    lm_init = [(y[j * n_ant:(j + 1) * n_ant].double().cpu().numpy() * SIGMA_PRIOR) for j in range(n_eval)]
    w_scale = [sim.w_scale] * n_eval
    batch = _abi.Batch(ctxs, vis, None, w_scale=w_scale, stream=stream)
    batch.psc_batch_autotune()
    zeros = [np.zeros_like(t) for t in truth]
    plain = _batch_rms_trace(batch, zeros, truth, max_iter)
    learned = _batch_rms_trace(batch, lm_init, truth, max_iter)
    # batched iteration time (graph replay), event-timed
    batch.psc_batch_begin(zeros)
    batch.psc_batch_iterate(2)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        batch.psc_batch_restart()
        batch.psc_batch_iterate(1)
    e1.record(stream)
    torch.cuda.synchronize()
    t_iter = e0.elapsed_time(e1) / reps / 1e3
    batch.close()
    for c in ctxs:
        c.close()

    def first_all(trace):
        ok = np.nonzero(np.all(trace <= target_arcsec, axis=1))[0]
        return int(ok[0]) if len(ok) else None

    def mean_first(trace):
        it = [np.nonzero(trace[:, j] <= target_arcsec)[0] for j in range(trace.shape[1])]
        return float(np.mean([x[0] if len(x) else np.nan for x in it]))

    kp, kl = first_all(plain), first_all(learned)
    # time to the target: the start evaluation plus k iterations (none if the
    # start already meets it); the learned arm adds its estimate
    tp = (kp + 1) * t_iter if kp is not None and kp > 0 else (0.0 if kp == 0 else None)
    tl = (t_init + ((kl + 1) * t_iter if kl > 0 else 0.0)) if kl is not None else None
    return {
        "n_eval": n_eval, "batched": True,
        "plain_iters_all": kp, "learned_iters_all": kl,
        "plain_mean_iters": mean_first(plain), "learned_mean_iters": mean_first(learned),
        "learned_init_rms_arcsec": float(np.median(learned[0])),
        "t_batch_iter_ms": 1e3 * t_iter, "t_learned_init_ms": 1e3 * t_init,
        "plain_intervals_per_s": n_eval / tp if tp else None,
        "learned_intervals_per_s": n_eval / tl if tl else None,
        "target_arcsec": target_arcsec,
    }


def run(n_train=2000, n_eval=50, steps=2000, batch=1024, lr=1e-3, n_geom=8, seed=0, time_stride=15, log=print,
        n_eval_batched=0):
    """Simulate, train and evaluate (per interval, and as one batch of
    n_eval_batched held-out intervals if > 0); returns (report, params)."""
    stream = torch.cuda.current_stream()
    sim = Simulator(n_geom=n_geom, seed=seed, stream=stream)
    t = time.perf_counter()
    X, T = make_dataset(sim, n_train, time_stride)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t
    net = _abi.Mlp(max(batch, sim.n_ant, n_eval_batched * sim.n_ant), stream=stream)
    net.psc_mlp_set_params(init_params(X, seed))
    t = time.perf_counter()
    losses = train(net, X, T, steps=steps, batch=batch, lr=lr, seed=seed, log_every=max(1, steps // 10))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t
    if log:
        log("train losses: " + ", ".join("%d:%.4f" % x for x in losses))
    # held-out evaluation draws continue the same seeded stream
    rep = evaluate(sim, net, n_eval, time_stride)
    if n_eval_batched > 0:
        rep["batched"] = evaluate_batched(sim, net, n_eval_batched, time_stride)
    rep.update({"n_train_intervals": n_train, "n_train_samples": int(X.shape[0]), "train_steps": steps,
                "batch": batch, "t_simulate_s": t_data, "t_train_s": t_train,
                "final_train_loss": losses[-1][1] if losses else None})
    params = net.psc_mlp_get_params()
    net.close()
    sim.close()
    return rep, params


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-intervals", type=int, default=2000)
    ap.add_argument("--eval-intervals", type=int, default=50)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    rep, _ = run(n_train=a.train_intervals, n_eval=a.eval_intervals, steps=a.steps, seed=a.seed)
    print(json.dumps(rep))
