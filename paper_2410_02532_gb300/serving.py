"""Continuous-batching serving loop for OPO simulations.

Requests (an ``OPOConfig`` plus a round-trip budget M) arrive over time.
Every tick the loop

1. moves arrived requests into the wait queue;
2. admits waiting requests first-come first-served while the SM budget (sum
   of cluster sizes of active fused instances, plus a fixed share per plain
   instance) and the device-memory budget allow: admission creates the
   instance's device state, which then stays on the device until it retires;
3. advances every active instance by the same K round trips: all fused
   instances in one batched launch (grouped by size class inside the
   library), instances too large for the fused path on the plain path on their
   own streams; the launches of newly admitted requests overlap with the work
   of those already running;
4. retires finished instances (output fields and trace copied to the host)
   and records latency = completion time - arrival time.

Each instance advances exactly as it would alone (same kernels, launch shape
and round-trip chunking do not change its arithmetic), so a result does not
depend on the mix it ran in; ``tests/test_gpu_serving.py`` checks this.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import opo
from . import workloads as W

SMS = 152


def instance_bytes(n, nfields, precision):
    """Device bytes of one context (fields, output, scratch, tables, staging)."""
    csz = 16 if precision == opo.OPO_FP64 else 8
    return csz * n * (5 * nfields + 2) + 16 * 2 * n * 2 + 4096 * 8 * 4


@dataclasses.dataclass
class Request:
    rid: int
    cfg: W.OPOConfig
    rounds: int
    arrival: float = 0.0


@dataclasses.dataclass
class Result:
    rid: int
    n: int
    nfields: int
    rounds: int
    arrival: float
    admitted: float
    finished: float
    path: int
    out_fields: np.ndarray
    trace: np.ndarray

    @property
    def latency(self):
        return self.finished - self.arrival


class _Active:
    def __init__(self, req, ctx, path, cluster, admitted):
        self.req = req
        self.ctx = ctx
        self.path = path
        self.cluster = cluster
        self.done = 0
        self.admitted = admitted
        self.trace = []


class Server:
    """Runs requests on one GPU with continuous batching.

    ``tick_rt``: round trips per tick (latency granularity).  ``sm_budget``:
    SMs the active fused instances may occupy (default: all).  ``hbm_budget``:
    device bytes for instance state (default: half of the free memory).
    ``launch``: optional callable ``(n, nfields, precision) -> (cluster,
    threads, rt_per_launch)`` (e.g. from the autotuner); default shapes
    otherwise.
    """

    def __init__(self, precision=opo.OPO_FP32_PH64, device=0, tick_rt=16, sm_budget=SMS,
                 hbm_budget=None, launch=None, plain_sm_share=16):
        import torch
        self.torch = torch
        self.precision = precision
        self.device = device
        self.tick_rt = int(tick_rt)
        self.sm_budget = int(sm_budget)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget = free // 2
        self.hbm_budget = int(hbm_budget)
        self.launch = launch
        self.plain_sm_share = plain_sm_share
        self.results = []
        self.ticks = 0
        self.busy_s = 0.0
        self.field_steps = 0.0

    # ---------------------------------------------------------------- admission
    def _shape(self, cfg):
        if self.launch is not None:
            shape = self.launch(cfg.n, cfg.nfields, self.precision)
            if shape:
                return shape
        return (0, 0, 0)

    def _admit(self, req, now, sm_used, mem_used):
        cfg = req.cfg
        need_mem = instance_bytes(cfg.n, cfg.nfields, self.precision)
        if mem_used + need_mem > self.hbm_budget:
            return None
        # a private stream per instance: plain-path instances overlap with the
        # batched fused launch, which fences each member's stream with events
        ctx = opo.Context(cfg, precision=self.precision, device=self.device)
        cl, th, rtpl = self._shape(cfg)
        path, cluster = opo.OPO_PATH_FUSED, 0
        try:
            ctx.set_path(opo.OPO_PATH_FUSED, cl, rtpl, th)
            _, cluster = opo.opo_fused_capacity(ctx.h, cl, th)
        except opo.OPOError:
            path, cluster = opo.OPO_PATH_PLAIN, 0
            ctx.set_path(opo.OPO_PATH_PLAIN)
        share = cluster if path == opo.OPO_PATH_FUSED else self.plain_sm_share
        if sm_used + share > self.sm_budget and sm_used > 0:
            ctx.close()
            return None
        a = _Active(req, ctx, path, cluster, now)
        a.mem = need_mem
        a.share = share
        return a

    # -------------------------------------------------------------------- loop
    def run(self, requests, time_scale=1.0, clock=time.perf_counter, max_wall_s=None):
        """Replay ``requests`` (arrival times in seconds, scaled by
        ``time_scale``) in real time; returns the list of ``Result``."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active = []
        sm_used = mem_used = 0
        t0 = clock()
        batch = None
        batch_members = None
        while pending or waiting or active:
            now = clock() - t0
            if max_wall_s is not None and now > max_wall_s:
                break
            while pending and pending[0].arrival * time_scale <= now:
                waiting.append(pending.popleft())
            while waiting:
                a = self._admit(waiting[0], now, sm_used, mem_used)
                if a is None:
                    break
                waiting.popleft()
                active.append(a)
                sm_used += a.share
                mem_used += a.mem
            if not active:
                if pending:
                    wait = pending[0].arrival * time_scale - (clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                continue
            k = min(self.tick_rt, min(a.req.rounds - a.done for a in active))
            fused = [a for a in active if a.path == opo.OPO_PATH_FUSED]
            plain = [a for a in active if a.path == opo.OPO_PATH_PLAIN]
            members = tuple(id(a) for a in fused)
            if members != batch_members:
                if batch is not None:
                    opo.opo_batch_destroy(batch)
                batch = opo.opo_batch_create([a.ctx.h for a in fused], 0, 0) if fused else None
                batch_members = members
            t_tick = clock()
            if batch is not None:
                opo.opo_batch_run(batch, k)
            for a in plain:
                opo.opo_run_roundtrips(a.ctx.h, k)
            for a in active:
                a.trace.append(a.ctx.trace(k))  # waits for this instance's stream
            self.busy_s += clock() - t_tick
            self.ticks += 1
            now = clock() - t0
            if any(a.done + k >= a.req.rounds for a in active) and batch is not None:
                # the batch points at its members: drop it before any retires
                opo.opo_batch_destroy(batch)
                batch, batch_members = None, None
            keep = []
            for a in active:
                a.done += k
                cfg = a.req.cfg
                self.field_steps += cfg.nfields * cfg.nz * k
                if a.done >= a.req.rounds:
                    out = a.ctx.get_fields(opo.OPO_OUTPUT)
                    self.results.append(Result(
                        a.req.rid, cfg.n, cfg.nfields, a.req.rounds, a.req.arrival * time_scale,
                        a.admitted, clock() - t0, a.path, out, np.concatenate(a.trace)))
                    sm_used -= a.share
                    mem_used -= a.mem
                    a.ctx.close()
                else:
                    keep.append(a)
            active = keep
        if batch is not None:
            opo.opo_batch_destroy(batch)
        for a in active:
            a.ctx.close()
        return self.results


def latency_stats(results):
    lat = np.array([r.latency for r in results])
    if lat.size == 0:
        return {"p50_s": None, "p99_s": None, "count": 0}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "count": int(lat.size)}


def poisson_trace(count, rate_hz, seed=20241008, n_exps=(12, 13, 14, 15), rounds=(100, 5000),
                  fields=(2, 3)):
    """Seeded request stream: Poisson arrivals, N = 2^e with e uniform over
    ``n_exps``, M uniform over ``rounds``, F uniform over ``fields``; CW or
    sech^2 pump with parameters drawn from the preset ranges."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    base16k = W.cw_sro_16k()
    for i in range(count):
        t += rng.exponential(1.0 / rate_hz)
        n = 1 << int(rng.choice(n_exps))
        F = int(rng.choice(fields))
        M = int(rng.integers(rounds[0], rounds[1] + 1))
        level = float(rng.uniform(1.5, 5.0))
        if F == 2:
            cfg = W.degenerate_2field(n=n, level=level).replace(nz=100, length=float(rng.uniform(5e-3, 30e-3)))
        else:
            cfg = W.OPOConfig(n=n, nz=100, length=float(rng.uniform(5e-3, 30e-3)),
                              dbeta1=base16k.dbeta1, beta2=base16k.beta2, beta3=base16k.beta3)
            if rng.random() < 0.5:
                cfg = cfg.replace(pump_kind=W.PUMP_SECH2, pump_fwhm=float(rng.uniform(0.2e-12, 2e-12)),
                                  eom_beta=0.5, eom_f=10e9, delay=float(rng.uniform(-20e-15, 20e-15)))
        cfg = cfg.replace(name="req%d" % i, seed=seed, instance=i)
        cfg = cfg.replace(pump_power=level * W.sro_threshold_power(cfg))
        reqs.append(Request(i, cfg, M, t))
    return reqs


def request_work(req):
    """Point-field-steps of a request."""
    c = req.cfg
    return c.n * c.nfields * c.nz * req.rounds


__all__ = ["Server", "Request", "Result", "latency_stats", "poisson_trace", "instance_bytes",
           "request_work"]
