"""Continuous-batching serving loop for OPO simulations.

Requests (an ``OPOConfig`` plus a round-trip budget M) arrive over time.
Every tick the loop

1. moves arrived requests into the wait queue;
2. admits waiting requests first-come first-served while the GPU share and
   the device-memory budget allow: a fused instance of a size class takes
   1/capacity of the GPU, capacity being how many clusters of that class can
   be resident at once (the library's occupancy query), a plain-path instance
   a fixed share; admission configures device state that then stays on the
   device until the request retires;
3. advances every active instance by the same K round trips in one batch:
   fused instances grouped by size class inside the library, instances too
   large for the fused path (or all of them, with ``path="plain"``) in
   batched plain-path groups; the launches of newly admitted requests overlap
   with the work of those already running;
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

def instance_bytes(n, nfields, precision):
    """Device bytes of one context (fields, output, scratch, tables, staging)."""
    csz = 16 if precision == opo.OPO_FP64 else 8
    return csz * n * (7 * nfields + 2) + 16 * 2 * n * 2 + 4096 * 8 * 4


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
        self.k = 0


class Server:
    """Runs requests on one GPU with continuous batching.

    ``tick_rt``: round trips per tick (latency granularity).  ``gpu_share``:
    fraction of the GPU the active instances may fill (1.0: as many as can be
    resident at once).  ``hbm_budget``:
    device bytes for instance state (default: half of the free memory).
    ``launch``: optional callable ``(n, nfields, precision) -> (cluster,
    threads, rt_per_launch)`` (e.g. from the autotuner); default shapes
    otherwise.  ``path="plain"`` runs every request on the batched plain
    path (one kernel per operation) with the same admission shares the fused
    path would get, so that the two forms are compared on the same trace.
    Device state of retired requests is kept in a pool per
    (N, field count) and reconfigured for the next request of that class, so
    admission allocates only when a class needs more instances than ever
    before.  The loop is pipelined: while a tick runs on the GPU, arrivals
    are admitted and prepared for the next tick.
    """

    def __init__(self, precision=opo.OPO_FP32_PH64, device=0, tick_rt=16, gpu_share=1.0,
                 hbm_budget=None, launch=None, plain_share=0.1, path="auto"):
        import torch
        self.precision = precision
        self.device = device
        self.tick_rt = int(tick_rt)
        self.gpu_share = float(gpu_share)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget = free // 2
        self.hbm_budget = int(hbm_budget)
        self.launch = launch
        self.plain_share = float(plain_share)
        if path not in ("auto", "plain"):
            raise ValueError("path is 'auto' or 'plain'")
        self.path = path
        self.capacity = {}  # (n, F, cluster, threads) -> resident clusters
        self.results = []
        self.ticks = 0
        self.busy_s = 0.0
        self.field_steps = 0.0
        self.pool = collections.defaultdict(list)   # (n, F) -> idle contexts
        self.pooled_bytes = 0
        self.allocations = 0

    # ---------------------------------------------------------------- admission
    def _shape(self, cfg):
        if self.launch is not None:
            shape = self.launch(cfg.n, cfg.nfields, self.precision)
            if shape:
                return shape
        return (0, 0, 0)

    def _context(self, cfg):
        key = (cfg.n, cfg.nfields)
        if self.pool[key]:
            ctx = self.pool[key].pop()
            self.pooled_bytes -= instance_bytes(cfg.n, cfg.nfields, self.precision)
            ctx.reset(cfg)
            return ctx
        self.allocations += 1
        # a private stream per instance: plain-path instances overlap with the
        # batched fused launch, which fences each member's stream with events
        return opo.Context(cfg, precision=self.precision, device=self.device)

    def _admit(self, req, now, share_used, mem_used):
        cfg = req.cfg
        need_mem = instance_bytes(cfg.n, cfg.nfields, self.precision)
        pooled = bool(self.pool[(cfg.n, cfg.nfields)])
        if not pooled and mem_used + self.pooled_bytes + need_mem > self.hbm_budget:
            return None
        ctx = self._context(cfg)
        cl, th, rtpl = self._shape(cfg)
        path, cluster = opo.OPO_PATH_FUSED, 0
        try:
            ctx.set_path(opo.OPO_PATH_FUSED, cl, rtpl, th)
            key = (cfg.n, cfg.nfields, cl, th)
            if key not in self.capacity:
                self.capacity[key] = opo.opo_fused_capacity(ctx.h, cl, th)
            cap, cluster = self.capacity[key]
            share = 1.0 / max(1, cap)
        except opo.OPOError:
            path, cluster = opo.OPO_PATH_PLAIN, 0
            share = self.plain_share
        if self.path == "plain":
            path, cluster = opo.OPO_PATH_PLAIN, 0
        if path == opo.OPO_PATH_PLAIN:
            ctx.set_path(opo.OPO_PATH_PLAIN)
        if share_used + share > self.gpu_share + 1e-9 and share_used > 0:
            self._release(ctx, cfg)
            return None
        a = _Active(req, ctx, path, cluster, now)
        a.mem = need_mem
        a.share = share
        return a

    def _release(self, ctx, cfg):
        self.pool[(cfg.n, cfg.nfields)].append(ctx)
        self.pooled_bytes += instance_bytes(cfg.n, cfg.nfields, self.precision)

    # -------------------------------------------------------------------- loop
    def run(self, requests, time_scale=1.0, clock=time.perf_counter, max_wall_s=None):
        """Replay ``requests`` (arrival times in seconds, scaled by
        ``time_scale``) in real time; returns the list of ``Result``."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active, ready = [], []
        budget = {"share": 0.0, "mem": 0}
        t0 = clock()
        batches = {}  # (k, member ids) -> batch handle

        def admit():
            now = clock() - t0
            while pending and pending[0].arrival * time_scale <= now:
                waiting.append(pending.popleft())
            while waiting:
                a = self._admit(waiting[0], now, budget["share"], budget["mem"])
                if a is None:
                    break
                waiting.popleft()
                ready.append(a)
                budget["share"] += a.share
                budget["mem"] += a.mem

        def drop_batches():
            for b in batches.values():
                opo.opo_batch_destroy(b)
            batches.clear()

        while pending or waiting or active or ready:
            if max_wall_s is not None and clock() - t0 > max_wall_s:
                break
            admit()
            active.extend(ready)
            ready.clear()
            if not active:
                if pending:
                    wait = pending[0].arrival * time_scale - (clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.005))
                continue
            # ---- launch one tick: instances finishing inside the tick run
            # their remainder in a batch of their own
            t_tick = clock()
            groups = collections.defaultdict(list)
            for a in active:
                a.k = min(self.tick_rt, a.req.rounds - a.done)
                groups[a.k].append(a)
            live = set()
            for k, members in groups.items():
                key = (k, tuple(id(a) for a in members))
                live.add(key)
                if key not in batches:
                    batches[key] = opo.opo_batch_create([a.ctx.h for a in members], 0, 0)
                opo.opo_batch_run(batches[key], k)
            for key in [kk for kk in batches if kk not in live]:
                opo.opo_batch_destroy(batches.pop(key))
            # ---- while the GPU works: admit and prepare the next arrivals
            admit()
            # ---- finish the tick
            for a in active:
                a.trace.append(a.ctx.trace(a.k))  # waits for this instance's stream
            self.busy_s += clock() - t_tick
            self.ticks += 1
            finished = [a for a in active if a.done + a.k >= a.req.rounds]
            if finished:
                drop_batches()  # batches point at their members
            keep = []
            for a in active:
                a.done += a.k
                cfg = a.req.cfg
                self.field_steps += cfg.nfields * cfg.nz * a.k
                if a.done >= a.req.rounds:
                    out = a.ctx.get_fields(opo.OPO_OUTPUT)
                    self.results.append(Result(
                        a.req.rid, cfg.n, cfg.nfields, a.req.rounds, a.req.arrival * time_scale,
                        a.admitted, clock() - t0, a.path, out, np.concatenate(a.trace)))
                    budget["share"] -= a.share
                    budget["mem"] -= a.mem
                    self._release(a.ctx, cfg)
                else:
                    keep.append(a)
            active = keep
        drop_batches()
        for a in active + ready:
            a.ctx.close()
        self.close()
        return self.results

    def close(self):
        for lst in self.pool.values():
            for ctx in lst:
                ctx.close()
        self.pool.clear()
        self.pooled_bytes = 0


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
