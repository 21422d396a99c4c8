"""Autotuner for the fused path: picks the launch shape of an instance class.

An instance class is (N, field count, precision, nonlinear-step variant:
chi(2) with a phase mismatch somewhere, chi(2) with dk = 0 in every crystal,
or with the Kerr terms -- the library runs each on its own kernel, and the
Kerr kernel prefers larger CTAs than the chi(2) ones).  Candidates are
(cluster size, threads per CTA, round trips per launch); each candidate that
the library accepts is timed on a batch that fills the GPU (as many
co-resident clusters as the occupancy query allows) with CUDA events on the
launch stream, and the one with the highest field-steps/s wins.  The choice
depends only on the class, never on the mix an instance later runs in, so a
result does not depend on which batch it was computed in.

Results are cached per process and optionally in a JSON file.
"""
from __future__ import annotations

import json
import os
import threading

from . import opo

CLUSTERS = (1, 2, 4, 8, 16)
THREADS = (0, 128, 192, 256, 384, 512)
RT_PER_LAUNCH = (16, 64)

_cache = {}
_lock = threading.Lock()


def variant(cfg):
    """The nonlinear-step variant of an ``OPOConfig``: "kerr" if any crystal
    has an n2, else "chi2" if any has a phase mismatch, else "chi2_dk0"."""
    crystals = (cfg,) + tuple(getattr(cfg, "extra_crystals", ()) or ())
    if any(getattr(k, "n2", 0.0) != 0.0 for k in crystals):
        return "kerr"
    if any(getattr(k, "dk", 0.0) != 0.0 for k in crystals):
        return "chi2"
    return "chi2_dk0"


def _key(n, nfields, precision, var="chi2_dk0"):
    return "%d/%d/%d/%s" % (int(n), int(nfields), int(precision), var)


def load(path):
    """Merge a JSON cache written by :func:`save`."""
    if path and os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
        with _lock:
            _cache.update(data)


def save(path):
    with _lock:
        data = dict(_cache)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(n, nfields, precision, var="chi2_dk0"):
    with _lock:
        return _cache.get(_key(n, nfields, precision, var))


def pick(results):
    """The winning shape of a list of timed candidates (dicts with
    "field_steps_per_s" and "threads"), tagged with the candidate count, or
    None for an empty list.  Shapes within 1% of the fastest are a tie: the
    one with the most threads per CTA wins (more warps to hide latency;
    heavier per-point work such as the Kerr terms keeps more of its speed
    there)."""
    if not results:
        return None
    top = max(r["field_steps_per_s"] for r in results)
    ties = [r for r in results if r["field_steps_per_s"] >= 0.99 * top]
    best = max(ties, key=lambda r: (r["threads"], r["field_steps_per_s"]))
    return dict(best, candidates=len(results))


def tune(cfg, precision=opo.OPO_FP32_PH64, device=0, round_trips=2, candidates=None, reps=3):
    """Time every accepted launch shape for the class of ``cfg``; return the
    best as ``{"cluster", "threads", "rt_per_launch", "field_steps_per_s"}``.

    ``cfg`` is an ``OPOConfig``; its physics only sets the work per step (all
    instances of a class cost the same).
    """
    import torch

    var = variant(cfg)
    hit = lookup(cfg.n, cfg.nfields, precision, var)
    if hit is not None:
        return hit
    stream = torch.cuda.Stream(device=device)
    results = []
    cands = candidates or [(c, t, r) for c in CLUSTERS for t in THREADS for r in RT_PER_LAUNCH]
    probe = opo.Context(cfg, precision=precision, device=device, stream=stream.cuda_stream)
    try:
        for (cl, th, rtpl) in cands:
            try:
                active, cl_used = opo.opo_fused_capacity(probe.h, cl, th)
            except opo.OPOError:
                continue
            if active < 1:
                continue
            ctxs = [probe] + [opo.Context(cfg.replace(instance=cfg.instance + i + 1),
                                          precision=precision, device=device,
                                          stream=stream.cuda_stream)
                              for i in range(active - 1)]
            try:
                for c in ctxs:
                    c.set_path(opo.OPO_PATH_FUSED, cl_used, rtpl, th)
                batch = opo.opo_batch_create([c.h for c in ctxs], cl_used, th)
                sec = float("inf")
                with torch.cuda.stream(stream):
                    opo.opo_batch_run(batch, 1)  # warm-up
                    # best of a few timings: one short timing is at the
                    # mercy of clock ramps and launch jitter, and shapes
                    # within a few percent of each other swap places
                    for _ in range(reps):
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        opo.opo_batch_run(batch, round_trips)
                        e1.record(stream)
                        e1.synchronize()
                        sec = min(sec, e0.elapsed_time(e1) * 1e-3)
                opo.opo_batch_destroy(batch)
                fs = active * cfg.nfields * cfg.nz * round_trips / sec
                results.append({"cluster": cl_used, "threads": th, "rt_per_launch": rtpl,
                                "field_steps_per_s": fs, "instances": active})
            except opo.OPOError:
                pass
            finally:
                for c in ctxs[1:]:
                    c.close()
    finally:
        probe.close()
    best = pick(results)
    if best is None:
        return None
    with _lock:
        _cache[_key(cfg.n, cfg.nfields, precision, var)] = best
    return best


__all__ = ["tune", "pick", "variant", "lookup", "load", "save"]
