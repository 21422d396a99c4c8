#!/usr/bin/env python
"""Benchmark of the OPO split-step hot path on GB300.

Workload: the 2^14-point singly resonant CW OPO (100 ps window, 3 fields,
20 mm crystal, 100 z-steps, GVM/GVD/TOD, intracavity GDD -500 fs^2, pump at
4x threshold), FP32 fields with FP64 phase arguments.  One step is one round
trip (entry, 100 split-step z-steps, observables, cavity) of a batch of
independent instances of that workload (seeds differ) sized to fill the GPU
with one thread-block cluster per instance, run by the fused persistent
kernel.  Metric: field-steps/s (one length-N field through one full z-step).

Also reported: the same instance alone on the fused and on the plain
(one-kernel-per-operation, graph-replayed) path; an end-to-end number
through the C ABI with host buffers; the FP64 CPU oracle as the CPU baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU (torchrun), each rank runs its own batch
(weak scaling, no collective on the data path); timing is the max over
ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SSFM field-steps/s at N=2^14 (fused, batched round trips)"
# (instances, cluster, threads requested) -> DRAM bytes per fused launch of the
# 2^14 workload (dram__bytes_read.sum + dram__bytes_write.sum of one ncu
# capture of the current kernel in that launch shape): 8-CTA clusters of 128
# threads (cluster size compiled in), 48.13 MB read + 0.80 MB written
PROFILED_SHAPES = {(36, 8, 128): 48932608.0}
UNIT = "field-steps/s"
PEAK_SM_MHZ = 2070.0          # GB300 maximum SM clock
SMS = 152
FP32_LANES = 128              # FP32 FMA lanes per SM
FP64_NOMINAL_TFLOPS = 1.25    # GB300 FP64 (non-tensor), nominal


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=0, help="instances per GPU (0: fill the GPU)")
    ap.add_argument("--cluster", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (0: default)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--workload", choices=["cw_sro_16k", "sync_pumped_131072"],
                    default="cw_sro_16k",
                    help="the timed batch's workload (default: the 2^14 CW SRO; the other is the "
                         "2^17-point sync-pumped OPO, for profiling its kernel)")
    ap.add_argument("--path", choices=["fused", "plain"], default="fused",
                    help="fused persistent kernel (default) or the batched plain chain, for "
                         "profiling")
    ap.add_argument("--skip-extras", action="store_true",
                    help="only the headline number (no plain/e2e/cpu legs)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-tune", action="store_true", help="default launch shape, no autotuning")
    ap.add_argument("--serving-full", type=int, default=0, metavar="COUNT",
                    help="also serve the request stream at its stated budgets (100-5000 round "
                         "trips): the 200/s trace for 90 s and COUNT requests at 0.7 capacity")
    return ap.parse_args()


def total_nz(cfg):
    """z-steps of one round trip: every crystal's."""
    return cfg.nz + sum(c.nz for c in getattr(cfg, "extra_crystals", ()))


def flops_per_roundtrip(cfg):
    """Algorithmic FLOPs of one round trip of one instance (the roofline's model).

    per point-field per z-step: two FFTs 2 * 5 log2 N, dispersion multiply 6,
    two RK4 half steps 2 * rk4 where rk4 = 58 (3 fields) / 62 (2 fields) per
    point-field, +24 / +18 with the e^{i dk z} factor, +52 / +44 with the Kerr
    terms; per round trip and
    point-field: cavity FFT pair 10 log2 N plus 6 (spectral factor) plus 6
    (mirror).
    """
    n, F, nz = cfg.n, cfg.nfields, total_nz(cfg)
    lg = math.log2(n)
    if F == 3:
        rk4 = 58.0 + (24.0 if cfg.dk != 0 else 0.0)
    else:
        rk4 = 62.0 + (18.0 if cfg.dk != 0 else 0.0)
    if getattr(cfg, "n2", 0.0) != 0.0:
        # Kerr terms per stage and point-field: |A|^2 (3), sum_y G_xy |A_y|^2
        # (2F), g A into the stage value (4)
        rk4 += 4.0 * (3.0 + 2.0 * F + 4.0)
    per_step = 10.0 * lg + 6.0 + 2.0 * rk4
    per_rt = 10.0 * lg + 12.0
    return n * F * (nz * per_step + per_rt)


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the timed region starts once the sampler is writing samples
        t0 = time.time()
        while time.time() - t0 < 3.0:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                break
            time.sleep(0.01)

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        out.update(sm_mhz=statistics.median(sm) if sm else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=sorted(reasons),
                   samples=len(rows))
        return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    """The FP64 CPU oracle as it stands, one round trip of one instance per
    step, single-threaded on the host."""
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    from oracle import oracle as orc
    from paper_2410_02532_gb300 import workloads as W
    cfg = W.cw_sro_16k()
    p = orc.params(cfg)
    pump = orc.pump_profile(p, cfg.pump_kind, cfg.pump_power, cfg.pump_fwhm)
    a = cfg.initial_fields()
    m = 0
    for _ in range(args.warmup):
        a, _, _, _ = orc.run(p, a, pump, m, 1)
        m += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        a, _, _, _ = orc.run(p, a, pump, m, 1)
        m += 1
    dt = time.perf_counter() - t0
    fs = cfg.nfields * cfg.nz * args.steps
    val = fs / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded noise)",
        "config": {"workload": cfg.name + " x1 instance (oracle sample)", "n": cfg.n,
                   "fields": cfg.nfields, "nz": cfg.nz, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d round trips of one 2^14-point instance" % args.steps},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(seconds):
    from oracle import oracle as orc
    from paper_2410_02532_gb300 import workloads as W
    cfg = W.cw_sro_16k()
    p = orc.params(cfg)
    pump = orc.pump_profile(p, cfg.pump_kind, cfg.pump_power, cfg.pump_fwhm)
    a = cfg.initial_fields()
    t0 = time.perf_counter()
    rts = 0
    while True:
        a, _, _, _ = orc.run(p, a, pump, rts, 1)
        rts += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": cfg.nfields * cfg.nz * rts / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d round trip(s) of one 2^14-point, 3-field, 100-step instance "
                      "(FP64, single thread, %.1f s)" % (rts, dt)}


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch
    from paper_2410_02532_gb300 import opo
    from paper_2410_02532_gb300 import shard
    from paper_2410_02532_gb300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    prec = opo.OPO_FP32_PH64 if args.precision == "fp32" else opo.OPO_FP64
    base = W.cw_sro_16k()
    if args.workload == "sync_pumped_131072":
        base = W.sync_pumped_64k(delay_fs=5.0).replace(
            n=1 << 17, name="sync_pumped_n131072_3f_L1mm_nz64_eom")
    plain = args.path == "plain"

    def make(i, s=stream):
        c = base.replace(instance=rank * 100000 + i)
        ctx = opo.Context(c, precision=prec, device=local, stream=s.cuda_stream if s else None)
        if plain:
            ctx.set_path(opo.OPO_PATH_PLAIN)
        return ctx

    tuned = None
    if (not args.no_tune and args.cluster == 0 and args.threads == 0 and not plain
            and args.workload == "cw_sro_16k"):
        from paper_2410_02532_gb300 import autotune
        tuned = autotune.tune(base.replace(instance=rank * 100000 + 50000), prec, device=local)
    cl_req = tuned["cluster"] if tuned else args.cluster
    th_req = tuned["threads"] if tuned else args.threads
    probe = make(0)
    if plain and args.batch > 0:
        # sizes without a fused form (FP64 at 2^17) have no fused capacity
        active, cluster = args.batch, args.cluster
    else:
        active, cluster = opo.opo_fused_capacity(probe.h, cl_req, th_req)
    B = args.batch if args.batch > 0 else max(1, active)
    # weak scaling: every rank owns its own block of B instances (seeds differ)
    ctxs = [probe] + [make(i) for i in range(1, B)]
    batch = opo.opo_batch_create([c.h for c in ctxs], cluster, th_req)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            opo.opo_batch_run(batch, 1)
        barrier()
        clocks = ClockSampler(local)
        clocks.start()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()  # evict L2 between timed steps (outside the events)
            evs[k][0].record(stream)
            opo.opo_batch_run(batch, 1)
            evs[k][1].record(stream)
        barrier()
        clk = clocks.stop()
    step_ms = [a.elapsed_time(b_) for a, b_ in evs]
    total_ms = shard.max_over_ranks(sum(step_ms), dist, device="cuda")
    ms_per_step = total_ms / args.steps
    field_steps = base.nfields * base.nz * B * world
    value = field_steps / (ms_per_step * 1e-3)
    for c in ctxs:
        c.sync()

    # DRAM bytes per launch of the fused kernel (dram__bytes_read.sum +
    # dram__bytes_write.sum) from one ncu capture of this workload in this
    # launch shape; reported only when the run uses that shape
    traffic = None
    if ((B, cluster, th_req) in PROFILED_SHAPES and prec == opo.OPO_FP32_PH64 and not plain
            and args.workload == "cw_sro_16k"):
        traffic = PROFILED_SHAPES[(B, cluster, th_req)]
    flops_rt = flops_per_roundtrip(base)
    achieved = flops_rt * B / (statistics.median(step_ms) * 1e-3) / 1e12
    peak = SMS * FP32_LANES * 2 * PEAK_SM_MHZ * 1e6 / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "note": "FP32 vector peak from 152 SMs x 128 lanes x 2 x 2070 MHz; achieved = "
                        "algorithmic FLOPs of the batch round trip / median step time "
                        "(the fused kernel plus one finalize launch)"}
    if plain:
        hbm, src = measured_hbm_gbs()
        gbs = plain_bytes_per_roundtrip(base, 16 if prec == opo.OPO_FP64 else 8) * B / (
            statistics.median(step_ms) * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                    "frac": gbs / hbm, "traffic": None,
                    "note": "batched plain chain; algorithmic bytes / median step time; peak: "
                            "%s copy bandwidth" % src}

    extras = {}
    if not args.skip_extras and rank == 0:
        # one instance alone, at the default cluster and the fastest of a few
        # CTA sizes
        extras = single_and_plain(args, opo, W, base, prec, local, torch)
        extras["e2e"] = e2e(args, opo, W, ctxs, batch, base, torch, np)
        pb = plain_batched_leg(opo, W, prec, local, torch, base, (B, 8 * B))
        extras["plain_batched"] = pb
        if "ms_per_round_trip" in pb.get("B%d" % B, {}):
            extras["fused_over_plain_batched"] = (pb["B%d" % B]["ms_per_round_trip"]
                                                  / statistics.median(step_ms))
        extras["batched_sweep"] = sweep_leg(opo, W, prec, local, torch, rounds=1000)
        extras["workloads"] = config_legs(opo, W, local, torch)
        extras["variants_2e14"] = rows_leg(opo, W, prec, local, torch, base, cluster, th_req)
        extras["serving"] = serving_leg(prec, local, value, base)
        if args.serving_full:
            extras["serving_full_budgets"] = serving_full_leg(
                prec, local, extras["serving"].pop("capacity"), args.serving_full)
        else:
            extras["serving"].pop("capacity", None)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == opo.OPO_FP32_PH64 else "f64",
            "data": "synthetic (seeded noise, random-phase start)",
            "config": {"workload": ("%s x %d instances per GPU (one cluster of %d CTAs each)"
                                    % (base.name, B, cluster)) if not plain else
                                   ("%s x %d instances per GPU, batched plain chain"
                                    % (base.name, B)),
                       "n": base.n, "fields": base.nfields, "nz": base.nz,
                       "instances_per_gpu": B, "cluster": cluster,
                       "threads_per_cta": th_req, "autotuned": tuned,
                       "precision": "fp32 fields + fp64 phase args" if prec else "fp64",
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": "instances sharded per GPU, no collective"},
            "round_trips_per_s": B * world / (ms_per_step * 1e-3),
            "roofline": roofline,
            "clocks": clk,
            "gpu_launches": 2 * args.steps,
        }
        line.update({k: v for k, v in extras.items() if k != "e2e"})
        if "e2e" in extras:
            line["e2e"] = extras["e2e"]
        if world == 1 and not args.skip_extras:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    opo.opo_batch_destroy(batch)
    for c in ctxs:
        c.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def plain_bytes_per_roundtrip(cfg, csz):
    """Algorithmic HBM bytes of one plain-path round trip of one instance:
    per z-step and point-field, RK4 half steps 2 x (read + write), forward and
    inverse FFT 2 x (read + write) for a field transformed whole in one CTA
    (N <= 2^14 in FP32, 2^13 in FP64) or 2 x (column pass + row pass) x
    (read + write) above, dispersion factor read + write + table read: 11 or
    15 csz; per round trip the entry, the power sums, the output copy, the
    cavity visit (FFT pair, factor) and the mirror/EOM pass, about 16 csz per
    point-field."""
    n, F = cfg.n, cfg.nfields
    whole = 256 <= n <= (8192 if csz == 16 else 16384)
    return n * F * csz * ((11 if whole else 15) * total_nz(cfg) + 16)


def measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def plain_batched_leg(opo, W, prec, local, torch, base, counts, steps=6):
    """The plain per-operation chain on batches of the headline workload: every
    launch applies one operation to all instances (one graph per round trip).
    Timed like the headline (one round trip per step, L2 flushed between
    steps, CUDA events on the launch stream, median step).  ``counts``: batch
    sizes; the first equals the fused headline batch, a larger one has a
    working set beyond L2, where the chain is bound by HBM bandwidth."""
    csz = 16 if prec == opo.OPO_FP64 else 8
    peak, peak_src = measured_hbm_gbs()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {}
    for B in counts:
        s = torch.cuda.Stream()
        ctxs = []
        try:
            for i in range(B):
                c = opo.Context(base.replace(instance=900000 + i), precision=prec, device=local,
                                stream=s.cuda_stream)
                c.set_path(opo.OPO_PATH_PLAIN)
                ctxs.append(c)
            b = opo.opo_batch_create([c.h for c in ctxs], 0, 0)
            times = []
            with torch.cuda.stream(s):
                for _ in range(2):
                    opo.opo_batch_run(b, 1)
                for _ in range(steps):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(s)
                    opo.opo_batch_run(b, 1)
                    e1.record(s)
                    e1.synchronize()
                    times.append(e0.elapsed_time(e1))
            opo.opo_batch_destroy(b)
            ms = statistics.median(times)
            gbs = plain_bytes_per_roundtrip(base, csz) * B / (ms * 1e-3) / 1e9
            out["B%d" % B] = {
                "instances": B, "ms_per_round_trip": ms,
                "field_steps_per_s": B * base.nfields * total_nz(base) / (ms * 1e-3),
                "working_set_MB": B * base.n * base.nfields * csz * 3 / 1e6,
                "algorithmic_GB_per_s": gbs, "hbm_peak_GB_per_s": peak,
                "hbm_peak": peak_src, "frac_hbm": gbs / peak}
        except opo.OPOError as e:
            out["B%d" % B] = {"error": str(e)}
        finally:
            for c in ctxs:
                c.close()
    return out


def single_and_plain(args, opo, W, base, prec, local, torch, cl_req=0):
    """One instance alone: fused and plain paths, round trips per second.  The
    library's default CTA size favours batches (two CTAs per SM where the
    shared memory allows); a lone instance runs faster on larger CTAs, so the
    fused path is timed at a few CTA sizes of the default cluster and the
    fastest is reported with its size."""
    out = {}
    s = torch.cuda.Stream()
    legs = [("single_fused", opo.OPO_PATH_FUSED, th) for th in (0, 256, 384, 512)]
    legs.append(("single_plain", opo.OPO_PATH_PLAIN, 0))
    for name, path, th in legs:
        ctx = opo.Context(base, precision=prec, device=local, stream=s.cuda_stream)
        try:
            if path == opo.OPO_PATH_FUSED:
                ctx.set_path(path, cl_req, 0, th)
            else:
                ctx.set_path(path)
        except opo.OPOError:
            ctx.close()
            continue
        steps = max(3, min(args.steps, 10))
        with torch.cuda.stream(s):
            for _ in range(2):
                opo.opo_run_roundtrips(ctx.h, 1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(steps):
                opo.opo_run_roundtrips(ctx.h, 1)
            e1.record(s)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        if name not in out or ms < out[name]["ms_per_round_trip"]:
            out[name] = {"ms_per_round_trip": ms, "round_trips_per_s": 1e3 / ms,
                         "field_steps_per_s": base.nfields * base.nz * 1e3 / ms}
            if path == opo.OPO_PATH_FUSED:
                out[name]["threads_per_cta"] = th if th else "default"
        ctx.close()
    out["fused_over_plain_single"] = (out["single_plain"]["ms_per_round_trip"]
                                      / out["single_fused"]["ms_per_round_trip"])
    return out


def e2e(args, opo, W, ctxs, batch, base, torch, np):
    """Through the C ABI with host buffers: every step copies all instances'
    fields from pinned host memory (one batch copy), runs one round trip and
    reads every instance's output signal field and trace row back to the host
    (one batch copy each).  The reported value uses opo_batch_step_io (the
    copies of a step overlap the neighbouring steps' round trips); the
    synchronous sequence of calls is reported beside it."""
    n, F = base.n, base.nfields
    B = len(ctxs)
    host_in = torch.empty((B, F, n, 2), dtype=torch.float64).pin_memory()
    host_out = torch.empty((B, n, 2), dtype=torch.float64).pin_memory()
    host_tr = torch.empty((B, 1, 4), dtype=torch.float64).pin_memory()
    for i, c in enumerate(ctxs):
        host_in[i].copy_(torch.from_numpy(np.stack([c.get_fields()[x].view(np.float64).reshape(n, 2)
                                                     for x in range(F)])))
    L = opo.lib()
    dp = lambda t: opo.ctypes.cast(t.data_ptr(), opo._DP)  # noqa: E731
    steps = max(3, min(args.steps, 10))

    def one_step():
        assert L.opo_batch_set_fields(batch, dp(host_in), B * F * n) == 0
        opo.opo_batch_run(batch, 1)
        assert L.opo_batch_get_fields(batch, 1, opo.OPO_OUTPUT, dp(host_out), B * n) == 0
        assert L.opo_batch_get_trace(batch, dp(host_tr), 1) == 0

    one_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one_step()
    torch.cuda.synchronize()
    dt_sync = (time.perf_counter() - t0) / steps

    # the same steps through opo_batch_step_io: each step's upload and
    # download run on copy streams beside the neighbouring steps' round trips
    # (two device staging slots; every byte still crosses per step)
    io_out = torch.empty(2 * B * n + 4 * B, dtype=torch.float64).pin_memory()
    pin = host_in.data_ptr()
    opo.opo_batch_step_io(batch, pin, io_out.data_ptr(), 1, 1)
    opo.opo_batch_io_wait(batch)
    steps_io = max(steps, 20)
    t0 = time.perf_counter()
    for _ in range(steps_io):
        opo.opo_batch_step_io(batch, pin, io_out.data_ptr(), 1, 1)
    opo.opo_batch_io_wait(batch)
    dt = (time.perf_counter() - t0) / steps_io
    return {"value": F * base.nz * B / dt, "unit": UNIT,
            "h2d_bytes_per_step": B * F * n * 16,
            "d2h_bytes_per_step": B * (n * 16 + 32),
            "ms_per_step": dt * 1e3,
            "api": "opo_batch_step_io (copies overlapped with the neighbouring steps)",
            "synchronous": {"value": F * base.nz * B / dt_sync, "ms_per_step": dt_sync * 1e3,
                            "api": "opo_batch_set_fields, opo_batch_run, "
                                   "opo_batch_get_fields, opo_batch_get_trace"}}


def rows_leg(opo, W, prec, local, torch, base, cluster, threads, rounds=2):
    """The widened entry and nonlinear-step variants on the 2^14 workload, in
    the headline's launch shape: ns-pulsed pump (the Gaussian slice evaluated
    at every entry), pump-resonant cavity (input added to the circulating
    pump), Kerr terms with fourth-order dispersion, the same steps in two
    crystals, the FP64 path, and the chi(2)-only workload timed the same way
    for comparison.  Batch throughput (best of
    three runs of ``rounds`` round trips, L2 not flushed) and the fraction of
    the FP32 peak by each variant's own FLOP count."""
    variants = {
        "chi2_only_same_leg": base,
        "ns_pulsed_pump": base.replace(pump_kind=W.PUMP_NS, pump_fwhm=10e-9,
                                       pump_t0=30e-9),
        "pump_resonant_tro": base.replace(resonant_mask=0b111, R=(0.9, 0.98, 0.98),
                                          pump_power=0.05 * base.pump_power),
        "kerr_beta4": base.replace(n2=2e-19, beta4=(4e-55, -3e-55, 2e-55)),
        # the same 100 steps in two crystals (the second with another phase
        # mismatch, d_eff and indices)
        "two_crystals": base.replace(length=base.length / 2, nz=base.nz // 2, extra_crystals=(
            W.Crystal(length=base.length / 2, nz=base.nz - base.nz // 2, dk=50.0,
                      deff=0.9 * base.deff, nidx=tuple(1.01 * x for x in base.nidx),
                      dbeta1=base.dbeta1, beta2=base.beta2, beta3=base.beta3),)),
    }
    peak = SMS * FP32_LANES * 2 * PEAK_SM_MHZ * 1e6 / 1e12
    out = {}
    # the FP64 path on the same workload, in its own default launch shape
    # (its fields need twice the shared memory); its fraction is still
    # quoted against the FP32 peak
    # every variant in the headline's launch shape; the Kerr variant also at
    # the shapes its heavier nonlinear step prefers (larger CTAs), reported
    # at the fastest; the FP64 path in its own default shape
    runs = [(name, cfg, prec, [(cluster, threads)]) for name, cfg in variants.items()]
    runs[3] = ("kerr_beta4", variants["kerr_beta4"], prec,
               [(cluster, threads), (4, 512), (8, 256), (4, 384), (8, 384)])
    runs.append(("chi2_only_fp64", base, opo.OPO_FP64, [(0, 0)]))
    for name, cfg, pr, shapes in runs:
        best = None
        for cl_req, th_req in shapes:
            r = time_batch(opo, cfg, pr, local, torch, cl_req, th_req, rounds)
            if "error" in r:
                best = best or r
                continue
            # the fastest shape by throughput (shapes hold different batches)
            if best is None or "error" in best or \
                    r["instances"] / r["seconds"] > best["instances"] / best["seconds"]:
                best = r
        if "error" not in best:
            sec, active = best.pop("seconds"), best["instances"]
            best["field_steps_per_s"] = active * cfg.nfields * total_nz(cfg) * rounds / sec
            best["tflops"] = flops_per_roundtrip(cfg) * active * rounds / sec / 1e12
            best["frac_fp32_peak"] = best["tflops"] / peak
            best["shapes_tried"] = len(shapes)
            if pr == opo.OPO_FP64:
                best["frac_fp64_peak"] = best["tflops"] / FP64_NOMINAL_TFLOPS
                best["fp64_peak_note"] = "nominal GB300 FP64 rate, not measured"
        out[name] = best
    return out


def time_batch(opo, cfg, pr, local, torch, cl_req, th_req, rounds):
    """A GPU-filling fused batch of ``cfg`` in one launch shape: best of three
    runs of ``rounds`` round trips (CUDA events on the launch stream)."""
    s = torch.cuda.Stream()
    probe = opo.Context(cfg, precision=pr, device=local, stream=s.cuda_stream)
    ctxs = [probe]
    try:
        active, cl = opo.opo_fused_capacity(probe.h, cl_req, th_req)
        ctxs += [opo.Context(cfg.replace(instance=i), precision=pr, device=local,
                             stream=s.cuda_stream) for i in range(1, active)]
        b = opo.opo_batch_create([c.h for c in ctxs], cl, th_req)
        sec = 1e30
        with torch.cuda.stream(s):
            opo.opo_batch_run(b, 1)
            for _ in range(3):  # best of three
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s)
                opo.opo_batch_run(b, rounds)
                e1.record(s)
                e1.synchronize()
                sec = min(sec, e0.elapsed_time(e1) * 1e-3)
        opo.opo_batch_destroy(b)
        return {"instances": active, "cluster": cl, "threads_per_cta": th_req or "default",
                "seconds": sec}
    except opo.OPOError as e:
        return {"error": str(e)}
    finally:
        for c in ctxs:
            c.close()


def config_legs(opo, W, local, torch):
    """The other workloads as whole runs.  The 1024-point FP64 parity
    workload (3 fields, 50 steps, 10 round trips): one instance on the plain
    and on the fused path, and a GPU-filling fused batch.  The synchronously
    pumped 2^16-point workload (sech^2 pump, EOM, FP32 fields with FP64
    phases): the five timing mismatches -20..+20 fs plus two more (a full
    wave of 16-CTA clusters), each for the whole 2000 round trips in one
    batch; throughput and each mismatch's mean output signal power over the
    last 200 round trips."""
    out = {}
    cfg1 = W.cw_sro_1024()
    leg = {}
    s = torch.cuda.Stream()
    for name, path in (("plain", opo.OPO_PATH_PLAIN), ("fused", opo.OPO_PATH_FUSED)):
        with opo.Context(cfg1, precision=opo.OPO_FP64, device=local, stream=s.cuda_stream) as ctx:
            ctx.set_path(path)
            with torch.cuda.stream(s):
                ctx.run(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                opo.opo_run_roundtrips(ctx.h, cfg1.M)
                e1.record(s)
                e1.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            leg["single_" + name] = {"round_trips": cfg1.M, "seconds": sec,
                                     "round_trips_per_s": cfg1.M / sec,
                                     "field_steps_per_s": cfg1.M * cfg1.nfields * cfg1.nz / sec}
    r = time_batch(opo, cfg1, opo.OPO_FP64, local, torch, 0, 0, cfg1.M)
    if "error" not in r:
        sec = r.pop("seconds")
        r["field_steps_per_s"] = r["instances"] * cfg1.nfields * cfg1.nz * cfg1.M / sec
        r["round_trips_per_s"] = r["instances"] * cfg1.M / sec
    leg["batch_fused"] = r
    out["cw_sro_n1024_fp64"] = leg
    delays = (-20.0, -10.0, 0.0, 10.0, 20.0, -15.0, 15.0)
    cfgs = [W.sync_pumped_64k(delay_fs=d).replace(instance=i) for i, d in enumerate(delays)]
    M = cfgs[0].M
    ctxs = [opo.Context(c, device=local, stream=s.cuda_stream) for c in cfgs]
    try:
        b = opo.opo_batch_create([c.h for c in ctxs], 0, 0)
        with torch.cuda.stream(s):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            opo.opo_batch_run(b, M)
            e1.record(s)
            e1.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
        tr = opo.opo_batch_get_trace(b, len(ctxs), M)
        opo.opo_batch_destroy(b)
        c0 = cfgs[0]
        out["sync_pumped_n65536"] = {
            "instances": len(cfgs), "round_trips": M, "seconds": sec,
            "round_trips_per_s": len(cfgs) * M / sec,
            "field_steps_per_s": len(cfgs) * M * c0.nfields * c0.nz / sec,
            "point_field_steps_per_s": len(cfgs) * M * c0.nfields * c0.nz * c0.n / sec,
            "signal_out_W_by_delay_fs": {("%+.0f" % d): float(tr[i, -200:, 1].mean())
                                         for i, d in enumerate(delays)}}
    except opo.OPOError as e:
        out["sync_pumped_n65536"] = {"error": str(e)}
    finally:
        for c in ctxs:
            c.close()
    return out


def sweep_leg(opo, W, prec, local, torch, rounds=2):
    """The batched sweep: 256 seeded instances (N 2^12..2^15, SRO/DRO/degenerate,
    1-5x threshold, +-50 fs, 5-30 mm), advanced together; point-field-steps/s."""
    cfgs = W.sweep_instances(256)
    s = torch.cuda.Stream()
    ctxs = [opo.Context(c, precision=prec, device=local, stream=s.cuda_stream) for c in cfgs]
    try:
        b = opo.opo_batch_create([c.h for c in ctxs], 0, 0)
        with torch.cuda.stream(s):
            opo.opo_batch_run(b, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            opo.opo_batch_run(b, rounds)
            e1.record(s)
            e1.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
        pfs = sum(c.n * c.nfields * c.nz for c in cfgs) * rounds
        fs = sum(c.nfields * c.nz for c in cfgs) * rounds
        out = {"instances": len(cfgs), "round_trips": rounds, "seconds": sec,
               "point_field_steps_per_s": pfs / sec, "field_steps_per_s": fs / sec,
               "round_trips_per_s": len(cfgs) * rounds / sec,
               "launches": "one persistent launch per size class, classes concurrent"}
        # the same sweep as one persistent launch of the generic fused kernel
        # (one cluster and CTA size, that of the largest member), over fewer
        # round trips
        r1 = 20
        try:
            opo.opo_batch_set_one_launch(b, True)
            with torch.cuda.stream(s):
                opo.opo_batch_run(b, 1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                opo.opo_batch_run(b, r1)
                e1.record(s)
                e1.synchronize()
            sec1 = e0.elapsed_time(e1) * 1e-3
            out["one_launch"] = {"round_trips": r1, "seconds": sec1,
                                 "point_field_steps_per_s": pfs / rounds * r1 / sec1,
                                 "round_trips_per_s": len(cfgs) * r1 / sec1}
        except opo.OPOError as e:
            out["one_launch"] = {"error": str(e)}
        opo.opo_batch_destroy(b)
        return out
    finally:
        for c in ctxs:
            c.close()


def serving_leg(prec, local, batch_value, base, count=1000):
    """Request stream through the continuous-batching server: N = 2^12..2^17
    (2^12..2^16 on the fused path, 2^17 on the plain path), 2 or 3 fields, CW
    or pulsed.  First a saturation run (all requests present at t = 0)
    measures the server's capacity on this mix; then ``count`` Poisson
    arrivals at 0.7 of that capacity give p50/p99 latency.  Round-trip
    budgets are 20..120 so that the run takes seconds."""
    from paper_2410_02532_gb300 import serving
    exps = (12, 13, 14, 15, 16, 17)
    rounds = (20, 120)
    sat = serving.poisson_trace(160, 1e6, seed=20241009, n_exps=exps, rounds=rounds)
    srv = serving.Server(precision=prec, device=local, tick_rt=16)
    t0 = time.perf_counter()
    res = srv.run(sat)
    sat_wall = time.perf_counter() - t0
    cap = sum(serving.request_work(r) for r in sat) / sat_wall   # point-field-steps/s
    probe = serving.poisson_trace(400, 1.0, n_exps=exps, rounds=rounds)
    mean_work = sum(serving.request_work(r) for r in probe) / len(probe)
    rate = 0.7 * cap / mean_work
    reqs = serving.poisson_trace(count, rate, n_exps=exps, rounds=rounds)
    srv = serving.Server(precision=prec, device=local, tick_rt=16)
    t0 = time.perf_counter()
    res = srv.run(reqs, max_wall_s=4 * count / rate)
    wall = time.perf_counter() - t0
    st = serving.latency_stats(res)
    done = {x.rid for x in res}
    work = sum(serving.request_work(r) for r in reqs if r.rid in done)
    # the stream of the full request mix (200 arrivals/s, 100..5000 round trips)
    full = serving.poisson_trace(400, 1.0, n_exps=exps, rounds=(100, 5000))
    full_load = 200.0 * sum(serving.request_work(r) for r in full) / len(full) / cap
    st.update({"requests": count, "completed": len(res), "rate_hz": rate,
               "offered_load": 0.7, "capacity_point_field_steps_per_s": cap,
               "rounds_range": list(rounds), "n_range": [1 << exps[0], 1 << exps[-1]],
               "wall_s": wall, "point_field_steps_per_s": work / wall,
               "field_steps_per_s": srv.field_steps / wall, "ticks": srv.ticks,
               "allocations": srv.allocations,
               "note": "rate = 0.7 x the server's saturated throughput on the same request mix; "
                       "200 requests/s with 100-5000 round trips would offer about %.0fx that "
                       "capacity" % full_load})
    # the same trace with every request on the batched plain path (same
    # admission shares): the plain chain's latency on the same stream
    srv = serving.Server(precision=prec, device=local, tick_rt=16, path="plain")
    t0 = time.perf_counter()
    res_p = srv.run(reqs, max_wall_s=3 * wall)
    wall_p = time.perf_counter() - t0
    stp = serving.latency_stats(res_p)
    done_p = {x.rid for x in res_p}
    stp.update({"completed": len(res_p), "wall_s": wall_p,
                "point_field_steps_per_s": sum(serving.request_work(r) for r in reqs
                                               if r.rid in done_p) / wall_p,
                "note": "same requests and arrival times on the batched plain path; requests "
                        "not finished within 3x the fused run's wall time are left out"})
    st["plain_path"] = stp
    if stp.get("p99_s") and len(res_p) == len(res):
        st["p99_plain_over_fused"] = stp["p99_s"] / st["p99_s"]
    st["capacity"] = cap
    return st


def serving_full_leg(prec, local, cap, count, window_s=90.0):
    """Config-5 request stream at its stated budgets (N = 2^12..2^17, 100..5000
    round trips, 2 or 3 fields, CW or pulsed).  (1) The first 2000 arrivals at
    200 requests/s, served for ``window_s`` seconds: the offered load is
    hundreds of times the capacity, so the report is how many finished and
    their latencies, with the rest still queued.  (2) ``count`` arrivals at
    0.7 of the capacity measured on the short-budget mix: p50/p99."""
    from paper_2410_02532_gb300 import serving
    exps = (12, 13, 14, 15, 16, 17)
    rounds = (100, 5000)
    out = {}
    reqs = serving.poisson_trace(2000, 200.0, seed=20241011, n_exps=exps, rounds=rounds)
    mean_work = sum(serving.request_work(r) for r in reqs) / len(reqs)
    srv = serving.Server(precision=prec, device=local, tick_rt=32)
    t0 = time.perf_counter()
    res = srv.run(reqs, max_wall_s=window_s)
    wall = time.perf_counter() - t0
    st = serving.latency_stats(res)
    st.update({"arrivals": len(reqs), "rate_hz": 200.0, "completed": len(res),
               "window_s": wall, "offered_over_capacity": 200.0 * mean_work / cap,
               "field_steps_per_s": srv.field_steps / wall,
               "note": "latencies of the requests finished inside the window only"})
    out["rate_200_per_s"] = st
    rate = 0.7 * cap / mean_work
    reqs = serving.poisson_trace(count, rate, seed=20241012, n_exps=exps, rounds=rounds)
    srv = serving.Server(precision=prec, device=local, tick_rt=32)
    t0 = time.perf_counter()
    res = srv.run(reqs, max_wall_s=6 * count / rate)
    wall = time.perf_counter() - t0
    st = serving.latency_stats(res)
    st.update({"requests": count, "completed": len(res), "rate_hz": rate, "offered_load": 0.7,
               "wall_s": wall, "field_steps_per_s": srv.field_steps / wall})
    out["rate_0p7_capacity"] = st
    return out


if __name__ == "__main__":
    sys.exit(main())
