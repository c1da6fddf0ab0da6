#!/usr/bin/env python3
"""Throughput of the progressive material cache on one GB300 (shading points / s).

Workload (one "step"): one progressive frame of 1920x1080 pixels x 16 samples, run as
16 passes (pmc_eval_batch calls) of 2,073,600 shading points each against a table of
2^24 slots (2^21 cells x 8 entries, 16 B each) that starts empty; 64 generated
material networks of 20-200 nodes (20 % shading-point dependent), materials per 8x8
tile from a Zipf(1.1) law, UV affine per tile with per-sample jitter.  Inputs (1.2 GB
of points) are resident in HBM and larger than L2; the table is 256 MB.

The JSON line reports the cached throughput (value), the same frame with the cache
off (uncached), the cached throughput through the host-buffer entry point with the
copies inside the timed region (e2e), the roofline of the dominant kernel from
CUDA events on the library's stream, and the CPU oracle on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2305_07238_gb300 import workload as W  # noqa: E402

METRIC = "shading points/sec (progressive material cache, cached)"
UNIT = "points/s"
WIDTH, HEIGHT, SPP = 1920, 1080, 16
N_MATS, NODES_LO, NODES_HI, SP_FRAC = 64, 20, 200, 0.2
N_CELLS, N_ENTRIES, LEVEL = 1 << 21, 8, 10
SAMPLE_ROWS = (0, 40)            # CPU-oracle sample: 40 full-width rows, all 16 passes
REF_ROWS = (0, 16)               # reference arm: 16 full-width rows per step, all 16 passes
# The cost threshold of the headline frame (FP32 operations per cacheable sub-graph): the
# break-even value the rule below gives on this frame with the per-cell-list insert
# (about 490, rounded to a multiple of 50). It is fixed, so that the reference arm and
# every leg run the same configuration; the line reports the live estimate beside it.
MIN_ROOT_COST = 500
REF_MIN_ROOT_COST = MIN_ROOT_COST   # reference arm: the same threshold
# DRAM bytes (read + written) per launch of each kernel, the mean of the two launches one
# ncu capture of that kernel takes from a four-pass frame of this workload at the bench's
# cost threshold; None while the kernel has changed since its capture
NCU_TRAFFIC = {"eval": 159.1e6, "eval_roots": 94.0e6, "lookup": 366.8e6}

FP32_LANES_PER_SM = 128          # Blackwell SM: 4 partitions x 32 FP32 lanes


def n_sms(torch, dev):
    """Streaming multiprocessors of the device, as the CUDA driver reports them."""
    return int(torch.cuda.get_device_properties(torch.device(dev)).multi_processor_count)


def workload(seed=0):
    mats = W.random_materials(N_MATS, NODES_LO, NODES_HI, SP_FRAC, seed=seed)
    frame = W.Frame(W.FrameSpec(width=WIDTH, height=HEIGHT, n_mats=N_MATS, seed=seed))
    return mats, frame


def config_dict(extra=None):
    d = {"workload": f"frame {WIDTH}x{HEIGHT}x{SPP}spp, 16 passes of {WIDTH * HEIGHT} points, "
                     f"{N_MATS} materials {NODES_LO}-{NODES_HI} nodes ({int(SP_FRAC * 100)}% SP), "
                     f"table {N_CELLS}x{N_ENTRIES} slots (256 MB), Zipf 1.1, lambda {LEVEL}",
         "points_per_step": WIDTH * HEIGHT * SPP, "batch": WIDTH * HEIGHT, "passes_per_step": SPP,
         "n_cells": N_CELLS, "n_entries": N_ENTRIES, "uv_level": LEVEL,
         "l2": "inputs larger than L2 (1.2 GB points + 256 MB table per step)"}
    if extra:
        d.update(extra)
    return d


# --------------------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


def max_over_ranks(torch, dist, secs, device):
    """The slowest rank's time (every rank gets it); `secs` itself on one process."""
    if dist is None:
        return secs
    t = torch.tensor([secs], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, secs_max):
    """Units of all replicas per second: every rank processes units_per_rank in the time
    of the slowest one."""
    return units_per_rank * world / secs_max


def run_frame(cache, dev_passes, outs, hits, stream):
    cache.reset(stream)
    for p in range(SPP):
        cache.eval_batch(dev_passes[p], outs, hits, stream)


def timed_steps(torch, cache, dev_passes, outs, hits, steps, dist_barrier):
    stream = torch.cuda.current_stream()
    dist_barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        run_frame(cache, dev_passes, outs, hits, stream)
    t1.record(stream)
    torch.cuda.synchronize()
    dist_barrier()
    return t0.elapsed_time(t1) / 1000.0


def timed_graph(torch, graph, steps, dist_barrier):
    stream = torch.cuda.current_stream()
    dist_barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        graph.launch(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    dist_barrier()
    return t0.elapsed_time(t1) / 1000.0


def ours(args, rank, world, local_rank, dist):
    import torch
    from paper_2305_07238_gb300 import build as B
    from paper_2305_07238_gb300 import pmc as P

    B.build()
    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    barrier = (lambda: dist.barrier()) if dist is not None else (lambda: None)

    mats, frame = workload(seed=rank)
    passes_host = [frame.points(p) for p in range(SPP)]
    dev_passes = [P.points_to_device(h, dev) for h in passes_host]
    n = WIDTH * HEIGHT
    outs = torch.empty((3, n), dtype=torch.float32, device=dev)
    hits = torch.empty(n, dtype=torch.int16, device=dev)

    uncached = None
    if "uncached" in args.legs.split(","):
        uncached = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, flags=P.PMC_CACHE_OFF, device=local_rank)
    pts_total = n * SPP * args.steps

    def measure(cache):
        """Warm-up frames, the schedule autotuned on a warm table, timed eager frames with
        per-phase events (the per-kernel times of the roofline), then the whole frame (reset +
        16 passes) as one CUDA graph."""
        for _ in range(args.warmup):
            run_frame(cache, dev_passes, outs, hits, None)
        cache.reset()
        for p in range(2):
            cache.eval_batch(dev_passes[p], outs, hits)
        tune = cache.autotune(dev_passes[2], reps=3)
        cache.sync()
        cache.read_timing()
        cache.set_timing(True)
        secs_eager = timed_steps(torch, cache, dev_passes, outs, hits, args.steps, barrier)
        cache.set_timing(False)
        timing = cache.read_timing()
        frame_stats = cache.stats()   # reset() zeroes the counters per frame: one frame's worth
        cache.reset()
        cache.eval_batch(dev_passes[0], outs, hits)
        pass0_stats = cache.stats()   # the empty-table pass: no lookup launch
        graph = cache.graph(dev_passes, [outs] * SPP, [hits] * SPP, reset=True)
        for _ in range(max(1, args.warmup)):
            graph.launch()
        cache.sync()
        cache.read_timing()
        secs = timed_graph(torch, graph, args.steps, barrier)
        g_launches = cache.read_timing()["launches"]
        graph.close()
        # passes 2..15 of a frame on the warm table, eager, CUDA events on the library's stream
        stream = torch.cuda.current_stream()
        cache.reset(stream)
        for p in range(2):
            cache.eval_batch(dev_passes[p], outs, hits, stream)
        cache.sync()
        st0 = cache.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for p in range(2, SPP):
            cache.eval_batch(dev_passes[p], outs, hits, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        st1 = cache.stats()
        warm = {"points_per_s": round(n * (SPP - 2) / (e0.elapsed_time(e1) / 1e3), 1),
                "hit_rate": round((st1["hits"] - st0["hits"]) / max(1, st1["lookups"] - st0["lookups"]), 4),
                "passes": f"2-{SPP - 1}", "launch": "eager"}
        # hit rate of every pass of one frame (untimed: the counters are read after each pass)
        cache.reset(stream)
        per_pass, prev = [], cache.stats()
        for p in range(SPP):
            cache.eval_batch(dev_passes[p], outs, hits, stream)
            cur = cache.stats()
            per_pass.append(round((cur["hits"] - prev["hits"]) / max(1, cur["lookups"] - prev["lookups"]), 4))
            prev = cur
        warm["hit_rate_per_pass"] = per_pass
        return dict(tune=tune, secs_eager=secs_eager, timing=timing, frame_stats=frame_stats,
                    pass0_stats=pass0_stats, secs=max_over_ranks(torch, dist, secs, dev), g_launches=g_launches,
                    warm=warm)

    with ClockSampler(local_rank) as clk:
        # the evaluation's cost per FP32 operation with the cache off (every node evaluated,
        # one eager frame with per-phase events)
        plain = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, flags=P.PMC_CACHE_OFF, device=local_rank)
        run_frame(plain, dev_passes, outs, hits, None)
        plain.sync()
        plain.read_timing()
        plain.set_timing(True)
        plain.reset()
        run_frame(plain, dev_passes, outs, hits, None)
        plain_ms = plain.read_timing()["ms"]
        t_flop = plain_ms["eval"] / max(1, plain.stats()["flops"])
        plain.close()
        # the rule of Sec. 3: every maximal UV-only node is cached
        m_all = measure(P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, device=local_rank))
        # break-even cost of a cacheable node: a probe (its lookup and insert, from the
        # all-roots run's phase times) against the evaluation a hit saves at the measured hit
        # rate
        ms_all, st_all = m_all["timing"]["ms"], m_all["frame_stats"]
        t_probe = (ms_all["lookup"] + ms_all["insert"]) / args.steps / max(1, st_all["lookups"])
        hit = st_all["hits"] / max(1, st_all["lookups"])
        break_even = t_probe / max(1e-30, hit * t_flop)
        min_root_cost = MIN_ROOT_COST
        cached = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, min_root_cost=min_root_cost, device=local_rank)
        m = measure(cached)
    tune, secs_eager, timing = m["tune"], m["secs_eager"], m["timing"]
    frame_stats, pass0_stats, g_launches = m["frame_stats"], m["pass0_stats"], m["g_launches"]
    secs_max = m["secs"]
    value = whole_job_rate(pts_total, world, secs_max)

    # ---- uncached --------------------------------------------------------------------
    legs = set(args.legs.split(","))
    usecs, u_value, u_warm = float("nan"), float("nan"), float("nan")
    if "uncached" in legs:
        uncached.autotune(dev_passes[2], reps=3)
        ugraph = uncached.graph(dev_passes, [outs] * SPP, [hits] * SPP, reset=True)
        for _ in range(max(1, args.warmup)):
            ugraph.launch()
        uncached.sync()
        usecs = timed_graph(torch, ugraph, args.steps, barrier)
        ugraph.close()
        # the same passes 2..15 as the cached warm-pass figure, eager
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for p in range(2, SPP):
            uncached.eval_batch(dev_passes[p], outs, hits, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        u_warm = n * (SPP - 2) / (e0.elapsed_time(e1) / 1e3)
        usecs = max_over_ranks(torch, dist, usecs, dev)
        u_value = whole_job_rate(pts_total, world, usecs)

    # ---- end to end through the host-buffer entry point --------------------------------
    e2e = None
    if "e2e" in legs:
        e2e = e2e_run(torch, P, mats, passes_host, args, local_rank, barrier, dist, dev, min_root_cost)

    # ---- roofline of the dominant kernel ------------------------------------------------
    hbm_peak, sm_mhz_max, peak_kind = peaks()
    ms = timing["ms"]
    per_launch_ms = {k: v / max(1, timing["batches"]) for k, v in ms.items()}
    # the first pass of a frame runs on an empty table: no lookup launch
    per_launch_ms["lookup"] = ms["lookup"] / max(1, timing["batches"] - args.steps)
    fp32_peak = n_sms(torch, dev) * FP32_LANES_PER_SM * 2 * sm_mhz_max * 1e6 / 1e12   # TFLOP/s
    # FP32 work of the per-point programs (k_eval) and of the batched misses (k_eval_roots)
    flops_missed = frame_stats["flops_missed"]
    flops_eval = frame_stats["flops"] - flops_missed
    eval_tflops = flops_eval * args.steps / (ms["eval"] / 1e3) / 1e12 if ms["eval"] else 0.0
    missed_tflops = flops_missed * args.steps / (ms["missed"] / 1e3) / 1e12 if ms["missed"] else 0.0
    # algorithmic bytes of the lookup kernel, which runs on passes 1..15 (the empty-table
    # first pass forms its descriptors in the evaluator): per point 12 B (u, v, material),
    # per probe 16 B for every slot examined up to the hit or the first empty slot (all N_e
    # of a full cell) plus a 16-B hit/value write -- the method's per-unit figure, for
    # 16-byte slots {hash2, r, g, b}.  This layout moves less per probe: 4 B per hash2 word
    # examined and 12 B per hit value (the "layout" figure below).
    pts_looked = n * (SPP - 1)
    look_probes = frame_stats["lookups"] - pass0_stats["lookups"]
    look_slots = frame_stats["slots_probed"] - pass0_stats["slots_probed"]
    look_hits = frame_stats["hits"] - pass0_stats["hits"]
    look_bytes_frame = 12 * pts_looked + 16 * look_slots + 16 * look_probes
    layout_bytes_frame = 8 * pts_looked + 4 * look_slots + 12 * look_hits + 16 * look_probes
    look_gbs = look_bytes_frame * args.steps / (ms["lookup"] / 1e3) / 1e9 if ms["lookup"] else 0.0
    layout_gbs = layout_bytes_frame * args.steps / (ms["lookup"] / 1e3) / 1e9 if ms["lookup"] else 0.0
    kernels = {
        "eval": {"bound": "alu", "achieved": round(eval_tflops, 3), "peak": round(fp32_peak, 2),
                 "unit": "TFLOP/s", "frac": round(eval_tflops / fp32_peak, 4),
                 "ms_per_launch": round(per_launch_ms["eval"], 4), "traffic": NCU_TRAFFIC["eval"]},
        "eval_roots": {"bound": "alu", "achieved": round(missed_tflops, 3), "peak": round(fp32_peak, 2),
                       "unit": "TFLOP/s", "frac": round(missed_tflops / fp32_peak, 4),
                       "ms_per_pass": round(per_launch_ms["missed"], 4), "traffic": NCU_TRAFFIC["eval_roots"]},
        "lookup": {"bound": "hbm", "achieved": round(look_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                   "frac": round(look_gbs / hbm_peak, 4), "ms_per_launch": round(per_launch_ms["lookup"], 4),
                   "traffic": NCU_TRAFFIC["lookup"],
                   "bytes_per_launch": round(look_bytes_frame / (SPP - 1)),
                   "slots_examined_per_probe": round(look_slots / max(1, look_probes), 3),
                   "achieved_layout_bytes": round(layout_gbs, 1),
                   "frac_layout_bytes": round(layout_gbs / hbm_peak, 4)},
    }
    # algorithmic bytes of the insert per frame: 24 B per candidate offered (its key, cell and
    # value) and 16 B per slot filled.  No ncu traffic figure: the captures of its resolve
    # cover the first two passes of a frame only, not a frame's mean launch.
    ins_bytes_frame = 24 * frame_stats["candidates"] + 16 * frame_stats["inserted"]
    ins_gbs = ins_bytes_frame * args.steps / (ms["insert"] / 1e3) / 1e9 if ms["insert"] else 0.0
    kernels["insert"] = {"bound": "hbm", "achieved": round(ins_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(ins_gbs / hbm_peak, 4), "ms_per_pass": round(per_launch_ms["insert"], 4),
                         "traffic": None, "bytes_per_pass": round(ins_bytes_frame / SPP)}
    phase_of = {"eval": "eval", "eval_roots": "missed", "lookup": "lookup"}
    dominant = max(phase_of, key=lambda k: ms[phase_of[k]])
    roof = dict(kernels[dominant])
    # the evaluators of the tuned schedule: two points per lane unless it is PMC_ONE_POINT
    one_point = bool(tune["schedule"]["flags"] & P.PMC_ONE_POINT)
    binned = bool(tune["schedule"]["flags"] & P.PMC_INSERT_BINNED)
    names = {"eval": "k_eval" if one_point else "k_eval2", "eval_roots": "k_eval_roots" if one_point else "k_eval_roots2",
             "lookup": "k_lookup",
             "insert": "k_bin_count .. k_bin_insert (binned)" if binned else "k_chain_link + k_chain_resolve"}
    for k in kernels:
        kernels[k]["kernel"] = names[k]
    roof["kernel"] = names[dominant]
    roof["peak_kind"] = "FP32 lanes x 2 x max SM clock" if dominant != "lookup" else peak_kind + " HBM copy"

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(secs_max / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict({"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                               "min_root_cost": min_root_cost}),
        "min_root_cost": {"value": min_root_cost, "rule": "break-even: (lookup + insert ms per probe, all-roots run) / "
                                                          "(hit rate x evaluation ms per FP32 op, cache off)",
                          "break_even_estimate": round(break_even, 1),
                          "probe_ns": round(t_probe * 1e6, 4), "flop_ns": round(t_flop * 1e6, 7),
                          "hit_rate": round(hit, 4)},
        "cached_all_roots": {"value": round(whole_job_rate(pts_total, world, m_all["secs"]), 1), "unit": UNIT,
                             "ms_per_step": round(m_all["secs"] / args.steps * 1e3, 3),
                             "hit_rate": round(hit, 4),
                             "lookups_per_point": round(st_all["lookups"] / (n * SPP), 3),
                             "phase_ms_per_step": {k: round(v / args.steps, 3) for k, v in ms_all.items()}},
        "uncached": {"value": round(u_value, 1), "unit": UNIT,
                     "ms_per_step": round(usecs / args.steps * 1e3, 3),
                     "speedup_cached_over_uncached": round(value / u_value, 3),
                     "speedup_all_roots_over_uncached": round(whole_job_rate(pts_total, world, m_all["secs"]) / u_value, 3)}
        if u_value == u_value else None,
        "hit_rate": round(frame_stats["hits"] / max(1, frame_stats["lookups"]), 4),
        "table": {k: frame_stats[k] for k in ("lookups", "hits", "inserted", "dropped_dup", "dropped_full")},
        "phase_ms_per_step": {k: round(v / args.steps, 3) for k, v in ms.items()},
        "roofline": roof,
        "kernels": kernels,
        "e2e": e2e,
        "gpu_launches": int(g_launches),
        "clocks": clk.summary(),
        "launch": "one CUDA graph per frame (reset + 16 passes); schedule from pmc_autotune",
        "schedule": tune["schedule"],
        "autotune_ms": {f"{t['flags']:#x}/rb{t['lookup_rb']}": round(t["ms"], 3) for t in tune["tried"]},
        "eager": {"value": round(pts_total * world / secs_eager, 1), "unit": UNIT,
                  "ms_per_step": round(secs_eager / args.steps * 1e3, 3),
                  "gpu_launches": int(timing["launches"])},
        # passes 2..15 on the warm table (the first two passes fill it), cached and uncached
        # both eager
        "warm_passes": dict(m["warm"], uncached_points_per_s=round(u_warm, 1) if u_warm == u_warm else None,
                            speedup_over_uncached=round(m["warm"]["points_per_s"] / u_warm, 3)
                            if u_warm == u_warm else None),
    }
    def guarded(name, fn):
        # an optional leg that raises reports its error instead of losing the whole line
        try:
            line[name] = fn()
        except Exception as exc:   # noqa: BLE001
            line[name] = {"error": f"{type(exc).__name__}: {exc}"}

    if "surr" in legs:
        guarded("surrogate", lambda: surrogate_leg(torch, P, dev, local_rank, seed=rank))
    if "f128" in legs:
        guarded("frame128", lambda: frame128_leg(torch, P, dev, local_rank, seed=rank, min_root_cost=min_root_cost))
    if "alg1" in legs:
        guarded("alg1", lambda: alg1_leg(torch, P, mats, dev_passes, outs, hits, local_rank))
        if u_value == u_value and "cached" in line["alg1"]:
            line["alg1"]["speedup_cached_over_uncached"] = round(line["alg1"]["cached"] / u_value, 3)
    if "cones" in legs:
        guarded("ray_cones", lambda: cones_leg(torch, P, dev, local_rank, seed=rank, min_root_cost=min_root_cost))
        if u_value == u_value and "offset0" in line["ray_cones"]:
            for key in [k for k in ("offset0", "offset-1", "offset0_threshold", "offset-1_threshold")
                        if k in line["ray_cones"]]:
                r = line["ray_cones"][key]
                r["speedup_cached_over_uncached"] = round(r["cached"] / u_value, 3)
    if "raycast" in legs:
        guarded("ray_caster", lambda: raycast_leg(torch, P, mats, dev, local_rank, seed=rank,
                                                  min_root_cost=min_root_cost))
    if "position" in legs:
        guarded("position_descriptor", lambda: position_leg(torch, P, mats, dev_passes, outs, hits, local_rank))
    if "replace" in legs:
        guarded("replacement", lambda: replace_leg(torch, P, dev, local_rank, seed=rank))
    if "sweep" in legs:
        guarded("scale_sweep", lambda: sweep_leg(torch, P, dev, local_rank, seed=rank))
    if "scale" in legs:
        guarded("scale", lambda: sweep_leg(torch, P, dev, local_rank, seed=rank, full=False,
                                           min_root_cost=min_root_cost))
    if "threshold" in legs:
        guarded("cost_threshold", lambda: threshold_leg(torch, P, mats, dev_passes, outs, hits, local_rank))
        if u_value == u_value and "runs" in line["cost_threshold"]:
            for r in line["cost_threshold"]["runs"]:
                r["speedup_over_uncached"] = round(r["points_per_s"] / u_value, 3)
    if rank == 0 and not args.no_cpu_baseline and "cpu" in legs:
        line["cpu_baseline"], line["max_abs_err_vs_fp64"] = cpu_baseline(P, torch, mats, frame, dev, min_root_cost)
    return line


F128_MATS, F128_LO, F128_HI, F128_PASSES, F128_CELLS = 1024, 5, 2000, 128, 1 << 23


def frame128_leg(torch, P, dev, local_rank, seed=0, min_root_cost=0):
    """1024 networks of 5-2000 nodes (20 % SP); one 1920x1080 frame rendered as 128 passes
    of one sample per pixel against a 1 GB table (2^23 cells x 8), cacheable nodes above the
    cost threshold `min_root_cost`.  Frame throughput with
    stream launches and as one CUDA graph; grouped by material vs unsorted; the autotuned
    schedule; the uncached frame.  Points come from the torch form of the frame generator
    (9.6 GB resident)."""
    from paper_2305_07238_gb300 import pmc as Pm
    mats = W.random_materials(F128_MATS, F128_LO, F128_HI, SP_FRAC, seed=seed + 300)
    frame = W.Frame(W.FrameSpec(width=WIDTH, height=HEIGHT, n_mats=F128_MATS, seed=seed + 300))
    passes = [frame.points_torch(p, dev) for p in range(F128_PASSES)]
    n = WIDTH * HEIGHT
    # materials are fixed per tile, so every pass needs the same number of probe records
    roots = np.array([len(P.analyze_material(m, min_root_cost=min_root_cost)["roots"]) for m in mats])
    need = max(1, int(roots[frame.tile_mat[frame.pix_tile]].sum()))
    outs = torch.empty((3, n), dtype=torch.float32, device=dev)
    hits = torch.empty(n, dtype=torch.int16, device=dev)
    pts_frame = n * F128_PASSES
    res = {"config": f"frame {WIDTH}x{HEIGHT}, {F128_PASSES} passes of 1 spp ({pts_frame} points), "
                     f"{F128_MATS} materials {F128_LO}-{F128_HI} nodes ({int(SP_FRAC * 100)}% SP), Zipf 1.1, "
                     f"table {F128_CELLS}x{N_ENTRIES} slots (1 GB), lambda {LEVEL}",
           "unit": UNIT, "probes_per_pass": need, "min_root_cost": min_root_cost}

    def make(flags=0):
        return P.Cache(mats, F128_CELLS, N_ENTRIES, uv_level=LEVEL, flags=flags, device=local_rank,
                       probe_capacity=need, min_root_cost=min_root_cost)

    def graph_rate(c, reps=2):
        g = c.graph(passes, [outs] * F128_PASSES, [hits] * F128_PASSES, reset=True)
        g.launch()
        c.sync()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(reps):
            g.launch()
        t1.record()
        torch.cuda.synchronize()
        c.sync()
        g.close()
        return pts_frame * reps / (t0.elapsed_time(t1) / 1e3)

    c = make()
    # stream launches, one event pair per pass: all passes and warm passes (>= 2)
    for rep in range(2):
        c.reset()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(F128_PASSES + 1)]
        ev[0].record()
        for p in range(F128_PASSES):
            c.eval_batch(passes[p], outs, hits)
            ev[p + 1].record()
        torch.cuda.synchronize()
    per_pass = [ev[p].elapsed_time(ev[p + 1]) for p in range(F128_PASSES)]
    st = c.stats()
    res["eager"] = round(pts_frame / (sum(per_pass) / 1e3), 1)
    res["eager_warm_passes"] = round(n * (F128_PASSES - 2) / (sum(per_pass[2:]) / 1e3), 1)
    res["hit_rate"] = round(st["hits"] / max(1, st["lookups"]), 4)
    res["graph_grouped"] = round(graph_rate(c), 1)
    # the per-point evaluator's work distribution: warp pairs of items (above), block-wide
    # tiles of one material, one point per lane
    c.set_schedule(Pm.PMC_BLOCK_ITEMS, 4)
    res["graph_block_per_material"] = round(graph_rate(c), 1)
    c.set_schedule(Pm.PMC_ONE_POINT, 4)
    res["graph_one_point_per_lane"] = round(graph_rate(c), 1)
    c.set_schedule(Pm.PMC_UNSORTED | Pm.PMC_EVAL_INLINE, 4)
    res["graph_unsorted"] = round(graph_rate(c), 1)
    c.set_schedule(0, 4)
    c.reset()
    for p in range(2):
        c.eval_batch(passes[p], outs, hits)
    tune = c.autotune(passes[2], reps=2)
    res["autotuned_schedule"] = tune["schedule"]
    res["graph_autotuned"] = round(graph_rate(c), 1)
    c.close()
    u = make(Pm.PMC_CACHE_OFF)
    res["uncached_graph_grouped"] = round(graph_rate(u, 1), 1)
    u.set_schedule(Pm.PMC_BLOCK_ITEMS, 4)
    res["uncached_graph_block_per_material"] = round(graph_rate(u, 1), 1)
    u.set_schedule(Pm.PMC_UNSORTED | Pm.PMC_EVAL_INLINE, 4)
    res["uncached_graph_unsorted"] = round(graph_rate(u, 1), 1)
    u.close()
    best = max(res["graph_grouped"], res["graph_unsorted"], res["graph_autotuned"], res["graph_block_per_material"],
               res["graph_one_point_per_lane"])
    res["speedup_cached_over_uncached"] = round(best / max(res["uncached_graph_grouped"], res["uncached_graph_unsorted"],
                                                           res["uncached_graph_block_per_material"]), 3)
    res["graph_over_eager"] = round(res["graph_grouped"] / res["eager"], 3)
    del passes
    torch.cuda.empty_cache()
    return res


def alg1_leg(torch, P, mats, dev_passes, outs, hits, local_rank):
    """The paper's concurrent update (Sec. 3.3, Alg. 1; PMC_ALG1) on the benchmark frame:
    8-byte slots {hash2, RGB9E5 value}, lookups and one-CAS inserts inside the evaluator,
    entries visible within the pass.  Cached points/s (whole frame as one CUDA graph, the
    schedule autotuned between grouped and unsorted), hit rate and counters of a frame."""
    n = WIDTH * HEIGHT
    c = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, flags=P.PMC_ALG1, device=local_rank)
    for p in range(2):
        c.eval_batch(dev_passes[p], outs, hits)
    tune = c.autotune(dev_passes[2], reps=2)
    c.reset()
    for p in range(SPP):
        c.eval_batch(dev_passes[p], outs, hits)
    st = c.stats()
    g = c.graph(dev_passes, [outs] * SPP, [hits] * SPP, reset=True)
    g.launch()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(3):
        g.launch()
    t1.record()
    torch.cuda.synchronize()
    g.close()
    c.close()
    return {"config": f"frame 1920x1080x16spp, table {N_CELLS}x{N_ENTRIES} slots of 8 B (128 MB), "
                      "RGB9E5 values, one 64-bit CAS per insert", "unit": UNIT,
            "cached": round(3 * n * SPP / (t0.elapsed_time(t1) / 1e3), 1),
            "schedule": tune["schedule"],
            "hit_rate": round(st["hits"] / max(1, st["lookups"]), 4),
            "table": {k: st[k] for k in ("inserted", "dropped_dup", "dropped_full", "dropped_race")}}


def raycast_leg(torch, P, mats, dev, local_rank, seed=0, min_root_cost=0):
    """Shading points from the library's ray caster instead of the synthetic stream: a
    closed room with 24 spheres, 64 materials (Zipf 1.1 over the objects), a 1920x1080
    pinhole camera, one primary ray per pixel per pass, 16 passes.  The caster alone
    (points/s and the HBM roofline of its 56 B of output per point), then cast + pass with
    per-point levels from the ray cones (Eq. 1), cached (every cacheable node, and above the
    cost threshold `min_root_cost`) and uncached, eager launches."""
    sc = W.Scene(W.SceneSpec(seed=seed))
    n = WIDTH * HEIGHT
    bufs = P.cast_rays(sc.objects, sc.camera, seed=seed + 1, pass_index=0)
    for p in range(3):
        P.cast_rays(sc.objects, sc.camera, seed=seed + 1, pass_index=p, out=bufs)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for p in range(SPP):
        P.cast_rays(sc.objects, sc.camera, seed=seed + 1, pass_index=p, out=bufs)
    t1.record()
    torch.cuda.synchronize()
    cast_s = t0.elapsed_time(t1) / 1e3
    hbm_peak, sm_mhz_max, peak_kind = peaks()
    gbs = 56.0 * n * SPP / cast_s / 1e9
    # FP32 operations per ray, counted from the caster's formulas (a multiply-add as 2):
    # 12 per plane, 24 per sphere, about 105 for the ray, the shading point and the cone
    n_planes = int((sc.objects["kind"] == W.KIND_PLANE).sum())
    flops_ray = 12 * n_planes + 24 * (len(sc.objects) - n_planes) + 105
    fp32_peak = n_sms(torch, dev) * FP32_LANES_PER_SM * 2 * sm_mhz_max * 1e6 / 1e12
    tflops = flops_ray * n * SPP / cast_s / 1e12
    res = {"config": f"room of 6 planes + 24 spheres, 64 materials, {WIDTH}x{HEIGHT} pinhole, {SPP} passes, "
                     f"table {N_CELLS}x{N_ENTRIES} slots, per-point levels from the ray cones", "unit": UNIT,
           "cast_points_per_s": round(n * SPP / cast_s, 1),
           "cast_roofline": {"kernel": "k_cast", "bound": "alu", "achieved": round(tflops, 2),
                             "peak": round(fp32_peak, 2), "unit": "TFLOP/s", "frac": round(tflops / fp32_peak, 4),
                             "flops_per_ray": flops_ray, "peak_kind": "FP32 lanes x 2 x max SM clock",
                             "output_gbs": round(gbs, 1), "output_frac_of_hbm": round(gbs / hbm_peak, 4),
                             "bytes_per_point": 56}}
    outs = torch.empty((3, n), dtype=torch.float32, device=dev)
    hits = torch.empty(n, dtype=torch.int16, device=dev)
    runs = [("cached", 0, 0), ("uncached", P.PMC_CACHE_OFF, 0)]
    if min_root_cost:
        runs.insert(1, ("cached_threshold", 0, min_root_cost))
    for name, flags, thr in runs:
        c = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, flags=flags, device=local_rank, min_root_cost=thr)
        for p in range(2):
            P.cast_rays(sc.objects, sc.camera, seed=seed + 1, pass_index=p, out=bufs)
            c.eval_batch(bufs, outs, hits)
        c.autotune(bufs, reps=2)
        c.reset()
        torch.cuda.synchronize()
        t0.record()
        for p in range(SPP):
            P.cast_rays(sc.objects, sc.camera, seed=seed + 1, pass_index=p, out=bufs)
            c.eval_batch(bufs, outs, hits)
        t1.record()
        torch.cuda.synchronize()
        st = c.stats()
        r = {"points_per_s": round(n * SPP / (t0.elapsed_time(t1) / 1e3), 1)}
        if name != "uncached":
            r.update(min_root_cost=thr, hit_rate=round(st["hits"] / max(1, st["lookups"]), 4),
                     inserted=st["inserted"], dropped_full=st["dropped_full"])
        c.close()
        res[name] = r
    res["speedup_cached_over_uncached"] = round(res["cached"]["points_per_s"] / res["uncached"]["points_per_s"], 3)
    if "cached_threshold" in res:
        res["speedup_threshold_over_uncached"] = round(res["cached_threshold"]["points_per_s"] /
                                                       res["uncached"]["points_per_s"], 3)
    return res


POS_LEVEL = 6   # world-position voxels of 1/64 unit: about 6 pixels of the frame per voxel edge


def position_leg(torch, P, mats, dev_passes, outs, hits, local_rank):
    """The benchmark frame with the world-position descriptor (Sec. 3.1 and Sec. 5): the
    networks' position noise (single FBM, Worley or checker nodes of the position) becomes
    cacheable under voxels of 2^-6 units.  Those are single nodes, so both cached runs take
    min_root_nodes = 1: UV descriptors only, UV and position descriptors, and uncached;
    the whole frame as one CUDA graph with the autotuned schedule."""
    n = WIDTH * HEIGHT
    res = {"config": f"frame 1920x1080x16spp, {N_MATS} materials, table {N_CELLS}x{N_ENTRIES} slots, "
                     f"min_root_nodes 1, position voxels of 2^-{POS_LEVEL}", "unit": UNIT}
    runs = (("uv_only", 0), ("uv_and_position", P.PMC_POSITION_DESCRIPTOR), ("uncached", P.PMC_CACHE_OFF))
    for name, flags in runs:
        c = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, flags=flags, min_root_nodes=1, pos_level=POS_LEVEL,
                    device=local_rank)
        for p in range(2):
            c.eval_batch(dev_passes[p], outs, hits)
        c.autotune(dev_passes[2], reps=2)
        c.reset()
        for p in range(SPP):
            c.eval_batch(dev_passes[p], outs, hits)
        st = c.stats()
        g = c.graph(dev_passes, [outs] * SPP, [hits] * SPP, reset=True)
        g.launch()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(3):
            g.launch()
        t1.record()
        torch.cuda.synchronize()
        g.close()
        c.close()
        r = {"points_per_s": round(3 * n * SPP / (t0.elapsed_time(t1) / 1e3), 1)}
        if name != "uncached":
            r.update(hit_rate=round(st["hits"] / max(1, st["lookups"]), 4),
                     lookups_per_point=round(st["lookups"] / (n * SPP), 3), inserted=st["inserted"],
                     dropped_full=st["dropped_full"])
        res[name] = r
    u = res["uncached"]["points_per_s"]
    res["speedup_uv_only_over_uncached"] = round(res["uv_only"]["points_per_s"] / u, 3)
    res["speedup_uv_and_position_over_uncached"] = round(res["uv_and_position"]["points_per_s"] / u, 3)
    return res


THRESHOLDS = (0, 150, 300, 450, 500, 550, 600, 900)


def threshold_leg(torch, P, mats, dev_passes, outs, hits, local_rank):
    """The benchmark frame with cacheable nodes restricted to sub-graphs of at least
    min_root_cost FP32 operations of the node cost model (0 = every node the rule of Sec. 3
    picks): probes per point, hit rate and frame throughput (one CUDA graph per frame,
    autotuned schedule) for each threshold."""
    n = WIDTH * HEIGHT
    res = {"config": f"frame 1920x1080x16spp, {N_MATS} materials, table {N_CELLS}x{N_ENTRIES} slots",
           "unit": UNIT, "runs": []}
    for thr in THRESHOLDS:
        c = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, min_root_cost=thr, device=local_rank)
        for p in range(2):
            c.eval_batch(dev_passes[p], outs, hits)
        c.autotune(dev_passes[2], reps=2)
        c.reset()
        for p in range(SPP):
            c.eval_batch(dev_passes[p], outs, hits)
        st = c.stats()
        g = c.graph(dev_passes, [outs] * SPP, [hits] * SPP, reset=True)
        g.launch()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(3):
            g.launch()
        t1.record()
        torch.cuda.synchronize()
        g.close()
        c.close()
        res["runs"].append({"min_root_cost": thr, "points_per_s": round(3 * n * SPP / (t0.elapsed_time(t1) / 1e3), 1),
                            "lookups_per_point": round(st["lookups"] / (n * SPP), 3),
                            "hit_rate": round(st["hits"] / max(1, st["lookups"]), 4),
                            "flops_per_point": round(st["flops"] / (n * SPP), 1)})
    return res


REPL_PASSES, REPL_BOUNCES = 8, (0.5, 0.25)


def replace_leg(torch, P, dev, local_rank, seed=0):
    """Path-traced passes of the benchmark frame (Sec. 5's case for prioritising directly
    visible shading points): each pass is one batch of the 2,073,600 directly visible
    samples (class 0) followed by the indirect shading points of two bounces (half and a
    quarter as many, each on the surface seen by a random pixel: classes 1 and 2); 8 passes,
    table 2^21 x 8.  Keep-first against replacement by visibility class: points/s of the
    whole sequence (reset + 8 passes) replayed as one CUDA graph, hit rate of all lookups
    and of the directly visible points' lookups over passes 1..7, entries replaced; and the
    same passes uncached."""
    mats, frame = workload(seed)
    host = [frame.points_paths(p, REPL_BOUNCES) for p in range(REPL_PASSES)]
    n = len(host[0]["u"])
    passes = [P.points_to_device(h, dev) for h in host]
    del host
    nroots = torch.tensor([len(P.analyze_material(m)["roots"]) for m in mats], dtype=torch.int64, device=dev)
    outs = torch.empty((3, n), dtype=torch.float32, device=dev)
    hits = [torch.empty(n, dtype=torch.int16, device=dev) for _ in passes]
    res = {"config": f"frame 1920x1080, {REPL_PASSES} path-traced passes of {n} points (2073600 direct + "
                     f"{n - WIDTH * HEIGHT} indirect of 2 bounces), {N_MATS} materials, "
                     f"table {N_CELLS}x{N_ENTRIES} slots", "unit": UNIT, "points_per_pass": n}
    for name, flags in (("keep_first", 0), ("replacement", P.PMC_REPLACE_VISIBILITY), ("uncached", P.PMC_CACHE_OFF)):
        c = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, flags=flags, device=local_rank)
        for p in range(2):
            c.eval_batch(passes[p], outs, hits[p])
        c.autotune(passes[2], reps=2)
        g = c.graph(passes, [outs] * REPL_PASSES, hits, reset=True)
        g.launch()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(3):
            g.launch()
        t1.record()
        torch.cuda.synchronize()
        g.close()
        r = {"points_per_s": round(3 * n * REPL_PASSES / (t0.elapsed_time(t1) / 1e3), 1)}
        if name != "uncached":
            c.reset()
            for p in range(REPL_PASSES):
                c.eval_batch(passes[p], outs, hits[p])
            st = c.stats()
            dh = dl = 0
            for p in range(1, REPL_PASSES):
                d = passes[p]["vis"] == 0
                dh += int(hits[p][d].long().sum())
                dl += int(nroots[passes[p]["mat"][d].long()].sum())
            r.update(hit_rate=round(st["hits"] / max(1, st["lookups"]), 4), direct_hit_rate=round(dh / max(1, dl), 4),
                     inserted=st["inserted"], replaced=st["replaced"], dropped_full=st["dropped_full"])
        c.close()
        res[name] = r
    res["speedup_replacement_over_keep_first"] = round(res["replacement"]["points_per_s"] /
                                                       res["keep_first"]["points_per_s"], 3)
    del passes
    torch.cuda.empty_cache()
    return res


def cones_leg(torch, P, dev, local_rank, seed=0, min_root_cost=0):
    """The benchmark frame with every shading point at its own mip level, from the
    texture-coordinate gradients of its ray-cone footprint (Eq. 1; footprint minor axis
    delta * 2^U(-1/2, 1/2), axis ratio log-uniform on [1, 4]), for level offsets 0 and -1,
    every cacheable node cached and with the cost threshold `min_root_cost` ("_threshold"):
    cached points/s (whole frame as one CUDA graph, autotuned schedule), hit rate and the
    levels the first pass uses.  Uncached evaluation does not depend on the level."""
    mats, frame = workload(seed)
    n = WIDTH * HEIGHT
    passes = [P.points_to_device(frame.points(p, cones=True), dev) for p in range(SPP)]
    outs = torch.empty((3, n), dtype=torch.float32, device=dev)
    hits = torch.empty(n, dtype=torch.int16, device=dev)
    lv = P.compute_levels(passes[0]["g1u"], passes[0]["g1v"], passes[0]["g2u"], passes[0]["g2v"])
    hist = torch.bincount(lv.long(), minlength=14).cpu().numpy()
    res = {"config": "frame 1920x1080x16spp, per-point mip level from ray-cone gradients, "
                     f"table {N_CELLS}x{N_ENTRIES} slots", "unit": UNIT,
           "levels_pass0": {int(k): int(v) for k, v in enumerate(hist) if v}}
    for off, thr in ((0, 0), (-1, 0), (0, min_root_cost), (-1, min_root_cost)):
        c = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, level_offset=off, device=local_rank,
                    min_root_cost=thr)
        for p in range(2):
            c.eval_batch(passes[p], outs, hits)
        c.autotune(passes[2], reps=2)
        c.reset()
        for p in range(SPP):
            c.eval_batch(passes[p], outs, hits)
        st = c.stats()
        g = c.graph(passes, [outs] * SPP, [hits] * SPP, reset=True)
        g.launch()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(3):
            g.launch()
        t1.record()
        torch.cuda.synchronize()
        g.close()
        c.close()
        res[f"offset{off}" + ("_threshold" if thr else "")] = {
            "cached": round(3 * n * SPP / (t0.elapsed_time(t1) / 1e3), 1), "min_root_cost": thr,
            "hit_rate": round(st["hits"] / max(1, st["lookups"]), 4),
            "inserted": st["inserted"], "dropped_full": st["dropped_full"]}
    del passes
    torch.cuda.empty_cache()
    return res


SCALE_MATS, SCALE_LO, SCALE_HI, SCALE_SP, SCALE_ZIPF, SCALE_SIDE, SCALE_BATCHES = 4096, 10, 2000, 0.4, 0.9, 2048, 64


def sweep_leg(torch, P, dev, local_rank, seed=0, full=True, min_root_cost=0):
    """The scale configuration: 4096 networks of 10-2000 nodes (40 % SP), materials
    Zipf(0.9) per 8x8 tile of a 2048x2048 stream, 2^28 points in 64 batches of 2^22.  With
    `full`, the table swept from 2^20 to 2^29 slots (16 MB - 8 GB); else 2^26 slots (1 GB)
    under the rule of Sec. 3 and under cost thresholds 300, 450, `min_root_cost` and 800.  Per run: points/s
    of the whole stream replayed as one CUDA graph, hit rate, inserted and dropped counts.
    Then the surrogate mix at 2^26 slots (with the cost threshold): networks trained for
    every material's candidate node, those validated within 1.6e-3 enabled."""
    from paper_2305_07238_gb300 import pmc as Pm
    t0 = time.perf_counter()
    mats = W.random_materials(SCALE_MATS, SCALE_LO, SCALE_HI, SCALE_SP, seed=seed + 500)
    frame = W.Frame(W.FrameSpec(width=SCALE_SIDE, height=SCALE_SIDE, n_mats=SCALE_MATS, zipf_s=SCALE_ZIPF,
                                seed=seed + 500))
    passes = [frame.points_torch(p, dev) for p in range(SCALE_BATCHES)]
    n = SCALE_SIDE * SCALE_SIDE
    roots = np.array([len(P.analyze_material(m)["roots"]) for m in mats])
    need = int(roots[frame.tile_mat[frame.pix_tile]].sum())
    outs = torch.empty((3, n), dtype=torch.float32, device=dev)
    hits = torch.empty(n, dtype=torch.int16, device=dev)
    total = n * SCALE_BATCHES
    res = {"config": f"{SCALE_MATS} materials {SCALE_LO}-{SCALE_HI} nodes ({int(SCALE_SP * 100)}% SP), "
                     f"Zipf {SCALE_ZIPF} per 8x8 tile of {SCALE_SIDE}x{SCALE_SIDE}, {SCALE_BATCHES} batches of {n} "
                     f"points ({total} points)",
           "unit": UNIT, "probes_per_batch": need, "setup_s": round(time.perf_counter() - t0, 1)}

    def rate(c):
        g = c.graph(passes, [outs] * SCALE_BATCHES, [hits] * SCALE_BATCHES, reset=True)
        g.launch()
        c.sync()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.launch()
        e1.record()
        torch.cuda.synchronize()
        g.close()
        return total / (e0.elapsed_time(e1) / 1e3)

    u = P.Cache(mats, 1 << 17, N_ENTRIES, uv_level=LEVEL, flags=Pm.PMC_CACHE_OFF, device=local_rank)
    res["uncached"] = round(rate(u), 1)
    u.close()
    rows = []
    thresholds = sorted({0, 300, 450, min_root_cost, 800})
    runs = [(ls, 0) for ls in range(20, 30)] if full else [(26, thr) for thr in thresholds]
    for log_slots, thr in runs:
        c = P.Cache(mats, 1 << (log_slots - 3), N_ENTRIES, uv_level=LEVEL, device=local_rank, probe_capacity=need,
                    min_root_cost=thr)
        r = rate(c)
        s = c.stats()
        rows.append({"slots": 1 << log_slots, "table_mb": (16 << log_slots) >> 20, "min_root_cost": thr,
                     "value": round(r, 1), "hit_rate": round(s["hits"] / max(1, s["lookups"]), 4),
                     "lookups_per_point": round(s["lookups"] / total, 3), "inserted": s["inserted"],
                     "dropped_full": s["dropped_full"], "speedup_over_uncached": round(r / res["uncached"], 3)})
        c.close()
    res["sweep" if full else "runs"] = rows
    c = P.Cache(mats, 1 << 23, N_ENTRIES, uv_level=LEVEL, device=local_rank, probe_capacity=need,
                min_root_cost=min_root_cost)
    t = time.perf_counter()
    rmse = c.train_surrogates(n_train=1 << 16, n_valid=1 << 13, epochs=16, lr=1e-2, seed=2)
    torch.cuda.synchronize()
    res["surrogate_mix"] = {"slots": 1 << 26, "min_root_cost": min_root_cost,
                            "train_s": round(time.perf_counter() - t, 2),
                            "candidates": int(np.sum(rmse >= 0)),
                            "enabled": int(np.sum((rmse >= 0) & (rmse <= 1.6e-3))),
                            "value": round(rate(c), 1)}
    s = c.stats()
    res["surrogate_mix"]["hit_rate"] = round(s["hits"] / max(1, s["lookups"]), 4)
    res["surrogate_mix"]["surrogate_evals"] = s["surrogate_evals"]
    res["surrogate_mix"]["speedup_over_uncached"] = round(res["surrogate_mix"]["value"] / res["uncached"], 3)
    c.close()
    del passes
    torch.cuda.empty_cache()
    return res


SURR_MATS, SURR_LO, SURR_HI, SURR_PASSES = 256, 500, 2000, 64
SURR_TRAIN, SURR_VALID, SURR_EPOCHS = 1 << 20, 1 << 16, 2
MLP_FLOPS_PER_POINT = 2 * (64 * 64 + 64 * 64 + 64 * 3)   # the network's multiply-adds, FMA = 2


def bf16_peak():
    """Dense BF16 tensor peak: the measured cuBLAS burst figure, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured cuBLAS BF16 burst"
    return 1900.0, "fallback"


def surrogate_leg(torch, P, dev, local_rank, seed=0):
    """Deep networks (256 of 500-2000 nodes, one cacheable node on a low-frequency UV tree
    each) shaded over 64 passes of 1920x1080 points: exact without cache, exact with the
    cache, and with surrogates trained on 2^20 pairs per network and validated on 2^16
    (cache on for any other node).  Training time, the fraction of networks enabled (a
    validation RMSE of at most 1.6e-3, a margin under the 2e-3 bar) and the median RMSE
    are reported."""
    mats = W.surrogate_materials(SURR_MATS, SURR_LO, SURR_HI, seed=seed)
    frame = W.Frame(W.FrameSpec(width=WIDTH, height=HEIGHT, n_mats=SURR_MATS, seed=seed + 100))
    passes = [frame.points_torch(p, dev) for p in range(SURR_PASSES)]
    n = WIDTH * HEIGHT
    outs = torch.empty((3, n), dtype=torch.float32, device=dev)
    res = {"config": f"{SURR_MATS} networks of {SURR_LO}-{SURR_HI} nodes, one cacheable node each on a "
                     f"low-frequency UV tree; {SURR_PASSES} passes of {n} points; table {N_CELLS}x{N_ENTRIES}"}

    def run(cache):
        cache.reset()
        for p in range(SURR_PASSES):
            cache.eval_batch(passes[p], outs)
        cache.sync()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cache.reset()
        t0.record()
        for p in range(SURR_PASSES):
            cache.eval_batch(passes[p], outs)
        t1.record()
        torch.cuda.synchronize()
        return n * SURR_PASSES / (t0.elapsed_time(t1) / 1e3)

    res["uncached"] = round(run(P.Cache(mats, N_CELLS, N_ENTRIES, flags=P.PMC_CACHE_OFF, device=local_rank)), 1)
    cached = P.Cache(mats, N_CELLS, N_ENTRIES, device=local_rank)
    res["cached"] = round(run(cached), 1)
    t = time.perf_counter()
    rmse = cached.train_surrogates(n_train=SURR_TRAIN, n_valid=SURR_VALID, epochs=SURR_EPOCHS, lr=1e-2, seed=1)
    torch.cuda.synchronize()
    res["train_s"] = round(time.perf_counter() - t, 3)
    res["train_pairs_per_network"] = SURR_TRAIN
    res["epochs"] = SURR_EPOCHS
    res["valid_pairs_per_network"] = SURR_VALID
    res["enabled_fraction"] = round(float(np.mean((rmse >= 0) & (rmse <= 1.6e-3))), 4)
    res["rmse_median"] = float(np.median(rmse[rmse >= 0])) if np.any(rmse >= 0) else None
    res["surrogate"] = round(run(cached), 1)
    # tensor-core roofline of the in-pass inference (k_surrogate_tc): with one cacheable node
    # per network and every network's surrogate enabled, the lookup phase is that kernel
    cached.reset()
    cached.sync()
    cached.read_timing()
    cached.set_timing(True)
    for p in range(SURR_PASSES):
        cached.eval_batch(passes[p], outs)
    cached.set_timing(False)
    tm = cached.read_timing()
    st = cached.stats()
    peak = bf16_peak()
    flops = MLP_FLOPS_PER_POINT * st["surrogate_evals"]
    ms_inf = tm["ms"]["lookup"]
    tf = flops / (ms_inf / 1e3) / 1e12 if ms_inf else 0.0
    res["tensor_roofline"] = {"kernel": "k_surrogate_tc", "bound": "tensor", "achieved": round(tf, 2),
                              "peak": peak[0], "unit": "TFLOP/s", "frac": round(tf / peak[0], 4),
                              "peak_kind": peak[1], "ms_per_pass": round(ms_inf / SURR_PASSES, 4),
                              "flops_per_point": MLP_FLOPS_PER_POINT}
    th = torch.tensor(cached.get_surrogate(0)["theta"], device=dev)
    u, v = passes[0]["u"], passes[0]["v"]
    for _ in range(3):
        P.mlp_forward(th, u, v)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        P.mlp_forward(th, u, v)
    e1.record()
    torch.cuda.synchronize()
    ms_fw = e0.elapsed_time(e1) / 10
    tf_fw = MLP_FLOPS_PER_POINT * n / (ms_fw / 1e3) / 1e12
    res["mlp_forward"] = {"points_per_s": round(n / (ms_fw / 1e3), 1), "achieved": round(tf_fw, 2),
                          "unit": "TFLOP/s", "frac": round(tf_fw / peak[0], 4)}
    res["unit"] = UNIT
    res["speedup_surrogate_over_uncached"] = round(res["surrogate"] / res["uncached"], 2)
    res["speedup_cached_over_uncached"] = round(res["cached"] / res["uncached"], 2)
    res["speedup_surrogate_over_cached"] = round(res["surrogate"] / res["cached"], 2)
    return res


def e2e_run(torch, P, mats, passes_host, args, local_rank, barrier, dist, dev, min_root_cost=0):
    """Same frame through pmc_eval_passes_host from pinned host buffers: every pass's points
    go in and its colours and hit counts come out inside the timed region, the copies of a
    pass overlapping the evaluation of its neighbours."""
    n = WIDTH * HEIGHT
    pinned = []
    for h in passes_host:
        d = {}
        for k in W.POINT_FIELDS:
            t = torch.from_numpy(h[k].view(np.int32) if k == "mat" else h[k]).pin_memory()
            d[k] = t.numpy().view(np.uint32) if k == "mat" else t.numpy()
        pinned.append(d)
    rgb = [torch.empty(3 * n, dtype=torch.float32).pin_memory().numpy() for _ in range(SPP)]
    hits = [torch.empty(n, dtype=torch.int16).pin_memory().numpy().view(np.uint16) for _ in range(SPP)]
    cache = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, min_root_cost=min_root_cost, device=local_rank)

    def frame_host():
        cache.reset()
        cache.eval_passes_host(pinned, rgb, hits)

    for _ in range(max(1, args.warmup)):
        frame_host()
    barrier()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        frame_host()
    torch.cuda.synchronize()
    secs = time.perf_counter() - t
    barrier()
    secs = max_over_ranks(torch, dist, secs, dev)
    world = dist.get_world_size() if dist is not None else 1
    cache.close()
    return {"value": round(whole_job_rate(n * SPP * args.steps, world, secs), 1), "unit": UNIT,
            "h2d_bytes_per_step": int(SPP * n * 36), "d2h_bytes_per_step": int(SPP * n * (12 + 2))}


def cpu_model():
    """The host CPU's model name, as the kernel reports it."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def oracle_rate(O, mats, passes, threads, min_root_cost=0):
    """Points/s of the FP64 oracle over a sequence of passes from an empty table."""
    ref = O.Cache(mats, N_CELLS, N_ENTRIES, level=LEVEL, threads=threads, min_root_cost=min_root_cost)
    npts, secs, outs = 0, 0.0, []
    for part in passes:
        t = time.perf_counter()
        outs.append(ref.run_batch(part)["rgb"])
        secs += time.perf_counter() - t
        npts += len(part["u"])
    return npts / secs, secs, npts, outs


def cpu_baseline(P, torch, mats, frame, dev, min_root_cost=0):
    """The FP64 oracle on the first SAMPLE_ROWS rows of all 16 passes (same table geometry and
    cost threshold as the headline), over all host cores (its points spread over OpenMP
    threads, the insert sequential) and on one core; the CUDA path runs the same sample for
    the error figure."""
    from oracle import oracle as O
    passes = [frame.points(p, rows=SAMPLE_ROWS) for p in range(SPP)]
    cores = os.cpu_count() or 1
    rate_all, secs_all, npts, outs = oracle_rate(O, mats, passes, cores, min_root_cost)
    rate_one, secs_one, _, _ = oracle_rate(O, mats, passes, 1, min_root_cost)
    gpu = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, min_root_cost=min_root_cost)
    err = 0.0
    for part, r in zip(passes, outs):
        d = P.points_to_device(part, dev)
        rgb = torch.empty((3, len(part["u"])), dtype=torch.float32, device=dev)
        gpu.eval_batch(d, rgb)
        gpu.sync()
        err = max(err, float(np.abs(rgb.cpu().numpy() - r).max()))
    gpu.close()
    rows = SAMPLE_ROWS[1] - SAMPLE_ROWS[0]
    sample = (f"rows {SAMPLE_ROWS[0]}-{SAMPLE_ROWS[1]} of all {SPP} passes ({rows * WIDTH} points/pass, "
              f"{npts} points), same table size and cost threshold ({min_root_cost})")
    return ({"value": round(rate_all, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
             "cpu": cpu_model(), "sample": f"{sample}; {secs_all:.1f} s on {cores} threads",
             "single_core": {"value": round(rate_one, 1), "unit": UNIT, "cores": 1,
                             "sample": f"{sample}; {secs_one:.1f} s"}},
            err)


PRIM_POINTS = 1 << 20


def primitive_materials():
    """Single-primitive networks for counting what each node costs on the device: for every
    primitive a chain of L copies (L = 1 and 9) fed by UV, each copy reading the previous one
    (two-input primitives read UV as their second input).  A checker must read UV itself,
    so its copies are joined by MIX nodes (the MIX chain is measured on its own).  With the
    cache off every node of a chain is evaluated for every point."""
    B = W.Builder
    specs = {
        "FBM1": (W.OP_FBM, dict(ip=[1, 5], fp=[4.0, 2.0, 0.5])),
        "FBM4": (W.OP_FBM, dict(ip=[4, 5], fp=[4.0, 2.0, 0.5])),
        "VORONOI": (W.OP_VORONOI, dict(ip=[0, 5], fp=[8.0])),
        "RAMP4": (W.OP_RAMP, dict(ip=[4], fp=[0.0, 0.3, 0.6, 1.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6,
                                                0.7, 0.8, 0.9, 0.2, 0.4, 0.6])),
        "MIX": (W.OP_MIX, dict(fp=[0.3])),
        "ADD": (W.OP_ADD, {}),
        "MUL": (W.OP_MUL, {}),
        "POW": (W.OP_POW, dict(fp=[1.5])),
        "FACING": (W.OP_FACING, dict(fp=[0.6, 0.8, 0.0])),
        "UV_AFFINE": (W.OP_UV_AFFINE, dict(fp=[0.8, -0.6, 0.6, 0.8, 0.25, 0.5])),
        "CHECKER": (W.OP_CHECKER, dict(fp=[8.0, 0.1, 0.2, 0.3, 0.9, 0.8, 0.7])),
    }
    out = []
    for name, (op, kw) in specs.items():
        for L in (1, 9):
            b = B()
            uv = b.add(W.OP_UV)
            prev = uv
            for _ in range(L):
                if op == W.OP_CHECKER:
                    ck = b.add(op, [uv], **kw)
                    prev = b.add(W.OP_MIX, [prev, ck], fp=[0.3])
                elif op in (W.OP_ADD, W.OP_MUL, W.OP_MIX):
                    prev = b.add(op, [prev, uv], **kw)
                else:
                    prev = b.add(op, [prev], **kw)
            out.append((name, L, b.build()))
    return out


def profile_primitives(only=""):
    """One cache-off pass of PRIM_POINTS uniform points per single-primitive network (of
    `only` alone if given), in the order printed after one warm-up pass, so that an ncu
    capture of k_eval that skips one launch gets one launch per (primitive, chain length): the per-node instruction and FP32 operation counts
    follow from the difference between the 9-copy and 1-copy chains."""
    import torch
    from paper_2305_07238_gb300 import build as B
    from paper_2305_07238_gb300 import pmc as P
    B.build()
    pts = P.points_to_device(W.points_uniform(PRIM_POINTS, seed=0))
    rgb = torch.empty((3, PRIM_POINTS), dtype=torch.float32, device="cuda")
    rows = []
    chains = [(name, L, mat) for name, L, mat in primitive_materials() if not only or name == only]
    w = P.Cache([chains[0][2]], 1, 1, flags=P.PMC_CACHE_OFF)     # one warm-up launch (ncu -s 1)
    w.eval_batch(pts, rgb)
    w.close()
    for name, L, mat in chains:
        c = P.Cache([mat], 1, 1, flags=P.PMC_CACHE_OFF)
        c.eval_batch(pts, rgb)
        st = c.stats()
        rows.append({"primitive": name, "chain": L, "nodes_per_point": st["nodes_evaluated"] / PRIM_POINTS,
                     "flops_per_point": st["flops"] / PRIM_POINTS})
        c.close()
    return {"profile": "primitives", "points": PRIM_POINTS, "launch_order": rows}


TRAIN_FLOPS_PER_STEP = 2 * 128 * (2 * (64 * 64 + 64 * 64 + 64 * 3) + (3 * 64 + 64 * 64))


def profile_train(args):
    """One network trained on 2^16 random (u, v, target) rows for `steps` minibatches of 128
    in one launch of the tensor-core training kernel (one CTA): per-step time and the
    useful tensor work per step (forward, backward to the hidden activations, weight
    gradients)."""
    import torch
    from paper_2305_07238_gb300 import build as B
    from paper_2305_07238_gb300 import pmc as P
    B.build()
    rng = np.random.default_rng(0)
    n = 1 << 16
    data = torch.tensor(rng.random((n, 5)), dtype=torch.float32, device="cuda")
    theta = torch.tensor(rng.normal(0, 0.1, 8515), dtype=torch.float32, device="cuda")
    m1, m2 = torch.zeros(8515, device="cuda"), torch.zeros(8515, device="cuda")
    steps = max(1, args.steps) * 128
    P.mlp_train(theta, m1, m2, data, steps, 0, steps, 1e-3)      # warm-up launch
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    P.mlp_train(theta, m1, m2, data, steps, steps, 2 * steps, 1e-3)
    t1.record()
    torch.cuda.synchronize()
    us = t0.elapsed_time(t1) * 1e3 / steps
    return {"profile": "surrogate training, one network", "steps": steps, "us_per_step": round(us, 3),
            "useful_tflops_per_cta": round(TRAIN_FLOPS_PER_STEP / (us * 1e-6) / 1e12, 3)}


def profile_run(args):
    """Eager frames only (default schedule, no autotuning, no graph, no other legs), so
    that an ncu launch list can select whole frames: W warm-up frames, then K frames.
    With --profile-surrogate: 32 deep networks with trained surrogates, K passes of
    2,073,600 points (the tensor-core inference kernel on a full pass)."""
    import torch
    from paper_2305_07238_gb300 import build as B
    from paper_2305_07238_gb300 import pmc as P
    B.build()
    if args.profile_surrogate:
        mats = W.surrogate_materials(32, SURR_LO, SURR_HI, seed=0)
        frame = W.Frame(W.FrameSpec(width=WIDTH, height=HEIGHT, n_mats=32, seed=100))
        n = WIDTH * HEIGHT
        outs = torch.empty((3, n), dtype=torch.float32, device="cuda")
        cache = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL)
        rmse = cache.train_surrogates(n_train=1 << 14, n_valid=1024, epochs=4, lr=1e-2, seed=1)
        for m in range(len(mats)):   # every network on, whatever its fit, for the kernel's sake
            cache.set_surrogate(m, cache.get_surrogate(m)["theta"])
        passes = [frame.points_torch(p, "cuda") for p in range(max(1, args.steps))]
        for d in passes:
            cache.eval_batch(d, outs)
        cache.sync()
        return {"profile": "surrogate passes", "passes": len(passes), "networks": len(mats),
                "surrogate_evals": cache.stats()["surrogate_evals"], "rmse_median": float(np.median(rmse))}
    mats, frame = workload(seed=0)
    n_pass = args.profile_passes or SPP
    dev_passes = [P.points_to_device(frame.points(p)) for p in range(n_pass)]
    n = WIDTH * HEIGHT
    outs = torch.empty((3, n), dtype=torch.float32, device="cuda")
    hits = torch.empty(n, dtype=torch.int16, device="cuda")
    flags = P.PMC_CACHE_OFF if args.profile_uncached else 0
    cache = P.Cache(mats, N_CELLS, N_ENTRIES, uv_level=LEVEL, flags=flags, min_root_cost=args.profile_min_root_cost)

    def frame_():
        cache.reset()
        for p in range(n_pass):
            cache.eval_batch(dev_passes[p], outs, hits)

    for _ in range(args.warmup):
        frame_()
    cache.sync()
    cache.read_timing()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        frame_()
    t1.record()
    torch.cuda.synchronize()
    secs = t0.elapsed_time(t1) / 1e3
    launches = cache.read_timing()["launches"]
    return {"profile": "eager frames" + (" (cache off)" if args.profile_uncached else ""),
            "min_root_cost": args.profile_min_root_cost,
            "passes_per_frame": n_pass, "value": round(n * n_pass * args.steps / secs, 1), "unit": UNIT,
            "steps": args.steps, "warmup": args.warmup, "launches_per_frame": launches // max(1, args.steps)}


# --------------------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# --------------------------------------------------------------------------------------
def reference(args):
    from oracle import oracle as O
    mats, frame = workload(seed=0)
    passes = [frame.points(p, rows=REF_ROWS) for p in range(SPP)]
    cores = os.cpu_count() or 1
    ref = O.Cache(mats, N_CELLS, N_ENTRIES, level=LEVEL, threads=cores, min_root_cost=REF_MIN_ROOT_COST)

    def step():
        ref.reset()
        for p in range(SPP):
            ref.run_batch(passes[p])

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    secs = time.perf_counter() - t
    npts = sum(len(p["u"]) for p in passes) * args.steps
    value = npts / secs
    rows = REF_ROWS[1] - REF_ROWS[0]
    sample = (f"rows {REF_ROWS[0]}-{REF_ROWS[1]} of all {SPP} passes per step "
              f"({rows * WIDTH} points/pass), same materials, table size and cost threshold")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(secs / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict({"parallelism": f"{cores} CPU threads (OpenMP), sequential insert",
                                   "min_root_cost": REF_MIN_ROOT_COST}),
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "cpu": cpu_model(), "sample": sample},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs",
                    default="cached,uncached,e2e,surr,f128,scale,threshold,alg1,cones,raycast,position,replace,cpu",
                    help="comma list of cached, uncached, e2e, surr, f128, scale, threshold, alg1, cones, raycast, "
                         "position, replace, sweep, cpu (sweep, the full table-size sweep of the scale "
                         "configuration, is not in the default: a few minutes more)")
    ap.add_argument("--profile", action="store_true",
                    help="eager frames only, for ncu launch lists (prints launches per frame)")
    ap.add_argument("--profile-surrogate", action="store_true",
                    help="with --profile: passes of 32 networks with surrogates (tensor-core kernel)")
    ap.add_argument("--profile-passes", type=int, default=0,
                    help="with --profile: passes per frame (default 16; fewer for small ncu captures)")
    ap.add_argument("--profile-uncached", action="store_true",
                    help="with --profile: the same frames with the cache off")
    ap.add_argument("--profile-primitives", action="store_true",
                    help="one cache-off pass per single-primitive network (per-node device costs)")
    ap.add_argument("--primitive", default="",
                    help="with --profile-primitives: only this primitive's two chains (two launches)")
    ap.add_argument("--profile-min-root-cost", type=int, default=0,
                    help="with --profile: the cost threshold of cacheable nodes")
    ap.add_argument("--profile-train", action="store_true",
                    help="one launch of the surrogate training kernel on one network (steps x 128 minibatches)")
    args = ap.parse_args()
    if args.profile_primitives:
        print(json.dumps(profile_primitives(args.primitive)), flush=True)
        return 0
    if args.profile_train:
        print(json.dumps(profile_train(args)), flush=True)
        return 0
    if args.profile:
        print(json.dumps(profile_run(args)), flush=True)
        return 0

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference(args)), flush=True)
        return 0

    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl", device_id=torch.device(f"cuda:{local_rank}"))
        dist = tdist
    line = ours(args, rank, world, local_rank, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
