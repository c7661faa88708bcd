#!/usr/bin/env python3
"""Benchmark of the DRT hot path on the full-3D canyon workload (one GB300 per rank).

Workload (the full-3D FP64 DRT case): urban canyon 20 m wide, 40 facades, 8 moving and yawing
vehicles, 512 ray chains of <= 3 interactions (R:D:S = 6:2:2, committed t0 path set), 60 GHz,
2000 steps x 0.5 ms, 512 frequency bins over 1 GHz, FP64 form.

One step = one drt_synthesize_H call on the resident link: pose table (a2), extrapolation of every
(path, time-step) with field coefficients and Doppler (a3-a8), H(t, f) synthesis (a9).
value = path-timesteps/s over all ranks (each rank runs its own link: weak scaling, no data-path
collective).  L2 (129 MB) is flushed by a 256 MB write between timed steps, outside the events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference implementation of this method here) on
the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2205_00237_gb300 import inputs as I  # noqa: E402

METRIC = "path-timesteps/s and H(t,f) samples/s at stated error vs FP64 oracle"
UNIT = "path-timesteps/s"
WORKLOAD = "canyon"
PATHSET = os.path.join(ROOT, "tests", "golden", "pathset_canyon_seed0.npz")

# Roofline of the dominant kernel (k_extrapolate_fp64, FP64-pipe bound; the H synthesis asks for no
# Doppler output, so its geometry runs on values).  FP64 FLOPs executed per path-step on this
# workload (DADD + DMUL + 2 DFMA thread-instructions counted by ncu, see
# profiles/k_extrapolate_fp64_canyon.md) and the FP64 peak of the GB300 derived from its unit counts:
# 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz = 1.26 TFLOP/s (no FP64 tensor path is used).  DRAM bytes
# per launch from the same capture (set to None whenever the kernel changes after the capture).
FP64_FLOP_PER_PATH_STEP = 1747.0
FP64_PEAK_FLOPS = 152 * 2 * 2 * 2.07e9
K1_DRAM_BYTES_PER_LAUNCH = 28.32e6
# the same capture: the FP64 pipe was busy this fraction of the launch (conversions, compares and the
# division / square-root sequences occupy it without counting as DADD / DMUL / DFMA FLOPs)
K1_FP64_PIPE_ACTIVE = 0.869
# FP32-bulk form (profiles/k_extrapolate_bulk_canyon.md, profiles/k_synth_canyon.md): FP32 FLOPs per
# path-step of k_extrapolate_bulk (FADD + FMUL + 2 FFMA, ncu) and 8 FLOP per synthesis term; FP32
# peak 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz = 80.5 TFLOP/s
FP32_FLOP_PER_PATH_STEP = 1733.0
FP32_PEAK_FLOPS = 152 * 128 * 2 * 2.07e9
SYNTH_FLOP_PER_TERM = 8.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-links", type=int, default=4096, help="links of the batched workload (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="measured serving window (0: skip)")
    ap.add_argument("--highway", action="store_true", help="also time the large highway batch (~1 min)")
    ap.add_argument("--highway-steps", type=int, default=1, help="timed runs of the highway batch")
    ap.add_argument("--serve-warmup", type=float, default=2.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="Poisson arrival rate, requests/s")
    return ap.parse_args()


def workload():
    scene = I.scene_canyon(0)
    paths = I.PathSet.from_npz(PATHSET)
    tg, fg = I.grids(WORKLOAD)
    return scene, paths, tg, fg


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(seconds: float, world: int, device=None) -> float:
    """The slowest rank's time (all ranks get it); every rank runs its own link, so the job takes as
    long as its slowest rank."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Units all ranks processed divided by the slowest rank's time (weak scaling)."""
    return world * units_per_rank / max_seconds


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def cpu_baseline(scene, paths, tg, fg, n_steps):
    """The FP64 oracle as it stands (O-DRT extrapolation + direct H sum) on all host cores."""
    import oracle as O
    cores = os.cpu_count() or 1
    sub = I.TimeGrid(tg.t_start, tg.dt, n_steps)
    t0 = time.perf_counter()
    rec = O.extrapolate(scene, paths, sub, fg.fc, n_threads=cores)
    O.synthesize_H(rec, fg, n_threads=cores)
    dt = time.perf_counter() - t0
    return {"value": paths.n_paths * n_steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{paths.n_paths} paths x {n_steps} of {tg.n_steps} steps x {fg.n_bins} bins "
                      f"(extrapolation + H), {dt:.2f} s wall on {cores} threads",
            "h_samples_per_s": n_steps * fg.n_bins / dt}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    scene, paths, tg, fg = workload()
    import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    n_sub = 64   # time steps per step: a bounded sample of the workload
    times = []
    for k in range(args.warmup + args.steps):
        sub = I.TimeGrid(tg.t_start + (k * n_sub % tg.n_steps) * tg.dt, tg.dt, n_sub)
        t0 = time.perf_counter()
        rec = O.extrapolate(scene, paths, sub, fg.fc, n_threads=cores)
        O.synthesize_H(rec, fg, n_threads=cores)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = paths.n_paths * n_sub * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "h_samples_per_s": n_sub * fg.n_bins * args.steps / total,
            "config": {"workload": "canyon-512paths-2000x0.5ms-512bins-60GHz-fp64",
                       "sample_per_step": f"{paths.n_paths} paths x {n_sub} steps x {fg.n_bins} bins"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                             "sample": f"{paths.n_paths} paths x {n_sub} consecutive steps per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_batched(args, ctx, drt, flush):
    """The batched FP32-bulk form over `--batch-links` uneven links (log-uniform 8..2048 paths,
    horizons uniform 100..5000 x 1 ms, 256 bins at 28 GHz): one drt_batch_run per step, replayed
    from its CUDA graph."""
    import torch
    w = I.BATCH
    spec = I.batch_links(args.batch_links, seed=0)
    sets = [(I.scene_link(k), I.PathSet.from_npz(os.path.join(ROOT, "tests", "golden", f"pathset_link_seed{k}.npz")))
            for k in range(I.LINK_SCENES)]
    t0 = time.perf_counter()
    loaded, links, tgs, fgs, Hs = {}, [], [], [], []
    for k, P, T in spec:
        if (k, P) not in loaded:
            loaded[(k, P)] = ctx.load(sets[k][0], sets[k][1].subset(np.arange(P)))
        links.append(loaded[(k, P)])
        tgs.append(I.TimeGrid(0.0, w["dt"], T))
        fgs.append(I.FreqGrid(w["fc"], w["bandwidth"], w["n_bins"]))
        Hs.append(torch.empty((T, w["n_bins"]), dtype=torch.complex64, device="cuda"))
    load_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = ctx.batch(links, tgs, fgs, Hs)
    plan_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    for _ in range(3):
        b.run(use_graph=True)
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.batch_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(use_graph=True)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    total_s = sum(a.elapsed_time(c) for a, c in evs) * 1e-3
    info = b.info(redo=True)
    ps_steps = sum(P * T for _, P, T in spec)
    h_samples = sum(T for _, _, T in spec) * w["n_bins"]
    out = {"value": ps_steps * args.batch_steps / total_s, "unit": UNIT,
           "h_samples_per_s": h_samples * args.batch_steps / total_s,
           "terms_per_s": ps_steps * w["n_bins"] * args.batch_steps / total_s,
           "ms_per_step": 1e3 * total_s / args.batch_steps, "steps": args.batch_steps,
           "workload": f"{len(spec)} links, paths log-U[8,2048] (mean {np.mean([p for _, p, _ in spec]):.0f}), "
                       f"steps U[100,5000] x 1 ms (mean {np.mean([t for _, _, t in spec]):.0f}), "
                       f"{w['n_bins']} bins over 400 MHz at 28 GHz",
           "path_steps_per_step": ps_steps, "precision": "DRT_FP32_BULK", "graph": True,
           "synth_tile_variant": info["variant"], "scratch_gb": info["scratch_bytes"] / 1e9,
           "redo_steps_per_step": info["redo_steps"], "load_s": load_s, "plan_and_autotune_s": plan_s,
           "l2": "flushed by a 256 MB write between timed steps (outside the events)"}
    b.close()
    del Hs
    for lk in loaded.values():
        lk.unload()
    return out


def run_power(args, link, tg, fg, drt, flush):
    """Power-Doppler (200 ms windows x 14.34 Hz bins over +-8 kHz) and power-delay (200 ms x 1 ns
    over 4.096 us) profiles of the canyon link, each one drt_power_profile call (extrapolation with
    Doppler and records, then the binning kernel)."""
    import torch
    stream = torch.cuda.current_stream()
    spb = max(1, int(round(0.2 / tg.dt)))
    cases = {"pdfp": (-8000.0, 14.34, 1116, drt.PP_DOPPLER), "pdp": (0.0, 1e-9, 4096, drt.PP_DELAY)}
    out = {"windows_steps": spb, "l2": "flushed between timed calls"}
    for prec, pname in ((drt.FP64, "fp64"), (drt.FP32_BULK, "fp32_bulk")):
        for name, (x0, dx, nb, kind) in cases.items():
            P = link.power_profile(tg, fg, spb, x0, dx, nb, kind, prec)
            for _ in range(2):
                link.power_profile(tg, fg, spb, x0, dx, nb, kind, prec, P=P)
            torch.cuda.synchronize()
            evs = []
            for _ in range(max(1, args.steps)):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                link.power_profile(tg, fg, spb, x0, dx, nb, kind, prec, P=P)
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
            ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
            out[f"{name}_{pname}"] = {"ms": ms, "path_steps_per_s": link.n_paths * tg.n_steps / (ms * 1e-3),
                                      "bins": nb}
    return out


def run_lifetime(args, link, tg, fg, drt, flush):
    """Multipath-lifetime management on the canyon link: the window plan (drt_lifetime_windows, share
    1e-5 of the power, windows of 10 to 150 ms) and H over those windows (drt_synthesize_H_windows),
    beside the plain H of the same form."""
    import torch
    stream = torch.cuda.current_stream()
    mn, mx = max(1, int(round(0.01 / tg.dt))), max(1, int(round(0.15 / tg.dt)))
    out = {"share": 1e-5, "min_steps": mn, "max_steps": mx, "l2": "flushed between timed calls"}
    H = torch.empty((tg.n_steps, fg.n_bins), dtype=torch.complex64, device="cuda")
    for prec, pname in ((drt.FP64, "fp64"), (drt.FP32_BULK, "fp32_bulk")):
        starts, major = link.lifetime_windows(tg, fg, 1e-5, mn, mx, prec)
        plan_ms = []
        for _ in range(max(1, args.steps)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            link.lifetime_windows(tg, fg, 1e-5, mn, mx, prec)
            plan_ms.append(1e3 * (time.perf_counter() - t0))
        for _ in range(2):
            link.synthesize_H_windows(tg, fg, starts, prec, H=H)
        torch.cuda.synchronize()
        evs = []
        for _ in range(max(1, args.steps)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            link.synthesize_H_windows(tg, fg, starts, prec, H=H)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
        out[pname] = {"windows": len(starts), "major_changes": int(major.sum()),
                      "plan_ms_wall": statistics.median(plan_ms), "windowed_H_ms": ms,
                      "path_steps_per_s": link.n_paths * tg.n_steps / (ms * 1e-3)}
    return out


def run_wideband(args, link, tg, fg, drt, flush, n_sub=4):
    """H with field coefficients per sub-band (drt_synthesize_H_wideband, 4 sub-bands) on the canyon
    link, both forms: one extrapolation and one synthesis per sub-band."""
    import torch
    stream = torch.cuda.current_stream()
    H = torch.empty((tg.n_steps, fg.n_bins), dtype=torch.complex64, device="cuda")
    out = {"n_sub": n_sub, "l2": "flushed between timed calls"}
    for prec, pname in ((drt.FP64, "fp64"), (drt.FP32_BULK, "fp32_bulk")):
        for _ in range(2):
            link.synthesize_H_wideband(tg, fg, n_sub, prec, H=H)
        torch.cuda.synchronize()
        evs = []
        for _ in range(max(1, args.steps)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            link.synthesize_H_wideband(tg, fg, n_sub, prec, H=H)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
        out[pname] = {"ms": ms, "path_steps_per_s": link.n_paths * tg.n_steps / (ms * 1e-3)}
    return out


def run_highway(args, ctx, drt, flush):
    """The large vehicular highway (64 links x 20300 paths, 28 and 60 GHz, 20000 x 0.1 ms, 1024
    bins, FP32-bulk) through one drt_batch_run per step, graph-replayed."""
    import torch
    hw = I.HIGHWAY
    rd = I.PathSet.from_npz(os.path.join(ROOT, "tests", "golden", "pathset_highway_rd_seed0.npz"))
    tg = I.TimeGrid(0.0, hw["dt"], hw["n_steps"])
    fgs = [I.FreqGrid(fc, hw["bandwidth"], hw["n_bins"]) for fc in hw["carriers"]]
    t0 = time.perf_counter()
    links = [ctx.load(I.scene_highway(0, l), I.highway_pathset(rd, l)) for l in range(hw["n_links"])]
    load_s = time.perf_counter() - t0
    entries = [(l, fg) for fg in fgs for l in range(hw["n_links"])]
    Hs = [torch.empty((tg.n_steps, fg.n_bins), dtype=torch.complex64, device="cuda") for _, fg in entries]
    t0 = time.perf_counter()
    b = ctx.batch([links[l] for l, _ in entries], [tg] * len(entries), [fg for _, fg in entries], Hs)
    plan_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    b.run(use_graph=True)
    torch.cuda.synchronize()
    evs = []
    for _ in range(max(1, args.highway_steps)):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(use_graph=True)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    sec = statistics.mean(a.elapsed_time(c) for a, c in evs) * 1e-3
    info = b.info(redo=True)
    P = rd.n_paths // hw["n_links"] + hw["n_tiles"]
    ps = len(entries) * P * tg.n_steps
    out = {"value": ps / sec, "unit": UNIT, "s_per_step": sec, "steps": len(evs),
           "h_samples_per_s": len(entries) * tg.n_steps * hw["n_bins"] / sec,
           "terms_per_s": ps * hw["n_bins"] / sec, "path_steps_per_step": ps,
           "workload": f"{hw['n_links']} links x {P} paths ({hw['n_tiles']} ER tiles + {hw['n_rd']} R/D), "
                       f"carriers {[f / 1e9 for f in hw['carriers']]} GHz, {tg.n_steps} x {tg.dt * 1e3} ms, "
                       f"{hw['n_bins']} bins over {hw['bandwidth'] / 1e6:.0f} MHz, FP32-bulk",
           "synth_tile_variant": info["variant"], "scratch_gb": info["scratch_bytes"] / 1e9,
           "redo_steps_per_step": info["redo_steps"], "load_s": load_s, "plan_and_autotune_s": plan_s}
    b.close()
    del Hs
    for lk in links:
        lk.unload()
    return out


def run_serving(args, drt):
    """Poisson-arriving prediction requests on resident canyon links (512, 128 and 32 paths),
    horizons U{50..500} x 1 ms from random start times, 512 bins at 60 GHz, HBM budget 64 GB."""
    import torch
    ctx = drt.Context(torch.cuda.current_device(), hbm_budget=64 << 30)
    scene = I.scene_canyon(0)
    paths = I.PathSet.from_npz(PATHSET)
    links = [ctx.load(scene, paths), ctx.load(scene, paths.subset(np.arange(128))),
             ctx.load(scene, paths.subset(np.arange(32)))]
    weights = np.array([0.6, 0.25, 0.15])
    ctx.serve_start(0, 4, 256)
    F, ring = 512, 2048
    bufs = [torch.empty((500, F), dtype=torch.complex64, device="cuda") for _ in range(ring)]
    rng = np.random.default_rng(11)
    duration = args.serve_warmup + args.serve_seconds
    n_req = int(args.serve_rate * duration * 1.2) + 16
    gaps = rng.exponential(1.0 / args.serve_rate, n_req)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < duration]
    li = rng.choice(len(links), len(arrivals), p=weights)
    hor = rng.integers(50, 501, len(arrivals))
    t_starts = rng.integers(0, 1000, len(arrivals)) * 1e-3
    tickets = [None] * len(arrivals)
    results = [None] * len(arrivals)
    fg = I.FreqGrid(60e9, 1e9, F)
    done_upto = [0]

    def collector():
        for i in range(len(arrivals)):
            while tickets[i] is None:
                time.sleep(1e-4)
            results[i] = ctx.wait(tickets[i], 60000)
            done_upto[0] = i + 1

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for i, ta in enumerate(arrivals):
        while time.perf_counter() - t0 < ta:
            pass
        while i - done_upto[0] >= ring - 1:      # the ring buffer slot is still in use
            time.sleep(1e-4)
        H = bufs[i % ring][:hor[i]]
        tickets[i] = ctx.submit(links[li[i]], I.TimeGrid(float(t_starts[i]), 1e-3, int(hor[i])), fg, H)
    th.join()
    t_end = time.perf_counter() - t0
    stats = ctx.serve_stats()
    ctx.serve_stop()
    n_paths = np.array([lk.n_paths for lk in links])
    sub = np.array([r["t_submit"] for r in results])
    t_first = sub.min()
    meas = (sub - t_first) >= args.serve_warmup
    lat = np.array([r["latency"] for r in results])[meas] * 1e3
    done_t = np.array([r["t_done"] for r in results])
    ps = (n_paths[li] * hor)[meas]
    span = done_t[meas].max() - sub[meas].min()
    ok = all(r["status"] == 0 for r in results)
    for lk in links:
        lk.unload()
    ctx.close()
    return {"requests": int(meas.sum()), "offered_req_per_s": args.serve_rate,
            "achieved_req_per_s": meas.sum() / span, "value": ps.sum() / span, "unit": UNIT,
            "h_samples_per_s": (hor[meas] * F).sum() / span,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                           "p99": float(np.percentile(lat, 99)), "max": float(lat.max())},
            "mean_batch_requests": float(np.mean([r["batch_requests"] for r in results])),
            "launches": stats["launches"], "arena_peak_gb": stats["arena_peak"] / 1e9, "all_ok": ok,
            "window_s": args.serve_seconds, "warmup_s": args.serve_warmup, "wall_s": t_end,
            "workload": "Poisson arrivals; canyon links of 512/128/32 paths (p = 0.6/0.25/0.15); horizons "
                        "U{50..500} x 1 ms from t_start U[0,1) s; 512 bins over 1 GHz at 60 GHz; FP32-bulk; "
                        "HBM budget 64 GB"}


def run_ours(args):
    import torch
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00237_gb300 import drt

    scene, paths, tg, fg = workload()
    P, T, F = paths.n_paths, tg.n_steps, fg.n_bins
    dev = torch.device("cuda", local_rank)
    ctx = drt.Context(local_rank)
    link = ctx.load(scene, paths)
    H = torch.empty((T, F), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        link.synthesize_H(tg, fg, drt.FP64, H)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read()
    sampler = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    evs = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        link.synthesize_H(tg, fg, drt.FP64, H)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier()
    clocks = sampler.stop()
    prof = ctx.profile_read()
    ctx.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_s = sum(step_ms) * 1e-3
    total_s = max_over_ranks(total_s, world, dev)
    value = whole_job_rate(P * T * args.steps, world, total_s)
    n_launch, k1_ms = prof["extrapolate"]
    k1_avg_s = k1_ms * 1e-3 / max(1, args.steps)
    kernel_launches = sum(v[0] for v in prof.values())

    # the FP32-bulk form on the same link (reported beside the FP64 headline)
    for _ in range(3):
        link.synthesize_H(tg, fg, drt.FP32_BULK, H)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read()
    evb = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        link.synthesize_H(tg, fg, drt.FP32_BULK, H)
        e1.record(stream)
        evb.append((e0, e1))
    torch.cuda.synchronize()
    profb = ctx.profile_read()
    ctx.profile(False)
    bulk_s = sum(a.elapsed_time(b) for a, b in evb) * 1e-3
    bulk_s = max_over_ranks(bulk_s, world, dev)
    fp32_bulk = {"value": whole_job_rate(P * T * args.steps, world, bulk_s), "unit": UNIT, "ms_per_step": 1e3 * bulk_s / args.steps,
                 "h_samples_per_s": world * T * F * args.steps / bulk_s, "precision": "DRT_FP32_BULK",
                 "kernel_ms": {k: (v[1] / args.steps) for k, v in profb.items() if v[0]},
                 "kernel_ms_note": "device time per step of each kernel kind (all its launches)"}
    ke, ks = fp32_bulk["kernel_ms"].get("extrapolate"), fp32_bulk["kernel_ms"].get("synth")
    if ke and ks:
        a1 = FP32_FLOP_PER_PATH_STEP * P * T / (ke * 1e-3)
        a3 = SYNTH_FLOP_PER_TERM * P * T * F / (ks * 1e-3)
        fp32_bulk["rooflines"] = {
            "k_extrapolate_bulk": {"bound": "alu", "achieved": a1 / 1e12, "peak": FP32_PEAK_FLOPS / 1e12,
                                   "unit": "TFLOP/s", "frac": a1 / FP32_PEAK_FLOPS},
            "k_synth": {"bound": "alu", "achieved": a3 / 1e12, "peak": FP32_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                        "frac": a3 / FP32_PEAK_FLOPS, "terms_per_s": P * T * F / (ks * 1e-3)}}

    # end to end through the public API with host buffers: load (H2D) + synthesize to host (D2H)
    h2d = sum(np.ascontiguousarray(a).nbytes for a in (scene.bodies, scene.materials, scene.faces, scene.edges,
                                                       scene.tiles, paths.n_int, paths.types, paths.prims, paths.s0))
    Hh = torch.empty((T, F), dtype=torch.complex64, pin_memory=True)
    torch.cuda.synchronize()
    e2e_s = []
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        lk = ctx.load(scene, paths)
        lk.synthesize_H_host(tg, fg, drt.FP64, Hh)
        lk.unload()
        e2e_s.append(time.perf_counter() - t0)
    e2e_val = world * P * T * len(e2e_s) / sum(e2e_s)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "h_samples_per_s": world * T * F * args.steps / total_s,
            "config": {"workload": "canyon-512paths-2000x0.5ms-512bins-60GHz-fp64", "paths": P, "steps": T,
                       "bins": F, "fc_hz": fg.fc, "bandwidth_hz": fg.bandwidth, "precision": "DRT_FP64",
                       "l2": "flushed by a 256 MB write between timed steps (outside the events)",
                       "parallelism": f"{world} independent links, one per GPU"},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(T * F * 8),
                    "note": "drt_load_paths + drt_synthesize_H_host + drt_unload per step, wall clock"},
            "gpu_launches": int(kernel_launches),
            "kernel_ms": {k: (v[1] / args.steps) for k, v in prof.items() if v[0]},
            "kernel_ms_note": "device time per step of each kernel kind (all its launches)",
            "wall_s": wall, "clocks": clocks, "fp32_bulk": fp32_bulk}
    if FP64_FLOP_PER_PATH_STEP:
        achieved = FP64_FLOP_PER_PATH_STEP * P * T / k1_avg_s
        line["roofline"] = {"bound": "alu", "kernel": "k_extrapolate_fp64", "achieved": achieved / 1e12,
                            "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_FLOPS,
                            "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz (no FP64 figure in "
                                           "MEASURED_PEAKS.json)",
                            "algorithmic": f"{FP64_FLOP_PER_PATH_STEP:.0f} FP64 FLOP per path-step x {P * T} path-steps",
                            "traffic": K1_DRAM_BYTES_PER_LAUNCH,
                            "ncu_fp64_pipe_active": K1_FP64_PIPE_ACTIVE}
    else:
        line["roofline"] = {"bound": "alu", "kernel": "k_extrapolate_fp64", "achieved": None,
                            "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s", "frac": None,
                            "traffic": None, "note": "per-path-step FLOP count not yet measured"}
    probe = ctx.probe_peak(0)
    line["roofline"]["probe_fp64_tflops"] = probe / 1e12
    line["power_profiles"] = run_power(args, link, tg, fg, drt, flush)
    line["lifetime"] = run_lifetime(args, link, tg, fg, drt, flush)
    line["wideband"] = run_wideband(args, link, tg, fg, drt, flush)
    if args.batch_links > 0:
        line["batched"] = run_batched(args, ctx, drt, flush)
    if args.highway:
        line["highway"] = run_highway(args, ctx, drt, flush)
    if args.serve_seconds > 0:
        line["serving"] = run_serving(args, drt)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, paths, tg, fg, n_steps=tg.n_steps)
    link.unload()
    ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
