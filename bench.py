"""Benchmark of the patch-decomposed PIC hot path on GB300.

Workload: the 2D3V LWFA-shaped run, 2048 x 512 cells (dx = 0.125,
dy = 0.5 c/w0, dt = 0.95 CFL), 32 x 32-cell patches, 4 particles per cell
(4 194 304 electrons at t = 0) on immobile ions with a 200 c/w0 linear
ramp, Gaussian laser a0 = 2 (waist 20, 30/w0 FWHM) entering at x_min,
moving window at c from t = 128.  The run is first advanced `--spinup`
steps untimed (so the timed steps see the moving window and the wake, not
a cold plasma at rest), then W warm-up steps, then exactly K timed steps;
the defaults (1000 + 10 + 990) cover the workload's 2000 steps.

One JSON line is printed on rank 0:
  value        particle-steps/s over all ranks (FP32 path, the headline)
  fp64         the same for the FP64 path (its own run)
  fp32_float_current  the FP32 path with float shared-atomic current
               accumulation instead of the default 32-bit fixed point
  roofline     dominant kernel (the patch particle step): algorithmic bytes
               per launch / mean launch time (CUDA events on the launching
               stream) against the measured HBM copy bandwidth
  e2e          the same metric through the C-ABI from host buffers over
               the same K steps: the state after the spin-up restored from
               page-locked host memory (H2D), K steps, D2H of fields and
               particles, all inside the timed region
  lwfa3d       the 3D3V config (1024x256x256, 67 M electrons, FP32)
  batching     64 small runs batched (one launch per kernel per step) vs
               the same runs stepped one after the other
  serving      the served ensemble (FP32 runs of four grid sizes, Poisson
               arrivals at 70% of the measured capacity, continuous
               batching): p50/p99 latency from arrival, throughput
  precision_study  FP32 against FP64 from identical inputs over the
               workload's 2000 steps: field and energy differences, both
               paths' continuity and Gauss residuals
  cpu_baseline the FP64 CPU oracle on a bounded sample of the workload
`--impl reference` times the oracle alone (the reference arm).

Multi-GPU: the path is run as independent replicas (one per rank, no
collective on the data path); value = particles x steps of all ranks /
max-over-ranks time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (push+deposit+FDTD) FP32 vs FP64; p50/p99 served-run latency"
WORKLOAD = ("2D3V LWFA-shaped: 2048x512 cells, dx=0.125, dy=0.5 c/w0, dt=0.95 CFL, "
            "32x32-cell patches, 4 ppc (4194304 electrons), immobile ions, 200 c/w0 ramp, "
            "Gaussian laser a0=2 waist 20 tau 30, moving window at c")
L2_BYTES = 129e6


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _code_only(text):
    """Source text without comments, trailing blanks and blank lines: what
    the compiler sees, so that the digest of a kernel does not change when
    only its comments do.  String literals are copied as they are."""
    out, i, n = [], 0, len(text)
    while i < n:
        if text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text[i] == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(text[i])
            i += 1
    lines = [ln.rstrip() for ln in "".join(out).split("\n")]
    return "\n".join(ln for ln in lines if ln)


def source_digest(files):
    """sha256 of the listed kernel sources (repo-relative), comments
    stripped."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()


def _summary_matches(text):
    """True when an ncu summary's recorded digest equals the digest of its
    kernel sources as they are now."""
    import re
    m = re.search(r"sha256 `([0-9a-f]+)` of (.*)", text)
    if not m:
        return False
    return source_digest(re.findall(r"`([^`]+)`", m.group(2))).startswith(m.group(1))


def moved_bytes(r, hbm):
    """The roofline against the bytes the particle step had to move: the
    algorithmic bytes less those of the particles in skipped calm slots
    (11 s each: nothing read or written), over the same launch time."""
    calm = r.get("calm_per_step", 0.0)
    b = r["kernel_bytes"] - calm * 11 * r["rs"]
    ach = b / (r["particle_step_ms"] * 1e-3) / 1e9
    return {"bytes_per_launch": b, "calm_particles_per_launch": calm,
            "calm_share": calm / r["np"] if r["np"] else 0.0,
            "achieved": ach, "frac": ach / hbm}


def profiled_traffic(name):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    from the committed ncu summary profiles/<name>, if the kernel sources
    it names still hash to the value recorded at capture time; else None."""
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", name)).read()
        if not _summary_matches(text):
            return None
        t = re.search(r"traffic = DRAM read \+ write per launch \| (\d+) bytes", text)
        return int(t.group(1)) if t else None
    except Exception:
        return None


def profiled_value(name, key):
    """An integer recorded as `key` in the committed ncu summary
    profiles/<name>, if its kernel sources still hash to the recorded
    value; else None."""
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", name)).read()
        if not _summary_matches(text):
            return None
        v = re.search(r"`" + key + r"` (\d+)", text)
        return int(v.group(1)) if v else None
    except Exception:
        return None


def over_ranks(v, dist, device, op="max"):
    """v reduced over all ranks (max or sum); v itself on a single rank.
    device: where the collective's tensor lives ("cuda:k" under NCCL, "cpu"
    under gloo)."""
    if not dist:
        return float(v)
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_this_rank, ms_this_rank, dist, device):
    """Units processed by all ranks / the slowest rank's time, per second."""
    units = over_ranks(units_this_rank, dist, device, "sum")
    ms_max = over_ranks(ms_this_rank, dist, device, "max")
    return units / (ms_max / 1e3), ms_max


def algorithmic_bytes(npart, ncell, rsize):
    """Bytes the method must move once per step: per particle read
    x, y, ux, uy, uz, w and write x, y, ux, uy, uz (11 words); per cell gather
    E and Bm (6), write J once (3), Yee read E, B, J (9), write E, B, Bm (9)."""
    per_particle_step = 11 * rsize
    per_cell_step = 27 * rsize
    per_particle_kernel = 11 * rsize      # the particle step kernel alone
    per_cell_kernel = 9 * rsize           # gather E, Bm (6) + J written once (3)
    return (npart * per_particle_step + ncell * per_cell_step,
            npart * per_particle_kernel + ncell * per_cell_kernel)


def run_gpu(prec, steps, warmup, spinup, device, rank, world, dist, cf=2.0, merge=-1, sort=0,
            chunk=0, current_float=False, deterministic=False):
    import torch

    from paper_1912_04064_gb300 import pic
    from paper_1912_04064_gb300 import workloads as W

    run, parts = W.lwfa_2d()
    npart0 = parts["x"].size
    ncell = run["n"][0] * run["n"][1]
    rs = 4 if prec == "fp32" else 8
    stream = torch.cuda.Stream(device=device)
    cfg = pic.config_from_run(run, prec, stream=stream.cuda_stream, device=device,
                              use_graph=True, timing=False, capacity_factor=cf, merge=merge,
                              sort_every=sort, task_chunk=chunk,
                              current_float=current_float, deterministic=deterministic)
    g = pic.Pic(cfg)
    g.pic_load_particles(parts)
    g.pic_set_background("neutralising")
    # clocks sampled over the whole GPU leg (spin-up, warm-up and the timed
    # steps): the timed region alone is too short for nvidia-smi's interval
    with ClockSampler(device) as clk:
        g.pic_step(spinup)
        g.pic_step(warmup)
        d0 = g.pic_diag()
        blob = g.pic_snapshot()   # the per-kernel timing pass replays the same steps
        if dist:
            dist.barrier()
        torch.cuda.synchronize(device)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        g.pic_step(steps)
        ev1.record(stream)
        torch.cuda.synchronize(device)
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    d1 = g.pic_diag()
    # per-kernel times over the same steps (replayed from the snapshot taken
    # before the timed region), CUDA events around each phase on the
    # launching stream (no graph replay)
    cfg_t = pic.config_from_run(run, prec, stream=stream.cuda_stream, device=device,
                                use_graph=False, timing=True, capacity_factor=cf, merge=merge,
                                sort_every=sort, task_chunk=chunk,
                                current_float=current_float, deterministic=deterministic)
    g.close()
    gt = pic.Pic(cfg_t)
    gt.pic_restore(blob)
    t0 = gt.pic_diag()
    gt.pic_step(steps)
    t1 = gt.pic_diag()
    gt.close()
    np_mean = 0.5 * (d0["np"] + d1["np"])
    value, ms_max = whole_job_rate(np_mean * steps, ms, dist, f"cuda:{device}")
    step_bytes, k_bytes = algorithmic_bytes(np_mean, ncell, rs)
    ps_ms = (t1["ms_particles"] - t0["ms_particles"]) / steps
    fd_ms = (t1["ms_fields"] - t0["ms_fields"]) / steps
    return {
        "value": value,
        "ms_per_step": ms_max / steps,
        "np": np_mean, "np0": npart0, "ncell": ncell, "rs": rs,
        "step_bytes": step_bytes, "kernel_bytes": k_bytes,
        "particle_step_ms": ps_ms, "fields_ms": fd_ms,
        "window_ms": (t1["ms_window"] - t0["ms_window"]) / steps,
        "sort_ms": (t1["ms_sort"] - t0["ms_sort"]) / steps,
        # kernels of the timed steps: the diagnostics call after them launched
        # 5 reductions (+1 deposit when the continuity residual is available)
        "launches": d1["launches"] - d0["launches"] - (5 + (0 if math.isnan(d1["continuity"]) else 1)),
        "shifts": d1["shifts"], "t": d1["t"], "max_patch": d1["max_patch_count"],
        "capacity": d1["capacity"], "grows_in_timed_region": d1["grows"] - d0["grows"],
        "clocks": clk.summary(),
        "energy": {"U_E": d1["U_E"], "U_B": d1["U_B"], "U_K": d1["U_K"]},
        # particle-steps of the timed steps that the calm-slot skip did no
        # work for (particles at rest in zero fields whose copy was kept)
        "calm_per_step": (d1["calm_particle_steps"] - d0["calm_particle_steps"]) / steps,
    }


def run_gpu3(prec, steps, warmup, spinup, device, cf=2.0):
    """Config 3 (3D3V LWFA-shaped): 1024 x 256 x 256 cells, 16^3 patches,
    plasma of 0.005 n_c filling the upper half of the transverse box (2 ppc,
    67 108 864 electrons, filled on the device), laser a0 = 3 waist 15,
    moving window; `spinup` untimed steps, `warmup`, then `steps` timed
    steps (graph replay, CUDA events on the library's stream), then the same
    steps replayed from a fresh run with per-phase timers."""
    import torch

    from paper_1912_04064_gb300 import pic
    from paper_1912_04064_gb300 import workloads as W

    run = W.lwfa_3d()
    ncell = run["n"][0] * run["n"][1] * run["n"][2]
    rs = 4 if prec == "fp32" else 8
    stream = torch.cuda.Stream(device=device)
    # the config's 16^3 SDMD patches set the window step (16 cells); the GPU
    # stores particles in 8 x 8 x 8 sub-patches: a patch's E and Bm tile
    # (46 KB) and current tile (26 KB) fit three blocks per SM
    sub = (8, 8, 8)
    g = pic.Pic(pic.config_from_run(run, prec, stream=stream.cuda_stream, device=device,
                                    capacity_factor=cf, patch=sub))
    g.pic_load_plasma()
    g.pic_step(spinup + warmup)
    d0 = g.pic_diag()
    torch.cuda.synchronize(device)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    g.pic_step(steps)
    ev1.record(stream)
    torch.cuda.synchronize(device)
    ms = ev0.elapsed_time(ev1)
    d1 = g.pic_diag()
    g.close()
    gt = pic.Pic(pic.config_from_run(run, prec, stream=stream.cuda_stream, device=device,
                                     capacity_factor=cf, timing=True, patch=sub))
    gt.pic_load_plasma()
    gt.pic_step(spinup + warmup)
    t0 = gt.pic_diag()
    gt.pic_step(steps)
    t1 = gt.pic_diag()
    gt.close()
    np_mean = 0.5 * (d0["np"] + d1["np"])
    step_bytes = np_mean * 13 * rs + ncell * 27 * rs
    ps_ms = (t1["ms_particles"] - t0["ms_particles"]) / steps
    return {"value": np_mean * steps / (ms / 1e3), "ms_per_step": ms / steps, "np": np_mean,
            "cells": ncell, "step_bytes": step_bytes, "particle_step_ms": ps_ms,
            "fields_ms": (t1["ms_fields"] - t0["ms_fields"]) / steps,
            "kernel_bytes": np_mean * 13 * rs + ncell * 9 * rs,
            "launches": d1["launches"] - d0["launches"] - 5, "t": d1["t"]}


def run_e2e(prec, steps, device, spinup, cf=2.0):
    """Through the public C-ABI from host buffers, over the same steps as the
    device-timed region: the run's state after `spinup` steps (a pic_snapshot
    taken untimed, held in page-locked host memory) restored into a new
    context (H2D), `steps` steps, then E, B and every particle read back
    (D2H), all inside the timed region."""
    import ctypes

    import torch

    from paper_1912_04064_gb300 import pic
    from paper_1912_04064_gb300 import workloads as W

    run, parts = W.lwfa_2d()
    cfg = pic.config_from_run(run, prec, device=device, use_graph=True, capacity_factor=cf)
    g0 = pic.Pic(cfg)
    g0.pic_load_particles(parts)
    g0.pic_set_background("neutralising")
    g0.pic_step(spinup)
    blob = g0.pic_snapshot()
    n_at = g0.pic_diag()["np"]
    g0.close()
    pinned = lambda shape, dt=torch.float64: torch.empty(shape, dtype=dt).pin_memory().numpy()  # noqa: E731
    state = pinned((len(blob),), torch.uint8)
    state[:] = np.frombuffer(blob, dtype=np.uint8)
    del blob
    # page-locked result buffers, allocated before the timed region like the
    # input (the library reads and writes page-locked host memory in place)
    fields_out = {k: pinned(W.field_shape(run)) for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")}
    parts_out = pinned((6, n_at + n_at // 2))
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    g = pic.Pic(cfg)
    g._check(pic.lib().pic_restore(g.h, ctypes.c_void_p(state.ctypes.data), state.size))
    g.pic_step(steps)
    out = {}
    for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        out[k] = g.pic_get_field(k, out=fields_out[k])
    p = g.pic_get_particles(out=parts_out)
    t1 = time.perf_counter()
    n_mean = 0.5 * (n_at + p["x"].size)
    g.close()
    h2d = state.nbytes
    d2h = sum(v.nbytes for v in out.values()) + 6 * 8 * p["x"].size
    return {"value": n_mean * steps / (t1 - t0), "unit": "particle-steps/s",
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "seconds": t1 - t0, "steps": steps, "from_step": spinup}


def run_serving(device, seconds, seed=5, probe=16, load=0.7, cf=4.0, steps_per_tick=10):
    """The served ensemble (FP32): first `probe` requests submitted at once
    and run to completion give the service capacity (requests/s); then
    requests arrive as a Poisson process at `load` x that capacity for
    `seconds` and the server drains.  Latency = completion - arrival."""
    from paper_1912_04064_gb300 import pic
    from paper_1912_04064_gb300 import workloads as W

    def cfg_of(run):
        return pic.config_from_run(run, "fp32", device=device, capacity_factor=cf)

    srv = pic.Server(device=device, steps_per_tick=steps_per_tick)
    # capacity probe
    probe_reqs = W.served_requests(probe, seed)
    t0 = srv.pic_server_clock()
    ps0 = srv.pic_server_get_stats()["particle_steps"]
    for run, steps, _ in probe_reqs:
        srv.pic_server_submit(cfg_of(run), steps)
    while True:
        srv.pic_server_tick()
        st = srv.pic_server_get_stats()
        if st["done"] + st["failed"] >= probe:
            break
    t_probe = srv.pic_server_clock() - t0
    cap_rps = probe / t_probe
    cap_ps = (st["particle_steps"] - ps0) / t_probe
    # Poisson arrivals at load x capacity
    lam = load * cap_rps
    rng = np.random.default_rng(seed + 1)
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=int(lam * seconds * 3) + 10))
    arrivals = arrivals[arrivals < seconds]
    reqs = W.served_requests(arrivals.size, seed + 2)
    ids = []
    base_done = st["done"] + st["failed"]
    ps1 = st["particle_steps"]
    t_start = srv.pic_server_clock()
    i = 0
    running = []
    while True:
        now = srv.pic_server_clock() - t_start
        while i < arrivals.size and arrivals[i] <= now:
            run, steps, _ = reqs[i]
            ids.append(srv.pic_server_submit(cfg_of(run), steps))
            i += 1
        st = srv.pic_server_get_stats()
        if i == arrivals.size and st["done"] + st["failed"] - base_done >= arrivals.size:
            break
        if st["running"] == 0 and st["queued"] == 0:
            time.sleep(max(0.0, min(arrivals[i] - now, 0.05)))
            continue
        running.append(srv.pic_server_tick())
    t_end = srv.pic_server_clock() - t_start
    lat, failed = [], 0
    for k, rid in enumerate(ids):
        info = srv.pic_server_info(rid)
        if info["state"] != pic.PIC_REQ_DONE:
            failed += 1
            continue
        lat.append(info["t_done"] - t_start - arrivals[k])
    st = srv.pic_server_get_stats()
    srv.close()
    lat = np.array(lat)
    return {
        "workload": ("served ensemble, FP32: grids {256x256, 512x256, 1024x512, 2048x512} "
                     "(32x32 patches), 1-8 ppc, 0.001-0.02 n_c uniform or ramped, laser a0 "
                     "0.5-4 with moving window in half, 200-2000 steps; plasma filled on the "
                     "device at admission; Poisson arrivals"),
        "arrival_rate_per_s": lam, "load_vs_capacity": load,
        "capacity_runs_per_s": cap_rps, "capacity_particle_steps_per_s": cap_ps,
        "probe_requests": probe, "requests": int(arrivals.size), "failed": failed,
        "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
        "mean_s": float(lat.mean()) if lat.size else None,
        "throughput_particle_steps_per_s": (st["particle_steps"] - ps1) / t_end,
        "runs_per_s": (lat.size) / t_end, "window_s": t_end,
        "max_concurrent_runs": max(running) if running else 0,
        "mean_concurrent_runs": float(np.mean(running)) if running else 0.0,
        "steps_per_tick": steps_per_tick, "capacity_factor": cf,
    }


def run_batching(device, nruns=64, steps=100):
    """Many small runs (64 LWFA-shaped runs of 256 x 128 cells, 32 x 32
    patches, 4 ppc, laser, FP32; 131 072 electrons each, plasma filled on
    the device) advanced `steps` steps: one batch (one launch per kernel per
    step for all runs) against the same runs stepped one after the other.
    Device time with CUDA events on the batch / run streams."""
    import torch

    from paper_1912_04064_gb300 import pic
    from paper_1912_04064_gb300 import workloads as W

    def runs_for(stream):
        out = []
        for k in range(nruns):
            run = W.lwfa_run(n=(256, 128), patch=(32, 32), ppc=(2, 2), n0=0.005 + 0.0002 * k,
                             ramp=20.0, a0=1.0 + 0.02 * k, waist=8.0, tau=10.0)
            g = pic.Pic(pic.config_from_run(run, "fp32", stream=stream.cuda_stream,
                                            device=device, capacity_factor=4.0))
            g.pic_load_plasma()
            out.append(g)
        return out

    stream = torch.cuda.Stream(device=device)
    alone = runs_for(stream)
    for g in alone:
        g.pic_step(3)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for g in alone:
        g.pic_step(steps)
    e1.record(stream)
    torch.cuda.synchronize(device)
    ms_alone = e0.elapsed_time(e1)
    np_total = sum(g.pic_diag()["np"] for g in alone)
    launches_alone = sum(g.pic_diag()["launches"] for g in alone)
    for g in alone:
        g.close()
    batched = runs_for(stream)
    b = pic.Batch(stream=stream.cuda_stream, device=device)
    b.pic_batch_set(batched)
    b.pic_batch_step(3)
    d0 = b.pic_batch_get_diag()
    torch.cuda.synchronize(device)
    e0.record(stream)
    b.pic_batch_step(steps)
    e1.record(stream)
    torch.cuda.synchronize(device)
    ms_batch = e0.elapsed_time(e1)
    d1 = b.pic_batch_get_diag()
    b.close()
    for g in batched:
        g.close()
    return {"workload": f"{nruns} LWFA-shaped runs of 256x128 cells (32x32 patches, 4 ppc, laser, "
                        f"FP32), {steps} steps each, plasma filled on the device",
            "particles": np_total, "steps": steps,
            "batched_particle_steps_per_s": np_total * steps / (ms_batch * 1e-3),
            "alone_particle_steps_per_s": np_total * steps / (ms_alone * 1e-3),
            "speedup": ms_alone / ms_batch,
            "launches_per_batched_step": (d1["launches"] - d0["launches"]) / steps,
            "grid": d1["grid"]}


def run_precision(device, steps=2000, every=50):
    """The precision study on the LWFA workload: the FP32 and FP64 paths
    advanced side by side from identical inputs (same particles, t = 0) for
    `steps` steps.  Every `every` steps (and after steps 1 and 10) the FP32
    fields are compared with the FP64 ones (||a - b||_inf / ||b||_inf per
    component; worst of the E, B and J components), with the particle count,
    both paths' FP64 continuity and Gauss residuals and their energies.
    Accumulated differences, not single-step errors: the FP32 run is never
    reset to the FP64 state.  The FP32 path runs twice: with its default
    fixed-point current tile and with float shared-atomic accumulation
    (`float_current`), for comparison."""
    import torch

    from paper_1912_04064_gb300 import pic
    from paper_1912_04064_gb300 import workloads as W

    run, parts = W.lwfa_2d()
    stream = torch.cuda.Stream(device=device)
    ctx = {}
    for name, prec, cf in (("fp64", "fp64", False), ("fp32", "fp32", False),
                           ("fp32f", "fp32", True)):
        g = pic.Pic(pic.config_from_run(run, prec, stream=stream.cuda_stream, device=device,
                                        use_graph=True, capacity_factor=4.0, current_float=cf))
        g.pic_load_particles(parts)
        g.pic_set_background("neutralising")
        ctx[name] = g
    shape = ctx["fp64"].shape
    bufs = {p: torch.empty(shape, dtype=torch.float64, device=f"cuda:{device}") for p in ctx}
    groups = {"E": ("Ex", "Ey", "Ez"), "B": ("Bx", "By", "Bz"), "J": ("Jx", "Jy", "Jz")}
    marks = sorted({1, 10, *range(every, steps + 1, every)})
    hist = {"fp32": [], "fp32f": []}
    done = 0
    for m in marks:
        for g in ctx.values():
            g.pic_step(m - done)
        done = m
        recs = {v: {"step": m} for v in hist}
        for grp, names in groups.items():
            worst = {v: 0.0 for v in hist}
            for k in names:
                for p, g in ctx.items():
                    g.pic_get_field(k, out=bufs[p])
                torch.cuda.synchronize(device)
                ref = bufs["fp64"].abs().max().item()
                for v in hist:
                    diff = (bufs[v] - bufs["fp64"]).abs().max().item()
                    worst[v] = max(worst[v], diff / ref if ref > 0 else diff)
            for v in hist:
                recs[v][grp] = worst[v]
        d64 = ctx["fp64"].pic_diag()
        # residuals not available at this step (e.g. right after a window
        # shift) are reported as null
        fin = lambda x: x if math.isfinite(x) else None  # noqa: E731
        for v in hist:
            d32 = ctx[v].pic_diag()
            for k in ("U_E", "U_B", "U_K"):
                recs[v][k] = abs(d32[k] - d64[k]) / max(abs(d64[k]), 1e-300)
            recs[v]["np"] = (d32["np"], d64["np"])
            recs[v]["continuity"] = (fin(d32["continuity"]), fin(d64["continuity"]))
            recs[v]["gauss"] = (fin(d32["gauss"]), fin(d64["gauss"]))
            hist[v].append(recs[v])
    for g in ctx.values():
        g.close()
    pick = [m for m in (1, 10, 100, 500, 1000, 2000) if m in marks]

    def summary(h):
        def at(step):
            r = next(x for x in h if x["step"] == step)
            return {k: r[k] for k in ("E", "B", "J", "U_E", "U_B", "U_K")}
        last = h[-1]
        return {"at_step": {str(m): at(m) for m in pick},
                "max_over_run": {k: max(x[k] for x in h) for k in ("E", "B", "J", "U_E", "U_B", "U_K")},
                "particles_at_end": {"fp32": last["np"][0], "fp64": last["np"][1]},
                "continuity_at_end": {"fp32": last["continuity"][0], "fp64": last["continuity"][1]},
                "gauss_at_end": {"fp32": last["gauss"][0], "fp64": last["gauss"][1]},
                "gauss_max_over_run": {p: max((x["gauss"][i] for x in h if x["gauss"][i] is not None),
                                              default=None) for i, p in enumerate(("fp32", "fp64"))}}

    out = {"workload": "the LWFA workload above, FP32 and FP64 from identical inputs at t = 0, "
                       f"{steps} steps, recorded every {every}",
           "metric": "||fp32 - fp64||_inf / ||fp64||_inf per field component (worst of each "
                     "group); relative energy difference"}
    out.update(summary(hist["fp32"]))
    out["float_current"] = summary(hist["fp32f"])
    out["float_current"]["note"] = ("the same FP32 path with the current tile accumulated by float "
                                    "shared atomics (pic_config.current_float = 1)")
    return out


def cpu_oracle(steps, threads=0, spinup=0):
    """The FP64 CPU oracle on the same workload: advanced by itself from the
    initial state through `spinup` untimed steps (the phase the GPU arm
    times: wake formed, laser inside the plasma), one warm-up step, then
    `steps` timed steps."""
    from oracle.oracle import Oracle
    from paper_1912_04064_gb300 import workloads as W

    run, parts = W.lwfa_2d()
    o = Oracle(run, nthreads=threads)
    o.load(parts)
    o.set_background("neutralising")
    t_spin = time.perf_counter()
    if spinup > 0:
        o.step(spinup)
    t_spin = time.perf_counter() - t_spin
    o.step(1)  # warm-up
    n0 = o.diag()["np"]
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    n1 = o.diag()["np"]
    cores = threads or (os.cpu_count() or 1)
    where = f"after {spinup} untimed steps (the GPU arm's phase)" if spinup else "from t=0"
    return {"value": 0.5 * (n0 + n1) * steps / dt, "unit": "particle-steps/s", "cores": cores,
            "kind": "oracle", "seconds": dt, "spinup_seconds": t_spin,
            "sample": f"{steps} steps of the full 2048x512 LWFA-shaped workload {where} "
                      f"(and 1 warm-up step), FP64, OpenMP over patches"}


def issue_roofline(launch_ms):
    """Secondary ceiling of the FP32 particle step, which is bound by
    instruction issue: warp instructions of one launch (ncu, step 1005)
    over the mean launch time, against 152 SMs x 4 schedulers x the
    measured maximum SM clock."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = json.load(f)["sm_max_mhz"]
    except Exception:
        mhz = 2070.0
    n = profiled_value("particle_step_instruction_mix_lwfa2048.md", "warp_instructions_fp32")
    peak = 152 * 4 * mhz * 1e6
    if n is None or not launch_ms:
        return {"bound": "issue", "achieved": None, "peak": peak, "unit": "warp instructions/s"}
    ach = n / (launch_ms * 1e-3)
    return {"bound": "issue", "achieved": ach, "peak": peak, "unit": "warp instructions/s",
            "frac": ach / peak, "warp_instructions_per_launch": n,
            "source": "profiles/particle_step_instruction_mix_lwfa2048.md (one launch, step 1005)"}


def shared_atomic_ceiling(launch_ms):
    """Shared-atomic throughput of the FP32 deposit: the shared-atomic
    wavefronts of one particle-step launch (ncu, step 1005) over the mean
    launch time, against the measured rate of conflict-free 32-bit integer
    shared reductions on this GPU (0.91 warp operations per clock per SM,
    one wavefront each) at the maximum SM clock."""
    import re
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = json.load(f)["sm_max_mhz"]
    except Exception:
        mhz = 2070.0
    peak = 0.91 * 152 * mhz * 1e6
    out = {"achieved": None, "peak": peak, "unit": "shared-atomic wavefronts/s",
           "peak_source": "integer red.shared probe, 0.91 per clock per SM"}
    try:
        text = open(os.path.join(ROOT, "profiles", "particle_step_fp32_lwfa2048.md")).read()
        if not _summary_matches(text) or not launch_ms:
            return out
        w = int(re.search(r"mem_shared_op_atom\.sum`\) \| (\d+)", text).group(1))
    except Exception:
        return out
    ach = w / (launch_ms * 1e-3)
    out.update({"achieved": ach, "frac": ach / peak, "wavefronts_per_launch": w,
                "source": "profiles/particle_step_fp32_lwfa2048.md (one launch, step 1005)"})
    return out


def alu_roofline_fp64(launch_ms):
    """The FP64 particle step is bound by GB300's FP64 unit: FP64 flops of
    one launch (2 FMA + add + mul thread instructions, ncu, step 1005)
    over the mean launch time, against the nominal 1.25 TFLOP/s."""
    n = profiled_value("particle_step_instruction_mix_lwfa2048.md", "fp64_flops")
    peak = 1250.0
    if n is None or not launch_ms:
        return {"bound": "alu", "achieved": None, "peak": peak, "unit": "GFLOP/s"}
    ach = n / (launch_ms * 1e-3) / 1e9
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "GFLOP/s", "frac": ach / peak,
            "peak_source": "nominal FP64 rate (profiling recipe)", "flops_per_launch": n}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=990)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--spinup", type=int, default=1000)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=100)
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--task-chunk", type=int, default=0,
                    help="particles per work item of the particle step (0 = library default)")
    ap.add_argument("--sort-every", type=int, default=0,
                    help="re-order particles into the interleaved cell order every N steps")
    ap.add_argument("--merge", type=int, default=-1,
                    help="deposit merging in registers: 1 on, 0 off, -1 library default")
    ap.add_argument("--capacity-factor", type=float, default=4.0,
                    help="patch capacity / fullest initial patch")
    ap.add_argument("--serve-seconds", type=float, default=20.0,
                    help="arrival window of the served-ensemble measurement (0: skip)")
    ap.add_argument("--steps3d", type=int, default=40,
                    help="timed steps of the 3D3V config-3 leg (0: skip)")
    ap.add_argument("--float-current", type=int, default=1,
                    help="1: also time the FP32 path with float shared-atomic current accumulation")
    ap.add_argument("--precision-steps", type=int, default=2000,
                    help="steps of the FP32-vs-FP64 precision study (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=100,
                    help="steps of the batching comparison (0: skip)")
    ap.add_argument("--det-steps", type=int, default=20,
                    help="timed steps of the deterministic-mode legs, FP32 and FP64 (0: skip)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        from oracle.oracle import Oracle  # noqa: F401  (builds the oracle)
        w = max(0, min(args.warmup, 1))
        steps = max(1, min(args.steps, args.cpu_steps))
        cb = cpu_oracle(steps, spinup=args.spinup)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "particle-steps/s",
                "n_gpus": args.gpus, "steps": steps, "warmup": w,
                "ms_per_step": 1e3 * cb["seconds"] / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "arm": "FP64 CPU oracle, OpenMP over patches",
                           "bounded_sample": cb["sample"]},
                "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "e2e": {"value": cb["value"], "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0},
                "wall_s": time.perf_counter() - t0}
        print(json.dumps(line), flush=True)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
        dist = tdist
    torch.cuda.set_device(local)
    from paper_1912_04064_gb300 import build as pic_build
    if rank == 0:
        pic_build.build()
    if dist:
        dist.barrier()

    r32 = run_gpu("fp32", args.steps, args.warmup, args.spinup, local, rank, world, dist,
                  args.capacity_factor, args.merge, args.sort_every, args.task_chunk)
    r32f = None
    if args.float_current:
        r32f = run_gpu("fp32", args.steps, args.warmup, args.spinup, local, rank, world, dist,
                       args.capacity_factor, args.merge, args.sort_every, args.task_chunk,
                       current_float=True)
    r64 = None
    if args.fp64_steps > 0:
        r64 = run_gpu("fp64", args.fp64_steps, max(3, args.warmup // 2), args.spinup, local, rank,
                      world, dist, args.capacity_factor, -1, args.sort_every, args.task_chunk)
    dets = {}
    if args.det_steps > 0:
        for prec in ("fp32", "fp64"):
            dets[prec] = run_gpu(prec, args.det_steps, 3, args.spinup, local, rank, world, dist,
                                 args.capacity_factor, -1, 0, 0, deterministic=True)
    e2e = (None if args.no_e2e else
           run_e2e("fp32", args.steps, local, args.spinup + args.warmup, args.capacity_factor))
    serving = run_serving(local, args.serve_seconds) if args.serve_seconds > 0 else None
    r3 = (run_gpu3("fp32", args.steps3d, 3, max(0, 500 - args.steps3d - 3), local)
          if args.steps3d > 0 else None)
    batching = run_batching(local, steps=args.batch_steps) if args.batch_steps > 0 else None
    precision = (run_precision(local, args.precision_steps)
                 if rank == 0 and args.precision_steps > 0 else None)
    cpu = cpu_oracle(args.cpu_steps, spinup=args.spinup) if rank == 0 and args.cpu_steps > 0 else None
    cpu1 = cpu_oracle(1, threads=1) if rank == 0 and args.cpu_steps > 0 else None
    if dist:
        dist.barrier()
    if rank != 0:
        return
    hbm, src = peaks()
    k_gbs = r32["kernel_bytes"] / (r32["particle_step_ms"] * 1e-3) / 1e9
    step_gbs = r32["step_bytes"] / (r32["ms_per_step"] * 1e-3) / 1e9
    ws = r32["np0"] * 3 * 6 * r32["rs"] + r32["ncell"] * 15 * r32["rs"]
    line = {
        "metric": METRIC, "value": r32["value"], "unit": "particle-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r32["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "prec": "fp32 (patch-relative positions, FP32 shared-memory J)",
                   "particles_mean": r32["np"], "cells": r32["ncell"], "spinup_steps": args.spinup,
                   "t_end": r32["t"], "window_shifts": r32["shifts"],
                   "patch_capacity": r32["capacity"], "max_patch_count": r32["max_patch"],
                   "capacity_grows_in_timed_region": r32["grows_in_timed_region"],
                   "l2": f"no flush: working set {ws / 1e6:.0f} MB > {L2_BYTES / 1e6:.0f} MB L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "kernel": "particle_step (TMA staging, gather, Boris, "
                                                "Esirkepov, J reduction, re-binning)",
                     "achieved": k_gbs, "peak": hbm, "unit": "GB/s", "frac": k_gbs / hbm,
                     "peak_source": src,
                     "traffic": profiled_traffic("particle_step_fp32_lwfa2048.md"),
                     "traffic_source": "ncu capture of one launch at step 1005 "
                                       "(profiles/particle_step_fp32_lwfa2048.md); null when "
                                       "the kernel sources changed since",
                     "bytes_per_launch": r32["kernel_bytes"], "launch_ms": r32["particle_step_ms"],
                     "moved": moved_bytes(r32, hbm),
                     "whole_step": {"achieved": step_gbs, "frac": step_gbs / hbm,
                                    "bytes_per_step": r32["step_bytes"]},
                     "issue": issue_roofline(r32["particle_step_ms"]),
                     "shared_atomics": shared_atomic_ceiling(r32["particle_step_ms"])},
        "phases_ms": {"particle_step": r32["particle_step_ms"], "fields": r32["fields_ms"],
                      "window": r32["window_ms"], "sort": r32["sort_ms"]},
        "fp64": None if r64 is None else {
            "value": r64["value"], "ms_per_step": r64["ms_per_step"], "steps": args.fp64_steps,
            "particle_step_ms": r64["particle_step_ms"], "fields_ms": r64["fields_ms"],
            "speedup_fp32_over_fp64": r32["value"] / r64["value"],
            "hbm_frac_whole_step": r64["step_bytes"] / (r64["ms_per_step"] * 1e-3) / 1e9 / hbm,
            "roofline": alu_roofline_fp64(r64["particle_step_ms"])},
        "fp32_float_current": None if r32f is None else {
            "value": r32f["value"], "ms_per_step": r32f["ms_per_step"],
            "particle_step_ms": r32f["particle_step_ms"],
            "note": "the same FP32 path and steps with the shared current tile accumulated by "
                    "float atomics (pic_config.current_float = 1) instead of 32-bit fixed point"},
        "gpu_launches": r32["launches"],
        "clocks": r32["clocks"],
    }
    if e2e:
        line["e2e"] = {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")}
        line["e2e"]["note"] = (f"C-ABI from page-locked host buffers over the device-timed steps: "
                               f"pic_restore of the state after step {e2e['from_step']} (H2D), "
                               f"{e2e['steps']} steps, D2H of E, B and all particles; "
                               f"context creation inside the timed region")
    if dets:
        line["deterministic"] = {
            "note": "pic_config.deterministic = 1 (bitwise reproducible; fixed-order current "
                    "reduction, one work item per patch, FP64 tiles in 64-bit fixed point), same "
                    "workload and phase"}
        for prec, r in dets.items():
            base = r32 if prec == "fp32" else r64
            line["deterministic"][prec] = {
                "value": r["value"], "ms_per_step": r["ms_per_step"], "steps": args.det_steps,
                "particle_step_ms": r["particle_step_ms"], "fields_ms": r["fields_ms"],
                "ms_per_step_default_mode": None if base is None else base["ms_per_step"]}
    if serving:
        line["serving"] = serving
    if batching:
        line["batching"] = batching
    if precision:
        line["precision_study"] = precision
    if r3:
        line["lwfa3d"] = {
            "workload": ("3D3V LWFA-shaped: 1024x256x256 cells, dx=0.125, dy=dz=0.5 c/w0, "
                         "dt=0.95 CFL, 16^3-cell patches (window step 16 cells; stored as "
                         "8x8x8 GPU sub-patches), 0.005 n_c in the upper half of the "
                         "transverse box, 2 ppc (67108864 electrons), immobile ions, laser a0=3 "
                         "waist 15, moving window at c"),
            "dtype": "f32", "value": r3["value"], "unit": "particle-steps/s",
            "ms_per_step": r3["ms_per_step"], "steps": args.steps3d,
            "spinup_steps": max(0, 500 - args.steps3d - 3), "warmup": 3, "t_end": r3["t"],
            "note": "the timed steps are the last ones of the config's 500",
            "particle_step_ms": r3["particle_step_ms"], "fields_ms": r3["fields_ms"],
            "roofline": {"bound": "hbm", "peak": hbm, "unit": "GB/s",
                         "achieved_whole_step": r3["step_bytes"] / (r3["ms_per_step"] * 1e-3) / 1e9,
                         "frac_whole_step": r3["step_bytes"] / (r3["ms_per_step"] * 1e-3) / 1e9 / hbm,
                         "achieved_particle_step": r3["kernel_bytes"] / (r3["particle_step_ms"] * 1e-3) / 1e9,
                         "frac_particle_step": r3["kernel_bytes"] / (r3["particle_step_ms"] * 1e-3) / 1e9 / hbm,
                         "bytes_per_step": r3["step_bytes"]}}
    if cpu:
        line["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
        if cpu1:
            line["cpu_baseline"]["one_thread"] = {k: cpu1[k] for k in ("value", "cores", "sample")}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
