"""Benchmark of the planar WCSPH hydrodynamic-ram step on B300.

Workload: the 300 x 150 mm channel at dx = 0.2 mm (1,125,000 fluid particles,
3 ghost layers per wall, 5 mm disk entering at 900 m/s with tau = 200 us),
stepped from t = 0 (impact phase).  One "step" is one pass of the whole hot
path: drift, counting sort, ghosts, fused interaction pass, probes and the CFL
gate, replayed from a CUDA graph.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  With --gpus N > 1 (launched by torchrun) every rank runs
an independent replica of the case (the path does not shard across GPUs), and
the value is the aggregate particle-steps/s over all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import casegen  # noqa: E402

METRIC = "particle-steps/s at 1M particles"
UNIT = "particle-steps/s"
DX = 2e-4
ALG_BYTES_PER_PARTICLE = 40      # {x, y, vx, vy, rho} read and written once
# algorithmic FP32 work of the interaction pass per particle-step: about 20
# interacting neighbours x ~70 flop of pair terms plus ~61 candidates x ~6
# flop of the support predicate (FMA counted as 2)
FLOP_PER_PARTICLE = 1700
FLOP_PER_PAIR = 58               # the pair terms alone, as the pass forms them
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "k_pass_channel300x150_dx0.2mm_traffic.txt")


def workload(dx=DX, Lx=None):
    p = casegen.config_scaling(dx)
    if Lx is not None:
        p["Lx"] = Lx
    xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], p["jitter"], p["seed"],
                               disk=(p["x_c0"], p["y_c0"], p["R_disk"]))
    return p, xy.astype(np.float32)


def workload_config(dx=DX, world=1):
    """The workload's description, the same on both arms of the benchmark."""
    p = casegen.config_scaling(dx)
    n = casegen.n_lattice(p["Lx"], p["W"], dx)
    return {"workload": "300 x 150 mm water channel, dx = %g mm, %d fluid particles, 5 mm disk "
                        "entering at 900 m/s, impact phase from t = 0" % (dx * 1e3, n),
            "particles": n, "dx_mm": dx * 1e3,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "256 MB buffer written between timed steps"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def fp32_peak_tflops(sm_mhz, sms, lanes=128):
    """FP32 peak from unit counts: SMs x FP32 lanes x 2 flop (FMA) x clock.
    sms is the device's multiprocessor count as the CUDA runtime reports it."""
    return sms * lanes * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.1)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[4:8]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def read_traffic(src_hash):
    """dram bytes per launch of k_pass from the committed ncu summary, or None
    when the kernel source changed since the counters were taken."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None
    vals = {}
    with open(PROFILE_TRAFFIC) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha1") != src_hash:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def kernel_source_hash():
    """sha1 of the kernel source without its comments and blank lines, so that
    the committed ncu traffic stays valid across edits of the comments only."""
    with open(os.path.join(ROOT, "paper_2609_05494_b300", "csrc", "hram_device.cuh")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    lines = [ln.split("//", 1)[0].rstrip() for ln in src.splitlines()]
    return hashlib.sha1("\n".join(ln for ln in lines if ln.strip()).encode()).hexdigest()


def max_over_ranks(total_ms, dist=None):
    """The timed region's duration as the maximum over ranks (every rank runs
    its own replica; the job is done when the slowest one is)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(total_ms)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world, particles, steps, total_ms):
    """Whole-job particle-steps/s: all ranks' particle-steps over the slowest rank's time."""
    return world * particles * steps / (total_ms * 1e-3)


def shard(items, rank, world):
    """Cases of an independent sweep split across ranks (no collective needed)."""
    return list(items)[rank::world]


def batch_steps_benchmark(stream, steps, n_cases=64):
    """The 64-case sweep as one batch (default cell grids and schedule), the
    first `steps` batched steps timed with CUDA events: for profiling the
    batched kernels alone."""
    import torch
    from paper_2609_05494_b300 import Batch, Case
    specs = []
    for p in casegen.sweep_draws(casegen.DEFAULT_SEED, n_cases):
        xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], p["jitter"], p["seed"],
                                   disk=(p["x_c0"], p["y_c0"], p["R_disk"]))
        specs.append((p, xy.astype(np.float32)))
    cases = [Case(p, xy, stream=stream) for p, xy in specs]
    with Batch(cases, 1.0, stream=stream) as b:      # no case reaches t = 1 s here
        b.run(max_steps=3)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            b.step()
        e.record(stream)
        e.synchronize()
        ms = a.elapsed_time(e) / steps
    n = sum(xy.shape[0] for _, xy in specs)
    for c in cases:
        c.close()
    return {"cases": n_cases, "particles": n, "steps": steps, "ms_per_batched_step": ms,
            "particle_steps_per_s": n / (ms * 1e-3)}


def sweep_benchmark(stream, rank=0, world=1, dist=None, n_cases=64, t_end=0.5e-3):
    """The batched coefficient sweep: n_cases cases from casegen.sweep_draws
    (alpha, c0, cutoff, v0, width; dx = 1 mm), each run to t_end, first one
    after another (each its own graph replays), then all together in one
    batch.  Wall-clock time of each, max over ranks for N > 1."""
    import torch
    from paper_2609_05494_b300 import Batch, Case, autotune
    specs = []
    for p in shard(casegen.sweep_draws(casegen.DEFAULT_SEED, n_cases), rank, world):
        xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], p["jitter"], p["seed"],
                                   disk=(p["x_c0"], p["y_c0"], p["R_disk"]))
        specs.append((p, xy.astype(np.float32)))
    # per-case cell grids and the batch's block schedule, picked by timing
    t0 = time.perf_counter()
    specs, schedule, tune_report = autotune.tune_sweep(specs, stream=stream)
    t_tune = time.perf_counter() - t0
    serial = [Case(p, xy, stream=stream) for p, xy in specs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps_serial = 0
    for c in serial:
        c.run(0, t_end)
        steps_serial += int(c.scalars()["step"])
    torch.cuda.synchronize()
    t_serial = time.perf_counter() - t0
    batched = [Case(p, xy, stream=stream) for p, xy in specs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with Batch(batched, t_end, stream=stream, schedule=schedule) as b:
        b.run()
        n_batched_steps = b.steps
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    same = all(np.array_equal(a.probe_pressure(), g.probe_pressure()) for a, g in
               zip(serial[:4], batched[:4]))
    # the same sweep as one persistent launch, block counts per case autotuned
    t0 = time.perf_counter()
    blocks, ptune = autotune.tune_persistent(specs, t_end, stream=stream)
    t_ptune = time.perf_counter() - t0
    # (the persistent kernel takes the 3 x 3 stencil: cases tuned to the 5 x 5
    # one run on cells of side 2h there, and are not compared bit for bit)
    pspecs = [(dict(p, cell_factor=max(float(p["cell_factor"]), 1.001)), xy) for p, xy in specs]
    persist = [Case(p, xy, stream=stream) for p, xy in pspecs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with Batch(persist, t_end, stream=stream, persistent=True, case_blocks=blocks) as b:
        b.run()
    torch.cuda.synchronize()
    t_persist = time.perf_counter() - t0
    same_p = all(np.array_equal(a.probe_pressure(), g.probe_pressure()) and
                 np.array_equal(a.get_state()["xy"], g.get_state()["xy"])
                 for a, g, (p, _), (q, _) in zip(serial, persist, specs, pspecs)
                 if p["cell_factor"] == q["cell_factor"])
    particles = sum(xy.shape[0] for _, xy in specs)
    t_serial = max_over_ranks(t_serial * 1e3, dist) * 1e-3
    t_batch = max_over_ranks(t_batch * 1e3, dist) * 1e-3
    t_persist = max_over_ranks(t_persist * 1e3, dist) * 1e-3
    for c in serial + batched + persist:
        c.close()
    return {"cases": n_cases, "cases_per_rank": len(specs), "t_end_s": t_end,
            "particles": particles, "serial_s": t_serial, "batched_s": t_batch,
            "speedup": t_serial / t_batch, "case_steps": steps_serial,
            "batched_launch_steps": n_batched_steps, "batched_equals_serial": bool(same),
            "persistent_s": t_persist, "persistent_speedup": t_serial / t_persist,
            "persistent_over_batched": t_batch / t_persist,
            "persistent_equals_serial": bool(same_p),
            "persistent_blocks": {"min": int(blocks.min()), "max": int(blocks.max()),
                                  "total": int(blocks.sum())},
            "persistent_autotune": ptune, "persistent_autotune_s": t_ptune,
            "autotune": tune_report, "autotune_s": t_tune}


def pass_variant_benchmark(stream, xy, p, flush, steps=50):
    """A/B of the interaction pass on the headline workload: candidates read
    through the read-only path from global memory (the default), their
    positions staged in shared memory (HR_FLAG_STAGE_POS), their whole
    records staged (HR_FLAG_STAGE_ALL), cells of side h with the 5 x 5
    stencil (cell_factor 0.5), and every fluid pair evaluated once
    (HR_FLAG_NEWTON3).  Each variant: the same flushed-L2 steps from
    t = 0, the kernel groups timed by the in-graph events.  The staged
    variants' end states are compared bit for bit with the default's; the
    5 x 5 stencil and the Newton-3 pass sum the same neighbours in another
    order, so their density is compared to rounding."""
    import torch
    from paper_2609_05494_b300 import Case
    out, ref = {}, None
    variants = (("global", 0, p, False), ("stage_pos", 1, p, False), ("stage_all", 2, p, False),
                ("cells_h_5x5", 0, dict(p, cell_factor=0.5), False), ("newton3", 0, p, True))
    for name, stage, q, n3 in variants:
        with torch.cuda.stream(stream):
            c = Case(q, xy, stream=stream, timing=True, stage=stage, newton3=n3,
                     probe_capacity=steps + 16)
        c.run(5)
        c.sync()
        gs = {}
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                c.step()
            stream.synchronize()
            for g, v in c.kernel_times().items():
                gs.setdefault(g, []).append(v)
        st = c.get_state()
        c.close()
        out[name] = {g + "_us": 1e3 * statistics.mean(v) for g, v in gs.items()}
        out[name]["step_us"] = sum(out[name].values())
        if ref is None:
            ref = st
        elif stage:
            out[name]["bitwise_equal"] = all(np.array_equal(ref[k], st[k]) for k in ref)
        else:
            out[name]["rho_max_rel_diff"] = float(np.abs(st["rho"] / ref["rho"] - 1.0).max())
    out["steps"] = steps
    return out


def close_benchmark(stream, flush, big_xy, big_p, steps=60, blocks=3, warmup=5):
    """A/B of the step close: inside each step's own graph
    (HR_FLAG_CLOSE_INLINE) against the default, deferred to the next step's
    graph beside its drift.  ms per step of the graphs without timing events
    (L2 flushed before every step; the two forms in alternating blocks of
    steps/blocks steps), and whether the end states and scalars are equal
    bit for bit."""
    import torch
    from paper_2609_05494_b300 import Case
    p1, xy1 = workload(1e-3)
    out = []
    for name, q, x in (("300 x 150 mm, dx = 1 mm", p1, xy1),
                       ("300 x 150 mm, dx = 0.2 mm", big_p, big_xy)):
        with torch.cuda.stream(stream):
            forms = {"inline": Case(q, x, stream=stream, close_inline=True,
                                    probe_capacity=steps + warmup + 8),
                     "deferred": Case(q, x, stream=stream, probe_capacity=steps + warmup + 8)}
        for c in forms.values():
            c.run(warmup)
        torch.cuda.synchronize()
        ms = {k: 0.0 for k in forms}
        per = steps // blocks
        for _ in range(blocks):
            for key, c in forms.items():
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(per)]
                for k in range(per):
                    with torch.cuda.stream(stream):
                        flush.fill_(k & 0xFF)
                        ev[k][0].record(stream)
                        c.step()
                        ev[k][1].record(stream)
                torch.cuda.synchronize()
                ms[key] += sum(a.elapsed_time(b) for a, b in ev)
        sa, sb = forms["inline"].get_state(), forms["deferred"].get_state()
        equal = (all(np.array_equal(sa[k], sb[k]) for k in sa) and
                 forms["inline"].scalars() == forms["deferred"].scalars())
        for c in forms.values():
            c.close()
        out.append({"case": name, "particles": int(x.shape[0]),
                    "inline_ms_per_step": ms["inline"] / (per * blocks),
                    "deferred_ms_per_step": ms["deferred"] / (per * blocks),
                    "bitwise_equal": equal})
    return out


def tangent_benchmark(stream, big_xy=None, big_p=None, big_steps=20):
    """Cost of the tangent-linear mode (derivatives of the peak probe pressure
    and the wall impulse along alpha, c0, tau): the 22,500-particle fixed-dt
    workload run for its 400 steps with and without HR_FLAG_TANGENT, and a few
    steps of the 1.125M-particle workload (fixed dt) both ways.  CUDA events on
    the case's stream around hr_run."""
    import torch
    from paper_2609_05494_b300 import Case

    def timed(p, xy, steps, tangent):
        with torch.cuda.stream(stream):
            c = Case(p, xy, stream=stream, tangent=tangent, probe_capacity=steps + 8)
        c.run(3)
        c.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c.run(steps)
        b.record(stream)
        c.sync()
        ms = a.elapsed_time(b)
        out = c.tangent_outputs() if tangent else None
        c.close()
        return ms, out

    p = casegen.config_adjoint()
    xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], p["jitter"], p["seed"],
                               disk=(p["x_c0"], p["y_c0"], p["R_disk"])).astype(np.float32)
    steps = int(p["n_steps"])
    f_ms, _ = timed(p, xy, steps, False)
    t_ms, out = timed(p, xy, steps, True)
    res = {"workload": "150 x 150 mm, dx = 1 mm, %d particles, %d steps, fixed dt"
                       % (xy.shape[0], steps),
           "forward_ms_per_step": f_ms / steps, "tangent_ms_per_step": t_ms / steps,
           "tangent_over_forward": t_ms / f_ms,
           "gradients_per_s": 1e3 / t_ms,
           "peak_Pa": out["peak"], "dpeak_dln": out["dpeak"].tolist(),
           "impulse": out["impulse"], "dimpulse_dln": out["dimpulse"].tolist()}
    if big_xy is not None:
        q = dict(big_p)
        q["dt_mode"] = 1
        f_ms, _ = timed(q, big_xy, big_steps, False)
        t_ms, _ = timed(q, big_xy, big_steps, True)
        res["large"] = {"particles": int(big_xy.shape[0]), "steps": big_steps,
                        "forward_ms_per_step": f_ms / big_steps,
                        "tangent_ms_per_step": t_ms / big_steps,
                        "tangent_over_forward": t_ms / f_ms}
    return res


def adjoint_benchmark(stream, big_xy=None, big_p=None, big_steps=20, every=20):
    """Cost of the reverse mode (hr_adjoint_forward + hr_adjoint_backward: the
    run with a checkpoint every `every` steps, then the reverse sweep that
    recomputes each segment) against the plain run of the same steps, on the
    22,500-particle fixed-dt workload (400 steps) and on a few steps of the
    1.125M-particle workload.  CUDA events on the case's stream."""
    import torch
    from paper_2609_05494_b300 import Case

    def timed(p, xy, steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(stream):
            plain = Case(p, xy, stream=stream, probe_capacity=steps + 8)
            adj = Case(p, xy, stream=stream, probe_capacity=steps + 8)
        torch.cuda.synchronize()
        ev[0].record(stream)
        plain.run(steps)
        ev[1].record(stream)
        plain.sync()
        ev[2].record(stream)
        y = adj.adjoint_forward(steps, every)
        g = adj.adjoint_backward()
        ev[3].record(stream)
        torch.cuda.synchronize()
        f_ms, a_ms = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
        plain.close()
        adj.close()
        return f_ms, a_ms, y, g

    p = casegen.config_adjoint()
    xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], p["jitter"], p["seed"],
                               disk=(p["x_c0"], p["y_c0"], p["R_disk"])).astype(np.float32)
    steps = int(p["n_steps"])
    timed(p, xy, 40)   # warm-up of the code paths
    f_ms, a_ms, y, g = timed(p, xy, steps)
    res = {"workload": "150 x 150 mm, dx = 1 mm, %d particles, %d steps, fixed dt, a checkpoint "
                       "every %d steps" % (xy.shape[0], steps, every),
           "forward_ms_per_step": f_ms / steps, "adjoint_ms_per_step": a_ms / steps,
           "adjoint_over_forward": a_ms / f_ms, "gradients_per_s": 1e3 / a_ms,
           "peak_Pa": y["peak"], "dpeak_dln": g["dpeak"].tolist(),
           "impulse": y["impulse"], "dimpulse_dln": g["dimpulse"].tolist()}
    if big_xy is not None:
        q = dict(big_p)
        q["dt_mode"] = 1
        f_ms, a_ms, _, _ = timed(q, big_xy, big_steps)
        res["large"] = {"particles": int(big_xy.shape[0]), "steps": big_steps,
                        "forward_ms_per_step": f_ms / big_steps,
                        "adjoint_ms_per_step": a_ms / big_steps,
                        "adjoint_over_forward": a_ms / f_ms}
    return res


def scaling_benchmark(stream, flush, dxs=(1e-3, 5e-4, 2.5e-4, 2e-4, 1e-4), steps=30, warmup=5):
    """The scaling sweep of the same channel at spacing dx (45,000 to 4.5M
    particles): ms per step (L2 flushed between steps, graph without timing
    events), particle-steps/s, and the algorithmic HBM rate of the whole step
    (40 B per particle-step)."""
    import torch
    from paper_2609_05494_b300 import Case
    out = []
    for dx in dxs:
        p, xy = workload(dx)
        with torch.cuda.stream(stream):
            c = Case(p, xy, stream=stream, probe_capacity=steps + warmup + 8)
        c.run(warmup)
        c.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
                c.step()
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        n = xy.shape[0]
        out.append({"dx_mm": dx * 1e3, "particles": n, "ms_per_step": ms,
                    "particle_steps_per_s": n / (ms * 1e-3),
                    "alg_hbm_gbs": ALG_BYTES_PER_PARTICLE * n / (ms * 1e-3) / 1e9,
                    "status": c.sync()})
        c.close()
    return out


def small_case_benchmark(stream, flush, steps=50, warmup=5):
    """Small, latency-bound cases with the pass split over 1, 2 or 4 lanes
    per particle (HR_FLAG_PASS_LANES2 / _LANES4): ms per step (graph without
    timing events, L2 flushed between steps) and the pass's own duration
    (in-graph events, a second case).  The 1,000-particle patch is this
    step's floor: seven kernels of one short wave each."""
    import torch
    from paper_2609_05494_b300 import Case
    cases = []
    p, xy = workload(1e-3)
    q = dict(p, Lx=0.04, W=0.025)
    cases.append(("patch 40 x 25 mm, dx = 1 mm", q, casegen.fluid_lattice(
        q["Lx"], q["W"], q["dx"], q["jitter"], q["seed"],
        disk=(q["x_c0"], q["y_c0"], q["R_disk"])).astype(np.float32)))
    q = casegen.config_adjoint()
    cases.append(("150 x 150 mm, dx = 1 mm", q, casegen.fluid_lattice(
        q["Lx"], q["W"], q["dx"], q["jitter"], q["seed"],
        disk=(q["x_c0"], q["y_c0"], q["R_disk"])).astype(np.float32)))
    cases.append(("300 x 150 mm, dx = 1 mm", p, xy))
    p5, xy5 = workload(5e-4)
    cases.append(("300 x 150 mm, dx = 0.5 mm", p5, xy5))
    out = []
    for name, q, x in cases:
        row = {"case": name, "particles": int(x.shape[0])}
        for lanes in (1, 2, 4):
            with torch.cuda.stream(stream):
                c = Case(q, x, stream=stream, lanes=lanes, probe_capacity=steps + warmup + 8)
                t = Case(q, x, stream=stream, lanes=lanes, timing=True,
                         probe_capacity=steps + warmup + 8)
            c.run(warmup)
            t.run(warmup)
            c.sync()
            t.sync()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            pt = []
            for k in range(steps):
                with torch.cuda.stream(stream):
                    flush.fill_(k & 0xFF)
                    ev[k][0].record(stream)
                    c.step()
                    ev[k][1].record(stream)
                    flush.fill_(k & 0xFF)
                    t.step()
                stream.synchronize()
                pt.append(t.kernel_times()["pass"])
            torch.cuda.synchronize()
            row["lanes%d_ms_per_step" % lanes] = sum(a.elapsed_time(b) for a, b in ev) / steps
            row["lanes%d_pass_us" % lanes] = 1e3 * statistics.mean(pt)
            c.close()
            t.close()
        out.append(row)
    return out


def production_benchmark(stream):
    """The production runs: 300 x 150 mm at dx = 0.5 mm (180,000 particles),
    1 ms of simulated time at v0 = 900 and 600 m/s; wall clock of the whole
    run (hr_run to t_end, synchronised) and the four wall probes' peaks."""
    import torch
    from paper_2609_05494_b300 import Case
    out = []
    for v0 in (900.0, 600.0):
        p = casegen.config_production(v0)
        xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], p["jitter"], p["seed"],
                                   disk=(p["x_c0"], p["y_c0"], p["R_disk"])).astype(np.float32)
        with torch.cuda.stream(stream):
            c = Case(p, xy, stream=stream, probe_capacity=1 << 16)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = c.run(0, p["t_end"])
        c.sync()
        wall = time.perf_counter() - t0
        steps = int(c.scalars()["step"])
        pr = c.probe_pressure()
        d = c.diagnostics()
        c.close()
        out.append({"v0": v0, "particles": int(xy.shape[0]), "t_end_s": p["t_end"],
                    "steps": steps, "wall_s": wall, "ms_per_step": 1e3 * wall / steps,
                    "probe_peaks_MPa": [float(x) * 1e-6 for x in pr.max(axis=0)],
                    "wall_impulse": d["wall_impulse"], "status": st})
    return out


def paper_event_benchmark(stream):
    """The paper's own set-up and closure (750 x 150 mm, cubic spline,
    summation density, Mie-Grueneisen water, drag law, centreline probes PTn
    and PTf) through its whole 150 us event: the production run (dx = 1.5 mm,
    alpha 0.03, 900 m/s; the paper times it at about 14 s on a TITAN RTX,
    Section "Speed"), the resolution sweep dx = 2.0 / 1.5 / 1.0 mm and the
    alpha sweep 0.01-0.10 at 900 and 600 m/s (Tables tab:convergence and
    tab:alpha-sweep, whose peaks are listed beside ours for magnitude only: a
    planar model's peaks are not parity targets).  Wall clock from the first
    step to the synchronised end."""
    import torch
    from paper_2609_05494_b300 import Batch, Case

    def setup(dx, alpha, v0):
        p = casegen.config_paper(v0)
        p.update(dx=float(dx), alpha=float(alpha))
        xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], p["jitter"], p["seed"],
                                   disk=(p["x_c0"], p["y_c0"], p["R_disk"])).astype(np.float32)
        return p, xy

    def event(dx, alpha, v0, lanes=1):
        p, xy = setup(dx, alpha, v0)
        with torch.cuda.stream(stream):
            c = Case(p, xy, stream=stream, lanes=lanes)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = c.run(0, p["t_end"])
        c.sync()
        wall = time.perf_counter() - t0
        steps = int(c.scalars()["step"])
        pr = c.probe_pressure()
        c.close()
        return {"dx_mm": dx * 1e3, "alpha": alpha, "v0": v0, "particles": int(xy.shape[0]),
                "steps": steps, "wall_s": wall, "ms_per_step": 1e3 * wall / steps,
                "ptn_peak_MPa": float(pr[:, 0].max()) * 1e-6,
                "ptf_peak_MPa": float(pr[:, 1].max()) * 1e-6, "status": st}

    main = event(1.5e-3, 0.03, 900.0)
    main.update(particle_steps_per_s=main["particles"] * main["steps"] / main["wall_s"],
                paper_wall_s_titan_rtx=14.0)
    # the same event with the pass on four lanes per particle (a small,
    # latency-bound case; its sums differ from the one-lane run's in order)
    l4 = event(1.5e-3, 0.03, 900.0, lanes=4)
    main["lanes4"] = {k: l4[k] for k in ("steps", "wall_s", "ms_per_step", "ptn_peak_MPa",
                                         "ptf_peak_MPa", "status")}
    # the paper's printed peaks (MPa) for the same runs
    paper_res = {2.0: (785.8, 658.0), 1.5: (850.3, 714.9), 1.0: (830.5, 737.5)}
    paper_alpha = {(900.0, 0.01): 855.7, (900.0, 0.03): 850.3, (900.0, 0.06): 893.7,
                   (900.0, 0.10): 871.9, (600.0, 0.01): 429.7, (600.0, 0.03): 446.0,
                   (600.0, 0.06): 371.4, (600.0, 0.10): 367.1}
    res = []
    for dx in (2.0e-3, 1.5e-3, 1.0e-3):
        r = main if dx == 1.5e-3 else event(dx, 0.03, 900.0)
        res.append({k: r[k] for k in ("dx_mm", "particles", "steps", "wall_s", "ptn_peak_MPa",
                                      "ptf_peak_MPa")})
        res[-1]["paper_ptn_MPa"], res[-1]["paper_ptf_MPa"] = paper_res[round(dx * 1e3, 1)]
    alph = []
    for v0 in (900.0, 600.0):
        for a in (0.01, 0.03, 0.06, 0.10):
            r = main if (v0 == 900.0 and a == 0.03) else event(1.5e-3, a, v0)
            alph.append({"v0": v0, "alpha": a, "ptn_peak_MPa": r["ptn_peak_MPa"],
                         "paper_ptn_MPa": paper_alpha[(v0, a)], "wall_s": r["wall_s"]})
    # the same eight alpha-sweep events as one batch (one launch per kernel
    # per step for all eight); the batched peaks must equal the lone runs'
    cases = []
    with torch.cuda.stream(stream):
        for r in alph:
            p, xy = setup(1.5e-3, r["alpha"], r["v0"])
            cases.append(Case(p, xy, stream=stream))
        b = Batch(cases, casegen.config_paper(900.0)["t_end"], stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = b.run()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    same = all(float(c.probe_pressure()[:, 0].max()) * 1e-6 == r["ptn_peak_MPa"]
               for c, r in zip(cases, alph))
    b.close()
    for c in cases:
        c.close()
    main["resolution"] = res
    main["alpha_sweep"] = alph
    lone = sum(r["wall_s"] for r in alph)
    main["alpha_sweep_batched"] = {"cases": len(alph), "wall_s": wall, "lone_wall_s": lone,
                                   "speedup": lone / wall, "peaks_identical": bool(same),
                                   "status": st}
    main["workload"] = ("paper set-up: 750 x 150 mm, dx = 1.5 mm, %d particles, 900 m/s, "
                        "closure 1, 150 us" % main["particles"])
    return main


def cpu_model():
    """The host CPU's model name (first 'model name' line of /proc/cpuinfo)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - not Linux
        return os.cpu_count() or 1


def _oracle_sample(args):
    """One host thread: the oracle on the first Lx of the channel for about
    `seconds` of stepping; returns (particles, steps, seconds, set-up seconds)."""
    seconds, Lx = args
    import oracle
    p, xy = workload(DX, Lx=Lx)
    t0 = time.perf_counter()
    o = oracle.OracleCase(p, xy.astype(np.float64))
    t1 = time.perf_counter()
    steps = 0
    while True:
        o.step()
        steps += 1
        if time.perf_counter() - t1 >= seconds:
            break
    return xy.shape[0], steps, time.perf_counter() - t1, t1 - t0


def _oracle_config_runs():
    """The oracle as it stands, one thread, on the two small workloads run in
    full: the 150 x 150 mm parity case (dx = 2 mm, 250 steps) and the
    22,500-particle derivative workload (dx = 1 mm, 400 steps, fixed dt)."""
    import oracle
    out = {}
    for name, p in (("parity_150x150_dx2mm_250_steps", casegen.config_parity()),
                    ("adjoint_150x150_dx1mm_400_steps", casegen.config_adjoint())):
        xy = casegen.fluid_lattice(p["Lx"], p["W"], p["dx"], p["jitter"], p["seed"],
                                   disk=(p["x_c0"], p["y_c0"], p["R_disk"])).astype(np.float32)
        o = oracle.OracleCase(p, xy.astype(np.float64))
        n = int(p["n_steps"])
        t0 = time.perf_counter()
        o.run(n)
        el = time.perf_counter() - t0
        out[name] = {"particles": int(xy.shape[0]), "steps": n, "seconds": el,
                     "particle_steps_per_s": xy.shape[0] * n / el}
    return out


def cpu_baseline(seconds=10.0, Lx=0.075):
    """The FP64 oracle as it stands on a bounded sample of the workload (the
    first Lx of the channel at the same spacing, from t = 0), timed on the
    host cores two ways: one thread, and one independent copy of the sample
    per host core at once (a process pool started with spawn), the
    aggregate particle-steps/s of all copies over the slowest copy's time.
    The oracle itself is single-threaded; the second leg is how it uses every
    core without being changed."""
    import multiprocessing as mp
    import oracle
    oracle.build()   # once, before the pool
    n, steps, el, setup = _oracle_sample((seconds, Lx))
    single = n * steps / el
    cores = min(host_cores(), 64)   # bounded: each copy holds its own oracle case
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_sample, [(seconds, Lx)] * cores)
    all_steps = sum(r[1] for r in res)
    all_el = max(r[2] for r in res)
    value = n * all_steps / all_el
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "single_thread": {"value": single, "cores": 1, "steps": steps, "seconds": el},
            "full_runs_single_thread": _oracle_config_runs(),
            "sample": "first %d mm of the 300 mm channel at dx = 0.2 mm (%d fluid particles) "
                      "from t = 0; %d independent copies at once (one per host core) for about "
                      "%.0f s each, %d steps in all (one thread alone: %d steps, set-up %.1f s)"
                      % (round(Lx * 1e3), n, cores, seconds, all_steps, steps, setup)}


def _oracle_steps(args):
    """One host thread: the oracle on the first Lx of the channel, `warmup`
    untimed steps then `steps` timed ones; returns (particles, seconds)."""
    warmup, steps, Lx = args
    import oracle
    p, xy = workload(DX, Lx=Lx)
    o = oracle.OracleCase(p, xy.astype(np.float64))
    for _ in range(warmup):
        o.step()
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step()
    return xy.shape[0], time.perf_counter() - t0


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import multiprocessing as mp
    import oracle
    oracle.build()   # once, before the pool
    Lx = 0.0375
    cores = min(host_cores(), 64)
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_steps, [(args.warmup, args.steps, Lx)] * cores)
    n = res[0][0]
    el = max(r[1] for r in res)
    value = cores * n * args.steps / el
    sample = ("FP64 C oracle as it stands, %d independent copies at once (one per host core, "
              "%s), each on the first %.1f mm of the 300 mm channel at dx = 0.2 mm (%d fluid "
              "particles) from t = 0; value = all copies' particle-steps over the slowest "
              "copy's time" % (cores, cpu_model(), Lx * 1e3, n))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(DX, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_only(args):
    """One leg alone (for profiling): the reverse mode or the tangent mode on
    the channel at --dx for --steps steps (fixed dt), or the 64-case sweep."""
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    if args.only == "sweep":
        out = sweep_benchmark(stream)
    elif args.only == "batch":
        out = batch_steps_benchmark(stream, args.steps)
    elif args.only == "scaling":
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        out = scaling_benchmark(stream, flush, steps=args.steps)
    elif args.only == "small":
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        out = small_case_benchmark(stream, flush, steps=args.steps)
    elif args.only == "close":
        p, xy = workload(args.dx)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        out = close_benchmark(stream, flush, xy, p, steps=args.steps)
    elif args.only == "passvar":
        p, xy = workload(args.dx)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        out = pass_variant_benchmark(stream, xy, p, flush, steps=args.steps)
    else:
        from paper_2609_05494_b300 import Case
        p, xy = workload(args.dx)
        p["dt_mode"] = 1
        with torch.cuda.stream(stream):
            c = Case(p, xy, stream=stream, probe_capacity=args.steps + 8,
                     tangent=args.only == "tangent")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        if args.only == "adjoint":
            y = c.adjoint_forward(args.steps, 20)
            g = c.adjoint_backward()
            res = {"peak": y["peak"], "impulse": y["impulse"], "dpeak": g["dpeak"].tolist(),
                   "dimpulse": g["dimpulse"].tolist()}
        else:
            c.run(args.steps)
            res = {k: (v.tolist() if hasattr(v, "tolist") else v)
                   for k, v in c.tangent_outputs().items()}
        b.record(stream)
        torch.cuda.synchronize()
        out = {"leg": args.only, "particles": int(xy.shape[0]), "steps": args.steps,
               "ms_per_step": a.elapsed_time(b) / args.steps, "result": res}
        c.close()
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--dx", type=float, default=DX)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-tangent", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    ap.add_argument("--no-scaling", action="store_true")
    ap.add_argument("--no-production", action="store_true")
    ap.add_argument("--no-passvar", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-close", action="store_true")
    ap.add_argument("--only", choices=("adjoint", "tangent", "sweep", "passvar", "small", "scaling",
                                       "batch", "close"),
                    help="run one leg alone on the channel at --dx for --steps steps "
                         "(profiling runs); prints that leg's JSON")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.only:
        return run_only(args)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2609_05494_b300 import Case

    p, xy = workload(args.dx)
    n = xy.shape[0]
    stream = torch.cuda.Stream()
    # the headline graph carries no timing events (each event node in a graph
    # costs about 2.6 us of step time); kernel durations come from a second
    # case whose graph records them (HR_FLAG_TIMING), run right after
    with torch.cuda.stream(stream):
        case = Case(p, xy, stream=stream, probe_capacity=args.steps + args.warmup + 8)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # the interaction pass runs split at this size (interior particles beside
    # the ghost pass, boundary particles after it): close + drift, scan,
    # reorder, ghost, boundary pass and sums, interior pass = 7 launches per
    # step (5 unsplit); the step's close runs in the next step's drift launch
    # (one launch more per step when a case closes inline)
    split = bool(case.info()["split"])
    deferred = bool(case.info()["close_deferred"])
    launches_per_step = (7 if split else 5) + (0 if deferred else 1)
    # pairs per step (for the flop count), from the neighbour lists of the start state
    off, _ = case.neighbours()
    pairs_fluid_rows = int(off[n] - off[0])
    for _ in range(args.warmup):
        case.step()
    # (the last warm-up step's close stays pending: the first timed step's
    # graph runs it, so the K timed steps hold K closes)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.__enter__()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)               # write 256 MB > L2 between timed steps
            ev[k][0].record(stream)
            case.step()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    total_ms = max_over_ranks(total_ms, dist)
    if dist:
        dist.barrier()
    status = case.sync()

    # end to end through the C-ABI with host buffers (pinned), K steps
    vel0 = np.zeros_like(xy)
    rho0 = np.full(n, p["rho0"], np.float32)
    h_xy = torch.from_numpy(xy).pin_memory().numpy()
    h_v = torch.from_numpy(vel0).pin_memory().numpy()
    h_r = torch.from_numpy(rho0).pin_memory().numpy()
    def pinned(shape):
        return torch.empty(shape, dtype=torch.float32).pin_memory().numpy()
    h_probes = pinned((args.steps + args.warmup + 8, max(len(p["probes"]), 1)))
    h_final = dict(xy=pinned((n, 2)), vel=pinned((n, 2)), rho=pinned((n,)), p=pinned((n,)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    case.set_state(h_xy, h_v, h_r)
    case.run(args.steps)
    probes = case.probe_pressure(out=h_probes)
    final = case.get_state(out=h_final)
    e2e_s = time.perf_counter() - t0
    h2d = h_xy.nbytes + h_v.nbytes + h_r.nbytes
    d2h = probes.nbytes + sum(v.nbytes for v in final.values())

    case.close()

    # kernel durations: the same workload, graph with timing events, the same
    # flushed-L2 steps; k_pass's mean duration feeds the roofline
    with torch.cuda.stream(stream):
        tcase = Case(p, xy, stream=stream, timing=True, probe_capacity=args.steps + args.warmup + 8)
    tcase.run(args.warmup)
    tcase.sync()
    k_timed = min(args.steps, 100)
    pass_ms, gsum = [], {}
    for k in range(k_timed):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
            tcase.step()
        stream.synchronize()
        kt = tcase.kernel_times()
        pass_ms.append(kt["pass"])
        for g, v in kt.items():
            gsum[g] = gsum.get(g, 0.0) + v
    groups = {g: v / k_timed for g, v in gsum.items()}
    groups["steps"] = k_timed
    tcase.close()
    clk.__exit__(None, None, None)
    sweep = None if args.no_sweep else sweep_benchmark(stream, rank, world, dist)
    tangent = None if args.no_tangent else tangent_benchmark(stream, xy, p)
    adjoint = None if args.no_adjoint else adjoint_benchmark(stream, xy, p)
    paper = None if args.no_paper else paper_event_benchmark(stream)
    scaling = None if args.no_scaling else scaling_benchmark(stream, flush)
    production = None if args.no_production else production_benchmark(stream)
    passvar = None if args.no_passvar else pass_variant_benchmark(stream, xy, p, flush)
    small = None if args.no_small else small_case_benchmark(stream, flush)
    close_ab = None if args.no_close else close_benchmark(stream, flush, xy, p)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    pk, src = peaks()
    value = aggregate_value(world, n, args.steps, total_ms)
    t_pass = statistics.mean(pass_ms) * 1e-3
    flops = n * FLOP_PER_PARTICLE
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    alu_peak = fp32_peak_tflops(pk.get("sm_max_mhz", 2032.0), n_sm)
    achieved_tf = flops / t_pass / 1e12
    hbm_achieved = ALG_BYTES_PER_PARTICLE * n / t_pass / 1e9
    traffic = read_traffic(kernel_source_hash())
    from paper_2609_05494_b300 import fp32_rate
    fma = {"scalar_tflops": fp32_rate(False, stream), "packed_f32x2_tflops": fp32_rate(True, stream)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args.dx, world),
        "timing": "step graph without timing events; kernel durations from a second run of "
                  "the workload with in-graph CUDA events; each step graph runs the previous "
                  "step's close in the first blocks of its drift launch (k_close_drift), so "
                  "the drift group holds it and the finalize group is empty",
        "status": status,
        "clocks": clk.summary(),
        "e2e": {"value": world * n * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps},
        "gpu_launches": launches_per_step * args.steps,
        "pass_split": split,
        "roofline": {"kernel": "k_pass", "bound": "alu", "achieved": achieved_tf,
                     "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved_tf / alu_peak,
                     "traffic": traffic,
                     "peak_source": "FP32 from unit counts: %d SM (as the device reports) x "
                                    "128 lanes x 2 x %.0f MHz" % (n_sm, pk.get("sm_max_mhz", 2032.0)),
                     "fp32_fma_measured": fma,
                     "flop_per_launch": flops, "flop_per_particle": FLOP_PER_PARTICLE,
                     "pair_terms_only": {"pairs": pairs_fluid_rows,
                                         "flop_per_pair": FLOP_PER_PAIR,
                                         "tflops": pairs_fluid_rows * FLOP_PER_PAIR / t_pass / 1e12},
                     "pass_ms": t_pass * 1e3,
                     "pass_group": "k_pass over the interior particles, with k_ghost, "
                                   "k_pass_boundary and k_pass_boundary_sums beside it on a "
                                   "high-priority branch (events around the group)"
                                   if split else "k_pass"},
        "roofline_hbm": {"kernel": "k_pass", "bound": "hbm", "achieved": hbm_achieved,
                         "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": hbm_achieved / pk["hbm_gbs"],
                         "step_frac": ALG_BYTES_PER_PARTICLE * value / world / 1e9 / pk["hbm_gbs"],
                         "peak_source": src, "bytes_per_particle": ALG_BYTES_PER_PARTICLE},
        "kernel_groups_ms": groups,
        "batched_sweep": sweep,
        "tangent": tangent,
        "adjoint": adjoint,
        "paper_event": paper,
        "size_sweep": scaling,
        "production": production,
        "pass_variants": passvar,
        "small_cases": small,
        "step_close": close_ab,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
