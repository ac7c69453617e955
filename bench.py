#!/usr/bin/env python
"""Benchmark: synaptic events delivered per second, real-time factor and HBM
roofline fraction of spike delivery on one GB300.

Default workload (one JSON line on stdout): the balanced random network with
112,500 neurons (90,000 E + 22,500 I), in-degree 11,250 (9,000 E + 2,250 I),
1.27e9 static synapses in 12-byte FP32 records, delay 1.5 ms (15 steps of
0.1 ms), Poisson drive tuned for about 8 Hz.  One step = 1 s of biological
time (10,000 grid steps = 667 update/deliver intervals) of the whole hot path:
fused update with spike compaction, then delivery, every interval.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference      # the FP64 oracle on all host cores

Under torchrun (N > 1) every rank simulates its own independent network
(replicas: the workload does not exchange data between GPUs); the reported
value is all ranks' events over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "synaptic events delivered/s & real-time factor on 1 GB300; % of HBM roofline"
UNIT = "events/s"
# Poisson drive giving ~8 Hz in the 112,500-neuron network (found with
# paper_2109_12855_gb300.tune on a GB300; fixed from then on)
NU_EXT_8HZ = 25757.293701171875

WORKLOADS = {
    # name: (network recipe, record format, bio ms per step, kind)
    "balanced-112500-fp32": (W.BALANCED_112500, 0, 1000.0, "simulate"),
    "balanced-112500-bf16": (W.BALANCED_112500, 1, 1000.0, "simulate"),
    "balanced-562500-bf16": (W.BALANCED_562500, 1, 500.0, "simulate"),
    "balanced-1250-fp32": (W.BALANCED_1250, 0, 1000.0, "simulate"),
    # long run: 10 s of biological time per step, rates per second and the
    # CV of the intervals from the FP64 accumulators (drift check)
    "long-112500-fp32": (W.BALANCED_112500, 0, 10000.0, "long"),
    # plastic variant: E->E synapses with power-law STDP (FP32 weights
    # updated at delivery), the other synapses static BF16
    "balanced-112500-stdp-bf16": (W.BALANCED_112500, 1, 1000.0, "simulate"),
    "deliver-112500-fp32": (W.BALANCED_112500, 0, 1000.0, "deliver"),
    "deliver-562500-bf16": (W.BALANCED_562500, 1, 500.0, "deliver"),
    # profiling case for the update kernel: all 112,500 neurons, in-degree
    # 1,125 (a 1.5 GB store)
    "update-112500": (W.Balanced("balanced-112500-k1125", 90000, 22500, 900,
                                 225, 15, 15, "fp32", 0.0, 1000.0),
                      0, 1000.0, "simulate"),
    # profiling case of the plastic kernel: 20,000 neurons with the
    # in-degree of the 112,500-neuron network (1.8 GB store)
    "stdp-20000-bf16": (W.Balanced("balanced-20000", 16000, 4000, 9000,
                                   2250, 15, 15, "bf16", 0.0, 150.0),
                        1, 150.0, "simulate"),
    # profiling case with the per-CTA shape of the 562,500-neuron delivery
    # (tiles of 1,234 targets, 20-step window, runs of ~25 records; replay
    # at 46.6 Hz gives its ~4,400 runs per tile) on a 1.4 GB store
    "deliver-93750-k1900-bf16": (W.Balanced("balanced-93750-k1900", 75000,
                                            18750, 1520, 380, 10, 20, "bf16",
                                            0.1, 100.0), 1, 100.0, "deliver"),
    # profiling case: the same segment length and launch size as the
    # 112,500-neuron delivery, with a store of 2.7 GB
    "deliver-20000-fp32": (W.Balanced("balanced-20000", 16000, 4000, 9000,
                                      2250, 15, 15, "fp32", 0.0, 150.0),
                           0, 150.0, "deliver"),
    # profiling case of the interval-list delivery: the same in-degree, runs
    # of ~74 records per spike and tile, a 2.7 GB store, simulated
    "balanced-20000-fp32": (W.Balanced("balanced-20000", 16000, 4000, 9000,
                                       2250, 15, 15, "fp32", 0.0, 150.0),
                            0, 150.0, "simulate"),
    # the same network driven to ~45 Hz: ~1,350 spikes per 15-step interval,
    # the launch shape of the 1.27e9-synapse delivery (152 tiles, runs of ~74
    # records) on a 2.7 GB store, simulated (interval-list kernel, update
    # prefetch included)
    "balanced-20000-fp32-45hz": (W.Balanced("balanced-20000", 16000, 4000,
                                            9000, 2250, 15, 15, "fp32", 0.0,
                                            150.0), 0, 150.0, "simulate"),
    # the same 45 Hz network with BF16 8-byte records (the launch shape of
    # the 1.27e9-synapse BF16 delivery)
    "balanced-20000-bf16-45hz": (W.Balanced("balanced-20000", 16000, 4000,
                                            9000, 2250, 15, 15, "bf16", 0.0,
                                            150.0), 1, 150.0, "simulate"),
    # 93,750 neurons, in-degree 1,900, delays 10..20, BF16 with spread,
    # driven to ~47 Hz: ~4,400 spikes per 10-step interval and runs of ~25
    # records, the per-CTA shape of the 6.3e9-synapse delivery, on a 1.4 GB
    # store, simulated
    "balanced-93750-k1900-bf16": (W.Balanced("balanced-93750-k1900", 75000,
                                             18750, 1520, 380, 10, 20, "bf16",
                                             0.1, 100.0), 1, 100.0, "simulate"),
}
# drive of the profiling cases above (found with paper_2109_12855_gb300.tune
# on a GB300 for the rates stated; all other workloads use NU_EXT_8HZ)
NU_EXT_OF = {"balanced-20000-fp32-45hz": 89526.3671875,
             "balanced-20000-bf16-45hz": 89526.3671875,
             "balanced-93750-k1900-bf16": 35632.32421875}
DEFAULT = "balanced-112500-fp32"
PLASTIC = {"balanced-112500-stdp-bf16", "stdp-20000-bf16"}
# STDP of the plastic workload: tau 20 ms, lambda 0.1, alpha 0.0513, mu 0.4;
# weights bounded by 100 pA; 16 post spikes kept per neuron.  For
# uncorrelated firing the rule drifts towards w0 alpha^(-1/(1-mu)); w0 is
# set so that this equals the initial excitatory weight (w0 = 1 pA would put
# it at 141 pA, six times the 0.1 mV weight, and the network runs away).
STDP_ALPHA, STDP_MU = 0.0513, 0.4


def stdp_config(w_e):
    return dict(tau_plus=20.0, tau_minus=20.0, lam=0.1, alpha=STDP_ALPHA,
                mu=STDP_MU, w0=w_e * STDP_ALPHA ** (1.0 / (1.0 - STDP_MU)),
                w_max=100.0, history=16)
# DRAM bytes (read + write) per synaptic event of k_deliver_tiled, measured
# by ncu on launches of a small simulated case (a few GB on the device; for
# the 1.27e9-synapse network, FP32 and BF16, with its launch shape:
# in-degree, runs per tile, window; for the 6.3e9 one a short-run BF16 case,
# whose runs are shorter than the full network's) and divided by those
# launches' events
# (profiles/dram_k_deliver_tiled_*.md); bench.py scales it by the events of
# an average full-size launch.  It
# stands for the kernel it was measured on: the entry is used only while the
# kernel sources (comments aside) hash to the recorded prefixes.
TRAFFIC_B_PER_EVENT = {
    "balanced-112500-fp32": (12.339, "09aa1a562d40154d", "19d84bddd44d9f03"),
    "balanced-112500-bf16": (8.332, "09aa1a562d40154d", "19d84bddd44d9f03"),
    "balanced-562500-bf16": (9.375, "09aa1a562d40154d", "19d84bddd44d9f03"),
}
# serving: a Poisson stream of independent balanced nets (BF16 records,
# N log-uniform in [1,250, 112,500], 100 ms - 1 s each), mean rate in req/s
SERVE_WORKLOADS = {"serve-poisson-20": 20.0}
# L2 reduction throughput (red.global.add.f32, the ring-buffer additions):
# buffers the size of the 112,500- and 562,500-neuron ring buffers (32 slots)
# and one far beyond L2, scattered and sweeping cells
PROBE_WORKLOADS = {"l2-red-probe": [(32 * 112500, "ring buffer, 112,500 neurons"),
                                    (32 * 562500, "ring buffer, 562,500 neurons"),
                                    (1 << 28, "1 GiB, beyond L2")]}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
# the nominal HBM3e bandwidth of the part, reported beside the measured copy
HBM_NOMINAL_GBS = 7900.0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(ms: float, events: int, extra: float = 0.0):
    """(max ms, sum events, sum extra) over the process group (or identity)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return ms, events, extra
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    e = torch.tensor([float(events), extra], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), int(e[0].item()), float(e[1].item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
def oracle_sample(wl, nu_ext, n_targets, seed=1, n_lists=50, rate_hz=8.0,
                  plastic=False):
    """The segments of the targets [0, n_targets) (what one NEST thread that
    owns those targets holds), the oracle's neuron model for them, and a pool
    of interval spike lists of all sources (Bernoulli at rate_hz) that the
    timed steps cycle through."""
    import oracle as O
    nm = O.Neuron()
    w_e = O.weight_for_psp(nm, wl.psp_mv)
    cp = O.Conn(wl.n_e, wl.n_i, wl.k_e, wl.k_i, w_e, -wl.g * w_e, wl.d_lo,
                wl.d_hi, seed + 1000, wfmt=1 if wl.weight_format == "fp32" else 2)
    store = O.build_fixed_indegree_targets(cp, 0, n_targets)
    lists = [W.bernoulli_spikes(wl.n, 0, wl.d_lo, rate_hz, 0.1, seed=100 + k)
             for k in range(n_lists)]
    st = O.State(O.init_v(nm, n_targets, seed), np.zeros(n_targets),
                 np.zeros(n_targets), np.zeros(n_targets, np.int32))
    ctx = {"O": O, "nm": nm, "w_e": w_e, "store": store, "n": n_targets,
           "lists": lists, "state": st, "rb_local": np.zeros((32, n_targets)),
           "rb": np.zeros((32, wl.n)), "t": 0, "plastic": plastic}
    if plastic:
        q = stdp_config(w_e)
        ctx["w"] = store.w.copy()
        ctx["hist"] = O.History(wl.n, cap=96)
        ctx["stdp"] = O.Stdp(n_exc=wl.n_e, tau_plus=q["tau_plus"],
                             tau_minus=q["tau_minus"], lam=q["lam"],
                             alpha=q["alpha"], mu=q["mu"], w0=q["w0"],
                             w_max=q["w_max"])
    return ctx


def oracle_step(ctx, wl, nu_ext, n_intervals, seed=1):
    """n_intervals of: the oracle's update of the sampled neurons for one
    interval, then Algorithm REF delivery of one interval's spike list of all
    sources onto the sampled targets.  Both phases are timed as they stand;
    the delivered input is not fed back into the sampled neurons.  Returns
    (events, seconds)."""
    O, D = ctx["O"], wl.d_lo
    events, secs = 0, 0.0
    for _ in range(n_intervals):
        t = ctx["t"]
        src, tt = ctx["lists"][(t // D) % len(ctx["lists"])]
        a = time.perf_counter()
        O.update(ctx["nm"], ctx["state"], ctx["rb_local"], t, D, nu_ext,
                 ctx["w_e"], seed)
        if ctx["plastic"]:
            ctx["hist"].add(src, tt + t)
            _, _, ev = O.deliver_stdp(ctx["store"], ctx["w"], ctx["stdp"],
                                      ctx["hist"], 32, src, tt + t,
                                      rb=ctx["rb"])
        else:
            _, _, _, ev = O.deliver_ref(ctx["store"], 32, src, tt + t,
                                        rb=ctx["rb"], counts=False)
        secs += time.perf_counter() - a
        events += ev
        ctx["t"] = t + D
    return events, secs


def host_info():
    """Host facts for the CPU baseline: hardware threads, CPU model, memory."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True,
                                 timeout=10).stdout
            for line in out.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    mem = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    return {"nproc": os.cpu_count(), "cpu": model, "mem_gb": round(mem / 1e9, 1)}


def mem_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")


def oracle_threaded(wl, nu_ext, threads, n_targets, seed=1, n_lists=50):
    """The oracle's thread-parallel form on all host threads (each owns a
    range of neurons and the segments onto them, Section 2.1).  The whole
    network when its FP64 store (16 B per synapse, twice that while it is
    built) fits in 60 % of the available host memory; otherwise the targets
    [0, threads x n_targets) with Bernoulli lists of all sources, as in the
    single-thread sample."""
    import oracle as O
    nm = O.Neuron()
    w_e = O.weight_for_psp(nm, wl.psp_mv)
    cp = O.Conn(wl.n_e, wl.n_i, wl.k_e, wl.k_i, w_e, -wl.g * w_e, wl.d_lo,
                wl.d_hi, seed + 1000, sd_e=wl.sd_rel * w_e,
                sd_i=wl.sd_rel * wl.g * w_e,
                wfmt=1 if wl.weight_format == "fp32" else 2)
    whole = 32 * wl.n_synapses <= 0.6 * mem_available()
    hi = wl.n if whole else min(wl.n, threads * n_targets)
    mt = O.Threaded(cp, threads, tgt_hi=hi)
    st = O.State(O.init_v(nm, wl.n, seed), np.zeros(wl.n), np.zeros(wl.n),
                 np.zeros(wl.n, np.int32))
    ctx = {"O": O, "nm": nm, "w_e": w_e, "mt": mt, "state": st,
           "rb": np.zeros((32, wl.n)), "t": 0, "whole": whole, "hi": hi,
           "threads": mt.n_threads}
    if not whole:
        ctx["lists"] = [W.bernoulli_spikes(wl.n, 0, wl.d_lo, 8.0, 0.1,
                                           seed=100 + k) for k in range(n_lists)]
    return ctx


def oracle_threaded_step(ctx, wl, nu_ext, bio_ms, seed=1):
    """bio_ms of biological time: the whole network's time-driven cycle, or
    per interval the sampled neurons' update and the delivery of one list of
    all sources onto them.  Returns (events, seconds, spikes)."""
    D = wl.d_lo
    n_steps = int(round(bio_ms / 0.1))
    mt, st, rb = ctx["mt"], ctx["state"], ctx["rb"]
    if ctx["whole"]:
        cap = wl.n * (n_steps // 21 + 2)   # one spike per refractory period
        a = time.perf_counter()
        src, _, ev = mt.simulate(ctx["nm"], D, st, rb, ctx["t"], n_steps, nu_ext,
                                 ctx["w_e"], seed, cap=cap)
        secs = time.perf_counter() - a
        ctx["t"] += n_steps
        return ev, secs, len(src)
    events, secs = 0, 0.0
    for _ in range(max(1, n_steps // D)):
        t = ctx["t"]
        src, tt = ctx["lists"][(t // D) % len(ctx["lists"])]
        a = time.perf_counter()
        mt.update(ctx["nm"], st, rb, t, D, nu_ext, ctx["w_e"], seed)
        _, ev = mt.deliver(src, tt + t, rb)
        secs += time.perf_counter() - a
        events += ev
        ctx["t"] = t + D
    return events, secs, 0


def threaded_text(ctx, wl, bio_ms):
    if ctx["whole"]:
        return (f"the whole {wl.name} network ({wl.n_synapses:,} synapses, FP64 "
                f"store on the host), {bio_ms:g} ms of biological time per "
                f"step from the initial state: the oracle's time-driven cycle "
                f"on {ctx['threads']} host threads, each owning a range of "
                f"neurons and the segments onto them (NEST's thread model)")
    return (f"targets [0, {ctx['hi']:,}) of {wl.name} "
            f"({ctx['hi'] * wl.k:,} synapses) on {ctx['threads']} host threads "
            f"(each owning a range of them): per {wl.d_lo}-step interval the "
            f"oracle update of those neurons + Algorithm REF delivery of an "
            f"8 Hz Bernoulli spike list of all {wl.n:,} sources, "
            f"{bio_ms:g} ms of biological time per step")


def precision_probe(net, wl, nu_ext, w_g, seed, n_sample=3000):
    """Error of the stored-weight format against the FP64 oracle with the
    unrounded weights, measured after the timed region from the net's
    current state: both sides deliver one 8 Hz Bernoulli interval list
    (emission steps [t0 - D, t0)) and update one interval with the same
    drive; ring-buffer cells and membrane potentials of the targets
    [0, n_sample) are compared (max and RMS), neurons whose spike decision
    differs are counted and left out of the potential figures."""
    import oracle as O
    from paper_2109_12855_gb300 import snn
    D = wl.d_lo
    src, tt = W.bernoulli_spikes(wl.n, 0, D, 8.0, 0.1, seed=77)
    t0 = net.stats().t_now
    V, I, J, refr = net.read_state()
    snn.snn_clear_rb(net.h)
    net.deliver(src, (tt + t0 - D).astype(np.int32))
    rb_g = net.read_rb()[:, :n_sample].astype(np.float64)
    snn.snn_update(net.h, t0, D)
    snn.snn_discard_pending(net.h)
    V_g, _, _, refr_g = net.read_state()
    nm = O.Neuron()
    w_o = O.weight_for_psp(nm, wl.psp_mv)
    cp = O.Conn(wl.n_e, wl.n_i, wl.k_e, wl.k_i, w_o, -wl.g * w_o, wl.d_lo,
                wl.d_hi, seed + 1000, sd_e=wl.sd_rel * w_o,
                sd_i=wl.sd_rel * wl.g * w_o, wfmt=0)
    store = O.build_fixed_indegree_targets(cp, 0, n_sample)
    rb_o, _, absw, _ = O.deliver_ref(store, 32, src, tt + t0 - D)
    st = O.State(V.astype(np.float64), I.astype(np.float64),
                 J.astype(np.float64), refr.copy())
    O.update_range(nm, st, rb_o.copy(), 0, n_sample, t0, D, nu_ext, w_o, seed)
    err = rb_g - rb_o[:, :n_sample]
    absw = absw[:, :n_sample]
    hit = absw > 0
    same = refr_g[:n_sample] == st.refr[:n_sample]
    dv = np.abs(V_g[:n_sample].astype(np.float64) - st.V[:n_sample])
    return {"against": "FP64 oracle, unrounded weights",
            "targets": n_sample, "cells": int(hit.sum()),
            "rb_max_abs_pa": float(np.abs(err).max()),
            "rb_rms_pa": float(np.sqrt(np.mean(err[hit] ** 2))),
            "rb_max_rel": float((np.abs(err)[hit] / absw[hit]).max()),
            "vm_max_abs_mv": float(dv[same].max()) if same.any() else None,
            "vm_rms_mv": float(np.sqrt(np.mean(dv[same] ** 2)))
            if same.any() else None,
            "spike_mismatch": int((~same).sum())}


def cpu_baseline_all_cores(args, wl, nu_ext):
    """All-cores oracle figures for cpu_baseline: events/s, the real-time
    factor (measured on the whole network, or extrapolated from the sample
    by N / sampled neurons), and the host."""
    threads = args.oracle_threads or os.cpu_count() or 1
    ctx = oracle_threaded(wl, nu_ext, threads, args.oracle_targets)
    try:
        oracle_threaded_step(ctx, wl, nu_ext, 10.0)            # warm-up
        ev, secs, _ = oracle_threaded_step(ctx, wl, nu_ext, args.oracle_bio_ms)
    finally:
        ctx["mt"].close()
    rtf = secs / (args.oracle_bio_ms * 1e-3)
    out = {"value": ev / secs, "unit": UNIT, "cores": ctx["threads"],
           "kind": "oracle", "seconds": secs,
           "sample": threaded_text(ctx, wl, args.oracle_bio_ms),
           "real_time_factor": rtf if ctx["whole"] else rtf * wl.n / ctx["hi"],
           "real_time_factor_kind": "measured on the whole network"
           if ctx["whole"] else
           f"extrapolated: sample wall time x {wl.n:,} / {ctx['hi']:,} neurons"}
    return out


def sample_text(wl, n_targets, n_intervals, plastic=False):
    how = ("plastic delivery (STDP of the E->E synapses against the full "
           "spike history)" if plastic else "Algorithm REF delivery")
    return (f"targets [0, {n_targets:,}) of {wl.name} "
            f"({n_targets * wl.k:,} synapses), {n_intervals} intervals of "
            f"{wl.d_lo} steps: oracle update of those neurons + {how} "
            f"of 8 Hz Bernoulli spike lists of all {wl.n:,} sources "
            f"onto them (single thread)")


def run_reference(args, wl, nu_ext):
    """--impl reference: the oracle as it stands, on all host cores (its
    thread-parallel form); each step a bounded sample of the workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    plastic = args.workload in PLASTIC
    if plastic:
        # the plastic oracle has no thread-parallel form: one core
        n_targets = args.oracle_targets
        ctx = oracle_sample(wl, nu_ext, n_targets, plastic=True)
        per_step = min(args.oracle_intervals, 20)
        for _ in range(args.warmup):
            oracle_step(ctx, wl, nu_ext, per_step)
        ev, secs = 0, 0.0
        for _ in range(args.steps):
            e, s_ = oracle_step(ctx, wl, nu_ext, per_step)
            ev += e
            secs += s_
        cores = 1
        sample = sample_text(wl, n_targets, per_step, True) + " per step"
    else:
        threads = args.oracle_threads or os.cpu_count() or 1
        ctx = oracle_threaded(wl, nu_ext, threads, args.oracle_targets)
        try:
            for _ in range(args.warmup):
                oracle_threaded_step(ctx, wl, nu_ext, args.oracle_bio_ms)
            ev, secs = 0, 0.0
            for _ in range(args.steps):
                e, s_, _ = oracle_threaded_step(ctx, wl, nu_ext,
                                                args.oracle_bio_ms)
                ev += e
                secs += s_
        finally:
            ctx["mt"].close()
        cores = ctx["threads"]
        sample = threaded_text(ctx, wl, args.oracle_bio_ms)
    value = ev / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": sample,
                             "host": host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def build_net(wl, fmt, nu_ext, seed, stream, log_cap=0, deliver_mode=0,
              plastic=False):
    from paper_2109_12855_gb300.tune import build_balanced
    from paper_2109_12855_gb300 import snn
    w_e0 = snn.snn_psc_weight_for_psp(snn.params(), wl.psp_mv)
    net, w_e = build_balanced(wl.n_e, wl.n_i, wl.k_e, wl.k_i, wl.d_lo, wl.d_hi,
                              fmt, wl.sd_rel, seed, stream, psp_mv=wl.psp_mv,
                              g=wl.g, nu_ext=nu_ext,
                              stdp=snn.stdp_params(**stdp_config(w_e0))
                              if plastic else None,
                              spike_log_capacity=log_cap,
                              deliver_mode=deliver_mode)
    snn.snn_set_drive(net.h, nu_ext, w_e)
    return net, w_e


def _code_only(text):
    """Source text without comments and with whitespace collapsed: edits of
    comments leave the compiled kernel, and so the hash, unchanged."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_sources_hash():
    import hashlib
    csrc = os.path.join(ROOT, "paper_2109_12855_gb300", "csrc")
    return tuple(hashlib.sha256(_code_only(open(os.path.join(csrc, f)).read())
                                .encode()).hexdigest()[:16]
                 for f in ("snn_kernels.cu", "snn_internal.cuh"))


def measured_traffic(workload, events_per_launch):
    """ncu-measured DRAM bytes per launch of the delivery kernel, or None
    when there is no capture for this workload or the kernel has changed."""
    ent = TRAFFIC_B_PER_EVENT.get(workload)
    if ent is None or kernel_sources_hash() != ent[1:]:
        return None
    return ent[0] * events_per_launch


def timed(torch, stream, fn, k):
    """Run fn k times between events on the library's stream; ms total."""
    barrier()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(k):
        fn()
    b.record(stream)
    b.synchronize()
    torch.cuda.synchronize()
    barrier()
    return a.elapsed_time(b)


def run_ours(args, wl, fmt, bio_ms, kind, nu_ext):
    import torch
    from paper_2109_12855_gb300 import snn

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    s = torch.cuda.Stream()
    torch.cuda.set_stream(s)
    stream = s.cuda_stream
    steps_per = int(round(bio_ms / 0.1))
    rec_bytes = 12 if fmt == 0 else 8
    expected_spikes = int(wl.n * 8.0 * bio_ms * 1e-3 * 4) + 100000
    # the log must hold every spike of the timed region (read once after it)
    log_cap = expected_spikes * (max(args.steps, 3) + 1)

    t_build = time.perf_counter()
    mode = {"tiled": 0, "atomic": 1}[args.deliver_mode]
    plastic = args.workload in PLASTIC
    net, w_e = build_net(wl, fmt, nu_ext, 1 + rank, stream, log_cap=log_cap,
                         deliver_mode=mode, plastic=plastic)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t_build
    h = net.h
    st0 = net.stats()
    st_tiles = st0
    D = st0.interval

    if args.launch_bytes:
        # per-launch algorithmic bytes of the delivery kernel, for comparison
        # with a profiler's per-launch DRAM counters on the same (bitwise
        # reproducible) launches: --launch-skip intervals, then one interval
        # per call with the counters read after each
        snn.snn_simulate(h, args.launch_skip * D)
        rows = []
        for _ in range(args.launch_bytes):
            a = net.stats()
            snn.snn_simulate(h, D)
            b = net.stats()
            ev, sp = b.events_delivered - a.events_delivered, b.spikes - a.spikes
            pl = b.plastic_events - a.plastic_events
            rows.append({"events": ev, "spikes": sp,
                         "bytes": rec_bytes * ev + 32 * sp + 8 * pl})
        net.close()
        if rank == 0:
            print(json.dumps({"workload": args.workload, "skip": args.launch_skip,
                              "kernel": "k_deliver_tiled", "launches": rows}),
                  flush=True)
        return

    if kind == "deliver":
        # record one step of the whole network's spikes (or draw Bernoulli
        # lists at --replay-rate), then replay them interval by interval
        # through snn_deliver from device memory
        if args.replay_rate:
            src, t = W.bernoulli_spikes(wl.n, 0, steps_per, args.replay_rate,
                                        0.1, seed=5)
        else:
            snn.snn_simulate(h, steps_per)
            src, t = net.read_spikes(log_cap)
        order = np.lexsort((src, t))
        src, t = src[order], t[order]
        iv = (t // D).astype(np.int64)
        bounds = np.searchsorted(iv, np.arange(iv.min(), iv.max() + 2)) \
            if len(iv) else np.zeros(1, np.int64)
        d_src = torch.from_numpy(src.astype(np.int32)).cuda()
        d_t = torch.from_numpy(t.astype(np.int32)).cuda()
        lists = [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:])]

        def step():
            for a, b in lists:
                if b > a:
                    snn.lib().snn_deliver(h, d_src.data_ptr() + 4 * a,
                                          d_t.data_ptr() + 4 * a, b - a,
                                          snn.SNN_MEM_DEVICE, None)
    elif kind == "long":
        # a long run in 1 s pieces: spikes per second for the drift check
        per_s = []
        one_s = int(round(1000.0 / 0.1))

        def step():
            for _ in range(int(round(bio_ms / 1000.0))):
                before = net.stats().spikes
                snn.snn_simulate(h, one_s)
                per_s.append((net.stats().spikes - before) / wl.n)
    else:
        def step():
            snn.snn_simulate(h, steps_per)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    net.read_spikes(log_cap)      # empty the log
    if kind == "long":
        per_s.clear()
        snn.snn_clear_spike_stats(h)

    # ---- timed region: production path (graphs) --------------------------
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
    clocks = Clocks(gpu_index)
    a = net.stats()
    clocks.start()
    ms = timed(torch, s, step, args.steps)
    clk = clocks.stop()
    b = net.stats()
    events = b.events_delivered - a.events_delivered
    spikes = b.spikes - a.spikes
    launches = b.kernel_launches - a.kernel_launches
    net.read_spikes(log_cap)
    ms_max, events_all, spikes_all = reduce_over_ranks(ms, events, spikes)
    value = events_all / (ms_max * 1e-3)
    long_run = None
    if kind == "long":
        r = np.array(per_s[:int(round(bio_ms / 1000.0))])
        _, n_isi, s1, s2 = snn.snn_read_spike_stats(h, wl.n)
        ok = n_isi >= 2
        m = s1[ok] / n_isi[ok]
        cv = float(np.mean(np.sqrt(np.maximum(s2[ok] / n_isi[ok] - m * m, 0)) / m))
        long_run = {"rate_hz_per_s": [round(float(x), 4) for x in r],
                    "max_rel_drift": float(np.max(np.abs(r / r.mean() - 1.0))),
                    "cv_isi": cv, "neurons_with_2_intervals": int(ok.sum())}

    # ---- roofline: the same steps with every launch between CUDA events ----
    snn.snn_set_profiling(h, True)
    a = net.stats()
    ms_prof = timed(torch, s, step, args.steps)
    b = net.stats()
    snn.snn_set_profiling(h, False)
    n_del = b.deliver_launches - a.deliver_launches
    ms_del = b.ms_deliver - a.ms_deliver
    ms_upd = b.ms_update - a.ms_update
    ev_prof = b.events_delivered - a.events_delivered
    sp_prof = b.spikes - a.spikes
    pl_prof = b.plastic_events - a.plastic_events
    net.read_spikes(log_cap)
    # algorithmic bytes: one record per event; per spike a list entry (16 B)
    # and its two row offsets (16 B); a plastic event also reads and writes
    # its FP32 weight (8 B)
    n_listed = sp_prof if kind != "deliver" else len(src) * args.steps
    alg_bytes = rec_bytes * ev_prof + 32 * n_listed + 8 * pl_prof
    per_launch_bytes = alg_bytes / max(n_del, 1)
    per_launch_s = ms_del * 1e-3 / max(n_del, 1)
    hbm, peak_kind = peaks()
    achieved = per_launch_bytes / per_launch_s / 1e9 if per_launch_s else 0.0

    # ---- end to end through the public API with host buffers --------------
    e2e = None
    if kind == "simulate":
        n = wl.n
        hV = torch.empty(n, dtype=torch.float32).pin_memory()
        hI = torch.empty(n, dtype=torch.float32).pin_memory()
        hJ = torch.empty(n, dtype=torch.float32).pin_memory()
        hR = torch.empty(n, dtype=torch.int32).pin_memory()
        hsrc = torch.empty(expected_spikes, dtype=torch.int32).pin_memory()
        ht = torch.empty(expected_spikes, dtype=torch.int32).pin_memory()
        snn.snn_read_state(h, hV, hI, hJ, hR)
        counts = {"spikes": 0}

        def e2e_step():
            snn.snn_write_state(h, hV, hI, hJ, hR)           # h2d
            snn.snn_simulate(h, steps_per)
            counts["spikes"] += snn.snn_read_spikes(h, hsrc, ht)  # d2h
            snn.snn_read_state(h, hV, hI, hJ, hR)            # d2h

        k_e2e = max(1, args.steps)
        a = net.stats()
        ms_e2e = timed(torch, s, e2e_step, k_e2e)
        b = net.stats()
        ev_e2e = b.events_delivered - a.events_delivered
        ms_e2e_max, ev_e2e_all, _ = reduce_over_ranks(ms_e2e, ev_e2e)
        e2e = {"value": ev_e2e_all / (ms_e2e_max * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": 16 * n,
               "d2h_bytes_per_step": int(16 * n + 8 * counts["spikes"] / k_e2e),
               "steps": k_e2e}
    st = net.stats()
    err = st.error_flags
    precision = None
    if ws == 1 and not args.no_cpu_baseline and kind != "deliver" and not plastic:
        precision = precision_probe(net, wl, nu_ext, w_e, 1 + rank)
    net.close()

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        ctx = oracle_sample(wl, nu_ext, args.oracle_targets, plastic=plastic)
        n_iv = args.cpu_intervals if not plastic else min(args.cpu_intervals, 150)
        oracle_step(ctx, wl, nu_ext, 5)
        e_c, s_c = oracle_step(ctx, wl, nu_ext, n_iv)
        one = {"value": e_c / s_c, "unit": UNIT, "cores": 1, "kind": "oracle",
               "seconds": s_c,
               "sample": sample_text(wl, args.oracle_targets, n_iv, plastic)}
        del ctx
        if plastic:   # the plastic oracle has no thread-parallel form
            cpu = dict(one, host=host_info())
        else:
            cpu = cpu_baseline_all_cores(args, wl, nu_ext)
            cpu["single_core"] = one
            cpu["host"] = host_info()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if fmt == 0 else "bf16-store/f32-accumulate",
        "data": "synthetic",
        "real_time_factor": (ms_max / args.steps) / bio_ms,
        "config": {"workload": args.workload, "neurons": wl.n,
                   "in_degree": wl.k, "synapses": wl.n_synapses,
                   "record_bytes": rec_bytes, "interval_steps": D,
                   "bio_ms_per_step": bio_ms, "nu_ext_hz": nu_ext,
                   "mean_rate_hz": spikes_all / ws / wl.n / (
                       args.steps * bio_ms * 1e-3),
                   "events_timed": events_all, "spikes_timed": int(spikes_all),
                   "plastic": plastic,
                   **({"stdp": stdp_config(w_e), "plastic_events_profiled": pl_prof,
                       "stdp_truncated": st.stdp_truncated} if plastic else {}),
                   "build_s": t_build,
                   "l2": "inputs larger than L2 (the record store is "
                         f"{wl.n_synapses * rec_bytes / 1e9:.1f} GB, streamed "
                         "from HBM every step)",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm,
                     "peak_source": peak_kind,
                     "frac_of_nominal": achieved / HBM_NOMINAL_GBS,
                     "traffic": measured_traffic(args.workload,
                                                 ev_prof / max(n_del, 1)),
                     "traffic_unit": "bytes per launch (ncu dram read+write)",
                     "algorithmic_bytes_per_launch": per_launch_bytes,
                     "kernel": "k_deliver_tiled" if args.deliver_mode == "tiled"
                               else "k_deliver",
                     "launches": n_del, "avg_launch_us": 1e3 * ms_del / max(n_del, 1),
                     "deliver_mode": args.deliver_mode,
                     "tiles": [st_tiles.n_tiles, st_tiles.tile_width,
                               st_tiles.window],
                     "bytes_per_event": rec_bytes + (8 * pl_prof / max(ev_prof, 1)),
                     "ms_deliver_share": ms_del / ms_prof if ms_prof else None,
                     "ms_update_share": ms_upd / ms_prof if ms_prof else None,
                     "profiled_value": ev_prof / (ms_prof * 1e-3)},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "error_flags": err,
    }
    if precision:
        line["precision"] = precision
    if long_run:
        line["long_run"] = long_run
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
def serve_requests(snn, stream_reqs, fmt, nu_ext, record, seed_offset=0):
    out = []
    for i, r in enumerate(stream_reqs):
        wl = r.net
        p = snn.params(n_exc=wl.n_e, n_inh=wl.n_i, weight_format=fmt,
                       seed=r.seed + seed_offset, nu_ext=nu_ext)
        w_e = snn.snn_psc_weight_for_psp(p, wl.psp_mv)
        p.w_ext = w_e
        c = snn.conn_params(k_exc=wl.k_e, k_inh=wl.k_i, w_exc=w_e,
                            w_inh=-wl.g * w_e, sd_exc=wl.sd_rel * w_e,
                            sd_inh=wl.sd_rel * wl.g * w_e, d_lo=wl.d_lo,
                            d_hi=wl.d_hi, seed=r.seed + seed_offset + 1000,
                            clip_exc=1, clip_inh=0)
        out.append(snn.request(p, c, int(round(wl.bio_ms / 0.1)), user_tag=i,
                               record_spikes=record))
    return out


def _lat_stats(lat):
    a = np.sort(np.asarray(lat)) * 1e3
    return {"p50_ms": float(np.percentile(a, 50)),
            "p99_ms": float(np.percentile(a, 99)),
            "max_ms": float(a[-1]), "mean_ms": float(a.mean())}


def serve_batched(snn, reqs, arrivals, budget, stream, clocks=None,
                  persistent=0, exclusive=0):
    """Continuous batching: submit each request at its arrival time, step the
    server until every request finished.  Latency = completion - arrival."""
    sv = snn.snn_server_create(budget, reqs[0].params.weight_format, stream)
    try:
        snn.snn_server_set_option(sv, snn.SNN_SERVE_OPT_PERSISTENT, persistent)
        snn.snn_server_set_option(sv, snn.SNN_SERVE_OPT_EXCLUSIVE, exclusive)
        ids, lag = [], []
        if clocks:
            clocks.start()
        t0 = time.perf_counter()
        nxt, n = 0, len(reqs)
        last_steps = -1
        while True:
            now = time.perf_counter() - t0
            while nxt < n and arrivals[nxt] <= now:
                ids.append(snn.snn_server_submit(sv, reqs[nxt]))
                lag.append(time.perf_counter() - t0 - arrivals[nxt])
                nxt += 1
            active = snn.snn_server_step(sv)
            st = snn.snn_server_get_stats(sv)
            if nxt == n and st.done + st.failed == n:
                break
            if active == 0:
                time.sleep(1e-4)          # nothing on the GPU yet
            elif st.steps == last_steps:
                time.sleep(2e-5)          # every lane busy: let the GPU run
            last_steps = st.steps
        wall = time.perf_counter() - t0
        clk = clocks.stop() if clocks else None
        res = [snn.snn_server_poll(sv, i) for i in ids]
        if any(r.state != snn.SNN_REQ_DONE for r in res):
            raise RuntimeError("served request failed: " + str(
                [(r.id, r.error) for r in res if r.state != snn.SNN_REQ_DONE]))
        lat = [r.t_done - r.t_submit + g for r, g in zip(res, lag)]
        spikes_read = sum(r.spikes for r in res)
        parts = {"queue_p50_ms": 1e3 * float(np.median([r.t_admit - r.t_submit for r in res])),
                 "build_p50_ms": 1e3 * float(np.median([r.t_start - r.t_admit for r in res])),
                 "run_p50_ms": 1e3 * float(np.median([r.t_done - r.t_start for r in res]))}
        return {"wall_s": wall, "events": sum(r.events for r in res),
                "spikes": spikes_read, "latency": _lat_stats(lat),
                "latency_parts": parts,
                "server_steps": st.steps, "intervals": st.intervals,
                "kernel_launches": st.kernel_launches, "gpu_ms": st.gpu_ms,
                "intervals_per_step": st.intervals_per_step,
                "tuned": st.tuned, "clocks": clk}
    finally:
        snn.snn_server_destroy(sv)


def serve_serial(snn, reqs, arrivals, stream):
    """The plain single-net path, one request at a time in arrival order:
    build, snn_simulate, read the spikes back, destroy."""
    t0 = time.perf_counter()
    lat, events, spikes = [], 0, 0
    for r, arr in zip(reqs, arrivals):
        now = time.perf_counter() - t0
        if now < arr:
            time.sleep(arr - now)
        p = snn.snn_params.from_buffer_copy(r.params)
        with snn.Net(p, stream) as net:
            net.connect_fixed_indegree(r.conn)
            net.finalize()
            snn.snn_simulate(net.h, r.n_steps)
            if p.spike_log_capacity:
                net.read_spikes()
            st = net.stats()
        events += st.events_delivered
        spikes += st.spikes
        lat.append(time.perf_counter() - t0 - arr)
    wall = time.perf_counter() - t0
    return {"wall_s": wall, "events": events, "spikes": spikes,
            "latency": _lat_stats(lat)}


def spike_log_bound(r):
    """Spike-log capacity that holds every spike of a request (each neuron
    fires at most once per refractory period plus one step)."""
    n = r.params.n_exc + r.params.n_inh
    refr = round(r.params.t_ref / r.params.h)
    return min(n * int((r.n_steps + refr) / (refr + 1)), 1 << 22)


def run_serve(args, rate_hz, nu_ext):
    import torch
    from paper_2109_12855_gb300 import snn

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    s = torch.cuda.Stream()
    torch.cuda.set_stream(s)
    stream = s.cuda_stream
    stream_reqs = W.serving_stream(args.requests, rate_hz, seed=7)
    arrivals = [r.arrival_s for r in stream_reqs]
    zero = [0.0] * len(arrivals)
    off = 1000000 * rank                  # replicas draw their own nets
    bf16 = serve_requests(snn, stream_reqs, 1, nu_ext, True, off)
    fp32 = serve_requests(snn, stream_reqs, 0, nu_ext, True, off)
    for r in fp32:                        # the single-net path sizes its log
        r.params.spike_log_capacity = spike_log_bound(r)
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.8 * free)

    # warm-up: short runs of the first requests through both paths
    for _ in range(max(args.warmup, 1)):
        warm = serve_requests(snn, stream_reqs[:3], 1, nu_ext, True, off)
        for r in warm:
            r.n_steps = 200
        serve_batched(snn, warm, [0.0] * 3, budget, stream)
        warm = serve_requests(snn, stream_reqs[:3], 0, nu_ext, False, off)
        for r in warm:
            r.n_steps = 200
        serve_serial(snn, warm, [0.0] * 3, stream)

    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    if cvd.isdigit():
        gpu_index = int(cvd)
    barrier()
    batched = serve_batched(snn, bf16, arrivals, budget, stream,
                            Clocks(gpu_index))
    persist = serve_batched(snn, bf16, arrivals, budget, stream, persistent=1)
    excl = serve_batched(snn, bf16, arrivals, budget, stream, exclusive=1)
    serial = serve_serial(snn, fp32, arrivals, stream)
    sat_batched = serve_batched(snn, bf16, zero, budget, stream)
    sat_persist = serve_batched(snn, bf16, zero, budget, stream, persistent=1)
    sat_excl = serve_batched(snn, bf16, zero, budget, stream, exclusive=1)
    sat_serial_bf16 = serve_serial(snn, [r for r in serve_requests(
        snn, stream_reqs, 1, nu_ext, False, off)], zero, stream)
    sat_serial = serve_serial(snn, fp32, zero, stream)
    barrier()

    wall, events_all, _ = reduce_over_ranks(1e3 * batched["wall_s"],
                                            batched["events"])
    value = events_all / (wall * 1e-3)
    if rank != 0:
        return

    def rate(x):
        return x["events"] / x["wall_s"]

    hbm, peak_kind = peaks()
    gpu_s = batched["gpu_ms"] * 1e-3
    alg_bytes = 8 * batched["events"] + 32 * batched["spikes"]
    achieved = alg_bytes / gpu_s / 1e9 if gpu_s else 0.0
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        big = max(stream_reqs, key=lambda r: r.net.n_synapses).net
        n_t = min(args.oracle_targets, big.n)
        ctx = oracle_sample(big, nu_ext, n_t)
        oracle_step(ctx, big, nu_ext, 5)
        e_c, s_c = oracle_step(ctx, big, nu_ext, args.cpu_intervals)
        cpu = {"value": e_c / s_c, "unit": UNIT, "cores": 1, "kind": "oracle",
               "seconds": s_c,
               "sample": sample_text(big, n_t, args.cpu_intervals)}
    n_req = len(stream_reqs)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": batched["server_steps"], "warmup": args.warmup,
        "ms_per_step": wall / max(batched["server_steps"], 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-store/f32-accumulate", "data": "synthetic",
        "config": {"workload": args.workload, "requests": n_req,
                   "arrival_rate_hz": rate_hz,
                   "neurons": [min(r.net.n for r in stream_reqs),
                               max(r.net.n for r in stream_reqs)],
                   "synapses_total": sum(r.net.n_synapses for r in stream_reqs),
                   "bio_ms_total": sum(r.net.bio_ms for r in stream_reqs),
                   "nu_ext_hz": nu_ext, "mem_budget_bytes": budget,
                   "step": "one server step: every running net advances by "
                           "the autotuned number of intervals",
                   "l2": "inputs larger than L2 (the resident stores total "
                         "several GB, streamed every interval)",
                   "parallelism": f"replicas x{ws}"},
        "latency": batched["latency"],
        "serving": {
            "batched_bf16": {"events_per_s": rate(batched), **batched},
            "batched_bf16_persistent": {"events_per_s": rate(persist),
                                        **persist},
            "exclusive_bf16": {"events_per_s": rate(excl), **excl},
            "serial_fp32": {"events_per_s": rate(serial), **serial},
            "saturated": {
                "batched_bf16": {"events_per_s": rate(sat_batched),
                                 "wall_s": sat_batched["wall_s"],
                                 "latency": sat_batched["latency"],
                                 "intervals_per_step":
                                     sat_batched["intervals_per_step"]},
                "batched_bf16_persistent": {
                    "events_per_s": rate(sat_persist),
                    "wall_s": sat_persist["wall_s"],
                    "latency": sat_persist["latency"]},
                "exclusive_bf16": {"events_per_s": rate(sat_excl),
                                   "wall_s": sat_excl["wall_s"],
                                   "latency": sat_excl["latency"]},
                "serial_bf16": {"events_per_s": rate(sat_serial_bf16),
                                "wall_s": sat_serial_bf16["wall_s"],
                                "latency": sat_serial_bf16["latency"]},
                "serial_fp32": {"events_per_s": rate(sat_serial),
                                "wall_s": sat_serial["wall_s"],
                                "latency": sat_serial["latency"]}}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm,
                     "peak_source": peak_kind, "traffic": None,
                     "kernel": "k_update_batch + k_deliver_tiled_batch "
                               "(GPU time of the server steps)",
                     "bytes_per_event": 8},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT,
                "h2d_bytes_per_step": int(n_req * ctypes_size(snn.snn_request)
                                          / max(batched["server_steps"], 1)),
                "d2h_bytes_per_step": int(8 * batched["spikes"]
                                          / max(batched["server_steps"], 1)),
                "note": "the serving value is already end to end: requests "
                        "enter as host structs and every spike train is read "
                        "back to host memory inside the timed region"},
        "gpu_launches": batched["kernel_launches"],
        "clocks": batched["clocks"],
    }
    print(json.dumps(line), flush=True)


def ctypes_size(t):
    import ctypes
    return ctypes.sizeof(t)


# ---------------------------------------------------------------------------
# target-partitioned network over the ranks (one partition per GPU)
# ---------------------------------------------------------------------------
def run_partitioned(args, wl, fmt, bio_ms, nu_ext):
    """Rank r simulates neurons split(N, world)[r] of ONE network with the
    synapses of all sources onto them; every interval the ranks all-gather
    their spike lists and deliver the union.  The union of the partitions
    equals the whole net bit for bit.  Strong scaling: the total work is
    fixed as the number of GPUs grows.

    Default exchange: the update writes its spikes into a fixed-size device
    buffer, one NCCL all_gather_into_tensor moves the buffers (none at
    N=1), the delivery reads them directly -- no host synchronisation per
    interval.  --host-exchange: read each pending list (counts through the
    host) and all-gather variable-length lists."""
    import torch
    from paper_2109_12855_gb300 import partition as PT
    from paper_2109_12855_gb300 import snn

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    s = torch.cuda.Stream()
    torch.cuda.set_stream(s)
    lo, hi = PT.split(wl.n, ws)[rank]
    # spike log: this rank's spikes of the warm-up, timed and end-to-end
    # steps (read back by the end-to-end steps)
    per_step = int((hi - lo) * 8.0 * bio_ms * 1e-3 * 4) + 100000
    p = snn.params(n_exc=wl.n_e, n_inh=wl.n_i, weight_format=fmt, seed=1,
                   nu_ext=nu_ext,
                   spike_log_capacity=per_step * (args.warmup + args.steps + 2))
    w_e = snn.snn_psc_weight_for_psp(p, wl.psp_mv)
    p.w_ext = w_e
    c = snn.conn_params(k_exc=wl.k_e, k_inh=wl.k_i, w_exc=w_e,
                        w_inh=-wl.g * w_e, sd_exc=wl.sd_rel * w_e,
                        sd_inh=wl.sd_rel * wl.g * w_e, d_lo=wl.d_lo,
                        d_hi=wl.d_hi, seed=1001, clip_exc=1, clip_inh=0)
    t_build = time.perf_counter()
    net = PT.create(p, c, lo, hi, s.cuda_stream)

    def reduce_max(v):
        import torch.distributed as dist
        x = torch.tensor([float(a) for a in v], dtype=torch.float64,
                         device="cuda")
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        return [x[0].item(), x[1].item(), x[2].item()]

    PT.agree_bounds([net], reduce_max if ws > 1 else None)
    net.finalize()
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t_build
    D = net.stats().interval
    d_src = torch.empty(max(net.n * D, 1), dtype=torch.int32, device="cuda")
    d_t = torch.empty_like(d_src)
    steps_per = int(round(bio_ms / 0.1))
    xch = None
    if not args.host_exchange:
        def cap_max(v):
            import torch.distributed as dist
            x = torch.tensor([int(v)], dtype=torch.int64, device="cuda")
            dist.all_reduce(x, op=dist.ReduceOp.MAX)
            return int(x.item())
        xch = PT.DeviceExchange([net], reduce_max=cap_max if ws > 1 else None)

    iv_per_step = -(-steps_per // D)

    def step(t0):
        if xch is not None:  # replays of 8-interval graphs, as snn_simulate
            PT.simulate_exchanged([net], xch, steps_per, interval=D,
                                  graph_intervals=8)
            return t0 + steps_per
        t = t0
        while t < t0 + steps_per:
            m = min(D, t0 + steps_per - t)
            snn.snn_update(net.h, t, m)
            k = snn.snn_read_pending(net.h, d_src, d_t)
            a_s, a_t = d_src[:k], d_t[:k]
            if ws > 1:
                a_s, a_t = PT.allgather_spikes(a_s, a_t)
            snn.snn_deliver_gathered(net.h, a_s, a_t, want_events=False)
            t += m
        return t

    t = 0
    for _ in range(args.warmup):
        t = step(t)
    torch.cuda.synchronize()
    a = net.stats()
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    clocks = Clocks(int(cvd) if cvd.isdigit() else local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        t = step(t)
    e1.record(s)
    e1.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms = e0.elapsed_time(e1)
    b = net.stats()
    events = b.events_delivered - a.events_delivered
    spikes = b.spikes - a.spikes
    # update + delivery per interval (graph replays are not counted by the
    # library's host counters)
    launches = (2 * iv_per_step * args.steps if xch is not None
                else b.kernel_launches - a.kernel_launches)
    ms_max, ev_all, sp_all = reduce_over_ranks(ms, events, spikes)
    if b.error_flags:
        raise RuntimeError(f"device error flags {b.error_flags:#x}")
    # end to end through the public API with host buffers: this rank's
    # neuron state in from pinned host memory, the step, its spikes and
    # state back
    e2e = None
    if xch is not None:
        n_loc = net.n
        hV = torch.empty(n_loc, dtype=torch.float32).pin_memory()
        hI = torch.empty_like(hV).pin_memory()
        hJ = torch.empty_like(hV).pin_memory()
        hR = torch.empty(n_loc, dtype=torch.int32).pin_memory()
        cap = per_step * (args.warmup + args.steps + 2)
        hsrc = torch.empty(cap, dtype=torch.int32).pin_memory()
        ht = torch.empty(cap, dtype=torch.int32).pin_memory()
        snn.snn_read_state(net.h, hV, hI, hJ, hR)
        snn.snn_read_spikes(net.h, hsrc, ht)
        sp_read = [0]

        def e2e_step():
            snn.snn_write_state(net.h, hV, hI, hJ, hR)
            step(0)
            sp_read[0] += snn.snn_read_spikes(net.h, hsrc, ht)
            snn.snn_read_state(net.h, hV, hI, hJ, hR)

        c0 = net.stats()
        ms_e2e = timed(torch, s, e2e_step, args.steps)
        c1 = net.stats()
        ms_e2e_max, ev_e2e_all, sp_e2e_all = reduce_over_ranks(
            ms_e2e, c1.events_delivered - c0.events_delivered, sp_read[0])
        e2e = {"value": ev_e2e_all / (ms_e2e_max * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": 16 * wl.n,
               "d2h_bytes_per_step": int(16 * wl.n + 8 * sp_e2e_all / args.steps),
               "steps": args.steps}
    if xch is not None:
        xch.close()
    net.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": ev_all / (ms_max * 1e-3), "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None,
        "dtype": "f32" if fmt == 0 else "bf16-store/f32-accumulate",
        "data": "synthetic", "real_time_factor": (ms_max / args.steps) / bio_ms,
        "config": {"workload": args.workload, "neurons": wl.n,
                   "synapses": wl.n_synapses, "bio_ms_per_step": bio_ms,
                   "mean_rate_hz": sp_all / wl.n / (args.steps * bio_ms * 1e-3),
                   "build_s": t_build,
                   "parallelism": f"target partition x{ws}: each GPU holds "
                                  "1/N of the neurons and the synapses onto "
                                  "them; spike lists all-gathered every "
                                  "interval",
                   "exchange": ("host lists (read + variable all-gather)"
                                if args.host_exchange else
                                "device buffers (fixed all_gather_into_tensor, "
                                "no host sync), 8-interval CUDA graphs")},
        "roofline": None, "cpu_baseline": None, "e2e": e2e,
        "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def use_partition(workload: str, kind: str, world: int, partition: bool,
                  replicas: bool) -> bool:
    """Several ranks split ONE network (target partition, strong scaling)
    unless replicas are asked for; one rank runs the whole net unless the
    partitioned path is asked for.  Plastic and replayed-list workloads do
    not partition."""
    partitionable = kind == "simulate" and "stdp" not in workload
    if partition and not partitionable:
        raise SystemExit(f"{workload} cannot be partitioned")
    return partitionable and (partition or (world > 1 and not replicas))


def run_probe(args, sizes):
    """Reductions per second of snn_probe_reductions per buffer size and
    pattern: median of --steps timed launches after --warmup ones; the line's
    value is the scattered rate at the first size."""
    import torch
    from paper_2109_12855_gb300 import snn
    torch.cuda.set_device(0)
    n_ops = 1 << 28
    clocks = Clocks(0)
    rows, launches = [], 0
    clocks.start()
    for n_cells, what in sizes:
        buf = torch.zeros(n_cells, device="cuda")
        for pattern, pname in ((snn.SNN_PROBE_SCATTER, "scatter"),
                               (snn.SNN_PROBE_SWEEP, "sweep")):
            for _ in range(args.warmup):
                snn.snn_probe_reductions(buf, n_ops, pattern)
            ms = sorted(snn.snn_probe_reductions(buf, n_ops, pattern)
                        for _ in range(args.steps))
            launches += args.warmup + args.steps
            med = ms[len(ms) // 2]
            rows.append({"cells": n_cells, "bytes": 4 * n_cells, "buffer": what,
                         "pattern": pname, "ops": n_ops, "ms": med,
                         "ops_per_s": n_ops / (med * 1e-3)})
        del buf
    clk = clocks.stop()
    first = rows[0]
    print(json.dumps({
        "metric": "L2 reductions/s (red.global.add.f32, the ring-buffer additions)",
        "value": first["ops_per_s"], "unit": "ops/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": first["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "ops_per_launch": n_ops,
                   "l2": "the two ring-buffer sizes are L2-resident (the "
                         "probe's own working set); the third exceeds L2"},
        "probe": rows, "roofline": None, "cpu_baseline": None, "e2e": None,
        "gpu_launches": launches, "clocks": clk}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) +
                    sorted(SERVE_WORKLOADS) + sorted(PROBE_WORKLOADS),
                    default=DEFAULT)
    ap.add_argument("--host-exchange", action="store_true",
                    help="with --partition: exchange through the host "
                         "(pending lists read back every interval)")
    ap.add_argument("--replicas", action="store_true",
                    help="with several ranks: independent copies of the "
                         "network (one per GPU) instead of one partitioned "
                         "network")
    ap.add_argument("--partition", action="store_true",
                    help="split one network over the ranks (target "
                         "partition, spike all-gather every interval) "
                         "instead of running independent replicas")
    ap.add_argument("--requests", type=int, default=40,
                    help="serving workloads: requests in the stream")
    ap.add_argument("--nu-ext", type=float, default=None)
    ap.add_argument("--oracle-targets", type=int, default=4500)
    ap.add_argument("--oracle-intervals", type=int, default=100,
                    help="oracle intervals per --impl reference step")
    ap.add_argument("--cpu-intervals", type=int, default=1500,
                    help="oracle intervals timed for cpu_baseline")
    ap.add_argument("--oracle-threads", type=int, default=0,
                    help="host threads of the all-cores oracle (0: all)")
    ap.add_argument("--oracle-bio-ms", type=float, default=100.0,
                    help="biological ms per all-cores oracle step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--launch-bytes", type=int, default=0,
                    help="print the algorithmic bytes of this many delivery "
                         "launches (one interval each) and exit")
    ap.add_argument("--launch-skip", type=int, default=200,
                    help="intervals simulated before --launch-bytes")
    ap.add_argument("--deliver-mode", choices=["tiled", "atomic"],
                    default="tiled")
    ap.add_argument("--replay-rate", type=float, default=0.0,
                    help="deliver workloads: Bernoulli lists at this rate "
                         "instead of a recorded run")
    args = ap.parse_args()
    nu_ext = args.nu_ext if args.nu_ext is not None else \
        NU_EXT_OF.get(args.workload, NU_EXT_8HZ)
    if args.workload in PROBE_WORKLOADS:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the probe measures the GPU's L2; it has no "
                              "CPU reference"}))
            return
        from paper_2109_12855_gb300 import build
        build()
        run_probe(args, PROBE_WORKLOADS[args.workload])
        return
    if args.workload in SERVE_WORKLOADS:
        if args.impl == "reference":
            big = max(W.serving_stream(args.requests), key=lambda r:
                      r.net.n_synapses).net
            run_reference(args, big, nu_ext)
        else:
            from paper_2109_12855_gb300 import build
            build()
            run_serve(args, SERVE_WORKLOADS[args.workload], nu_ext)
        return
    wl, fmt, bio_ms, kind = WORKLOADS[args.workload]
    args.partition = use_partition(args.workload, kind, dist_env()[0],
                                   args.partition, args.replicas)
    if args.partition and args.impl != "reference":
        from paper_2109_12855_gb300 import build
        build()
        run_partitioned(args, wl, fmt, bio_ms, nu_ext)
        return
    if args.impl == "reference":
        run_reference(args, wl, nu_ext)
    else:
        from paper_2109_12855_gb300 import build
        build()
        run_ours(args, wl, fmt, bio_ms, kind, nu_ext)


if __name__ == "__main__":
    main()
