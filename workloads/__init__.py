"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds none of the method's arithmetic: it only draws random
inputs (spike lists, edge lists, neuron states) with numpy's PCG64 so that the
CUDA path and the oracle can be fed identical data.  The network's own random
numbers (connections, initial potentials, Poisson drive) are not drawn here:
both sides generate those from the counter-based Philox4x32-10 definition.

Workload recipes (balanced random network, Section 2.2 of the paper; the
parameters follow the benchmark configurations):

* ``BALANCED_1250``   N = 1,250 (1,000 E + 250 I), K = 100 (80 E + 20 I),
  delays uniform in 10..20 steps (1.0-2.0 ms at h = 0.1 ms).
* ``BALANCED_112500`` N = 112,500 (90,000 E + 22,500 I), K = 11,250
  (9,000 E + 2,250 I), delay 15 steps (1.5 ms), FP32 records.
* ``BALANCED_562500`` N = 562,500 (450,000 E + 112,500 I), K = 11,250,
  delays 10..20 steps, BF16 records with weights N(J, 0.1 J) (E, clipped at 0)
  and N(-5 J, 0.5 J) (I).
* ``serving_stream``  a Poisson stream of independent balanced nets (mean
  20 requests/s): N log-uniform in [1,250, 112,500] with 4:1 E:I,
  K = min(N/10, 11,250) with 4:1 E:I, BF16 records with the spread above,
  delays 10..20 steps, 100 ms to 1 s of biological time, one seed each.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Balanced:
    name: str
    n_e: int
    n_i: int
    k_e: int
    k_i: int
    d_lo: int
    d_hi: int
    weight_format: str      # "fp32" (12-byte records) or "bf16" (8-byte)
    sd_rel: float           # relative weight spread (0: fixed weights)
    bio_ms: float           # simulated biological time of the workload
    g: float = 5.0          # inhibitory weight = -g * excitatory weight
    psp_mv: float = 0.1     # J_E: peak membrane response of one E synapse

    @property
    def n(self) -> int:
        return self.n_e + self.n_i

    @property
    def k(self) -> int:
        return self.k_e + self.k_i

    @property
    def n_synapses(self) -> int:
        return self.n * self.k


BALANCED_1250 = Balanced("balanced-1250", 1000, 250, 80, 20, 10, 20, "fp32",
                         0.0, 1000.0)
BALANCED_112500 = Balanced("balanced-112500", 90000, 22500, 9000, 2250, 15, 15,
                           "fp32", 0.0, 1000.0)
BALANCED_562500 = Balanced("balanced-562500", 450000, 112500, 9000, 2250, 10,
                           20, "bf16", 0.1, 500.0)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def bernoulli_spikes(n: int, t0: int, n_steps: int, rate_hz: float, h_ms: float,
                     seed: int, sources: np.ndarray | None = None):
    """Spike list of an interval [t0, t0 + n_steps): each neuron (or each of
    ``sources``) fires independently with probability rate * h per step.
    Returns (src uint32, t int64), step-major then neuron-minor."""
    g = rng(seed)
    pool = np.arange(n, dtype=np.uint32) if sources is None else \
        np.asarray(sources, np.uint32)
    p = rate_hz * h_ms * 1e-3
    src, tt = [], []
    for s in range(n_steps):
        hit = pool[g.random(len(pool)) < p]
        src.append(hit)
        tt.append(np.full(len(hit), t0 + s, np.int64))
    if not src:
        return np.zeros(0, np.uint32), np.zeros(0, np.int64)
    return np.concatenate(src).astype(np.uint32), np.concatenate(tt)


def random_spikes(n: int, n_spikes: int, t_lo: int, t_hi: int, seed: int):
    """``n_spikes`` uniformly random (source, step) pairs, duplicates allowed."""
    g = rng(seed)
    src = g.integers(0, n, n_spikes, dtype=np.uint32) if n else \
        np.zeros(0, np.uint32)
    tt = g.integers(t_lo, t_hi, n_spikes).astype(np.int64)
    return src, tt


def random_edges(n: int, n_edges: int, d_lo: int, d_hi: int, seed: int,
                 w_scale: float = 20.0, hub: int | None = None,
                 hub_edges: int = 0):
    """Random edge list (src, tgt, delay, w) with optional hub source that
    gets ``hub_edges`` extra out-edges (a long target segment)."""
    g = rng(seed)
    src = g.integers(0, n, n_edges, dtype=np.uint32)
    tgt = g.integers(0, n, n_edges, dtype=np.uint32)
    if hub is not None and hub_edges:
        src = np.concatenate([src, np.full(hub_edges, hub, np.uint32)])
        tgt = np.concatenate([tgt, g.integers(0, n, hub_edges, dtype=np.uint32)])
    m = len(src)
    delay = g.integers(d_lo, d_hi + 1, m).astype(np.int32)
    w = g.normal(0.0, w_scale, m)
    return src, tgt, delay, w


def random_state(n: int, seed: int, v_lo: float = 0.0, v_hi: float = 20.0,
                 refr_max: int = 20):
    """Neuron state (V mV, I pA, J pA/ms, refractory count)."""
    g = rng(seed)
    V = g.uniform(v_lo, v_hi, n)
    I = g.normal(0.0, 50.0, n)
    J = g.normal(0.0, 200.0, n)
    refr = np.where(g.random(n) < 0.2, g.integers(1, refr_max + 1, n), 0)
    return V, I, J, refr.astype(np.int32)


@dataclass(frozen=True)
class ServeRequest:
    arrival_s: float        # offset from the start of the stream
    net: Balanced
    seed: int


def serving_stream(n_requests: int, rate_hz: float = 20.0, seed: int = 7,
                   n_lo: int = 1250, n_hi: int = 112500,
                   bio_lo_ms: float = 100.0, bio_hi_ms: float = 1000.0):
    """Poisson arrivals (exponential gaps of mean 1/rate_hz; all at 0 when
    rate_hz is 0) of balanced nets with log-uniform sizes."""
    g = rng(seed)
    out, t = [], 0.0
    for i in range(n_requests):
        if rate_hz > 0 and i > 0:
            t += g.exponential(1.0 / rate_hz)
        n = int(round(np.exp(g.uniform(np.log(n_lo), np.log(n_hi))) / 5)) * 5
        n = min(max(n, n_lo), n_hi)
        k = min(n // 10, 11250)
        k_e = k * 4 // 5
        bio = float(round(g.uniform(bio_lo_ms, bio_hi_ms), 1))
        net = Balanced(f"serve-{i}", n * 4 // 5, n - n * 4 // 5, k_e, k - k_e,
                       10, 20, "bf16", 0.1, bio)
        out.append(ServeRequest(t, net, 1000 + i))
    return out
