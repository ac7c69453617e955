"""FP64 CPU oracle for spike delivery (arXiv 2109.12855), TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2109_12855_gb300``) and never imports it.

The arithmetic lives in ``snn_oracle.c`` (plain C, FP64); this module only
compiles it with gcc and marshals numpy arrays through ctypes.  Each wrapper
names the passage of the paper it follows:

* ``deliver_ref``            -- Section 3.2, Algorithm REF.
* ``deliver_bwrb/lagrb/bwts`` -- Sections 4.1-4.4 (bwRB*, lagRB, bwTS,
  bwTSRB*), order-preserving rewrites of REF kept as self-checks.
* ``build_fixed_indegree``   -- Section 2.2 (balanced random network,
  random connectivity) and Section 3.1 (source-specific target segments).
* ``update`` / ``simulate``  -- Section 1 and Section 2.1 (time-driven
  cycle: update for one min-delay interval, then deliver; exact
  integration of the linear subthreshold dynamics).
* ``Threaded``               -- Section 2.1 (the thread model: each thread
  owns a range of neurons and the segments onto them); bitwise the results
  of ``simulate`` / ``deliver_ref``, on all host cores.
* ``deliver_stdp`` / ``simulate_stdp`` -- Section 6 (plasticity as an update
  scheme driven by presynaptic spikes, weights computed at delivery; the
  cited pair-based power-law rule), with the readings stated in the C source.

Pins: the paper prints no worked example, so none of these can be checked
against numbers it prints; every one is pinned in
``tests/test_oracle_pins.py`` (and ``tests/test_oracle_stdp.py``,
``tests/test_oracle_threaded.py``) by closed forms, library routines, brute
force and invariants.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``snn_oracle.c`` into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fno-fast-math",
           "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm",
           "-pthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB_PATH)
        _declare(_lib)
    return _lib


class NeuronC(C.Structure):
    _fields_ = [("h", C.c_double), ("tau_m", C.c_double), ("c_m", C.c_double),
                ("v_th", C.c_double), ("v_reset", C.c_double),
                ("t_ref", C.c_double), ("tau_syn", C.c_double)]


class ConnC(C.Structure):
    _fields_ = [("n_e", C.c_uint32), ("n_i", C.c_uint32), ("k_e", C.c_uint32),
                ("k_i", C.c_uint32), ("w_e", C.c_double), ("w_i", C.c_double),
                ("sd_e", C.c_double), ("sd_i", C.c_double),
                ("d_lo", C.c_int32), ("d_hi", C.c_int32), ("seed", C.c_uint64),
                ("clip_e", C.c_int32), ("clip_i", C.c_int32),
                ("wfmt", C.c_int32)]


class StoreC(C.Structure):
    _fields_ = [("n", C.c_uint32), ("n_slots", C.c_int32),
                ("row_ptr", C.c_void_p), ("tgt", C.c_void_p),
                ("delay", C.c_void_p), ("w", C.c_void_p)]


_P = C.c_void_p


def _declare(lib):
    lib.orc_philox4x32_10.argtypes = [_P, _P, _P]
    lib.orc_round_f32.argtypes = [C.c_double]
    lib.orc_round_f32.restype = C.c_double
    lib.orc_round_bf16.argtypes = [C.c_double]
    lib.orc_round_bf16.restype = C.c_double
    lib.orc_propagators.argtypes = [C.POINTER(NeuronC), _P]
    lib.orc_psp_unit.argtypes = [C.POINTER(NeuronC), C.c_double]
    lib.orc_psp_unit.restype = C.c_double
    lib.orc_psp_peak.argtypes = [C.POINTER(NeuronC), C.POINTER(C.c_double)]
    lib.orc_psp_peak.restype = C.c_double
    lib.orc_refractory_steps.argtypes = [C.POINTER(NeuronC)]
    lib.orc_refractory_steps.restype = C.c_int
    lib.orc_poisson_table.argtypes = [C.c_double, _P, C.c_int]
    lib.orc_poisson_table.restype = C.c_int
    lib.orc_poisson_count.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, _P,
                                      C.c_int]
    lib.orc_poisson_count.restype = C.c_int
    lib.orc_init_v.argtypes = [C.POINTER(NeuronC), C.c_uint32, C.c_uint64, _P]
    lib.orc_draw_synapse.argtypes = [C.POINTER(ConnC), C.c_uint32, C.c_uint32,
                                     _P, _P, _P]
    lib.orc_incoming.argtypes = [C.POINTER(ConnC), C.c_uint32, _P, _P, _P]
    lib.orc_build_fixed_indegree.argtypes = [C.POINTER(ConnC), _P, _P, _P, _P]
    lib.orc_build_fixed_indegree.restype = C.c_int
    lib.orc_build_fixed_indegree_targets.argtypes = [
        C.POINTER(ConnC), C.c_uint32, C.c_uint32, _P, _P, _P, _P]
    lib.orc_build_fixed_indegree_targets.restype = C.c_int
    lib.orc_build_edges.argtypes = [C.c_uint32, C.c_uint64, _P, _P, _P, _P,
                                    _P, _P, _P, _P]
    lib.orc_build_edges.restype = C.c_int
    for name in ("orc_deliver_bwrb", "orc_deliver_lagrb"):
        getattr(lib, name).argtypes = [C.POINTER(StoreC), C.c_uint64, _P, _P,
                                       _P, C.c_int]
        getattr(lib, name).restype = C.c_uint64
    lib.orc_deliver_ref.argtypes = [C.POINTER(StoreC), C.c_uint64, _P, _P, _P,
                                    _P, _P]
    lib.orc_deliver_ref.restype = C.c_uint64
    lib.orc_deliver_bwts.argtypes = [C.POINTER(StoreC), C.c_uint64, _P, _P,
                                     _P, C.c_int, C.c_int]
    lib.orc_deliver_bwts.restype = C.c_uint64
    lib.orc_update.argtypes = [C.POINTER(NeuronC), C.c_uint32, C.c_int32, _P,
                               _P, _P, _P, _P, C.c_int64, C.c_int32,
                               C.c_double, C.c_double, C.c_uint64, _P, _P,
                               C.c_uint64]
    lib.orc_update.restype = C.c_uint64
    lib.orc_simulate.argtypes = [C.POINTER(NeuronC), C.POINTER(StoreC),
                                 C.c_int32, _P, _P, _P, _P, _P, C.c_int64,
                                 C.c_int64, C.c_double, C.c_double, C.c_uint64,
                                 _P, _P, C.c_uint64, C.POINTER(C.c_uint64)]
    lib.orc_simulate.restype = C.c_uint64
    lib.orc_update_range.argtypes = [C.POINTER(NeuronC), C.c_uint32,
                                     C.c_uint32, C.c_uint32, C.c_int32, _P, _P,
                                     _P, _P, _P, C.c_int64, C.c_int32,
                                     C.c_double, C.c_double, C.c_uint64, _P,
                                     _P, C.c_uint64]
    lib.orc_update_range.restype = C.c_uint64
    lib.orc_mt_create.argtypes = [C.POINTER(ConnC), C.c_int, C.c_int32,
                                  C.c_uint32, C.c_uint32]
    lib.orc_mt_create.restype = C.c_void_p
    lib.orc_mt_destroy.argtypes = [C.c_void_p]
    lib.orc_mt_threads.argtypes = [C.c_void_p]
    lib.orc_mt_threads.restype = C.c_int
    lib.orc_mt_range.argtypes = [C.c_void_p, C.c_int, _P, _P]
    lib.orc_mt_simulate.argtypes = [C.c_void_p, C.POINTER(NeuronC), C.c_int32,
                                    _P, _P, _P, _P, _P, C.c_int64, C.c_int64,
                                    C.c_double, C.c_double, C.c_uint64, _P, _P,
                                    C.c_uint64, C.POINTER(C.c_uint64)]
    lib.orc_mt_simulate.restype = C.c_uint64
    lib.orc_mt_deliver.argtypes = [C.c_void_p, C.c_uint64, _P, _P, _P]
    lib.orc_mt_deliver.restype = C.c_uint64
    lib.orc_mt_update.argtypes = [C.c_void_p, C.POINTER(NeuronC), _P, _P, _P,
                                  _P, _P, C.c_int64, C.c_int32, C.c_double,
                                  C.c_double, C.c_uint64]
    lib.orc_mt_update.restype = C.c_uint64
    _declare_stdp(lib)


class StdpC(C.Structure):
    _fields_ = [("h", C.c_double), ("tau_plus", C.c_double),
                ("tau_minus", C.c_double), ("lam", C.c_double),
                ("alpha", C.c_double), ("mu", C.c_double), ("w0", C.c_double),
                ("w_max", C.c_double), ("n_exc", C.c_uint32)]


class HistC(C.Structure):
    _fields_ = [("n", C.c_uint32), ("cap", C.c_uint32), ("t", C.c_void_p),
                ("count", C.c_void_p)]


def _declare_stdp(lib):
    lib.orc_hist_add.argtypes = [C.POINTER(HistC), C.c_uint64, _P, _P]
    lib.orc_hist_add.restype = C.c_int
    lib.orc_deliver_stdp.argtypes = [C.POINTER(StoreC), _P, C.POINTER(StdpC),
                                     C.POINTER(HistC), C.c_uint64, _P, _P, _P,
                                     _P]
    lib.orc_deliver_stdp.restype = C.c_uint64


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# Model parameters
# --------------------------------------------------------------------------
@dataclass
class Neuron:
    """iaf_psc_alpha parameters (resting potential 0 mV)."""
    h: float = 0.1          # ms
    tau_m: float = 10.0     # ms
    c_m: float = 250.0      # pF
    v_th: float = 20.0      # mV
    v_reset: float = 0.0    # mV
    t_ref: float = 2.0      # ms
    tau_syn: float = 0.5    # ms

    def c(self) -> NeuronC:
        return NeuronC(self.h, self.tau_m, self.c_m, self.v_th, self.v_reset,
                       self.t_ref, self.tau_syn)


@dataclass
class Conn:
    """Fixed in-degree rule (see ``orc_draw_synapse`` in the C source)."""
    n_e: int
    n_i: int
    k_e: int
    k_i: int
    w_e: float
    w_i: float
    d_lo: int
    d_hi: int
    seed: int
    sd_e: float = 0.0
    sd_i: float = 0.0
    clip_e: bool = True
    clip_i: bool = False
    wfmt: int = 0           # 0 FP64, 1 FP32-rounded, 2 BF16-rounded

    def c(self) -> ConnC:
        return ConnC(self.n_e, self.n_i, self.k_e, self.k_i, self.w_e,
                     self.w_i, self.sd_e, self.sd_i, self.d_lo, self.d_hi,
                     self.seed, int(self.clip_e), int(self.clip_i), self.wfmt)


@dataclass
class Store:
    """Source-major connection store: row ``i`` is ``[row_ptr[i], row_ptr[i+1])``."""
    n: int
    row_ptr: np.ndarray   # uint64 [n+1]
    tgt: np.ndarray       # uint32
    delay: np.ndarray     # int32
    w: np.ndarray         # float64

    def c(self, n_slots: int) -> StoreC:
        return StoreC(self.n, n_slots, self.row_ptr.ctypes.data,
                      self.tgt.ctypes.data, self.delay.ctypes.data,
                      self.w.ctypes.data)


# --------------------------------------------------------------------------
# Wrappers
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def round_f32(x: float) -> float:
    return _load().orc_round_f32(x)


def round_bf16(x: float) -> float:
    return _load().orc_round_bf16(x)


def propagators(nm: Neuron) -> np.ndarray:
    """Closed-form exact propagator entries (P11, P21, P22, P31, P32, P33)."""
    out = np.zeros(6)
    _load().orc_propagators(C.byref(nm.c()), _ptr(out))
    return out


def psp_unit(nm: Neuron, t: float) -> float:
    return _load().orc_psp_unit(C.byref(nm.c()), t)


def psp_peak(nm: Neuron):
    tp = C.c_double()
    v = _load().orc_psp_peak(C.byref(nm.c()), C.byref(tp))
    return v, tp.value


def weight_for_psp(nm: Neuron, psp_mv: float) -> float:
    """PSC amplitude (pA) whose membrane response peaks at ``psp_mv``."""
    return psp_mv / psp_peak(nm)[0]


def refractory_steps(nm: Neuron) -> int:
    return _load().orc_refractory_steps(C.byref(nm.c()))


def poisson_table(lam: float, cap: int = 256) -> np.ndarray:
    thr = np.zeros(cap, dtype=np.uint64)
    n = _load().orc_poisson_table(lam, _ptr(thr), cap)
    return thr[:n].copy()


def poisson_count(seed: int, neuron: int, step: int, thr: np.ndarray) -> int:
    thr = np.ascontiguousarray(thr, dtype=np.uint64)
    return _load().orc_poisson_count(seed, neuron, step, _ptr(thr), len(thr))


def init_v(nm: Neuron, n: int, seed: int) -> np.ndarray:
    V = np.zeros(n)
    _load().orc_init_v(C.byref(nm.c()), n, seed, _ptr(V))
    return V


def draw_synapse(cp: Conn, tgt: int, k: int):
    s = np.zeros(1, np.uint32)
    d = np.zeros(1, np.int32)
    w = np.zeros(1)
    _load().orc_draw_synapse(C.byref(cp.c()), tgt, k, _ptr(s), _ptr(d), _ptr(w))
    return int(s[0]), int(d[0]), float(w[0])


def incoming(cp: Conn, tgt: int):
    """All K_E + K_I incoming synapses of one target: (src, delay, w) arrays."""
    kk = cp.k_e + cp.k_i
    src = np.zeros(max(kk, 1), np.uint32)
    dl = np.zeros(max(kk, 1), np.int32)
    w = np.zeros(max(kk, 1))
    _load().orc_incoming(C.byref(cp.c()), tgt, _ptr(src), _ptr(dl), _ptr(w))
    return src[:kk], dl[:kk], w[:kk]


def build_fixed_indegree(cp: Conn) -> Store:
    n = cp.n_e + cp.n_i
    m = n * (cp.k_e + cp.k_i)
    rp = np.zeros(n + 1, np.uint64)
    tg = np.zeros(max(m, 1), np.uint32)
    dl = np.zeros(max(m, 1), np.int32)
    w = np.zeros(max(m, 1))
    rc = _load().orc_build_fixed_indegree(C.byref(cp.c()), _ptr(rp), _ptr(tg),
                                          _ptr(dl), _ptr(w))
    if rc != 0:
        raise MemoryError("oracle store build failed (%d)" % rc)
    return Store(n, rp, tg[:m], dl[:m], w[:m])


def build_fixed_indegree_targets(cp: Conn, tgt_lo: int, tgt_hi: int) -> Store:
    n = cp.n_e + cp.n_i
    m = (tgt_hi - tgt_lo) * (cp.k_e + cp.k_i)
    rp = np.zeros(n + 1, np.uint64)
    tg = np.zeros(max(m, 1), np.uint32)
    dl = np.zeros(max(m, 1), np.int32)
    w = np.zeros(max(m, 1))
    rc = _load().orc_build_fixed_indegree_targets(
        C.byref(cp.c()), tgt_lo, tgt_hi, _ptr(rp), _ptr(tg), _ptr(dl), _ptr(w))
    if rc != 0:
        raise MemoryError("oracle store build failed (%d)" % rc)
    return Store(n, rp, tg[:m], dl[:m], w[:m])


def build_edges(n: int, src, tgt, delay, w) -> Store:
    src = np.ascontiguousarray(src, np.uint32)
    tgt = np.ascontiguousarray(tgt, np.uint32)
    delay = np.ascontiguousarray(delay, np.int32)
    w = np.ascontiguousarray(w, np.float64)
    m = len(src)
    rp = np.zeros(n + 1, np.uint64)
    tg = np.zeros(max(m, 1), np.uint32)
    dl = np.zeros(max(m, 1), np.int32)
    ww = np.zeros(max(m, 1))
    rc = _load().orc_build_edges(n, m, _ptr(src), _ptr(tgt), _ptr(delay),
                                 _ptr(w), _ptr(rp), _ptr(tg), _ptr(dl), _ptr(ww))
    if rc != 0:
        raise ValueError("oracle edge-list build failed (%d)" % rc)
    return Store(n, rp, tg[:m], dl[:m], ww[:m])


def _spikes(src, t):
    src = np.ascontiguousarray(src, np.uint32)
    t = np.ascontiguousarray(t, np.int64)
    assert len(src) == len(t)
    return src, t


def deliver_ref(st: Store, n_slots: int, src, t, rb=None, counts=True):
    """Algorithm REF.  Returns (rb[S][N] float64, cnt[S][N] uint32, absw[S][N],
    events).  ``rb`` is accumulated into when given."""
    src, t = _spikes(src, t)
    if rb is None:
        rb = np.zeros((n_slots, st.n))
    cnt = np.zeros((n_slots, st.n), np.uint32) if counts else None
    absw = np.zeros((n_slots, st.n)) if counts else None
    ev = _load().orc_deliver_ref(
        C.byref(st.c(n_slots)), len(src), _ptr(src), _ptr(t), _ptr(rb),
        _ptr(cnt) if counts else None, _ptr(absw) if counts else None)
    return rb, cnt, absw, int(ev)


def deliver_bwrb(st: Store, n_slots: int, src, t, b_rb: int):
    src, t = _spikes(src, t)
    rb = np.zeros((n_slots, st.n))
    ev = _load().orc_deliver_bwrb(C.byref(st.c(n_slots)), len(src), _ptr(src),
                                  _ptr(t), _ptr(rb), b_rb)
    return rb, int(ev)


def deliver_lagrb(st: Store, n_slots: int, src, t, b_rb: int):
    src, t = _spikes(src, t)
    rb = np.zeros((n_slots, st.n))
    ev = _load().orc_deliver_lagrb(C.byref(st.c(n_slots)), len(src), _ptr(src),
                                   _ptr(t), _ptr(rb), b_rb)
    return rb, int(ev)


def deliver_bwts(st: Store, n_slots: int, src, t, b_ts: int, b_rb: int = 0):
    src, t = _spikes(src, t)
    rb = np.zeros((n_slots, st.n))
    ev = _load().orc_deliver_bwts(C.byref(st.c(n_slots)), len(src), _ptr(src),
                                  _ptr(t), _ptr(rb), b_ts, b_rb)
    return rb, int(ev)


@dataclass
class State:
    V: np.ndarray
    I: np.ndarray
    J: np.ndarray
    refr: np.ndarray

    @staticmethod
    def zeros(n: int) -> "State":
        return State(np.zeros(n), np.zeros(n), np.zeros(n),
                     np.zeros(n, np.int32))

    def copy(self) -> "State":
        return State(self.V.copy(), self.I.copy(), self.J.copy(),
                     self.refr.copy())


def update(nm: Neuron, st: State, rb: np.ndarray, t0: int, n_steps: int,
           nu_ext_hz: float, w_ext: float, seed: int, cap: int | None = None):
    """Exact-integration update of all neurons for ``n_steps`` steps (in place).
    Returns (spike sources, spike steps) in step-major, neuron-minor order."""
    n = len(st.V)
    n_slots = rb.shape[0]
    cap = n * max(n_steps, 1) if cap is None else cap
    src = np.zeros(max(cap, 1), np.uint32)
    tt = np.zeros(max(cap, 1), np.int64)
    ns = _load().orc_update(C.byref(nm.c()), n, n_slots, _ptr(st.V), _ptr(st.I),
                            _ptr(st.J), _ptr(st.refr), _ptr(rb), t0, n_steps,
                            nu_ext_hz, w_ext, seed, _ptr(src), _ptr(tt), cap)
    ns = min(int(ns), cap)
    return src[:ns].copy(), tt[:ns].copy()


def update_range(nm: Neuron, st: State, rb: np.ndarray, lo: int, hi: int,
                 t0: int, n_steps: int, nu_ext_hz: float, w_ext: float,
                 seed: int, cap: int | None = None):
    """``update`` of the neurons [lo, hi) only (arrays indexed globally, in
    place; the drive keyed by the global index)."""
    n = len(st.V)
    assert 0 <= lo <= hi <= n and rb.shape[1] == n
    cap = (hi - lo) * max(n_steps, 1) if cap is None else cap
    src = np.zeros(max(cap, 1), np.uint32)
    tt = np.zeros(max(cap, 1), np.int64)
    ns = _load().orc_update_range(C.byref(nm.c()), lo, hi, n, rb.shape[0],
                                  _ptr(st.V), _ptr(st.I), _ptr(st.J),
                                  _ptr(st.refr), _ptr(rb), t0, n_steps,
                                  nu_ext_hz, w_ext, seed, _ptr(src), _ptr(tt),
                                  cap)
    ns = min(int(ns), cap)
    return src[:ns].copy(), tt[:ns].copy()


def simulate(nm: Neuron, store: Store, n_slots: int, interval: int, st: State,
             rb: np.ndarray, t0: int, n_steps: int, nu_ext_hz: float,
             w_ext: float, seed: int, cap: int = 1 << 24):
    """Time-driven cycle (update one interval, deliver with REF).  In place on
    ``st`` and ``rb``.  Returns (spike sources, spike steps, events)."""
    src = np.zeros(cap, np.uint32)
    tt = np.zeros(cap, np.int64)
    ev = C.c_uint64()
    ns = _load().orc_simulate(C.byref(nm.c()), C.byref(store.c(n_slots)),
                              interval, _ptr(st.V), _ptr(st.I), _ptr(st.J),
                              _ptr(st.refr), _ptr(rb), t0, n_steps, nu_ext_hz,
                              w_ext, seed, _ptr(src), _ptr(tt), cap,
                              C.byref(ev))
    ns = min(int(ns), cap)
    return src[:ns].copy(), tt[:ns].copy(), int(ev.value)


class Threaded:
    """The fixed in-degree network on ``n_threads`` host threads (NEST's
    thread model, Section 2.1): the threads split the neurons
    [tgt_lo, tgt_hi) (default: all N) evenly in order and each holds the
    segments of all sources onto its own neurons.  ``simulate`` (whole
    population only) and ``deliver`` return bitwise what ``simulate`` /
    ``deliver_ref`` return on the full store; ``update`` runs the owned
    neurons.  Close it (or use ``with``) to free the stores."""

    def __init__(self, cp: Conn, n_threads: int, n_slots: int = 32,
                 tgt_lo: int = 0, tgt_hi: int | None = None):
        self.n = cp.n_e + cp.n_i
        self.n_slots = n_slots
        hi = self.n if tgt_hi is None else tgt_hi
        self._cp = cp.c()          # kept alive: the C side holds a pointer
        self._h = _load().orc_mt_create(C.byref(self._cp), n_threads, n_slots,
                                        tgt_lo, hi)
        if not self._h:
            raise MemoryError("oracle: per-thread stores do not fit")
        self.n_threads = _load().orc_mt_threads(self._h)

    def ranges(self):
        out = []
        for k in range(self.n_threads):
            lo, hi = np.zeros(1, np.uint32), np.zeros(1, np.uint32)
            _load().orc_mt_range(self._h, k, _ptr(lo), _ptr(hi))
            out.append((int(lo[0]), int(hi[0])))
        return out

    def simulate(self, nm: Neuron, interval: int, st: State, rb: np.ndarray,
                 t0: int, n_steps: int, nu_ext_hz: float, w_ext: float,
                 seed: int, cap: int = 1 << 24):
        """Like ``simulate`` (in place on ``st`` and ``rb``); the threads
        must own the whole population."""
        rg = self.ranges()
        if rg[0][0] != 0 or rg[-1][1] != self.n:
            raise ValueError("a closed-network run needs every neuron")
        assert rb.shape == (self.n_slots, self.n) and rb.dtype == np.float64
        src = np.zeros(cap, np.uint32)
        tt = np.zeros(cap, np.int64)
        ev = C.c_uint64()
        ns = _load().orc_mt_simulate(self._h, C.byref(nm.c()), interval,
                                     _ptr(st.V), _ptr(st.I), _ptr(st.J),
                                     _ptr(st.refr), _ptr(rb), t0, n_steps,
                                     nu_ext_hz, w_ext, seed, _ptr(src),
                                     _ptr(tt), cap, C.byref(ev))
        if ns == 2 ** 64 - 1:
            raise MemoryError("oracle: interval lists do not fit")
        ns = min(int(ns), cap)
        return src[:ns].copy(), tt[:ns].copy(), int(ev.value)

    def update(self, nm: Neuron, st: State, rb: np.ndarray, t0: int,
               n_steps: int, nu_ext_hz: float, w_ext: float, seed: int) -> int:
        """The owned neurons' update (arrays indexed globally, in place);
        returns the number of spikes (not kept)."""
        assert rb.shape == (self.n_slots, self.n) and len(st.V) == self.n
        return int(_load().orc_mt_update(
            self._h, C.byref(nm.c()), _ptr(st.V), _ptr(st.I), _ptr(st.J),
            _ptr(st.refr), _ptr(rb), t0, n_steps, nu_ext_hz, w_ext, seed))

    def deliver(self, src, t, rb=None):
        """Algorithm REF of one list onto all targets; returns (rb, events)."""
        src, t = _spikes(src, t)
        if rb is None:
            rb = np.zeros((self.n_slots, self.n))
        ev = _load().orc_mt_deliver(self._h, len(src), _ptr(src), _ptr(t),
                                    _ptr(rb))
        return rb, int(ev)

    def close(self):
        if self._h:
            _load().orc_mt_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# Plasticity (Section 6; readings in the C source)
# --------------------------------------------------------------------------
@dataclass
class Stdp:
    """Pair-based power-law STDP of E->E synapses."""
    n_exc: int
    tau_plus: float = 20.0   # ms
    tau_minus: float = 20.0  # ms
    lam: float = 0.1
    alpha: float = 0.0513
    mu: float = 0.4
    w0: float = 1.0          # pA
    w_max: float = 100.0     # pA
    h: float = 0.1           # ms

    def c(self) -> StdpC:
        return StdpC(self.h, self.tau_plus, self.tau_minus, self.lam,
                     self.alpha, self.mu, self.w0, self.w_max, self.n_exc)


class History:
    """Every spike of every neuron so far (``cap`` per neuron)."""

    def __init__(self, n: int, cap: int = 4096):
        self.n, self.cap = n, cap
        self.t = np.zeros((n, cap), np.int64)
        self.count = np.zeros(n, np.uint32)

    def c(self) -> HistC:
        return HistC(self.n, self.cap, self.t.ctypes.data, self.count.ctypes.data)

    def add(self, src, t):
        src, t = _spikes(src, t)
        h = self.c()
        if _load().orc_hist_add(C.byref(h), len(src), _ptr(src), _ptr(t)) != 0:
            raise ValueError("spike history full")

    def spikes(self, i: int) -> np.ndarray:
        return self.t[i, :self.count[i]].copy()


def deliver_stdp(st: Store, w: np.ndarray, p: Stdp, hist: History,
                 n_slots: int, src, t, rb=None):
    """Delivery with plastic E->E weights (``w`` updated in place; the
    history must hold every spike up to the list's steps).  Returns
    (rb, absw, events)."""
    src, t = _spikes(src, t)
    assert w.dtype == np.float64 and len(w) == len(st.tgt)
    if rb is None:
        rb = np.zeros((n_slots, st.n))
    absw = np.zeros((n_slots, st.n))
    ev = _load().orc_deliver_stdp(C.byref(st.c(n_slots)), _ptr(w),
                                  C.byref(p.c()), C.byref(hist.c()), len(src),
                                  _ptr(src), _ptr(t), _ptr(rb), _ptr(absw))
    return rb, absw, int(ev)


def simulate_stdp(nm: Neuron, store: Store, w: np.ndarray, p: Stdp,
                  n_slots: int, interval: int, st: State, rb: np.ndarray,
                  t0: int, n_steps: int, nu_ext_hz: float, w_ext: float,
                  seed: int, hist: History):
    """Time-driven cycle with plastic delivery: update one interval, record
    its spikes, deliver them (weights in ``w`` change).  In place.  Returns
    (spike sources, spike steps, events)."""
    out_s, out_t, events = [], [], 0
    t = t0
    while t < t0 + n_steps:
        m = min(interval, t0 + n_steps - t)
        s_i, s_t = update(nm, st, rb, t, m, nu_ext_hz, w_ext, seed)
        hist.add(s_i, s_t)
        _, _, ev = deliver_stdp(store, w, p, hist, n_slots, s_i, s_t, rb)
        events += ev
        out_s.append(s_i)
        out_t.append(s_t)
        t += m
    return np.concatenate(out_s), np.concatenate(out_t), events
