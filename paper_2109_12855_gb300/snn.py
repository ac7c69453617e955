"""Thin ctypes binding of libsnn (``include/snn.h``): same names, argument
marshalling only.  Every computation runs in the CUDA library; there is no
fallback -- importing this module without the built library raises.

Buffers may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); the binding passes the matching ``SNN_MEM_*`` flag.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .native import lib_path

LIB = lib_path()

SNN_OK = 0
SNN_E_OOM, SNN_E_ARG, SNN_E_STATE, SNN_E_TIMEOUT, SNN_E_OVERFLOW, SNN_E_CUDA = \
    -1, -2, -3, -4, -5, -6
SNN_MEM_HOST, SNN_MEM_DEVICE = 0, 1
SNN_T_DEVICE = -1  # snn_update: start at the device clock
SNN_W_FP32_12B, SNN_W_BF16_8B = 0, 1
SNN_DELIVER_TILED, SNN_DELIVER_ATOMIC = 0, 1
SNN_ERRF_SPIKE_LIST, SNN_ERRF_SPIKE_LOG, SNN_ERRF_BAD_SOURCE, SNN_ERRF_CHUNKS = \
    1, 2, 4, 8
SNN_ERRF_TIMEOUT = 16
SNN_ERRF_SCALES = 32
SNN_ERRF_CHECK = 64

EXPORTS = [
    "snn_abi_version", "snn_last_error", "snn_default_params",
    "snn_psc_weight_for_psp", "snn_create", "snn_connect_fixed_indegree",
    "snn_connect_edges", "snn_finalize", "snn_update", "snn_deliver_pending",
    "snn_discard_pending", "snn_deliver", "snn_deliver_noalloc",
    "snn_simulate", "snn_read_spikes",
    "snn_read_rb", "snn_write_rb", "snn_read_counts", "snn_clear_rb",
    "snn_read_state", "snn_write_state", "snn_read_store", "snn_state_size",
    "snn_save_state", "snn_load_state", "snn_set_drive",
    "snn_set_time",
    "snn_set_profiling", "snn_get_stats", "snn_clear_errors", "snn_sync",
    "snn_destroy", "snn_server_create", "snn_server_submit", "snn_server_step",
    "snn_server_poll", "snn_server_spikes", "snn_server_release",
    "snn_server_get_stats", "snn_server_destroy", "snn_set_stdp",
    "snn_read_weights", "snn_read_spike_stats", "snn_clear_spike_stats",
    "snn_read_pending", "snn_get_bounds", "snn_set_bounds",
    "snn_deliver_gathered", "snn_server_set_option", "snn_server_cancel",
    "snn_debug_fail_allocations", "snn_exchange_capacity",
    "snn_set_exchange", "snn_deliver_exchanged", "snn_get_stream",
    "snn_checked", "snn_debug_check_failures", "snn_debug_poke_record",
    "snn_probe_reductions",
]
SNN_REQ_QUEUED, SNN_REQ_BUILDING, SNN_REQ_RUNNING, SNN_REQ_DONE = 0, 1, 2, 3
SNN_REQ_FAILED = -1
SNN_REQ_CANCELLED = 4


class SnnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libsnn error {code}: {msg}")
        self.code = code


class snn_params(C.Structure):
    _fields_ = [("n_exc", C.c_uint32), ("n_inh", C.c_uint32),
                ("h", C.c_double), ("tau_m", C.c_double), ("c_m", C.c_double),
                ("v_th", C.c_double), ("v_reset", C.c_double),
                ("t_ref", C.c_double), ("tau_syn", C.c_double),
                ("nu_ext", C.c_double), ("w_ext", C.c_double),
                ("seed", C.c_uint64), ("weight_format", C.c_int32),
                ("n_slots", C.c_int32), ("interval", C.c_int32),
                ("init_v_random", C.c_int32), ("count_events", C.c_int32),
                ("deliver_mode", C.c_int32), ("spike_log_capacity", C.c_uint64),
                ("tile_width", C.c_int32), ("stream_priority", C.c_int32),
                ("part_lo", C.c_uint32), ("part_hi", C.c_uint32),
                ("acc_words", C.c_int32), ("build_yield", C.c_int32)]


class snn_conn_params(C.Structure):
    _fields_ = [("k_exc", C.c_uint32), ("k_inh", C.c_uint32),
                ("w_exc", C.c_double), ("w_inh", C.c_double),
                ("sd_exc", C.c_double), ("sd_inh", C.c_double),
                ("d_lo", C.c_int32), ("d_hi", C.c_int32), ("seed", C.c_uint64),
                ("clip_exc", C.c_int32), ("clip_inh", C.c_int32)]


class snn_stats(C.Structure):
    _fields_ = [("events_delivered", C.c_uint64), ("spikes", C.c_uint64),
                ("n_synapses", C.c_uint64), ("t_now", C.c_int64),
                ("interval", C.c_int32), ("min_delay", C.c_int32),
                ("max_delay", C.c_int32), ("error_flags", C.c_uint32),
                ("kernel_launches", C.c_uint64),
                ("update_launches", C.c_uint64),
                ("deliver_launches", C.c_uint64), ("ms_update", C.c_double),
                ("ms_deliver", C.c_double), ("bytes_per_record", C.c_uint64),
                ("store_bytes", C.c_uint64), ("n_tiles", C.c_uint32),
                ("tile_width", C.c_uint32), ("window", C.c_int32),
                ("deliver_mode", C.c_int32), ("plastic_events", C.c_uint64),
                ("stdp_truncated", C.c_uint64), ("first_neuron", C.c_uint32),
                ("n_sources", C.c_uint32), ("acc_words", C.c_int32),
                ("reserved_", C.c_int32)]


class snn_bounds(C.Structure):
    _fields_ = [("mult_max", C.c_uint32), ("k_in_max", C.c_uint32),
                ("max_abs_w", C.c_float), ("reserved_", C.c_uint32)]


class snn_stdp_params(C.Structure):
    _fields_ = [("tau_plus", C.c_double), ("tau_minus", C.c_double),
                ("lam", C.c_double), ("alpha", C.c_double), ("mu", C.c_double),
                ("w0", C.c_double), ("w_max", C.c_double),
                ("history", C.c_int32), ("reserved_", C.c_int32)]


class snn_request(C.Structure):
    _fields_ = [("params", snn_params), ("conn", snn_conn_params),
                ("n_steps", C.c_int64), ("user_tag", C.c_uint64),
                ("record_spikes", C.c_int32), ("pad_", C.c_int32)]


class snn_result(C.Structure):
    _fields_ = [("id", C.c_uint64), ("user_tag", C.c_uint64),
                ("state", C.c_int32), ("error", C.c_int32),
                ("n_neurons", C.c_uint64), ("n_synapses", C.c_uint64),
                ("spikes", C.c_uint64), ("events", C.c_uint64),
                ("n_steps", C.c_int64), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double), ("bytes", C.c_uint64)]


class snn_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("done", C.c_uint64),
                ("failed", C.c_uint64), ("active", C.c_uint64),
                ("queued", C.c_uint64), ("steps", C.c_uint64),
                ("intervals", C.c_uint64), ("kernel_launches", C.c_uint64),
                ("events", C.c_uint64), ("spikes", C.c_uint64),
                ("mem_budget", C.c_uint64), ("mem_used", C.c_uint64),
                ("intervals_per_step", C.c_int32), ("tuned", C.c_int32),
                ("gpu_ms", C.c_double)]


_P = C.c_void_p
_lib = None


def lib():
    """Load libsnn.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(
                f"{LIB} is missing: run `python -m paper_2109_12855_gb300.native` "
                "(there is no CPU fallback)")
        L = C.CDLL(LIB)
        sig = {
            "snn_abi_version": ([], C.c_int),
            "snn_last_error": ([], C.c_char_p),
            "snn_default_params": ([C.POINTER(snn_params)], C.c_int),
            "snn_psc_weight_for_psp": ([C.POINTER(snn_params), C.c_double,
                                        C.POINTER(C.c_double)], C.c_int),
            "snn_create": ([C.POINTER(snn_params), _P, C.POINTER(_P)], C.c_int),
            "snn_connect_fixed_indegree": ([_P, C.POINTER(snn_conn_params)],
                                           C.c_int),
            "snn_connect_edges": ([_P, _P, _P, _P, _P, C.c_uint64, C.c_int],
                                  C.c_int),
            "snn_finalize": ([_P], C.c_int),
            "snn_update": ([_P, C.c_int64, C.c_int32], C.c_int),
            "snn_deliver_pending": ([_P], C.c_int),
            "snn_discard_pending": ([_P], C.c_int),
            "snn_deliver": ([_P, _P, _P, C.c_uint32, C.c_int,
                             C.POINTER(C.c_uint64)], C.c_int),
            "snn_deliver_noalloc": ([_P, _P, _P, C.c_uint32,
                                     C.POINTER(C.c_uint64)], C.c_int),
            "snn_simulate": ([_P, C.c_int64], C.c_int),
            "snn_read_spikes": ([_P, _P, _P, C.c_uint64, C.POINTER(C.c_uint64),
                                 C.c_int], C.c_int),
            "snn_read_rb": ([_P, _P, C.c_int], C.c_int),
            "snn_write_rb": ([_P, _P, C.c_int], C.c_int),
            "snn_read_counts": ([_P, _P, C.c_int], C.c_int),
            "snn_clear_rb": ([_P], C.c_int),
            "snn_read_state": ([_P, _P, _P, _P, _P, C.c_int], C.c_int),
            "snn_write_state": ([_P, _P, _P, _P, _P, C.c_int], C.c_int),
            "snn_read_store": ([_P, _P, _P, _P, _P, C.c_int], C.c_int),
            "snn_state_size": ([_P, C.POINTER(C.c_uint64)], C.c_int),
            "snn_save_state": ([_P, _P, C.c_uint64], C.c_int),
            "snn_load_state": ([_P, _P, C.c_uint64], C.c_int),
            "snn_set_drive": ([_P, C.c_double, C.c_double], C.c_int),
            "snn_set_time": ([_P, C.c_int64], C.c_int),
            "snn_set_profiling": ([_P, C.c_int], C.c_int),
            "snn_get_stats": ([_P, C.POINTER(snn_stats)], C.c_int),
            "snn_clear_errors": ([_P], C.c_int),
            "snn_sync": ([_P], C.c_int),
            "snn_destroy": ([_P], C.c_int),
            "snn_set_stdp": ([_P, C.POINTER(snn_stdp_params)], C.c_int),
            "snn_read_weights": ([_P, _P, C.c_int32], C.c_int),
            "snn_read_spike_stats": ([_P, _P, _P, _P, _P], C.c_int),
            "snn_clear_spike_stats": ([_P], C.c_int),
            "snn_read_pending": ([_P, _P, _P, C.c_uint64,
                                  C.POINTER(C.c_uint64), C.c_int32], C.c_int),
            "snn_get_bounds": ([_P, C.POINTER(snn_bounds)], C.c_int),
            "snn_deliver_gathered": ([_P, _P, _P, C.c_uint32, C.c_int32,
                                      C.POINTER(C.c_uint64)], C.c_int),
            "snn_set_bounds": ([_P, C.POINTER(snn_bounds)], C.c_int),
            "snn_server_create": ([C.c_uint64, C.c_int32, _P, C.POINTER(_P)],
                                  C.c_int),
            "snn_server_submit": ([_P, C.POINTER(snn_request),
                                   C.POINTER(C.c_uint64)], C.c_int),
            "snn_server_step": ([_P, C.POINTER(C.c_int32)], C.c_int),
            "snn_server_poll": ([_P, C.c_uint64, C.POINTER(snn_result)], C.c_int),
            "snn_server_spikes": ([_P, C.c_uint64, _P, _P, C.c_uint64,
                                   C.POINTER(C.c_uint64)], C.c_int),
            "snn_server_release": ([_P, C.c_uint64], C.c_int),
            "snn_server_get_stats": ([_P, C.POINTER(snn_server_stats)], C.c_int),
            "snn_server_destroy": ([_P], C.c_int),
            "snn_server_set_option": ([_P, C.c_int32, C.c_double], C.c_int),
            "snn_server_cancel": ([_P, C.c_uint64], C.c_int),
            "snn_exchange_capacity": ([_P, C.POINTER(C.c_uint64)], C.c_int),
            "snn_get_stream": ([_P, C.POINTER(C.c_void_p)], C.c_int),
            "snn_checked": ([], C.c_int),
            "snn_debug_check_failures": ([], C.c_uint64),
            "snn_probe_reductions": ([C.c_void_p, C.c_uint64, C.c_uint64,
                                      C.c_int, C.c_void_p,
                                      C.POINTER(C.c_float)], C.c_int),
            "snn_debug_poke_record": ([_P, C.c_uint64, C.c_int, C.c_uint32],
                                      C.c_int),
            "snn_set_exchange": ([_P, _P, C.c_uint64], C.c_int),
            "snn_deliver_exchanged": ([_P, _P, C.c_uint32, C.c_uint64],
                                      C.c_int),
            "snn_debug_fail_allocations": ([C.c_int64, C.c_int64], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc: int):
    if rc != SNN_OK:
        raise SnnError(rc, lib().snn_last_error().decode(errors="replace"))
    return rc


def _buf(x, dtype=None):
    """(pointer, mem kind) of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None, SNN_MEM_HOST
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "array must be contiguous"
        if dtype is not None:
            assert x.dtype == dtype, f"expected {dtype}, got {x.dtype}"
        return x.ctypes.data, SNN_MEM_HOST
    # torch tensor
    assert x.is_contiguous(), "tensor must be contiguous"
    return x.data_ptr(), (SNN_MEM_DEVICE if x.is_cuda else SNN_MEM_HOST)


def _mem_of(*xs):
    kinds = {_buf(x)[1] for x in xs if x is not None}
    assert len(kinds) <= 1, "buffers of one call must share a memory kind"
    return kinds.pop() if kinds else SNN_MEM_HOST


# --- same-named wrappers ----------------------------------------------------
def snn_abi_version() -> int:
    return lib().snn_abi_version()


def snn_default_params() -> snn_params:
    p = snn_params()
    _check(lib().snn_default_params(C.byref(p)))
    return p


def snn_psc_weight_for_psp(p: snn_params, psp_mv: float) -> float:
    w = C.c_double()
    _check(lib().snn_psc_weight_for_psp(C.byref(p), psp_mv, C.byref(w)))
    return w.value


def snn_create(p: snn_params, stream: int | None = None):
    h = _P()
    _check(lib().snn_create(C.byref(p), stream or None, C.byref(h)))
    return h


def snn_connect_fixed_indegree(net, c: snn_conn_params):
    _check(lib().snn_connect_fixed_indegree(net, C.byref(c)))


def snn_connect_edges(net, src, tgt, delay, w):
    mem = _mem_of(src, tgt, delay, w)
    _check(lib().snn_connect_edges(net, _buf(src)[0], _buf(tgt)[0],
                                   _buf(delay)[0], _buf(w)[0], len(src), mem))


def snn_finalize(net):
    _check(lib().snn_finalize(net))


def snn_update(net, t0: int, n_steps: int):
    _check(lib().snn_update(net, t0, n_steps))


def snn_deliver_pending(net):
    _check(lib().snn_deliver_pending(net))


def snn_discard_pending(net):
    _check(lib().snn_discard_pending(net))


def snn_deliver(net, src, t_emit, want_events: bool = True):
    mem = _mem_of(src, t_emit)
    ev = C.c_uint64()
    _check(lib().snn_deliver(net, _buf(src)[0], _buf(t_emit)[0], len(src), mem,
                             C.byref(ev) if want_events else None))
    return ev.value if want_events else None


# the scratch capacity, SNN_NOALLOC_MAX_SPIKES of include/snn.h (a test
# checks that the two agree)
SNN_NOALLOC_MAX_SPIKES = 1 << 18


def snn_deliver_noalloc(net, src, t_emit, want_events: bool = True):
    """Allocation-free delivery; src/t_emit must be CUDA tensors."""
    ps, ms = _buf(src)
    pt, mt = _buf(t_emit)
    if not (ms == mt == SNN_MEM_DEVICE):
        raise ValueError("snn_deliver_noalloc: spike arrays must be device "
                         "memory (CUDA tensors)")
    ev = C.c_uint64()
    _check(lib().snn_deliver_noalloc(net, ps, pt, len(src),
                                     C.byref(ev) if want_events else None))
    return ev.value if want_events else None


def snn_simulate(net, n_steps: int):
    _check(lib().snn_simulate(net, n_steps))


def snn_read_spikes(net, src, t):
    """Fills src/t (capacity len(src)); returns the number logged."""
    n = C.c_uint64()
    mem = _mem_of(src, t)
    rc = lib().snn_read_spikes(net, _buf(src)[0], _buf(t)[0], len(src),
                               C.byref(n), mem)
    if rc not in (SNN_OK, SNN_E_OVERFLOW):
        _check(rc)
    return n.value


def snn_read_rb(net, dst):
    p, mem = _buf(dst)
    _check(lib().snn_read_rb(net, p, mem))


def snn_write_rb(net, src):
    p, mem = _buf(src)
    _check(lib().snn_write_rb(net, p, mem))


def snn_read_counts(net, dst):
    p, mem = _buf(dst)
    _check(lib().snn_read_counts(net, p, mem))


def snn_clear_rb(net):
    _check(lib().snn_clear_rb(net))


def snn_read_state(net, V=None, I=None, J=None, refr=None):
    mem = _mem_of(V, I, J, refr)
    _check(lib().snn_read_state(net, _buf(V)[0], _buf(I)[0], _buf(J)[0],
                                _buf(refr)[0], mem))


def snn_write_state(net, V=None, I=None, J=None, refr=None):
    mem = _mem_of(V, I, J, refr)
    _check(lib().snn_write_state(net, _buf(V)[0], _buf(I)[0], _buf(J)[0],
                                 _buf(refr)[0], mem))


def snn_read_store(net, row_ptr=None, tgt=None, delay=None, w=None):
    mem = _mem_of(row_ptr, tgt, delay, w)
    _check(lib().snn_read_store(net, _buf(row_ptr)[0], _buf(tgt)[0],
                                _buf(delay)[0], _buf(w)[0], mem))


def stdp_params(**kw) -> snn_stdp_params:
    """Power-law STDP defaults (tau 20 ms, lambda 0.1, alpha 0.0513,
    mu 0.4, w0 1 pA, w_max 100 pA, 16 post spikes kept) with overrides."""
    q = snn_stdp_params(20.0, 20.0, 0.1, 0.0513, 0.4, 1.0, 100.0, 16, 0)
    for k, v in kw.items():
        if not hasattr(q, k):
            raise AttributeError(k)
        setattr(q, k, v)
    return q


def snn_set_stdp(net, q: snn_stdp_params):
    _check(lib().snn_set_stdp(net, C.byref(q)))


def snn_read_weights(net, w):
    mem = _mem_of(w)
    _check(lib().snn_read_weights(net, _buf(w)[0], mem))


def snn_read_spike_stats(net, n: int):
    """(spikes, intervals, interval sum, interval square sum) per neuron."""
    a = np.zeros(n, np.uint32)
    b = np.zeros(n, np.uint32)
    c = np.zeros(n, np.float64)
    d = np.zeros(n, np.float64)
    _check(lib().snn_read_spike_stats(net, a.ctypes.data, b.ctypes.data,
                                      c.ctypes.data, d.ctypes.data))
    return a, b, c, d


def snn_clear_spike_stats(net):
    _check(lib().snn_clear_spike_stats(net))


def snn_read_pending(net, src, t) -> int:
    """Pending interval list into src / t (numpy or device tensors); returns
    the number of spikes."""
    mem = _mem_of(src, t)
    n = C.c_uint64()
    cap = len(src) if hasattr(src, "__len__") else src.numel()
    _check(lib().snn_read_pending(net, _buf(src)[0], _buf(t)[0], cap,
                                  C.byref(n), mem))
    return n.value


def snn_deliver_gathered(net, src, t, want_events: bool = True) -> int:
    """Deliver the gathered interval list (numpy uint32/int32 or device
    int32 tensors); returns the events this partition received (0 when
    want_events is false, which saves two synchronisations)."""
    mem = _mem_of(src, t)
    ev = C.c_uint64()
    n = len(src)
    _check(lib().snn_deliver_gathered(net, _buf(src)[0] if n else None,
                                      _buf(t)[0] if n else None, n, mem,
                                      C.byref(ev) if want_events else None))
    return ev.value


def snn_checked() -> bool:
    """True for the bounds-checked build of the library."""
    return bool(lib().snn_checked())


def snn_debug_check_failures() -> int:
    return int(lib().snn_debug_check_failures())


def snn_debug_poke_record(net, index: int, field: int, value: int):
    """Bounds-checked builds: corrupt one record's target (field 0) or delay
    (field 1)."""
    _check(lib().snn_debug_poke_record(net, index, field, value))


SNN_PROBE_SCATTER, SNN_PROBE_SWEEP = 0, 1


def snn_probe_reductions(buf, n_ops: int, pattern: int, stream: int = 0) -> float:
    """Time n_ops L2 reductions (+1.0f) into the device float tensor buf
    (scattered or sweeping cells); returns the launch's CUDA-event ms."""
    ptr, mem = _buf(buf)
    if mem != SNN_MEM_DEVICE or str(buf.dtype) != "torch.float32":
        raise ValueError("buf must be a float32 device tensor")
    ms = C.c_float()
    _check(lib().snn_probe_reductions(ptr, buf.numel(), n_ops, pattern,
                                      C.c_void_p(stream or None), C.byref(ms)))
    return float(ms.value)


def snn_get_stream(net) -> int:
    """The cudaStream_t (as an int; 0 for the legacy default stream) the
    net's work is enqueued on."""
    p = C.c_void_p()
    _check(lib().snn_get_stream(net, C.byref(p)))
    return p.value or 0


def snn_exchange_capacity(net) -> int:
    """Entries an exchange buffer of this partition needs (never overflows)."""
    n = C.c_uint64()
    _check(lib().snn_exchange_capacity(net, C.byref(n)))
    return n.value


def snn_set_exchange(net, buf, cap_entries: int | None = None):
    """Attach a device exchange buffer (a CUDA tensor of at least 16 + 8 cap
    bytes) or detach it (buf None)."""
    if buf is None:
        _check(lib().snn_set_exchange(net, None, 0))
        return
    ptr, mem = _buf(buf)
    if mem != SNN_MEM_DEVICE:
        raise ValueError("the exchange buffer must be a CUDA tensor")
    nbytes = buf.numel() * buf.element_size()
    if cap_entries is None:
        cap_entries = (nbytes - 16) // 8
    if nbytes < 16 + 8 * cap_entries:
        raise ValueError(f"{nbytes} bytes hold fewer than {cap_entries} entries")
    _check(lib().snn_set_exchange(net, ptr, cap_entries))


def snn_deliver_exchanged(net, parts, n_parts: int | None = None,
                          stride_bytes: int | None = None):
    """Deliver the pending interval from gathered exchange buffers: a CUDA
    tensor whose first dimension is the parts (each row one buffer), or a
    raw device pointer with n_parts and stride_bytes."""
    if isinstance(parts, int):
        ptr = parts
    else:
        ptr, mem = _buf(parts)
        if mem != SNN_MEM_DEVICE:
            raise ValueError("gathered exchange buffers must be a CUDA tensor")
        if n_parts is None:
            n_parts = parts.shape[0]
        if stride_bytes is None:
            stride_bytes = parts.stride(0) * parts.element_size()
    _check(lib().snn_deliver_exchanged(net, ptr, n_parts, stride_bytes))


def snn_get_bounds(net) -> snn_bounds:
    b = snn_bounds()
    _check(lib().snn_get_bounds(net, C.byref(b)))
    return b


def snn_set_bounds(net, b: snn_bounds):
    _check(lib().snn_set_bounds(net, C.byref(b)))


def snn_state_size(net) -> int:
    n = C.c_uint64()
    _check(lib().snn_state_size(net, C.byref(n)))
    return n.value


def snn_save_state(net) -> bytes:
    """Checkpoint image of the net's dynamic state (bytes)."""
    n = snn_state_size(net)
    buf = (C.c_char * n)()
    _check(lib().snn_save_state(net, buf, n))
    return bytes(buf)


def snn_load_state(net, image: bytes):
    buf = C.create_string_buffer(image, len(image))
    _check(lib().snn_load_state(net, buf, len(image)))


def snn_set_drive(net, nu_ext: float, w_ext: float):
    _check(lib().snn_set_drive(net, nu_ext, w_ext))


def snn_set_time(net, t: int):
    _check(lib().snn_set_time(net, t))


def snn_set_profiling(net, on: bool):
    _check(lib().snn_set_profiling(net, int(on)))


def snn_get_stats(net) -> snn_stats:
    s = snn_stats()
    _check(lib().snn_get_stats(net, C.byref(s)))
    return s


def snn_clear_errors(net):
    _check(lib().snn_clear_errors(net))


def snn_sync(net):
    _check(lib().snn_sync(net))


def snn_destroy(net):
    _check(lib().snn_destroy(net))


# --- convenience ------------------------------------------------------------
def params(**kw) -> snn_params:
    """Defaults of ``snn_default_params`` with fields overridden by ``kw``."""
    p = snn_default_params()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def conn_params(**kw) -> snn_conn_params:
    c = snn_conn_params()
    c.clip_exc = 1
    for k, v in kw.items():
        if not hasattr(c, k):
            raise AttributeError(k)
        setattr(c, k, v)
    return c


class Net:
    """Owning wrapper around an ``snn_net*`` handle."""

    def __init__(self, p: snn_params, stream: int | None = None):
        self.p = p
        part = p.part_hi != 0 or p.part_lo != 0
        self.n_src = p.n_exc + p.n_inh          # store rows: every source
        self.n = p.part_hi - p.part_lo if part else self.n_src  # local
        self.h = snn_create(p, stream)

    def close(self):
        if self.h:
            snn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # pass-throughs
    def connect_fixed_indegree(self, c):
        snn_connect_fixed_indegree(self.h, c)

    def connect_edges(self, src, tgt, delay, w):
        snn_connect_edges(self.h, np.ascontiguousarray(src, np.uint32),
                          np.ascontiguousarray(tgt, np.uint32),
                          np.ascontiguousarray(delay, np.uint8),
                          np.ascontiguousarray(w, np.float64))

    def finalize(self):
        snn_finalize(self.h)

    def stats(self) -> snn_stats:
        return snn_get_stats(self.h)

    def read_rb(self) -> np.ndarray:
        out = np.zeros((self.p.n_slots, self.n), np.float32)
        snn_read_rb(self.h, out)
        return out

    def read_counts(self) -> np.ndarray:
        out = np.zeros((self.p.n_slots, self.n), np.uint32)
        snn_read_counts(self.h, out)
        return out

    def read_state(self):
        V = np.zeros(self.n, np.float32)
        I = np.zeros(self.n, np.float32)
        J = np.zeros(self.n, np.float32)
        r = np.zeros(self.n, np.int32)
        snn_read_state(self.h, V, I, J, r)
        return V, I, J, r

    def write_state(self, V, I, J, refr):
        snn_write_state(self.h, np.ascontiguousarray(V, np.float32),
                        np.ascontiguousarray(I, np.float32),
                        np.ascontiguousarray(J, np.float32),
                        np.ascontiguousarray(refr, np.int32))

    def read_store(self):
        st = self.stats()
        m = st.n_synapses
        rp = np.zeros(self.n_src + 1, np.uint64)
        tg = np.zeros(max(m, 1), np.uint32)
        dl = np.zeros(max(m, 1), np.uint8)
        w = np.zeros(max(m, 1), np.float32)
        snn_read_store(self.h, rp, tg, dl, w)
        return rp, tg[:m], dl[:m], w[:m]

    def read_weights(self):
        m = self.stats().n_synapses
        w = np.zeros(max(m, 1), np.float32)
        snn_read_weights(self.h, w)
        return w[:m]

    def deliver(self, src, t):
        return snn_deliver(self.h, np.ascontiguousarray(src, np.uint32),
                           np.ascontiguousarray(t, np.int32))

    def read_spikes(self, cap: int | None = None):
        cap = cap or max(self.p.spike_log_capacity, 1)
        src = np.zeros(cap, np.uint32)
        t = np.zeros(cap, np.int32)
        n = snn_read_spikes(self.h, src, t)
        k = min(n, cap)
        return src[:k], t[:k]


# --- serving ----------------------------------------------------------------
def snn_server_create(mem_budget: int, weight_format: int, stream=None):
    h = _P()
    _check(lib().snn_server_create(mem_budget, weight_format, stream or None,
                                   C.byref(h)))
    return h


def snn_server_submit(sv, req: snn_request) -> int:
    i = C.c_uint64()
    _check(lib().snn_server_submit(sv, C.byref(req), C.byref(i)))
    return i.value


def snn_server_step(sv) -> int:
    n = C.c_int32()
    _check(lib().snn_server_step(sv, C.byref(n)))
    return n.value


def snn_server_poll(sv, rid: int) -> snn_result:
    r = snn_result()
    _check(lib().snn_server_poll(sv, rid, C.byref(r)))
    return r


def snn_server_spikes(sv, rid: int):
    n = C.c_uint64()
    rc = lib().snn_server_spikes(sv, rid, None, None, 0, C.byref(n))
    if rc not in (SNN_OK, SNN_E_OVERFLOW):
        _check(rc)
    src = np.zeros(max(n.value, 1), np.uint32)
    t = np.zeros(max(n.value, 1), np.int32)
    _check(lib().snn_server_spikes(sv, rid, src.ctypes.data, t.ctypes.data,
                                   n.value, C.byref(n)))
    return src[:n.value], t[:n.value]


def snn_server_release(sv, rid: int):
    _check(lib().snn_server_release(sv, rid))


def snn_server_get_stats(sv) -> snn_server_stats:
    st = snn_server_stats()
    _check(lib().snn_server_get_stats(sv, C.byref(st)))
    return st


SNN_SERVE_OPT_PERSISTENT, SNN_SERVE_OPT_SPIN_LIMIT, SNN_SERVE_OPT_STEP_US = 0, 1, 2
SNN_SERVE_OPT_EXCLUSIVE = 3


def snn_server_set_option(sv, option: int, value: float):
    _check(lib().snn_server_set_option(sv, option, float(value)))


def snn_server_cancel(sv, rid: int):
    _check(lib().snn_server_cancel(sv, rid))


def snn_debug_fail_allocations(after: int, count: int = 1):
    _check(lib().snn_debug_fail_allocations(after, count))


def snn_server_destroy(sv):
    _check(lib().snn_server_destroy(sv))


def request(params: snn_params, conn: snn_conn_params, n_steps: int,
            user_tag: int = 0, record_spikes: bool = False) -> snn_request:
    r = snn_request()
    r.params = params
    r.conn = conn
    r.n_steps = n_steps
    r.user_tag = user_tag
    r.record_spikes = int(record_spikes)
    return r
