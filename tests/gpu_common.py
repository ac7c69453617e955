"""Helpers shared by the GPU parity tests (not a test module)."""
import numpy as np
import pytest

import oracle as O

S = 32


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2109_12855_gb300 as pkg
    pkg.build()
    return torch


def stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def fixed_net(n_e, n_i, k_e, k_i, w_e, w_i, d_lo, d_hi, seed, fmt=0,
              sd_e=0.0, sd_i=0.0, **pkw):
    """GPU net + matching oracle connection rule (weights rounded as stored)."""
    from paper_2109_12855_gb300 import snn
    pkw.setdefault("count_events", 1)
    p = snn.params(n_exc=n_e, n_inh=n_i, weight_format=fmt, **pkw)
    net = snn.Net(p, stream())
    net.connect_fixed_indegree(snn.conn_params(
        k_exc=k_e, k_inh=k_i, w_exc=w_e, w_inh=w_i, sd_exc=sd_e, sd_inh=sd_i,
        d_lo=d_lo, d_hi=d_hi, seed=seed, clip_exc=1, clip_inh=0))
    net.finalize()
    cp = O.Conn(n_e, n_i, k_e, k_i, w_e, w_i, d_lo, d_hi, seed, sd_e=sd_e,
                sd_i=sd_i, clip_e=True, clip_i=False, wfmt=1 if fmt == 0 else 2)
    return net, cp


def edge_net(n, edges, fmt=0, **pkw):
    from paper_2109_12855_gb300 import snn
    src, tgt, d, w = edges
    p = snn.params(n_exc=n, n_inh=0, weight_format=fmt, count_events=1, **pkw)
    net = snn.Net(p, stream())
    net.connect_edges(src, tgt, d, w)
    net.finalize()
    rnd = O.round_f32 if fmt == 0 else O.round_bf16
    wr = np.array([rnd(float(x)) for x in w])
    store = O.build_edges(n, src, tgt, d, wr)
    return net, store


def check_delivery(net, store, src, t, n_slots=S, reset=True):
    """Deliver (src, t) on the GPU and through Algorithm REF; event count and
    per-cell counts bit-exact, values within 1e-5 sum|w| per cell."""
    from paper_2109_12855_gb300 import snn
    if reset:
        snn.snn_clear_rb(net.h)
    ev = net.deliver(src, np.asarray(t, np.int32))
    rb = net.read_rb()
    cnt = net.read_counts()
    rb_o, cnt_o, absw, ev_o = O.deliver_ref(store, n_slots, src,
                                            np.asarray(t, np.int64))
    assert ev == ev_o
    assert np.array_equal(cnt.astype(np.int64), cnt_o.astype(np.int64))
    err = np.abs(rb.astype(np.float64) - rb_o)
    assert np.all(err <= 1e-5 * absw), float((err - 1e-5 * absw).max())
    return ev, rb, rb_o, absw
