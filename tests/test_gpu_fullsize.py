"""Delivery at the benchmark sizes, in the launch configuration the benchmark
times: 112,500 neurons x 11,250 synapses (1.27e9, FP32 12-byte records,
delay 15 steps) and 562,500 x 11,250 (6.3e9, BF16 8-byte records, delays
10..20, weights N(J, 0.1 J) / N(-5 J, 0.5 J)).  The oracle cannot hold these
stores; it regenerates the incoming synapses of sampled targets from the
connection rule's definition and computes their ring-buffer columns one by
one.  Properties that hold at any size are checked for every target."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import S, need_gpu, stream

pytestmark = pytest.mark.gpu

NM = O.Neuron()
W_E = O.weight_for_psp(NM, 0.1)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _column(cp, j, spikes_by_src):
    """Oracle ring-buffer column of target j: (rb[S], counts[S], sum|w|[S])."""
    src, d, w = O.incoming(cp, j)
    col = np.zeros(S)
    cnt = np.zeros(S, np.int64)
    absw = np.zeros(S)
    for s, dd, ww in zip(src.tolist(), d.tolist(), w.tolist()):
        for t in spikes_by_src.get(s, ()):
            slot = (t + dd) % S
            col[slot] += ww
            cnt[slot] += 1
            absw[slot] += abs(ww)
    return col, cnt, absw


def _by_src(src, t):
    out = {}
    for s, tt in zip(src.tolist(), t.tolist()):
        out.setdefault(s, []).append(tt)
    return out


def _run(wl, fmt, sd, seed):
    from paper_2109_12855_gb300 import snn
    p = snn.params(n_exc=wl.n_e, n_inh=wl.n_i, weight_format=fmt,
                   count_events=1)
    net = snn.Net(p, stream())
    c = snn.conn_params(k_exc=wl.k_e, k_inh=wl.k_i, w_exc=W_E,
                        w_inh=-wl.g * W_E, sd_exc=sd * W_E,
                        sd_inh=sd * wl.g * W_E, d_lo=wl.d_lo, d_hi=wl.d_hi,
                        seed=seed, clip_exc=1, clip_inh=0)
    net.connect_fixed_indegree(c)
    net.finalize()
    cp = O.Conn(wl.n_e, wl.n_i, wl.k_e, wl.k_i, W_E, -wl.g * W_E, wl.d_lo,
                wl.d_hi, seed, sd_e=sd * W_E, sd_i=sd * wl.g * W_E,
                clip_e=True, clip_i=False, wfmt=1 if fmt == 0 else 2)
    return net, cp


def _check_sampled(net, cp, wl, src, t, n_targets, seed):
    from paper_2109_12855_gb300 import snn
    snn.snn_clear_rb(net.h)
    ev = net.deliver(src, t.astype(np.int32))
    rb = net.read_rb()
    cnt = net.read_counts()
    rp = np.zeros(wl.n + 1, np.uint64)
    snn.snn_read_store(net.h, rp)
    deg = np.diff(rp.astype(np.int64))
    assert ev == int(deg[src].sum())
    assert int(cnt.sum(dtype=np.int64)) == ev
    sp = _by_src(src, t)
    g = W.rng(seed)
    for j in g.choice(wl.n, n_targets, replace=False).tolist():
        col, c, absw = _column(cp, j, sp)
        assert np.array_equal(cnt[:, j].astype(np.int64), c), j
        assert np.all(np.abs(rb[:, j] - col) <= 1e-5 * absw), j
    return rb, cnt


def test_balanced_112500_fp32_delivery():
    wl = W.BALANCED_112500
    net, cp = _run(wl, 0, 0.0, seed=2)
    with net:
        st = net.stats()
        assert st.n_synapses == wl.n_synapses == 1_265_625_000
        assert st.interval == 15 and st.min_delay == st.max_delay == 15
        # one interval of ~8 Hz activity (about 1,350 spikes)
        src, t = W.bernoulli_spikes(wl.n, 300, 15, 8.0, 0.1, seed=3)
        _check_sampled(net, cp, wl, src, t, 48, seed=4)
        # every source fires once: each target receives exactly K events in
        # slot 15 (complete in-degree check of the whole store)
        src = np.arange(wl.n, dtype=np.uint32)
        from paper_2109_12855_gb300 import snn
        snn.snn_clear_rb(net.h)
        ev = net.deliver(src, np.zeros(wl.n, np.int32))
        assert ev == wl.n_synapses
        cnt = net.read_counts()
        assert np.all(cnt[15] == wl.k) and cnt.sum(dtype=np.int64) == ev
        rb = net.read_rb()
        want = wl.k_e * np.float32(W_E) - wl.k_i * np.float32(wl.g * W_E)
        absw = wl.k_e * W_E + wl.k_i * wl.g * W_E
        # 11,250 FP32 additions per cell: compared at 1e-4 sum|w|
        assert np.all(np.abs(rb[15] - want) <= 1e-4 * absw)


def test_balanced_562500_bf16_delivery():
    wl = W.BALANCED_562500
    net, cp = _run(wl, 1, wl.sd_rel, seed=6)
    with net:
        st = net.stats()
        assert st.n_synapses == wl.n_synapses == 6_328_125_000
        assert st.interval == 10 and st.store_bytes >= 8 * wl.n_synapses
        src, t = W.bernoulli_spikes(wl.n, 5000, 10, 8.0, 0.1, seed=7)
        _check_sampled(net, cp, wl, src, t, 24, seed=8)
        from paper_2109_12855_gb300 import snn
        snn.snn_clear_rb(net.h)
        ev = net.deliver(np.arange(wl.n, dtype=np.uint32),
                         np.zeros(wl.n, np.int32))
        assert ev == wl.n_synapses
        cnt = net.read_counts()
        assert np.all(cnt.sum(axis=0, dtype=np.int64) == wl.k)
        assert not cnt[:10].any() and not cnt[21:].any()
