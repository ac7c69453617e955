"""Plastic delivery (pair-based power-law STDP of E->E synapses, Section 6)
on the GPU against the oracle.

Forced-spike protocol: with no drive and 0.1 mV synapses no neuron reaches
threshold by itself, so the spikes are exactly the ones the test forces
(membrane potential set above threshold before an interval): both sides see
the same spike trains, and every plastic weight can be compared synapse by
synapse (FP32 traces and weights against FP64).  Counts of plastic updates
are exact; ring buffers stay within 1e-5 sum|w| per cell."""
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


def _nets(fmt, hist, lam, alpha, w_max, n_e=480, n_i=120, k_e=48, k_i=12,
          seed=21):
    from paper_2109_12855_gb300 import snn
    p = snn.params(n_exc=n_e, n_inh=n_i, weight_format=fmt, seed=seed,
                   init_v_random=0, spike_log_capacity=1 << 20)
    net = snn.Net(p, stream())
    q = snn.stdp_params(lam=lam, alpha=alpha, w_max=w_max, history=hist)
    snn.snn_set_stdp(net.h, q)
    cp = snn.conn_params(k_exc=k_e, k_inh=k_i, w_exc=W_E, w_inh=-5 * W_E,
                         d_lo=10, d_hi=20, seed=seed + 1000)
    net.connect_fixed_indegree(cp)
    net.finalize()
    ocp = O.Conn(n_e, n_i, k_e, k_i, W_E, -5 * W_E, 10, 20, seed + 1000,
                 wfmt=1 if fmt == 0 else 2)
    store = O.build_fixed_indegree(ocp)
    ost = O.Stdp(n_exc=n_e, lam=lam, alpha=alpha, w_max=w_max)
    return net, store, ost


def _canonical(row_ptr, tgt, delay, w):
    """Per row, (target, delay, weight) sorted: synapses sharing (source,
    target, delay) start equal and see the same spikes, so they stay equal."""
    out = []
    for i in range(len(row_ptr) - 1):
        a, b = int(row_ptr[i]), int(row_ptr[i + 1])
        o = np.lexsort((w[a:b], delay[a:b], tgt[a:b]))
        out.append(np.stack([tgt[a:b][o], delay[a:b][o], w[a:b][o]], 1))
    return out


def _run_forced(net, store, ost, n_iv, rate, seed, D=10):
    from paper_2109_12855_gb300 import snn
    n = net.n
    g = W.rng(seed)
    hist = O.History(n)
    w_o = store.w.copy()
    st = O.State.zeros(n)
    rb_o = np.zeros((S, n))
    n_plastic = 0
    srcs = np.repeat(np.arange(n), np.diff(store.row_ptr.astype(np.int64)))
    e2e = (srcs < ost.n_exc) & (store.tgt < ost.n_exc)
    pl_per_src = np.bincount(srcs[e2e], minlength=n)
    for k in range(n_iv):
        t0 = k * D
        forced = np.flatnonzero(g.random(n) < rate)
        V, I, J, refr = net.read_state()
        V = V.copy()
        V[forced] = 100.0
        net.write_state(V, I, J, refr)
        st.V[forced] = 100.0
        snn.snn_update(net.h, t0, D)
        snn.snn_deliver_pending(net.h)
        gs, gt = net.read_spikes()
        os_, ot = O.update(NM, st, rb_o, t0, D, 0.0, 0.0, 1)
        assert sorted(zip(gs.tolist(), gt.tolist())) == \
            sorted(zip(os_.tolist(), ot.tolist()))
        assert set(os_.tolist()) == set(forced.tolist())
        hist.add(os_, ot)
        O.deliver_stdp(store, w_o, ost, hist, S, os_, ot, rb_o)
        n_plastic += int(pl_per_src[os_].sum())
    return w_o, rb_o, n_plastic


@pytest.mark.parametrize("fmt", [0, 1], ids=["fp32", "bf16"])
@pytest.mark.parametrize("lam,alpha,w_max,bound", [(1.0, 0.2, 30.0, "zero"),
                                                    (1.0, 0.0, 25.0, "cap")],
                         ids=["depress", "potentiate"])
def test_forced_spikes_weights_match_oracle(fmt, lam, alpha, w_max, bound):
    net, store, ost = _nets(fmt, hist=16, lam=lam, alpha=alpha, w_max=w_max)
    with net:
        w_o, rb_o, n_pl = _run_forced(net, store, ost, 80, 0.12, seed=5)
        st = net.stats()
        assert st.error_flags == 0
        assert st.plastic_events == n_pl > 10000
        assert st.stdp_truncated == 0
        rp, tg, dl, _ = net.read_store()
        w_g = net.read_weights()
        got = _canonical(rp, tg, dl, w_g.astype(np.float64))
        want = _canonical(store.row_ptr, store.tgt, store.delay, w_o)
        w0 = _canonical(store.row_ptr, store.tgt, store.delay, store.w)
        n_e = ost.n_exc
        changed = hit = 0
        for i, (a, b, c) in enumerate(zip(got, want, w0)):
            assert np.array_equal(a[:, :2], b[:, :2])
            assert np.allclose(a[:, 2], b[:, 2], rtol=2e-5, atol=2e-5)
            pl = (b[:, 0] < n_e) if i < n_e else np.zeros(len(b), bool)
            assert np.array_equal(b[~pl, 2], c[~pl, 2])   # static: unchanged
            changed += int((b[pl, 2] != c[pl, 2]).sum())
            hit += int((b[pl, 2] == (0.0 if bound == "zero" else w_max)).sum())
        # the protocol moves the plastic weights and reaches the bound
        assert changed > 10000 and hit > 100
        rb = net.read_rb()
        assert np.all(np.abs(rb - rb_o) <= 1e-4 * (np.abs(rb_o) + 1.0))


def _plastic_geometry(n, n_exc, tw0, sms, k=4):
    """The tile layout a plastic net takes (written out here from the rule:
    the narrowest width, from max(64, ceil(n_exc / SMs)) up to the uniform
    one, whose plastic tiles, one CTA each, plus the static tiles k to a CTA
    fit one wave)."""
    for tw in range(min(max(64, -(-n_exc // sms)), tw0), tw0 + 1):
        nt, pt = -(-n // tw), -(-n_exc // tw)
        if pt + -(-(nt - pt) // k) <= sms:
            return tw, nt
    return tw0, -(-n // tw0)


@pytest.mark.parametrize("fmt", [0, 1], ids=["fp32", "bf16"])
def test_narrowed_plastic_tiles_weights_match_oracle(fmt):
    """20,300 neurons: the plastic tiles narrow below the uniform width and
    the static ones share CTAs four at a time (on 152 SMs: 142 plastic tiles
    of 113 targets, 38 static ones, the last group of two); every plastic
    weight still matches the oracle synapse by synapse."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n_e, n_i = 16000, 4300
    net, store, ost = _nets(fmt, hist=16, lam=1.0, alpha=0.2, w_max=30.0,
                            n_e=n_e, n_i=n_i, k_e=48, k_i=12, seed=31)
    with net:
        st = net.stats()
        tw0 = max(-(-(n_e + n_i) // sms), 64)
        tw, nt = _plastic_geometry(n_e + n_i, n_e, tw0, sms)
        assert (st.tile_width, st.n_tiles) == (tw, nt)
        assert tw < tw0
        w_o, rb_o, n_pl = _run_forced(net, store, ost, 24, 0.05, seed=8)
        st = net.stats()
        assert st.error_flags == 0 and st.plastic_events == n_pl > 10000
        rp, tg, dl, _ = net.read_store()
        got = _canonical(rp, tg, dl, net.read_weights().astype(np.float64))
        want = _canonical(store.row_ptr, store.tgt, store.delay, w_o)
        for a, b in zip(got, want):
            assert np.array_equal(a[:, :2], b[:, :2])
            assert np.allclose(a[:, 2], b[:, 2], rtol=2e-5, atol=2e-5)
        rb = net.read_rb()
        assert np.all(np.abs(rb - rb_o) <= 1e-4 * (np.abs(rb_o) + 1.0))


def test_short_history_counts_truncated_windows():
    # two post spikes kept: windows that reach further are counted
    net, store, ost = _nets(1, hist=2, lam=0.5, alpha=0.1, w_max=60.0)
    with net:
        from paper_2109_12855_gb300 import snn
        g = W.rng(9)
        for k in range(40):
            V, I, J, refr = net.read_state()
            V = V.copy()
            # post neurons fire every interval, pre neurons every 8th
            V[g.random(net.n) < (0.9 if k % 8 else 1.0)] = 100.0
            net.write_state(V, I, J, refr)
            snn.snn_update(net.h, 10 * k, 10)
            snn.snn_deliver_pending(net.h)
        assert net.stats().stdp_truncated > 0


def test_plastic_net_rejects_caller_lists_and_checkpoints():
    from paper_2109_12855_gb300 import snn
    net, _, _ = _nets(0, hist=8, lam=0.1, alpha=0.05, w_max=50.0)
    with net:
        with pytest.raises(snn.SnnError) as e:
            net.deliver([1, 2], [0, 0])
        assert e.value.code == snn.SNN_E_STATE
        with pytest.raises(snn.SnnError):
            snn.snn_save_state(net.h)
        # parameters: after connecting, and out of range
        with pytest.raises(snn.SnnError):
            snn.snn_set_stdp(net.h, snn.stdp_params())
    p = snn.params(n_exc=10, n_inh=0)
    with snn.Net(p, stream()) as n2:
        for bad in (dict(history=1), dict(history=33), dict(history=12), dict(mu=1.5),
                    dict(tau_plus=0.0), dict(w_max=-1.0)):
            with pytest.raises(snn.SnnError) as e:
                snn.snn_set_stdp(n2.h, snn.stdp_params(**bad))
            assert e.value.code == snn.SNN_E_ARG


def test_zero_lambda_plastic_net_equals_static_net():
    """lambda = 0: the plastic kernels deliver the stored weights; the whole
    simulation equals the static one bit for bit."""
    from paper_2109_12855_gb300 import snn
    runs = []
    for plastic in (False, True):
        p = snn.params(n_exc=4000, n_inh=1000, weight_format=1, seed=3,
                       nu_ext=20000.0, w_ext=W_E, spike_log_capacity=1 << 20)
        net = snn.Net(p, stream())
        if plastic:
            snn.snn_set_stdp(net.h, snn.stdp_params(lam=0.0))
        net.connect_fixed_indegree(snn.conn_params(
            k_exc=400, k_inh=100, w_exc=W_E, w_inh=-5 * W_E, d_lo=10, d_hi=20,
            seed=4))
        net.finalize()
        with net:
            snn.snn_simulate(net.h, 1500)
            s, t = net.read_spikes(1 << 20)
            o = np.lexsort((s, t))
            runs.append((s[o], t[o], net.read_rb(), net.stats()))
    (s0, t0, rb0, st0), (s1, t1, rb1, st1) = runs
    assert len(s0) > 1000
    assert np.array_equal(s0, s1) and np.array_equal(t0, t1)
    assert np.array_equal(rb0.view(np.uint32), rb1.view(np.uint32))
    assert st1.plastic_events > 0 and st0.plastic_events == 0


def test_network_statistics_match_oracle():
    """A driven balanced net with STDP: chaotic, so compared statistically
    (mean rate within 2 %, mean change of the E->E weights within 5 %)."""
    from paper_2109_12855_gb300 import snn
    n_e, n_i, k_e, k_i, steps = 1000, 250, 80, 20, 4000
    lam, alpha = 0.1, 0.0513
    g_rates, o_rates, g_dw, o_dw = [], [], [], []
    for seed in range(1, 4):
        p = snn.params(n_exc=n_e, n_inh=n_i, weight_format=0, seed=seed,
                       nu_ext=20000.0, w_ext=W_E, spike_log_capacity=1 << 22)
        with snn.Net(p, stream()) as net:
            snn.snn_set_stdp(net.h, snn.stdp_params(lam=lam, alpha=alpha))
            net.connect_fixed_indegree(snn.conn_params(
                k_exc=k_e, k_inh=k_i, w_exc=W_E, w_inh=-5 * W_E, d_lo=10,
                d_hi=20, seed=seed + 1000))
            net.finalize()
            snn.snn_simulate(net.h, steps)
            st = net.stats()
            assert st.stdp_truncated == 0
            g_rates.append(st.spikes / (n_e + n_i) / (steps * 1e-4))
            rp, tg, _, w0 = net.read_store()
            w = net.read_weights()
            srcs = np.repeat(np.arange(n_e + n_i), np.diff(rp.astype(np.int64)))
            e2e = (srcs < n_e) & (tg < n_e)
            g_dw.append(float(np.mean(w[e2e]) - W_E))
        cp = O.Conn(n_e, n_i, k_e, k_i, W_E, -5 * W_E, 10, 20, seed + 1000,
                    wfmt=1)
        store = O.build_fixed_indegree(cp)
        w_o = store.w.copy()
        st_o = O.State.zeros(n_e + n_i)
        st_o.V[:] = O.init_v(NM, n_e + n_i, seed)
        rb = np.zeros((S, n_e + n_i))
        s_o, _, _ = O.simulate_stdp(NM, store, w_o, O.Stdp(n_exc=n_e, lam=lam,
                                    alpha=alpha), S, 10, st_o, rb, 0, steps,
                                    20000.0, W_E, seed, O.History(n_e + n_i))
        o_rates.append(len(s_o) / (n_e + n_i) / (steps * 1e-4))
        srcs = np.repeat(np.arange(n_e + n_i), np.diff(store.row_ptr.astype(np.int64)))
        e2e = (srcs < n_e) & (store.tgt < n_e)
        o_dw.append(float(np.mean(w_o[e2e]) - W_E))
    assert np.mean(g_rates) == pytest.approx(np.mean(o_rates), rel=0.02)
    assert abs(np.mean(o_dw)) > 1e-3
    assert np.mean(g_dw) == pytest.approx(np.mean(o_dw), rel=0.05)
