"""Whole-network runs: deterministic timing pins and statistical parity with
the oracle (spiking is chaotic, so only statistics can be compared)."""
import numpy as np
import pytest

import oracle as O
from gpu_common import S, need_gpu, stream

pytestmark = pytest.mark.gpu

NM = O.Neuron()
W_E = O.weight_for_psp(NM, 0.1)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def test_spike_arrives_at_emission_plus_delay_on_gpu():
    """0 -> 1 with delay 7 and weight 6000 pA: neuron 1 fires at 7 + n*,
    n* the first grid step where the closed-form PSP crosses threshold."""
    from paper_2109_12855_gb300 import snn
    d, w = 7, 6000.0
    n_star = next(n for n in range(1, 500)
                  if w * O.psp_unit(NM, n * NM.h) >= NM.v_th)
    p = snn.params(n_exc=2, n_inh=0, init_v_random=0, spike_log_capacity=64)
    with snn.Net(p, stream()) as net:
        net.connect_edges([0], [1], [d], [w])
        net.finalize()
        net.write_state([100.0, 0.0], [0, 0], [0, 0], [0, 0])
        snn.snn_simulate(net.h, 200)
        src, t = net.read_spikes()
        assert sorted(zip(t.tolist(), src.tolist())) == [(0, 0), (d + n_star, 1)]
        st = net.stats()
        assert st.events_delivered == 1 and st.spikes == 2 and st.t_now == 200


def _rates_cv(src, t, n, steps):
    rate = len(src) / n / (steps * NM.h * 1e-3)
    cvs = []
    order = np.lexsort((t, src))
    s, tt = src[order], t[order]
    bounds = np.flatnonzero(np.diff(s)) + 1
    for a, b in zip(np.r_[0, bounds], np.r_[bounds, len(s)]):
        if b - a > 2:
            isi = np.diff(tt[a:b])
            cvs.append(isi.std() / isi.mean())
    return rate, float(np.mean(cvs)) if cvs else float("nan")


@pytest.mark.parametrize("nu,fmt", [(15000.0, 0), (20000.0, 0), (15000.0, 1)])
def test_balanced_net_statistics_match_oracle(nu, fmt):
    """N = 1,250, K = 100, 1 s: mean rate within 2 % and mean CV of the ISI
    within 5 % of the oracle's, averaged over 5 seeds."""
    from paper_2109_12855_gb300 import snn
    steps = 10000
    g_r, g_c, o_r, o_c = [], [], [], []
    for seed in range(1, 6):
        p = snn.params(n_exc=1000, n_inh=250, weight_format=fmt, nu_ext=nu,
                       w_ext=W_E, seed=100 + seed, spike_log_capacity=1 << 22)
        with snn.Net(p, stream()) as net:
            net.connect_fixed_indegree(snn.conn_params(
                k_exc=80, k_inh=20, w_exc=W_E, w_inh=-5 * W_E, d_lo=10,
                d_hi=20, seed=seed))
            net.finalize()
            snn.snn_simulate(net.h, steps)
            src, t = net.read_spikes()
            st = net.stats()
            assert st.error_flags == 0
            deg_check = st.events_delivered
        r, c = _rates_cv(src, t, 1250, steps)
        g_r.append(r)
        g_c.append(c)
        cp = O.Conn(1000, 250, 80, 20, W_E, -5 * W_E, 10, 20, seed,
                    wfmt=1 if fmt == 0 else 2)
        store = O.build_fixed_indegree(cp)
        s = O.State(O.init_v(NM, 1250, 100 + seed), np.zeros(1250),
                    np.zeros(1250), np.zeros(1250, np.int32))
        osrc, ot, oev = O.simulate(NM, store, S, 10, s, np.zeros((S, 1250)), 0,
                                   steps, nu, W_E, 100 + seed)
        r, c = _rates_cv(osrc, ot, 1250, steps)
        o_r.append(r)
        o_c.append(c)
        # events delivered are the out-degrees of the spikes (invariant)
        deg = np.diff(store.row_ptr.astype(np.int64))
        assert deg_check == int(deg[src].sum())
    gr, orr = np.mean(g_r), np.mean(o_r)
    gc, oc = np.mean(g_c), np.mean(o_c)
    assert abs(gr - orr) <= 0.02 * orr, (gr, orr)
    assert abs(gc - oc) <= 0.05 * oc, (gc, oc)


def test_benchmark_drive_of_the_tiny_net_is_subthreshold():
    """At the 8 kHz drive of the 1,250-neuron benchmark configuration the
    free membrane potential stays far below threshold: no spikes, on both
    sides."""
    from paper_2109_12855_gb300 import snn
    p = snn.params(n_exc=1000, n_inh=250, nu_ext=8000.0, w_ext=W_E, seed=3,
                   spike_log_capacity=1 << 16)
    with snn.Net(p, stream()) as net:
        net.connect_fixed_indegree(snn.conn_params(
            k_exc=80, k_inh=20, w_exc=W_E, w_inh=-5 * W_E, d_lo=10, d_hi=20,
            seed=1))
        net.finalize()
        snn.snn_simulate(net.h, 10000)
        assert net.stats().spikes == 0
        V = net.read_state()[0]
    assert 5.0 < V.mean() < 15.0


def test_simulation_counters_and_partial_intervals():
    from paper_2109_12855_gb300 import snn
    p = snn.params(n_exc=1000, n_inh=250, nu_ext=20000.0, w_ext=W_E, seed=7,
                   spike_log_capacity=1 << 20)
    with snn.Net(p, stream()) as net:
        net.connect_fixed_indegree(snn.conn_params(
            k_exc=80, k_inh=20, w_exc=W_E, w_inh=-5 * W_E, d_lo=10, d_hi=20,
            seed=2))
        net.finalize()
        for n in (3, 10, 97, 1000, 5):     # graph and non-graph paths
            snn.snn_simulate(net.h, n)
        st = net.stats()
        assert st.t_now == 1115 and st.error_flags == 0
        src, t = net.read_spikes()
        assert len(src) == st.spikes > 0
        assert t.min() >= 0 and t.max() < 1115
        rp = net.read_store()[0].astype(np.int64)
        assert st.events_delivered == int((rp[src + 1] - rp[src]).sum())
