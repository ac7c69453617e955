"""Long-run spike statistics: per-neuron spike and inter-spike-interval
counts with FP64 sums kept by the update kernel.  Intervals are integer
step counts, so the sums are exact and must equal, bit for bit, the sums
computed from the spike log.  A 10 s biological run of the balanced network
is compared with the oracle for drift: per-second rates stay flat, and the
mean rate (2 %) and CV of the intervals (5 %) agree."""
import numpy as np
import pytest

import oracle as O
from gpu_common import need_gpu, stream

pytestmark = pytest.mark.gpu

NM = O.Neuron()
W_E = O.weight_for_psp(NM, 0.1)
S = 32


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _net(n_e=4000, n_i=1000, k_e=400, k_i=100, nu=20000.0, seed=7, log=1 << 22):
    from paper_2109_12855_gb300 import snn
    p = snn.params(n_exc=n_e, n_inh=n_i, nu_ext=nu, w_ext=W_E, seed=seed,
                   spike_log_capacity=log)
    net = snn.Net(p, stream())
    net.connect_fixed_indegree(snn.conn_params(
        k_exc=k_e, k_inh=k_i, w_exc=W_E, w_inh=-5 * W_E, d_lo=10, d_hi=20,
        seed=seed + 1000))
    net.finalize()
    return net


def _from_log(n, src, t, t_lo=None):
    """Per neuron: spikes (at or after t_lo), intervals ending at or after
    t_lo, and the exact integer sums of those intervals and their squares."""
    o = np.lexsort((t, src))
    src, t = src[o].astype(np.int64), t[o].astype(np.int64)
    spikes = np.zeros(n, np.int64)
    cnt = np.zeros(n, np.int64)
    s1 = np.zeros(n, np.int64)
    s2 = np.zeros(n, np.int64)
    lo = -1 if t_lo is None else t_lo
    keep = t >= lo
    np.add.at(spikes, src[keep], 1)
    same = src[1:] == src[:-1]
    d = (t[1:] - t[:-1])[same]
    who = src[1:][same]
    end = t[1:][same]
    m = end >= lo
    np.add.at(cnt, who[m], 1)
    np.add.at(s1, who[m], d[m])
    np.add.at(s2, who[m], d[m] * d[m])
    return spikes, cnt, s1, s2


def test_accumulators_equal_the_spike_log_exactly():
    from paper_2109_12855_gb300 import snn
    with _net() as net:
        snn.snn_simulate(net.h, 3000)
        src, t = net.read_spikes(1 << 22)
        a, b, c, d = snn.snn_read_spike_stats(net.h, net.n)
        sp, cnt, s1, s2 = _from_log(net.n, src, t)
        assert sp.sum() > 10000 and cnt.sum() > 5000
        assert np.array_equal(a, sp) and np.array_equal(b, cnt)
        assert np.array_equal(c, s1.astype(np.float64))
        assert np.array_equal(d, s2.astype(np.float64))


def test_clear_counts_from_then_on_with_the_spanning_interval():
    from paper_2109_12855_gb300 import snn
    with _net(seed=8) as net:
        snn.snn_simulate(net.h, 1000)
        snn.snn_clear_spike_stats(net.h)
        snn.snn_simulate(net.h, 1000)
        src, t = net.read_spikes(1 << 22)
        a, b, c, d = snn.snn_read_spike_stats(net.h, net.n)
        sp, cnt, s1, s2 = _from_log(net.n, src, t, t_lo=1000)
        assert np.array_equal(a, sp) and np.array_equal(b, cnt)
        assert np.array_equal(c, s1.astype(np.float64))
        assert np.array_equal(d, s2.astype(np.float64))


def _cv(cnt, s1, s2):
    ok = cnt >= 2
    m = s1[ok] / cnt[ok]
    var = s2[ok] / cnt[ok] - m * m
    return float(np.mean(np.sqrt(np.maximum(var, 0.0)) / m))


def test_ten_seconds_without_drift_against_oracle():
    from paper_2109_12855_gb300 import snn
    n_e, n_i, k_e, k_i, nu = 1000, 250, 80, 20, 15000.0
    n = n_e + n_i
    steps_s = 10000
    g_rate, g_cv, o_rate, o_cv = [], [], [], []
    for seed in (1, 2, 3):
        with _net(n_e, n_i, k_e, k_i, nu, seed=seed, log=0) as net:
            per_s = []
            prev = 0
            for _ in range(10):
                snn.snn_simulate(net.h, steps_s)
                sp = net.stats().spikes
                per_s.append((sp - prev) / n)
                prev = sp
            _, b, c, d = snn.snn_read_spike_stats(net.h, n)
            g_rate.append(per_s)
            g_cv.append(_cv(b, c, d))
        cp = O.Conn(n_e, n_i, k_e, k_i, W_E, -5 * W_E, 10, 20, seed + 1000,
                    wfmt=1)
        store = O.build_fixed_indegree(cp)
        st = O.State.zeros(n)
        st.V[:] = O.init_v(NM, n, seed)
        rb = np.zeros((S, n))
        src, t, _ = O.simulate(NM, store, S, 10, st, rb, 0, 10 * steps_s, nu,
                               W_E, seed)
        o_rate.append(np.bincount(t // steps_s, minlength=10)[:10] / n)
        _, cnt, s1, s2 = _from_log(n, src, t)
        o_cv.append(_cv(cnt, s1.astype(np.float64), s2.astype(np.float64)))
    g_rate, o_rate = np.array(g_rate), np.array(o_rate)
    assert g_rate.mean() > 2.0
    assert g_rate.mean() == pytest.approx(o_rate.mean(), rel=0.02)
    assert np.mean(g_cv) == pytest.approx(np.mean(o_cv), rel=0.05)
    # no drift: every second within 10 % of the run's mean, on both sides
    for r in (g_rate.mean(0), o_rate.mean(0)):
        assert np.all(np.abs(r / r.mean() - 1.0) < 0.10)
