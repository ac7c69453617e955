"""Pins of the oracle's plastic delivery (pair-based power-law STDP of E->E
synapses, evaluated at delivery; Section 6 of the paper and the rule it
cites).  Readings: the whole delay is dendritic (a synapse sees a pre spike
at t_e and a post spike at t_p + d); pairs with D = (t_p + d - t_e) h > 0
potentiate by lambda w0^(1-mu) w^mu exp(-D/tau_plus), pairs with D <= 0
depress by lambda alpha w exp(D/tau_minus); weights stay in [0, w_max].

Pinned by: hand-evaluated closed forms of one and two pairs; an independent
brute-force enumeration of every pre/post pair (in the small-lambda limit
the weight change divided by lambda is the plain pair sum); bounds; static
synapses and lambda = 0 reducing to Algorithm REF bit for bit."""
import numpy as np
import pytest

import oracle as O
import workloads as W

H = 0.1
S = 32


def _one_synapse(d, w=20.0, n=2, n_exc=None, lam=0.1, alpha=0.0513,
                 w_max=100.0):
    st = O.build_edges(n, [0], [1], [d], [w])
    p = O.Stdp(n_exc=n if n_exc is None else n_exc, lam=lam, alpha=alpha,
               w_max=w_max)
    return st, st.w.copy(), p


def _deliver_pre(st, w, p, hist, pre_times):
    for te in pre_times:
        O.deliver_stdp(st, w, p, hist, S, [0], [te])


def test_potentiation_then_depression_closed_form():
    d = 10
    st, w, p = _one_synapse(d)
    hist = O.History(2)
    hist.add([0, 1, 0], [0, 30, 100])
    _deliver_pre(st, w, p, hist, [0, 100])
    w1 = 20.0 + 0.1 * 1.0 ** 0.6 * 20.0 ** 0.4 * np.exp(-(30 + d - 0) * H / 20.0)
    w2 = w1 * (1.0 - 0.1 * 0.0513 * np.exp(-(100 - 30 - d) * H / 20.0))
    assert w[0] == pytest.approx(w2, rel=1e-14)


def test_depression_only_and_same_step_pair_depresses():
    d = 10
    st, w, p = _one_synapse(d)
    hist = O.History(2)
    # post seen at the synapse at 50 + 10 = 60 = the pre spike: D = 0
    hist.add([1, 0], [50, 60])
    _deliver_pre(st, w, p, hist, [60])
    assert w[0] == pytest.approx(20.0 * (1 - 0.1 * 0.0513), rel=1e-14)


def test_pair_seen_one_step_later_potentiates_at_next_pre():
    d = 10
    st, w, p = _one_synapse(d)
    hist = O.History(2)
    hist.add([0, 1, 0], [60, 51, 200])   # post seen at 61 > 60
    _deliver_pre(st, w, p, hist, [60])
    assert w[0] == 20.0                   # nothing before the first pre spike
    _deliver_pre(st, w, p, hist, [200])
    w1 = 20.0 + 0.1 * 20.0 ** 0.4 * np.exp(-1 * H / 20.0)
    w2 = w1 * (1 - 0.1 * 0.0513 * np.exp(-(200 - 61) * H / 20.0))
    assert w[0] == pytest.approx(w2, rel=1e-14)


def _pair_sum(pre, post, d, w, p):
    """Every pair that the event-driven scheme has applied once the pre
    spikes ``pre`` were delivered, summed with the weight held at w."""
    pre = np.sort(np.asarray(pre))
    last = pre[-1]
    tot = 0.0
    for tp in post:
        seen = tp + d
        for te in pre:
            D = (seen - te) * H
            if D > 0:
                if seen <= last:   # applied at the first pre spike >= seen
                    tot += p.w0 ** (1 - p.mu) * w ** p.mu * np.exp(-D / p.tau_plus)
            else:
                tot -= p.alpha * w * np.exp(D / p.tau_minus)
    return tot


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_small_lambda_limit_equals_brute_force_pair_sum(seed):
    g = W.rng(seed)
    d = int(g.integers(1, 30))
    pre = np.unique(g.integers(0, 3000, 25))
    post = np.unique(g.integers(0, 3000, 30))
    # force exact coincidences D = 0 and D = 1 step
    post = np.unique(np.concatenate([post, pre[[3, 7]] - d, pre[[5]] - d + 1]))
    lam = 1e-7
    st, w, p = _one_synapse(d, lam=lam, w_max=1e9)
    hist = O.History(2)
    tt = np.concatenate([pre, post])
    ii = np.concatenate([np.zeros(len(pre), np.uint32), np.ones(len(post), np.uint32)])
    o = np.argsort(tt, kind="stable")
    hist.add(ii[o], tt[o])
    _deliver_pre(st, w, p, hist, pre)
    want = _pair_sum(pre, post, d, 20.0, p)
    assert abs(want) > 1e-3
    assert (w[0] - 20.0) / lam == pytest.approx(want, rel=1e-5)


def test_weights_stay_in_bounds():
    d = 5
    st, w, p = _one_synapse(d, lam=50.0, w_max=37.5)
    hist = O.History(2)
    hist.add([0, 1, 0], [0, 1, 100])
    _deliver_pre(st, w, p, hist, [0, 100])
    # potentiation hits the cap; depression of 50 * 0.0513 * exp(-9.4/20) ~ 1.6
    # then drives the weight to zero, where the power law keeps it
    assert w[0] == 0.0
    st, w, p = _one_synapse(d, lam=50.0, alpha=0.0, w_max=37.5)
    hist = O.History(2)
    hist.add([0, 1, 0], [0, 1, 100])
    _deliver_pre(st, w, p, hist, [0, 100])
    assert w[0] == 37.5


def test_static_synapses_and_zero_lambda_reduce_to_ref():
    n = 300
    src, tgt, dl, ww = W.random_edges(n, 6000, 1, 20, seed=4)
    # excitatory sources (< 240) have non-negative weights, as in the network
    ww = np.where(np.asarray(src) < 240, np.abs(ww), -np.abs(ww))
    st = O.build_edges(n, src, tgt, dl, ww)
    g = W.rng(8)
    # spikes of all neurons over 400 steps, delivered in intervals of 20
    sp_t = np.sort(g.integers(0, 400, 900))
    sp_i = g.integers(0, n, 900).astype(np.uint32)
    hist = O.History(n)
    hist.add(sp_i, sp_t)
    # lambda = 0: REF bit for bit, weights unchanged
    w = st.w.copy()
    p0 = O.Stdp(n_exc=240, lam=0.0)
    rb = np.zeros((S, n))
    rb_ref = np.zeros((S, n))
    for k in range(0, 400, 20):
        m = (sp_t >= k) & (sp_t < k + 20)
        O.deliver_stdp(st, w, p0, hist, S, sp_i[m], sp_t[m], rb)
        O.deliver_ref(st, S, sp_i[m], sp_t[m], rb=rb_ref, counts=False)
    assert np.array_equal(rb.view(np.uint64), rb_ref.view(np.uint64))
    assert np.array_equal(w, st.w)
    # lambda > 0: only E->E synapses change
    w = st.w.copy()
    p = O.Stdp(n_exc=240, lam=0.1)
    for k in range(0, 400, 20):
        m = (sp_t >= k) & (sp_t < k + 20)
        O.deliver_stdp(st, w, p, hist, S, sp_i[m], sp_t[m])
    srcs = np.repeat(np.arange(n), np.diff(st.row_ptr.astype(np.int64)))
    plastic = (srcs < 240) & (st.tgt < 240)
    assert np.array_equal(w[~plastic], st.w[~plastic])
    assert (w[plastic] != st.w[plastic]).mean() > 0.5


def test_simulation_with_zero_lambda_equals_static_simulation():
    nm = O.Neuron()
    w_e = O.weight_for_psp(nm, 0.1)
    cp = O.Conn(400, 100, 40, 10, w_e, -5 * w_e, 10, 20, seed=6)
    store = O.build_fixed_indegree(cp)
    sa, sb = O.State.zeros(500), O.State.zeros(500)
    sa.V[:] = sb.V[:] = O.init_v(nm, 500, 3)
    rba, rbb = np.zeros((S, 500)), np.zeros((S, 500))
    a = O.simulate(nm, store, S, 10, sa, rba, 0, 600, 20000.0, w_e, 3)
    w = store.w.copy()
    b = O.simulate_stdp(nm, store, w, O.Stdp(n_exc=400, lam=0.0), S, 10, sb,
                        rbb, 0, 600, 20000.0, w_e, 3, O.History(500))
    assert len(a[0]) > 200
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2] == b[2]
    assert np.array_equal(sa.V, sb.V)


def test_history_overflow_raises():
    h = O.History(2, cap=2)
    h.add([0, 0], [1, 2])
    with pytest.raises(ValueError):
        h.add([0], [3])
