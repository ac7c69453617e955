"""The oracle's thread-parallel form (Section 2.1, NEST's thread model: each
thread owns a range of neurons and the target segments onto them) against
its single-thread form: bitwise equal ring buffers, spike trains, states and
event counts, for several thread counts (uneven ranges, more threads than
there are spiking neurons) and a partial last interval."""
import numpy as np
import pytest

import oracle as O
import workloads as W

NM = O.Neuron()
S = 32


def _net(seed=7, d_lo=10, d_hi=20):
    cp = O.Conn(400, 100, 40, 10, 22.4, -112.0, d_lo, d_hi, seed, wfmt=1)
    return cp, O.build_fixed_indegree(cp)


def _state(n, seed):
    return O.State(O.init_v(NM, n, seed), np.zeros(n), np.zeros(n),
                   np.zeros(n, np.int32))


@pytest.mark.parametrize("threads", [1, 2, 3, 7, 16])
def test_threaded_simulation_is_bitwise_the_single_thread_one(threads):
    cp, store = _net()
    s0, rb0 = _state(500, 3), np.zeros((S, 500))
    a0, b0, e0 = O.simulate(NM, store, S, 10, s0, rb0, 0, 2995, 20000.0, 22.4, 5)
    assert len(a0) > 1000 and e0 > 0
    with O.Threaded(cp, threads) as mt:
        assert mt.n_threads == threads
        rg = mt.ranges()
        assert rg[0][0] == 0 and rg[-1][1] == 500
        assert all(a[1] == b[0] for a, b in zip(rg, rg[1:]))
        s1, rb1 = _state(500, 3), np.zeros((S, 500))
        a1, b1, e1 = mt.simulate(NM, 10, s1, rb1, 0, 2995, 20000.0, 22.4, 5)
    assert e1 == e0
    assert np.array_equal(a1, a0) and np.array_equal(b1, b0)
    for x, y in ((s1.V, s0.V), (s1.I, s0.I), (s1.J, s0.J), (s1.refr, s0.refr),
                 (rb1, rb0)):
        assert np.array_equal(x, y)


def test_threaded_simulation_continues_like_one_long_run():
    """Two calls on the same stores equal one call of their total length."""
    cp, store = _net(seed=11, d_lo=15, d_hi=15)
    s0, rb0 = _state(500, 4), np.zeros((S, 500))
    a0, b0, e0 = O.simulate(NM, store, S, 15, s0, rb0, 0, 3000, 20000.0, 22.4, 6)
    with O.Threaded(cp, 4) as mt:
        s1, rb1 = _state(500, 4), np.zeros((S, 500))
        a1, b1, e1 = mt.simulate(NM, 15, s1, rb1, 0, 1500, 20000.0, 22.4, 6)
        a2, b2, e2 = mt.simulate(NM, 15, s1, rb1, 1500, 1500, 20000.0, 22.4, 6)
    assert e1 + e2 == e0
    assert np.array_equal(np.r_[a1, a2], a0) and np.array_equal(np.r_[b1, b2], b0)
    assert np.array_equal(s1.V, s0.V) and np.array_equal(rb1, rb0)


@pytest.mark.parametrize("threads", [1, 5, 8])
def test_threaded_delivery_is_bitwise_algorithm_ref(threads):
    cp, store = _net(seed=13)
    src, t = W.random_spikes(500, 3000, -40, 40, seed=2)   # wraps the ring
    rb0, _, _, e0 = O.deliver_ref(store, S, src, t)
    with O.Threaded(cp, threads) as mt:
        rb1, e1 = mt.deliver(src, t)
        # a second list adds onto the first
        src2, t2 = W.random_spikes(500, 10, 0, 3, seed=4)
        rb1, e2 = mt.deliver(src2, t2, rb1)
    O.deliver_ref(store, S, src2, t2, rb=rb0)
    assert e1 == e0
    assert np.array_equal(rb1, rb0)


def test_more_threads_than_neurons_is_clamped():
    cp = O.Conn(3, 1, 2, 1, 22.4, -112.0, 10, 20, 1, wfmt=1)
    with O.Threaded(cp, 9) as mt:
        assert mt.n_threads == 4
        rb, ev = mt.deliver([0, 1, 2, 3], [0, 0, 0, 0])
    rb0, _, _, ev0 = O.deliver_ref(O.build_fixed_indegree(cp), S,
                                   [0, 1, 2, 3], [0, 0, 0, 0])
    assert ev == ev0 and np.array_equal(rb, rb0)


def test_threads_over_a_target_range():
    """Threads that own only [100, 400): delivery writes exactly those
    columns of Algorithm REF's ring buffer, the update advances exactly
    those neurons as the whole-population update does, and a closed-network
    simulation is refused."""
    cp, store = _net(seed=17)
    src, t = W.random_spikes(500, 2000, 0, 10, seed=8)
    rb0, _, _, _ = O.deliver_ref(store, S, src, t)
    with O.Threaded(cp, 3, tgt_lo=100, tgt_hi=400) as mt:
        assert mt.ranges()[0][0] == 100 and mt.ranges()[-1][1] == 400
        rb1, ev = mt.deliver(src, t)
        assert np.array_equal(rb1[:, 100:400], rb0[:, 100:400])
        assert not rb1[:, :100].any() and not rb1[:, 400:].any()
        tg = store.tgt.astype(np.int64)
        rp = store.row_ptr.astype(np.int64)
        owned = sum(int(((tg[rp[s]:rp[s + 1]] >= 100) &
                         (tg[rp[s]:rp[s + 1]] < 400)).sum()) for s in src)
        assert ev == owned
        V, I, J, refr = W.random_state(500, seed=3)
        s0 = O.State(V.copy(), I.copy(), J.copy(), refr.copy())
        s1 = O.State(V.copy(), I.copy(), J.copy(), refr.copy())
        r0, r1 = rb0.copy(), rb0.copy()
        osrc, _ = O.update(NM, s0, r0, 5, 10, 20000.0, 22.4, 9)
        n_sp = mt.update(NM, s1, r1, 5, 10, 20000.0, 22.4, 9)
        own = slice(100, 400)
        assert n_sp == int(((osrc >= 100) & (osrc < 400)).sum())
        for a, b, x in ((s1.V, s0.V, V), (s1.J, s0.J, J), (s1.refr, s0.refr, refr)):
            assert np.array_equal(a[own], b[own])
            assert np.array_equal(a[:100], x[:100]) and np.array_equal(a[400:], x[400:])
        assert np.array_equal(r1[:, own], r0[:, own])
        with pytest.raises(ValueError):
            mt.simulate(NM, 10, s1, r1, 0, 10, 0.0, 0.0, 1)
