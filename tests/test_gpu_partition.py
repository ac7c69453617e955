"""Target-partitioned network (Section 2.1: neurons spread over processes,
synapses stored with their targets, one spike exchange per interval): two
or three partitions of one network, run in one process with the exchange
done by concatenation, equal the whole net bit for bit -- spike trains,
neuron state, ring buffers and event counts -- because every random stream
is keyed by global neuron index and the partitions agree on the bounds of
the exact fixed-point accumulation."""
import numpy as np
import pytest

import oracle as O
from gpu_common import need_gpu, stream

pytestmark = pytest.mark.gpu

W_E = O.weight_for_psp(O.Neuron(), 0.1)
N = 5000


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _params(fmt):
    from paper_2109_12855_gb300 import snn
    return snn.params(n_exc=4000, n_inh=1000, weight_format=fmt, seed=13,
                      nu_ext=20000.0, w_ext=W_E, spike_log_capacity=1 << 21)


def _conn(fmt):
    from paper_2109_12855_gb300 import snn
    sd = 0.1 if fmt == 1 else 0.0
    return snn.conn_params(k_exc=400, k_inh=100, w_exc=W_E, w_inh=-5 * W_E,
                           sd_exc=sd * W_E, sd_inh=sd * 5 * W_E, d_lo=10,
                           d_hi=20, seed=77)


def _sorted(src, t):
    o = np.lexsort((src, t))
    return src[o], t[o]


def _run_whole(fmt, steps):
    from paper_2109_12855_gb300 import snn
    with snn.Net(_params(fmt), stream()) as net:
        net.connect_fixed_indegree(_conn(fmt))
        net.finalize()
        snn.snn_simulate(net.h, steps)
        return (net.stats().events_delivered, _sorted(*net.read_spikes(1 << 21)),
                net.read_state(), net.read_rb())


def _run_parts(fmt, cuts, steps):
    from paper_2109_12855_gb300 import partition as PT
    nets = [PT.create(_params(fmt), _conn(fmt), lo, hi, stream())
            for lo, hi in zip(cuts[:-1], cuts[1:])]
    try:
        PT.agree_bounds(nets)
        for net in nets:
            net.finalize()
        ev = PT.simulate(nets, steps, t0=0)
        logs = [net.read_spikes(1 << 21) for net in nets]
        states = [net.read_state() for net in nets]
        rbs = [net.read_rb() for net in nets]
        stats = [net.stats() for net in nets]
    finally:
        for net in nets:
            net.close()
    src = np.concatenate([s for s, _ in logs])
    t = np.concatenate([tt for _, tt in logs])
    return ev, _sorted(src, t), states, rbs, stats


@pytest.mark.parametrize("fmt", [0, 1], ids=["fp32", "bf16"])
@pytest.mark.parametrize("cuts", [[0, 2500, N], [0, 1700, 3333, N]],
                         ids=["2-parts", "3-parts"])
def test_partitions_equal_the_whole_net(fmt, cuts):
    steps = 1500
    w_ev, (ws, wt), wstate, wrb = _run_whole(fmt, steps)
    ev, (ps, pt), states, rbs, stats = _run_parts(fmt, cuts, steps)
    assert len(ws) > 2000
    assert np.array_equal(ws, ps) and np.array_equal(wt, pt)
    assert ev == w_ev
    assert sum(st.events_delivered for st in stats) == w_ev
    for k, (lo, hi) in enumerate(zip(cuts[:-1], cuts[1:])):
        assert stats[k].first_neuron == lo and stats[k].n_sources == N
        for a, b in zip(wstate, states[k]):
            assert np.array_equal(a[lo:hi].view(np.uint32) if a.dtype == np.float32
                                  else a[lo:hi], b.view(np.uint32)
                                  if b.dtype == np.float32 else b)
        assert np.array_equal(wrb[:, lo:hi].view(np.uint32), rbs[k].view(np.uint32))


def test_partition_rejects_bad_ranges_and_features():
    from paper_2109_12855_gb300 import snn
    p = _params(0)
    for lo, hi in ((10, 10), (4000, 6000), (3000, 2000)):
        q = snn.snn_params.from_buffer_copy(p)
        q.part_lo, q.part_hi = lo, hi
        with pytest.raises(snn.SnnError) as e:
            snn.Net(q, stream())
        assert e.value.code == snn.SNN_E_ARG
    q = snn.snn_params.from_buffer_copy(p)
    q.part_lo, q.part_hi = 0, 2500
    with snn.Net(q, stream()) as net:
        with pytest.raises(snn.SnnError):
            snn.snn_set_stdp(net.h, snn.stdp_params())
        with pytest.raises(snn.SnnError):
            net.connect_edges([0], [1], [10], [1.0])
        net.connect_fixed_indegree(_conn(0))
        net.finalize()
        # a gathered list needs a pending update; sources are global
        with pytest.raises(snn.SnnError) as e:
            snn.snn_deliver_gathered(net.h, np.array([1], np.uint32),
                                     np.array([0], np.int32))
        assert e.value.code == snn.SNN_E_STATE
        snn.snn_update(net.h, 0, 10)
        with pytest.raises(snn.SnnError) as e:
            snn.snn_deliver_gathered(net.h, np.array([N], np.uint32),
                                     np.array([0], np.int32))
        assert e.value.code == snn.SNN_E_ARG
        assert snn.snn_deliver_gathered(net.h, np.array([4999], np.uint32),
                                        np.array([3], np.int32)) > 0


def test_accumulator_word_count_parameter_is_checked():
    """snn_params.acc_words accepts 0 (automatic) and 2 (two words) only."""
    from paper_2109_12855_gb300 import snn
    for bad in (1, 3, -1):
        q = snn.snn_params.from_buffer_copy(_params(1))
        q.acc_words = bad
        with pytest.raises(snn.SnnError) as e:
            snn.Net(q, stream())
        assert e.value.code == snn.SNN_E_ARG
