"""Target-partitioned network (Section 2.1: neurons spread over processes,
synapses stored with their targets, one spike exchange per interval): two
or three partitions of one network, run in one process with the exchange
done by concatenation on the host or through the device exchange buffers,
equal the whole net bit for bit -- spike trains, neuron state, ring buffers
and event counts -- because every random stream is keyed by global neuron
index and the partitions agree on the bounds of the exact fixed-point
accumulation."""
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


def _run_parts_exchanged(fmt, cuts, steps, params=None, graph=0):
    """The partitions advanced with the device exchange (in one process the
    gathered rows are the local rows: no copy, no host synchronisation),
    eagerly or replaying captured groups of `graph` intervals."""
    import torch
    from paper_2109_12855_gb300 import partition as PT
    pp = params or _params(fmt)
    s = torch.cuda.Stream()  # one stream for every partition
    nets = [PT.create(pp, _conn(fmt), lo, hi, s.cuda_stream)
            for lo, hi in zip(cuts[:-1], cuts[1:])]
    try:
        PT.agree_bounds(nets)
        for net in nets:
            net.finalize()
        xch = PT.DeviceExchange(nets)
        replays = PT.simulate_exchanged(nets, xch, steps, graph_intervals=graph)
        assert (replays > 0) == (graph > 0)
        s.synchronize()
        logs = [net.read_spikes(1 << 21) for net in nets]
        states = [net.read_state() for net in nets]
        rbs = [net.read_rb() for net in nets]
        stats = [net.stats() for net in nets]
        xch.close()
    finally:
        for net in nets:
            net.close()
    src = np.concatenate([s for s, _ in logs])
    t = np.concatenate([tt for _, tt in logs])
    return _sorted(src, t), states, rbs, stats


@pytest.mark.parametrize("fmt", [0, 1], ids=["fp32", "bf16"])
@pytest.mark.parametrize("cuts,graph", [([0, N], 0), ([0, 2500, N], 0),
                                        ([0, 1700, 3333, N], 0), ([0, N], 8),
                                        ([0, 1700, 3333, N], 8)],
                         ids=["1-part", "2-parts", "3-parts", "1-part-graph",
                              "3-parts-graph"])
def test_device_exchange_equals_the_whole_net(fmt, cuts, graph):
    """Update -> device exchange buffers -> delivery read straight from the
    gathered buffers, eagerly or as replayed CUDA graphs (updates from the
    device clock): the union equals the whole net bit for bit (spikes,
    state, ring buffers, events counted on the device)."""
    steps = 1505  # 150 intervals of 10 steps and a short one
    w_ev, (ws, wt), wstate, wrb = _run_whole(fmt, steps)
    (ps, pt), states, rbs, stats = _run_parts_exchanged(fmt, cuts, steps,
                                                        graph=graph)
    assert len(ws) > 2000
    assert np.array_equal(ws, ps) and np.array_equal(wt, pt)
    assert sum(st.events_delivered for st in stats) == w_ev
    for k, (lo, hi) in enumerate(zip(cuts[:-1], cuts[1:])):
        assert stats[k].error_flags == 0
        assert stats[k].t_now == steps
        for a, b in zip(wstate, states[k]):
            assert np.array_equal(a[lo:hi].view(np.uint32) if a.dtype == np.float32
                                  else a[lo:hi], b.view(np.uint32)
                                  if b.dtype == np.float32 else b)
        assert np.array_equal(wrb[:, lo:hi].view(np.uint32), rbs[k].view(np.uint32))


def test_device_exchange_needs_one_stream():
    """Partitions on different streams could read a buffer before its update
    wrote it: DeviceExchange refuses them."""
    import torch
    from paper_2109_12855_gb300 import partition as PT
    from paper_2109_12855_gb300 import snn
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    nets = [PT.create(_params(0), _conn(0), 0, 2500, s1.cuda_stream),
            PT.create(_params(0), _conn(0), 2500, N, s2.cuda_stream)]
    try:
        for net in nets:
            net.finalize()
        assert snn.snn_get_stream(nets[0].h) == s1.cuda_stream
        with pytest.raises(ValueError):
            PT.DeviceExchange(nets)
    finally:
        for net in nets:
            net.close()


def test_exchange_buffer_holds_the_pending_list():
    """After snn_update the attached buffer holds the interval's spikes (the
    pending list's entries, as a multiset), count word first."""
    import torch
    from paper_2109_12855_gb300 import partition as PT
    from paper_2109_12855_gb300 import snn
    net = PT.create(_params(0), _conn(0), 1200, 3900, stream())
    try:
        net.finalize()
        cap = snn.snn_exchange_capacity(net.h)
        # interval 10 steps, refractory 20: one spike per neuron at most
        assert cap == 2700
        buf = torch.zeros(PT.exchange_words(cap), dtype=torch.int32,
                          device="cuda")
        torch.cuda.synchronize()  # the net runs on a stream of its own
        snn.snn_set_exchange(net.h, buf, cap)
        total = 0
        for k in range(40):
            snn.snn_update(net.h, 10 * k, 10)
            src, t = PT._pending(net)
            xs, xt = PT.decode_exchange(buf.view(1, -1))
            assert buf[0].item() == len(src)
            a = np.lexsort((src, t))
            b = np.lexsort((xs, xt))
            assert np.array_equal(src[a], xs[b]) and np.array_equal(t[a], xt[b])
            assert np.all((src >= 1200) & (src < 3900))
            total += len(src)
            snn.snn_deliver_exchanged(net.h, buf.view(1, -1))
        assert total > 100
        assert net.stats().error_flags == 0
        # detached: the buffer is left alone
        snn.snn_set_exchange(net.h, None)
        before = buf.clone()
        snn.snn_update(net.h, 400, 10)
        snn.snn_deliver_pending(net.h)
        snn.snn_sync(net.h)
        assert torch.equal(before, buf)
    finally:
        net.close()


def test_exchanged_delivery_checks_its_arguments_and_entries():
    """Bad calls are refused; entries of a caller's buffer with a source
    outside the population or a step outside the interval are skipped and
    flagged, the valid ones delivered as a gathered list would be."""
    import torch
    from paper_2109_12855_gb300 import partition as PT
    from paper_2109_12855_gb300 import snn
    nets = [PT.create(_params(0), _conn(0), 0, 2500, stream()) for _ in range(2)]
    try:
        for net in nets:
            net.finalize()
        a, b = nets
        cap = 64
        rows = torch.zeros((2, PT.exchange_words(cap)), dtype=torch.int32,
                           device="cuda")
        # no pending update
        with pytest.raises(snn.SnnError) as e:
            snn.snn_deliver_exchanged(a.h, rows)
        assert e.value.code == snn.SNN_E_STATE
        with pytest.raises(ValueError):
            snn.snn_set_exchange(a.h, torch.zeros(64, dtype=torch.int32))
        with pytest.raises(snn.SnnError) as e:
            snn.snn_set_exchange(a.h, rows[0], 0)
        assert e.value.code == snn.SNN_E_ARG
        with pytest.raises(snn.SnnError) as e:
            snn.snn_set_exchange(a.h, rows[0][1:], 8)  # misaligned
        assert e.value.code == snn.SNN_E_ARG
        snn.snn_update(a.h, 0, 10)
        snn.snn_update(b.h, 0, 10)
        for bad in (dict(n_parts=0), dict(n_parts=65), dict(stride_bytes=8),
                    dict(stride_bytes=40)):
            with pytest.raises(snn.SnnError) as e:
                snn.snn_deliver_exchanged(a.h, rows, **bad)
            assert e.value.code == snn.SNN_E_ARG
        host = np.zeros(64, np.int32)
        with pytest.raises(snn.SnnError) as e:
            snn.snn_deliver_exchanged(a.h, host.ctypes.data, 1, 256)
        assert e.value.code == snn.SNN_E_ARG
        # a pending update refuses re-attaching
        with pytest.raises(snn.SnnError) as e:
            snn.snn_set_exchange(a.h, rows[0], cap)
        assert e.value.code == snn.SNN_E_STATE
        # crafted rows: row 0 {valid, bad source, bad step}, row 1 {valid x2}
        h = np.zeros((2, PT.exchange_words(cap)), np.int32)
        ent = [[(17, 3), (N + 5, 4), (30, 10)], [(4999, 0), (2600, 9)]]
        for r, es in enumerate(ent):
            h[r, 0] = len(es)
            for k, (s_, t_) in enumerate(es):
                h[r, 4 + 2 * k], h[r, 5 + 2 * k] = s_, t_
        rows.copy_(torch.from_numpy(h))
        torch.cuda.synchronize()  # the nets run on streams of their own
        snn.snn_deliver_exchanged(a.h, rows)
        snn.snn_deliver_gathered(b.h, np.array([17, 4999, 2600], np.uint32),
                                 np.array([3, 0, 9], np.int32))
        sa, sb = a.stats(), b.stats()
        assert sa.error_flags & snn.SNN_ERRF_BAD_SOURCE
        assert (sb.error_flags & snn.SNN_ERRF_BAD_SOURCE) == 0
        assert sa.events_delivered == sb.events_delivered > 0
        assert np.array_equal(a.read_rb().view(np.uint32), b.read_rb().view(np.uint32))
    finally:
        for net in nets:
            net.close()


def test_undersized_exchange_buffer_is_flagged():
    """A buffer smaller than the interval's spikes keeps its first cap
    entries and raises SNN_ERRF_SPIKE_LIST."""
    import torch
    from paper_2109_12855_gb300 import partition as PT
    from paper_2109_12855_gb300 import snn
    net = PT.create(_params(0), _conn(0), 0, N, stream())
    try:
        net.finalize()
        buf = torch.zeros(PT.exchange_words(2), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        snn.snn_set_exchange(net.h, buf, 2)
        seen = 0
        for k in range(50):
            snn.snn_update(net.h, 10 * k, 10)
            src, _ = PT._pending(net)
            seen = max(seen, len(src))
            snn.snn_deliver_exchanged(net.h, buf.view(1, -1))
        assert seen > 2
        assert net.stats().error_flags & snn.SNN_ERRF_SPIKE_LIST
    finally:
        net.close()


def test_exchanged_delivery_needs_tiled_static_nets():
    import torch
    from paper_2109_12855_gb300 import partition as PT
    from paper_2109_12855_gb300 import snn
    p = _params(0)
    p.deliver_mode = snn.SNN_DELIVER_ATOMIC
    net = PT.create(p, _conn(0), 0, 2500, stream())
    try:
        net.finalize()
        rows = torch.zeros((1, PT.exchange_words(8)), dtype=torch.int32,
                           device="cuda")
        snn.snn_update(net.h, 0, 10)
        with pytest.raises(snn.SnnError) as e:
            snn.snn_deliver_exchanged(net.h, rows)
        assert e.value.code == snn.SNN_E_STATE
    finally:
        net.close()


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
