"""Serving: independent simulation requests batched onto one GPU.

By default a server step runs lanes of batched update and batched
tiled-delivery launches, one each per interval; the persistent mode makes a
step one launch of the persistent serving kernel, which advances every
running net by its own number of intervals (CTAs claim the ready update
blocks and delivery tiles of the nets); the exclusive mode runs one net per
step alone (least remaining work first) with the single-net kernels.
Because tiled delivery sums in exact fixed point and every random
draw is keyed by (neuron, step), a request's spike train must equal, bit for
bit, the same net simulated alone through the single-net path, whatever
else shares its batch, when it was admitted, and how many intervals a step
runs."""
import numpy as np
import pytest

import oracle as O
from gpu_common import need_gpu, stream

pytestmark = pytest.mark.gpu

W_E = O.weight_for_psp(O.Neuron(), 0.1)
GB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _req(n, seed, n_steps, fmt=0, d=(10, 20), nu=20000.0, tag=0):
    from paper_2109_12855_gb300 import snn
    ne = n * 4 // 5
    p = snn.params(n_exc=ne, n_inh=n - ne, weight_format=fmt, nu_ext=nu,
                   w_ext=W_E, seed=seed)
    k = max(1, n // 10)
    ke = k * 4 // 5
    c = snn.conn_params(k_exc=ke, k_inh=k - ke, w_exc=W_E, w_inh=-5 * W_E,
                        d_lo=d[0], d_hi=d[1], seed=seed + 1000)
    return snn.request(p, c, n_steps, user_tag=tag, record_spikes=True)


def _solo(r):
    """The same request run alone through snn_simulate."""
    from paper_2109_12855_gb300 import snn
    p = snn.snn_params.from_buffer_copy(r.params)
    p.spike_log_capacity = 1 << 22
    with snn.Net(p, stream()) as net:
        net.connect_fixed_indegree(r.conn)
        net.finalize()
        snn.snn_simulate(net.h, r.n_steps)
        src, t = net.read_spikes(1 << 22)
        st = net.stats()
        return _sorted(src, t), st.spikes, st.events_delivered


def _sorted(src, t):
    o = np.lexsort((src, t))
    return np.asarray(src)[o], np.asarray(t)[o]


def _drain(sv, ids, max_steps=100000, watch=None):
    from paper_2109_12855_gb300 import snn
    for _ in range(max_steps):
        snn.snn_server_step(sv)
        if watch:
            watch(snn.snn_server_get_stats(sv))
        states = [snn.snn_server_poll(sv, i).state for i in ids]
        if all(s in (snn.SNN_REQ_DONE, snn.SNN_REQ_FAILED,
                     snn.SNN_REQ_CANCELLED) for s in states):
            return
    raise AssertionError("server did not finish")


def _check_equal_to_solo(sv, rid, r):
    from paper_2109_12855_gb300 import snn
    res = snn.snn_server_poll(sv, rid)
    assert res.state == snn.SNN_REQ_DONE, res.error
    (ss, st), sp, ev = _solo(r)
    gs, gt = _sorted(*snn.snn_server_spikes(sv, rid))
    assert len(gs) == res.spikes == sp
    assert res.events == ev
    assert np.array_equal(gs, ss) and np.array_equal(gt, st)
    assert gt.max() < r.n_steps
    return res


def _set_mode(snn, sv, mode):
    snn.snn_server_set_option(sv, snn.SNN_SERVE_OPT_PERSISTENT,
                              int(mode == "persistent"))
    snn.snn_server_set_option(sv, snn.SNN_SERVE_OPT_EXCLUSIVE,
                              int(mode == "exclusive"))


@pytest.mark.parametrize("mode", ["persistent", "lanes", "exclusive"])
@pytest.mark.parametrize("fmt", [0, 1], ids=["fp32", "bf16"])
def test_batched_requests_equal_solo_runs(fmt, mode):
    """Mixed sizes, seeds, delay ranges and lengths (one not a multiple of
    its interval); two requests join while the first two are running."""
    from paper_2109_12855_gb300 import snn
    reqs = [_req(1250, 1, 600, fmt, (10, 20), tag=11),
            _req(5000, 2, 1000, fmt, (15, 25), tag=12),
            _req(3000, 3, 733, fmt, (10, 20), tag=13),
            _req(11250, 4, 400, fmt, (12, 30), nu=15000.0, tag=14)]
    sv = snn.snn_server_create(8 * GB, fmt, stream())
    try:
        _set_mode(snn, sv, mode)
        ids = [snn.snn_server_submit(sv, r) for r in reqs[:2]]
        for _ in range(5):
            snn.snn_server_step(sv)
        ids += [snn.snn_server_submit(sv, r) for r in reqs[2:]]
        _drain(sv, ids)
        for rid, r in zip(ids, reqs):
            res = _check_equal_to_solo(sv, rid, r)
            assert res.user_tag == r.user_tag
            assert res.n_neurons == r.params.n_exc + r.params.n_inh
            assert 0 <= res.t_submit <= res.t_admit <= res.t_start <= res.t_done
            assert res.spikes > 100
        st = snn.snn_server_get_stats(sv)
        assert st.done == 4 and st.failed == 0 and st.active == 0
        assert st.mem_used == 0
        if mode == "persistent":  # one launch per step, several intervals each
            assert st.kernel_launches == st.steps < st.intervals
        else:
            assert st.kernel_launches == 2 * st.intervals
    finally:
        snn.snn_server_destroy(sv)


def test_memory_budget_admits_one_at_a_time():
    from paper_2109_12855_gb300 import snn
    reqs = [_req(3000, 10 + k, 300) for k in range(3)]
    sv = snn.snn_server_create(GB, 0, stream())
    try:
        probe = snn.snn_server_submit(sv, reqs[0])
        need = snn.snn_server_poll(sv, probe).bytes
        _drain(sv, [probe])
        snn.snn_server_release(sv, probe)
    finally:
        snn.snn_server_destroy(sv)
    budget = need + need // 2             # room for one request, not two
    seen = []
    sv = snn.snn_server_create(budget, 0, stream())
    try:
        ids = [snn.snn_server_submit(sv, r) for r in reqs]
        _drain(sv, ids, watch=lambda s: seen.append((s.active, s.mem_used)))
        assert max(a for a, _ in seen) == 1
        assert max(m for _, m in seen) <= budget
        for rid, r in zip(ids, reqs):
            _check_equal_to_solo(sv, rid, r)
        # admission in arrival order
        t_admit = [snn.snn_server_poll(sv, i).t_admit for i in ids]
        assert t_admit == sorted(t_admit)
    finally:
        snn.snn_server_destroy(sv)


def test_autotuner_settles_and_graph_steps_stay_exact():
    """A long request outlives the tuning phase (candidates of 1, 2, 4, 8, 16
    intervals per step); intervals that ran as captured graphs give the same
    spikes as the solo run."""
    from paper_2109_12855_gb300 import snn
    r = _req(5000, 21, 2500)
    sv = snn.snn_server_create(4 * GB, 0, stream())
    try:
        rid = snn.snn_server_submit(sv, r)
        _drain(sv, [rid])
        st = snn.snn_server_get_stats(sv)
        assert st.tuned == 1 and st.intervals_per_step in (1, 2, 4, 8, 16)
        assert st.intervals == 250 and st.steps < 250
        assert st.gpu_ms > 0
        _check_equal_to_solo(sv, rid, r)
    finally:
        snn.snn_server_destroy(sv)


def test_requests_rejected_or_failed():
    from paper_2109_12855_gb300 import snn
    sv = snn.snn_server_create(GB, 0, stream())
    try:
        bad = [_req(1000, 1, 100, fmt=1),            # format differs
               _req(1000, 1, 0),                     # no steps
               _req(200000, 1, 100)]                 # above the budget
        r = _req(1000, 1, 100)
        r.params.deliver_mode = snn.SNN_DELIVER_ATOMIC
        bad.append(r)
        for r in bad:
            with pytest.raises(snn.SnnError) as e:
                snn.snn_server_submit(sv, r)
            assert e.value.code == snn.SNN_E_ARG
        # accepted, then the build rejects delays beyond the ring buffer
        broken = _req(1000, 1, 100, d=(10, 40))
        good = _req(1000, 2, 100)
        ids = [snn.snn_server_submit(sv, broken), snn.snn_server_submit(sv, good)]
        with pytest.raises(snn.SnnError) as e:
            snn.snn_server_spikes(sv, ids[1])
        assert e.value.code == snn.SNN_E_STATE
        _drain(sv, ids)
        res = snn.snn_server_poll(sv, ids[0])
        assert res.state == snn.SNN_REQ_FAILED and res.error == snn.SNN_E_ARG
        _check_equal_to_solo(sv, ids[1], good)
        st = snn.snn_server_get_stats(sv)
        assert (st.done, st.failed, st.mem_used) == (1, 1, 0)
        snn.snn_server_release(sv, ids[1])
        with pytest.raises(snn.SnnError):
            snn.snn_server_poll(sv, ids[1])
    finally:
        snn.snn_server_destroy(sv)


def test_persistent_steps_pace_nets_by_their_own_interval_time():
    """A long small net and a long large net in one persistent kernel: the
    step-length tuner settles, every net runs several intervals per launch,
    and both equal their solo runs."""
    from paper_2109_12855_gb300 import snn
    small, large = _req(2000, 31, 20000, 1), _req(40000, 32, 3000, 1)
    sv = snn.snn_server_create(16 * GB, 1, stream())
    try:
        snn.snn_server_set_option(sv, snn.SNN_SERVE_OPT_PERSISTENT, 1)
        ids = [snn.snn_server_submit(sv, r) for r in (large, small)]
        _drain(sv, ids)
        st = snn.snn_server_get_stats(sv)
        assert st.tuned == 1 and st.intervals_per_step > 1, \
            (st.tuned, st.steps, st.intervals, st.intervals_per_step)
        assert st.intervals == 2000 + 300 and 2 * st.steps < st.intervals
        for rid, r in zip(ids, (large, small)):
            _check_equal_to_solo(sv, rid, r)
        # the small net (2,000 intervals) took less time than the large one
        # (300 intervals) would have at its own pace
        rs, rl = (snn.snn_server_poll(sv, i) for i in (ids[1], ids[0]))
        assert rs.t_done - rs.t_start < (rl.t_done - rl.t_start) * 2000 / 300
    finally:
        snn.snn_server_destroy(sv)


def test_persistent_kernel_wait_limit_fails_the_step_not_the_gpu():
    """A spin limit of one poll makes the persistent kernel give up at once
    (a CTA finds no ready item): its launch ends, the requests it ran fail
    with SNN_E_TIMEOUT, and the server serves the next request normally."""
    from paper_2109_12855_gb300 import snn
    sv = snn.snn_server_create(4 * GB, 0, stream())
    try:
        snn.snn_server_set_option(sv, snn.SNN_SERVE_OPT_PERSISTENT, 1)
        snn.snn_server_set_option(sv, snn.SNN_SERVE_OPT_SPIN_LIMIT, 1)
        bad = [_req(3000, 41 + k, 500) for k in range(2)]
        ids = [snn.snn_server_submit(sv, r) for r in bad]
        _drain(sv, ids)
        for i in ids:
            res = snn.snn_server_poll(sv, i)
            assert res.state == snn.SNN_REQ_FAILED
            assert res.error == snn.SNN_E_TIMEOUT
        snn.snn_server_set_option(sv, snn.SNN_SERVE_OPT_SPIN_LIMIT, 1 << 22)
        good = _req(3000, 45, 500)
        rid = snn.snn_server_submit(sv, good)
        _drain(sv, [rid])
        _check_equal_to_solo(sv, rid, good)
        st = snn.snn_server_get_stats(sv)
        assert (st.done, st.failed, st.mem_used) == (1, 2, 0)
    finally:
        snn.snn_server_destroy(sv)


@pytest.mark.parametrize("mode", ["lanes", "persistent", "exclusive"])
def test_cancel_queued_and_running_requests(mode):
    """Cancelling a queued request removes it before it is built; cancelling
    a running one drops it from its batch (freed once its launched work has
    completed); the others still equal their solo runs; the budget is
    returned; a finished request cannot be cancelled."""
    from paper_2109_12855_gb300 import snn
    keep = _req(3000, 51, 800)
    run_long = _req(5000, 52, 200000)         # would run for a long time
    queued = _req(2000, 53, 500)
    sv = snn.snn_server_create(4 * GB, 0, stream())
    try:
        _set_mode(snn, sv, mode)
        ids = [snn.snn_server_submit(sv, r) for r in (keep, run_long)]
        for _ in range(2000):                 # until both run
            snn.snn_server_step(sv)
            if all(snn.snn_server_poll(sv, i).state == snn.SNN_REQ_RUNNING
                   for i in ids):
                break
        qid = snn.snn_server_submit(sv, queued)
        snn.snn_server_cancel(sv, qid)        # queued or building
        snn.snn_server_cancel(sv, ids[1])     # running
        with pytest.raises(snn.SnnError) as e:
            snn.snn_server_cancel(sv, ids[1])  # already cancelled
        assert e.value.code == snn.SNN_E_STATE
        _drain(sv, ids + [qid])
        for i in (qid, ids[1]):
            assert snn.snn_server_poll(sv, i).state == snn.SNN_REQ_CANCELLED
        _check_equal_to_solo(sv, ids[0], keep)
        with pytest.raises(snn.SnnError) as e:
            snn.snn_server_cancel(sv, ids[0])  # finished
        assert e.value.code == snn.SNN_E_STATE
        st = snn.snn_server_get_stats(sv)
        assert st.done == 1 and st.active == 0 and st.mem_used == 0
        snn.snn_server_release(sv, qid)
    finally:
        snn.snn_server_destroy(sv)


def test_injected_allocation_failures():
    """Host-side fault injection: a device allocation that fails makes
    snn_create and a server's build fail with SNN_E_OOM and leaves the
    library usable (the next net and the next request succeed)."""
    from paper_2109_12855_gb300 import snn
    try:
        snn.snn_debug_fail_allocations(3, 1)  # the 4th allocation fails
        with pytest.raises(snn.SnnError) as e:
            snn.Net(snn.params(n_exc=100, n_inh=25), stream())
        assert e.value.code == snn.SNN_E_OOM
        with snn.Net(snn.params(n_exc=100, n_inh=25), stream()) as net:
            net.finalize()                    # allocations succeed again
        sv = snn.snn_server_create(4 * GB, 0, stream())
        try:
            snn.snn_debug_fail_allocations(0, 1)  # the build's first one
            bad = snn.snn_server_submit(sv, _req(2000, 61, 300))
            _drain(sv, [bad])
            res = snn.snn_server_poll(sv, bad)
            assert res.state == snn.SNN_REQ_FAILED
            assert res.error == snn.SNN_E_OOM
            good = _req(2000, 62, 300)
            rid = snn.snn_server_submit(sv, good)
            _drain(sv, [rid])
            _check_equal_to_solo(sv, rid, good)
            assert snn.snn_server_get_stats(sv).mem_used == 0
        finally:
            snn.snn_server_destroy(sv)
    finally:
        snn.snn_debug_fail_allocations(-1, 0)
