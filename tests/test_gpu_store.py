"""GPU connection store vs the oracle's: integer parts bit-exact, weights as
stored (FP32 or BF16 rounding of the same FP64 value)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import edge_net, fixed_net, need_gpu, stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _canonical(tg, dl, w, a, b):
    """Row [a, b) sorted by (delay, target, weight)."""
    order = np.lexsort((w[a:b], tg[a:b], dl[a:b]))
    return tg[a:b][order], dl[a:b][order], w[a:b][order]


def _compare(net, store, exact_w=True, fmt=0):
    """Same rows as the oracle's store (order within a row may differ: the
    GPU store is sorted by target tile first); each GPU row is sorted by
    (tile, delay, target)."""
    rp, tg, dl, w = net.read_store()
    st = net.stats()
    assert np.array_equal(rp, store.row_ptr)
    differ = 0
    tw = st.tile_width
    wo = store.w.astype(np.float32)
    dlo = store.delay.astype(np.uint8)
    for i in range(len(rp) - 1):
        a, b = int(rp[i]), int(rp[i + 1])
        if a == b:
            continue
        key = ((tg[a:b] // tw).astype(np.int64) << 40) | \
            (dl[a:b].astype(np.int64) << 32) | tg[a:b]
        assert np.all(np.diff(key) >= 0), i
        gt, gd, gw = _canonical(tg, dl, w, a, b)
        ot, od, ow = _canonical(store.tgt, dlo, wo, a, b)
        assert np.array_equal(gt, ot) and np.array_equal(gd, od), i
        if exact_w:
            assert np.array_equal(gw, ow), i
        else:
            # FP64 normals come from CUDA's and the host's log/cos, which may
            # differ in the last FP64 bit; after rounding to the stored
            # format at most a one-ulp difference can remain, and rarely
            ulp = np.spacing(np.abs(ow)) * (65536.0 if fmt == 1 else 1.0)
            assert np.all(np.abs(gw - ow) <= ulp), i
            differ += int(np.count_nonzero(gw != ow))
    # BF16 stores decide most roundings from an FP32 evaluation with an error
    # bound (the FP64 one only near a rounding boundary): the result is the
    # FP64 path's, so a differing weight stays as rare as a last-bit FP64
    # difference between the two math libraries
    if not exact_w and fmt == 1:
        assert differ <= 1e-4 * max(len(tg), 1), differ


@pytest.mark.parametrize("fmt", [0, 1])
def test_fixed_indegree_store_small(fmt):
    net, cp = fixed_net(400, 100, 40, 10, 22.4, -112.0, 10, 20, seed=3,
                        fmt=fmt)
    with net:
        _compare(net, O.build_fixed_indegree(cp))
        st = net.stats()
        assert st.min_delay == 10 and st.max_delay == 20 and st.interval == 10
        assert st.n_synapses == 500 * 50
        assert st.window == 20 and st.n_tiles * st.tile_width >= 500


@pytest.mark.parametrize("fmt", [0, 1])
def test_fixed_indegree_store_weight_spread(fmt):
    net, cp = fixed_net(800, 200, 80, 20, 22.4, -112.0, 10, 20, seed=17,
                        fmt=fmt, sd_e=2.24, sd_i=11.2)
    with net:
        _compare(net, O.build_fixed_indegree(cp), exact_w=False, fmt=fmt)


@pytest.mark.parametrize("fmt", [0, 1])
def test_fixed_indegree_store_wide_spread_clipped(fmt):
    """Spreads as large as the means: excitatory weights clipped at zero
    (about a sixth of them), inhibitory ones crossing zero -- the BF16
    rounding decided from FP32 near zero and at the clip, against the
    oracle's FP64 values."""
    net, cp = fixed_net(3000, 750, 300, 75, 22.4, -112.0, 10, 20, seed=29,
                        fmt=fmt, sd_e=22.4, sd_i=112.0)
    with net:
        _compare(net, O.build_fixed_indegree(cp), exact_w=False, fmt=fmt)
        w = net.read_store()[3]
        assert np.count_nonzero(w == 0.0) > 0.05 * len(w)


def test_fixed_indegree_store_medium_fixed_delay():
    net, cp = fixed_net(4000, 1000, 400, 100, 22.4, -112.0, 15, 15, seed=5)
    with net:
        _compare(net, O.build_fixed_indegree(cp))
        assert net.stats().interval == 15


@pytest.mark.parametrize("fmt", [0, 1])
def test_edge_store_with_long_segment(fmt):
    # the hub's segment (20,000 synapses) exceeds the shared-memory sort and
    # takes the global-memory path; delays span the full ring
    edges = W.random_edges(3000, 40000, 1, 32, seed=4, hub=77,
                           hub_edges=20000)
    net, store = edge_net(3000, edges, fmt)
    with net:
        _compare(net, store)
        assert net.stats().interval == 1


def test_edge_store_rejects_bad_edges():
    from paper_2109_12855_gb300 import snn
    from gpu_common import stream
    p = snn.params(n_exc=10, n_inh=0)
    with snn.Net(p, stream()) as net:
        with pytest.raises(snn.SnnError) as e:
            net.connect_edges([1], [10], [3], [1.0])       # target >= N
        assert e.value.code == snn.SNN_E_ARG
        with pytest.raises(snn.SnnError):
            net.connect_edges([1], [2], [33], [1.0])       # delay > n_slots
        with pytest.raises(snn.SnnError):
            net.connect_edges([1], [2], [0], [1.0])        # delay 0
        net.connect_edges([1], [2], [3], [1.0])
        with pytest.raises(snn.SnnError) as e:
            net.connect_edges([1], [2], [3], [1.0])        # second connect
        assert e.value.code == snn.SNN_E_STATE


def test_empty_store():
    from paper_2109_12855_gb300 import snn
    from gpu_common import stream
    p = snn.params(n_exc=50, n_inh=0, count_events=1)
    with snn.Net(p, stream()) as net:
        net.finalize()
        st = net.stats()
        assert st.n_synapses == 0 and st.interval == 32
        assert net.deliver([1, 2, 3], [0, 0, 5]) == 0
        assert not net.read_rb().any()


@pytest.mark.parametrize("fmt", [0, 1])
def test_yielding_build_gives_the_same_store(fmt):
    """build_yield (short whole-SM build CTAs, as a server's builds use)
    changes the launch shape, not the store: fixed in-degree and edge-list
    stores (with a segment longer than shared memory) equal the normal
    build bit for bit."""
    from paper_2109_12855_gb300 import snn
    stores = []
    for y in (0, 1):
        p = snn.params(n_exc=4000, n_inh=1000, weight_format=fmt, build_yield=y)
        with snn.Net(p, stream()) as net:
            net.connect_fixed_indegree(snn.conn_params(
                k_exc=400, k_inh=100, w_exc=22.4, w_inh=-112.0, sd_exc=2.0,
                sd_inh=10.0, d_lo=10, d_hi=20, seed=5, clip_exc=1))
            net.finalize()
            stores.append(net.read_store() + (net.stats().tile_width,))
        src, tgt, d, w = W.random_edges(3000, 40000, 1, 20, seed=9, hub=7,
                                        hub_edges=20000)
        p = snn.params(n_exc=3000, n_inh=0, weight_format=fmt, build_yield=y)
        with snn.Net(p, stream()) as net:
            net.connect_edges(src, tgt, d, w)
            net.finalize()
            stores.append(net.read_store())
    fixed, edges = stores[0::2], stores[1::2]
    for other in fixed[1:]:
        assert all(np.array_equal(x, y) for x, y in zip(fixed[0], other))
    for other in edges[1:]:
        assert all(np.array_equal(x, y) for x, y in zip(edges[0], other))
