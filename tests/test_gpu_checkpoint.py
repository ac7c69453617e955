"""Determinism and checkpoint/restore.  With tiled delivery the ring-buffer
sums are exact fixed-point integers (order-independent) and every random
draw is a Philox call keyed by (neuron, step), so a simulation is bitwise
reproducible, and a run that is saved, restored into a fresh net and
continued equals the uninterrupted run bit for bit."""
import numpy as np
import pytest

import oracle as O
from gpu_common import need_gpu, stream

pytestmark = pytest.mark.gpu

W_E = O.weight_for_psp(O.Neuron(), 0.1)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _net(fmt=0, seed=7):
    from paper_2109_12855_gb300 import snn
    p = snn.params(n_exc=4000, n_inh=1000, weight_format=fmt, nu_ext=20000.0,
                   w_ext=W_E, seed=seed, spike_log_capacity=1 << 20)
    net = snn.Net(p, stream())
    net.connect_fixed_indegree(snn.conn_params(
        k_exc=400, k_inh=100, w_exc=W_E, w_inh=-5 * W_E, d_lo=10, d_hi=20,
        seed=11))
    net.finalize()
    return net


def _spikes(net):
    src, t = net.read_spikes(1 << 20)
    order = np.lexsort((src, t))
    return src[order], t[order]


@pytest.mark.parametrize("fmt", [0, 1])
def test_simulation_is_bitwise_reproducible(fmt):
    from paper_2109_12855_gb300 import snn
    runs = []
    for _ in range(2):
        with _net(fmt) as net:
            snn.snn_simulate(net.h, 1234)
            runs.append((_spikes(net), net.read_state(), net.read_rb()))
    (s0, st0, rb0), (s1, st1, rb1) = runs
    assert len(s0[0]) > 1000
    assert np.array_equal(s0[0], s1[0]) and np.array_equal(s0[1], s1[1])
    for a, b in zip(st0, st1):
        assert np.array_equal(a, b)
    assert np.array_equal(rb0.view(np.uint32), rb1.view(np.uint32))


def test_checkpoint_restore_continues_bit_for_bit():
    from paper_2109_12855_gb300 import snn
    T1, T2 = 770, 1000        # T1 a multiple of the 10-step interval
    with _net() as a:
        snn.snn_simulate(a.h, T1 + T2)
        sa, ta = _spikes(a)
        full = (a.read_state(), a.read_rb())
    with _net() as b:
        snn.snn_simulate(b.h, T1)
        _spikes(b)
        image = snn.snn_save_state(b.h)
        assert len(image) == snn.snn_state_size(b.h) == 64 + 16 * 5000 + 4 * 32 * 5000
    with _net() as c:
        # scramble the fresh net's state: the image must replace all of it
        g = np.random.default_rng(3)
        c.write_state(g.uniform(0, 20, 5000), g.normal(0, 9, 5000),
                      g.normal(0, 9, 5000), g.integers(0, 20, 5000))
        snn.snn_write_rb(c.h, g.normal(0, 5, (32, 5000)).astype(np.float32))
        snn.snn_set_time(c.h, 123)
        snn.snn_load_state(c.h, image)
        assert c.stats().t_now == T1
        snn.snn_simulate(c.h, T2)
        sc, tc = _spikes(c)
        m = ta >= T1
        assert np.array_equal(sa[m], sc) and np.array_equal(ta[m], tc)
        st, rb = c.read_state(), c.read_rb()
        for x, y in zip(full[0], st):
            assert np.array_equal(x, y)
        assert np.array_equal(full[1].view(np.uint32), rb.view(np.uint32))


def test_restore_rejects_a_foreign_image():
    from paper_2109_12855_gb300 import snn
    p = snn.params(n_exc=10, n_inh=0)
    with snn.Net(p, stream()) as small, _net() as big:
        image = snn.snn_save_state(big.h)
        small.finalize()
        with pytest.raises(snn.SnnError) as e:
            snn.snn_load_state(small.h, image)
        assert e.value.code == snn.SNN_E_ARG
        with pytest.raises(snn.SnnError):
            snn.snn_load_state(big.h, b"x" * len(image))
