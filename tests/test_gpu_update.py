"""Fused neuron update (exact integration, drive, threshold, refractoriness,
spike compaction) vs the oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import S, need_gpu, stream

pytestmark = pytest.mark.gpu

NM = O.Neuron()


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _bare_net(n, **kw):
    """A net without synapses: interval = n_slots, so updates of up to 32
    steps are allowed."""
    from paper_2109_12855_gb300 import snn
    base = dict(n_exc=n, n_inh=0, init_v_random=0, spike_log_capacity=1 << 20)
    base.update(kw)
    net = snn.Net(snn.params(**base), stream())
    net.finalize()
    return net


def test_closed_form_psp_on_the_gpu():
    """One input of w at step 3: V at step 3 + n equals w psp(n h) within
    1e-6 of the PSP peak (the closed-form pin of the exact integration, on
    the device in FP32).  Bound: the float32 rounding of the propagator
    entries alone moves V by at most 3.3e-7 of the peak over these 400 steps,
    and float32 arithmetic (with or without fused multiply-adds) by a similar
    amount."""
    from paper_2109_12855_gb300 import snn
    w, t_kick = 37.5, 3
    with _bare_net(1, v_th=1e9) as net:
        rb = np.zeros((S, 1), np.float32)
        rb[t_kick] = w
        snn.snn_write_rb(net.h, rb)
        peak = w * O.psp_peak(NM)[0]
        V = []
        for t in range(t_kick + 400):
            snn.snn_simulate(net.h, 1)
            V.append(net.read_state()[0][0])
        for k in range(1, 399):
            want = w * O.psp_unit(NM, k * NM.h)
            assert abs(V[t_kick + k] - want) <= 1e-6 * peak, k


@pytest.mark.parametrize("nu", [8000.0, 30000.0, 120000.0])
def test_poisson_drive_counts_bit_exact(nu):
    """Drive counts are integer decisions on the same Philox word: recover
    each neuron's count from J after one step and compare with the oracle's
    inversion."""
    from paper_2109_12855_gb300 import snn
    n = 4096
    with _bare_net(n, v_th=1e9, nu_ext=nu, w_ext=1.0, seed=99) as net:
        thr = O.poisson_table(nu * 0.1e-3)
        psc = np.float32(np.e / 0.5)
        for t in (0, 1, 2, 3, 4, 1001, 77777):
            snn.snn_write_state(net.h, np.zeros(n, np.float32),
                                np.zeros(n, np.float32),
                                np.zeros(n, np.float32),
                                np.zeros(n, np.int32))
            snn.snn_set_time(net.h, t)
            snn.snn_simulate(net.h, 1)
            J = net.read_state()[2]
            k_gpu = np.rint(J / psc).astype(np.int64)
            k_orc = np.array([O.poisson_count(99, i, t, thr) for i in range(n)])
            assert np.array_equal(k_gpu, k_orc), t
        lam = nu * 1e-4
        assert abs(k_gpu.mean() - lam) < 5 * np.sqrt(lam / n)


@pytest.mark.parametrize("n_steps", [1, 7, 15, 32])
def test_update_from_random_state_matches_oracle(n_steps):
    from paper_2109_12855_gb300 import snn
    n = 3000
    V, I, J, refr = W.random_state(n, seed=n_steps)
    g = W.rng(100 + n_steps)
    rb = g.normal(0, 40.0, (S, n)).astype(np.float32)
    with _bare_net(n, nu_ext=15000.0, w_ext=22.4, seed=5) as net:
        V32, I32, J32 = (x.astype(np.float32) for x in (V, I, J))
        net.write_state(V32, I32, J32, refr)
        snn.snn_write_rb(net.h, rb)
        t0 = 1234
        snn.snn_update(net.h, t0, n_steps)
        gV, gI, gJ, gR = net.read_state()
        gsrc, gt = net.read_spikes()
        snn.snn_discard_pending(net.h)
        grb = net.read_rb()
    st = O.State(V32.astype(np.float64), I32.astype(np.float64),
                 J32.astype(np.float64), refr.copy())
    orb = rb.astype(np.float64)
    osrc, ot = O.update(NM, st, orb, t0, n_steps, 15000.0, 22.4, 5)
    assert sorted(zip(gsrc.tolist(), gt.tolist())) == \
        sorted(zip(osrc.tolist(), ot.tolist()))
    assert np.array_equal(gR, st.refr)
    np.testing.assert_allclose(gV, st.V, rtol=1e-5, atol=2e-4)
    np.testing.assert_allclose(gI, st.I, rtol=1e-5, atol=1e-3)
    np.testing.assert_allclose(gJ, st.J, rtol=1e-5, atol=1e-2)
    # the slots of the updated steps were read and cleared, the rest kept
    used = [(t0 + s) % S for s in range(n_steps)]
    assert not grb[used].any()
    keep = [s for s in range(S) if s not in used]
    assert np.array_equal(grb[keep], rb[keep])


def test_refractory_clamp_and_reset_on_gpu():
    from paper_2109_12855_gb300 import snn
    with _bare_net(1) as net:
        net.write_state([100.0], [0.0], [500.0], [0])
        snn.snn_simulate(net.h, 1)
        V, I, J, r = net.read_state()
        assert V[0] == 0.0 and r[0] == 20
        Vs = []
        for _ in range(25):
            snn.snn_simulate(net.h, 1)
            Vs.append(net.read_state()[0][0])
        assert all(v == 0.0 for v in Vs[:20]) and Vs[20] > 0.0
        src, t = net.read_spikes()
        assert list(t) == [0]


def test_update_requires_delivery_of_pending_spikes():
    from paper_2109_12855_gb300 import snn
    with _bare_net(10) as net:
        snn.snn_update(net.h, 0, 5)
        with pytest.raises(snn.SnnError) as e:
            snn.snn_update(net.h, 5, 5)
        assert e.value.code == snn.SNN_E_STATE
        snn.snn_deliver_pending(net.h)
        snn.snn_update(net.h, 5, 5)
        snn.snn_discard_pending(net.h)
        with pytest.raises(snn.SnnError):
            snn.snn_update(net.h, 10, 33)      # longer than the interval
