"""Whole-network statistical parity at the benchmark size: the balanced
random network of 112,500 neurons with 1.27e9 synapses (FP32 12-byte
records, delay 1.5 ms, Poisson drive tuned for ~8 Hz; the paper's benchmark
network of Section 2.2) simulated for 1 s of biological time on the GPU and
by the FP64 oracle.  Spiking is chaotic, so the two spike trains diverge
after a few milliseconds; what must agree is the statistics of the
asynchronous irregular state: mean rate within 2 % and mean coefficient of
variation of the inter-spike intervals within 5 %.

The oracle runs in its thread-parallel form (each host thread owns a range
of neurons and the segments onto them), which is bitwise its single-thread
form (tests/test_oracle_threaded.py); it holds the 1.27e9 FP64 synapses in
about 20 GB of host memory."""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import S, need_gpu, stream

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NM = O.Neuron()
# the drive the benchmark uses for ~8 Hz in this network
NU_EXT_8HZ = 25757.293701171875


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _rate_cv(src, t, n, steps):
    rate = len(src) / n / (steps * NM.h * 1e-3)
    order = np.lexsort((t, src))
    s, tt = np.asarray(src)[order], np.asarray(t, np.int64)[order]
    bounds = np.flatnonzero(np.diff(s)) + 1
    cvs = []
    for a, b in zip(np.r_[0, bounds], np.r_[bounds, len(s)]):
        if b - a > 2:
            isi = np.diff(tt[a:b])
            cvs.append(isi.std() / isi.mean())
    return rate, float(np.mean(cvs)), len(cvs)


def test_balanced_112500_one_second_statistics_match_oracle():
    from paper_2109_12855_gb300 import snn
    from paper_2109_12855_gb300.tune import build_balanced
    wl = W.BALANCED_112500
    steps = 10000
    seed = 1
    net, w_e = build_balanced(wl.n_e, wl.n_i, wl.k_e, wl.k_i, wl.d_lo,
                              wl.d_hi, 0, 0.0, seed, stream(),
                              nu_ext=NU_EXT_8HZ, spike_log_capacity=1 << 22)
    with net:
        snn.snn_set_drive(net.h, NU_EXT_8HZ, w_e)
        snn.snn_simulate(net.h, steps)
        g_src, g_t = net.read_spikes(1 << 22)
        st = net.stats()
        assert st.error_flags == 0 and st.t_now == steps
        g_events = st.events_delivered
    g_rate, g_cv, g_n = _rate_cv(g_src, g_t, wl.n, steps)

    w_o = O.weight_for_psp(NM, wl.psp_mv)
    cp = O.Conn(wl.n_e, wl.n_i, wl.k_e, wl.k_i, w_o, -wl.g * w_o, wl.d_lo,
                wl.d_hi, seed + 1000, wfmt=1)
    with O.Threaded(cp, os.cpu_count() or 1) as mt:
        ost = O.State(O.init_v(NM, wl.n, seed), np.zeros(wl.n),
                      np.zeros(wl.n), np.zeros(wl.n, np.int32))
        rb = np.zeros((S, wl.n))
        o_src, o_t, o_events = mt.simulate(NM, wl.d_lo, ost, rb, 0, steps,
                                           NU_EXT_8HZ, w_o, seed,
                                           cap=1 << 22)
    o_rate, o_cv, o_n = _rate_cv(o_src, o_t, wl.n, steps)
    msg = (f"GPU {g_rate:.4f} Hz CV {g_cv:.4f} ({g_n} neurons, {g_events} "
           f"events); oracle {o_rate:.4f} Hz CV {o_cv:.4f} ({o_n}, {o_events})")
    assert 7.0 < o_rate < 9.0, msg            # the tuned ~8 Hz state
    assert abs(g_rate / o_rate - 1.0) <= 0.02, msg
    assert abs(g_cv / o_cv - 1.0) <= 0.05, msg
    # events follow the spikes: every spike delivers its source's segment
    assert abs(g_events / o_events - 1.0) <= 0.03, msg
