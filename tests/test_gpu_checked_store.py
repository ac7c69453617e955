"""Bounds-checked build (libsnn_check.so, compiled with SNN_CHECK): a store
corrupted on purpose -- one record's target outside the net, another's delay
outside the store's delay range -- is delivered without touching memory out
of bounds: both records are skipped, SNN_ERRF_CHECK is raised, and every
other synapse is delivered as Algorithm REF (the FP64 oracle) delivers the
store without the two records.

Runs only in a process that loaded the checked library (SNN_CHECKED=1, as
tests/test_gpu_checked.py starts it): the production kernels trust the
store, so the library refuses the corruption there."""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import need_gpu, stream

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("SNN_CHECKED") != "1",
                                 reason="needs the bounds-checked library")]
S = 32


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    from paper_2109_12855_gb300 import snn
    assert snn.snn_checked()


@pytest.mark.parametrize("fmt", [0, 1], ids=["fp32", "bf16"])
@pytest.mark.parametrize("mode", [0, 1], ids=["tiled", "atomic"])
def test_corrupt_records_are_skipped_and_flagged(fmt, mode):
    from paper_2109_12855_gb300 import snn
    n = 3000
    p = snn.params(n_exc=2400, n_inh=600, weight_format=fmt, deliver_mode=mode,
                   count_events=0, seed=3)
    c = snn.conn_params(k_exc=240, k_inh=60, w_exc=20.0, w_inh=-100.0,
                        sd_exc=2.0, sd_inh=10.0, d_lo=10, d_hi=20, seed=41)
    with snn.Net(p, stream()) as net:
        net.connect_fixed_indegree(c)
        net.finalize()
        rp, tg, dl, w = net.read_store()
        rp = rp.astype(np.int64)
        # two records in the segments of sources that spike below
        bad_t = int(rp[5] + 3)      # target -> outside the net
        bad_d = int(rp[1234] + 7)   # delay  -> above the largest delay
        snn.snn_debug_poke_record(net.h, bad_t, 0, n + 7)
        snn.snn_debug_poke_record(net.h, bad_d, 1, 27)
        src, t = W.random_spikes(n, 400, 0, 10, seed=8)
        src = np.concatenate([src, [5, 1234]]).astype(np.uint32)
        t = np.concatenate([t, [4, 6]]).astype(np.int32)
        net.deliver(src, t)
        st = net.stats()
        assert st.error_flags & snn.SNN_ERRF_CHECK
        assert st.deliver_mode == mode
        keep = np.ones(len(tg), bool)
        keep[[bad_t, bad_d]] = False
        srcs = np.repeat(np.arange(n), np.diff(rp))
        store = O.build_edges(n, srcs[keep], tg[keep], dl[keep].astype(np.int32),
                              w[keep].astype(np.float64))
        rb_o, _, absw, _ = O.deliver_ref(store, S, src, t)
        rb = net.read_rb()
        assert np.all(np.abs(rb - rb_o) <= 1e-5 * absw + 1e-6)


def test_production_library_refuses_corruption_here_only():
    """The checked library reports itself and counts flagged nets."""
    from paper_2109_12855_gb300 import snn
    assert snn.snn_checked()
    assert snn.snn_debug_check_failures() >= 0
