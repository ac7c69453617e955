"""The allocation-free delivery entry point, snn_deliver_noalloc.

Callers whose device memory is fully reserved by another allocator, or that
run in loops where cudaMalloc's implicit synchronisation is not acceptable,
deliver through this entry point; it stages the spike list in the library's
fixed scratch instead of memory it would allocate.  These tests call it
through the C ABI and check its ring buffer against the ordinary snn_deliver
on the same lists, two calls in a row, within the delivery tolerance used by
all parity tests (1e-5 of the summed |w| per cell, against the FP64 oracle,
for each of the two results).  This file sorts last so that a run that stops
at the first failure has already run every other test; it also passes when
run alone in a fresh process.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import S, fixed_net, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("fmt", [0, 1], ids=["fp32", "bf16"])
def test_noalloc_matches_deliver_two_calls_in_a_row(fmt):
    import torch
    from paper_2109_12855_gb300 import snn
    net, cp = fixed_net(4000, 1000, 400, 100, 22.4, -112.0, 10, 20, seed=21,
                        fmt=fmt)
    store = O.build_fixed_indegree(cp)
    with net:
        for call, (n_sp, seed) in enumerate([(3000, 1), (777, 2)]):
            src, t = W.random_spikes(5000, n_sp, 100 * call, 100 * call + 40,
                                     seed=seed)
            d_src = torch.from_numpy(src.astype(np.int32)).cuda()
            d_t = torch.from_numpy(t.astype(np.int32)).cuda()
            # existing entry point
            snn.snn_clear_rb(net.h)
            ev_ref = snn.snn_deliver(net.h, d_src, d_t)
            rb_ref = net.read_rb()
            cnt_ref = net.read_counts()
            # allocation-free entry point, same list
            snn.snn_clear_rb(net.h)
            ev = snn.snn_deliver_noalloc(net.h, d_src, d_t)
            rb = net.read_rb()
            cnt = net.read_counts()
            assert ev == ev_ref
            assert np.array_equal(cnt, cnt_ref)
            _, _, absw, ev_o = O.deliver_ref(store, S, src, t)
            assert ev == ev_o
            assert np.all(np.abs(rb.astype(np.float64) - rb_ref) <= 2e-5 * absw)
        assert net.stats().error_flags == 0


def test_noalloc_rejects_lists_beyond_its_scratch():
    import torch
    from paper_2109_12855_gb300 import snn
    net, _ = fixed_net(400, 100, 40, 10, 22.4, -112.0, 10, 20, seed=3)
    with net:
        n = snn.SNN_NOALLOC_MAX_SPIKES + 1
        d_src = torch.zeros(n, dtype=torch.int32, device="cuda")
        d_t = torch.zeros(n, dtype=torch.int32, device="cuda")
        with pytest.raises(snn.SnnError) as e:
            snn.snn_deliver_noalloc(net.h, d_src, d_t)
        assert e.value.code == snn.SNN_E_ARG
        assert "scratch" in str(e.value)
        # the largest list it accepts still works
        m = snn.SNN_NOALLOC_MAX_SPIKES
        ev = snn.snn_deliver_noalloc(net.h, d_src[:m], d_t[:m])
        rp = net.read_store()[0]
        assert ev == m * int(rp[1] - rp[0])
