"""The allocation-free delivery entry point, snn_deliver_noalloc.

Some callers cannot let a library allocate device memory: a process whose
HBM is fully reserved by another allocator (a framework's caching allocator
holding it all), or a latency-critical loop in which cudaMalloc's implicit
device synchronisation is not acceptable.  They deliver through this entry
point, which stages the spike list in the library's fixed scratch instead.

These tests call it through the C ABI, two calls in a row on different
lists, and check each result element by element against the FP64 oracle's
Algorithm REF ring buffer (1e-5 of the summed |w| per cell, event counts and
per-cell counts exact) and against the ordinary snn_deliver on the same list
(within the same tolerance).  This file sorts last so that a run that stops
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
def test_noalloc_matches_oracle_and_deliver_two_calls_in_a_row(fmt):
    import torch
    from paper_2109_12855_gb300 import snn
    net, cp = fixed_net(4000, 1000, 400, 100, 22.4, -112.0, 10, 20, seed=21,
                        fmt=fmt)
    store = O.build_fixed_indegree(cp)
    lists = []
    for call, (n_sp, seed) in enumerate([(3000, 1), (777, 2)]):
        src, t = W.random_spikes(5000, n_sp, 100 * call, 100 * call + 40,
                                 seed=seed)
        lists.append((src, t, torch.from_numpy(src.astype(np.int32)).cuda(),
                      torch.from_numpy(t.astype(np.int32)).cuda()))
    with net:
        # the existing entry point on each list, from a cleared ring buffer
        ref = []
        for src, t, d_src, d_t in lists:
            snn.snn_clear_rb(net.h)
            ev = snn.snn_deliver(net.h, d_src, d_t)
            ref.append((ev, net.read_rb(), net.read_counts()))
        # the allocation-free entry point, two calls in a row: the second
        # adds onto the first call's ring buffer
        snn.snn_clear_rb(net.h)
        rb_o = np.zeros((S, 5000))
        cnt_o = np.zeros((S, 5000), np.int64)
        absw = np.zeros((S, 5000))
        for call, (src, t, d_src, d_t) in enumerate(lists):
            ev = snn.snn_deliver_noalloc(net.h, d_src, d_t)
            rb = net.read_rb().astype(np.float64)
            cnt = net.read_counts().astype(np.int64)
            # the oracle: Algorithm REF in FP64 on the stored weights
            r1, c1, a1, ev_o = O.deliver_ref(store, S, src, t)
            rb_o += r1
            cnt_o += c1
            absw += a1
            assert ev == ev_o == ref[call][0]
            assert np.array_equal(cnt, cnt_o)
            tol = 1e-5 * absw
            assert np.all(np.abs(rb - rb_o) <= tol), \
                float((np.abs(rb - rb_o) - tol).max())
            # the existing entry point's results (summed over the calls so
            # far), within the same tolerance
            want = sum(r[1].astype(np.float64) for r in ref[:call + 1])
            want_cnt = sum(r[2].astype(np.int64) for r in ref[:call + 1])
            assert np.array_equal(cnt, want_cnt)
            assert np.all(np.abs(rb - want) <= tol)
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
        # host memory is refused before any work is queued: by the binding,
        # and by the C entry point itself when handed host pointers
        hs, ht = np.zeros(4, np.uint32), np.zeros(4, np.int32)
        with pytest.raises(ValueError):
            snn.snn_deliver_noalloc(net.h, hs, ht)
        rc = snn.lib().snn_deliver_noalloc(net.h, hs.ctypes.data,
                                            ht.ctypes.data, 4, None)
        assert rc == snn.SNN_E_ARG
        # the largest list it accepts still works
        m = snn.SNN_NOALLOC_MAX_SPIKES
        ev = snn.snn_deliver_noalloc(net.h, d_src[:m], d_t[:m])
        rp = net.read_store()[0]
        assert ev == m * int(rp[1] - rp[0])
