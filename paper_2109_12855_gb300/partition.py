"""Target-partitioned simulation of one network (Section 2.1 of arXiv
2109.12855: neurons are distributed over processes, synapses are stored
with their targets, and the spikes of each min-delay interval are exchanged
once before delivery).

A partition is a net created with ``snn_params.part_lo / part_hi``: it
integrates neurons ``[lo, hi)`` and holds the synapses of every source onto
them.  One interval of the partitioned network is::

    update every partition          (snn_update)
    read each pending list          (snn_read_pending: global sources)
    gather the lists of all parts   (concatenation, or an all-gather)
    deliver the union to each part  (snn_deliver_gathered)

Random streams are keyed by global neuron index and delivery sums are exact
once the partitions agree on the accumulation bounds (``agree_bounds``), so
the union of the partitions is bit-identical to the whole net.  The exchange
is the only collective: ``allgather_spikes`` does it with torch.distributed
(gloo with host tensors, NCCL with device tensors); this module only moves
data, the simulation runs in the library.
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np

from . import snn


def split(n: int, parts: int) -> list[tuple[int, int]]:
    """Boundaries of ``parts`` contiguous ranges covering [0, n)."""
    cuts = [(n * k) // parts for k in range(parts + 1)]
    return [(cuts[k], cuts[k + 1]) for k in range(parts)]


def create(params, conn, lo: int, hi: int, stream=None):
    """A connected (not yet finalized) partition net holding [lo, hi)."""
    p = snn.snn_params.from_buffer_copy(params)
    p.part_lo, p.part_hi = lo, hi
    net = snn.Net(p, stream)
    net.connect_fixed_indegree(conn)
    return net


def local_bounds(nets) -> snn.snn_bounds:
    b = snn.snn_bounds()
    for net in nets:
        x = snn.snn_get_bounds(net.h)
        b.mult_max = max(b.mult_max, x.mult_max)
        b.k_in_max = max(b.k_in_max, x.k_in_max)
        b.max_abs_w = max(b.max_abs_w, x.max_abs_w)
    return b


def agree_bounds(nets, reduce_max: Callable | None = None):
    """Give every partition the largest bounds of all (``reduce_max`` maps
    a (mult_max, k_in_max, max_abs_w) triple to its maximum over ranks)."""
    b = local_bounds(nets)
    if reduce_max is not None:
        m, k, w = reduce_max((b.mult_max, b.k_in_max, b.max_abs_w))
        b.mult_max, b.k_in_max, b.max_abs_w = int(m), int(k), float(w)
    for net in nets:
        snn.snn_set_bounds(net.h, b)


def _pending(net):
    cap = net.n * max(net.stats().interval, 1)
    src = np.zeros(max(cap, 1), np.uint32)
    t = np.zeros(max(cap, 1), np.int32)
    k = snn.snn_read_pending(net.h, src, t)
    return src[:k], t[:k]


def concat_gather(lists: Sequence[tuple[np.ndarray, np.ndarray]]):
    """Exchange for partitions in one process: the union of their lists."""
    if not lists:
        return np.zeros(0, np.uint32), np.zeros(0, np.int32)
    return (np.concatenate([s for s, _ in lists]).astype(np.uint32),
            np.concatenate([t for _, t in lists]).astype(np.int32))


def allgather_spikes(src, t, group=None):
    """Variable-length all-gather of one rank's (src, t) list over
    torch.distributed: counts first, then lists padded to the longest;
    returns the concatenation in rank order.  Host (numpy / CPU) inputs
    travel as CPU tensors (gloo); CUDA tensors stay on the device (NCCL)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    dev = src.device if isinstance(src, torch.Tensor) else torch.device("cpu")
    s = src if isinstance(src, torch.Tensor) else torch.from_numpy(
        np.ascontiguousarray(src, np.int64).astype(np.int32))
    tt = t if isinstance(t, torch.Tensor) else torch.from_numpy(
        np.ascontiguousarray(t, np.int32))
    s = s.to(dev, torch.int32)
    tt = tt.to(dev, torch.int32)
    n = torch.tensor([s.numel()], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(n) for _ in range(ws)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    m = max(max(counts), 1)
    pad = torch.zeros(2, m, dtype=torch.int32, device=dev)
    pad[0, :s.numel()] = s
    pad[1, :tt.numel()] = tt
    out = [torch.zeros_like(pad) for _ in range(ws)]
    dist.all_gather(out, pad, group=group)
    all_s = torch.cat([o[0, :c] for o, c in zip(out, counts)])
    all_t = torch.cat([o[1, :c] for o, c in zip(out, counts)])
    if isinstance(src, torch.Tensor):
        return all_s, all_t
    return (all_s.numpy().astype(np.uint32), all_t.numpy().astype(np.int32))


def run_interval(nets, t0: int, steps: int, gather=None) -> int:
    """One interval of the partitioned network; ``gather`` maps the local
    partitions' union (src, t) to the union over all ranks (None: this
    process holds every partition).  Returns the events the local
    partitions received."""
    lists = []
    for net in nets:
        snn.snn_update(net.h, t0, steps)
        lists.append(_pending(net))
    src, t = concat_gather(lists)
    if gather is not None:
        src, t = gather(src, t)
    events = 0
    for net in nets:
        events += snn.snn_deliver_gathered(net.h, src, t)
    return events


def simulate(nets, n_steps: int, t0: int | None = None, gather=None):
    """Advance the partitions by n_steps (intervals of the nets' interval
    length, a shorter last one).  Returns the events delivered locally."""
    st = nets[0].stats()
    D = st.interval
    t = st.t_now if t0 is None else t0
    end = t + n_steps
    events = 0
    while t < end:
        m = min(D, end - t)
        events += run_interval(nets, t, m, gather)
        t += m
    return events
