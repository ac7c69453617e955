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

``DeviceExchange`` runs the same cycle without any host round trip: each
update also writes its spikes into a fixed-capacity device buffer
(``snn_set_exchange``), the buffers of all partitions are gathered on the
device (one ``all_gather_into_tensor`` on the current stream across ranks;
nothing at all when this process holds every partition), and each delivery
reads the gathered buffers directly (``snn_deliver_exchanged``)::

    update every partition          (snn_update: also fills its buffer)
    all-gather the fixed buffers    (NCCL, device to device; none in-process)
    deliver from the gathered rows  (snn_deliver_exchanged)

The updates start at the device clock (``SNN_T_DEVICE``), so a run of
intervals can be captured into one CUDA graph and replayed
(``DeviceExchange.graph``), as the single-net simulation replays its own.
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


# ---------------------------------------------------------------------------
# device-resident exchange (no host synchronisation per interval)

EXCHANGE_HEADER_WORDS = 4  # count word + 3 alignment words before the entries


def exchange_words(cap: int) -> int:
    """32-bit words of one exchange buffer of at least ``cap`` entries
    (rows of whole 16-byte units)."""
    w = EXCHANGE_HEADER_WORDS + 2 * cap
    return (w + 3) // 4 * 4


def row_capacity(words: int) -> int:
    """Entries a row of ``words`` words holds: the clamp the delivery applies
    to a row's count (a producer writing the row takes the same capacity)."""
    return (words - EXCHANGE_HEADER_WORDS) // 2


class DeviceExchange:
    """Exchange buffers of the local partitions ``nets`` (all on this
    process's current CUDA device and on the stream the caller runs them on:
    the collective and the library calls must be ordered on one stream).

    ``local`` holds one row per local partition, ``gathered`` the rows of
    every partition of every rank in rank order: the all-gather's output,
    a device copy of ``local`` for several partitions in one process (a
    delivery clears its own row when it completes), or ``local`` itself for
    a single partition.  ``cap`` entries per row: by default the largest
    ``snn_exchange_capacity`` of all partitions (``reduce_max`` maps it to
    the maximum over ranks), which can never overflow."""

    def __init__(self, nets, cap: int | None = None, group=None,
                 reduce_max: Callable | None = None):
        import torch
        import torch.distributed as dist
        self.nets = list(nets)
        self.world = (dist.get_world_size(group)
                      if dist.is_available() and dist.is_initialized() else 1)
        # one stream orders every update before every delivery that reads
        # its buffer (and, across ranks, the collective between them)
        streams = {snn.snn_get_stream(net.h) for net in self.nets}
        self.stream = next(iter(streams))
        self._tstream = (torch.cuda.ExternalStream(self.stream) if self.stream
                         else torch.cuda.default_stream())
        self._graphs = {}
        if len(streams) > 1:
            raise ValueError("partitions sharing exchange buffers must run on "
                             "one stream (pass it to create())")
        if self.world > 1 and streams != {torch.cuda.current_stream().cuda_stream}:
            raise ValueError("the partitions must run on the current CUDA "
                             "stream, where the all-gather is ordered")
        if cap is None:
            cap = max(snn.snn_exchange_capacity(net.h) for net in self.nets)
            if reduce_max is not None:
                cap = int(reduce_max(cap))
        words = exchange_words(int(cap))
        self.cap = row_capacity(words)  # the readers' clamp, whole row
        self.group = group
        dev = torch.device("cuda", torch.cuda.current_device())
        self.local = torch.zeros((len(self.nets), words), dtype=torch.int32,
                                 device=dev)
        self.gathered = (self.local if self.world == 1 and len(self.nets) == 1
                         else torch.zeros((self.world * len(self.nets), words),
                                          dtype=torch.int32, device=dev))
        torch.cuda.current_stream().synchronize()  # zeroed before first use
        for k, net in enumerate(self.nets):
            snn.snn_set_exchange(net.h, self.local[k], self.cap)

    def gather(self):
        """All-gather the local rows into ``gathered`` on the nets' stream
        (asynchronous; a device copy in one process, nothing for a single
        partition)."""
        if self.gathered is self.local:
            return
        import torch
        with torch.cuda.stream(self._tstream):
            if self.world > 1:
                allgather_rows(self.local, self.gathered, self.group)
            else:
                self.gathered.copy_(self.local)

    def graph(self, intervals: int, steps: int):
        """A CUDA graph of ``intervals`` exchanged intervals of ``steps``
        steps each (updates from the device clock), captured on the nets'
        stream once and cached; None if this process cannot capture it (the
        caller then runs the intervals eagerly).  Capture happens after at
        least one eager interval has run (pointer checks and kernel
        attributes are then settled)."""
        import torch
        key = (intervals, steps)
        if key not in self._graphs:
            t_now = [net.stats().t_now for net in self.nets]
            g = torch.cuda.CUDAGraph()
            try:
                with torch.cuda.graph(g, stream=self._tstream):
                    for _ in range(intervals):
                        run_interval_exchanged(self.nets, self, steps)
            except RuntimeError:
                # nothing of the capture ran: clear a pending flag the
                # interrupted sequence left and put the clocks back
                g = None
                for net, t in zip(self.nets, t_now):
                    snn.snn_discard_pending(net.h)
                    snn.snn_set_time(net.h, t)
            self._graphs[key] = g
        return self._graphs[key]

    def replay(self, g):
        """Replay a captured graph on the nets' stream (torch launches a
        graph on its current stream)."""
        import torch
        with torch.cuda.stream(self._tstream):
            g.replay()

    def close(self):
        self._graphs.clear()
        for net in self.nets:
            if net.h:
                snn.snn_set_exchange(net.h, None)
        self.nets = []


def allgather_rows(local, gathered=None, group=None):
    """All-gather of fixed-size exchange rows over torch.distributed: every
    rank's ``local`` (rows x words) into ``gathered`` (ranks x rows x words,
    rank-major), one collective with no size exchange before it (NCCL for
    CUDA tensors, gloo for CPU tensors).  Returns ``gathered``."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    if gathered is None:
        gathered = torch.empty((ws * local.shape[0],) + tuple(local.shape[1:]),
                               dtype=local.dtype, device=local.device)
    dist.all_gather_into_tensor(gathered, local, group=group)
    return gathered


def run_interval_exchanged(nets, xch: DeviceExchange, steps: int,
                           t0: int = snn.SNN_T_DEVICE):
    """One interval of the partitioned network with the device exchange:
    asynchronous, no host synchronisation (t0: the interval's first step,
    by default the device clock)."""
    ptr = xch.gathered.data_ptr()
    rows = xch.gathered.shape[0]
    stride = xch.gathered.stride(0) * xch.gathered.element_size()
    for net in nets:
        snn.snn_update(net.h, t0, steps)
    xch.gather()
    for net in nets:
        snn.snn_deliver_exchanged(net.h, ptr, rows, stride)


def simulate_exchanged(nets, xch: DeviceExchange, n_steps: int,
                       interval: int | None = None, graph_intervals: int = 0):
    """Advance the partitions by n_steps from their device clock with the
    device exchange (intervals of the nets' interval length, a shorter last
    one).  graph_intervals > 0 replays a captured CUDA graph of that many
    intervals while whole groups remain (after one eager interval).
    Asynchronous: read the events afterwards from the nets' statistics.
    Returns the number of graph replays."""
    if interval is None:
        interval = nets[0].stats().interval
    left, replays = n_steps, 0
    while left > 0:
        m = min(interval, left)
        g = None
        if (graph_intervals > 0 and left < n_steps
                and left >= graph_intervals * interval):
            g = xch.graph(graph_intervals, interval)
        if g is not None:
            xch.replay(g)
            replays += 1
            left -= graph_intervals * interval
            continue
        run_interval_exchanged(nets, xch, m)
        left -= m
    return replays


def encode_exchange(src, t, cap: int) -> np.ndarray:
    """One exchange row (int32 words, ``exchange_words(cap)`` of them) holding
    the list (src, t); a list longer than the row keeps its count and the
    entries that fit, as an overflowing update does."""
    src = np.asarray(src, np.uint32)
    t = np.asarray(t, np.int32)
    row = np.zeros(exchange_words(cap), np.uint32)
    row[0] = len(src)
    k = min(len(src), row_capacity(len(row)))
    e = row[EXCHANGE_HEADER_WORDS:EXCHANGE_HEADER_WORDS + 2 * k]
    e[0::2] = src[:k]
    e[1::2] = t[:k].view(np.uint32)
    return row.view(np.int32)


def decode_exchange(rows):
    """(src, t) lists of exchange rows (a CPU int32 array or tensor whose
    rows are buffers), concatenated in row order; counts above a row's
    capacity are clamped as the delivery clamps them."""
    a = np.asarray(rows.cpu() if hasattr(rows, "cpu") else rows)
    a = a.reshape(-1, a.shape[-1]).view(np.uint32)
    cap = row_capacity(a.shape[1])
    srcs, ts = [], []
    for r in a:
        n = min(int(r[0]), cap)
        e = r[EXCHANGE_HEADER_WORDS:EXCHANGE_HEADER_WORDS + 2 * n]
        srcs.append(e[0::2])
        ts.append(e[1::2].view(np.int32))
    return (np.concatenate(srcs).astype(np.uint32) if srcs else
            np.zeros(0, np.uint32),
            np.concatenate(ts).astype(np.int32) if ts else np.zeros(0, np.int32))
