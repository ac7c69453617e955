"""Host side of the partitioned network's exchange step on the CPU: two
gloo ranks all-gather variable-length spike lists (one of them empty in one
round) and receive the concatenation in rank order; ranges split the
population exactly."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2109_12855_gb300.partition import allgather_spikes
    res = []
    for rnd in range(3):
        n = 0 if (rnd == 1 and rank == 0) else 5 + 7 * rank + rnd
        src = np.arange(n, dtype=np.uint32) + 1000 * rank
        t = np.full(n, 10 * rnd + rank, np.int32)
        s_all, t_all = allgather_spikes(src, t)
        res.append((s_all.tolist(), t_all.tolist(), str(s_all.dtype)))
    out[rank] = res
    dist.destroy_process_group()


def test_two_rank_allgather_of_spike_lists():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    for rnd, (s_all, t_all, dt) in enumerate(res[0]):
        n0 = 0 if rnd == 1 else 5 + rnd
        n1 = 12 + rnd
        assert s_all == list(range(n0)) + list(range(1000, 1000 + n1))
        assert t_all == [10 * rnd] * n0 + [10 * rnd + 1] * n1
        assert dt == "uint32"


def test_split_covers_the_population():
    from paper_2109_12855_gb300.partition import split
    for n, p in ((5000, 3), (7, 7), (112500, 8), (10, 4)):
        r = split(n, p)
        assert r[0][0] == 0 and r[-1][1] == n and len(r) == p
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert max(h - l for l, h in r) - min(h - l for l, h in r) <= 1


def _rank_rows(rank, world, port, out):
    """Each rank encodes two partitions' lists into fixed-size rows and the
    ranks all-gather the rows (no size exchange first)."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    from paper_2109_12855_gb300 import partition as PT
    cap = 9
    res = []
    for rnd in range(3):
        rows = []
        for part in range(2):
            n = 0 if (rnd == 1 and rank == 0 and part == 1) else 3 + rank + part + rnd
            src = np.arange(n, dtype=np.uint32) + 1000 * rank + 100 * part
            t = np.full(n, 10 * rnd + 2 * rank + part, np.int32)
            rows.append(PT.encode_exchange(src, t, cap))
        local = torch.from_numpy(np.stack(rows))
        g = PT.allgather_rows(local)
        s_all, t_all = PT.decode_exchange(g)
        res.append((tuple(g.shape), s_all.tolist(), t_all.tolist()))
    out[rank] = res
    dist.destroy_process_group()


def test_two_rank_allgather_of_fixed_exchange_rows():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_rows, args=(2, port, out), nprocs=2,
                           join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    for rnd, (shape, s_all, t_all) in enumerate(res[0]):
        assert shape == (4, 24)
        exp_s, exp_t = [], []
        for rank in range(2):
            for part in range(2):
                n = 0 if (rnd == 1 and rank == 0 and part == 1) else 3 + rank + part + rnd
                n = min(n, 9)
                exp_s += list(range(1000 * rank + 100 * part,
                                    1000 * rank + 100 * part + n))
                exp_t += [10 * rnd + 2 * rank + part] * n
        assert s_all == exp_s and t_all == exp_t


def test_exchange_rows_round_trip_and_clamp():
    """Rows are 16-byte multiples; a count above the capacity keeps the
    first cap entries, as the delivery reads them."""
    from paper_2109_12855_gb300 import partition as PT
    for cap in (1, 2, 5, 6):
        w = PT.exchange_words(cap)
        assert w % 4 == 0 and w >= 4 + 2 * cap
        assert cap <= PT.row_capacity(w) <= cap + 1
    src = np.array([5, 7, 2**31 + 3, 11], np.uint32)
    t = np.array([-1, 0, 2**31 - 1, 4], np.int32)
    for cap, keep in ((2, 2), (3, 4), (6, 4)):
        row = PT.encode_exchange(src, t, cap)
        assert row.dtype == np.int32 and row.view(np.uint32)[0] == 4
        s2, t2 = PT.decode_exchange(row[None])
        assert s2.tolist() == src[:keep].tolist()
        assert t2.tolist() == t[:keep].tolist()
    row = PT.encode_exchange(src, t, 2)
    s3, _ = PT.decode_exchange(np.stack([PT.encode_exchange([], [], 2), row]))
    assert s3.tolist() == src[:2].tolist()
