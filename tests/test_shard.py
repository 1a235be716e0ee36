"""Sharding one search across ranks (host logic, CPU): contiguous entry ranges
balanced by cost, and the candidate merge; a 2-rank gloo run in which each
rank computes its range with the oracle must reproduce the single-process
top candidates."""
import os
import socket

import numpy as np
import pytest

from paper_1703_05581_gb300 import shard, synth


def _plain(orc):
    ts = synth.PLAIN["tsamp"]
    return orc.Config(tsamp=ts, period_min=256 * ts, period_max=512 * ts, widths=(1, 2, 4, 8, 16))


def test_split_entries_cover_and_balance(orc):
    rows, _, _ = orc.plan(orc.Config(tsamp=64e-6, period_min=1.0, period_max=30.0, duty=0.1), 1 << 26)
    for parts in (1, 2, 3, 8):
        rg = shard.split_entries(rows, parts)
        assert rg[0][0] == 0 and rg[-1][1] == len(rows)
        assert all(a[1] == b[0] for a, b in zip(rg, rg[1:]))
        cost = shard.entry_cost(rows)
        per = [cost[b:e].sum() for b, e in rg]
        assert max(per) - min(per) <= 2 * cost.max() + 1e-9 * cost.sum()


def test_merge_candidates_order():
    dt = np.dtype([("trial", "<i8"), ("snr", "<f4")])
    a = np.array([(5, 9.0), (1, 7.0)], dt)
    b = np.array([(3, 9.0), (8, 8.0)], dt)
    m = shard.merge_candidates([a, b], 3)
    assert m["trial"].tolist() == [3, 5, 8]


def _top(records, first, k):
    order = np.lexsort((np.arange(records.size) + first, -records["snr"]))
    return [(int(first + i), float(records["snr"][i])) for i in order[:k]]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle as orc
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    cfg = _plain(orc)
    x = synth.plain_series(seed=5)
    rows, _, _ = orc.plan(cfg, x.size)
    b, e = shard.split_entries(rows, world)[rank]
    z = orc.octave_series(cfg, x)
    rec = orc.fold_score_rows(orc.FOLD_F64, z, rows[b:e], nthreads=2)
    dtype = np.dtype([("trial", "<i8"), ("snr", "<f8")])
    local = np.array(_top(rec, int(rows["first_trial"][b]), 10), dtype)
    gathered = [None] * world
    dist.all_gather_object(gathered, local)
    if rank == 0:
        q.put(shard.merge_candidates(gathered, 10)["trial"].tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_search_matches_single(orc):
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    cfg = _plain(orc)
    ref = orc.search(cfg, synth.plain_series(seed=5), nthreads=os.cpu_count())
    assert got == [t for t, _ in _top(ref, 0, 10)]
