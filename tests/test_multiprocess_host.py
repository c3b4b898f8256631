"""Multi-process paths on CPU with gloo ranks on 127.0.0.1: the benchmark's
replicas (max of step times, disjoint query batches, no data-path
collective), and an object-sharded search whose per-shard lists are gathered
and merged exactly (Sec. 3.4's result merge as the exchange step)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import synth
    r, w, local = bench.dist_setup()
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    mx = bench.max_over_ranks(10.0 + rank * 5.0, w)
    # each rank's batch: its own slice of one query stream
    full = synth.lsh(2000, 8 * world, 5, config=2)
    mine = full.subset(np.arange(rank * 8, (rank + 1) * 8))
    out[rank] = (mx, mine.q_kw.copy())
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_split_queries():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 15.0
    assert not np.array_equal(out[0][1], out[1][1])
    import synth
    full = synth.lsh(2000, 16, 5, config=2)
    assert np.array_equal(np.concatenate([out[0][1], out[1][1]]), full.q_kw)


def _shard_main(rank, world, port, out):
    """One rank of an object-sharded search: the oracle's top-k over this
    rank's object shard stands in for the rank's GPU search; the lists meet on
    rank 0 through the product's exchange (gather + exact host merge)."""
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    import oracle
    import synth
    from paper_1603_08390_gb300 import _build, runner
    _build.build()
    dist.init_process_group("gloo")
    w = synth.sets(3001, (4, 24), 300, 12, (3, 20), 15, config=77)  # ties at the k-th count
    lo, hi = runner.shard_range(w.n_objects, rank, world)
    part = oracle.topk(w, k=15, obj_range=(lo, hi))  # global ids of this shard
    merged = runner.gather_merge(part["ids"], part["counts"], 15)
    if rank == 0:
        out[0] = tuple(np.asarray(a).copy() for a in merged)
    dist.destroy_process_group()


def test_object_sharded_search_merges_exactly_over_gloo_ranks():
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    world = 3
    procs = [ctx.Process(target=_shard_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    ids, counts, nv = out[0]
    w = synth.sets(3001, (4, 24), 300, 12, (3, 20), 15, config=77)
    ref = oracle.topk(w, k=15)
    assert np.array_equal(nv, ref["n_valid"])
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(counts, ref["counts"])
    # the shards' lists alone do not give it: some query's top-k spans shards
    assert any(len({int(i) * 3 // w.n_objects for i in ids[q, :nv[q]]}) > 1 for q in range(len(nv)))
