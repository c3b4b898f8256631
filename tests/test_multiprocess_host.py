"""The N > 1 benchmark path on CPU: two gloo ranks on 127.0.0.1 take the max
of their step times and slice disjoint query batches (weak scaling, no
data-path collective)."""
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
