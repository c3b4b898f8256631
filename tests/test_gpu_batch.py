"""The persistent, graph-captured batch path and the autotuner (GPU)."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1603_08390_gb300 import _build, genie, runner

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    genie.load()


def _same(a, b):
    for key in ("ids", "counts", "n_valid"):
        assert np.array_equal(a[key], b[key]), key


def _check_oracle(res, ref):
    for q in range(len(ref["n_valid"])):
        n = int(ref["n_valid"][q])
        assert res["n_valid"][q] == n
        assert np.array_equal(res["ids"][q, :n], ref["ids"][q, :n])
        assert np.array_equal(res["counts"][q, :n], ref["counts"][q, :n])
        assert np.all(res["ids"][q, n:] == 0xFFFFFFFF)


def _run_batch(batch, qs, k, d_k=None):
    out = runner.Outputs(qs.n_queries, k)
    batch.run(qs, out.ids, out.counts, out.n_valid, d_k=d_k)
    torch.cuda.synchronize()
    return out.host()


def test_batch_equals_search_and_oracle_across_replays():
    w = synth.sets(250_000, (16, 256), 1 << 16, 300, (8, 512), 10, config=30)
    idx = runner.build_index(w)
    first, second = w.subset(np.arange(0, 150)), w.subset(np.arange(150, 300))
    batch = genie.Batch(idx, 256, 256, 10)
    for part in (first, second, first):  # graph replays with new descriptors
        qs = runner.compile_queries(idx, part)
        got = _run_batch(batch, qs, 10)
        _same(got, runner.search(idx, qs, 10).host())
        _check_oracle(got, oracle.topk(part))


def test_batch_shapes_and_per_query_k():
    w = synth.lsh(90_000, 64, 50, config=31)
    rng = np.random.default_rng(1)
    ks = rng.integers(1, 51, w.n_queries).astype(np.uint32)
    idx = runner.build_index(w, 13)
    qs = runner.compile_queries(idx, w)
    ref = oracle.topk(w, k=ks)
    for threads, unroll, shift in ((768, 2, 0), (1024, 4, 14), (512, 8, 13)):
        opts = genie.BatchOpts(block_shift=shift, threads=threads, unroll=unroll)
        batch = genie.Batch(idx, 64, qs.max_bound, 50, opts)
        assert batch.info.threads == threads and batch.info.unroll == unroll
        _check_oracle(_run_batch(batch, qs, 50, d_k=runner.to_dev(ks)), ref)


def test_batch_limits_are_statuses():
    w = synth.sets(20_000, (4, 20), 2000, 40, (1, 30), 5, config=32)
    idx = runner.build_index(w)
    qs = runner.compile_queries(idx, w)
    small = genie.Batch(idx, 8, 64, 5)
    out = runner.Outputs(qs.n_queries, 5)
    with pytest.raises(genie.GenieError) as e:
        small.run(qs, out.ids, out.counts, out.n_valid)
    assert e.value.status == genie.GENIE_ERR_CAPACITY
    with pytest.raises(genie.GenieError) as e:
        genie.Batch(idx, 8, 5000, 5)
    assert e.value.status == genie.GENIE_ERR_INVALID_ARG


def test_autotune_and_its_cache(tmp_path):
    w = synth.lsh(120_000, 48, 20, config=33)
    idx = runner.build_index(w, 13)
    qs = runner.compile_queries(idx, w)
    cache = str(tmp_path / "tune.txt")
    a = genie.genie_autotune(idx, qs, 20, cache)
    assert a.from_cache == 0 and a.tuned_ms > 0
    assert a.threads in (512, 768, 896, 1024) and a.unroll in (2, 4, 8)
    b = genie.genie_autotune(idx, qs, 20, cache)
    assert b.from_cache == 1
    assert (b.block_shift, b.threads, b.unroll, b.ht_slots) == (a.block_shift, a.threads, a.unroll,
                                                                 a.ht_slots)
    with open(cache) as f:
        assert len(f.read().strip().splitlines()) == 1
    batch = genie.Batch(idx, 48, qs.max_bound, 20, a)
    _check_oracle(_run_batch(batch, qs, 20), oracle.topk(w))
