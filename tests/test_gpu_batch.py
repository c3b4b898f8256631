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


def test_batch_dense_repeats_per_query_k_and_changing_batches():
    """Zipf sets with object bitmaps (the dense graph): repeated keywords
    count once per occurrence, per-query k, and batches of different sizes
    replayed on one plan, against the oracle and the plain search."""
    w = synth.sets(300_000, (16, 256), 1 << 16, 96, (8, 512), 10, config=33)
    rng = np.random.default_rng(5)
    # repeat a few keywords inside some queries (multisets)
    q_kw, q_off = [], [0]
    for q in range(w.n_queries):
        kw = w.q_kw[w.q_off[q]:w.q_off[q + 1]]
        if q % 3 == 0 and len(kw):
            kw = np.concatenate([kw, kw[: rng.integers(1, min(len(kw), 4) + 1)]])
        q_kw.append(kw)
        q_off.append(q_off[-1] + len(kw))
    w.q_kw = np.concatenate(q_kw).astype(np.uint32)
    w.q_off = np.array(q_off, dtype=np.uint32)
    w.k = rng.integers(1, 11, w.n_queries).astype(np.uint32)
    idx = runner.build_index(w, dense_min_df=2000)
    assert idx.info.dense_keywords > 0
    batch = genie.Batch(idx, 96, 1024, 10)
    parts = (w.subset(np.arange(0, 96)), w.subset(np.arange(0, 96, 2)), w.subset(np.arange(40, 41)))
    for part in parts:
        qs = runner.compile_queries(idx, part)
        assert 2 * qs.n_dense_entries >= qs.n_entries  # the dense graph runs
        d_k = runner.to_dev(np.asarray(part.k, dtype=np.uint32))
        ref = oracle.topk(part)
        _check_oracle(_run_batch(batch, qs, 10, d_k=d_k), ref)
        _check_oracle(runner.search(idx, qs, part.k).host(), ref)
