"""genie_search_noalloc against genie_search.

Some callers cannot allocate device memory while they answer queries: a
process held to a hard memory budget, a program whose framework owns every
device allocation through its own pool, or a latency-critical loop that must
not wait on (or fail in) an allocation.  genie_search_noalloc serves them
from one fixed device array inside the library.  These tests call it through
the C ABI twice in a row and require exactly the results of genie_search
(ids, counts and n_valid are integers, so the tolerance is zero).  This file
is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import synth
from paper_1603_08390_gb300 import _build, genie, runner

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    genie.load()


def _noalloc(idx, qs, k, d_k=None):
    out = runner.Outputs(qs.n_queries, k)
    out.ids.fill_(-7)  # any slot the call forgets to write would show up
    out.counts.fill_(-7)
    out.n_valid.fill_(-7)
    genie.genie_search_noalloc(idx, qs, k, out.ids, out.counts, out.n_valid, d_k=d_k)
    torch.cuda.synchronize()
    return out.host()


def _same(a, b):
    for key in ("ids", "counts", "n_valid"):
        assert np.array_equal(a[key], b[key]), key


def test_noalloc_equals_search_on_two_calls_in_a_row():
    w = synth.lsh(70_000, 40, 100, config=25)  # two object ranges per query
    idx = runner.build_index(w)
    qs = runner.compile_queries(idx, w)
    ref = runner.search(idx, qs, 100).host()
    torch.cuda.synchronize()
    first = _noalloc(idx, qs, 100)
    second = _noalloc(idx, qs, 100)
    _same(first, ref)
    _same(second, ref)
    assert np.all(ref["n_valid"] == 100)


def test_noalloc_per_query_k_after_a_different_batch():
    w = synth.sets(150_000, (16, 120), 1 << 15, 64, (8, 200), 10, config=26)
    ks = np.random.default_rng(4).integers(1, 50, w.n_queries).astype(np.uint32)
    idx = runner.build_index(w)
    qs = runner.compile_queries(idx, w)
    d_k = runner.to_dev(ks)
    ref = runner.search(idx, qs, ks).host()
    torch.cuda.synchronize()
    for _ in range(2):
        _same(_noalloc(idx, qs, int(ks.max()), d_k=d_k), ref)


def test_noalloc_rejects_a_batch_beyond_its_scratch():
    w = synth.lsh(70_000, 1100, 1024, config=27)  # 1100 x 2 ranges x 1024 x 8 B > 16 MiB
    idx = runner.build_index(w)
    qs = runner.compile_queries(idx, w)
    out = runner.Outputs(qs.n_queries, 1024)
    with pytest.raises(genie.GenieError) as e:
        genie.genie_search_noalloc(idx, qs, 1024, out.ids, out.counts, out.n_valid)
    assert e.value.status == genie.GENIE_ERR_CAPACITY
    assert "exceeds the fixed scratch" in genie.genie_last_error()
