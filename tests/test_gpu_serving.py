"""The continuous-batching serving loop (GPU): every result is the same alone
and in a mix of overlapping requests, equal to genie_search and the oracle;
the counter budget bounds the queries in flight; bad requests are statuses."""
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


@pytest.fixture(scope="module")
def served():
    w = synth.sets(300_000, (64, 64), 1 << 18, 240, (8, 512), 10, config=40)
    rng = np.random.default_rng(5)
    w.k = np.array([1, 10, 100], dtype=np.uint32)[rng.integers(0, 3, w.n_queries)]
    idx = runner.build_index(w)
    return w, idx


def _row(ids, cnt, n):
    return ids[:n].tolist(), cnt[:n].tolist()


def test_each_result_is_the_same_alone_and_in_the_mix(served):
    w, idx = served
    n_obj = w.n_objects
    # budget for 8 queries of 8-bit counters in flight: a quarter of one slot's batch, so the
    # burst below must be held back however fast the device serves it
    opts = genie.ServerOpts(bc_budget_bytes=8 * n_obj, bits_per_object=8, max_batch=32,
                            k_max=100, streams=3)
    srv = genie.Server(idx, opts)
    q_off = w.q_off.astype(np.int64)
    # alone: one request at a time
    alone = {}
    for i in range(w.n_queries):
        srv.submit(w.q_kw[q_off[i]:q_off[i + 1]], int(w.k[i]), i)
        got = []
        while not got:
            got = srv.poll(4, 200000)
        info, ids, cnt = got[0]
        assert info.tag == i and info.k == w.k[i]
        alone[i] = (info.n_valid,) + _row(ids, cnt, info.n_valid)
    # in the mix: Poisson arrivals at 5M requests/s, all within about 50 us, so
    # requests queue while earlier batches run and the budget holds some back
    rng = np.random.default_rng(6)
    arrival = np.cumsum(rng.exponential(1.0 / 5e6, w.n_queries))
    lat, ids, cnt, nv = srv.replay(w.q_off, w.q_kw, w.k, arrival)
    st = srv.stats()
    assert st.max_queries_in_flight <= 8
    assert st.deferred_admissions > 0       # the budget held requests back
    assert st.launches < 2 * w.n_queries    # requests were batched together
    assert np.all(lat > 0)
    for i in range(w.n_queries):
        assert (nv[i],) + _row(ids[i], cnt[i], nv[i]) == alone[i], i
    # and both equal the library search and the oracle
    qs = runner.compile_queries(idx, w)
    ref = runner.search(idx, qs, w.k).host()
    torch.cuda.synchronize()
    orc = oracle.topk(w)
    for i in range(w.n_queries):
        n = int(orc["n_valid"][i])
        assert nv[i] == n == ref["n_valid"][i]
        assert np.array_equal(ids[i, :n], orc["ids"][i, :n])
        assert np.array_equal(cnt[i, :n], orc["counts"][i, :n])
        assert np.array_equal(ref["ids"][i, :n], orc["ids"][i, :n])
    srv.close()


def test_bad_requests_are_statuses(served):
    w, idx = served
    srv = genie.Server(idx, genie.ServerOpts(bc_budget_bytes=w.n_objects // 2, bits_per_object=8,
                                             k_max=10))
    with pytest.raises(genie.GenieError) as e:
        srv.submit(np.array([1, 2, 3]), 5, 0)      # one query's counters exceed the budget
    assert e.value.status == genie.GENIE_ERR_CAPACITY
    srv.close()
    srv = genie.Server(idx, genie.ServerOpts(k_max=10))
    for kw, k in ((np.array([w.vocab]), 1), (np.array([1]), 0), (np.array([1]), 11)):
        with pytest.raises(genie.GenieError) as e:
            srv.submit(kw, k, 0)
        assert e.value.status == genie.GENIE_ERR_INVALID_ARG
    srv.submit(np.array([], dtype=np.uint32), 3, 7)   # an empty query has no results
    info, ids, cnt = srv.poll(1, 1000000)[0]
    assert info.tag == 7 and info.n_valid == 0 and np.all(ids == 0xFFFFFFFF)
    srv.close()
