"""The continuous-batching serving loop (GPU): every result is the same alone
and in a mix of overlapping requests, equal to genie_search and the oracle;
the device-memory budget bounds the requests in flight, each charged the slot
memory it occupies; bad requests are statuses."""
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
    # a request is charged exactly its share of a launch slot's device buffers:
    # the per-query rows (request_bytes_base) for each of max_batch requests,
    # 4 bytes per keyword of the slot's keyword buffer, and the offsets' end word
    probe = genie.Server(idx, genie.ServerOpts(max_batch=32, k_max=100, streams=3))
    st0 = probe.stats()
    probe.close()
    assert st0.slot_bytes == 32 * st0.request_bytes_base + 4 * 32 * 4096 + 4
    assert st0.mem_budget_bytes == 3 * st0.slot_bytes  # default: every slot's memory
    # a budget of a quarter of one slot, so the burst below must be held back
    # however fast the device serves it
    budget = st0.slot_bytes // 4
    opts = genie.ServerOpts(mem_budget_bytes=budget, max_batch=32, k_max=100, streams=3)
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
    min_request = st0.request_bytes_base + 4 * int(np.diff(w.q_off.astype(np.int64)).min())
    assert st.max_queries_in_flight <= budget // min_request
    assert st.deferred_admissions > 0       # the budget held requests back
    assert st.reserved_bytes == 0 and st.bc_bytes_in_flight == 0  # all returned
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
    srv = genie.Server(idx, genie.ServerOpts(mem_budget_bytes=1000, k_max=10))
    with pytest.raises(genie.GenieError) as e:
        srv.submit(np.array([1, 2, 3]), 5, 0)      # one request's memory exceeds the budget
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
