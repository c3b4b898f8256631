"""GEN-SPQ ablation (Sec. 6.1.2, Appendix A) and the host-buffer entry point,
on the GPU through the C ABI, against the CPU oracle: ids, counts, padding and
n_valid bit for bit under (count desc, id asc)."""
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


def assert_same(res, ref):
    n_q = len(ref["n_valid"])
    stride = res["ids"].shape[1]
    for q in range(n_q):
        n = int(ref["n_valid"][q])
        assert res["n_valid"][q] == n, (q, res["n_valid"][q], n)
        assert np.array_equal(res["ids"][q, :n], ref["ids"][q, :n]), q
        assert np.array_equal(res["counts"][q, :n], ref["counts"][q, :n]), q
        assert np.all(res["ids"][q, n:stride] == 0xFFFFFFFF), q
        assert np.all(res["counts"][q, n:stride] == 0), q


def spq(idx, w, k=None, buckets=0, max_bytes=0):
    qs = runner.compile_queries(idx, w)
    k = w.k if k is None else k
    if np.isscalar(k):
        kmax, d_k = int(k), None
    else:
        kmax, d_k = int(np.max(k)), runner.to_dev(np.asarray(k, dtype=np.uint32))
    out = runner.Outputs(qs.n_queries, kmax)
    info = genie.genie_search_spq(idx, qs, kmax, out.ids, out.counts, out.n_valid, d_k=d_k,
                                  buckets=buckets, max_bytes=max_bytes)
    torch.cuda.synchronize()
    return out.host(), info


@pytest.mark.parametrize("buckets", [2, 16, 32])
def test_spq_lsh_equals_oracle(buckets):
    w = synth.lsh(150_000, 48, 100, config=61)
    idx = runner.build_index(w)
    res, info = spq(idx, w, buckets=buckets)
    assert_same(res, oracle.topk(w))
    assert info.count_table_bytes_per_query == 4 * w.n_objects
    assert info.list_bytes_per_query == 8 * w.n_objects
    assert info.mean_iterations >= 1


def test_spq_ties_per_query_k_and_passes():
    # many ties at the k-th count (small vocabulary), per-query k, and a memory
    # cap that forces several passes of 7 queries
    w = synth.sets(90_001, (8, 40), 600, 40, (4, 30), 25, config=62)
    rng = np.random.default_rng(3)
    w.k = np.array([1, 10, 25, 64], dtype=np.uint32)[rng.integers(0, 4, w.n_queries)]
    idx = runner.build_index(w)
    res, info = spq(idx, w, max_bytes=7 * 12 * w.n_objects)
    assert info.queries_per_pass == 7 and info.passes == (w.n_queries + 6) // 7
    assert_same(res, oracle.topk(w))


def test_spq_relational_and_k_beyond_n():
    w = synth.relational(n_objects=500, n_queries=16, config=63)
    idx = runner.build_index(w)
    res, _ = spq(idx, w, k=700)  # k > N: every matching object, then padding
    ref = oracle.topk(w, k=700)
    assert_same(res, ref)
    res2 = runner.search(idx, runner.compile_queries(idx, w), 700).host()
    for x in ("ids", "counts", "n_valid"):
        assert np.array_equal(res[x], res2[x])


def test_spq_empty_queries_and_capacity():
    w = synth.sets(20_000, (8, 16), 4096, 6, (1, 5), 10, config=64)
    w.q_off = np.array([0, 0, 3, 3, 5, 5, 8], dtype=np.uint32)  # empty queries in between
    w.q_kw = np.ascontiguousarray(w.obj_kw[:8])
    idx = runner.build_index(w)
    res, _ = spq(idx, w)
    assert_same(res, oracle.topk(w))
    with pytest.raises(genie.GenieError) as e:
        spq(idx, w, max_bytes=1000)
    assert e.value.status == genie.GENIE_ERR_CAPACITY


def test_search_host_equals_device_path_and_oracle():
    w = synth.lsh(120_000, 40, 50, config=65)
    rng = np.random.default_rng(7)
    karr = np.array([1, 7, 50], dtype=np.uint32)[rng.integers(0, 3, w.n_queries)]
    idx = runner.build_index(w)
    Q, k = w.n_queries, 50
    h_q_off = torch.from_numpy(w.q_off.view(np.int32)).pin_memory()
    h_q_kw = torch.from_numpy(w.q_kw.view(np.int32)).pin_memory()
    h_k = torch.from_numpy(karr.view(np.int32)).pin_memory()
    h_ids = torch.empty(Q * k, dtype=torch.int32).pin_memory()
    h_cnt = torch.empty(Q * k, dtype=torch.int32).pin_memory()
    h_nv = torch.empty(Q, dtype=torch.int32).pin_memory()
    for _ in range(2):  # the call returns with the results in host memory
        genie.genie_search_host(idx, h_q_off, h_q_kw, Q, k, h_ids, h_cnt, h_nv, h_k=h_k)
        res = {"ids": h_ids.numpy().view(np.uint32).reshape(Q, k),
               "counts": h_cnt.numpy().view(np.uint32).reshape(Q, k),
               "n_valid": h_nv.numpy().view(np.uint32)}
        w.k = karr
        assert_same(res, oracle.topk(w))
    # pageable host memory works too
    ids = np.zeros(Q * k, dtype=np.uint32)
    cnt = np.zeros(Q * k, dtype=np.uint32)
    nv = np.zeros(Q, dtype=np.uint32)
    addr = lambda a: a.ctypes.data
    genie.genie_search_host(idx, addr(w.q_off), addr(w.q_kw), Q, k, addr(ids), addr(cnt), addr(nv))
    w.k = k
    assert_same({"ids": ids.reshape(Q, k), "counts": cnt.reshape(Q, k), "n_valid": nv},
                oracle.topk(w))
    bad = w.q_off.copy()
    bad[0] = 1
    with pytest.raises(genie.GenieError) as e:
        genie.genie_search_host(idx, addr(bad), addr(w.q_kw), Q, k, addr(ids), addr(cnt), addr(nv))
    assert e.value.status == genie.GENIE_ERR_INVALID_ARG
