"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: the worked
examples of the paper (tests/golden), pure-Python evaluations of Definition
2.1 on tiny inputs, an independent inverted-index scan, a matrix product with
the incidence matrix, closed-form identities, and the invariants of Lemma 3.1
and Theorem 3.1 on a serial replay of Algorithm 1.
"""
import json
import os
import random
from collections import Counter

import numpy as np
import pytest

import oracle
import synth
from oracle import cpq

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _relational_workload(values, queries, k, vpd=64):
    values = np.asarray(values, dtype=np.uint32)
    n, d = values.shape
    item_off = np.zeros(len(queries) + 1, dtype=np.uint32)
    item_off[1:] = np.cumsum([len(q) for q in queries])
    flat = [it for q in queries for it in q]
    return synth.Workload(
        "golden", "relational", n, d * vpd,
        (np.arange(n + 1) * d).astype(np.uint32),
        (np.arange(d, dtype=np.uint32)[None, :] * vpd + values).ravel(),
        len(queries), k, values=values, values_per_dim=vpd, item_off=item_off,
        item_dim=np.array([it[0] for it in flat], dtype=np.uint32),
        item_lo=np.array([it[1] for it in flat], dtype=np.int32),
        item_hi=np.array([it[2] for it in flat], dtype=np.int32))


def _keyword_workload(objects, queries, vocab, k):
    obj_off = np.zeros(len(objects) + 1, dtype=np.uint32)
    obj_off[1:] = np.cumsum([len(o) for o in objects])
    q_off = np.zeros(len(queries) + 1, dtype=np.uint32)
    q_off[1:] = np.cumsum([len(q) for q in queries])
    return synth.Workload(
        "tiny", "keywords", len(objects), vocab, obj_off,
        np.array([e for o in objects for e in o], dtype=np.uint32), len(queries), k,
        q_off=q_off, q_kw=np.array([e for q in queries for e in q], dtype=np.uint32))


def _random_keyword_workload(rng, n_obj, vocab, n_q, obj_len, q_len, k):
    objects = [rng.sample(range(vocab), rng.randint(*obj_len)) for _ in range(n_obj)]
    # queries are multisets: repeated keywords are allowed and count per item
    queries = [[rng.randrange(vocab) for _ in range(rng.randint(*q_len))] for _ in range(n_q)]
    return _keyword_workload(objects, queries, vocab, k), objects, queries


def _python_topk(objects, queries, k):
    """Definition 2.1 with Python sets: MC = sum over items r of |r & O|."""
    out = []
    for q in queries:
        mc = [sum(len({r} & set(o)) for r in q) for o in objects]
        ranked = sorted((c, i) for i, c in enumerate(mc) if c >= 1)
        ranked.sort(key=lambda t: (-t[0], t[1]))
        out.append((mc, ranked[:k]))
    return out


def _check_against(res, expected, k):
    for q, (mc, top) in enumerate(expected):
        n = len(top)
        assert res["n_valid"][q] == n
        assert list(res["ids"][q, :n]) == [i for _, i in top]
        assert list(res["counts"][q, :n]) == [c for c, _ in top]
        assert np.all(res["ids"][q, n:k] == 0xFFFFFFFF)
        assert np.all(res["counts"][q, n:k] == 0)
        assert res["mcsum"][q] == sum(mc)
        nz = sorted((c for c in mc if c >= 1), reverse=True)
        assert res["tk"][q] == (nz[k - 1] if len(nz) >= k else 0)


# --------------------------------------------------------------------------
# worked examples
# --------------------------------------------------------------------------

def test_definition_2_1_example():
    g = _golden("example_2_1.json")
    w = _relational_workload([g["objects"]["O1"]], [g["query"]], k=1)
    res = oracle.topk(w)
    assert res["mcsum"][0] == g["expected_mc"]
    assert res["counts"][0, 0] == g["expected_mc"] and res["ids"][0, 0] == 0
    # one item at a time gives C(r, O1)
    for item, c in zip(g["query"], g["expected_item_counts"]):
        wi = _relational_workload([g["objects"]["O1"]], [[item]], k=1)
        assert oracle.topk(wi)["mcsum"][0] == c


def test_example_3_2_counts_and_top1():
    g = _golden("example_3_2.json")
    objs = [g["objects"][n] for n in ("O1", "O2", "O3")]
    w = _relational_workload(objs, [g["query"]], k=3)
    res = oracle.topk(w)
    by_id = dict(zip(res["ids"][0][:3].tolist(), res["counts"][0][:3].tolist()))
    assert [by_id[i] for i in range(3)] == g["expected_mc"]
    top = oracle.topk(w, k=g["k"])
    assert top["ids"][0, 0] == g["expected_top1"]["id"]
    assert top["counts"][0, 0] == g["expected_top1"]["count"]
    assert top["tk"][0] == g["expected_top1"]["count"]


def test_example_3_2_lists_follow_from_the_tuples():
    g = _golden("example_3_2.json")
    objs = [g["objects"][n] for n in ("O1", "O2", "O3")]
    for (d, lo, hi), lst in zip(g["query"], g["lists_in_scan_order"]):
        assert [i for i, o in enumerate(objs) if lo <= o[d] <= hi] == lst


def test_example_3_2_algorithm_1_trace():
    g = _golden("example_3_2.json")
    state, trace = cpq.replay(g["lists_in_scan_order"], 3, g["maxcount"], g["k"])
    assert len(trace) == len(g["trace"])
    for got, want in zip(trace, g["trace"]):
        assert got["AT"] == want["AT"]
        assert got["ZA"] == want["ZA"]
        assert got["HT"] == {int(o): c for o, c in want["HT"].items()}
        assert got["BC"] == want["BC"]
    assert cpq.select(state) == [(g["expected_top1"]["count"], g["expected_top1"]["id"])]
    # Theorem 3.1: the k-th count is AT - 1
    assert state["AT"] - 1 == g["expected_top1"]["count"]


# --------------------------------------------------------------------------
# brute force vs independent evaluations
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_oracle_equals_python_sets(seed):
    rng = random.Random(seed)
    n_obj = rng.randint(1, 64)
    vocab = rng.randint(4, 40)
    w, objects, queries = _random_keyword_workload(rng, n_obj, vocab, 8, (0, min(vocab, 12)),
                                                   (0, 20), 1)
    for k in (1, 2, 5, n_obj, n_obj + 3):
        res = oracle.topk(w, k=k)
        _check_against(res, _python_topk(objects, queries, k), k)


@pytest.mark.parametrize("seed", range(4))
def test_relational_oracle_equals_python(seed):
    rng = np.random.default_rng(seed)
    n, d, vpd = 200, 6, 16
    values = rng.integers(0, vpd, size=(n, d))
    queries = []
    for _ in range(10):
        q = []
        for _ in range(rng.integers(0, 9)):  # dims may repeat; ranges may leave [0, vpd)
            dim = int(rng.integers(0, d))
            lo = int(rng.integers(-4, vpd + 2))
            q.append((dim, lo, lo + int(rng.integers(-2, 6))))
        queries.append(q)
    for k in (1, 7, n + 1):
        res = oracle.topk(_relational_workload(values, queries, k, vpd))
        for qi, q in enumerate(queries):
            mc = [sum(1 for (dd, lo, hi) in q if lo <= values[o, dd] <= hi) for o in range(n)]
            top = sorted(((c, o) for o, c in enumerate(mc) if c >= 1), key=lambda t: (-t[0], t[1]))
            _check_against({kk: v[qi:qi + 1] for kk, v in res.items()}, [(mc, top[:k])], k)


@pytest.mark.parametrize("seed", range(3))
def test_oracle_equals_cpuidx(seed):
    rng = random.Random(100 + seed)
    w, _, _ = _random_keyword_workload(rng, 3000, 400, 40, (1, 60), (1, 120), 1)
    for k in (1, 10, 100, 5000):
        a, b = oracle.topk(w, k=k), oracle.cpuidx_topk(w, k=k)
        for key in ("ids", "counts", "n_valid", "tk", "mcsum"):
            assert np.array_equal(a[key], b[key]), key


def test_counts_are_the_incidence_product():
    rng = random.Random(7)
    w, _, _ = _random_keyword_workload(rng, 300, 90, 20, (1, 30), (1, 50), 1)
    mc = oracle.counts(w.obj_off, w.obj_kw, w.vocab, w.q_off, w.q_kw).astype(np.int64)
    inc = np.zeros((w.n_objects, w.vocab), dtype=np.int64)
    for o in range(w.n_objects):
        inc[o, w.obj_kw[w.obj_off[o]:w.obj_off[o + 1]]] = 1
    mult = np.zeros((w.n_queries, w.vocab), dtype=np.int64)
    for q in range(w.n_queries):
        np.add.at(mult[q], w.q_kw[w.q_off[q]:w.q_off[q + 1]].astype(np.int64), 1)
    assert np.array_equal(mc, mult @ inc.T)


def test_special_cases_argmax_and_full_sort():
    rng = random.Random(11)
    w, _, _ = _random_keyword_workload(rng, 500, 60, 30, (1, 25), (1, 40), 1)
    mc = oracle.counts(w.obj_off, w.obj_kw, w.vocab, w.q_off, w.q_kw).astype(np.int64)
    top1 = oracle.topk(w, k=1)
    full = oracle.topk(w, k=w.n_objects)
    for q in range(w.n_queries):
        if mc[q].max() >= 1:  # np.argmax returns the first (smallest id) maximum
            assert top1["ids"][q, 0] == np.argmax(mc[q])
            assert top1["counts"][q, 0] == mc[q].max()
        order = np.lexsort((np.arange(w.n_objects), -mc[q]))  # stable: count desc, id asc
        order = order[mc[q][order] >= 1]
        n = len(order)
        assert full["n_valid"][q] == n
        assert np.array_equal(full["ids"][q, :n], order)


def test_checksum_is_sum_of_document_frequencies():
    w = synth.lsh(20_000, 16, 10, config=2)
    df = np.bincount(w.obj_kw, minlength=w.vocab).astype(np.int64)
    res = oracle.topk(w)
    for q in range(w.n_queries):
        kws = w.q_kw[w.q_off[q]:w.q_off[q + 1]]
        assert res["mcsum"][q] == df[kws].sum()
        # a count never exceeds the number of query items
        assert res["counts"][q].max() <= len(kws)


def test_object_range_ranks_only_that_range():
    rng = random.Random(5)
    w, objects, queries = _random_keyword_workload(rng, 400, 50, 12, (1, 20), (1, 30), 1)
    lo, hi = 123, 301
    res = oracle.topk(w, k=9, obj_range=(lo, hi))
    for q, (mc, _) in enumerate(_python_topk(objects, queries, 9)):
        top = sorted(((c, o) for o, c in enumerate(mc) if c >= 1 and lo <= o < hi),
                     key=lambda t: (-t[0], t[1]))[:9]
        assert list(res["ids"][q, :len(top)]) == [o for _, o in top]


def test_per_query_k():
    rng = random.Random(9)
    w, objects, queries = _random_keyword_workload(rng, 100, 30, 6, (1, 10), (1, 15), 1)
    ks = np.array([1, 3, 10, 1, 100, 7], dtype=np.uint32)
    res = oracle.topk(w, k=ks)
    assert res["ids"].shape == (6, 100)
    for q in range(6):
        mc, top = _python_topk(objects, [queries[q]], int(ks[q]))[0]
        assert list(res["ids"][q, :len(top)]) == [o for _, o in top]


def test_rejects_bad_input():
    w = _keyword_workload([[0, 1]], [[5]], vocab=3, k=1)
    with pytest.raises(ValueError):
        oracle.topk(w)
    w = _keyword_workload([[0, 1]], [[1]], vocab=3, k=1)
    with pytest.raises(ValueError):
        oracle.topk(w, k=0)


# --------------------------------------------------------------------------
# c-PQ: Lemma 3.1, Theorem 3.1 and the tie / concurrency readings
# --------------------------------------------------------------------------

def _lists_of(objects, query):
    return [[o for o, obj in enumerate(objects) if kw in obj] for kw in query]


@pytest.mark.parametrize("seed", range(20))
def test_algorithm_1_invariants_and_readout(seed):
    rng = random.Random(1000 + seed)
    n_obj, vocab = rng.randint(5, 60), rng.randint(4, 25)
    objects = [rng.sample(range(vocab), rng.randint(1, vocab)) for _ in range(n_obj)]
    query = [rng.randrange(vocab) for _ in range(rng.randint(1, 12))]
    k = rng.randint(1, 8)
    state, _ = cpq.replay(_lists_of(objects, query), n_obj, len(query), k)
    za, at = state["ZA"], state["AT"]
    mc, top = _python_topk(objects, [query], k)[0]
    nz = sorted((c for c in mc if c >= 1), reverse=True)
    tk = nz[k - 1] if len(nz) >= k else 0
    assert za[at] < k                          # Lemma 3.1
    if at > 1:
        assert za[at - 1] >= k                 # Lemma 3.1
    assert at - 1 == tk                        # Theorem 3.1
    assert cpq.finalize(state) == at           # serial run: nothing left to finalise
    # the HT holds every object with count >= AT, with its exact count
    assert {o: c for o, c in state["HT"].items() if c >= at} == \
        {o: c for o, c in enumerate(mc) if c >= at}
    assert len(state["HT"]) <= k * max(at, 1) + k  # size O(k * AT)
    assert cpq.select(state) == top


@pytest.mark.parametrize("stale", [1, 3, 17, 200])
@pytest.mark.parametrize("seed", range(8))
def test_stale_gate_reads_still_give_exact_topk(stale, seed):
    """Reading of the concurrent update: a gate that sees an old AT only lets
    more objects in; the final pass recomputes AT and the read-out is exact."""
    rng = random.Random(2000 + seed)
    n_obj, vocab = rng.randint(20, 120), rng.randint(6, 30)
    objects = [rng.sample(range(vocab), rng.randint(1, vocab)) for _ in range(n_obj)]
    query = [rng.randrange(vocab) for _ in range(rng.randint(2, 16))]
    k = rng.randint(1, 10)
    lists = _lists_of(objects, query)
    # interleave postings of different lists, as parallel blocks would
    postings = [(i, o) for i, lst in enumerate(lists) for o in lst]
    rng.shuffle(postings)
    state, _ = cpq.replay([[o for _, o in postings]], n_obj, len(query), k, stale=stale)
    assert cpq.select(state) == _python_topk(objects, [query], k)[0][1]
    at_f = cpq.finalize(state)
    nz = sorted((c for c in state["BC"] if c >= 1), reverse=True)
    assert at_f - 1 == (nz[k - 1] if len(nz) >= k else 0)


@pytest.mark.parametrize("seed", range(8))
def test_seeded_gate_is_exact_when_seed_not_above_kth_count(seed):
    """Seeding AT at s <= t_k keeps the read-out exact; AT_f > s or s = 1
    certifies it."""
    rng = random.Random(3000 + seed)
    n_obj, vocab = 80, 12
    objects = [rng.sample(range(vocab), rng.randint(3, vocab)) for _ in range(n_obj)]
    query = [rng.randrange(vocab) for _ in range(10)]
    k = 5
    mc, top = _python_topk(objects, [query], k)[0]
    nz = sorted((c for c in mc if c >= 1), reverse=True)
    tk = nz[k - 1] if len(nz) >= k else 0
    for s in range(1, len(query) + 2):
        state, _ = cpq.replay(_lists_of(objects, query), n_obj, len(query), k, at0=s)
        at_f = cpq.finalize(state)
        certified = s == 1 or at_f > s
        assert certified == (s <= tk or s == 1)
        if certified:
            assert cpq.select(state) == top


def test_serial_equals_counter_semantics():
    """Algorithm 1 BC equals the brute-force count of every object."""
    rng = random.Random(4)
    objects = [rng.sample(range(15), rng.randint(1, 15)) for _ in range(40)]
    query = [rng.randrange(15) for _ in range(9)]
    state, _ = cpq.replay(_lists_of(objects, query), 40, 9, 3)
    assert state["BC"] == [sum(Counter(query)[e] for e in o) for o in objects]
