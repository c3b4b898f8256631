"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer results must match bit for bit: ids, counts, padding and n_valid of
every result slot, under the order (count desc, id asc).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import mlp as mlp_ref
from paper_1603_08390_gb300 import _build, genie, runner

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    genie.load()


def assert_same(res, ref, rows=None):
    """res: runner output dict; ref: oracle dict; rows: query ids of ref in res."""
    karr = ref["k"]
    n_q = len(ref["n_valid"])
    rows = np.arange(n_q) if rows is None else np.asarray(rows)
    stride = res["ids"].shape[1]
    for j in range(n_q):
        q = rows[j]
        kq = int(karr[j])
        n = int(ref["n_valid"][j])
        assert res["n_valid"][q] == n, (q, res["n_valid"][q], n)
        assert np.array_equal(res["ids"][q, :n], ref["ids"][j, :n]), q
        assert np.array_equal(res["counts"][q, :n], ref["counts"][j, :n]), q
        assert np.all(res["ids"][q, n:stride] == 0xFFFFFFFF), q
        assert np.all(res["counts"][q, n:stride] == 0), q
        assert n <= kq


def run(w, k=None, chunk_shift=0, opts=None, index=None):
    idx = index or runner.build_index(w, chunk_shift)
    qs = runner.compile_queries(idx, w)
    out = runner.search(idx, qs, w.k if k is None else k, opts=opts)
    torch.cuda.synchronize()
    return out.host(), idx, qs


# ---------------------------------------------------------------------------
# the five workload shapes at test sizes
# ---------------------------------------------------------------------------

def test_relational_tiny_config_full():
    w = synth.config(1)
    res, _, qs = run(w)
    assert qs.max_bound <= 255
    assert_same(res, oracle.topk(w))


@pytest.mark.parametrize("block_shift", [12, 13, 0])
def test_relational_many_ranges_ragged(block_shift):
    w = synth.relational(n_objects=70_001, n_queries=48, config=11)
    res, _, _ = run(w, chunk_shift=12, opts=genie.make_opts(block_shift=block_shift))
    assert_same(res, oracle.topk(w))


@pytest.mark.parametrize("block_shift", [12, 14, 0])
def test_lsh_keywords_small(block_shift):
    w = synth.lsh(60_000, 40, 100, config=12)
    opts = genie.make_opts(block_shift=block_shift)
    res, _, qs = run(w, chunk_shift=12, opts=opts)
    assert qs.max_bound == 256  # 16-bit lanes
    assert_same(res, oracle.topk(w))


def test_zipf_sets_16bit():
    w = synth.sets(200_000, (16, 256), 1 << 16, 96, (8, 512), 10, config=13)
    res, _, qs = run(w)
    assert 16 <= qs.max_bound <= 256
    assert_same(res, oracle.topk(w))


def test_zipf_sets_8bit_per_query_k():
    w = synth.sets(150_000, (64, 64), 1 << 18, 64, (8, 512), 10, config=15)
    rng = np.random.default_rng(3)
    w.k = np.array([1, 10, 100], dtype=np.uint32)[rng.integers(0, 3, w.n_queries)]
    res, _, qs = run(w, chunk_shift=14, opts=genie.make_opts(block_shift=15))
    assert qs.max_bound <= 64
    assert_same(res, oracle.topk(w))


def test_4bit_lanes_short_queries():
    w = synth.sets(90_000, (8, 40), 4096, 70, (1, 15), 25, config=16)
    res, _, qs = run(w, chunk_shift=13)
    assert qs.max_bound <= 15
    assert_same(res, oracle.topk(w))


# Small vocabularies make counts reach the bound B.  B = 7, 127 (and 256 in
# 16-bit lanes) leave every lane's top bit free, so the Gate tests whole
# counter words; B = 8, 15, 128, 255 do not, so it tests each posting's lane.
@pytest.mark.parametrize("vocab,obj_len,b", [
    (12, (3, 11), 7), (20, (5, 18), 8), (20, (5, 19), 15),
    (160, (60, 150), 127), (300, (100, 290), 128), (300, (100, 290), 255),
    (300, (100, 290), 256)])
def test_gate_test_on_both_sides_of_lane_headroom(vocab, obj_len, b):
    w = synth.sets(50_000, obj_len, vocab, 32, (b, b), 10, config=200 + b)
    res, _, qs = run(w, chunk_shift=12)
    assert qs.max_bound == b
    ref = oracle.topk(w)
    assert ref["counts"][:, 0].max() >= b - 3  # counts near the bound
    assert_same(res, ref)


# Every launch shape the library compiles (threads x 16-byte loads per lane),
# on both sides of the lane-headroom limit, with ragged sublists and per-query k.
@pytest.mark.parametrize("threads,unroll", [(768, 2), (768, 4), (896, 2), (1024, 2), (1024, 4),
                                            (512, 2), (512, 4), (512, 8)])
@pytest.mark.parametrize("b", [127, 200])
def test_every_launch_shape(threads, unroll, b):
    w = synth.sets(70_001, (60, 240), 260, 24, (b, b), 10, config=300 + b)
    rng = np.random.default_rng(b)
    w.k = np.array([1, 10, 37], dtype=np.uint32)[rng.integers(0, 3, w.n_queries)]
    res, _, qs = run(w, chunk_shift=13,
                     opts=genie.make_opts(threads=threads, unroll=unroll, block_shift=15))
    assert qs.max_bound == b
    assert_same(res, oracle.topk(w))


def test_search_shape_reports_the_automatic_choice():
    # short sublists (LSH buckets, one object range): 1024 threads, two loads per lane
    w = synth.lsh(60_000, 8, 10, config=12)
    idx = runner.build_index(w)
    qs = runner.compile_queries(idx, w)
    sh = genie.genie_search_shape(idx, qs, 10)
    assert (sh.counter_bits, sh.threads, sh.unroll) == (16, 1024, 2)
    assert sh.kernel_name() == "scan_cpq_kernel<4, 2, 1024, %s>" % ("true" if sh.dense else "false")
    blocks = genie.make_opts()
    runner.search(idx, qs, 10, opts=blocks)
    torch.cuda.synchronize()
    assert blocks._blocks.value == sh.n_groups == 1
    # explicit tuning is taken as given, and checked
    sh = genie.genie_search_shape(idx, qs, 10, genie.make_opts(threads=1024, unroll=4))
    assert (sh.threads, sh.unroll) == (1024, 4)
    with pytest.raises(genie.GenieError) as e:
        genie.genie_search_shape(idx, qs, 10, genie.make_opts(threads=896, unroll=4))
    assert e.value.status == genie.GENIE_ERR_INVALID_ARG
    # long sublists (a small vocabulary, no bitmaps): 512 threads, eight loads per lane
    w = synth.sets(50_000, (100, 290), 300, 8, (128, 128), 10, config=201)
    idx = runner.build_index(w, dense_min_df=genie.GENIE_NO_DENSE)
    qs = runner.compile_queries(idx, w)
    sh = genie.genie_search_shape(idx, qs, 10)
    assert (sh.counter_bits, sh.threads, sh.unroll, sh.dense) == (8, 512, 8, 0)
    # the same lists as bitmaps: nothing long is left to scan, so the short
    # shape (one object range: it cannot be halved)
    idx = runner.build_index(w)
    qs = runner.compile_queries(idx, w)
    sh = genie.genie_search_shape(idx, qs, 10)
    assert (sh.counter_bits, sh.threads, sh.unroll, sh.dense) == (8, 1024, 2, 1)
    assert_same(runner.search(idx, qs, 10).host(), oracle.topk(w))
    # bitmaps with 8-bit counters over several ranges: two 512-thread blocks
    # per SM with two loads per lane, each over half the usual object range
    w = synth.sets(300_000, (16, 64), 1 << 12, 24, (8, 100), 10, config=202)
    idx = runner.build_index(w)
    qs = runner.compile_queries(idx, w)
    sh = genie.genie_search_shape(idx, qs, 10)
    assert (sh.counter_bits, sh.threads, sh.unroll, sh.dense) == (8, 512, 2, 1)
    assert sh.block_shift == 16 and sh.n_groups == 5
    assert_same(runner.search(idx, qs, 10).host(), oracle.topk(w))
    assert_same(runner.search(idx, qs, 10).host(), oracle.topk(w))
    # 4-bit counters keep 768 threads for short sublists (3 items of 5 values: B = 15)
    w = synth.relational(n_objects=70_001, n_queries=8, config=11, items_per_query=3)
    idx = runner.build_index(w)
    qs = runner.compile_queries(idx, w)
    assert qs.max_bound <= 15
    sh = genie.genie_search_shape(idx, qs, 10)
    assert (sh.counter_bits, sh.threads, sh.unroll) == (4, 768, 2)
    assert_same(runner.search(idx, qs, 10).host(), oracle.topk(w))


# ---------------------------------------------------------------------------
# c-PQ invariants on the device state
# ---------------------------------------------------------------------------

def test_final_audit_threshold_is_kth_count_plus_one_per_range():
    """Theorem 3.1 per object range: AT_f - 1 is the range's k-th count."""
    w = synth.lsh(50_000, 12, 20, config=17)
    shift = 13
    idx = runner.build_index(w, 12)
    qs = runner.compile_queries(idx, w)
    groups = (w.n_objects + (1 << shift) - 1) >> shift
    at = torch.zeros(w.n_queries * groups, dtype=torch.int32, device="cuda")
    opts = genie.make_opts(block_shift=shift, d_chunk_at=at, flags=genie.GENIE_SEARCH_PER_RANGE_AT)
    runner.search(idx, qs, w.k, opts=opts)
    at = runner.u32(at).reshape(w.n_queries, groups)
    for g in range(groups):
        lo, hi = g << shift, min(w.n_objects, (g + 1) << shift)
        ref = oracle.topk(w, obj_range=(lo, hi))
        assert np.array_equal(at[:, g] - 1, ref["tk"]), g


def test_shared_audit_threshold_starts_no_higher_than_the_kth_count():
    """With the ranges of a query sharing their k-th counts, each range's
    final AT is at least its own k-th count + 1 and at most the query's."""
    w = synth.lsh(50_000, 12, 20, config=17)
    shift = 13
    idx = runner.build_index(w, 12)
    qs = runner.compile_queries(idx, w)
    groups = (w.n_objects + (1 << shift) - 1) >> shift
    at = torch.zeros(w.n_queries * groups, dtype=torch.int32, device="cuda")
    res = runner.search(idx, qs, w.k, opts=genie.make_opts(block_shift=shift, d_chunk_at=at)).host()
    at = runner.u32(at).reshape(w.n_queries, groups)
    full = oracle.topk(w)
    assert_same(res, full)
    for g in range(groups):
        lo, hi = g << shift, min(w.n_objects, (g + 1) << shift)
        local = oracle.topk(w, obj_range=(lo, hi))
        assert np.all(at[:, g] - 1 >= local["tk"])
        assert np.all(at[:, g] - 1 <= np.maximum(full["tk"], local["tk"]))


def test_compiler_facts_match_the_oracle():
    w = synth.sets(120_000, (16, 200), 1 << 15, 80, (8, 300), 10, config=18)
    idx = runner.build_index(w)
    qs = runner.compile_queries(idx, w)
    facts = runner.query_facts(qs)
    ref = oracle.topk(w)
    # postings scanned by a query = sum over objects of its match count
    assert np.array_equal(facts["entries"], ref["mcsum"])
    assert qs.n_entries == int(ref["mcsum"].sum())
    max_len = int(np.diff(w.obj_off.astype(np.int64)).max())
    qlen = np.diff(w.q_off.astype(np.int64))
    assert np.array_equal(facts["bound"], np.minimum(qlen, max_len))
    assert np.all(ref["counts"].max(axis=1) <= facts["bound"])
    df = np.bincount(w.obj_kw, minlength=w.vocab)
    want = mlp_ref.features(df[w.q_kw], w.q_off)
    assert np.array_equal(facts["features"], want.astype(np.float32))


def test_index_is_the_transpose_of_the_objects():
    w = synth.sets(30_000, (5, 60), 5000, 1, (1, 2), 1, config=19)
    idx = runner.build_index(w)
    kw_off = torch.empty(w.vocab + 1, dtype=torch.int64, device="cuda")
    post = torch.empty(w.nnz, dtype=torch.int32, device="cuda")
    genie.genie_index_export(idx, kw_off, post)
    owner = np.repeat(np.arange(w.n_objects, dtype=np.uint32), np.diff(w.obj_off.astype(np.int64)))
    order = np.lexsort((owner, w.obj_kw))
    want_off = np.concatenate([[0], np.cumsum(np.bincount(w.obj_kw, minlength=w.vocab))])
    assert np.array_equal(kw_off.cpu().numpy(), want_off)
    assert np.array_equal(runner.u32(post), owner[order])
    assert idx.max_object_len == int(np.diff(w.obj_off.astype(np.int64)).max())


@pytest.mark.parametrize("vocab", [1, 2, 256, 257, 70_001, 1 << 25])
def test_index_transpose_every_digit_count(vocab):
    """The 8-bit radix build for vocabularies of 0 to 4 digit passes (the last
    one partial), hot keywords that fill whole warps with one digit, and a
    ragged last tile: lists equal a stable sort of the pairs by keyword."""
    rng = np.random.default_rng(vocab)
    n = 23_457
    lens = rng.integers(0, min(vocab, 40) + 1, n)
    hot = rng.integers(0, vocab, 3)
    objs = []
    for L in lens:
        kw = np.concatenate([hot[: rng.integers(0, 4)], rng.integers(0, vocab, L)])
        objs.append(np.unique(kw)[:max(int(L), 1)] if L else kw[:0])
    obj_off = np.concatenate([[0], np.cumsum([len(o) for o in objs])]).astype(np.uint32)
    obj_kw = np.concatenate(objs).astype(np.uint32)
    w = synth.Workload("radix", "keywords", n, vocab, obj_off, obj_kw, 1, 1,
                       q_off=np.array([0, 1], dtype=np.uint32), q_kw=obj_kw[:1].copy())
    idx = runner.build_index(w)
    kw_off = torch.empty(vocab + 1, dtype=torch.int64, device="cuda")
    post = torch.empty(max(w.nnz, 1), dtype=torch.int32, device="cuda")
    genie.genie_index_export(idx, kw_off, post)
    owner = np.repeat(np.arange(n, dtype=np.uint32), np.diff(obj_off.astype(np.int64)))
    order = np.argsort(obj_kw, kind="stable")
    want_off = np.concatenate([[0], np.cumsum(np.bincount(obj_kw, minlength=vocab))])
    assert np.array_equal(kw_off.cpu().numpy(), want_off)
    assert np.array_equal(runner.u32(post)[: w.nnz], owner[order])


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def _kw_workload(objects, queries, vocab, k):
    obj_off = np.concatenate([[0], np.cumsum([len(o) for o in objects])]).astype(np.uint32)
    q_off = np.concatenate([[0], np.cumsum([len(q) for q in queries])]).astype(np.uint32)
    flat = lambda ll: np.array([e for x in ll for e in x], dtype=np.uint32)
    return synth.Workload("edge", "keywords", len(objects), vocab, obj_off, flat(objects),
                          len(queries), k, q_off=q_off, q_kw=flat(queries))


def test_edge_cases_small():
    objects = [[0, 1, 2], [], [1, 2], [2], [0, 2, 5], [5], [], [3, 4]]
    queries = [[], [6], [2, 2, 2], [0, 1, 2, 5], [3], [1, 1], [7, 6], [0, 1, 2, 3, 4, 5, 6, 7]]
    for k in (1, 2, 3, 8, 9, 50):
        w = _kw_workload(objects, queries, 8, k)
        res, _, _ = run(w)
        assert_same(res, oracle.topk(w))


def test_all_objects_tie():
    n = 40_000
    objects = [[7, 9] for _ in range(n)]
    w = _kw_workload(objects, [[7], [9, 7], [1], [7, 7, 7]], 10, 100)
    res, _, _ = run(w, chunk_shift=12, opts=genie.make_opts(block_shift=12))
    assert_same(res, oracle.topk(w))
    assert list(res["ids"][1, :5]) == [0, 1, 2, 3, 4]


def test_k_larger_than_objects_and_repeat_determinism():
    w = synth.sets(3000, (4, 30), 600, 20, (1, 60), 1, config=20)
    idx = runner.build_index(w)
    for k in (1, 7, 1000, 1024):
        qs = runner.compile_queries(idx, w)
        a = runner.search(idx, qs, k).host()
        b = runner.search(idx, qs, k).host()
        torch.cuda.synchronize()
        for key in a:
            assert np.array_equal(a[key], b[key])
        assert_same(a, oracle.topk(w, k=k))


def test_two_streams_share_one_index():
    w = synth.lsh(40_000, 32, 50, config=21)
    idx = runner.build_index(w)
    qs = runner.compile_queries(idx, w)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    o1 = runner.Outputs(w.n_queries, 50)
    o2 = runner.Outputs(w.n_queries, 50)
    torch.cuda.synchronize()
    genie.genie_search(idx, qs, 50, o1.ids, o1.counts, o1.n_valid, stream=s1)
    genie.genie_search(idx, qs, 50, o2.ids, o2.counts, o2.n_valid, stream=s2)
    torch.cuda.synchronize()
    a, b = o1.host(), o2.host()
    for key in a:
        assert np.array_equal(a[key], b[key])
    assert_same(a, oracle.topk(w))


def test_hash_table_overflow_falls_back_exactly():
    w = synth.lsh(80_000, 24, 100, config=22)
    stats = torch.zeros(8, dtype=torch.int64, device="cuda")
    # per-range AT: every block runs the Gate, so the fallback is the hash table's
    res, _, _ = run(w, chunk_shift=13, opts=genie.make_opts(block_shift=13, ht_slots=32,
                                                             d_stats=stats,
                                                             flags=genie.GENIE_SEARCH_PER_RANGE_AT))
    assert_same(res, oracle.topk(w))
    st = stats.cpu().numpy()
    assert st[4] == w.n_queries * ((w.n_objects + 8191) >> 13)
    assert st[2] > 0  # the Bitmap-Counter selection ran
    assert st[5] == 0  # no inconsistent ids
    assert st[6] == 0  # no block skipped the Gate


def test_seeded_gate_verify_and_rerun():
    w = synth.lsh(60_000, 32, 30, config=23)
    ref = oracle.topk(w)
    idx = runner.build_index(w, 12)
    qs = runner.compile_queries(idx, w)
    rng = np.random.default_rng(5)
    tk = ref["tk"].astype(np.int64)
    for seeds in (np.maximum(tk, 1), tk + 1, np.ones_like(tk), tk + rng.integers(-3, 4, len(tk)),
                  np.full_like(tk, 300)):
        seeds = np.clip(seeds, 0, 1000).astype(np.uint32)
        stats = torch.zeros(8, dtype=torch.int64, device="cuda")
        d_seed = runner.to_dev(seeds)
        out = runner.search(idx, qs, w.k, opts=genie.make_opts(d_seed=d_seed, block_shift=13,
                                                               d_stats=stats))
        torch.cuda.synchronize()
        assert_same(out.host(), ref)
        reruns = int(stats.cpu().numpy()[3])
        expect = int(np.sum((seeds > 1) & (seeds > tk)))
        assert reruns == expect


# ---------------------------------------------------------------------------
# errors are statuses, never faults
# ---------------------------------------------------------------------------

def _expect(status, fn, *a, **kw):
    with pytest.raises(genie.GenieError) as e:
        fn(*a, **kw)
    assert e.value.status == status
    assert genie.genie_last_error()


def test_invalid_inputs_return_status():
    d = runner.to_dev
    off = d(np.array([0, 2, 3], np.uint32))
    E = genie.GENIE_ERR_INVALID_ARG
    _expect(E, genie.genie_build_index, off, d(np.array([0, 9, 1], np.uint32)), 2, 5)  # kw >= vocab
    _expect(E, genie.genie_build_index, off, d(np.array([1, 1, 0], np.uint32)), 2, 5)  # repeat in set
    _expect(E, genie.genie_build_index, d(np.array([0, 3, 2], np.uint32)),
            d(np.array([0, 1, 2], np.uint32)), 2, 5)                                    # offsets
    _expect(E, genie.genie_build_index, d(np.array([1, 2, 3], np.uint32)),
            d(np.array([0, 1, 2], np.uint32)), 2, 5)                                    # off[0] != 0
    _expect(E, genie.genie_build_index, off, d(np.array([0, 1, 2], np.uint32)), 2, 5, 30)  # shift
    idx = genie.genie_build_index(off, d(np.array([0, 1, 2], np.uint32)), 2, 5)
    _expect(E, genie.genie_make_queries, idx, d(np.array([0, 1], np.uint32)),
            d(np.array([5], np.uint32)), 1)                                             # kw >= vocab
    _expect(E, genie.genie_make_queries, idx, d(np.array([0, 2, 1], np.uint32)),
            d(np.array([1, 2], np.uint32)), 2)                                          # offsets
    long_q = np.zeros(5000, np.uint32)
    big = genie.genie_build_index(d(np.arange(0, 5000 * 1 + 1, 1).astype(np.uint32)),
                                  d(np.zeros(5000, np.uint32)), 5000, 1)
    _expect(E, genie.genie_make_queries, big, d(np.array([0, 5000], np.uint32)), d(long_q), 1)
    qs = genie.genie_make_queries(idx, d(np.array([0, 2], np.uint32)), d(np.array([1, 2], np.uint32)), 1)
    o = runner.Outputs(1, 4)
    _expect(E, genie.genie_search, idx, qs, 0, o.ids, o.counts, o.n_valid)
    _expect(E, genie.genie_search, idx, qs, 2000, o.ids, o.counts, o.n_valid)
    _expect(E, genie.genie_search, idx, qs, 4, o.ids, o.counts, o.n_valid,
            d_k=d(np.array([5], np.uint32)))                                            # k_q > k
    _expect(E, genie.genie_search, idx, qs, 4, o.ids, o.counts, o.n_valid,
            opts=genie.make_opts(ht_slots=100))                                         # not pow2
    other = genie.genie_build_index(off, d(np.array([0, 1, 2], np.uint32)), 2, 5)
    _expect(E, genie.genie_search, other, qs, 4, o.ids, o.counts, o.n_valid)          # foreign
    rel = genie.genie_build_index(d(np.array([0, 2], np.uint32)), d(np.array([1, 66], np.uint32)), 1, 128)
    io = d(np.array([0, 1], np.uint32))
    _expect(E, genie.genie_compile_ranges, rel, 64, io, d(np.array([0], np.uint32)),
            d(np.array([5], np.int32)), d(np.array([4], np.int32)), 1)                 # lo > hi
    _expect(E, genie.genie_compile_ranges, rel, 64, io, d(np.array([2], np.uint32)),
            d(np.array([0], np.int32)), d(np.array([4], np.int32)), 1)                 # dim
    # still usable afterwards
    genie.genie_search(idx, qs, 4, o.ids, o.counts, o.n_valid)
    torch.cuda.synchronize()
    assert runner.u32(o.n_valid)[0] == 2


# ---------------------------------------------------------------------------
# full-size workloads, in the launch configuration the benchmark uses
# ---------------------------------------------------------------------------

def _sampled(w, n_sample, seed):
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(w.n_queries, size=n_sample, replace=False))
    return rows, oracle.topk(w.subset(rows))


def test_full_lsh_1m_sampled():
    w = synth.config(2)
    res, idx, qs = run(w)
    rows, ref = _sampled(w, 24, 0)
    assert_same(res, ref, rows)
    assert np.all(res["n_valid"] == 100)


def test_full_zipf_4m_sampled():
    w = synth.config(3)
    res, idx, qs = run(w)
    rows, ref = _sampled(w, 12, 1)
    assert_same(res, ref, rows)


def test_full_lsh_4m_sampled():
    w = synth.config(4)
    res, idx, qs = run(w)
    rows, ref = _sampled(w, 8, 2)
    assert_same(res, ref, rows)


def test_full_serving_index_8m_per_query_k_sampled():
    w = synth.config(5)
    res, idx, qs = run(w)
    assert qs.max_bound <= 64  # 8-bit counters
    rows, ref = _sampled(w, 12, 3)
    assert_same(res, ref, rows)


@pytest.mark.parametrize("maker", [lambda: synth.lsh(60_000, 32, 100, config=34),
                                   lambda: synth.sets(150_000, (16, 256), 1 << 16, 48, (8, 512), 10,
                                                      config=35),
                                   lambda: synth.relational(n_objects=40_000, n_queries=32,
                                                            config=36)])
def test_gateless_ablation_selects_the_same_topk(maker):
    """Counting first and selecting from the Bitmap Counter alone (the
    GEN-SPQ-style ablation) gives exactly the c-PQ results."""
    w = maker()
    res, _, _ = run(w, chunk_shift=13, opts=genie.make_opts(block_shift=14,
                                                             flags=genie.GENIE_SEARCH_NO_GATE))
    assert_same(res, oracle.topk(w))


def test_calibration_measures_a_positive_atomic_rate():
    cal = genie.genie_calibrate()
    assert cal.sms >= 1 and cal.seconds > 0
    assert 1e9 < cal.smem_atomics_per_s < 1e14


# ---------------------------------------------------------------------------
# dense keywords: object bitmaps added whole instead of their lists scanned
# ---------------------------------------------------------------------------

def _index_info(idx):
    return idx.info


@pytest.mark.parametrize("maker,k", [
    (lambda: synth.lsh(150_000, 40, 100, config=51), 100),                       # 16-bit lanes
    (lambda: synth.sets(120_000, (16, 200), 1 << 12, 48, (8, 300), 10, config=52), 10),
    (lambda: synth.sets(90_000, (8, 40), 2000, 40, (4, 60), 25, config=53), 25),  # 8-bit lanes
    (lambda: synth.relational(n_objects=60_000, values_per_dim=16, n_queries=32, config=54), 10)])
def test_dense_bitmaps_give_the_counts_of_the_lists(maker, k):
    """The default index stores dense keywords also as bitmaps; a search adds
    them whole.  Results equal the index without bitmaps, the search told to
    scan every list, and the oracle; the statistics show bitmaps were added."""
    w = maker()
    dense = runner.build_index(w)
    plain = runner.build_index(w, dense_min_df=genie.GENIE_NO_DENSE)
    assert dense.info.dense_keywords > 0 and plain.info.dense_keywords == 0
    assert dense.info.dense_min_df == max(64, (w.n_objects + 31) // 32)
    qd, qp = runner.compile_queries(dense, w), runner.compile_queries(plain, w)
    st = torch.zeros(8, dtype=torch.int64, device="cuda")
    a = runner.search(dense, qd, k, opts=genie.make_opts(d_stats=st,
                                                         flags=genie.GENIE_SEARCH_DENSE)).host()
    b = runner.search(plain, qp, k).host()
    c = runner.search(dense, qd, k, opts=genie.make_opts(flags=genie.GENIE_SEARCH_NO_DENSE)).host()
    d = runner.search(dense, qd, k).host()  # the library's own choice
    torch.cuda.synchronize()
    assert int(st[7].item()) > 0
    for x in ("ids", "counts", "n_valid"):
        assert np.array_equal(a[x], b[x]) and np.array_equal(a[x], c[x])
        assert np.array_equal(a[x], d[x])
    assert_same(a, oracle.topk(w, k=k))


@pytest.mark.parametrize("min_df,shift", [(1, 0), (1, 13), (40, 14)])
def test_every_keyword_dense_and_long_queries(min_df, shift):
    """Bitmaps for (almost) every keyword: queries with more than 255 (and
    more than 1024) dense keywords take several batches of adders; ranges of
    every width; per-query k."""
    w = synth.sets(70_001, (60, 240), 1500, 16, (300, 1200), 10, config=55)
    rng = np.random.default_rng(5)
    w.k = np.array([1, 10, 37], dtype=np.uint32)[rng.integers(0, 3, w.n_queries)]
    idx = runner.build_index(w, 13, dense_min_df=min_df)
    assert idx.info.dense_keywords > 0
    res, _, qs = run(w, index=idx, opts=genie.make_opts(block_shift=shift,
                                                         flags=genie.GENIE_SEARCH_DENSE))
    assert_same(res, oracle.topk(w))


def test_dense_gate_state_per_range():
    """With bitmaps and every range running the Gate from AT = 1, the
    ZipperArray set from the bitmap counts keeps Theorem 3.1: AT_f - 1 is each
    range's k-th count; and 8-bit lanes without headroom (B = 200)."""
    for w, shift in ((synth.lsh(50_000, 12, 20, config=17), 13),
                     (synth.sets(50_000, (100, 290), 300, 10, (200, 200), 10, config=56), 14)):
        idx = runner.build_index(w, 12, dense_min_df=100)
        assert idx.info.dense_keywords > 0
        qs = runner.compile_queries(idx, w)
        groups = (w.n_objects + (1 << shift) - 1) >> shift
        at = torch.zeros(w.n_queries * groups, dtype=torch.int32, device="cuda")
        opts = genie.make_opts(block_shift=shift, d_chunk_at=at,
                               flags=genie.GENIE_SEARCH_PER_RANGE_AT | genie.GENIE_SEARCH_DENSE)
        res = runner.search(idx, qs, w.k, opts=opts).host()
        at = runner.u32(at).reshape(w.n_queries, groups)
        assert_same(res, oracle.topk(w))
        for g in range(groups):
            lo, hi = g << shift, min(w.n_objects, (g + 1) << shift)
            ref = oracle.topk(w, obj_range=(lo, hi))
            assert np.array_equal(at[:, g] - 1, ref["tk"]), g


def test_dense_with_seeds_batch_and_noalloc():
    """The seeded search (verify and rerun), the persistent batch and the
    no-alloc entry point all add bitmaps the same way."""
    w = synth.lsh(120_000, 64, 50, config=57)
    idx = runner.build_index(w, dense_min_df=1500)
    assert idx.info.dense_keywords > 0
    qs = runner.compile_queries(idx, w)
    ref = oracle.topk(w)
    seeds = np.maximum(1, ref["tk"].astype(np.int64) - np.arange(w.n_queries) % 3)
    seeds[::7] += 5  # some seeds above the k-th count: those queries rerun
    st = torch.zeros(8, dtype=torch.int64, device="cuda")
    res = runner.search(idx, qs, 50, opts=genie.make_opts(
        d_seed=runner.to_dev(seeds.astype(np.uint32)), d_stats=st,
        flags=genie.GENIE_SEARCH_DENSE)).host()
    torch.cuda.synchronize()
    assert_same(res, ref)
    assert int(st[3].item()) > 0
    batch = genie.Batch(idx, w.n_queries, qs.max_bound, 50, None)
    out = runner.Outputs(w.n_queries, 50)
    batch.run(qs, out.ids, out.counts, out.n_valid)
    torch.cuda.synchronize()
    assert_same(out.host(), ref)
    out2 = runner.Outputs(w.n_queries, 50)
    genie.genie_search_noalloc(idx, qs, 50, out2.ids, out2.counts, out2.n_valid)
    torch.cuda.synchronize()
    assert_same(out2.host(), ref)


def test_dense_instantiation_chosen_for_zipf_sets_in_search_and_batch():
    """Where dense keywords carry most of a batch's postings (Zipf sets), the
    search and the persistent batch both add their bitmaps (the dense
    instantiation and graph), and the results stay the oracle's."""
    w = synth.sets(150_000, (16, 200), 1 << 12, 64, (8, 300), 10, config=58)
    idx = runner.build_index(w)
    qs = runner.compile_queries(idx, w)
    qi = genie.QueriesInfo()
    genie.load().genie_queries_get_info(qs.handle, genie.ctypes.byref(qi))
    assert 2 * qi.n_dense_entries >= qi.n_entries > 0
    assert genie.genie_search_shape(idx, qs, 10).dense == 1
    ref = oracle.topk(w)
    st = torch.zeros(8, dtype=torch.int64, device="cuda")
    assert_same(runner.search(idx, qs, 10, opts=genie.make_opts(d_stats=st)).host(), ref)
    assert int(st[7].item()) > 0
    batch = genie.Batch(idx, w.n_queries, qs.max_bound, 10, None)
    out = runner.Outputs(w.n_queries, 10)
    for _ in range(2):  # a replayed graph starts from a clean state
        batch.run(qs, out.ids, out.counts, out.n_valid)
        torch.cuda.synchronize()
        assert_same(out.host(), ref)
