"""Pins of the sequence-search oracle (Sec. 5.1): ordered n-grams, edit
distance, the n-gram bound of Theorem 5.1, Lemma 5.1, and the verification
of Algorithm 2 with the certificate of Theorem 5.2 (CPU only)."""
import functools
import itertools
import json
import os
from collections import Counter

import numpy as np
import pytest

import oracle
import synth
from oracle import sa

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_example_ordered_3grams():
    ex = json.load(open(os.path.join(GOLDEN, "example_5_1.json")))
    got = sa.ordered_ngrams(ex["sequence"].encode(), ex["n"])
    want = [(tuple(g.encode()), i) for g, i in ex["expected"]]
    assert got == want


def test_keyword_encoding_matches_the_ordered_ngrams():
    rng = np.random.default_rng(0)
    for n, sigma in ((1, 2), (2, 3), (3, 4), (4, 5)):
        seqs = [rng.integers(0, sigma, rng.integers(0, 30)).astype(np.uint8) for _ in range(60)]
        off = np.concatenate([[0], np.cumsum([len(x) for x in seqs])]).astype(np.uint32)
        chars = np.concatenate(seqs).astype(np.uint8)
        kw_off, kw = sa.grams(off, chars, n, sigma, 64)
        for t, x in enumerate(seqs):
            want = []
            for g, i in sa.ordered_ngrams(list(x), n):
                v = 0
                for c in g:
                    v = v * sigma + int(c)
                want.append(v * 64 + i)
            assert list(kw[kw_off[t]:kw_off[t + 1]]) == want


def test_repeats_beyond_R_are_rejected():
    off = np.array([0, 5], np.uint32)
    chars = np.zeros(5, np.uint8)  # 'aaaaa': the 2-gram aa occurs 4 times
    sa.grams(off, chars, 2, 2, 4)
    with pytest.raises(ValueError):
        sa.grams(off, chars, 2, 2, 3)


@functools.lru_cache(maxsize=None)
def _ed_rec(a, b):
    """Levenshtein distance by its recursive definition (short strings)."""
    if not a:
        return len(b)
    if not b:
        return len(a)
    return min(_ed_rec(a[1:], b) + 1, _ed_rec(a, b[1:]) + 1,
               _ed_rec(a[1:], b[1:]) + (a[0] != b[0]))


def test_edit_distance_textbook_values():
    assert sa.ed(b"kitten", b"sitting") == 3
    assert sa.ed(b"flaw", b"lawn") == 2
    assert sa.ed(b"intention", b"execution") == 5
    assert sa.ed(b"", b"abc") == 3 and sa.ed(b"abc", b"") == 3 and sa.ed(b"", b"") == 0


def test_edit_distance_equals_the_recursive_definition_exhaustively():
    for la in range(0, 5):
        for lb in range(0, 5):
            for a in itertools.product(b"ab", repeat=la):
                for b in itertools.product(b"abc", repeat=lb):
                    assert sa.ed(bytes(a), bytes(b)) == _ed_rec(bytes(a), bytes(b))


def test_edit_distance_pairs_symmetry_and_triangle():
    rng = np.random.default_rng(1)
    seqs = [rng.integers(0, 4, rng.integers(0, 150)).astype(np.uint8) for _ in range(40)]
    off = np.concatenate([[0], np.cumsum([len(x) for x in seqs])]).astype(np.uint32)
    chars = np.concatenate(seqs).astype(np.uint8)
    pairs = np.array([(i, j) for i in range(40) for j in range(40)], np.uint32)
    d = sa.ed_pairs(off, chars, off, chars, pairs).reshape(40, 40).astype(np.int64)
    assert np.all(np.diag(d) == 0)
    assert np.array_equal(d, d.T)
    lens = np.array([len(x) for x in seqs])
    assert np.all(d >= np.abs(lens[:, None] - lens[None, :]))
    assert np.all(d <= np.maximum(lens[:, None], lens[None, :]))
    for i, j, k in rng.integers(0, 40, (300, 3)):
        assert d[i, k] <= d[i, j] + d[j, k]


def test_lemma_5_1_match_count_is_the_multiset_intersection():
    rng = np.random.default_rng(2)
    for _ in range(200):
        n = int(rng.integers(1, 4))
        a = rng.integers(0, 3, rng.integers(0, 25)).tolist()
        b = rng.integers(0, 3, rng.integers(0, 25)).tolist()
        ca = Counter(tuple(a[p:p + n]) for p in range(len(a) - n + 1))
        cb = Counter(tuple(b[p:p + n]) for p in range(len(b) - n + 1))
        assert sa.shared_ngrams(a, b, n) == sum((ca & cb).values())


def test_theorem_5_1_ngram_bound_holds():
    rng = np.random.default_rng(3)
    for _ in range(400):
        n = int(rng.integers(1, 5))
        a = rng.integers(0, 4, rng.integers(0, 40)).astype(np.uint8)
        b = a.copy().tolist()
        for _ in range(int(rng.integers(0, 6))):  # a few random edits
            op = rng.integers(0, 3)
            if op == 0 and b:
                b[int(rng.integers(0, len(b)))] = int(rng.integers(0, 4))
            elif op == 1:
                b.insert(int(rng.integers(0, len(b) + 1)), int(rng.integers(0, 4)))
            elif b:
                del b[int(rng.integers(0, len(b)))]
        tau = sa.ed(a, np.array(b, np.uint8))
        mc = sa.shared_ngrams(a.tolist(), b, n)
        assert mc >= max(len(a), len(b)) - n + 1 - tau * n


def _candidates(seqs, n, K):
    """Keyword workload of the sequences' ordered n-grams and its top-K."""
    kw_off, kw = sa.grams(seqs.s_off, seqs.s_chars, n, seqs.sigma, 64)
    q_kw_off, q_kw = sa.grams(seqs.q_off, seqs.q_chars, n, seqs.sigma, 64)
    w = synth.Workload("seq", "keywords", seqs.n_seqs, seqs.sigma ** n * 64, kw_off, kw,
                       seqs.n_queries, K, q_off=q_kw_off, q_kw=q_kw)
    return oracle.topk(w)


def test_theorem_5_2_certified_queries_have_the_true_topk():
    n, K = 3, 40
    seqs = synth.sequences(3000, (10, 40), 6, 60, (0, 4), config=70)
    top = _candidates(seqs, n, K)
    s_len = np.diff(seqs.s_off.astype(np.int64))
    q_len = np.diff(seqs.q_off.astype(np.int64))
    for k in (1, 3):
        truth = sa.topk_ed(seqs.s_off, seqs.s_chars, seqs.q_off, seqs.q_chars, k)
        n_cert = 0
        for q in range(seqs.n_queries):
            m = int(top["n_valid"][q])
            ids = top["ids"][q, :m]
            pairs = np.stack([np.full(m, q, np.uint32), ids], 1)
            eds = sa.ed_pairs(seqs.q_off, seqs.q_chars, seqs.s_off, seqs.s_chars, pairs)
            r = sa.verify(int(q_len[q]), ids, top["counts"][q, :m], m, s_len[ids], eds, K, k, n)
            # the k best among the candidates, ties by candidate order
            order = sorted(range(m), key=lambda j: (int(eds[j]), j))[:k]
            assert r["ed"] == [int(eds[j]) for j in order]
            if r["certified"]:
                n_cert += 1
                assert r["ed"] == list(truth["ed"][q])  # Theorem 5.2
        if k == 1:  # near-duplicate queries are mostly certified
            assert n_cert > seqs.n_queries // 2


def test_verification_breaks_on_the_filtering_bound():
    # three candidates in count order; after the first (ed 0) theta = |Q| - n + 1 + n
    q_len, n = 10, 2
    counts = np.array([9, 2, 1], np.uint32)
    r = sa.verify(q_len, np.array([5, 6, 7]), counts, 3, np.array([10, 10, 10]),
                  np.array([0, 3, 4]), 3, 1, n)
    assert r["ids"] == [5] and r["ed"] == [0] and r["examined"] == 1
