"""Sequence search by ordered n-grams (GPU, Sec. 5.1): the n-gram keywords are
the oracle's bit for bit, and the whole shotgun-and-assembly pipeline (n-grams,
top-K by match count, the verification of Algorithm 2, the certificate of
Theorem 5.2) returns what the oracle pipeline returns."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import sa
from paper_1603_08390_gb300 import _build, genie, runner

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    genie.load()


@pytest.mark.parametrize("n,sigma,R", [(2, 4, 64), (3, 26, 16), (4, 5, 32)])
def test_grams_equal_the_oracle(n, sigma, R):
    seqs = synth.sequences(20_000, (0, 120), sigma, 8, (1, 3), config=80 + n)
    d_kw_off, d_kw, total = runner.sa_grams(runner.to_dev(seqs.s_off), runner.to_dev(seqs.s_chars),
                                            seqs.s_off, n, sigma, R)
    torch.cuda.synchronize()
    ref_off, ref_kw = sa.grams(seqs.s_off, seqs.s_chars, n, sigma, R)
    assert total == len(ref_kw)
    assert np.array_equal(runner.u32(d_kw_off), ref_off)
    assert np.array_equal(runner.u32(d_kw)[:total], ref_kw)


def test_grams_reject_bad_input():
    off = np.array([0, 6, 9], np.uint32)
    chars = np.array([0, 0, 0, 0, 0, 1, 2, 1, 5], np.uint8)
    d_off, d_chars = runner.to_dev(off), runner.to_dev(chars)
    with pytest.raises(genie.GenieError) as e:      # character 5 >= sigma 4
        runner.sa_grams(d_off, d_chars, off, 2, 4, 8)
    assert e.value.status == genie.GENIE_ERR_INVALID_ARG
    ok = np.array([0, 0, 0, 0, 0, 1, 2, 1, 3], np.uint8)
    with pytest.raises(genie.GenieError) as e:      # 'aa' occurs 4 times, R = 3
        runner.sa_grams(d_off, runner.to_dev(ok), off, 2, 4, 3)
    assert e.value.status == genie.GENIE_ERR_INVALID_ARG
    with pytest.raises(genie.GenieError) as e:      # sigma^n * R > 2^31
        runner.sa_grams(d_off, runner.to_dev(ok), off, 8, 256, 2)
    assert e.value.status == genie.GENIE_ERR_INVALID_ARG
    d_kw_off = torch.empty(3, dtype=torch.int32, device="cuda")
    d_kw = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(genie.GenieError) as e:      # 7 keywords, room for 4
        genie.genie_sa_grams(d_off, runner.to_dev(ok), 2, 2, 4, 8, d_kw_off, d_kw, 4)
    assert e.value.status == genie.GENIE_ERR_CAPACITY


def _oracle_pipeline(seqs, n, R, K, k):
    kw_off, kw = sa.grams(seqs.s_off, seqs.s_chars, n, seqs.sigma, R)
    q_kw_off, q_kw = sa.grams(seqs.q_off, seqs.q_chars, n, seqs.sigma, R)
    w = synth.Workload("seq", "keywords", seqs.n_seqs, seqs.sigma ** n * R, kw_off, kw,
                       seqs.n_queries, K, q_off=q_kw_off, q_kw=q_kw)
    top = oracle.topk(w)
    s_len = np.diff(seqs.s_off.astype(np.int64))
    q_len = np.diff(seqs.q_off.astype(np.int64))
    res = []
    for q in range(seqs.n_queries):
        m = int(top["n_valid"][q])
        ids = top["ids"][q, :m]
        pairs = np.stack([np.full(m, q, np.uint32), ids], 1)
        eds = sa.ed_pairs(seqs.q_off, seqs.q_chars, seqs.s_off, seqs.s_chars, pairs)
        res.append(sa.verify(int(q_len[q]), ids, top["counts"][q, :m], m, s_len[ids], eds, K, k,
                             n))
    return top, res


@pytest.mark.parametrize("length,k,R", [((20, 60), 1, 32), ((100, 500), 3, 256)])
def test_pipeline_equals_the_oracle_pipeline(length, k, R):
    n, K = 3, 64
    seqs = synth.sequences(30_000, length, 8, 48, (0, 6), config=90 + k)
    si = runner.SeqIndex(seqs.s_off, seqs.s_chars, n, seqs.sigma, R, chunk_shift=13)
    got = runner.sa_search(si, seqs.q_off, seqs.q_chars, K, k).host()
    torch.cuda.synchronize()
    top, ref = _oracle_pipeline(seqs, n, R, K, k)
    cand = got["candidates"]
    for key in ("ids", "counts", "n_valid"):
        assert np.array_equal(cand[key], top[key][:, :K] if key != "n_valid" else top[key]), key
    truth = sa.topk_ed(seqs.s_off, seqs.s_chars, seqs.q_off, seqs.q_chars, k)
    n_cert = 0
    for q in range(seqs.n_queries):
        r = ref[q]
        nb = len(r["ids"])
        assert got["n_out"][q] == nb
        assert list(got["ids"][q, :nb]) == r["ids"], q
        assert list(got["ed"][q, :nb]) == r["ed"], q
        assert np.all(got["ids"][q, nb:] == 0xFFFFFFFF)
        assert bool(got["certified"][q]) == r["certified"], q
        assert got["examined"][q] == r["examined"], q
        if r["certified"]:
            n_cert += 1
            assert list(got["ed"][q]) == list(truth["ed"][q])  # Theorem 5.2
    if k == 1:  # beyond the near-duplicate, random sequences are far: only k = 1 certifies
        assert n_cert > seqs.n_queries // 2
