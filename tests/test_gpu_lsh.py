"""LSH keywords on the GPU (Sec. 4.1): p-stable hashing and random binning
give the oracle's keywords bit for bit, and searching them gives the oracle's
top-k."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import lsh
from paper_1603_08390_gb300 import _build, genie, runner

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    genie.load()


def _pts(n, dim, config, scale=1.0):
    if dim == 128:
        _, v, _ = synth.lsh_keywords(n, config, 1, n_hash=1, want_vectors=True)
        return v
    rng = np.random.default_rng(config)
    return (rng.standard_normal((n, dim)) * scale).astype(np.float32)


def _gpu_pstable(pts, pp, D):
    n, dim = pts.shape
    m = pp["a"].shape[0]
    kw = torch.empty(n * m, dtype=torch.int32, device="cuda")
    genie.genie_lsh_pstable(torch.from_numpy(pts).cuda(), n, dim, torch.from_numpy(pp["a"]).cuda(),
                            torch.from_numpy(pp["b"]).cuda(), m, float(pp["w"]), D, kw)
    return kw


@pytest.mark.parametrize("n,dim,m", [(20_000, 128, 256), (3_001, 100, 70)])
def test_pstable_keywords_equal_the_oracle(n, dim, m):
    pts = _pts(n, dim, 21, scale=3.0)
    pp = synth.lsh_params("pstable", dim, m, 4.0, config=21)
    got = runner.u32(_gpu_pstable(pts, pp, 8192)).reshape(n, m)
    torch.cuda.synchronize()
    assert np.array_equal(got, lsh.pstable(pts, pp["a"], pp["b"], 4.0, 8192))


@pytest.mark.parametrize("n,dim,m,sigma", [(5_000, 32, 64, 10.0), (1_500, 1156, 40, 400.0)])
def test_rbh_keywords_equal_the_oracle(n, dim, m, sigma):
    rng = np.random.default_rng(22)
    pts = (rng.random((n, dim)) * 100).astype(np.float32)
    rp = synth.lsh_params("rbh", dim, m, sigma, config=22)
    kw = torch.empty(n * m, dtype=torch.int32, device="cuda")
    genie.genie_lsh_rbh(torch.from_numpy(pts).cuda(), n, dim, torch.from_numpy(rp["g"]).cuda(),
                        torch.from_numpy(rp["u"]).cuda(), runner.to_dev(rp["key"]), m, 8192, kw)
    got = runner.u32(kw).reshape(n, m)
    torch.cuda.synchronize()
    assert np.array_equal(got, lsh.rbh(pts, rp["g"], rp["u"], rp["key"], 8192))


def test_keywords_from_the_gpu_search_like_the_oracle():
    n, q, m, D = 60_000, 32, 128, 8192
    _, pts, _ = synth.lsh_keywords(n, 23, 1, n_hash=1, want_vectors=True)
    _, qpts, _ = synth.lsh_keywords(q, 23, 2, n_hash=1, want_vectors=True)
    pp = synth.lsh_params("pstable", 128, m, 4.0, config=23)
    d_kw = _gpu_pstable(pts, pp, D)
    d_qkw = _gpu_pstable(qpts, pp, D)
    off = (np.arange(n + 1, dtype=np.uint64) * m).astype(np.uint32)
    qoff = (np.arange(q + 1, dtype=np.uint64) * m).astype(np.uint32)
    idx = genie.genie_build_index(runner.to_dev(off), d_kw, n, m * D, 0, None)
    qs = genie.genie_make_queries(idx, runner.to_dev(qoff), d_qkw, q, None)
    got = runner.search(idx, qs, 20).host()
    torch.cuda.synchronize()
    w = synth.Workload("lsh", "keywords", n, m * D, off,
                       lsh.pstable(pts, pp["a"], pp["b"], 4.0, D).ravel(), q, 20, q_off=qoff,
                       q_kw=lsh.pstable(qpts, pp["a"], pp["b"], 4.0, D).ravel())
    ref = oracle.topk(w)
    for key in ("ids", "counts", "n_valid"):
        assert np.array_equal(got[key], ref[key]), key


def test_lsh_inputs_are_checked():
    x = torch.zeros(4, device="cuda")
    kw = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(genie.GenieError) as e:     # m * D > 2^32
        genie.genie_lsh_pstable(x, 1, 1, x, x, 2, 1.0, 1 << 31 | 1, kw)
    assert e.value.status == genie.GENIE_ERR_INVALID_ARG
    with pytest.raises(genie.GenieError) as e:     # w <= 0
        genie.genie_lsh_pstable(x, 1, 1, x, x, 1, 0.0, 8, kw)
    assert e.value.status == genie.GENIE_ERR_INVALID_ARG
