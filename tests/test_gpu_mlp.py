"""GPU checks of the k-th-count network against the float64 reference
(oracle/mlp.py), and of the learned seeded search against the CPU oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import mlp as ref
from paper_1603_08390_gb300 import _build, genie, learned, runner

pytestmark = pytest.mark.gpu

N_PARAMS = 128 * 64 + 128 + 128 + 1


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    genie.load()


def _split(theta):
    W1 = theta[:8192].reshape(128, 64)
    return W1, theta[8192:8320], theta[8320:8448], float(theta[8448])


def _rounded(theta):
    W1, b1, w2, b2 = _split(theta.astype(np.float32))
    return ref.bf16_round(W1), b1, ref.bf16_round(w2), b2


def _net(seed):
    rng = np.random.default_rng(seed)
    theta = (rng.normal(0, 0.2, N_PARAMS)).astype(np.float32)
    m = genie.MLP(seed)
    assert m.n_params == N_PARAMS
    m.set_params(torch.from_numpy(theta).cuda())
    return m, theta, rng


def test_forward_matches_reference():
    m, theta, rng = _net(1)
    x = rng.normal(0, 1, (1000, 64)).astype(np.float32)
    y = torch.empty(1000, dtype=torch.float32, device="cuda")
    m.forward(torch.from_numpy(x).cuda(), 1000, y)
    got = y.cpu().numpy()
    want, _ = ref.forward(x, *_rounded(theta))
    assert np.allclose(got, want, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("n", [1, 37, 1000])
def test_gradients_match_reference(n):
    m, theta, rng = _net(2 + n)
    x = rng.normal(0, 1, (n, 64)).astype(np.float32)
    t = rng.normal(2, 3, n).astype(np.float32)
    g = torch.empty(N_PARAMS + 1, dtype=torch.float32, device="cuda")
    m.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), n, g)
    got = g.cpu().numpy()
    W1, b1, w2, b2 = _rounded(theta)
    y, cache = ref.forward(x, W1, b1, w2, b2)
    gW1, gb1, gw2, gb2 = ref.backward(y, t, cache, W1, w2)
    want = np.concatenate([gW1.ravel(), gb1, gw2, [gb2]])
    scale = np.abs(want).max()
    assert np.abs(got[:N_PARAMS] - want).max() <= 1e-4 * scale
    assert np.isclose(got[N_PARAMS], np.sum((y - t) ** 2), rtol=1e-4)


def test_adam_step_matches_reference():
    m, theta, rng = _net(5)
    x = rng.normal(0, 1, (200, 64)).astype(np.float32)
    t = rng.normal(1, 2, 200).astype(np.float32)
    g = torch.empty(N_PARAMS + 1, dtype=torch.float32, device="cuda")
    m.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), 200, g)
    m.adam_step(1e-2)
    out = torch.empty(N_PARAMS, dtype=torch.float32, device="cuda")
    m.get_params(out)
    grad = g.cpu().numpy()[:N_PARAMS].astype(np.float64)
    want, _, _ = ref.adam(theta.astype(np.float64), grad, np.zeros(N_PARAMS), np.zeros(N_PARAMS),
                          step=1, lr=1e-2)
    assert np.allclose(out.cpu().numpy(), want, rtol=1e-5, atol=1e-6)


def test_training_fits_a_teacher():
    rng = np.random.default_rng(9)
    x = np.abs(rng.normal(0, 1, (4096, 64))).astype(np.float32)
    w_true = rng.normal(0, 1, 64)
    t = (x @ w_true + 5.0).astype(np.float32)
    m = genie.MLP(3)
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    g = torch.empty(N_PARAMS + 1, dtype=torch.float32, device="cuda")
    m.gradients(dx, dt, 4096, g)
    loss0 = 0.5 * float(g[N_PARAMS].item()) / 4096
    loss = m.train(dx, dt, 4096, epochs=40, batch=256, lr=3e-3)
    assert loss < loss0 / 20
    theta = torch.empty(N_PARAMS, dtype=torch.float32, device="cuda")
    m.get_params(theta)
    y, _ = ref.forward(x, *_rounded(theta.cpu().numpy()))
    assert np.isclose(loss, ref.loss(y, t), rtol=1e-3)


def test_learned_seeds_keep_results_exact_and_cut_gate_work():
    w = synth.lsh(200_000, 128, 20, config=28)
    idx = runner.build_index(w)
    tq_off, tq_kw = synth.lsh_training_queries(3000, config=28)
    tr = learned.train_predictor(idx, tq_off, tq_kw, 20, epochs=40, batch=128, lr=2e-3)
    assert tr["margin"] >= 0
    qs = runner.compile_queries(idx, w)
    # seeds follow the stated rule from the network's own (float32) output
    feats = runner.query_facts(qs)
    y = torch.empty(w.n_queries, dtype=torch.float32, device="cuda")
    tr["mlp"].forward(torch.from_numpy(feats["features"]).cuda(), w.n_queries, y)
    seeds = torch.empty(w.n_queries, dtype=torch.int32, device="cuda")
    tr["mlp"].seeds(qs, tr["margin"], seeds)
    yv = y.cpu().numpy()
    p = yv - np.float32(tr["margin"])
    want = np.where(p >= 1, np.minimum(np.floor(p), feats["bound"] + 1), 1).astype(np.uint32)
    assert np.array_equal(runner.u32(seeds), want)
    # Against the search the library ships without the network (the default
    # plain search: each range seeds its AuditThreshold from the query's
    # finished ranges, and a query's first ranges count without the Gate):
    # identical results, equal to the oracle, and the seeds replace that
    # warm-up -- no range runs unseeded, and every range's AuditThreshold
    # starts at or above the seed, a lower bound of the k-th count.
    st_plain = torch.zeros(8, dtype=torch.int64, device="cuda")
    st_seed = torch.zeros(8, dtype=torch.int64, device="cuda")
    plain = runner.search(idx, qs, 20, opts=genie.make_opts(d_stats=st_plain)).host()
    seeded = learned.seeded_search(idx, qs, tr["mlp"], tr["margin"], 20, stats=st_seed).host()
    torch.cuda.synchronize()
    ref_res = oracle.topk(w)
    for res in (plain, seeded):
        for x in ("ids", "counts", "n_valid"):
            assert np.array_equal(res[x], plain[x])
        for q in range(w.n_queries):
            n = int(ref_res["n_valid"][q])
            assert res["n_valid"][q] == n
            assert np.array_equal(res["ids"][q, :n], ref_res["ids"][q, :n])
            assert np.array_equal(res["counts"][q, :n], ref_res["counts"][q, :n])
    sp, ss = st_plain.cpu().numpy(), st_seed.cpu().numpy()
    assert ss[3] <= 0.1 * w.n_queries  # reruns (mispredictions)
    assert sp[6] >= w.n_queries        # plain: each query's first range ran unseeded
    kth = ref_res["tk"].astype(np.int64)
    good = want.astype(np.int64) <= np.maximum(kth, 1)   # seeds that certify
    assert good.mean() >= 0.9
    assert ss[6] < sp[6]  # unseeded ranges: only queries seeded at 1 and the reruns keep some
    # the seeds sit close to the k-th count: they start each query's Gate
    # where the plain search gets only after its first ranges
    assert np.mean(want[good]) >= 0.6 * np.mean(kth[good])
