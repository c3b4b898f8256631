"""Multiple loadings (GPU): an index split into parts by object id, held in
pinned host memory and searched part by part (Sec. 3.4), returns exactly the
oracle's top-k of the whole object set; the part store checks its inputs."""
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


def _check(res, ref):
    for q in range(len(ref["n_valid"])):
        n = int(ref["n_valid"][q])
        assert res["n_valid"][q] == n, q
        assert np.array_equal(res["ids"][q, :n], ref["ids"][q, :n]), q
        assert np.array_equal(res["counts"][q, :n], ref["counts"][q, :n]), q
        assert np.all(res["ids"][q, n:] == 0xFFFFFFFF)
        assert np.all(res["counts"][q, n:] == 0)


def test_uneven_parts_equal_one_index_and_the_oracle():
    w = synth.sets(150_000, (16, 128), 1 << 16, 120, (8, 300), 10, config=50)
    ranges = [(0, 61_000), (61_000, 118_500), (118_500, 150_000)]
    parts = runner.build_parts(w, ranges, chunk_shift=13)
    info = parts.info
    assert info.n_parts == 3 and info.n_objects == w.n_objects and info.vocab == w.vocab
    got = runner.search_parts(parts, w, 10).host()
    torch.cuda.synchronize()
    _check(got, oracle.topk(w))
    idx = runner.build_index(w, 13)
    whole = runner.search(idx, runner.compile_queries(idx, w), 10).host()
    for key in got:
        assert np.array_equal(got[key], whole[key]), key
    # a second search reuses the device slots
    again = runner.search_parts(parts, w, 10).host()
    for key in got:
        assert np.array_equal(got[key], again[key]), key
    parts.close()


def test_parts_with_an_id_gap_and_per_query_k():
    w = synth.lsh(60_000, 40, 30, config=51)
    rng = np.random.default_rng(3)
    ks = rng.integers(1, 31, w.n_queries).astype(np.uint32)
    # objects 20_000 .. 24_999 hold no keyword: they belong to no part
    off = w.obj_off.astype(np.int64)
    lens = np.diff(off)
    lens[20_000:25_000] = 0
    keep = np.ones(len(w.obj_kw), dtype=bool)
    keep[off[20_000]:off[25_000]] = False
    w.obj_kw = w.obj_kw[keep]
    w.obj_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint32)
    parts = runner.build_parts(w, [(0, 20_000), (25_000, 60_000)], chunk_shift=12)
    got = runner.search_parts(parts, w, ks).host()
    torch.cuda.synchronize()
    _check(got, oracle.topk(w, k=ks))
    parts.close()


def test_part_store_inputs_are_checked():
    w = synth.sets(10_000, (4, 16), 500, 8, (2, 10), 5, config=52)
    off = w.obj_off.astype(np.int64)
    parts = genie.Parts()
    with pytest.raises(genie.GenieError) as e:   # no part yet
        runner.search_parts(parts, w, 5)
    assert e.value.status == genie.GENIE_ERR_INVALID_ARG
    a = genie.genie_build_index(runner.to_dev(w.obj_off), runner.to_dev(w.obj_kw), w.n_objects,
                                w.vocab, 0, None)
    parts.add(a, 0)
    with pytest.raises(genie.GenieError) as e:   # overlapping id range
        parts.add(a, w.n_objects - 1)
    assert e.value.status == genie.GENIE_ERR_INVALID_ARG
    b = genie.genie_build_index(runner.to_dev(w.obj_off), runner.to_dev(w.obj_kw), w.n_objects,
                                w.vocab + 7, 0, None)
    with pytest.raises(genie.GenieError) as e:   # another vocabulary
        parts.add(b, w.n_objects)
    assert e.value.status == genie.GENIE_ERR_INVALID_ARG
    with pytest.raises(genie.GenieError) as e:   # ids past 2^32 - 2
        parts.add(a, 0xFFFFFFFF - 5)
    assert e.value.status == genie.GENIE_ERR_INVALID_ARG
    got = runner.search_parts(parts, w, 5).host()   # the one valid part
    torch.cuda.synchronize()
    _check(got, oracle.topk(w))
    for x in (a, b, parts):
        x.close()
    del off


@pytest.mark.parametrize("chunk_shift", [12, 16, 17])
def test_parts_carry_16_bit_places_or_full_ids(chunk_shift):
    """With object ranges of at most 2^16 ids a part keeps each id's place in
    its range (16 bits) in host memory and the device rebuilds the ids from
    the sublist map; wider ranges keep the full ids.  Both equal the oracle.
    At 2^12 ids per range the middle part spans 37 ranges, more than one
    warp-wide read of a keyword's row of the sublist map."""
    w = synth.sets(300_000, (16, 64), 1 << 16, 40, (8, 100), 10, config=53)
    ranges = [(0, 100_000), (100_000, 250_001), (250_001, 300_000)]
    parts = runner.build_parts(w, ranges, chunk_shift=chunk_shift)
    got = runner.search_parts(parts, w, 10).host()
    torch.cuda.synchronize()
    _check(got, oracle.topk(w))
    again = runner.search_parts(parts, w, 10).host()   # the staging buffers are reused
    for key in got:
        assert np.array_equal(got[key], again[key]), key
    nnz = int(w.obj_off[-1])
    pad = sum(((int(w.obj_off[b]) - int(w.obj_off[a]) + 3) & ~3) + 4 for a, b in ranges)
    other = parts.info.host_bytes - (pad - nnz) * (2 if chunk_shift <= 16 else 4)
    post = nnz * (2 if chunk_shift <= 16 else 4)
    # kw_off and the sublist map are the rest of the pinned bytes
    n_ch = sum(-(-(b - a) >> chunk_shift) + 1 for a, b in ranges)
    assert other - post == 3 * (w.vocab + 1) * 8 + w.vocab * n_ch * 4
    parts.close()


@pytest.mark.parametrize("n_parts", [2, 4])
def test_parts_kept_in_their_slots_between_calls(n_parts):
    """Parts still in a device slot are not copied again, and with an even
    number of parts the last part's search overlaps the copy of part 0 for
    the next call.  Three calls in a row (k = 10, per-query k, k = 1), then a
    part larger than the others appended (the slots grow and are refilled)
    and two more calls: all equal the oracle."""
    w = synth.lsh(80_000, 40, 30, config=54)
    N, half = w.n_objects, w.n_objects // 2
    cuts = [i * half // n_parts for i in range(n_parts + 1)]
    parts = runner.build_parts(w, list(zip(cuts[:-1], cuts[1:])))
    ks = np.random.default_rng(5).integers(1, 31, w.n_queries).astype(np.uint32)
    for k in (10, ks, 1):
        got = runner.search_parts(parts, w, k).host()
        torch.cuda.synchronize()
        _check(got, oracle.topk(w, k=k, obj_range=(0, half)))
    off = w.obj_off.astype(np.int64)
    sub_off = (off[half:] - off[half]).astype(np.uint32)
    idx = genie.genie_build_index(runner.to_dev(sub_off), runner.to_dev(w.obj_kw[off[half]:]),
                                  N - half, w.vocab, 0, None)
    parts.add(idx, half)
    idx.close()
    for _ in range(2):
        got = runner.search_parts(parts, w, 10).host()
        torch.cuda.synchronize()
        _check(got, oracle.topk(w, k=10))
    parts.close()
