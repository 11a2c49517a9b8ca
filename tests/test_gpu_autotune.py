"""Autotuner (bang_autotune) on the GPU: the settings it returns reproduce the
recall it reports, satisfy its criterion, and come back from its cache."""
import numpy as np
import pytest

import oracle
from tests import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_11324_gb300 as bang  # noqa: E402


@pytest.fixture(scope="module")
def setup():
    w = cases.clustered(n=20_000, nq=300, ncomp=8)
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    q = torch.from_numpy(np.ascontiguousarray(w["queries"])).cuda()
    yield w, ix, q
    ix.close()


def _recall_with(ix, q, w, r, k=10):
    ids = torch.empty((q.shape[0], k), dtype=torch.int32, device="cuda")
    dist = torch.empty((q.shape[0], k), dtype=torch.float32, device="cuda")
    p = bang.make_params(bloom_log2=r["bloom_log2"], mode=r["mode"], table_source=r["table_source"])
    ix.search(q, k, r["L"], ids, dist, p)
    torch.cuda.synchronize()
    return oracle.recall_at_k(ids.cpu().numpy().view(np.uint32), w["gt_ids"], k)


def test_fixed_L_within_tolerance(setup):
    w, ix, q = setup
    truth = np.ascontiguousarray(w["gt_ids"][:, :10])
    r = ix.autotune(q, 10, 64, truth=truth, bloom_min=14, bloom_max=16)
    assert r["L"] == 64 and r["mode"] in (0, 1, 3) and 14 <= r["bloom_log2"] <= 16
    assert r["recall"] >= r["ref_recall"] - 0.005 - 1e-6
    assert r["candidates"] >= 9 and r["ms"] > 0 and r["ref_ms"] > 0
    assert abs(_recall_with(ix, q, w, r) - r["recall"]) < 1e-6


def test_target_recall_picks_smallest_sufficient_L(setup):
    w, ix, q = setup
    truth = np.ascontiguousarray(w["gt_ids"][:, :10])
    r = ix.autotune(q, 10, 0, truth=truth, target_recall=0.8, modes=(1 << 3), bloom_min=15,
                    bloom_max=15)
    assert r["mode"] == 3 and r["bloom_log2"] == 15 and r["recall"] >= 0.8
    assert abs(_recall_with(ix, q, w, r) - r["recall"]) < 1e-6
    sweep = [16, 24, 32, 48, 64, 96, 128, 160, 192, 256, 320, 384, 512, 768, 1024]
    i = sweep.index(r["L"])
    if i > 0:                                   # the next smaller worklist misses the target
        smaller = dict(r, L=sweep[i - 1])
        assert _recall_with(ix, q, w, smaller) < 0.8


def test_without_truth_and_cache(setup, tmp_path):
    w, ix, q = setup
    path = str(tmp_path / "tune.jsonl")
    r1 = ix.autotune(q, 10, 48, bloom_min=15, bloom_max=16, cache_path=path)
    assert r1["from_cache"] == 0
    r2 = ix.autotune(q, 10, 48, bloom_min=15, bloom_max=16, cache_path=path)
    assert r2["from_cache"] == 1
    for f in ("mode", "bloom_log2", "table_source", "grid_mult", "L", "candidates"):
        assert r1[f] == r2[f]
    assert abs(r1["ms"] - r2["ms"]) <= 1e-4 * r1["ms"]
    assert open(path).read().count("\n") == 1


def test_batched_grid(setup):
    w, ix, q = setup
    truth = np.ascontiguousarray(w["gt_ids"][:, :10])
    r = ix.autotune(q, 10, 64, truth=truth, batched=1, modes=(1 << 1), bloom_min=16, bloom_max=16,
                    try_tensor_tables=0)
    assert r["grid_mult"] in (1, 2, 4) and r["mode"] == 1


def test_packed_rows_as_a_candidate(setup):
    w, ix, q = setup
    truth = np.ascontiguousarray(w["gt_ids"][:, :10])
    r = ix.autotune(q, 10, 64, truth=truth, modes=(1 << 3), bloom_min=15, bloom_max=15,
                    try_packed_graph=1)
    assert r["graph_packed"] in (0, 1) and r["candidates"] == 2
    # the index's own placement is back: unpacked results as before
    assert abs(_recall_with(ix, q, w, r) - r["recall"]) < 1e-6


def test_node_records_timed_on_the_winner(setup):
    w, ix, q = setup
    truth = np.ascontiguousarray(w["gt_ids"][:, :10])
    r = ix.autotune(q, 10, 64, truth=truth, modes=(1 << 3), bloom_min=15, bloom_max=15,
                    try_packed_graph=1, try_node_records=1)
    # two layouts, then the winner once more with its rows and vectors as records
    assert r["node_records"] in (0, 1) and r["candidates"] == 3
    assert abs(_recall_with(ix, q, w, r) - r["recall"]) < 1e-6
    flags = (bang.BANG_GRAPH_PACKED if r["graph_packed"] else 0) | (
        bang.BANG_NODE_RECORDS if r["node_records"] else 0)
    ix.set_placement(flags)
    try:
        assert abs(_recall_with(ix, q, w, r) - r["recall"]) < 1e-6
    finally:
        ix.set_placement(0)


def test_rejects_bad_options(setup):
    w, ix, q = setup
    for kw in (dict(target_recall=1.5), dict(bloom_min=17, bloom_max=14), dict(modes=1 << 7)):
        with pytest.raises(bang.BangError):
            ix.autotune(q, 10, 64, **kw)
    with pytest.raises(bang.BangError):
        ix.autotune(q, 10, 5)                    # L < k without a target recall


def test_structure_timed_on_the_winner(setup, tmp_path):
    # early code rows and the staged re-rank are timed on the winner; each
    # leaves the results unchanged, so the chosen settings reproduce the
    # reported recall with them set, and the cache returns them
    w, ix, q = setup
    truth = np.ascontiguousarray(w["gt_ids"][:, :10])
    path = str(tmp_path / "tune.jsonl")
    r = ix.autotune(q, 10, 64, truth=truth, bloom_min=15, bloom_max=16, try_structure=1, cache_path=path)
    assert r["early_codes"] in (0, 1) and r["rerank"] in (0, 1)
    assert r["candidates"] >= 8
    ids = torch.empty((q.shape[0], 10), dtype=torch.int32, device="cuda")
    dist = torch.empty((q.shape[0], 10), dtype=torch.float32, device="cuda")
    p = bang.make_params(bloom_log2=r["bloom_log2"], mode=r["mode"], table_source=r["table_source"],
                         early_codes=r["early_codes"], rerank=r["rerank"])
    ix.search(q, 10, r["L"], ids, dist, p)
    torch.cuda.synchronize()
    assert abs(oracle.recall_at_k(ids.cpu().numpy().view(np.uint32), w["gt_ids"], 10) - r["recall"]) < 1e-6
    r2 = ix.autotune(q, 10, 64, truth=truth, bloom_min=15, bloom_max=16, try_structure=1, cache_path=path)
    assert r2["from_cache"] == 1
    for f in ("mode", "bloom_log2", "L", "early_codes", "rerank"):
        assert r2[f] == r[f], f
