"""The synthetic workload generator (stand-in for the datasets and the
prebuilt index): valid graph, deterministic across thread counts, ground
truth and medoid equal to the oracle's independent brute force."""
import os
import subprocess
import sys

import numpy as np

import oracle
import workload

NONE = workload.NONE


def _small(tmp_path, monkeypatch):
    monkeypatch.setenv("BANG_WORKLOAD_CACHE", str(tmp_path))
    return workload.clustered_workload(2, n=6000, nq=50, ncomp=6, k=20)


def test_graph_is_valid_and_navigable(tmp_path, monkeypatch):
    w = _small(tmp_path, monkeypatch)
    adj, n = w["adj"], w["base"].shape[0]
    assert adj.shape == (n, 64)
    for i in range(0, n, 7):
        row = adj[i]
        ids = row[row != NONE]
        assert (row[len(ids):] == NONE).all()
        assert (ids < n).all() and i not in ids.tolist() and len(set(ids.tolist())) == len(ids)
    seen = np.zeros(n, bool)
    seen[w["medoid"]] = True
    fr = np.array([w["medoid"]])
    while len(fr):
        nb = adj[fr].ravel()
        nb = np.unique(nb[nb != NONE])
        nb = nb[~seen[nb]]
        seen[nb] = True
        fr = nb
    assert seen.mean() > 0.99


def test_ground_truth_and_medoid_match_oracle(tmp_path, monkeypatch):
    w = _small(tmp_path, monkeypatch)
    ids, dist = oracle.bruteforce_knn(w["base"], w["queries"], 20)
    assert (ids == w["gt_ids"]).all() and (dist == w["gt_dist"]).all()
    assert oracle.medoid(w["base"]) == w["medoid"]


def test_deterministic_across_thread_counts(tmp_path):
    code = ("import workload, hashlib, sys; "
            "w = workload.clustered_workload(2, n=3000, nq=10, ncomp=3, k=10); "
            "h = hashlib.sha1(); [h.update(w[f].tobytes()) for f in "
            "('base','queries','codebook','codes','adj','gt_ids')]; print(h.hexdigest())")
    out = []
    for th, sub in (("1", "a"), ("3", "b")):
        env = dict(os.environ, OMP_NUM_THREADS=th, BANG_WORKLOAD_CACHE=str(tmp_path / sub),
                   PYTHONPATH=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        out.append(subprocess.check_output([sys.executable, "-c", code], env=env, text=True))
    assert out[0] == out[1]


def test_mixed_cluster_links_of_configuration_4():
    # configuration 4's links between clusters: per point, half to clusters
    # among its cluster's nearest (by medoid distance) and half to random
    # other clusters; per medoid, its nh/2 nearest and nh/2 distinct random
    # ones; never its own cluster
    ng, nx, nh = 64, 4, 32
    w = workload.make_data(4, n=20_000, nq=4, ncomp=ng)
    gi = workload.graph_inputs(4, w["base"], w["labels"], ng, nx, nh)
    own = w["labels"].astype(np.int64)
    xclu, hclu, meds = gi["xclu"].astype(np.int64), gi["hclu"].astype(np.int64), gi["medoids"]
    assert xclu.shape == (20_000, nx) and hclu.shape == (ng, nh)
    assert (xclu != own[:, None]).all() and (xclu < ng).all()
    mv = w["base"][meds.astype(np.int64)].astype(np.int64)
    dm = ((mv[:, None, :] - mv[None, :, :]) ** 2).sum(-1)        # exact integers
    np.fill_diagonal(dm, np.iinfo(np.int64).max)
    near = np.argsort(dm, axis=1, kind="stable")
    for c in range(ng):
        assert c not in hclu[c] and len(set(hclu[c].tolist())) == nh
        assert (hclu[c, :nh // 2] == near[c, :nh // 2]).all()
    for p in range(0, 20_000, 97):
        assert set(xclu[p, :nx // 2].tolist()) <= set(near[own[p], :nx].tolist())
    # deterministic: the same inputs twice
    gi2 = workload.graph_inputs(4, w["base"], w["labels"], ng, nx, nh)
    assert (gi2["xclu"] == gi["xclu"]).all() and (gi2["hclu"] == gi["hclu"]).all()


def test_large_data_same_bytes_in_huge_page_memory():
    # the benchmark allocates configuration 5's base vectors with
    # bang_host_alloc (no GPU needed); the generated bytes do not depend on
    # where they are written
    import paper_2401_11324_gb300 as bang
    a = workload.large_data(5, n=20_000, nq=50, ncomp=64)
    b = workload.large_data(5, n=20_000, nq=50, ncomp=64, alloc=bang.host_empty)
    assert (a["base"] == b["base"]).all() and (a["queries"] == b["queries"]).all()
    assert b["base"].ctypes.data % (2 << 20) == 0
    assert a["medoid"] == b["medoid"]
