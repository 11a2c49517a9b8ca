"""GPU index build against the oracle, bit for bit: the clustered graph
construction (and, through the workload generator's independent build, the
graphs the other GPU tests search)."""
import numpy as np
import pytest

import oracle
import workload
from tests import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_11324_gb300 as bang  # noqa: E402


def _random_clusters(rng, dt, n, d, ng, hi):
    if dt == "f32":
        X = rng.normal(size=(n, d)).astype(np.float32)
    elif dt == "i8":
        X = rng.integers(-hi, hi, size=(n, d)).astype(np.int8)
    else:
        X = rng.integers(0, hi, size=(n, d)).astype(np.uint8)
    lab = rng.integers(0, ng, size=n)
    members = np.argsort(lab, kind="stable").astype(np.uint32)
    gstart = np.concatenate([[0], np.cumsum(np.bincount(lab, minlength=ng))]).astype(np.uint64)
    medoids = np.array([members[gstart[g] + (gstart[g + 1] - gstart[g]) // 2] for g in range(ng)],
                       np.uint32)
    return X, members, gstart, medoids


@pytest.mark.parametrize("dt,alpha,hi,d,R,nx,nh", [
    ("u8", 1.0, 6, 8, 12, 2, 3),          # small integers: distance ties decide
    ("u8", 1.2, 256, 128, 24, 4, 5),
    ("i8", 1.2, 128, 100, 20, 3, 2),      # rows of 100 bytes, padded on the device
    ("f32", 1.2, 0, 96, 16, 2, 2),
    ("f32", 1.0, 0, 7, 10, 0, 0),         # odd dimension, no medoid links
])
def test_cluster_graph_bit_exact(dt, alpha, hi, d, R, nx, nh):
    rng = np.random.default_rng(hash((dt, alpha, d)) % 2 ** 32)
    ng, n = 5, 900
    X, members, gstart, medoids = _random_clusters(rng, dt, n, d, ng, hi)
    xclu = rng.integers(0, ng + 1, size=(n, nx)).astype(np.uint32)    # includes out-of-range ids
    hclu = rng.integers(0, ng, size=(ng, nh)).astype(np.uint32)
    ref = oracle.cluster_graph(X, members, gstart, medoids, R, alpha, nx, xclu, nh, hclu)
    got = bang.bang_build_cluster_graph(X, members, gstart, medoids, R, alpha, nx, xclu, nh, hclu)
    assert (got == ref).all(), np.argwhere(got != ref)[:5]


def test_cluster_graph_tiny_and_device_buffers():
    rng = np.random.default_rng(41)
    X, members, gstart, medoids = _random_clusters(rng, "u8", 60, 16, 7, 256)
    gstart = np.array([0, 1, 2, 4, 20, 21, 40, 60], np.uint64)    # clusters of 1, 1, 2, 16, 1, 19, 20
    members = np.arange(60, dtype=np.uint32)
    medoids = np.array([0, 1, 2, 4, 20, 21, 40], np.uint32)
    ref = oracle.cluster_graph(X, members, gstart, medoids, 8, 1.2, 1, np.zeros((60, 1), np.uint32),
                               2, np.ones((7, 2), np.uint32))
    Xd = torch.from_numpy(X).cuda()
    adj = torch.zeros((60, 8), dtype=torch.int32, device="cuda")
    bang.bang_build_cluster_graph(Xd, members, gstart, medoids, 8, 1.2, 1,
                                  np.zeros((60, 1), np.uint32), 2, np.ones((7, 2), np.uint32), adj=adj)
    torch.cuda.synchronize()
    assert (adj.cpu().numpy().view(np.uint32) == ref).all()


def test_reproduces_the_generated_workload_graph():
    # the clustered workload the parity tests search, rebuilt on the GPU from
    # the same inputs, equals the generator's graph
    w = cases.clustered(n=20_000, nq=10, ncomp=8)
    c = workload.CONFIGS[2]
    gi = workload.graph_inputs(2, w["base"], w["labels"], 8, c["nx"], c["nh"])
    got = bang.bang_build_cluster_graph(w["base"], gi["members"], gi["gstart"], gi["medoids"],
                                        w["adj"].shape[1], c["alpha"], c["nx"], gi["xclu"],
                                        gi["hclu"].shape[1], gi["hclu"])
    assert (got == w["adj"]).all()


def test_rejects_inconsistent_inputs():
    X = np.zeros((10, 4), np.uint8)
    members = np.arange(10, dtype=np.uint32)
    ok = dict(members=members, gstart=[0, 10], medoids=[0], R=4, alpha=1.2)
    for bad in (dict(members=np.r_[members[:-1], 3].astype(np.uint32)),     # not a permutation
                dict(gstart=[0, 9]), dict(medoids=[10]), dict(R=129), dict(alpha=0.0)):
        kw = dict(ok, **bad)
        with pytest.raises(bang.BangError):
            bang.bang_build_cluster_graph(X, **kw)


@pytest.mark.parametrize("dt,d,M", [("u8", 32, 8), ("i8", 100, 30), ("f32", 96, 48), ("f32", 20, 3)])
def test_pq_build_bit_exact(dt, d, M):
    rng = np.random.default_rng(d * 7 + M)
    n = 3000
    if dt == "f32":
        X = (rng.normal(size=(n, d)) * 3).astype(np.float32)
    elif dt == "i8":
        X = rng.integers(-128, 128, size=(n, d)).astype(np.int8)
    else:
        X = rng.integers(0, 256, size=(n, d)).astype(np.uint8)
    sample = np.sort(rng.choice(n, size=1500, replace=False)).astype(np.uint64)
    init = np.stack([rng.choice(n, size=256, replace=False) for _ in range(M)]).astype(np.uint64)
    cb_ref = oracle.pq_train(X.astype(np.float32), M, sample, init, 4)
    codes_ref = oracle.pq_encode(X, M, cb_ref)
    cb, codes = bang.bang_build_pq(X, M, sample, init, 4)
    assert (cb.view(np.uint32) == cb_ref.view(np.uint32)).all()
    assert (codes == codes_ref).all()


def test_pq_build_rejects_bad_ids():
    X = np.zeros((300, 8), np.uint8)
    init = np.zeros((2, 256), np.uint64)
    with pytest.raises(bang.BangError):
        bang.bang_build_pq(X, 2, np.array([0, 300], np.uint64), init)
    with pytest.raises(bang.BangError):
        bang.bang_build_pq(X, 2, np.array([0, 1], np.uint64), init + 300)
    with pytest.raises(bang.BangError):
        bang.bang_build_pq(np.zeros((300, 40), np.uint8), 2, np.array([0], np.uint64), init)   # 20-wide


@pytest.mark.parametrize("dt,n,d,k,nq", [
    ("u8", 20_000, 128, 10, 50),           # rows held in registers
    ("i8", 20_000, 100, 100, 30),          # 32-bit words, int8 offset
    ("i8", 5_000, 99, 7, 20),              # bytes
    ("f32", 20_000, 96, 10, 40),           # FP64 in the oracle's order
    ("u8", 300_000, 32, 16, 20),           # more points than the threshold sample
    ("u8", 5, 16, 10, 4),                  # fewer points than k: padding
])
def test_ground_truth_bit_exact(dt, n, d, k, nq):
    rng = np.random.default_rng(n + d + k)
    if dt == "f32":
        X = rng.normal(size=(n, d)).astype(np.float32)
        Q = rng.normal(size=(nq, d)).astype(np.float32)
    elif dt == "i8":
        X = rng.integers(-128, 128, size=(n, d)).astype(np.int8)
        Q = rng.integers(-128, 128, size=(nq, d)).astype(np.int8)
    else:
        X = rng.integers(0, 8, size=(n, d)).astype(np.uint8)          # many distance ties
        Q = rng.integers(0, 8, size=(nq, d)).astype(np.uint8)
    ids_o, dist_o = oracle.bruteforce_knn(X, Q, k)
    ids, dist = bang.bang_ground_truth(X, Q, k)
    assert (ids == ids_o).all(), np.argwhere(ids != ids_o)[:5]
    fin = np.isfinite(dist_o)
    assert (np.isfinite(dist) == fin).all() and (dist[fin] == dist_o[fin]).all()
