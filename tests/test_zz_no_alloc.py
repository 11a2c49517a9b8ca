"""The allocation-free batched search, checked against bang_search_batched.

bang_search_batched_noalloc exists for callers that cannot let the library
call cudaMalloc: a serving loop that must not stall on the device-wide
synchronisation an allocation can cause, work recorded under global stream
capture (where allocations are refused), or a framework that owns the whole
device-memory budget.  Its scratch lives in one file-scope device array that
all calls share, so this test makes two calls in a row with different
batches and checks both against the allocating entry point (FP32 form: the
same ids, distances and iteration counts).  The file sorts last so that a run
stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

from tests import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_11324_gb300 as bang  # noqa: E402


def _batch(w, n, seed):
    rng = np.random.default_rng(seed)
    sel = rng.choice(w["queries"].shape[0], n, replace=False)
    k = rng.choice([1, 10, 100], size=n).astype(np.uint32)
    L = np.maximum(rng.choice([32, 64, 128, 256], size=n), k).astype(np.uint32)
    return np.ascontiguousarray(w["queries"][sel]), k, L


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a if dtype is None else a.view(dtype)))
    return t.cuda()


def test_noalloc_matches_allocating_batched_search_twice():
    w = cases.clustered(n=20_000, nq=300, ncomp=8)
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    s = torch.cuda.Stream()
    for seed, n in ((1, 200), (2, 77)):
        Q, k, L = _batch(w, n, seed)
        kmax, Lmax = int(k.max()), int(L.max())
        q, kd, Ld = _dev(Q), _dev(k, np.int32), _dev(L, np.int32)
        out = {}
        for name, fn in (("ref", bang.bang_search_batched), ("noalloc", bang.bang_search_batched_noalloc)):
            ids = torch.full((n, kmax), -7, dtype=torch.int32, device="cuda")
            dist = torch.full((n, kmax), -7.0, dtype=torch.float32, device="cuda")
            iters = torch.zeros(n, dtype=torch.int32, device="cuda")
            status = torch.full((n,), 9, dtype=torch.int32, device="cuda")
            p = bang.make_params(out_iters=iters, out_status=status)
            fn(ix.h, q, n, kd, Ld, kmax, Lmax, p, ids, dist, stream=s.cuda_stream)
            s.synchronize()
            out[name] = [t.cpu().numpy() for t in (ids, dist, iters, status)]
        r, z = out["ref"], out["noalloc"]
        assert (z[0] == r[0]).all()
        fin = np.isfinite(r[1])
        assert (np.isfinite(z[1]) == fin).all()
        np.testing.assert_allclose(z[1][fin], r[1][fin], rtol=1e-5, atol=0)
        assert (z[2] == r[2]).all() and (z[3] == r[3]).all() and (z[3] == 0).all()
    ix.close()


def _run(fn, ix, q, kd, Ld, n, kmax, Lmax, s):
    ids = torch.full((n, kmax), -7, dtype=torch.int32, device="cuda")
    dist = torch.full((n, kmax), -7.0, dtype=torch.float32, device="cuda")
    iters = torch.zeros(n, dtype=torch.int32, device="cuda")
    status = torch.full((n,), 9, dtype=torch.int32, device="cuda")
    p = bang.make_params(out_iters=iters, out_status=status)
    fn(ix.h, q, n, kd, Ld, kmax, Lmax, p, ids, dist, stream=s.cuda_stream)
    s.synchronize()
    return [t.cpu().numpy() for t in (ids, dist, iters, status)]


def test_noalloc_large_batch_with_out_of_range_rows():
    """A batch of 3,000 queries (more than the order kernel's 1,024 threads,
    so its strided loops run) in which some rows have L = 0, L > L_max or
    k > k_max: those rows are padded with status -1, and every other row
    equals bang_search_batched's."""
    w = cases.clustered(n=20_000, nq=300, ncomp=8)
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    s = torch.cuda.Stream()
    n, kmax, Lmax = 3000, 16, 64
    rng = np.random.default_rng(11)
    Q = np.ascontiguousarray(w["queries"][rng.integers(0, w["queries"].shape[0], n)])
    k = rng.choice([1, 5, 10, 16], size=n).astype(np.uint32)
    L = np.maximum(rng.choice([16, 32, 48, 64], size=n), k).astype(np.uint32)
    bad = rng.choice(n, 60, replace=False)
    L[bad[:20]] = 0                  # out of range: bucket 0 of the order
    L[bad[20:40]] = Lmax + 1 + rng.integers(0, 500, 20)
    k[bad[40:]] = kmax + 1
    q, kd, Ld = _dev(Q), _dev(k, np.int32), _dev(L, np.int32)
    r = _run(bang.bang_search_batched, ix, q, kd, Ld, n, kmax, Lmax, s)
    z = _run(bang.bang_search_batched_noalloc, ix, q, kd, Ld, n, kmax, Lmax, s)
    assert (z[3][bad] == -1).all() and (z[0][bad] == -1).all() and np.isinf(z[1][bad]).all()
    assert (z[2][bad] == 0).all()
    good = np.setdiff1d(np.arange(n), bad)
    assert (z[3][good] == 0).all()
    for a, b in zip(z, r):
        assert (a == b).all()
    ix.close()


def test_noalloc_at_its_capacity():
    """nq = 65,536, the static scratch's capacity: every result equals the
    allocating entry point's."""
    w = cases.clustered(n=20_000, nq=300, ncomp=8)
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    s = torch.cuda.Stream()
    n = 65536
    rng = np.random.default_rng(12)
    Q = np.ascontiguousarray(w["queries"][rng.integers(0, w["queries"].shape[0], n)])
    k = np.full(n, 10, np.uint32)
    L = rng.choice([16, 32], size=n).astype(np.uint32)
    q, kd, Ld = _dev(Q), _dev(k, np.int32), _dev(L, np.int32)
    r = _run(bang.bang_search_batched, ix, q, kd, Ld, n, 10, 32, s)
    z = _run(bang.bang_search_batched_noalloc, ix, q, kd, Ld, n, 10, 32, s)
    for a, b in zip(z, r):
        assert (a == b).all()
    assert (z[3] == 0).all()
    ix.close()


def test_noalloc_replayed_from_a_cuda_graph():
    """After one ordinary call (which looks up the scratch address), the
    entry point is recorded under stream capture and the graph replayed
    twice; each replay gives the allocating entry point's results."""
    w = cases.clustered(n=20_000, nq=300, ncomp=8)
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    Q, k, L = _batch(w, 250, 5)
    n, kmax, Lmax = 250, int(k.max()), int(L.max())
    q, kd, Ld = _dev(Q), _dev(k, np.int32), _dev(L, np.int32)
    s = torch.cuda.Stream()
    r = _run(bang.bang_search_batched, ix, q, kd, Ld, n, kmax, Lmax, s)
    ids = torch.full((n, kmax), -7, dtype=torch.int32, device="cuda")
    dist = torch.full((n, kmax), -7.0, dtype=torch.float32, device="cuda")
    iters = torch.zeros(n, dtype=torch.int32, device="cuda")
    status = torch.full((n,), 9, dtype=torch.int32, device="cuda")
    p = bang.make_params(out_iters=iters, out_status=status)
    bang.bang_search_batched_noalloc(ix.h, q, n, kd, Ld, kmax, Lmax, p, ids, dist,
                                     stream=s.cuda_stream)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bang.bang_search_batched_noalloc(ix.h, q, n, kd, Ld, kmax, Lmax, p, ids, dist,
                                         stream=s.cuda_stream)
    for _ in range(2):
        ids.fill_(-7)
        dist.fill_(-7.0)
        iters.zero_()
        status.fill_(9)
        g.replay()
        torch.cuda.synchronize()
        z = [t.cpu().numpy() for t in (ids, dist, iters, status)]
        for a, b in zip(z, r):
            assert (a == b).all()
    del g
    ix.close()


def test_noalloc_rejects_what_it_cannot_serve():
    w = cases.clustered(n=20_000, nq=300, ncomp=8)
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    Q, k, L = _batch(w, 8, 3)
    ids = torch.zeros((8, 100), dtype=torch.int32, device="cuda")
    dist = torch.zeros((8, 100), dtype=torch.float32, device="cuda")
    with pytest.raises(bang.BangError) as e:           # host arrays would need staging
        bang.bang_search_batched_noalloc(ix.h, Q, 8, k, L, 100, 256, None, ids, dist)
    assert e.value.code == bang.BANG_EINVAL
    with pytest.raises(bang.BangError) as e:           # beyond the static scratch
        bang.bang_search_batched_noalloc(ix.h, _dev(Q), 65537, _dev(k, np.int32),
                                         _dev(L, np.int32), 100, 256, None, ids, dist)
    assert e.value.code == bang.BANG_EINVAL and "65536" in str(e.value)
    ix.close()
