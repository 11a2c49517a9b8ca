"""Serving with continuous batching: requests submitted from several threads
while others run are packed into overlapping launches, and every request's
result equals the same request searched alone (FP32 form: bit for bit)."""
import threading

import numpy as np
import pytest

from tests import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_11324_gb300 as bang  # noqa: E402


@pytest.fixture(scope="module")
def index():
    w = cases.clustered(n=20_000, nq=300, ncomp=8)
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    yield w, ix
    ix.close()


def _alone(ix, Q, k, L, kmax, Lmax, mode=0):
    ids = np.zeros((len(Q), kmax), np.uint32)
    dist = np.zeros((len(Q), kmax), np.float32)
    ix.search_batched(np.ascontiguousarray(Q), k, L, kmax, Lmax, ids, dist, bang.make_params(mode=mode))
    return ids, dist


@pytest.mark.parametrize("mode,early", [(0, 0), (0, 1), (1, 1)])
def test_each_result_same_alone_and_in_the_mix(index, mode, early):
    # FP32 and BF16 tables, code rows after the filter or early: the alone
    # search is the allocating batched form with early code rows off, whose
    # results early code rows do not change
    w, ix = index
    kmax, Lmax = 10, 128
    srv = bang.Server(ix, kmax, Lmax, max_batch=96, streams=3, mode=mode, early_codes=early)
    rng = np.random.default_rng(11)
    reqs = []
    for _ in range(60):
        n = int(rng.integers(1, 40))
        sel = rng.choice(w["queries"].shape[0], n, replace=False)
        k = rng.choice([1, 5, 10], size=n).astype(np.uint32)
        L = np.maximum(rng.choice([16, 64, 128], size=n), k).astype(np.uint32)
        reqs.append((w["queries"][sel], k, L))
    tickets = [None] * len(reqs)

    def submitter(part):
        for i in part:
            tickets[i] = srv.submit(*reqs[i])

    th = [threading.Thread(target=submitter, args=(range(j, len(reqs), 2),)) for j in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    lat = []
    for i, (Q, k, L) in enumerate(reqs):
        ids, dist, ms = srv.wait(tickets[i], timeout_ms=60_000)
        ids_a, dist_a = _alone(ix, Q, k, L, kmax, Lmax, mode)
        assert (ids == ids_a).all(), i
        fin = np.isfinite(dist_a)
        assert (dist[fin] == dist_a[fin]).all() and np.isinf(dist[~fin]).all()
        lat.append(ms)
    assert min(lat) > 0
    srv.stop()


def test_server_rejects_oversized_requests(index):
    w, ix = index
    srv = bang.Server(ix, 10, 64, max_batch=8, streams=1)
    with pytest.raises(bang.BangError) as e:
        srv.submit(w["queries"][:9], np.full(9, 10, np.uint32), np.full(9, 64, np.uint32))
    assert e.value.code == bang.BANG_EINVAL
    t = srv.submit(w["queries"][:8], np.full(8, 10, np.uint32), np.full(8, 64, np.uint32))
    ids, _, _ = srv.wait(t)
    assert (ids != bang.BANG_NONE).any()
    srv.stop()


def test_requests_wait_for_a_busy_slot(index):
    """One slot and more work than it holds: requests submitted at once queue
    behind the running launch (a zero-timeout wait on the last one reports
    BANG_ETIMEOUT and keeps its ticket), then every request completes with
    the result it has alone."""
    w, ix = index
    kmax, Lmax = 10, 128
    srv = bang.Server(ix, kmax, Lmax, max_batch=64, streams=1)
    rng = np.random.default_rng(21)
    reqs = []
    for _ in range(24):
        sel = rng.choice(w["queries"].shape[0], 64, replace=False)
        k = np.full(64, 10, np.uint32)
        L = np.full(64, 128, np.uint32)
        reqs.append((w["queries"][sel], k, L))
    tickets = [srv.submit(*r) for r in reqs]
    with pytest.raises(bang.BangError) as e:
        srv.wait(tickets[-1], timeout_ms=0)
    assert e.value.code == bang.BANG_ETIMEOUT
    lat = []
    for i, (Q, k, L) in enumerate(reqs):
        ids, dist, ms = srv.wait(tickets[i], timeout_ms=60_000)
        ids_a, dist_a = _alone(ix, Q, k, L, kmax, Lmax)
        assert (ids == ids_a).all(), i
        assert (dist == dist_a).all(), i
        lat.append(ms)
    # queued behind the single slot: later requests waited longer
    assert lat[-1] > lat[0]
    srv.stop()


def test_admission_by_device_memory(index):
    """A memory budget of about one and a half full batches with four
    streams: small requests run several at a time, full-size ones wait for
    memory to be released (first in, first out), a request larger than the
    budget is refused, and every result equals the request searched alone."""
    w, ix = index
    kmax, Lmax, d = 10, 64, w["base"].shape[1]
    per_q = d + 8 + 8 * kmax                       # bytes of one query's buffers
    srv = bang.Server(ix, kmax, Lmax, max_batch=256, streams=4, mem_bytes=int(1.5 * 256 * per_q) + 4096)
    rng = np.random.default_rng(31)
    reqs = []
    for i in range(40):
        n = 256 if i % 5 == 0 else int(rng.integers(1, 64))
        sel = rng.choice(w["queries"].shape[0], n, replace=True)
        reqs.append((w["queries"][sel], np.full(n, 10, np.uint32), np.full(n, 64, np.uint32)))
    tickets = [srv.submit(*r) for r in reqs]
    for i, (Q, k, L) in enumerate(reqs):
        ids, dist, _ = srv.wait(tickets[i], timeout_ms=60_000)
        ids_a, dist_a = _alone(ix, Q, k, L, kmax, Lmax)
        assert (ids == ids_a).all(), i
        assert (dist == dist_a).all(), i
    srv.stop()
    small = bang.Server(ix, kmax, Lmax, max_batch=256, streams=2, mem_bytes=64 * per_q + 4096)
    with pytest.raises(bang.BangError) as e:      # 256 queries need more than the budget
        small.submit(w["queries"][:256], np.full(256, 10, np.uint32), np.full(256, 64, np.uint32))
    assert e.value.code == bang.BANG_EINVAL
    t = small.submit(w["queries"][:32], np.full(32, 10, np.uint32), np.full(32, 64, np.uint32))
    ids, _, _ = small.wait(t, timeout_ms=60_000)
    assert (ids != bang.BANG_NONE).any()
    small.stop()
