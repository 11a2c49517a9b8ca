"""GPU path against the oracle, element by element, through the C ABI.

FP32 form: ids, visit sequence, iteration counts and distance-computation
counts are bit-exact; distances agree within 1e-5 relative (they are in fact
computed in the same order and compared exactly where the test says so)."""
import numpy as np
import pytest

import oracle
from tests import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_11324_gb300 as bang  # noqa: E402

RTOL = 1e-5


def gpu_search(w, Q, k, L, log2z=16, iter_cap=0, trace_cap=0, host=False, M=None, mode=0,
               placement=0, prefetch_depth=0, phases=False, early_codes=0, rerank=0, table_source=0,
               carveout=0, table_subspaces=0):
    M = M or w["M"]
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], M)
    if placement:
        ix.set_placement(placement)
    nq = Q.shape[0]
    dev = "cpu" if host else "cuda"
    if host:
        q = np.ascontiguousarray(Q)
    else:
        q = torch.from_numpy(np.ascontiguousarray(Q)).to(dev)
    ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
    dist = torch.empty((nq, k), dtype=torch.float32, device=dev)
    iters = torch.empty(nq, dtype=torch.int32, device=dev)
    status = torch.empty(nq, dtype=torch.int32, device=dev)
    ndist = torch.empty(nq, dtype=torch.int32, device=dev)
    trace = torch.zeros((nq, max(trace_cap, 1)), dtype=torch.int32, device=dev)
    ph = torch.zeros((nq, len(bang.PHASES)), dtype=torch.int64, device=dev) if phases else None
    p = bang.make_params(bloom_log2=log2z, iter_cap=iter_cap, out_iters=iters, out_status=status,
                         out_ndist=ndist, trace=trace if trace_cap else None, trace_cap=trace_cap,
                         mode=mode, prefetch_depth=prefetch_depth, out_phase_cycles=ph,
                         early_codes=early_codes, rerank=rerank, table_source=table_source,
                         smem_carveout=carveout, table_subspaces=table_subspaces)
    ix.search(q, k, L, ids, dist, p)
    torch.cuda.synchronize()
    out = dict(ids=ids.cpu().numpy().view(np.uint32), dist=dist.cpu().numpy(),
               iters=iters.cpu().numpy().view(np.uint32), status=status.cpu().numpy(),
               ndist=ndist.cpu().numpy().view(np.uint32), trace=trace.cpu().numpy().view(np.uint32))
    if phases:
        out["phases"] = ph.cpu().numpy()
    ix.close()
    return out


def oracle_search(w, Q, k, L, log2z=16, iter_cap=None, trace_cap=0, M=None, exact=False, q8=False,
                  bf16=False, rerank_list=False):
    M = M or w["M"]
    ix = oracle.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], M)
    return ix.search(Q, k, L, log2z=log2z, iter_cap=iter_cap, trace_cap=trace_cap, exact=exact,
                     q8=q8, bf16=bf16, rerank_list=rerank_list)


def assert_parity(g, o, trace_cap=0, exact_dist=True):
    assert (g["ids"] == o["ids"]).all(), np.argwhere(g["ids"] != o["ids"])[:5]
    assert (g["iters"] == o["iters"]).all()
    assert (g["status"] == o["status"]).all()
    assert (g["ndist"].astype(np.uint64) == o["ndist"]).all()
    fin = np.isfinite(o["dist"])
    assert (np.isfinite(g["dist"]) == fin).all()
    if exact_dist:
        assert (g["dist"][fin] == o["dist"][fin]).all()
    else:
        np.testing.assert_allclose(g["dist"][fin], o["dist"][fin], rtol=RTOL)
    if trace_cap:
        for i in range(len(g["iters"])):
            m = min(int(o["iters"][i]), trace_cap)
            assert (g["trace"][i, :m] == o["trace"][i, :m]).all()


@pytest.fixture(scope="module")
def cfg1():
    return cases.config1()


def test_config1_fp32_bit_exact(cfg1):
    Q = cfg1["queries"]
    g = gpu_search(cfg1, Q, 10, 64, trace_cap=1024)
    o = oracle_search(cfg1, Q, 10, 64, trace_cap=1024)
    assert_parity(g, o, trace_cap=1024)


@pytest.mark.parametrize("k,L,log2z", [(1, 1, 16), (10, 16, 12), (10, 64, 16), (32, 200, 18),
                                       (100, 256, 20)])
def test_config1_sweep(cfg1, k, L, log2z):
    Q = cfg1["queries"][:37]                           # ragged batch
    assert_parity(gpu_search(cfg1, Q, k, L, log2z), oracle_search(cfg1, Q, k, L, log2z))


@pytest.fixture(scope="module")
def u8small():
    return cases.clustered(n=20_000, nq=300, ncomp=8)


def test_clustered_u8_bit_exact(u8small):
    Q = u8small["queries"]
    for k, L in ((10, 32), (10, 128)):
        g = gpu_search(u8small, Q, k, L, trace_cap=600)
        o = oracle_search(u8small, Q, k, L, trace_cap=600)
        assert_parity(g, o, trace_cap=600)
        assert oracle.recall_at_k(g["ids"], u8small["gt_ids"], 10) > 0.5


def test_host_buffers_match_device_buffers(u8small):
    Q = u8small["queries"][:65]
    g_dev = gpu_search(u8small, Q, 10, 48)
    g_host = gpu_search(u8small, Q, 10, 48, host=True)
    for f in ("ids", "dist", "iters", "status", "ndist"):
        assert (g_dev[f] == g_host[f]).all()


def test_int8_uneven_subspaces():
    w = cases.clustered(n=8_000, nq=40, ncomp=4, dtype="i8", d=100, M=30, R=40,
                        centre="uniform100")
    Q = w["queries"]
    assert_parity(gpu_search(w, Q, 10, 40, trace_cap=200), oracle_search(w, Q, 10, 40, trace_cap=200),
                  trace_cap=200)


def test_f32_d96_M48_R68():
    w = cases.clustered(n=6_000, nq=50, ncomp=4, dtype="f32", d=96, M=48, R=68,
                        centre="uniform255")
    Q = w["queries"]
    assert_parity(gpu_search(w, Q, 10, 64, trace_cap=300), oracle_search(w, Q, 10, 64, trace_cap=300),
                  trace_cap=300)


def test_long_worklist(cfg1):
    Q = cfg1["queries"][:20]
    assert_parity(gpu_search(cfg1, Q, 64, 512, 17, trace_cap=900),
                  oracle_search(cfg1, Q, 64, 512, 17, trace_cap=900), trace_cap=900)


def test_f32_d200_wide_vectors():
    # d > 128: four 128-dimension chunks per lane in the exact distance
    w = cases.clustered(n=5_000, nq=30, ncomp=4, dtype="f32", d=200, M=50, R=48,
                        centre="uniform255")
    Q = w["queries"]
    assert_parity(gpu_search(w, Q, 10, 48, trace_cap=200), oracle_search(w, Q, 10, 48, trace_cap=200),
                  trace_cap=200)


def test_u8_d130_unaligned_rows():
    # d % 4 != 0: rows are not 4-byte aligned, scalar loads; 5 dims per subspace
    w = cases.clustered(n=5_000, nq=30, ncomp=4, dtype="u8", d=130, M=26, R=32,
                        centre="uniform255")
    Q = w["queries"]
    assert_parity(gpu_search(w, Q, 10, 40, trace_cap=200), oracle_search(w, Q, 10, 40, trace_cap=200),
                  trace_cap=200)


def test_iteration_cap_and_single_query(u8small):
    Q = u8small["queries"][:1]
    g = gpu_search(u8small, Q, 5, 64, iter_cap=7)
    o = oracle_search(u8small, Q, 5, 64, iter_cap=7)
    assert g["status"][0] == 1 and g["iters"][0] == 7
    assert_parity(g, o)


def test_isolated_medoid_pads_results(u8small):
    w = dict(u8small)
    adj = w["adj"].copy()
    adj[w["medoid"]] = bang.BANG_NONE
    w["adj"] = adj
    Q = w["queries"][:3]
    g = gpu_search(w, Q, 4, 8)
    assert (g["ids"][:, 0] == w["medoid"]).all() and (g["ids"][:, 1:] == bang.BANG_NONE).all()
    assert np.isinf(g["dist"][:, 1:]).all() and (g["iters"] == 1).all()


def test_rejects_bad_arguments(u8small):
    w = u8small
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    q = torch.from_numpy(w["queries"][:2]).cuda()
    ids = torch.empty((2, 10), dtype=torch.int32, device="cuda")
    dist = torch.empty((2, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(bang.BangError) as e:
        ix.search(q, 10, 5, ids, dist)              # L < k
    assert e.value.code == bang.BANG_EINVAL
    with pytest.raises(bang.BangError):
        ix.search(q, 10, 64, ids, dist, bang.make_params(bloom_log2=30))
    bad = w["adj"].copy()
    bad[5, 0] = w["base"].shape[0] + 3
    h = bang.bang_create(0)
    bang.bang_load_pq(h, w["base"].shape[1], w["M"], w["codebook"], w["codes"], w["base"].shape[0])
    with pytest.raises(bang.BangError) as e:
        bang.bang_register_graph(h, bad, bad.shape[1], w["medoid"])
    assert e.value.code == bang.BANG_EINVAL
    bang.bang_destroy(h)
    ix.close()


def test_empty_batch(u8small):
    w = u8small
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    q = torch.empty((0, w["base"].shape[1]), dtype=torch.uint8, device="cuda")
    ids = torch.empty((0, 10), dtype=torch.int32, device="cuda")
    dist = torch.empty((0, 10), dtype=torch.float32, device="cuda")
    ix.search(q, 10, 32, ids, dist)
    ix.close()


# ---------------------------------------------------------------- other forms

def test_in_memory_placement_matches_host_placement(u8small):
    # §5.1: graph and/or vectors read from HBM instead of host memory
    Q = u8small["queries"][:100]
    ref = gpu_search(u8small, Q, 10, 64, trace_cap=300)
    for flags in (bang.BANG_GRAPH_IN_HBM, bang.BANG_GRAPH_IN_HBM | bang.BANG_VECTORS_IN_HBM,
                  bang.BANG_VECTORS_IN_HBM, bang.BANG_VECTORS_IN_HBM | bang.BANG_GRAPH_PACKED):
        g = gpu_search(u8small, Q, 10, 64, trace_cap=300, placement=flags)
        for f in ("ids", "dist", "iters", "ndist", "trace"):
            assert (g[f] == ref[f]).all()


@pytest.mark.parametrize("mode", [0, 2, 3])
def test_packed_graph_rows_give_identical_results(u8small, cfg1, mode):
    # ids packed to the fewest bits (15 at n = 20,000; 14 at n = 10,000),
    # read from host memory or HBM: the same visits and results
    for w, Q, L in ((u8small, u8small["queries"][:120], 64), (cfg1, cfg1["queries"], 64)):
        ref = gpu_search(w, Q, 10, L, trace_cap=400, mode=mode)
        for flags in (bang.BANG_GRAPH_PACKED, bang.BANG_GRAPH_PACKED | bang.BANG_GRAPH_IN_HBM):
            g = gpu_search(w, Q, 10, L, trace_cap=400, mode=mode, placement=flags)
            for f in ("ids", "dist", "iters", "ndist", "trace"):
                assert (g[f] == ref[f]).all(), (mode, flags, f)


@pytest.mark.parametrize("mode", [0, 1, 3])
def test_neighbor_code_layout_gives_identical_results(u8small, cfg1, mode):
    # the codes of every node's neighbours side by side in HBM, alone or with
    # packed rows or the graph in HBM: the same visits and results
    for w, Q, L in ((u8small, u8small["queries"][:120], 64), (cfg1, cfg1["queries"], 64)):
        ref = gpu_search(w, Q, 10, L, trace_cap=400, mode=mode)
        for flags in (bang.BANG_NEIGHBOR_CODES, bang.BANG_NEIGHBOR_CODES | bang.BANG_GRAPH_PACKED,
                      bang.BANG_NEIGHBOR_CODES | bang.BANG_GRAPH_IN_HBM | bang.BANG_VECTORS_IN_HBM):
            g = gpu_search(w, Q, 10, L, trace_cap=400, mode=mode, placement=flags)
            for f in ("ids", "dist", "iters", "ndist", "trace"):
                assert (g[f] == ref[f]).all(), (mode, flags, f)


def test_placement_transitions_and_reregistration(u8small):
    # one index moved through every layout and back, then given its graph
    # again (which drops the layouts built from the old rows): same results
    w = u8small
    Q = np.ascontiguousarray(w["queries"][:64])
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    q = torch.from_numpy(Q).cuda()

    def run():
        ids = torch.empty((len(Q), 10), dtype=torch.int32, device="cuda")
        dist = torch.empty((len(Q), 10), dtype=torch.float32, device="cuda")
        ix.search(q, 10, 64, ids, dist, bang.make_params(mode=3, bloom_log2=15))
        torch.cuda.synchronize()
        return ids.cpu().numpy(), dist.cpu().numpy()

    ref = run()
    P, H, V, N = (bang.BANG_GRAPH_PACKED, bang.BANG_GRAPH_IN_HBM, bang.BANG_VECTORS_IN_HBM,
                  bang.BANG_NEIGHBOR_CODES)
    D = bang.BANG_NODE_RECORDS
    for flags in (P, P | H, H, N | H | V, N | P, 0, N, P | N | H | V, D | P, D, D | N, P, 0):
        ix.set_placement(flags)
        got = run()
        assert (got[0] == ref[0]).all() and (got[1] == ref[1]).all(), flags
    ix.set_placement(P | N)
    bang.bang_register_graph(ix.h, ix.adj, ix.R, ix.medoid)      # drops packed rows and codes
    got = run()
    assert (got[0] == ref[0]).all()
    with pytest.raises(bang.BangError):
        ix.set_placement(32)                                     # unknown flag
    ix.close()


def test_neighbor_code_layout_limits():
    w = cases.clustered(n=6_000, nq=5, ncomp=4, dtype="f32", d=96, M=48, R=68,
                        centre="uniform255")
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], 48)
    with pytest.raises(bang.BangError):
        ix.set_placement(bang.BANG_NEIGHBOR_CODES)        # R = 68 > 64 and M = 48 > 32
    ix.close()


@pytest.mark.parametrize("mode,flags", [(0, 0), (3, 0), (3, 4), (1, 11), (2, 3)])
def test_speculative_prefetch_gives_identical_results(u8small, cfg1, mode, flags):
    # prefetch_depth 2 also requests the first unvisited worklist entry at
    # the start of each iteration; visits and results are unchanged
    for w, Q, L in ((u8small, u8small["queries"][:120], 64), (cfg1, cfg1["queries"], 64)):
        ref = gpu_search(w, Q, 10, L, trace_cap=400, mode=mode, placement=flags)
        g = gpu_search(w, Q, 10, L, trace_cap=400, mode=mode, placement=flags, prefetch_depth=2)
        for f in ("ids", "dist", "iters", "ndist", "trace"):
            assert (g[f] == ref[f]).all(), (mode, flags, f)


@pytest.mark.parametrize("mode,flags", [(0, 0), (1, 0), (3, 0), (0, 3), (3, 3), (3, 4), (1, 6),
                                        (0, 16), (3, 8)])
def test_early_code_rows_give_identical_results(u8small, cfg1, mode, flags):
    # early_codes requests every neighbour's code row as soon as the node's
    # row arrives (the neighbour-code layout, flag 8, takes precedence);
    # visits, counts and results are unchanged and equal to the oracle's
    for w, Q, L in ((u8small, u8small["queries"][:120], 64), (cfg1, cfg1["queries"], 64)):
        ref = gpu_search(w, Q, 10, L, trace_cap=400, mode=mode, placement=flags)
        g = gpu_search(w, Q, 10, L, trace_cap=400, mode=mode, placement=flags, early_codes=1)
        for f in ("ids", "dist", "iters", "ndist", "trace"):
            assert (g[f] == ref[f]).all(), (mode, flags, f)
        o = oracle_search(w, Q, 10, L, trace_cap=400, q8=mode == 3, bf16=mode == 1)
        assert (g["ids"] == o["ids"]).all() and (g["iters"] == o["iters"]).all()


@pytest.mark.parametrize("mode,flags", [(0, 0), (1, 0), (2, 3), (3, 4)])
def test_phase_clock_instantiation_gives_identical_results(u8small, mode, flags):
    # out_phase_cycles selects a separate instantiation of the kernel with
    # the per-phase clock; visits and results are those of the plain one, and
    # the phases (table and loop) add up to at most the whole query's cycles
    Q = u8small["queries"][:100]
    ref = gpu_search(u8small, Q, 10, 64, trace_cap=300, mode=mode, placement=flags)
    g = gpu_search(u8small, Q, 10, 64, trace_cap=300, mode=mode, placement=flags, phases=True)
    for f in ("ids", "dist", "iters", "ndist", "trace"):
        assert (g[f] == ref[f]).all(), (mode, flags, f)
    ph = g["phases"]
    assert (ph >= 0).all()
    assert (ph[:, -1] > 0).all()
    assert (ph[:, :-1].sum(1) <= ph[:, -1]).all()


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_node_records_give_identical_results(u8small, cfg1, mode):
    # BANG_NODE_RECORDS: each node's row and vector in one host record
    R, P, N = bang.BANG_NODE_RECORDS, bang.BANG_GRAPH_PACKED, bang.BANG_NEIGHBOR_CODES
    for w, Q in ((u8small, u8small["queries"][:120]), (cfg1, cfg1["queries"])):
        ref = gpu_search(w, Q, 10, 64, trace_cap=400, mode=mode)
        for flags in (R, R | P, R | N, R | P | N):
            if (flags & N) and mode == 2:
                continue
            g = gpu_search(w, Q, 10, 64, trace_cap=400, mode=mode, placement=flags)
            for f in ("ids", "dist", "iters", "ndist", "trace"):
                assert (g[f] == ref[f]).all(), (mode, flags, f)


def test_node_records_f32_wide_rows_and_limits():
    # R = 68 f32 rows (272-byte rows before each vector) and d = 200 vectors
    for kw in (dict(dtype="f32", d=96, M=48, R=68), dict(dtype="f32", d=200, M=50, R=32)):
        w = cases.clustered(n=6_000, nq=40, ncomp=4, centre="uniform255", **kw)
        Q = w["queries"]
        for mode in (0, 2):
            ref = gpu_search(w, Q, 10, 48, trace_cap=200, mode=mode, M=kw["M"])
            for flags in (bang.BANG_NODE_RECORDS, bang.BANG_NODE_RECORDS | bang.BANG_GRAPH_PACKED):
                g = gpu_search(w, Q, 10, 48, trace_cap=200, mode=mode, M=kw["M"], placement=flags)
                for f in ("ids", "dist", "iters", "ndist", "trace"):
                    assert (g[f] == ref[f]).all(), (kw, mode, flags, f)
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    for bad in (bang.BANG_NODE_RECORDS | bang.BANG_GRAPH_IN_HBM,
                bang.BANG_NODE_RECORDS | bang.BANG_VECTORS_IN_HBM):
        with pytest.raises(bang.BangError):
            ix.set_placement(bad)
    ix.close()


def test_packed_graph_rows_wide_rows():
    # R = 68 (four neighbours per lane), 13-bit ids straddling word boundaries
    w = cases.clustered(n=6_000, nq=50, ncomp=4, dtype="f32", d=96, M=48, R=68,
                        centre="uniform255")
    Q = w["queries"]
    o = oracle_search(w, Q, 10, 64, trace_cap=300)
    g = gpu_search(w, Q, 10, 64, trace_cap=300, placement=bang.BANG_GRAPH_PACKED)
    assert_parity(g, o, trace_cap=300)


def _placed(a, offset):
    """Copy of `a` starting `offset` bytes past a 4096-byte boundary."""
    buf = np.empty(a.nbytes + 8192, np.uint8)
    start = (-buf.ctypes.data) % 4096 + offset
    v = buf[start:start + a.nbytes].view(a.dtype).reshape(a.shape)
    v[...] = a
    return v


def test_host_arrays_aligned_in_place_or_copied(u8small):
    # 128-byte-aligned graph and vectors are read in place; others are copied
    # once into aligned page-locked memory; the results are the same
    Q = u8small["queries"][:80]
    ref = gpu_search(u8small, Q, 10, 64, trace_cap=300)
    for off in (0, 16, 64, 128):
        w = dict(u8small, adj=_placed(u8small["adj"], off), base=_placed(u8small["base"], off))
        g = gpu_search(w, Q, 10, 64, trace_cap=300)
        for f in ("ids", "dist", "iters", "ndist", "trace"):
            assert (g[f] == ref[f]).all()


@pytest.mark.parametrize("placement", [0, 3])
def test_exact_mode_bit_exact(u8small, cfg1, placement):
    # §5.2: exact distances in the loop, no table, no re-rank
    for w, Q, L in ((u8small, u8small["queries"][:120], 48), (cfg1, cfg1["queries"], 64)):
        g = gpu_search(w, Q, 10, L, trace_cap=400, mode=bang.BANG_MODE_EXACT, placement=placement)
        o = oracle_search(w, Q, 10, L, trace_cap=400, exact=True)
        assert_parity(g, o, trace_cap=400)


def test_exact_mode_int8_rows_of_16_byte_multiples():
    # d = 96 int8: the one-lane-per-neighbour integer path, bias included
    w = cases.clustered(n=8_000, nq=40, ncomp=4, dtype="i8", d=96, M=24, R=40,
                        centre="uniform100")
    Q = w["queries"]
    for placement in (0, 3):
        g = gpu_search(w, Q, 10, 40, trace_cap=200, mode=bang.BANG_MODE_EXACT, placement=placement)
        assert_parity(g, oracle_search(w, Q, 10, 40, trace_cap=200, exact=True), trace_cap=200)


def test_exact_mode_int8():
    w = cases.clustered(n=8_000, nq=40, ncomp=4, dtype="i8", d=100, M=30, R=40,
                        centre="uniform100")
    Q = w["queries"]
    g = gpu_search(w, Q, 10, 40, trace_cap=200, mode=bang.BANG_MODE_EXACT)
    assert_parity(g, oracle_search(w, Q, 10, 40, trace_cap=200, exact=True), trace_cap=200)


@pytest.mark.parametrize("placement", [0, 3])
def test_bf16_mode_bit_exact(u8small, cfg1, placement):
    # the per-warp BF16 table rounds the FP32 entries to nearest (ties to
    # even) and sums them in the FP32 order: bit-exact with the oracle's mode
    for w, Q, L in ((u8small, u8small["queries"], 32), (u8small, u8small["queries"][:150], 128),
                    (cfg1, cfg1["queries"], 64)):
        g = gpu_search(w, Q, 10, L, trace_cap=600, mode=bang.BANG_MODE_PQ_BF16, placement=placement)
        o = oracle_search(w, Q, 10, L, trace_cap=600, bf16=True)
        assert_parity(g, o, trace_cap=600)


def test_bf16_mode_uneven_subspaces_and_wide_rows():
    for w, L in ((cases.clustered(n=8_000, nq=40, ncomp=4, dtype="i8", d=100, M=30, R=40,
                                  centre="uniform100"), 40),
                 (cases.clustered(n=6_000, nq=50, ncomp=4, dtype="f32", d=96, M=48, R=68,
                                  centre="uniform255"), 64)):
        Q = w["queries"]
        for k, LL, log2z in ((10, L, 16), (1, 1, 12), (40, 2 * L, 18)):
            g = gpu_search(w, Q, k, LL, log2z, trace_cap=300, mode=bang.BANG_MODE_PQ_BF16)
            assert_parity(g, oracle_search(w, Q, k, LL, log2z, trace_cap=300, bf16=True),
                          trace_cap=300)


def test_bf16_table_recall_within_tolerance(u8small):
    # reduced-precision form: judged by recall@10 against the FP32 form
    Q = u8small["queries"]
    gt = u8small["gt_ids"]
    for L in (32, 96):
        o = oracle_search(u8small, Q, 10, L)
        g = gpu_search(u8small, Q, 10, L, mode=bang.BANG_MODE_PQ_BF16)
        r_o = oracle.recall_at_k(o["ids"], gt, 10)
        r_g = oracle.recall_at_k(g["ids"], gt, 10)
        assert abs(r_g - r_o) <= 0.005 + 1.0 / (10 * len(Q)), (L, r_g, r_o)
        # the re-rank makes the returned distances exact for the ids returned
        ex = ((u8small["base"][g["ids"]].astype(np.int64) -
               Q[:, None, :].astype(np.int64)) ** 2).sum(-1)
        assert (g["dist"] == ex.astype(np.float32)).all()


# ---------------------------------------------------------------- 8-bit table form

@pytest.mark.parametrize("placement", [0, 3])
def test_q8_mode_bit_exact(u8small, cfg1, placement):
    # the 8-bit table is computed from the FP32 table in FP32 and summed in
    # integers, so the whole search is bit-exact with the oracle's mode
    for w, Q, L in ((u8small, u8small["queries"], 32), (u8small, u8small["queries"][:150], 128),
                    (cfg1, cfg1["queries"], 64)):
        g = gpu_search(w, Q, 10, L, trace_cap=600, mode=bang.BANG_MODE_PQ_Q8, placement=placement)
        o = oracle_search(w, Q, 10, L, trace_cap=600, q8=True)
        assert_parity(g, o, trace_cap=600)


def test_q8_mode_uneven_subspaces_and_wide_rows():
    for w, L in ((cases.clustered(n=8_000, nq=40, ncomp=4, dtype="i8", d=100, M=30, R=40,
                                  centre="uniform100"), 40),
                 (cases.clustered(n=6_000, nq=50, ncomp=4, dtype="f32", d=96, M=48, R=68,
                                  centre="uniform255"), 64)):
        Q = w["queries"]
        for k, LL, log2z in ((10, L, 16), (1, 1, 12), (40, 2 * L, 18)):
            g = gpu_search(w, Q, k, LL, log2z, trace_cap=300, mode=bang.BANG_MODE_PQ_Q8)
            assert_parity(g, oracle_search(w, Q, k, LL, log2z, trace_cap=300, q8=True), trace_cap=300)


# ---------------------------------------------------------------- batched form

def _mixed_kl(nq, seed):
    rng = np.random.default_rng(seed)
    k = rng.choice([1, 10, 100], size=nq).astype(np.uint32)
    L = np.maximum(rng.choice([32, 64, 128, 256], size=nq), k).astype(np.uint32)
    return k, L


def _oracle_mixed(w, Q, k, L, mode_exact=False, q8=False):
    kmax = int(k.max())
    ids = np.full((len(Q), kmax), bang.BANG_NONE, np.uint32)
    dist = np.full((len(Q), kmax), np.inf, np.float32)
    iters = np.zeros(len(Q), np.uint32)
    for kk in np.unique(k):
        for LL in np.unique(L[k == kk]):
            sel = np.where((k == kk) & (L == LL))[0]
            o = oracle_search(w, Q[sel], int(kk), int(LL), exact=mode_exact, q8=q8)
            ids[sel, :kk] = o["ids"]
            dist[sel, :kk] = o["dist"]
            iters[sel] = o["iters"]
    return ids, dist, iters


def test_batched_uneven_k_and_L_host_arrays(u8small):
    Q = u8small["queries"][:160]
    k, L = _mixed_kl(len(Q), 5)
    ids_o, dist_o, iters_o = _oracle_mixed(u8small, Q, k, L)
    ix = bang.Index(u8small["base"], u8small["codebook"], u8small["codes"], u8small["adj"],
                    u8small["medoid"], u8small["M"])
    kmax, Lmax = int(k.max()), int(L.max())
    for mult in (0, 3):
        ids = np.zeros((len(Q), kmax), np.uint32)
        dist = np.zeros((len(Q), kmax), np.float32)
        iters = np.zeros(len(Q), np.uint32)
        ix.search_batched(np.ascontiguousarray(Q), k, L, kmax, Lmax, ids, dist,
                          bang.make_params(out_iters=iters, grid_mult=mult))
        assert (ids == ids_o).all() and (iters == iters_o).all()
        fin = np.isfinite(dist_o)
        assert (np.isfinite(dist) == fin).all() and (dist[fin] == dist_o[fin]).all()
    ix.close()


def test_batched_q8_uneven_k_and_L(u8small):
    Q = u8small["queries"][:160]
    k, L = _mixed_kl(len(Q), 9)
    ids_o, dist_o, iters_o = _oracle_mixed(u8small, Q, k, L, q8=True)
    ix = bang.Index(u8small["base"], u8small["codebook"], u8small["codes"], u8small["adj"],
                    u8small["medoid"], u8small["M"])
    kmax, Lmax = int(k.max()), int(L.max())
    ids = np.zeros((len(Q), kmax), np.uint32)
    dist = np.zeros((len(Q), kmax), np.float32)
    iters = np.zeros(len(Q), np.uint32)
    ix.search_batched(np.ascontiguousarray(Q), k, L, kmax, Lmax, ids, dist,
                      bang.make_params(out_iters=iters, mode=bang.BANG_MODE_PQ_Q8))
    ix.close()
    assert (ids == ids_o).all() and (iters == iters_o).all()
    fin = np.isfinite(dist_o)
    assert (np.isfinite(dist) == fin).all() and (dist[fin] == dist_o[fin]).all()


def test_batched_cuda_graph_replay(u8small):
    Q = u8small["queries"][:128]
    k, L = _mixed_kl(len(Q), 6)
    ids_o, _, _ = _oracle_mixed(u8small, Q, k, L)
    ix = bang.Index(u8small["base"], u8small["codebook"], u8small["codes"], u8small["adj"],
                    u8small["medoid"], u8small["M"])
    kmax, Lmax = int(k.max()), int(L.max())
    q = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    kd = torch.from_numpy(k.view(np.int32)).cuda()
    Ld = torch.from_numpy(L.view(np.int32)).cuda()
    ids = torch.zeros((len(Q), kmax), dtype=torch.int32, device="cuda")
    dist = torch.zeros((len(Q), kmax), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    p = bang.make_params()
    with torch.cuda.stream(s):
        ix.search_batched(q, kd, Ld, kmax, Lmax, ids, dist, p, stream=s.cuda_stream)  # allocates
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ix.search_batched(q, kd, Ld, kmax, Lmax, ids, dist, p, stream=s.cuda_stream)
    for _ in range(2):
        ids.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert (ids.cpu().numpy().view(np.uint32) == ids_o).all()
    ix.close()


def test_batched_invalid_rows_are_flagged(u8small):
    Q = u8small["queries"][:4]
    k = np.array([10, 0, 10, 5], np.uint32)
    L = np.array([64, 64, 5, 64], np.uint32)           # row 1: k=0, row 2: L<k
    ix = bang.Index(u8small["base"], u8small["codebook"], u8small["codes"], u8small["adj"],
                    u8small["medoid"], u8small["M"])
    ids = np.zeros((4, 10), np.uint32)
    dist = np.zeros((4, 10), np.float32)
    status = np.zeros(4, np.int32)
    ix.search_batched(np.ascontiguousarray(Q), k, L, 10, 64, ids, dist,
                      bang.make_params(out_status=status))
    assert status.tolist() == [0, -1, -1, 0]
    assert (ids[1] == bang.BANG_NONE).all() and (ids[2] == bang.BANG_NONE).all()
    o = oracle_search(u8small, Q[[0]], 10, 64)
    assert (ids[0] == o["ids"][0]).all()
    o5 = oracle_search(u8small, Q[[3]], 5, 64)
    assert (ids[3, :5] == o5["ids"][0]).all() and (ids[3, 5:] == bang.BANG_NONE).all()
    ix.close()


# ---- staged re-rank (§4.8 as a separate kernel after the search)

def _same(g, ref, fields=("ids", "dist", "iters", "status", "ndist", "trace")):
    for f in fields:
        assert (g[f] == ref[f]).all(), (f, np.argwhere(g[f] != ref[f])[:5])


@pytest.mark.parametrize("mode", [0, 1, 3])
@pytest.mark.parametrize("flags", [0, 3, 3 | 4, 16, 8])
def test_staged_rerank_equals_fused_and_oracle(u8small, cfg1, mode, flags):
    # the loop records its expanded nodes and a second kernel ranks them:
    # the same visits, counts and results as the fused re-rank, and the
    # oracle's ids and distances
    for w, Q, L in ((u8small, u8small["queries"][:150], 64), (cfg1, cfg1["queries"], 64)):
        ref = gpu_search(w, Q, 10, L, trace_cap=400, mode=mode, placement=flags)
        g = gpu_search(w, Q, 10, L, trace_cap=400, mode=mode, placement=flags, rerank=1)
        _same(g, ref)
        o = oracle_search(w, Q, 10, L, trace_cap=400, q8=mode == 3, bf16=mode == 1)
        assert (g["ids"] == o["ids"]).all() and (g["iters"] == o["iters"]).all()
        fin = np.isfinite(o["dist"])
        assert (g["dist"][fin] == o["dist"][fin]).all()


@pytest.mark.parametrize("k,L", [(1, 1), (32, 64), (33, 80), (100, 256)])
def test_staged_rerank_k_beyond_registers(u8small, k, L):
    # k <= 32 keeps the top-k in registers, larger k in shared memory; L = k = 1 too
    Q = u8small["queries"][:70]
    ref = gpu_search(u8small, Q, k, L, trace_cap=0)
    g = gpu_search(u8small, Q, k, L, rerank=1)
    _same(g, ref, ("ids", "dist", "iters", "status", "ndist"))
    o = oracle_search(u8small, Q, k, L)
    assert (g["ids"] == o["ids"]).all()


@pytest.mark.parametrize("shape", ["i8_d100_M30", "f32_d96_M48", "f32_d200_M50", "u8_d130_M26",
                                   "i8_d128_M32", "u8_d64_M16"])
def test_staged_rerank_element_types_and_widths(shape):
    # int8 (biased lanes), FP32 (the 32-lane summation order), d > 128 (four
    # chunks per lane), rows that are not 4-byte aligned, and integer rows of
    # 16-byte multiples (one lane per candidate row)
    spec = {"i8_d128_M32": dict(n=6_000, nq=50, ncomp=4, dtype="i8", d=128, M=32, R=40, centre="uniform100"),
            "u8_d64_M16": dict(n=6_000, nq=50, ncomp=4, dtype="u8", d=64, M=16, R=32, centre="uniform255"),
            "i8_d100_M30": dict(n=6_000, nq=40, ncomp=4, dtype="i8", d=100, M=30, R=40, centre="uniform100"),
            "f32_d96_M48": dict(n=5_000, nq=40, ncomp=4, dtype="f32", d=96, M=48, R=68, centre="uniform255"),
            "f32_d200_M50": dict(n=4_000, nq=30, ncomp=4, dtype="f32", d=200, M=50, R=48, centre="uniform255"),
            "u8_d130_M26": dict(n=4_000, nq=30, ncomp=4, dtype="u8", d=130, M=26, R=32, centre="uniform255")}[shape]
    w = cases.clustered(**spec)
    Q = w["queries"]
    for mode in (0, 3):
        ref = gpu_search(w, Q, 10, 48, trace_cap=300, mode=mode)
        g = gpu_search(w, Q, 10, 48, trace_cap=300, mode=mode, rerank=1)
        _same(g, ref)
    o = oracle_search(w, Q, 10, 48)
    g = gpu_search(w, Q, 10, 48, rerank=1)
    assert (g["ids"] == o["ids"]).all()
    fin = np.isfinite(o["dist"])
    assert (g["dist"][fin] == o["dist"][fin]).all()


def test_staged_rerank_iteration_cap_and_host_buffers(u8small):
    # a capped search (status 1) keeps the candidates it expanded; host
    # buffers are staged like the fused form's
    Q = u8small["queries"][:50]
    ref = gpu_search(u8small, Q, 10, 64, iter_cap=7)
    g = gpu_search(u8small, Q, 10, 64, iter_cap=7, rerank=1)
    _same(g, ref, ("ids", "dist", "iters", "status", "ndist"))
    assert (g["status"] == 1).all()
    gh = gpu_search(u8small, Q, 10, 64, host=True, rerank=1)
    gd = gpu_search(u8small, Q, 10, 64)
    _same(gh, gd, ("ids", "dist", "iters", "status", "ndist"))


def test_staged_rerank_batched_uneven_k_and_L(u8small):
    Q = u8small["queries"][:160]
    k, L = _mixed_kl(len(Q), 12)
    k[3], L[5] = 0, 2000                                  # two invalid rows
    ix = bang.Index(u8small["base"], u8small["codebook"], u8small["codes"], u8small["adj"],
                    u8small["medoid"], u8small["M"])
    kmax, Lmax = 100, 256
    out = []
    for rr in (0, 1):
        ids = np.zeros((len(Q), kmax), np.uint32)
        dist = np.zeros((len(Q), kmax), np.float32)
        status = np.zeros(len(Q), np.int32)
        ix.search_batched(np.ascontiguousarray(Q), k, L, kmax, Lmax, ids, dist,
                          bang.make_params(out_status=status, rerank=rr))
        out.append((ids, dist, status))
    ix.close()
    (i0, d0, s0), (i1, d1, s1) = out
    assert (i0 == i1).all() and (s0 == s1).all()
    assert (np.isfinite(d0) == np.isfinite(d1)).all() and (d0[np.isfinite(d0)] == d1[np.isfinite(d1)]).all()
    assert s1[3] == -1 and s1[5] == -1 and (i1[3] == bang.BANG_NONE).all()
    ok = np.array([i for i in range(len(Q)) if i not in (3, 5)])
    ids_o, _, _ = _oracle_mixed(u8small, Q[ok], k[ok], L[ok])
    assert (i1[ok, :ids_o.shape[1]] == ids_o).all()


def test_staged_rerank_graph_capture_and_rejections(u8small):
    Q = u8small["queries"][:64]
    ref = gpu_search(u8small, Q, 10, 64)
    ix = bang.Index(u8small["base"], u8small["codebook"], u8small["codes"], u8small["adj"],
                    u8small["medoid"], u8small["M"])
    q = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    ids = torch.zeros((64, 10), dtype=torch.int32, device="cuda")
    dist = torch.zeros((64, 10), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    p = bang.make_params(rerank=1)
    ix.search(q, 10, 64, ids, dist, p, stream=s.cuda_stream)       # allocates the candidate lists
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ix.search(q, 10, 64, ids, dist, p, stream=s.cuda_stream)
    for _ in range(2):
        ids.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert (ids.cpu().numpy().view(np.uint32) == ref["ids"]).all()
    for bad in (bang.make_params(rerank=3), bang.make_params(rerank=1, mode=bang.BANG_MODE_EXACT),
                bang.make_params(rerank=2, mode=bang.BANG_MODE_EXACT)):
        with pytest.raises(bang.BangError):
            ix.search(q, 10, 64, ids, dist, bad)
    kd = torch.full((64,), 10, dtype=torch.int32, device="cuda")
    Ld = torch.full((64,), 64, dtype=torch.int32, device="cuda")
    with pytest.raises(bang.BangError):
        bang.bang_search_batched_noalloc(ix.h, q, 64, kd, Ld, 10, 64, bang.make_params(rerank=1), ids, dist)
    ix.close()


# ---- FP32 form without a table (table_source 3): entries computed from the
# codebook when a distance needs them, in the table build's arithmetic

@pytest.mark.parametrize("flags,early", [(0, 0), (3, 1), (3, 0), (3 | 4, 1), (16, 1), (8, 0)])
def test_table_free_fp32_equals_table_and_oracle(u8small, cfg1, flags, early):
    for w, Q, L in ((u8small, u8small["queries"][:150], 64), (cfg1, cfg1["queries"], 64)):
        ref = gpu_search(w, Q, 10, L, trace_cap=400, placement=flags, early_codes=early)
        g = gpu_search(w, Q, 10, L, trace_cap=400, placement=flags, early_codes=early, table_source=3)
        _same(g, ref)
        o = oracle_search(w, Q, 10, L, trace_cap=400)
        assert_parity(g, o, trace_cap=400)


@pytest.mark.parametrize("shape", ["i8_d100_M30", "f32_d96_M48", "f32_d200_M50", "u8_d130_M26"])
def test_table_free_fp32_subspace_shapes(shape):
    # uneven subspaces (offsets read per entry), 2, 4 and 5 dimensions per
    # subspace, d > 128, rows that are not 4-byte aligned
    spec = {"i8_d100_M30": dict(n=6_000, nq=40, ncomp=4, dtype="i8", d=100, M=30, R=40, centre="uniform100"),
            "f32_d96_M48": dict(n=5_000, nq=40, ncomp=4, dtype="f32", d=96, M=48, R=68, centre="uniform255"),
            "f32_d200_M50": dict(n=4_000, nq=30, ncomp=4, dtype="f32", d=200, M=50, R=48, centre="uniform255"),
            "u8_d130_M26": dict(n=4_000, nq=30, ncomp=4, dtype="u8", d=130, M=26, R=32, centre="uniform255")}[shape]
    w = cases.clustered(**spec)
    Q = w["queries"]
    g = gpu_search(w, Q, 10, 48, trace_cap=300, table_source=3)
    _same(g, gpu_search(w, Q, 10, 48, trace_cap=300))
    assert_parity(g, oracle_search(w, Q, 10, 48, trace_cap=300), trace_cap=300)


@pytest.mark.parametrize("carveout", [0, 25, 60, 100])
def test_carveout_hint_leaves_results_unchanged(u8small, carveout):
    Q = u8small["queries"][:100]
    ref = gpu_search(u8small, Q, 10, 64, trace_cap=300, placement=3)
    for ts in (0, 3):
        g = gpu_search(u8small, Q, 10, 64, trace_cap=300, placement=3, table_source=ts, carveout=carveout)
        _same(g, ref)


def test_table_free_fp32_long_lists_batched_and_noalloc(u8small, cfg1):
    Q = cfg1["queries"][:20]
    assert_parity(gpu_search(cfg1, Q, 64, 512, 17, trace_cap=900, table_source=3),
                  oracle_search(cfg1, Q, 64, 512, 17, trace_cap=900), trace_cap=900)
    Q = u8small["queries"][:160]
    k, L = _mixed_kl(len(Q), 21)
    ids_o, dist_o, iters_o = _oracle_mixed(u8small, Q, k, L)
    ix = bang.Index(u8small["base"], u8small["codebook"], u8small["codes"], u8small["adj"],
                    u8small["medoid"], u8small["M"])
    kmax, Lmax = int(k.max()), int(L.max())
    ids = np.zeros((len(Q), kmax), np.uint32)
    dist = np.zeros((len(Q), kmax), np.float32)
    iters = np.zeros(len(Q), np.uint32)
    ix.search_batched(np.ascontiguousarray(Q), k, L, kmax, Lmax, ids, dist,
                      bang.make_params(out_iters=iters, table_source=3))
    assert (ids == ids_o).all() and (iters == iters_o).all()
    q = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    kd = torch.from_numpy(k.view(np.int32)).cuda()
    Ld = torch.from_numpy(L.view(np.int32)).cuda()
    idd = torch.zeros((len(Q), kmax), dtype=torch.int32, device="cuda")
    dd = torch.zeros((len(Q), kmax), dtype=torch.float32, device="cuda")
    bang.bang_search_batched_noalloc(ix.h, q, len(Q), kd, Ld, kmax, Lmax,
                                     bang.make_params(table_source=3, smem_carveout=50), idd, dd)
    torch.cuda.synchronize()
    assert (idd.cpu().numpy().view(np.uint32) == ids_o).all()
    for bad in (bang.make_params(table_source=3, mode=bang.BANG_MODE_PQ_BF16),
                bang.make_params(table_source=3, mode=bang.BANG_MODE_PQ_Q8),
                bang.make_params(smem_carveout=101), bang.make_params(table_source=4)):
        with pytest.raises(bang.BangError):
            ix.search(q, 10, 64, idd[:, :10].contiguous(), dd[:, :10].contiguous(), bad)
    ix.close()


@pytest.mark.parametrize("ntab", [1, 8, 16, 31, 32, 40])
def test_partial_table_equals_table_and_oracle(u8small, cfg1, ntab):
    # the first ntab subspaces from the table, the others computed: the same
    # bits as the whole table (ntab >= M is the whole table)
    for w, Q in ((u8small, u8small["queries"][:120]), (cfg1, cfg1["queries"])):
        for early in (0, 1):
            ref = gpu_search(w, Q, 10, 64, trace_cap=400, placement=3, early_codes=early)
            g = gpu_search(w, Q, 10, 64, trace_cap=400, placement=3, early_codes=early, table_source=3,
                           table_subspaces=ntab)
            _same(g, ref)
    o = oracle_search(cfg1, cfg1["queries"], 10, 64, trace_cap=400)
    assert_parity(g, o, trace_cap=400)


def test_partial_table_uneven_subspaces():
    w = cases.clustered(n=6_000, nq=40, ncomp=4, dtype="i8", d=100, M=30, R=40, centre="uniform100")
    Q = w["queries"]
    ref = gpu_search(w, Q, 10, 48, trace_cap=300)
    for ntab in (7, 10, 29):
        _same(gpu_search(w, Q, 10, 48, trace_cap=300, table_source=3, table_subspaces=ntab), ref)


@pytest.mark.parametrize("mode,flags", [(0, 0), (0, 3), (1, 3), (3, 3), (0, 3 | 4), (0, 16), (1, 6)])
def test_speculated_row_with_early_code_rows(u8small, cfg1, mode, flags):
    # prefetch depth 2 with early code rows: the first unvisited worklist
    # entry's row is requested at the start of an iteration and, when it is
    # chosen, its neighbours' code rows at once; visits and results unchanged
    for w, Q, L in ((u8small, u8small["queries"][:150], 96), (cfg1, cfg1["queries"], 64)):
        ref = gpu_search(w, Q, 10, L, trace_cap=600, mode=mode, placement=flags)
        g = gpu_search(w, Q, 10, L, trace_cap=600, mode=mode, placement=flags, early_codes=1,
                       prefetch_depth=2)
        _same(g, ref)
        g2 = gpu_search(w, Q, 10, L, trace_cap=600, mode=mode, placement=flags, early_codes=1,
                        prefetch_depth=2, rerank=1)
        _same(g2, ref)
        o = oracle_search(w, Q, 10, L, trace_cap=600, q8=mode == 3, bf16=mode == 1)
        assert (g["ids"] == o["ids"]).all() and (g["iters"] == o["iters"]).all()


# ---- staged re-rank of the final worklist only (rerank = 2)

@pytest.mark.parametrize("mode", [0, 1, 3])
@pytest.mark.parametrize("flags", [0, 3, 3 | 4, 16])
def test_final_worklist_rerank_equals_oracle(u8small, cfg1, mode, flags):
    for w, Q, L in ((u8small, u8small["queries"][:150], 64), (cfg1, cfg1["queries"], 48)):
        g = gpu_search(w, Q, 10, L, trace_cap=400, mode=mode, placement=flags, rerank=2)
        o = oracle_search(w, Q, 10, L, trace_cap=400, q8=mode == 3, bf16=mode == 1, rerank_list=True)
        assert_parity(g, o, trace_cap=400)
        ref = gpu_search(w, Q, 10, L, trace_cap=400, mode=mode, placement=flags)
        _same(g, ref, ("iters", "status", "ndist", "trace"))      # same search, other candidates


@pytest.mark.parametrize("k,L,cap", [(1, 1, 0), (10, 64, 9), (32, 40, 0), (50, 100, 0), (100, 256, 30)])
def test_final_worklist_rerank_k_and_cap(u8small, k, L, cap):
    # registers and shared-memory top-k; a capped search re-ranks a worklist
    # with unexpanded entries (the cap below L sizes the lists by L)
    Q = u8small["queries"][:60]
    g = gpu_search(u8small, Q, k, L, iter_cap=cap, rerank=2)
    o = oracle_search(u8small, Q, k, L, iter_cap=cap or None, rerank_list=True)
    assert_parity(g, o)


def test_final_worklist_rerank_other_types_and_batched(u8small):
    for spec in (dict(n=4_000, nq=30, ncomp=4, dtype="f32", d=96, M=48, R=68, centre="uniform255"),
                 dict(n=4_000, nq=30, ncomp=4, dtype="i8", d=128, M=32, R=40, centre="uniform100")):
        w = cases.clustered(**spec)
        assert_parity(gpu_search(w, w["queries"], 10, 48, rerank=2),
                      oracle_search(w, w["queries"], 10, 48, rerank_list=True))
    Q = u8small["queries"][:120]
    k, L = _mixed_kl(len(Q), 33)
    ix = bang.Index(u8small["base"], u8small["codebook"], u8small["codes"], u8small["adj"],
                    u8small["medoid"], u8small["M"])
    kmax, Lmax = int(k.max()), int(L.max())
    ids = np.zeros((len(Q), kmax), np.uint32)
    dist = np.zeros((len(Q), kmax), np.float32)
    ix.search_batched(np.ascontiguousarray(Q), k, L, kmax, Lmax, ids, dist, bang.make_params(rerank=2))
    ix.close()
    for kk in np.unique(k):
        for LL in np.unique(L[k == kk]):
            sel = np.where((k == kk) & (L == LL))[0]
            o = oracle_search(u8small, Q[sel], int(kk), int(LL), rerank_list=True)
            assert (ids[sel, :kk] == o["ids"]).all()
