"""CPU oracle for the BANG search path (arXiv 2401.11324).

TEST INFRASTRUCTURE ONLY.  A plain C restatement of the paper's search
(Alg. 1, Alg. 2, §4.1-§4.8) plus the offline steps it consumes (PQ training
and encoding, medoid, Vamana), wrapped with ctypes for the tests.  Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the product path never does.  It shares
no code with the CUDA implementation.

Parity status of each function (see the C file for the passage it follows):
  pq_train, pq_encode, medoid, adc_table, adc_dist, adc_table_q8, adc_dist_q8, round_bf16,
  adc_table_bf16, exact_dist, bloom,
  search, bruteforce_knn : pinned by tests/test_oracle_*.py
  cluster_graph          : pinned by closed forms (a line with alpha = 1 gives
                           the chain; a huge alpha gives the exact nearest
                           lists) and by the generator's independent build
  vamana_build           : pinned by hand-worked builds (the chain at alpha = 1,
                           a reverse-edge overflow pruned back, an edge the
                           second pass restores) and invariants
  shard_graph            : pinned by closed forms (nearest-centre assignment,
                           complete rows when nothing is pruned, the chain at
                           alpha = 1), a hand-worked build that separates the
                           two passes' parameters, and invariants
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bang_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

U8, I8, F32 = 0, 1, 2
NONE = 0xFFFFFFFF

_DT = {np.dtype(np.uint8): U8, np.dtype(np.int8): I8, np.dtype(np.float32): F32}


def build(force=False):
    """Compile the oracle with gcc (plain C99, no FMA contraction, OpenMP
    across independent queries only)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "bang_oracle.h"))):
        return _LIB
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-Wall", "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.check_call(cmd, cwd=_HERE)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


class OrcIndex(ctypes.Structure):
    _fields_ = [("d", ctypes.c_uint32), ("M", ctypes.c_uint32), ("R", ctypes.c_uint32),
                ("medoid", ctypes.c_uint32), ("n", ctypes.c_uint64), ("dtype", ctypes.c_int),
                ("off", ctypes.c_void_p), ("codebook", ctypes.c_void_p),
                ("codes", ctypes.c_void_p), ("adj", ctypes.c_void_p), ("base", ctypes.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB points the pins at a deliberately broken copy of the
        # oracle (tests/test_oracle_mutants.py); normally unset.
        path = os.environ.get("ORACLE_LIB") or build()
        L = ctypes.CDLL(path)
        vp, u32, u64, i32, f32 = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                  ctypes.c_int, ctypes.c_float)
        L.orc_chunk_offsets.argtypes = [u32, u32, vp]
        L.orc_pq_train.argtypes = [vp, u32, u32, vp, vp, u64, vp, u32, vp, vp]
        L.orc_pq_train.restype = i32
        L.orc_pq_encode.argtypes = [vp, i32, u64, u32, u32, vp, vp, vp]
        L.orc_medoid.argtypes = [vp, i32, u64, u32]
        L.orc_medoid.restype = u32
        L.orc_robust_prune.argtypes = [vp, u32, u32, vp, u32, f32, u32, vp]
        L.orc_robust_prune.restype = u32
        L.orc_vamana_build.argtypes = [vp, u64, u32, u32, u32, f32, u32, vp, vp, vp]
        L.orc_vamana_build.restype = i32
        L.orc_cluster_graph.argtypes = [vp, i32, u32, u64, vp, vp, u32, vp, u32, f32, u32, vp,
                                        u32, vp, vp]
        L.orc_cluster_graph.restype = i32
        L.orc_shard_graph.argtypes = [vp, i32, u64, u32, vp, u32, u32, u32, u32, f32, f32, u32,
                                      u32, vp, vp, i32]
        L.orc_shard_graph.restype = i32
        L.orc_adc_table_f32.argtypes = [vp, u32, vp, vp, vp]
        L.orc_adc_dist_f32.argtypes = [vp, u32, vp]
        L.orc_adc_dist_f32.restype = f32
        L.orc_round_bf16.argtypes = [f32]
        L.orc_round_bf16.restype = f32
        L.orc_adc_table_bf16.argtypes = [vp, u32, vp]
        L.orc_adc_table_q8.argtypes = [vp, u32, vp]
        L.orc_adc_dist_q8.argtypes = [vp, u32, vp]
        L.orc_adc_dist_q8.restype = u32
        L.orc_exact_dist.argtypes = [vp, vp, i32, u32]
        L.orc_exact_dist.restype = ctypes.c_double
        L.orc_fnv1a32_bytes.argtypes = [ctypes.c_char_p, u32]
        L.orc_fnv1a32_bytes.restype = u32
        L.orc_fnv1a64_bytes.argtypes = [ctypes.c_char_p, u32]
        L.orc_fnv1a64_bytes.restype = u64
        L.orc_bloom_positions.argtypes = [u32, u32, vp]
        L.orc_bloom_test.argtypes = [vp, u32, u32]
        L.orc_bloom_test.restype = i32
        L.orc_bloom_insert.argtypes = [vp, u32, u32]
        L.orc_search.argtypes = [ctypes.POINTER(OrcIndex), vp, i32, u32, u32, u32, u32, u32, vp,
                                 vp, vp, vp, vp, vp, u32, i32]
        L.orc_search.restype = i32
        L.orc_search_rr.argtypes = L.orc_search.argtypes + [i32]
        L.orc_search_rr.restype = i32
        L.orc_max_threads.restype = i32
        L.orc_bruteforce_knn.argtypes = [vp, vp, i32, u64, u32, u32, u32, vp, vp, i32]
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def chunk_offsets(d, M):
    off = np.zeros(M + 1, np.uint32)
    lib().orc_chunk_offsets(d, M, _p(off))
    return off


def pq_train(X, M, sample, init, iters, return_trace=False):
    """k-means PQ codebook (256 centroids per subspace).  ``sample`` indexes
    the training points in X; ``init`` (M x 256) indexes X for the initial
    centroids of each subspace."""
    X = _c(X, np.float32)
    n, d = X.shape
    off = chunk_offsets(d, M)
    sample = _c(sample, np.uint64)
    init = _c(init, np.uint64).reshape(M, 256)
    cb = np.zeros(256 * d, np.float32)
    trace = np.zeros(M * max(iters, 1), np.float64)
    rc = lib().orc_pq_train(_p(X), d, M, _p(off), _p(sample), len(sample), _p(init), iters,
                            _p(cb), _p(trace))
    assert rc == 0
    if return_trace:
        return cb, trace.reshape(M, max(iters, 1))[:, :iters]
    return cb


def pq_encode(X, M, codebook):
    X = np.ascontiguousarray(X)
    n, d = X.shape
    off = chunk_offsets(d, M)
    codes = np.zeros((n, M), np.uint8)
    codebook = _c(codebook, np.float32)
    lib().orc_pq_encode(_p(X), _DT[X.dtype], n, d, M, _p(off), _p(codebook), _p(codes))
    return codes


def medoid(X):
    X = np.ascontiguousarray(X)
    return int(lib().orc_medoid(_p(X), _DT[X.dtype], X.shape[0], X.shape[1]))


def robust_prune(X, p, cand, alpha, R):
    X = _c(X, np.float32)
    cand = _c(cand, np.uint32)
    out = np.zeros(max(R, 1), np.uint32)
    k = lib().orc_robust_prune(_p(X), X.shape[1], p, _p(cand), len(cand), alpha, R, _p(out))
    return out[:k].copy()


def vamana_build(X, R, Lb, alpha, medoid_id, init_adj, order):
    X = _c(X, np.float32)
    n, d = X.shape
    init_adj = _c(init_adj, np.uint32).reshape(n, R)
    order = _c(order, np.uint32)
    adj = np.zeros((n, R), np.uint32)
    rc = lib().orc_vamana_build(_p(X), n, d, R, Lb, alpha, medoid_id, _p(init_adj), _p(order),
                                _p(adj))
    assert rc == 0
    return adj


def shard_graph(X, centres, ell, R, Lb, alpha, batch_frac=0.02, log2z=16, iter_cap=0,
                nthreads=0):
    """Overlapping-shard graph (orc_shard_graph, §2.2): n x R adjacency and
    the n x ell shard assignment (nearest centre first)."""
    X = np.ascontiguousarray(X)
    n, d = X.shape
    centres = _c(centres, np.float32).reshape(-1, d)
    S = centres.shape[0]
    adj = np.zeros((n, R), np.uint32)
    sh = np.zeros((n, ell), np.uint32)
    rc = lib().orc_shard_graph(_p(X), _DT[X.dtype], n, d, _p(centres), S, ell, R, Lb,
                               ctypes.c_float(alpha), ctypes.c_float(batch_frac), log2z,
                               iter_cap or (2 * Lb + 64), _p(adj), _p(sh), nthreads)
    assert rc == 0, rc
    return adj, sh


def cluster_graph(X, members, gstart, medoids, R, alpha, nx=0, xclu=None, nh=0, hclu=None):
    """Clustered construction (see orc_cluster_graph): n x R adjacency."""
    X = np.ascontiguousarray(X)
    n, d = X.shape
    members = _c(members, np.uint32)
    gstart = _c(gstart, np.uint64)
    medoids = _c(medoids, np.uint32)
    ng = len(medoids)
    xclu = _c(xclu if xclu is not None else np.zeros((n, 0)), np.uint32)
    hclu = _c(hclu if hclu is not None else np.zeros((ng, 0)), np.uint32)
    adj = np.zeros((n, R), np.uint32)
    rc = lib().orc_cluster_graph(_p(X), _DT[X.dtype], d, n, _p(members), _p(gstart), ng,
                                 _p(medoids), R, alpha, nx, _p(xclu), nh, _p(hclu), _p(adj))
    assert rc == 0
    return adj


def adc_table(q, M, codebook):
    q = _c(q, np.float32)
    d = q.shape[0]
    off = chunk_offsets(d, M)
    T = np.zeros((M, 256), np.float32)
    codebook = _c(codebook, np.float32)
    lib().orc_adc_table_f32(_p(q), M, _p(off), _p(codebook), _p(T))
    return T


def adc_dist(T, code):
    T = _c(T, np.float32)
    code = _c(code, np.uint8)
    return float(lib().orc_adc_dist_f32(_p(T), T.shape[0], _p(code)))


def round_bf16(x):
    return float(lib().orc_round_bf16(ctypes.c_float(x)))


def adc_table_bf16(T):
    T = _c(T, np.float32)
    out = np.zeros_like(T)
    lib().orc_adc_table_bf16(_p(T), T.shape[0], _p(out))
    return out


def adc_table_q8(T):
    """8-bit form of an FP32 table (per-subspace offset, one scale)."""
    T = _c(T, np.float32)
    Q = np.zeros(T.shape, np.uint8)
    lib().orc_adc_table_q8(_p(T), T.shape[0], _p(Q))
    return Q


def adc_dist_q8(Q, code):
    Q = _c(Q, np.uint8)
    code = _c(code, np.uint8)
    return int(lib().orc_adc_dist_q8(_p(Q), Q.shape[0], _p(code)))


def exact_dist(q, x):
    q = np.ascontiguousarray(q)
    x = np.ascontiguousarray(x, dtype=q.dtype)
    return float(lib().orc_exact_dist(_p(q), _p(x), _DT[q.dtype], q.shape[0]))


def fnv1a32(b):
    return int(lib().orc_fnv1a32_bytes(bytes(b), len(b)))


def fnv1a64(b):
    return int(lib().orc_fnv1a64_bytes(bytes(b), len(b)))


class Bloom:
    def __init__(self, log2z):
        self.log2z = log2z
        self.bits = np.zeros(max(1, (1 << log2z) // 32), np.uint32)

    def positions(self, i):
        p = np.zeros(2, np.uint32)
        lib().orc_bloom_positions(i, self.log2z, _p(p))
        return int(p[0]), int(p[1])

    def test(self, i):
        return bool(lib().orc_bloom_test(_p(self.bits), self.log2z, i))

    def insert(self, i):
        lib().orc_bloom_insert(_p(self.bits), self.log2z, i)


class Index:
    """Host-side index as the search reads it (arrays owned by this object)."""

    def __init__(self, base, codebook, codes, adj, medoid_id, M):
        self.base = np.ascontiguousarray(base)
        self.n, self.d = self.base.shape
        self.M = M
        self.off = chunk_offsets(self.d, M)
        self.codebook = _c(codebook, np.float32)
        self.codes = _c(codes, np.uint8).reshape(self.n, M)
        self.adj = _c(adj, np.uint32).reshape(self.n, -1)
        self.R = self.adj.shape[1]
        self.medoid = int(medoid_id)
        self.dtype = _DT[self.base.dtype]
        self._s = OrcIndex(self.d, self.M, self.R, self.medoid, self.n, self.dtype,
                           self.off.ctypes.data, self.codebook.ctypes.data,
                           self.codes.ctypes.data, self.adj.ctypes.data,
                           self.base.ctypes.data)

    def search(self, queries, k, L, log2z=16, iter_cap=None, trace_cap=0, nthreads=0, exact=False,
               q8=False, bf16=False, rerank_list=False):
        """Alg. 2 search; exact=True runs the Exact-distance variant (§5.2),
        q8=True the search on the 8-bit table, bf16=True on the BF16 table;
        rerank_list=True re-ranks the final worklist instead of the expanded
        nodes (PQ modes)."""
        assert exact + q8 + bf16 <= 1
        mode = 1 if exact else (2 if q8 else (3 if bf16 else 0))
        q = np.ascontiguousarray(queries, dtype=self.base.dtype)
        nq = q.shape[0]
        if iter_cap is None:
            iter_cap = 8 * L + 64
        ids = np.zeros((nq, k), np.uint32)
        dist = np.zeros((nq, k), np.float32)
        iters = np.zeros(nq, np.uint32)
        status = np.zeros(nq, np.int32)
        ndist = np.zeros(nq, np.uint64)
        trace = np.zeros((nq, trace_cap), np.uint32) if trace_cap else None
        rc = lib().orc_search_rr(ctypes.byref(self._s), _p(q), mode, nq, k, L, log2z,
                                 iter_cap, _p(ids),
                                 _p(dist), _p(iters), _p(status), _p(ndist), _p(trace), trace_cap,
                                 nthreads, 1 if rerank_list else 0)
        if rc != 0:
            raise ValueError("oracle search rejected its arguments")
        out = dict(ids=ids, dist=dist, iters=iters, status=status, ndist=ndist)
        if trace_cap:
            out["trace"] = trace
        return out


def bruteforce_knn(base, queries, k, nthreads=0):
    base = np.ascontiguousarray(base)
    q = np.ascontiguousarray(queries, dtype=base.dtype)
    nq = q.shape[0]
    ids = np.zeros((nq, k), np.uint32)
    dist = np.zeros((nq, k), np.float64)
    lib().orc_bruteforce_knn(_p(base), _p(q), _DT[base.dtype], base.shape[0], nq, base.shape[1],
                             k, _p(ids), _p(dist), nthreads)
    return ids, dist


def max_threads():
    return int(lib().orc_max_threads())


def recall_at_k(found, truth, k):
    """k-recall@k = |S ∩ S~| / k averaged over queries (§6.3)."""
    found = np.asarray(found)[:, :k]
    truth = np.asarray(truth)[:, :k]
    hits = [len(set(f.tolist()) & set(t.tolist())) for f, t in zip(found, truth)]
    return float(np.mean(hits)) / k
