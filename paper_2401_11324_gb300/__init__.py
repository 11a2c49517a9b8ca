"""GB300-native BANG search path (arXiv 2401.11324): Python binding.

Argument marshalling over the C ABI declared in ``include/bang.h``; every step
of the search runs in the CUDA library ``csrc/libbang.so``.  There is no CPU
fallback: importing this package without the compiled library raises.

Functions carry the C names (``bang_create``, ``bang_load_pq``, ...).  Buffers
may be numpy arrays (host) or torch tensors (host or CUDA); the library
detects where each one lives.  ``Index`` is a thin convenience wrapper that
keeps the host arrays the library reads in place alive.
"""
import ctypes
import os

import numpy as np

from . import build as _build

BANG_OK, BANG_EINVAL, BANG_ENOMEM, BANG_ECUDA, BANG_ETIMEOUT, BANG_ESTATE = 0, -1, -2, -3, -4, -5
BANG_U8, BANG_I8, BANG_F32 = 0, 1, 2
BANG_NONE = 0xFFFFFFFF

_lib = None


class BangError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (status %d)" % (msg, code))
        self.code = code


class bang_search_params(ctypes.Structure):
    _fields_ = [("bloom_log2", ctypes.c_uint32), ("iter_cap", ctypes.c_uint32),
                ("out_iters", ctypes.c_void_p), ("out_status", ctypes.c_void_p),
                ("out_ndist", ctypes.c_void_p), ("trace", ctypes.c_void_p),
                ("trace_cap", ctypes.c_uint32), ("out_phase_cycles", ctypes.c_void_p),
                ("mode", ctypes.c_uint32), ("grid_mult", ctypes.c_uint32),
                ("table_source", ctypes.c_uint32), ("prefetch_depth", ctypes.c_uint32),
                ("early_codes", ctypes.c_uint32), ("rerank", ctypes.c_uint32),
                ("smem_carveout", ctypes.c_uint32), ("table_subspaces", ctypes.c_uint32)]


class bang_link_probe(ctypes.Structure):
    _fields_ = [("h2d_copy_gbs", ctypes.c_double), ("gather_gbs", ctypes.c_double),
                ("latency_ns", ctypes.c_double), ("gather_row_bytes", ctypes.c_uint32),
                ("cpu_gather_gbs", ctypes.c_double), ("cpu_threads", ctypes.c_uint32)]


def bang_probe_host_link(device=0, nbytes=1 << 30, row_bytes=256):
    out = bang_link_probe()
    _check(lib().bang_probe_host_link(device, nbytes, row_bytes, ctypes.byref(out)))
    return dict(h2d_copy_gbs=out.h2d_copy_gbs, gather_gbs=out.gather_gbs,
                latency_ns=out.latency_ns, gather_row_bytes=out.gather_row_bytes,
                cpu_gather_gbs=out.cpu_gather_gbs, cpu_threads=out.cpu_threads)


class bang_server_config(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_uint32), ("L_max", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32), ("streams", ctypes.c_uint32),
                ("mode", ctypes.c_uint32), ("bloom_log2", ctypes.c_uint32),
                ("mem_bytes", ctypes.c_uint64), ("early_codes", ctypes.c_uint32)]


class bang_autotune_opts(ctypes.Structure):
    _fields_ = [("modes", ctypes.c_uint32), ("bloom_min", ctypes.c_uint32),
                ("bloom_max", ctypes.c_uint32), ("try_tensor_tables", ctypes.c_uint32),
                ("batched", ctypes.c_uint32), ("reps", ctypes.c_uint32),
                ("target_recall", ctypes.c_float), ("recall_tolerance", ctypes.c_float),
                ("cache_path", ctypes.c_char_p), ("try_packed_graph", ctypes.c_uint32),
                ("try_neighbor_codes", ctypes.c_uint32), ("try_prefetch_depth", ctypes.c_uint32),
                ("try_node_records", ctypes.c_uint32), ("try_structure", ctypes.c_uint32)]


class bang_autotune_result(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("bloom_log2", ctypes.c_uint32),
                ("table_source", ctypes.c_uint32), ("grid_mult", ctypes.c_uint32),
                ("L", ctypes.c_uint32), ("ms", ctypes.c_float), ("recall", ctypes.c_float),
                ("ref_ms", ctypes.c_float), ("ref_recall", ctypes.c_float),
                ("candidates", ctypes.c_uint32), ("from_cache", ctypes.c_uint32),
                ("graph_packed", ctypes.c_uint32), ("neighbor_codes", ctypes.c_uint32),
                ("prefetch_depth", ctypes.c_uint32), ("node_records", ctypes.c_uint32),
                ("early_codes", ctypes.c_uint32), ("rerank", ctypes.c_uint32)]


def library_path():
    return _build.LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise ImportError("libbang.so is not built (%s); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % _build.LIB)
    L = ctypes.CDLL(_build.LIB)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    L.bang_create.argtypes = [i32, ctypes.POINTER(vp)]
    L.bang_load_pq.argtypes = [vp, u32, u32, vp, vp, u64]
    L.bang_register_graph.argtypes = [vp, vp, u32, u32]
    L.bang_register_vectors.argtypes = [vp, vp, i32]
    L.bang_search.argtypes = [vp, vp, u32, u32, u32, ctypes.POINTER(bang_search_params), vp, vp,
                              vp]
    L.bang_destroy.argtypes = [vp]
    L.bang_set_placement.argtypes = [vp, u32]
    L.bang_search_batched.argtypes = [vp, vp, u32, vp, vp, u32, u32,
                                      ctypes.POINTER(bang_search_params), vp, vp, vp]
    L.bang_search_batched_noalloc.argtypes = L.bang_search_batched.argtypes
    L.bang_index_info.argtypes = [vp, vp, vp, vp, vp, vp]
    L.bang_pq_tables.argtypes = [vp, vp, u32, vp, u32, vp]
    L.bang_server_start.argtypes = [vp, ctypes.POINTER(bang_server_config), ctypes.POINTER(vp)]
    L.bang_server_submit.argtypes = [vp, vp, u32, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
    L.bang_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_int32, vp, vp,
                                   ctypes.POINTER(ctypes.c_double)]
    L.bang_server_stop.argtypes = [vp]
    L.bang_build_cluster_graph.argtypes = [i32, vp, i32, u64, u32, vp, vp, u32, vp, u32,
                                           ctypes.c_float, u32, vp, u32, vp, vp, vp]
    L.bang_ground_truth.argtypes = [i32, vp, vp, i32, u64, u32, u32, u32, vp, vp, vp]
    L.bang_build_shard_graph.argtypes = [i32, vp, i32, u64, u32, vp, u32, u32, u32, u32,
                                         ctypes.c_float, ctypes.c_float, u32, u32, vp, vp, vp]
    L.bang_build_pq.argtypes = [i32, vp, i32, u64, u32, u32, vp, u64, vp, u32, vp, vp, vp]
    L.bang_autotune.argtypes = [vp, vp, u32, u32, u32, vp, ctypes.POINTER(bang_autotune_opts),
                                ctypes.POINTER(bang_autotune_result), vp]
    L.bang_probe_host_link.argtypes = [i32, u64, u32, ctypes.POINTER(bang_link_probe)]
    L.bang_probe_host_link.restype = i32
    L.bang_host_alloc.argtypes = [u64, ctypes.POINTER(ctypes.c_void_p)]
    L.bang_host_alloc.restype = i32
    L.bang_host_free.argtypes = [vp]
    L.bang_host_free.restype = i32
    L.bang_last_error.restype = ctypes.c_char_p
    for f in ("bang_create", "bang_load_pq", "bang_register_graph", "bang_register_vectors",
              "bang_search", "bang_destroy", "bang_set_placement", "bang_search_batched",
              "bang_search_batched_noalloc", "bang_index_info", "bang_server_start", "bang_pq_tables",
              "bang_server_submit", "bang_server_wait", "bang_server_stop", "bang_autotune",
              "bang_build_cluster_graph", "bang_build_pq", "bang_ground_truth",
              "bang_build_shard_graph"):
        getattr(L, f).restype = i32
    _lib = L
    return L


def lib():
    return _load()


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to the library must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    raise TypeError("unsupported buffer type %r" % type(x))


def _check(rc):
    if rc != BANG_OK:
        raise BangError(rc, lib().bang_last_error().decode(errors="replace"))
    return rc


def bang_last_error():
    return lib().bang_last_error().decode(errors="replace")


def bang_create(device=0):
    h = ctypes.c_void_p()
    _check(lib().bang_create(device, ctypes.byref(h)))
    return h


def bang_load_pq(ix, d, M, codebook, codes, n):
    return _check(lib().bang_load_pq(ix, d, M, _ptr(codebook), _ptr(codes), n))


def bang_register_graph(ix, adj, R, medoid):
    return _check(lib().bang_register_graph(ix, _ptr(adj), R, medoid))


def bang_register_vectors(ix, base, dtype):
    return _check(lib().bang_register_vectors(ix, _ptr(base), dtype))


PHASES = ("table", "select", "filter", "distance", "next", "rerank", "merge", "merge_rank",
          "merge_shift", "total")


BANG_MODE_PQ_F32, BANG_MODE_PQ_BF16, BANG_MODE_EXACT, BANG_MODE_PQ_Q8 = 0, 1, 2, 3
BANG_GRAPH_IN_HBM, BANG_VECTORS_IN_HBM, BANG_GRAPH_PACKED, BANG_NEIGHBOR_CODES = 1, 2, 4, 8
BANG_NODE_RECORDS = 16


def make_params(bloom_log2=0, iter_cap=0, out_iters=None, out_status=None, out_ndist=None,
                trace=None, trace_cap=0, out_phase_cycles=None, mode=0, grid_mult=0,
                table_source=0, prefetch_depth=0, early_codes=0, rerank=0, smem_carveout=0,
                table_subspaces=0):
    return bang_search_params(bloom_log2, iter_cap, _ptr(out_iters), _ptr(out_status),
                              _ptr(out_ndist), _ptr(trace), trace_cap, _ptr(out_phase_cycles), mode,
                              grid_mult, table_source, prefetch_depth, early_codes, rerank,
                              smem_carveout, table_subspaces)


def bang_search(ix, queries, nq, k, L, params, out_ids, out_dist, stream=None):
    p = ctypes.byref(params) if params is not None else None
    s = ctypes.c_void_p(stream) if isinstance(stream, int) else stream
    return _check(lib().bang_search(ix, _ptr(queries), nq, k, L, p, _ptr(out_ids),
                                    _ptr(out_dist), s))


def bang_search_batched(ix, queries, nq, k_per_q, L_per_q, k_max, L_max, params, out_ids,
                        out_dist, stream=None):
    p = ctypes.byref(params) if params is not None else None
    s = ctypes.c_void_p(stream) if isinstance(stream, int) else stream
    return _check(lib().bang_search_batched(ix, _ptr(queries), nq, _ptr(k_per_q), _ptr(L_per_q),
                                            k_max, L_max, p, _ptr(out_ids), _ptr(out_dist), s))


def bang_search_batched_noalloc(ix, queries, nq, k_per_q, L_per_q, k_max, L_max, params, out_ids,
                                out_dist, stream=None):
    """bang_search_batched without any allocation (device buffers only); see
    include/bang.h for who needs it and its limits."""
    p = ctypes.byref(params) if params is not None else None
    s = ctypes.c_void_p(stream) if isinstance(stream, int) else stream
    return _check(lib().bang_search_batched_noalloc(ix, _ptr(queries), nq, _ptr(k_per_q),
                                                    _ptr(L_per_q), k_max, L_max, p, _ptr(out_ids),
                                                    _ptr(out_dist), s))


def host_empty(shape, dtype):
    """A numpy array in memory from bang_host_alloc (advised for transparent
    huge pages, zero-filled), for the graph and vectors an index reads in
    place from host memory; the memory is unmapped when the array and every
    view of it are gone (destroy indexes that registered it first)."""
    import weakref
    dtype = np.dtype(dtype)
    nbytes = max(1, int(np.prod(shape)) * dtype.itemsize)
    ptr = ctypes.c_void_p()
    _check(lib().bang_host_alloc(nbytes, ctypes.byref(ptr)))
    holder = (ctypes.c_uint8 * nbytes).from_address(ptr.value)
    fin = weakref.finalize(holder, lib().bang_host_free, ctypes.c_void_p(ptr.value))
    fin.atexit = False                 # at exit the process's mappings go anyway
    return np.frombuffer(holder, np.uint8)[:int(np.prod(shape)) * dtype.itemsize].view(dtype).reshape(shape)


def bang_pq_tables(ix, queries, nq, out, out_bf16=0, stream=None):
    s = ctypes.c_void_p(stream) if isinstance(stream, int) else stream
    return _check(lib().bang_pq_tables(ix, _ptr(queries), nq, _ptr(out), out_bf16, s))


def bang_autotune(ix, queries, nq, k, L, truth=None, modes=0, bloom_min=0, bloom_max=0,
                  try_tensor_tables=1, batched=0, reps=0, target_recall=0.0, recall_tolerance=0.0,
                  cache_path=None, try_packed_graph=0, try_neighbor_codes=0, try_prefetch_depth=0,
                  try_node_records=0, try_structure=0, stream=None):
    """Returns the chosen settings as a dict (fields of bang_autotune_result)."""
    s = ctypes.c_void_p(stream) if isinstance(stream, int) else stream
    o = bang_autotune_opts(modes, bloom_min, bloom_max, try_tensor_tables, batched, reps,
                           target_recall, recall_tolerance,
                           cache_path.encode() if cache_path else None, try_packed_graph,
                           try_neighbor_codes, try_prefetch_depth, try_node_records, try_structure)
    t = None if truth is None else np.ascontiguousarray(truth, np.uint32)
    r = bang_autotune_result()
    _check(lib().bang_autotune(ix, _ptr(queries), nq, k, L, _ptr(t), ctypes.byref(o),
                               ctypes.byref(r), s))
    return {f: getattr(r, f) for f, _ in bang_autotune_result._fields_}


def bang_build_cluster_graph(base, members, gstart, medoids, R, alpha, nx=0, xclu=None, nh=0,
                             hclu=None, adj=None, device=0, stream=None):
    """Clustered graph built on the GPU; returns adj (n x R uint32, numpy
    unless a device tensor is passed)."""
    n, d = base.shape
    dt = _DTYPES[np.dtype(str(base.dtype).replace("torch.", ""))]
    members = np.ascontiguousarray(members, np.uint32)
    gstart = np.ascontiguousarray(gstart, np.uint64)
    medoids = np.ascontiguousarray(medoids, np.uint32)
    xclu = np.ascontiguousarray(xclu if xclu is not None else np.zeros((n, 0)), np.uint32)
    hclu = np.ascontiguousarray(hclu if hclu is not None else np.zeros((len(medoids), 0)), np.uint32)
    if adj is None:
        adj = np.zeros((n, R), np.uint32)
    s = ctypes.c_void_p(stream) if isinstance(stream, int) else stream
    _check(lib().bang_build_cluster_graph(device, _ptr(base), dt, n, d, _ptr(members), _ptr(gstart),
                                          len(medoids), _ptr(medoids), R, alpha, nx, _ptr(xclu), nh,
                                          _ptr(hclu), _ptr(adj), s))
    return adj


def bang_build_shard_graph(base, centres, ell, R, Lb, alpha, batch_frac=0.02, log2z=16, iter_cap=0,
                           adj=None, device=0, stream=None):
    """Overlapping-shard graph built on the GPU (§2.2); returns (adj n x R
    uint32, numpy unless a device tensor is passed, shard assignment n x ell)."""
    n, d = base.shape
    dt = _DTYPES[np.dtype(str(base.dtype).replace("torch.", ""))]
    centres = np.ascontiguousarray(centres, np.float32)
    if adj is None:
        adj = np.zeros((n, R), np.uint32)
    sh = np.zeros((n, ell), np.uint32)
    s = ctypes.c_void_p(stream) if isinstance(stream, int) else stream
    _check(lib().bang_build_shard_graph(device, _ptr(base), dt, n, d, _ptr(centres),
                                        centres.shape[0], ell, R, Lb, alpha, batch_frac, log2z,
                                        iter_cap, _ptr(adj), _ptr(sh), s))
    return adj, sh


def bang_build_pq(base, M, sample, init, iters=10, device=0, stream=None):
    """PQ codebook (256*d float32) and codes (n x M uint8) built on the GPU."""
    n, d = base.shape
    dt = _DTYPES[np.dtype(str(base.dtype).replace("torch.", ""))]
    sample = np.ascontiguousarray(sample, np.uint64)
    init = np.ascontiguousarray(init, np.uint64)
    cb = np.zeros(256 * d, np.float32)
    codes = np.zeros((n, M), np.uint8)
    s = ctypes.c_void_p(stream) if isinstance(stream, int) else stream
    _check(lib().bang_build_pq(device, _ptr(base), dt, n, d, M, _ptr(sample), len(sample),
                               _ptr(init), iters, _ptr(cb), _ptr(codes), s))
    return cb, codes


def bang_ground_truth(base, queries, k, device=0, stream=None):
    """Exact k-NN on the GPU: (ids uint32 nq x k, distances float64 nq x k)."""
    n, d = base.shape
    nq = queries.shape[0]
    dt = _DTYPES[np.dtype(str(base.dtype).replace("torch.", ""))]
    ids = np.zeros((nq, k), np.uint32)
    dist = np.zeros((nq, k), np.float64)
    s = ctypes.c_void_p(stream) if isinstance(stream, int) else stream
    _check(lib().bang_ground_truth(device, _ptr(base), _ptr(queries), dt, n, nq, d, k, _ptr(ids),
                                   _ptr(dist), s))
    return ids, dist


def bang_set_placement(ix, flags):
    return _check(lib().bang_set_placement(ix, flags))


def bang_destroy(ix):
    return _check(lib().bang_destroy(ix))


_DTYPES = {np.dtype(np.uint8): BANG_U8, np.dtype(np.int8): BANG_I8,
           np.dtype(np.float32): BANG_F32}


class Index:
    """Owns a bang_index and the host arrays it reads in place."""

    def __init__(self, base, codebook, codes, adj, medoid, M, device=0):
        self.base = np.ascontiguousarray(base)
        self.n, self.d = self.base.shape
        self.M = M
        self._codebook = np.ascontiguousarray(codebook, np.float32)
        self._codes = np.ascontiguousarray(codes, np.uint8).reshape(self.n, M)
        self.adj = np.ascontiguousarray(adj, np.uint32).reshape(self.n, -1)
        self.R = self.adj.shape[1]
        self.medoid = int(medoid)
        self.dtype = _DTYPES[self.base.dtype]
        self.h = bang_create(device)
        bang_load_pq(self.h, self.d, M, self._codebook, self._codes, self.n)
        bang_register_graph(self.h, self.adj, self.R, self.medoid)
        bang_register_vectors(self.h, self.base, self.dtype)

    def search_batched(self, queries, k_per_q, L_per_q, k_max, L_max, out_ids, out_dist,
                       params=None, stream=None):
        nq = queries.shape[0]
        return bang_search_batched(self.h, queries, nq, k_per_q, L_per_q, k_max, L_max, params,
                                   out_ids, out_dist, stream)

    def set_placement(self, flags):
        return bang_set_placement(self.h, flags)

    def autotune(self, queries, k, L, truth=None, stream=None, **opts):
        """bang_autotune over these queries; returns the chosen settings."""
        return bang_autotune(self.h, queries, queries.shape[0], k, L, truth=truth, stream=stream,
                             **opts)

    def search(self, queries, k, L, out_ids, out_dist, params=None, stream=None):
        nq = queries.shape[0]
        return bang_search(self.h, queries, nq, k, L, params, out_ids, out_dist, stream)

    def close(self):
        if self.h is not None:
            bang_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server over an Index (see bang_server_* in bang.h).
    submit() copies host queries and returns a ticket; wait() returns the
    request's ids, distances (nq x k_max) and latency in milliseconds."""

    def __init__(self, index, k_max, L_max, max_batch=1024, streams=8, mode=0, bloom_log2=0,
                 mem_bytes=0, early_codes=0):
        self.index = index
        self.k_max = k_max
        cfg = bang_server_config(k_max, L_max, max_batch, streams, mode, bloom_log2, mem_bytes,
                                 early_codes)
        h = ctypes.c_void_p()
        _check(lib().bang_server_start(index.h, ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h

    def submit(self, queries, k_per_q, L_per_q):
        q = np.ascontiguousarray(queries)
        k = np.ascontiguousarray(k_per_q, np.uint32)
        L = np.ascontiguousarray(L_per_q, np.uint32)
        t = ctypes.c_uint64()
        _check(lib().bang_server_submit(self.h, _ptr(q), q.shape[0], _ptr(k), _ptr(L),
                                        ctypes.byref(t)))
        return t.value, q.shape[0]

    def wait(self, ticket, timeout_ms=-1):
        t, nq = ticket
        ids = np.zeros((nq, self.k_max), np.uint32)
        dist = np.zeros((nq, self.k_max), np.float32)
        lat = ctypes.c_double()
        _check(lib().bang_server_wait(self.h, t, timeout_ms, _ptr(ids), _ptr(dist),
                                      ctypes.byref(lat)))
        return ids, dist, lat.value

    def stop(self):
        if self.h is not None:
            _check(lib().bang_server_stop(self.h))
            self.h = None
