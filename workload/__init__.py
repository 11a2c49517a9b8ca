"""Seeded synthetic workloads for the BANG search path (arXiv 2401.11324).

The paper measures on SIFT-1B (uint8, d=128), Deep-1B (float, d=96),
MSSPACEV-1B (int8, d=100) and Text-to-Image-1B (§6.2), searched through a
Vamana index and PQ codes built beforehand by DiskANN (§1, §6.3).  None of
those files exist here, so this module stands in for them: seeded Gaussian
mixtures with the datasets' element types and dimensions, the index the
search consumes (PQ codebooks and codes, graph, medoid) and exact ground
truth.  It holds none of the search's arithmetic; the oracle and the CUDA
path both read what it writes.

Configurations (the recipe of each is in ``CONFIGS``):
  1  n=10,000 f32 d=128, 16 components, centres ~N(0, 4I), unit variance,
     100 queries; PQ M=32; Vamana R=32 (built by the oracle in the tests).
  2  n=1,000,000 u8 d=128, 256 components, centres ~U[0,255]^d; each component
     low-rank like SIFT descriptors: x = c + A z + 4 e, A (d x 12) with
     N(0, 20^2/12) entries, z ~ N(0, I_12), e ~ N(0, I_d); rounded and
     clipped to 0..255; 10,000 queries; PQ M=32; clustered graph R=64.
  3  n=10,000,000 f32 d=96, 1,024 components, centres ~N(0, I) scaled to unit
     length, x = normalise(c + 0.1 z); 10,000 queries; PQ M=48; clustered
     graph with 64 in-cluster neighbours and 4 medoid links (R=68).
  4  n=100,000,000 int8 d=100, 4,096 components, centres ~U[-100,100]^d,
     low-rank components as in 2 (A: d x 12 with N(0, 16^2/12) entries, noise
     4), rounded and clipped to -128..127; 10,000 queries; PQ M=50; clustered
     graph R=64 (built on the GPU: the host cores would take days).
  5  n=200,000,000 u8 d=128 (the largest size the GPU machine's host memory holds
     with room for the index; the configuration names 1B), 16,384 low-rank
     components as in 2; 10,000 queries; PQ M=32; overlapping-shard graph R=64.
Configurations 4 and 5 come from the counter-based generator (large_data)
and take the overlapping-shard graph (32 shards, each point in its 2 nearest,
GreedySearch worklist 64, alpha 1.2) built on the GPU.
Seeds: data 1000+cfg, queries 2000+cfg, PQ 3000+cfg, graph 4000+cfg.
"""
import ctypes
import hashlib
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "indexgen.c")
_LIB = os.path.join(_HERE, "libwlgen.so")
NONE = 0xFFFFFFFF

CONFIGS = {
    1: dict(n=10_000, nq=100, d=128, dtype="f32", ncomp=16, centre="normal", centre_scale=2.0,
            sigma=1.0, M=32, R=32, Lb=64, alpha=1.2, k=10, L=64),
    2: dict(n=1_000_000, nq=10_000, d=128, dtype="u8", ncomp=256, centre="uniform255",
            centre_scale=None, sigma=20.0, rank=12, noise=4.0, M=32, R=64, alpha=1.2, nx=4,
            nh=32, k=10, L=64),
    # precision form: unit-normalised mixture under L2; 64 in-cluster
    # neighbours plus 4 links to other clusters' medoids (degree <= 68)
    3: dict(n=10_000_000, nq=10_000, d=96, dtype="f32", ncomp=1024, centre="unitnormal",
            centre_scale=None, sigma=0.1, normalise=True, M=48, R=68, alpha=1.2, nx=4, nh=32,
            k=10, L=128),
    # batched form: int8 mixture clipped to -128..127; 60 in-cluster neighbours
    # plus 4 links to other clusters' medoids (R = 64), half to nearby
    # clusters and half to random ones
    4: dict(n=100_000_000, nq=10_000, d=100, dtype="i8", ncomp=4096, centre="uniform100",
            centre_scale=None, sigma=16.0, rank=12, noise=4.0, M=50, R=64, alpha=1.2, nx=4,
            nh=32, k=10, L=128, links="mixed", shards=32, ell=2, Lb=64, batch_frac=0.02,
            bloom_build=16),
    # serving at the largest size the GPU machine's host memory holds with room
    # for the index (200M of the 1B points; SIFT's type and dimension),
    # overlapping-shard graph (§2.2), built on the GPU
    5: dict(n=200_000_000, nq=10_000, d=128, dtype="u8", ncomp=16384, centre="uniform255",
            centre_scale=None, sigma=20.0, rank=12, noise=4.0, M=32, R=64, alpha=1.2, k=10,
            L=64, shards=32, ell=2, Lb=64, batch_frac=0.02, bloom_build=16),
}

_DTN = {"u8": np.uint8, "i8": np.int8, "f32": np.float32}
_DTC = {"u8": 0, "i8": 1, "f32": 2}


def build(force=False):
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    subprocess.check_call(["gcc", "-std=c99", "-O3", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fopenmp", "-Wall", "-o", _LIB + ".tmp", _SRC, "-lm"], cwd=_HERE)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, u32, u64, i32, f32 = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                  ctypes.c_float)
        L.wl_pq_train.argtypes = [vp, u64, u32, u32, vp, vp, u32, vp]
        L.wl_pq_encode.argtypes = [vp, i32, u64, u32, u32, vp, vp, vp]
        L.wl_medoids.argtypes = [vp, i32, u32, vp, vp, u32, vp]
        L.wl_cluster_graph.argtypes = [vp, i32, u32, u64, vp, vp, u32, vp, u32, f32, u32, vp, u32,
                                       vp, vp]
        L.wl_cluster_graph.restype = i32
        L.wl_bruteforce.argtypes = [vp, vp, i32, u64, u32, u32, u32, vp, vp]
        L.wl_max_threads.restype = i32
        L.wl_mixture.argtypes = [vp, i32, u64, u32, vp, u32, vp, u32, f32, u64, vp]
        L.wl_mixture.restype = i32
        L.wl_scale_index.argtypes = [i32, u64, u32, u32, u32, u32, u32, u32, u64, vp, vp, vp, vp, vp]
        L.wl_scale_index.restype = i32
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def chunk_offsets(d, M):
    """Contiguous PQ subspaces; the first d % M take one extra dimension."""
    base, extra = divmod(d, M)
    return np.concatenate([[0], np.cumsum([base + (s < extra) for s in range(M)])]).astype(
        np.uint32)


def _mixture(rng, n, d, centres, sigma, dtype, factors=None, noise=0.0, chunk=131072,
             normalise=False):
    """Equal-weight Gaussian mixture; integer types are rounded and clipped.
    Isotropic components (sigma per dimension), or, with ``factors``
    (ncomp x d x r), low-rank components x = c + A z + noise*e with
    z ~ N(0, I_r) and e ~ N(0, I_d).  ``normalise`` scales every point to
    unit length."""
    lab = rng.integers(0, centres.shape[0], size=n).astype(np.uint32)
    out = np.empty((n, d), dtype=_DTN[dtype])
    for i in range(0, n, chunk):
        j = min(n, i + chunk)
        if factors is None:
            x = centres[lab[i:j]] + sigma * rng.standard_normal((j - i, d), dtype=np.float32)
        else:
            z = rng.standard_normal((j - i, factors.shape[2]), dtype=np.float32)
            x = centres[lab[i:j]] + np.einsum("ndr,nr->nd", factors[lab[i:j]], z)
            x += noise * rng.standard_normal((j - i, d), dtype=np.float32)
        if normalise:
            x /= np.maximum(np.linalg.norm(x, axis=1, keepdims=True), np.float32(1e-30))
        if dtype == "u8":
            out[i:j] = np.clip(np.rint(x), 0, 255).astype(np.uint8)
        elif dtype == "i8":
            out[i:j] = np.clip(np.rint(x), -128, 127).astype(np.int8)
        else:
            out[i:j] = x.astype(np.float32)
    return out, lab


def _centres(rng, c):
    if c["centre"] == "normal":
        cen = rng.standard_normal((c["ncomp"], c["d"]), dtype=np.float32) * c["centre_scale"]
    elif c["centre"] == "uniform255":
        cen = rng.uniform(0.0, 255.0, size=(c["ncomp"], c["d"])).astype(np.float32)
    elif c["centre"] == "unitnormal":
        cen = rng.standard_normal((c["ncomp"], c["d"]), dtype=np.float32)
        cen /= np.linalg.norm(cen, axis=1, keepdims=True)
    elif c["centre"] == "uniform100":
        cen = rng.uniform(-100.0, 100.0, size=(c["ncomp"], c["d"])).astype(np.float32)
    else:
        raise ValueError(c["centre"])
    return cen


def make_data(cfg, n=None, nq=None, ncomp=None, **over):
    """Base vectors, their mixture labels and the queries of a configuration
    (optionally shrunk: n points, nq queries, ncomp components)."""
    c = dict(CONFIGS[cfg])
    if n is not None:
        c["n"] = n
    if nq is not None:
        c["nq"] = nq
    if ncomp is not None:
        c["ncomp"] = ncomp
    c.update(over)
    rng = np.random.default_rng(1000 + cfg)
    cen = _centres(rng, c)
    fac = None
    if c.get("rank", 0):
        fac = (rng.standard_normal((c["ncomp"], c["d"], c["rank"]), dtype=np.float32) *
               np.float32(c["sigma"] / np.sqrt(c["rank"])))
    nrm = c.get("normalise", False)
    base, lab = _mixture(rng, c["n"], c["d"], cen, c["sigma"], c["dtype"], fac, c.get("noise", 0),
                         normalise=nrm)
    queries, _ = _mixture(np.random.default_rng(2000 + cfg), c["nq"], c["d"], cen, c["sigma"],
                          c["dtype"], fac, c.get("noise", 0), normalise=nrm)
    return dict(cfg=cfg, params=c, base=base, labels=lab, queries=queries)


def pq_random_choices(cfg, n, M, train_n):
    """The PQ training sample and the initial centroids (indices into the
    sample), drawn with the PQ seed."""
    rng = np.random.default_rng(3000 + cfg)
    ns = min(n, train_n)
    sample = np.sort(rng.choice(n, size=ns, replace=False)).astype(np.uint64)
    init = np.stack([rng.choice(ns, size=256, replace=False) for _ in range(M)]).astype(np.uint64)
    return sample, init


def build_pq(base, M, sample, init, iters=10):
    d = base.shape[1]
    off = chunk_offsets(d, M)
    Xs = np.ascontiguousarray(base[sample.astype(np.int64)], dtype=np.float32)
    cb = np.zeros(256 * d, np.float32)
    init = np.ascontiguousarray(init, np.uint64)
    lib().wl_pq_train(_p(Xs), Xs.shape[0], d, M, _p(off), _p(init), iters, _p(cb))
    codes = np.zeros((base.shape[0], M), np.uint8)
    lib().wl_pq_encode(_p(base), _DTC[_dtname(base)], base.shape[0], d, M, _p(off), _p(cb),
                       _p(codes))
    return cb, codes


def _dtname(a):
    return {np.dtype(np.uint8): "u8", np.dtype(np.int8): "i8", np.dtype(np.float32): "f32"}[a.dtype]


def medoids_of_groups(base, labels, ng):
    order = np.argsort(labels, kind="stable").astype(np.uint32)
    counts = np.bincount(labels, minlength=ng)
    gstart = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64)
    out = np.zeros(ng, np.uint32)
    lib().wl_medoids(_p(base), _DTC[_dtname(base)], base.shape[1], _p(order), _p(gstart), ng,
                     _p(out))
    return order, gstart, out


def graph_inputs(cfg, base, labels, ng, nx, nh):
    """Inputs of the clustered construction: members grouped by cluster,
    cluster offsets, cluster medoids, and the clusters whose medoids each
    point (nx) and each cluster medoid (nh) links to, drawn with the graph
    seed."""
    n = base.shape[0]
    order, gstart, meds = medoids_of_groups(base, labels, ng)
    rng = np.random.default_rng(4000 + cfg)
    own = labels.astype(np.int64)
    if CONFIGS.get(cfg, {}).get("links") == "mixed":
        # half of the links go to clusters whose medoids are near this
        # cluster's (each point: nx/2 of the nx nearest; each medoid: its
        # nh/2 nearest), half to random other clusters, so that greedy routing
        # has both long jumps and local steps.  Squared distances between
        # integer medoids are exact in FP64 (integers below 2^53), so the
        # order is the same on every machine.
        mv = base[meds.astype(np.int64)].astype(np.float64)
        g = mv @ mv.T
        sq = np.diag(g).copy()
        dm = sq[:, None] + sq[None, :] - 2.0 * g
        np.fill_diagonal(dm, np.inf)
        near = np.argsort(dm, axis=1, kind="stable")
        xn = nx // 2
        xclu = np.concatenate([
            near[own[:, None], rng.integers(0, min(nx, ng - 1), size=(n, xn))],
            (own[:, None] + 1 + rng.integers(0, ng - 1, size=(n, nx - xn))) % ng], axis=1)
        if nh:
            hn = min(nh // 2, ng - 1)
            rows = []
            for c in range(ng):
                others = np.setdiff1d(np.arange(ng), np.concatenate([[c], near[c, :hn]]))
                k = min(nh - hn, len(others))
                rows.append(np.concatenate([near[c, :hn], rng.choice(others, size=k, replace=False)]))
            hclu = np.stack(rows)
        else:
            hclu = np.zeros((ng, 0), np.int64)
    else:
        xclu = (own[:, None] + 1 + rng.integers(0, ng - 1, size=(n, nx))) % ng
        hclu = np.stack([(g + 1 + rng.choice(ng - 1, size=min(nh, ng - 1), replace=False)) % ng
                         for g in range(ng)]) if nh else np.zeros((ng, 0), np.int64)
    return dict(members=order, gstart=gstart, medoids=meds,
                xclu=np.ascontiguousarray(xclu, np.uint32), hclu=np.ascontiguousarray(hclu, np.uint32))


def build_cluster_graph(cfg, base, labels, ng, R, alpha, nx, nh):
    """Clustered graph (per-cluster exact candidates -> RobustPrune -> reverse
    edges; nx links per point and nh links per cluster medoid to other
    clusters' medoids, those clusters drawn with the graph seed)."""
    n, d = base.shape
    gi = graph_inputs(cfg, base, labels, ng, nx, nh)
    order, gstart, meds, xclu, hclu = gi["members"], gi["gstart"], gi["medoids"], gi["xclu"], gi["hclu"]
    nh_eff = hclu.shape[1]
    adj = np.zeros((n, R), np.uint32)
    rc = lib().wl_cluster_graph(_p(base), _DTC[_dtname(base)], d, n, _p(order), _p(gstart), ng,
                                _p(meds), R, alpha, nx, _p(xclu), nh_eff, _p(hclu), _p(adj))
    if rc != 0:
        raise MemoryError("cluster graph build failed (%d)" % rc)
    _, _, gmed = medoids_of_groups(base, np.zeros(n, np.uint32), 1)
    return adj, int(gmed[0])


def ground_truth(base, queries, k):
    nq = queries.shape[0]
    ids = np.zeros((nq, k), np.uint32)
    dist = np.zeros((nq, k), np.float64)
    queries = np.ascontiguousarray(queries)
    lib().wl_bruteforce(_p(base), _p(queries), _DTC[_dtname(base)],
                        base.shape[0], nq, base.shape[1], k, _p(ids), _p(dist))
    return ids, dist


def aligned_empty(shape, dtype, align=4096):
    """Uninitialised array whose data starts on an `align`-byte boundary."""
    dtype = np.dtype(dtype)
    nbytes = int(np.prod(shape)) * dtype.itemsize
    buf = np.empty(nbytes + align, np.uint8)
    start = (-buf.ctypes.data) % align
    return buf[start:start + nbytes].view(dtype).reshape(shape)


def scale_index(n, d, dtype, M, R, nx=4, ng=1024, nq=1000, seed=5):
    """An index of the full configuration sizes for parity checks, built
    without nearest-neighbour work (wl_scale_index): cluster-local graph rows
    plus links to other clusters, uniform vectors and codes.  Arrays are
    page-aligned, so the search library reads them in place."""
    base = aligned_empty((n, d), _DTN[dtype])
    queries = aligned_empty((nq, d), _DTN[dtype])
    codebook = np.zeros(256 * d, np.float32)
    codes = aligned_empty((n, M), np.uint8)
    adj = aligned_empty((n, R), np.uint32)
    rc = lib().wl_scale_index(_DTC[dtype], n, d, M, R, nx, ng, nq, seed, _p(base), _p(queries),
                              _p(codebook), _p(codes), _p(adj))
    if rc != 0:
        raise ValueError("scale_index: clusters too small for R")
    return dict(base=base, queries=queries, codebook=codebook, codes=codes, adj=adj, medoid=0, M=M)


def clustered_data(cfg=2, n=None, nq=None, ncomp=None, k=100, train_n=256_000, verbose=False,
                   **over):
    """Data, exact ground truth and the inputs of the index construction
    (PQ sample and initial centroids as rows of base; clustered-graph inputs)
    of a clustered configuration, for building the index elsewhere.  Cached
    on disk by its parameters."""
    c = dict(CONFIGS[cfg])
    c.update(over)
    n = n or c["n"]
    nq = nq or c["nq"]
    ncomp = ncomp or c["ncomp"]
    key = hashlib.sha1(repr(("data", cfg, n, nq, ncomp, k, train_n, sorted(c.items()),
                             os.path.getmtime(_SRC) // 1, 1)).encode()).hexdigest()[:16]
    path = os.path.join(cache_dir(), "cfg%d_data_%s.npz" % (cfg, key))
    if os.path.exists(path):
        z = np.load(path)
        out = {f: z[f] for f in z.files}
        out["medoid"] = int(out["medoid"])
        out["params"] = dict(c, n=n, nq=nq, ncomp=ncomp)
        return out
    t0 = time.time()
    w = make_data(cfg, n=n, nq=nq, ncomp=ncomp, **over)
    sample, init = pq_random_choices(cfg, n, c["M"], train_n)
    gi = graph_inputs(cfg, w["base"], w["labels"], ncomp, c["nx"], c["nh"])
    _, _, gmed = medoids_of_groups(w["base"], np.zeros(n, np.uint32), 1)
    t1 = time.time()
    if k > 0:
        gt_ids, gt_dist = ground_truth(w["base"], w["queries"], k)
    else:                                       # the caller computes the ground truth
        gt_ids, gt_dist = np.zeros((nq, 0), np.uint32), np.zeros((nq, 0))
    t2 = time.time()
    if verbose:
        print("data cfg%d n=%d: data %.1fs gt %.1fs (threads %d)" % (
            cfg, n, t1 - t0, t2 - t1, lib().wl_max_threads()), flush=True)
    out = dict(base=w["base"], queries=w["queries"], labels=w["labels"], gt_ids=gt_ids,
               gt_dist=gt_dist, pq_sample=sample, pq_init=sample[init.astype(np.int64)],
               members=gi["members"], gstart=gi["gstart"], medoids=gi["medoids"], xclu=gi["xclu"],
               hclu=gi["hclu"], medoid=np.int64(gmed[0]))
    if w["base"].nbytes <= (2 << 30):          # larger datasets are regenerated, not cached
        tmp = path + ".tmp.npz"
        np.savez(tmp, **out)
        os.replace(tmp, path)
    out["medoid"] = int(gmed[0])
    out["params"] = dict(c, n=n, nq=nq, ncomp=ncomp)
    return out


def large_data(cfg, n=None, nq=None, ncomp=None, train_n=256_000, verbose=False, alloc=None, **over):
    """Data of a large configuration (4 or 5) from the counter-based generator
    (wl_mixture: same bytes for any thread count and on x86 and Arm hosts),
    with the inputs of its index build: the PQ training sample and initial
    centroids, the shard centres (seeded data points) and the global medoid.
    The index itself (PQ codes, overlapping-shard graph) and the ground truth
    are built by the caller (on the GPU).  `alloc(shape, dtype)` allocates the
    base vectors (default: page-aligned numpy memory)."""
    c = dict(CONFIGS[cfg])
    c.update(over)
    n = n or c["n"]
    nq = nq or c["nq"]
    ncomp = ncomp or c["ncomp"]
    c.update(n=n, nq=nq, ncomp=ncomp)
    t0 = time.time()
    rng = np.random.default_rng(1000 + cfg)
    cen = np.ascontiguousarray(_centres(rng, c), np.float32)
    fac = rng.standard_normal((ncomp, c["d"], c["rank"]), dtype=np.float32) * np.float32(
        c["sigma"] / np.sqrt(c["rank"]))
    fac = np.ascontiguousarray(fac.transpose(0, 2, 1))         # rank-major per component
    base = (alloc or aligned_empty)((n, c["d"]), _DTN[c["dtype"]])
    queries = aligned_empty((nq, c["d"]), _DTN[c["dtype"]])
    for arr, rows, seed in ((base, n, 1000 + cfg), (queries, nq, 2000 + cfg)):
        rc = lib().wl_mixture(_p(arr), _DTC[c["dtype"]], rows, c["d"], _p(cen), ncomp, _p(fac),
                              c["rank"], c["noise"], seed, None)
        if rc != 0:
            raise ValueError("wl_mixture rejected its arguments")
    t1 = time.time()
    sample, init = pq_random_choices(cfg, n, c["M"], train_n)
    srng = np.random.default_rng(4000 + cfg)
    shard_ids = np.sort(srng.choice(n, size=c["shards"], replace=False))
    out = np.zeros(1, np.uint32)
    everyone = np.arange(n, dtype=np.uint32)
    bounds = np.array([0, n], np.uint64)
    lib().wl_medoids(_p(base), _DTC[c["dtype"]], c["d"], _p(everyone), _p(bounds), 1, _p(out))
    del everyone
    t2 = time.time()
    if verbose:
        print("data cfg%d n=%d: generator %.1fs, build inputs and medoid %.1fs (threads %d)" % (
            cfg, n, t1 - t0, t2 - t1, lib().wl_max_threads()), flush=True)
    return dict(base=base, queries=queries, pq_sample=sample,
                pq_init=sample[init.astype(np.int64)],
                shard_centres=np.ascontiguousarray(base[shard_ids], np.float32),
                medoid=int(out[0]), params=c)


def cache_dir():
    d = os.environ.get("BANG_WORKLOAD_CACHE", "/tmp/bang_workload_cache")
    os.makedirs(d, exist_ok=True)
    return d


def clustered_workload(cfg=2, n=None, nq=None, ncomp=None, k=100, train_n=256_000, verbose=False,
                       **over):
    """Data, PQ index, clustered graph and ground truth (k nearest) of a
    clustered configuration, cached on disk by its parameters."""
    c = dict(CONFIGS[cfg])
    c.update(over)
    n = n or c["n"]
    nq = nq or c["nq"]
    ncomp = ncomp or c["ncomp"]
    key = hashlib.sha1(repr((cfg, n, nq, ncomp, k, train_n, sorted(c.items()),
                             os.path.getmtime(_SRC) // 1, 1)).encode()).hexdigest()[:16]
    path = os.path.join(cache_dir(), "cfg%d_%s.npz" % (cfg, key))
    if os.path.exists(path):
        z = np.load(path)
        out = {f: z[f] for f in z.files}
        out["medoid"] = int(out["medoid"])
        out["params"] = dict(c, n=n, nq=nq, ncomp=ncomp)
        return out
    t0 = time.time()
    w = make_data(cfg, n=n, nq=nq, ncomp=ncomp, **over)
    t1 = time.time()
    sample, init = pq_random_choices(cfg, n, c["M"], train_n)
    cb, codes = build_pq(w["base"], c["M"], sample, init)
    t2 = time.time()
    adj, med = build_cluster_graph(cfg, w["base"], w["labels"], ncomp, c["R"], c["alpha"], c["nx"],
                                   c["nh"])
    t3 = time.time()
    gt_ids, gt_dist = ground_truth(w["base"], w["queries"], k)
    t4 = time.time()
    if verbose:
        print("workload cfg%d n=%d: data %.1fs pq %.1fs graph %.1fs gt %.1fs (threads %d)" % (
            cfg, n, t1 - t0, t2 - t1, t3 - t2, t4 - t3, lib().wl_max_threads()), flush=True)
    out = dict(base=w["base"], queries=w["queries"], labels=w["labels"], codebook=cb, codes=codes,
               adj=adj, medoid=np.int64(med), gt_ids=gt_ids, gt_dist=gt_dist)
    tmp = path + ".tmp.npz"
    np.savez(tmp, **out)
    os.replace(tmp, path)
    out["medoid"] = med
    out["params"] = dict(c, n=n, nq=nq, ncomp=ncomp)
    return out
