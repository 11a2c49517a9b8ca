"""Seeded test cases shared by the parity tests: data from the workload
generator, index pieces from the oracle (configuration 1) or the workload
generator (clustered configurations).  Cached under the workload cache."""
import hashlib
import os

import numpy as np

import oracle
import workload


def _cache(name, fn):
    path = os.path.join(workload.cache_dir(), name + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        return {f: z[f] for f in z.files}
    out = fn()
    np.savez(path + ".tmp.npz", **out)
    os.replace(path + ".tmp.npz", path)
    return out


def config1(n=None, nq=None):
    """Configuration 1: f32 d=128 mixture, PQ M=32 trained by the oracle
    (10 Lloyd iterations), Vamana R=32, L_build=64, alpha=1.2 built by the
    oracle from a seeded random initial graph, medoid entry."""
    c = workload.CONFIGS[1]
    n = n or c["n"]
    nq = nq or c["nq"]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "bang_oracle.c")).read()
    key = hashlib.sha1((src + repr((n, nq, sorted(c.items())))).encode()).hexdigest()[:12]

    def make():
        w = workload.make_data(1, n=n, nq=nq)
        X = w["base"]
        rng = np.random.default_rng(3001)
        init = np.stack([rng.choice(n, 256, replace=False) for _ in range(c["M"])])
        cb = oracle.pq_train(X, c["M"], np.arange(n), init, 10)
        codes = oracle.pq_encode(X, c["M"], cb)
        med = oracle.medoid(X)
        g = np.random.default_rng(4001)
        R = c["R"]
        init_adj = np.empty((n, R), np.uint32)
        for i in range(n):
            cand = g.choice(n - 1, R, replace=False)
            init_adj[i] = cand + (cand >= i)
        order = g.permutation(n).astype(np.uint32)
        adj = oracle.vamana_build(X, R, c["Lb"], c["alpha"], med, init_adj, order)
        gt, gtd = oracle.bruteforce_knn(X, w["queries"], 100)
        return dict(base=X, queries=w["queries"], codebook=cb, codes=codes, adj=adj,
                    medoid=np.int64(med), gt_ids=gt, gt_dist=gtd)

    out = _cache("cfg1_%s" % key, make)
    out["medoid"] = int(out["medoid"])
    out["M"] = c["M"]
    return out


def clustered(n, nq, ncomp, dtype="u8", d=128, M=32, R=64, **over):
    """A clustered workload (configuration 2's recipe) of a chosen size."""
    w = workload.clustered_workload(2, n=n, nq=nq, ncomp=ncomp, dtype=dtype, d=d, M=M, R=R,
                                    **over)
    w["M"] = M
    return w
