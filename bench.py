"""Benchmark: queries/s at recall@10 >= 0.9 of the GB300 BANG search path.

Workload: the mid-scale plain-method configuration (n = 1,000,000 uint8
points, d = 128, 256-component mixture, 10,000 queries, PQ M = 32 on the
device, clustered graph R = 64 and full vectors in page-locked host memory,
k = 10).  The worklist size L is the smallest of the sweep
{16, 24, 32, 48, 64, 80, 96, 112, 128, 160, 192, 224, 256, 288, 320, 384, 512, 768, 1024} (values
>= k) whose mean recall@k reaches 0.9 (ground truth: exact k-NN); a step is one
search of the whole batch at that L.  `--k 100` measures 100-recall@100 and
`--M` another PQ code size (the paper's second workload and compression study).

Forms timed: the plain method (FP32 table), the reduced-precision tables
(BF16 per warp or on the tensor cores, 8-bit), and the settings bang_autotune
picks for recall@k >= 0.9 (table precision and source, Bloom filter size,
L); the fastest form reaching the target is the headline.  The In-memory and
Exact-distance variants (§5.1, §5.2) are timed beside them, and the autotuned
settings with only the full vectors in HBM (the graph rows still read from
host memory).  With `--L` the sweep and the autotuner are skipped.

Timed: `--steps` searches of the device-resident batch, each bracketed by CUDA
events on the launching stream, an L2 flush (a 512 MB write) between them.
`e2e`: the same search through the C ABI with pinned host queries and
results (copies inside the timed region).  `cpu_baseline`: the CPU oracle on
the host cores.  `--impl reference` times that oracle alone.

Multi-GPU (torchrun): every rank searches its own replica (weak scaling, no
data-path collective); the slowest rank's time is reported.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_SWEEP = (16, 24, 32, 48, 64, 80, 96, 112, 128, 160, 192, 224, 256, 288, 320, 384, 512, 768, 1024)
TARGET_RECALL = 0.9
K = 10                      # k of the search and of recall@k (--k)
def workload_name(args):
    if args.config == 5:
        return ("serving at the largest size the host holds: n=%d u8 d=128, 16384 low-rank "
                "components, %d queries, PQ M=32, overlapping-shard Vamana graph R=64, k=%d"
                % (args.n or 200_000_000, args.nq or 10_000, K))
    if args.config == 4:
        return ("batched form: n=%d int8 d=100, 4096 components, %d queries, PQ M=%d, R=64, k=%d"
                % (args.n or 100_000_000, args.nq or 10_000, args.M or 50, K))
    if args.config == 3:
        return ("precision form: n=%d f32 d=96 unit-normalised, 1024 components, %d queries, "
                "PQ M=%d, R=68 (64 in-cluster + 4 medoid links), k=%d" % (
                    args.n or 10_000_000, args.nq or 10_000, args.M or 48, K))
    n = args.n or 1_000_000
    return "mid-scale plain method: n=%s u8 d=128, %d queries, PQ M=%d, R=64, k=%d" % (
        "1M" if n == 1_000_000 else str(n), args.nq or 10_000, args.M or 32, K)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=("gb300", "reference"))
    ap.add_argument("--n", type=int, default=None, help="shrink the workload (testing only)")
    ap.add_argument("--nq", type=int, default=None)
    ap.add_argument("--ncomp", type=int, default=None)
    ap.add_argument("--L", type=int, default=None, help="fix L instead of sweeping")
    ap.add_argument("--bloom-log2", type=int, default=16)
    ap.add_argument("--cpu-sample", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--k", type=int, default=10, help="k of the search and of k-recall@k")
    ap.add_argument("--M", type=int, default=None, help="PQ subspaces (bytes per code)")
    ap.add_argument("--gpu-build", action="store_true",
                    help="build the PQ codes and the clustered graph with the library's GPU "
                         "builder instead of the host generator (data and ground truth stay on "
                         "the host)")
    ap.add_argument("--gpu-truth", action="store_true",
                    help="with --gpu-build: exact k-NN by bang_ground_truth on the GPU, checked "
                         "against the oracle's brute force on sampled queries")
    ap.add_argument("--packed", action="store_true",
                    help="fixed forms read packed graph rows (BANG_GRAPH_PACKED)")
    ap.add_argument("--records", action="store_true",
                    help="fixed host forms read each node's row and vector as one record "
                         "(BANG_NODE_RECORDS)")
    ap.add_argument("--config", type=int, default=5, choices=(2, 3, 4, 5),
                    help="5: serving at the largest size the host holds (200M u8, the headline); "
                         "2: mid-scale u8 (1M); 3: the precision form (f32 d=96); 4: the batched "
                         "form (100M int8, d=100)")
    args = ap.parse_args()
    global K
    K = args.k
    return args


def metric_name():
    return "queries/s at recall@%d=0.9" % K


def sweep_values():
    return [L for L in L_SWEEP if L >= K]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_throughput(units_per_rank, steps, total_ms_local, world, dist=None, device="cpu"):
    """Whole-job units/s for replicas: every rank processed units_per_rank per
    step; the job took as long as the slowest rank.  Returns (units/s, ms)."""
    t = float(total_ms_local)
    if world > 1:
        import torch
        x = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return units_per_rank * world * steps / (t / 1e3), t


def gpu_built_workload(args, kw, device):
    """Data and ground truth from the host generator; PQ codebook, codes and
    the clustered graph from bang_build_pq / bang_build_cluster_graph."""
    import workload
    import paper_2401_11324_gb300 as bang
    if args.gpu_truth:
        kw = dict(kw, k=0)
    w = workload.clustered_data(args.config, verbose=True, **kw)
    c = w["params"]
    if args.gpu_truth:
        import oracle
        t0 = time.perf_counter()
        w["gt_ids"], w["gt_dist"] = bang.bang_ground_truth(w["base"], w["queries"], max(100, K),
                                                           device=device)
        t_gt = time.perf_counter() - t0
        sel = np.linspace(0, w["queries"].shape[0] - 1, 16).astype(np.int64)
        ids_o, dist_o = oracle.bruteforce_knn(w["base"], w["queries"][sel], max(100, K))
        if not ((ids_o == w["gt_ids"][sel]).all() and (dist_o == w["gt_dist"][sel]).all()):
            raise RuntimeError("GPU ground truth differs from the oracle's brute force")
        w["truth"] = ("GPU (bang_ground_truth) in %.1f s; 16 sampled queries equal to the oracle's "
                      "brute force" % t_gt)
    t0 = time.perf_counter()
    cb, codes = bang.bang_build_pq(w["base"], c["M"], w["pq_sample"],
                                   w["pq_init"].reshape(c["M"], 256), 10, device=device)
    t1 = time.perf_counter()
    adj = workload.aligned_empty((w["base"].shape[0], c["R"]), np.uint32)   # read in place later
    bang.bang_build_cluster_graph(w["base"], w["members"], w["gstart"], w["medoids"], c["R"],
                                  c["alpha"], c["nx"], w["xclu"], w["hclu"].shape[1], w["hclu"],
                                  adj=adj, device=device)
    t2 = time.perf_counter()
    w.update(codebook=cb, codes=codes, adj=adj,
             index_build={"pq_s": round(t1 - t0, 2), "graph_s": round(t2 - t1, 2),
                          "where": "GPU (bang_build_pq, bang_build_cluster_graph)"})
    return w


def load_workload(args, rank, world, barrier):
    import workload
    kw = dict(n=args.n, nq=args.nq, ncomp=args.ncomp, k=max(100, K))
    if args.M is not None:
        kw["M"] = args.M
    if args.gpu_build:
        return gpu_built_workload(args, kw, int(os.environ.get("LOCAL_RANK", "0")))
    if rank == 0:
        w = workload.clustered_workload(args.config, verbose=True, **kw)
    barrier()
    if rank != 0:
        w = workload.clustered_workload(args.config, **kw)
    return w


def dist_error(ids, dist, base, queries):
    """Max and mean relative error of returned distances against FP64 exact
    squared distances of the same ids."""
    ids = np.asarray(ids).astype(np.int64)
    ok = ids != 0xFFFFFFFF
    q = np.repeat(np.arange(ids.shape[0]), ids.shape[1]).reshape(ids.shape)[ok]
    ex = ((base[ids[ok]].astype(np.float64) - queries[q].astype(np.float64)) ** 2).sum(1)
    err = np.abs(np.asarray(dist, np.float64)[ok] - ex) / np.maximum(ex, 1e-300)
    return {"max_rel": float(err.max()) if err.size else 0.0,
            "mean_rel": float(err.mean()) if err.size else 0.0}


def recall(found, truth, k=None):
    k = k or K
    f = np.asarray(found)[:, :k].astype(np.int64)
    t = np.asarray(truth)[:, :k].astype(np.int64)
    hits = (f[:, :, None] == t[:, None, :]).any(-1).sum()
    return float(hits) / (k * len(f))


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def serving(bang, ix, w, L, mode, capacity_qps, log2z, seconds=2.0, early=0):
    """Continuous batching under Poisson arrivals of requests of 1..1024
    queries (uniform), k = 10, at fractions of the measured batch throughput:
    achieved queries/s and p50/p99 latency (submit to results on the host)."""
    import threading
    srv = bang.Server(ix, K, L, max_batch=1024, streams=8, mode=mode, bloom_log2=log2z,
                      early_codes=early)
    rng = np.random.default_rng(7)
    nqall = w["queries"].shape[0]
    out = []
    for frac in (0.3, 0.6, 0.9):
        rate_q = frac * capacity_qps
        mean_req = 512.5
        nreq = max(20, int(rate_q / mean_req * seconds))
        sizes = rng.integers(1, 1025, size=nreq)
        gaps = rng.exponential(mean_req / rate_q, size=nreq)
        starts = rng.integers(0, nqall - 1024, size=nreq)
        tickets, lat = [None] * nreq, [0.0] * nreq
        done_t = [0.0]

        def waiter():
            for i in range(nreq):
                while tickets[i] is None:
                    time.sleep(5e-5)
                lat[i] = srv.wait(tickets[i])[2]
            done_t[0] = time.perf_counter()

        th = threading.Thread(target=waiter)
        th.start()
        t0 = time.perf_counter()
        t_next = t0
        for i in range(nreq):
            t_next += gaps[i]
            while time.perf_counter() < t_next:
                time.sleep(min(2e-4, max(0.0, t_next - time.perf_counter())))
            n = int(sizes[i])
            q = w["queries"][starts[i]:starts[i] + n]
            tickets[i] = srv.submit(q, np.full(n, K, np.uint32), np.full(n, L, np.uint32))
        th.join()
        span = done_t[0] - t0
        out.append({"offered_qps": rate_q, "achieved_qps": float(sizes.sum()) / span,
                    "requests": nreq, "p50_ms": float(np.percentile(lat, 50)),
                    "p99_ms": float(np.percentile(lat, 99))})
    srv.stop()
    return {"what": "Poisson arrivals of 1..1024-query requests, k=10, L=%d, 8 streams, "
                    "max 1024 queries per launch" % L, "points": out}


def cpu_baseline(w, L, sample, log2z):
    """The oracle's search as it stands, OpenMP over queries on all host cores."""
    import oracle
    ix = oracle.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["codes"].shape[1])
    Q = w["queries"][:sample]
    t0 = time.perf_counter()
    r = ix.search(Q, K, L, log2z=log2z)
    dt = time.perf_counter() - t0
    return {"value": len(Q) / dt, "unit": "queries/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": "%d of the %d queries at L=%d (same index, same Bloom size); recall@%d %.4f"
                      % (len(Q), w["queries"].shape[0], L, K, recall(r["ids"], w["gt_ids"][:len(Q)]))}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import workload  # noqa: F401
    if args.config in (4, 5):       # the index (input to the timed search) is built on the GPU
        w = large_workload(args, int(os.environ.get("LOCAL_RANK", "0")))
    else:
        w = load_workload(args, 0, 1, lambda: None)
    import oracle
    ix = oracle.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["codes"].shape[1])
    nq = w["queries"].shape[0]
    L = args.L
    if L is None:
        L = sweep_values()[-1]
        for Lc in sweep_values():
            r = ix.search(w["queries"][:1000], K, Lc, log2z=args.bloom_log2)
            if recall(r["ids"], w["gt_ids"][:1000]) >= TARGET_RECALL:
                L = Lc
                break
    sample = min(args.cpu_sample, nq)
    Q = w["queries"][:sample]
    for _ in range(args.warmup):
        ix.search(Q[:200], K, L, log2z=args.bloom_log2)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ix.search(Q, K, L, log2z=args.bloom_log2)
    dt = time.perf_counter() - t0
    v = sample * args.steps / dt
    line = {"metric": metric_name(), "value": v, "unit": "queries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args), "L": L, "bloom_log2": args.bloom_log2,
                       "step": "%d queries (bounded sample of the 10k batch)" % sample},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "queries/s", "cores": oracle.max_threads(),
                             "kind": "oracle",
                             "sample": "%d queries per step at L=%d" % (sample, L)},
            "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# Traffic per launch of the head kernel from one ncu capture of the current
# kernel version at the default workload, keyed by (mode, bloom_log2, L, placement):
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) and host-memory
# bytes (32-byte sysmem read sectors).  Cleared whenever the kernel changes.
NCU_TRAFFIC = {(3, 15, 160, 4): 33481984 + 0}
NCU_HOST_TRAFFIC = {(3, 15, 160, 4): 18247564 * 32}

FORMS = {
    # name: (distance mode, placement flags, what it is)
    "fp32": (0, 0, "plain method: FP32 PQ table, graph and vectors in host memory (Alg. 2)"),
    "bf16": (1, 0, "reduced precision: BF16 PQ table summed in FP32, host graph and vectors"),
    "bf16_tc": (1, 0, "reduced precision with the BF16 tables of the whole batch built on the "
                      "tensor cores (tcgen05) first"),
    "q8": (3, 0, "reduced precision: 8-bit PQ table (per-subspace offset, one scale per query) "
                 "summed exactly in integers, host graph and vectors"),
    "in_memory": (0, 3, "In-memory variant (§5.1): FP32 PQ table, graph and vectors in HBM"),
    "exact": (2, 3, "Exact-distance variant (§5.2): exact distances, graph and vectors in HBM"),
}


def large_workload(args, device):
    """Configurations 4 and 5: data from the counter-based generator; PQ
    codebook and codes, the overlapping-shard graph (§2.2) and the exact
    100 nearest neighbours of every query built on the GPU; 16 sampled ground
    truth rows checked against the oracle's brute force."""
    import workload
    import paper_2401_11324_gb300 as bang
    n_req = args.n
    _, world, _ = dist_env()
    if n_req is None and world > 1:
        # every replica holds the data and graph in host memory while it
        # builds (about 420 bytes per point): fit all ranks on this node
        avail = 0
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
        n_req = int(min(workload.CONFIGS[args.config]["n"], 0.7 * avail / (world * 420)))
        n_req -= n_req % 1_000_000
    # graph and vectors in host memory advised for huge pages (bang_host_alloc)
    w = workload.large_data(args.config, n=n_req, nq=args.nq, ncomp=args.ncomp, verbose=True,
                            alloc=bang.host_empty)
    c = w["params"]
    n = w["base"].shape[0]
    t0 = time.perf_counter()
    cb, codes = bang.bang_build_pq(w["base"], c["M"], w["pq_sample"],
                                   w["pq_init"].reshape(c["M"], 256), 10, device=device)
    t1 = time.perf_counter()
    adj = bang.host_empty((n, c["R"]), np.uint32)                 # read in place later
    bang.bang_build_shard_graph(w["base"], w["shard_centres"], c["ell"], c["R"], c["Lb"], c["alpha"],
                                c["batch_frac"], c["bloom_build"], adj=adj, device=device)
    t2 = time.perf_counter()
    gt_ids, gt_dist = bang.bang_ground_truth(w["base"], w["queries"], 100, device=device)
    t3 = time.perf_counter()
    import oracle
    sel = np.linspace(0, w["queries"].shape[0] - 1, 16).astype(np.int64)
    ids_o, dist_o = oracle.bruteforce_knn(w["base"], w["queries"][sel], 100)
    if not ((ids_o == gt_ids[sel]).all() and (dist_o == gt_dist[sel]).all()):
        raise RuntimeError("GPU ground truth differs from the oracle's brute force")
    deg = (adj != 0xFFFFFFFF).sum(1)
    w.update(codebook=cb, codes=codes, adj=adj, gt_ids=gt_ids, gt_dist=gt_dist,
             index_build={"where": "GPU: bang_build_pq, bang_build_shard_graph (%d shards, each point "
                                   "in its %d nearest, GreedySearch worklist %d, alpha %.1f, batch "
                                   "fraction %.2f), bang_ground_truth" % (
                                       c["shards"], c["ell"], c["Lb"], c["alpha"], c["batch_frac"]),
                          "pq_s": round(t1 - t0, 1), "graph_s": round(t2 - t1, 1),
                          "ground_truth_s": round(t3 - t2, 1),
                          "mean_degree": round(float(deg.mean()), 2), "max_degree": int(deg.max())},
             truth="GPU (bang_ground_truth); 16 sampled queries equal to the oracle's brute force")
    return w


# Forms of the large configurations: (name, distance mode, placement, Bloom
# log2, what).  Results do not depend on the placement (tested), so every
# operating point is found with graph and vectors in HBM.
# early: request every neighbour's code row as soon as the node's row arrives
# (early_codes; same results; measured faster with the FP32 and BF16 tables,
# slower with the 8-bit table).
def _form(name, mode, placement, lz, early, tsrc, what, rerank=0):
    return dict(name=name, mode=mode, placement=placement, lz=lz, early=early, tsrc=tsrc,
                rerank=rerank, what=what)


LARGE_FORMS = [
    _form("fp32_hbm", 0, 3, 16, 1, 0, "FP32 PQ table (the paper's precision), graph and vectors in HBM "
                                      "(the In-memory variant, §5.1)"),
    _form("bf16_hbm", 1, 3, 16, 1, 0, "BF16 PQ table (reduced precision) summed in FP32, graph and "
                                      "vectors in HBM"),
    _form("q8_hbm", 3, 3, 15, 0, 0, "8-bit PQ table (reduced precision) summed in integers, graph and "
                                    "vectors in HBM"),
    _form("exact_hbm", 2, 3, 16, 0, 0, "Exact-distance variant (§5.2): exact distances in the loop, no "
                                       "table and no re-rank, graph and vectors in HBM"),
    _form("fp32_tc_hbm", 0, 3, 16, 1, 1, "FP32 search on tables built by the tensor cores (three-way "
                                         "BF16 splits, about FP32), graph and vectors in HBM"),
    _form("tf32_tc_hbm", 0, 3, 16, 1, 2, "TF32 tables: the tensor-core contraction with both operands "
                                         "rounded to TF32 and FP32 accumulation, FP32 search, HBM"),
    _form("fp32_staged_hbm", 0, 3, 16, 1, 0, "FP32 table with the re-rank staged as a separate kernel "
                                             "after the search (§4.8), graph and vectors in HBM",
          rerank=1),
    _form("fp32_toplist_hbm", 0, 3, 16, 1, 0, "FP32 table, staged re-rank of the final worklist only "
                                              "(the top-L by PQ distance), graph and vectors in HBM",
          rerank=2),
]


# FP32 (the paper's precision) first, then the reduced and tensor-core table forms
PRECISION_FORMS = ("fp32_hbm", "bf16_hbm", "q8_hbm", "tf32_tc_hbm", "fp32_tc_hbm")


def run_large(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    import paper_2401_11324_gb300 as bang
    w = large_workload(args, local)
    barrier()
    c = w["params"]
    nq, d = w["queries"].shape
    n = w["base"].shape[0]
    M, R = w["codes"].shape[1], w["adj"].shape[1]
    esz = w["base"].dtype.itemsize
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], M, device=local)
    stream = torch.cuda.Stream(device=dev)
    sptr = stream.cuda_stream
    q_dev = torch.from_numpy(w["queries"]).to(dev)
    ids = torch.empty((nq, K), dtype=torch.int32, device=dev)
    dout = torch.empty((nq, K), dtype=torch.float32, device=dev)
    iters = torch.empty(nq, dtype=torch.int32, device=dev)
    ndist = torch.empty(nq, dtype=torch.int32, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    placement = [None]

    def place(flags):
        if placement[0] != flags:
            ix.set_placement(flags)
            placement[0] = flags

    early = [0]                     # early_codes of the form being measured
    tsrc = [0]                      # table_source of the form being measured
    rerank = [0]                    # re-rank of the form being measured (0 fused, 1 staged)

    def search(L, mode, lz, nsub=None, stats=False):
        p = bang.make_params(bloom_log2=lz, mode=mode, out_iters=iters if stats else None,
                             out_ndist=ndist if stats else None, early_codes=early[0],
                             table_source=tsrc[0], rerank=rerank[0])
        m = nsub or nq
        ix.search(q_dev[:m], K, L, ids[:m], dout[:m], p, stream=sptr)

    def rec_now(m=None):
        m = m or nq
        return recall(ids[:m].cpu().numpy().view(np.uint32), w["gt_ids"][:m])

    def operating_point(mode, lz):
        sweep = []
        if args.L is not None:
            return args.L, sweep
        for Lc in sweep_values():
            search(Lc, mode, lz)
            stream.synchronize()
            rc = rec_now()
            sweep.append({"L": Lc, "recall@%d" % K: round(rc, 4)})
            if rc >= TARGET_RECALL:
                return Lc, sweep
        return sweep_values()[-1], sweep

    def timed(L, mode, lz, steps, nsub=None):
        for _ in range(args.warmup):
            search(L, mode, lz, nsub)
        stream.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        barrier()
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter()
        for a_, b_ in evs:
            with torch.cuda.stream(stream):
                flush.fill_(3)
                a_.record(stream)
            search(L, mode, lz, nsub)
            b_.record(stream)
        stream.synchronize()
        t_wall = time.perf_counter() - t_wall
        torch.cuda.synchronize(dev)
        barrier()
        ms = [a_.elapsed_time(b_) for a_, b_ in evs]
        _, total_ms = job_throughput(nsub or nq, steps, sum(ms), world, dist, dev)
        return (nsub or nq) * world * steps / (total_ms / 1e3), total_ms / steps, t_wall

    res = {}
    with ClockSampler(local) as clk:
        for f in LARGE_FORMS:
            name, mode, pl, lz, ec, ts, what = (f["name"], f["mode"], f["placement"], f["lz"],
                                                f["early"], f["tsrc"], f["what"])
            early[0] = ec
            tsrc[0] = ts
            rerank[0] = f["rerank"]
            place(pl)
            L, sweep = operating_point(mode, lz)
            search(L, mode, lz, stats=True)
            stream.synchronize()
            r = rec_now()
            ids_np, dout_np = ids.cpu().numpy().view(np.uint32), dout.cpu().numpy()
            derr = dist_error(ids_np, dout_np, w["base"], w["queries"])
            digest = hash((ids_np.tobytes(), dout_np.tobytes()))
            it = iters.cpu().numpy().astype(np.int64)
            nd = ndist.cpu().numpy().astype(np.int64)
            value, ms, t_wall = timed(L, mode, lz, args.steps)
            res[name] = dict(form=name, what=what, mode=mode, placement=pl, lz=lz, early=ec, tsrc=ts,
                             rerank=f["rerank"], L=L, sweep=sweep,
                             recall=round(r, 4), dist_error=derr, iters=it, ndist=nd, value=value,
                             ms_per_step=ms, t_wall=t_wall, digest=digest)
    # sampled queries of the FP32, 8-bit and Exact-distance forms at their
    # operating points, bit for bit against the oracle on the same index
    import oracle
    oix = oracle.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], M)
    sel = np.linspace(0, nq - 1, 16).astype(np.int64)
    parity = {}
    for name, okw in (("fp32_hbm", {}), ("q8_hbm", {"q8": True}), ("exact_hbm", {"exact": True}),
                      ("fp32_staged_hbm", {}), ("fp32_toplist_hbm", {"rerank_list": True})):
        r = res[name]
        early[0] = r["early"]
        tsrc[0] = r["tsrc"]
        rerank[0] = r["rerank"]
        search(r["L"], r["mode"], r["lz"], stats=True)
        stream.synchronize()
        o = oix.search(w["queries"][sel], K, r["L"], log2z=r["lz"], **okw)
        gi = ids.cpu().numpy().view(np.uint32)[sel]
        gd = dout.cpu().numpy()[sel]
        git = iters.cpu().numpy().view(np.uint32)[sel]
        parity[name] = bool((gi == o["ids"]).all() and (git == o["iters"]).all() and
                            np.array_equal(gd, o["dist"]))
    del oix

    # the paper's placement (graph and vectors read in place from page-locked
    # host memory), and the vectors alone in HBM, each at the FP32 form's
    # operating point, on a bounded sample of the batch (the same results)
    fp = res["fp32_hbm"]
    early[0] = fp["early"]
    tsrc[0] = fp["tsrc"]
    rerank[0] = fp["rerank"]
    host = {}
    for name, pl, what in (("fp32_host", 0, "FP32 PQ table, graph and vectors read in place from "
                                           "page-locked host memory (the paper's placement, Alg. 2)"),
                           ("fp32_vectors_hbm", 2 | 4, "FP32 PQ table, vectors in HBM, graph rows "
                                                       "(packed ids) read in place from host memory")):
        place(pl)
        m = min(nq, 1000)
        t0 = time.perf_counter()
        search(fp["L"], 0, fp["lz"], nsub=200)
        stream.synchronize()
        est = 200 / max(1e-6, time.perf_counter() - t0)
        m = int(min(nq, max(200, min(1000, est * 2.0))))      # about two seconds per step
        value, ms, _ = timed(fp["L"], 0, fp["lz"], 2, nsub=m)
        host[name] = dict(what=what, value=value, ms_per_step=ms, L=fp["L"], queries=m,
                          placement=pl)
    place(3)

    # autotuned settings (table precision, Bloom size, L) for recall@10 >= 0.9 in HBM
    early[0] = 0
    tsrc[0] = 0
    rerank[0] = 0
    t0 = time.perf_counter()
    try:
        tune = ix.autotune(q_dev, K, 0, truth=np.ascontiguousarray(w["gt_ids"][:, :K]),
                           target_recall=TARGET_RECALL, bloom_min=14, bloom_max=17, try_structure=1,
                           stream=sptr)
        tune["seconds"] = round(time.perf_counter() - t0, 2)
        early[0], rerank[0], tsrc[0] = tune["early_codes"], tune["rerank"], tune["table_source"]
        search(tune["L"], tune["mode"], tune["bloom_log2"])
        stream.synchronize()
        tune_rec = rec_now()
        tv, tms, _ = timed(tune["L"], tune["mode"], tune["bloom_log2"], args.steps)
        tuned = dict(value=tv, ms_per_step=tms, L=tune["L"], mode=tune["mode"],
                     bloom_log2=tune["bloom_log2"], table_source=tune["table_source"],
                     early_codes=tune["early_codes"], rerank=tune["rerank"], recall=round(tune_rec, 4),
                     seconds=tune["seconds"], candidates=tune["candidates"])
    except bang.BangError as e:
        tuned = {"failed": str(e)}
    early[0] = tsrc[0] = rerank[0] = 0

    # batched form: per-query k in {1, 10, 100} and L in {32, ..., 256} (at
    # least k), one persistent launch replayed from a CUDA graph
    q8 = res["q8_hbm"]
    rng = np.random.default_rng(44)
    kq = rng.choice([1, 10, 100], size=nq).astype(np.uint32)
    lmix = [q8["L"], q8["L"] * 5 // 4, q8["L"] * 3 // 2, 2 * q8["L"]]   # the operating point up to 2x
    lmix = [min(x, 1024) for x in lmix]
    Lq = np.maximum(rng.choice(lmix, size=nq), kq).astype(np.uint32)
    Lmax_b = int(Lq.max())
    kd = torch.from_numpy(kq.view(np.int32)).to(dev)
    Ld = torch.from_numpy(Lq.view(np.int32)).to(dev)
    bids = torch.empty((nq, 100), dtype=torch.int32, device=dev)
    bdist = torch.empty((nq, 100), dtype=torch.float32, device=dev)
    bp = bang.make_params(bloom_log2=q8["lz"], mode=q8["mode"])
    ix.search_batched(q_dev, kd, Ld, 100, Lmax_b, bids, bdist, bp, stream=sptr)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        ix.search_batched(q_dev, kd, Ld, 100, Lmax_b, bids, bdist, bp, stream=sptr)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(max(3, min(args.steps, 10)))]
    for a_, b_ in evs:
        with torch.cuda.stream(stream):
            flush.fill_(3)
            a_.record(stream)
            graph.replay()
            b_.record(stream)
    stream.synchronize()
    bms = statistics.mean(a_.elapsed_time(b_) for a_, b_ in evs)
    got = bids.cpu().numpy().view(np.uint32)
    brec = {}
    for kk in (1, 10, 100):
        sel = np.where(kq == kk)[0]
        brec["recall@%d" % kk] = round(recall(got[sel, :kk], w["gt_ids"][sel], kk), 4)
    batched = {"value": nq / (bms / 1e3), "unit": "queries/s", "ms_per_step": bms,
               "launch": "one persistent launch (bang_search_batched) replayed from a CUDA graph, "
                         "8-bit table, graph and vectors in HBM",
               "k_mix": "uniform over {1, 10, 100}",
               "L_mix": "uniform over {%s} (the 8-bit form's operating point up to twice it), at least k"
                        % ", ".join(str(x) for x in lmix), **brec}
    del graph

    # the headline: the faster of the two FP32-table forms (re-rank fused or
    # staged: the same results), at the operating point of the target recall
    st_ = res["fp32_staged_hbm"]
    head = st_ if st_["value"] > fp["value"] and st_["digest"] == fp["digest"] else fp
    it, nd = head["iters"], head["ndist"]
    launch_s = head["ms_per_step"] / 1e3
    # end to end through the C ABI: pinned host queries and results
    q_host = torch.from_numpy(w["queries"]).pin_memory()
    ids_h = torch.empty((nq, K), dtype=torch.int32).pin_memory()
    dist_h = torch.empty((nq, K), dtype=torch.float32).pin_memory()
    hp = bang.make_params(bloom_log2=head["lz"], mode=head["mode"], early_codes=head["early"],
                          table_source=head["tsrc"], rerank=head["rerank"])
    for _ in range(2):
        ix.search(q_host, K, head["L"], ids_h, dist_h, hp, stream=sptr)
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ix.search(q_host, K, head["L"], ids_h, dist_h, hp, stream=sptr)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    early[0] = head["early"]
    tsrc[0] = head["tsrc"]
    rerank[0] = head["rerank"]
    search(head["L"], head["mode"], head["lz"])
    stream.synchronize()
    assert (ids_h.numpy() == ids.cpu().numpy()).all()

    # serving: continuous batching in HBM with the BF16 table (the reduced
    # precision whose recall stays within 0.005 of FP32) and with the 8-bit table
    serving_rec = serving_q8 = None
    bf = res["bf16_hbm"]
    if not args.no_serving:
        serving_rec = serving(bang, ix, w, bf["L"], bf["mode"], bf["value"], bf["lz"], early=bf["early"])
        serving_q8 = serving(bang, ix, w, q8["L"], q8["mode"], q8["value"], q8["lz"], early=q8["early"])

    # rooflines: HBM binds the headline (graph, vectors and codes in HBM);
    # per expansion the row (R ids), the vector and one code row per new
    # neighbour (M bytes; nd counts them)
    row_bytes = R * 4
    hbm_bytes = int(it.sum()) * (row_bytes + d * esz) + int(nd.sum()) * M + nq * d * esz + nq * K * 8
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_gbs = hbm_bytes / launch_s / 1e9
    link = bang.bang_probe_host_link(local, 1 << 30, row_bytes)
    foot = int(min(n * (row_bytes + d * esz), 32 << 30))
    link_far = bang.bang_probe_host_link(local, foot, row_bytes)
    hf = host["fp32_host"]
    host_bytes_q = float(it.mean()) * (row_bytes + d * esz)
    host_gbs = hf["value"] * host_bytes_q / 1e9

    def brief(r):
        return {"what": r["what"], "value": r["value"], "ms_per_step": r["ms_per_step"],
                "L": r["L"], "recall@%d" % K: r["recall"], "sweep": r["sweep"],
                "mean_iterations": float(r["iters"].mean()),
                "dist_error_vs_fp64": r["dist_error"]}

    served = served_q8 = None
    if serving_rec is not None:
        top = serving_rec["points"][-1]
        served = {"what": "continuous batching (bang_server_*), BF16 table, graph and vectors in "
                          "HBM, L=%d, recall@%d %.4f (FP32: %.4f)" % (bf["L"], K, bf["recall"],
                                                                    fp["recall"]),
                  "achieved_qps": top["achieved_qps"], "p50_ms": top["p50_ms"], "p99_ms": top["p99_ms"],
                  "offered_qps": top["offered_qps"],
                  "vs_plain_form": top["achieved_qps"] / hf["value"],
                  "vs_fp32_hbm": top["achieved_qps"] / fp["value"]}
        t8 = serving_q8["points"][-1]
        served_q8 = {"what": "continuous batching, 8-bit table, graph and vectors in HBM, L=%d, "
                             "recall@%d %.4f" % (q8["L"], K, q8["recall"]),
                     "achieved_qps": t8["achieved_qps"], "p50_ms": t8["p50_ms"], "p99_ms": t8["p99_ms"],
                     "vs_plain_form": t8["achieved_qps"] / hf["value"]}
    summary = {
        "plain_form": {"value": hf["value"], "L": fp["L"], "recall@%d" % K: fp["recall"],
                       "what": "FP32 table, graph and vectors in page-locked host memory"},
        "fp32_hbm": {"value": fp["value"], "L": fp["L"], "recall@%d" % K: fp["recall"]},
        "bf16_hbm": {"value": res["bf16_hbm"]["value"], "L": res["bf16_hbm"]["L"],
                     "recall@%d" % K: res["bf16_hbm"]["recall"]},
        "q8_hbm": {"value": q8["value"], "L": q8["L"], "recall@%d" % K: q8["recall"]},
        "exact_hbm": {"value": res["exact_hbm"]["value"], "L": res["exact_hbm"]["L"],
                      "recall@%d" % K: res["exact_hbm"]["recall"]},
        "rerank_ablation": {"fused_value": fp["value"], "staged_value": res["fp32_staged_hbm"]["value"],
                            "staged_over_fused": res["fp32_staged_hbm"]["value"] / fp["value"],
                            "L": fp["L"], "same_results": res["fp32_staged_hbm"]["digest"] == fp["digest"],
                            "final_worklist_only": {"value": res["fp32_toplist_hbm"]["value"],
                                                    "L": res["fp32_toplist_hbm"]["L"],
                                                    "recall@%d" % K: res["fp32_toplist_hbm"]["recall"]},
                            "what": "FP32 table: re-rank fused into the loop vs staged as a separate "
                                    "kernel over the recorded candidates (§4.8)"},
        "tensor_core_tables": {f: {"value": res[f]["value"], "L": res[f]["L"],
                                   "recall@%d" % K: res[f]["recall"],
                                   "recall_vs_fp32": round(res[f]["recall"] - fp["recall"], 4)}
                               for f in ("fp32_tc_hbm", "tf32_tc_hbm")},
        "served": None if served is None else {k_: served[k_] for k_ in (
            "achieved_qps", "p50_ms", "p99_ms", "vs_plain_form", "vs_fp32_hbm")},
        "served_q8": None if served_q8 is None else {k_: served_q8[k_] for k_ in (
            "achieved_qps", "p50_ms", "p99_ms", "vs_plain_form")},
        "batched": {"value": batched["value"], "recall@10": batched["recall@10"]},
        "precision": {"tolerance": "reduced forms within 0.005 of FP32's recall@10",
                      "within": {f: abs(res[f]["recall"] - fp["recall"]) <= 0.005
                                 for f in PRECISION_FORMS[1:]},
                      "recall@10": {f: res[f]["recall"] for f in PRECISION_FORMS},
                      "L": {f: res[f]["L"] for f in PRECISION_FORMS},
                      "max_rel_dist_error_vs_fp64": max(res[f]["dist_error"]["max_rel"]
                                                        for f in PRECISION_FORMS)},
    }
    line = {
        "metric": metric_name(), "value": head["value"], "unit": "queries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(args), "form": head["form"], "form_what": head["what"],
                   "L": head["L"], "recall@%d" % K: head["recall"], "k": K, "bloom_log2": head["lz"],
                   "early_codes": head["early"], "rerank": "staged" if head["rerank"] else "fused",
                   "mean_iterations": float(it.mean()), "mean_pq_distances": float(nd.mean()),
                   "n": n, "nq": nq, "parallelism": "replica per GPU" if world > 1 else "single GPU",
                   "l2": "512 MB flush written between timed steps; the index (77 GB) is larger "
                         "than L2",
                   "index_build": w["index_build"], "ground_truth": w["truth"],
                   "parity": {"what": "16 sampled queries: ids, distances and iteration counts "
                                      "equal to the oracle's on this index", **parity},
                   "summary": summary},
        "forms": {f: brief(r) for f, r in res.items()},
        "host_forms": host,
        "autotuned": tuned,
        "batched_form": batched,
        "roofline": {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": hbm_gbs / hbm_peak, "traffic": None,
                     "traffic_note": "not captured at this size (83 GB in HBM); at 8M points "
                                     "and L = 224 the staged headline's search read 1.917 GB and "
                                     "its re-rank 0.303 GB of DRAM per step for 1.543 GB "
                                     "algorithmic (1.44x: each 32-byte code row costs a 64-byte "
                                     "DRAM access); the fused form's search read 2.305 GB",
                     "peak_source": "measured (MEASURED_PEAKS.json)" if "hbm_gbs" in peaks
                                    else "fallback",
                     "algorithmic_bytes_per_launch": hbm_bytes,
                     "per_unit": "%d B per expansion (row %d B + vector %d B) + %d B per PQ distance"
                                 % (row_bytes + d * esz, row_bytes, d * esz, M),
                     "units_per_launch": int(it.sum())},
        "host_link": {"plain_form_gbs": host_gbs, "gather_gbs_1GiB": link["gather_gbs"],
                      "gather_gbs_index_footprint": link_far["gather_gbs"],
                      "footprint_bytes": foot, "copy_engine_gbs": link["h2d_copy_gbs"],
                      "host_threads_gather_gbs": link["cpu_gather_gbs"],
                      "load_latency_ns": link["latency_ns"],
                      "load_latency_ns_index_footprint": link_far["latency_ns"],
                      "note": "random %d-byte row gathers in place from page-locked host memory: "
                              "the GPU reaches 1 GiB at full speed and the index's footprint far "
                              "slower, which is why the headline keeps graph and vectors in HBM"
                              % row_bytes},
        "e2e": {"value": nq / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": nq * d * esz,
                "d2h_bytes_per_step": nq * K * 8},
        "gpu_launches": args.steps * (2 if head["rerank"] else 1),   # search (+ re-rank) per step
        "clocks": clk.summary(),
        "wall_s_timed_region": sum(r["t_wall"] for r in res.values()),
    }
    if serving_rec is not None:
        line["serving"] = serving_rec
        line["serving_q8"] = serving_q8
        line["served_form"] = served
        line["served_form_q8"] = served_q8
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, fp["L"], min(args.cpu_sample, nq), 16)
    line["plain_form"] = summary["plain_form"]
    ix.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config in (4, 5):
        return run_large(args)
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    import paper_2401_11324_gb300 as bang
    w = load_workload(args, rank, world, barrier)
    nq, d = w["queries"].shape
    M = w["codes"].shape[1]
    R = w["adj"].shape[1]
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], M, device=local)
    stream = torch.cuda.Stream(device=dev)
    sptr = stream.cuda_stream
    q_dev = torch.from_numpy(w["queries"]).to(dev)
    ids = torch.empty((nq, K), dtype=torch.int32, device=dev)
    dist_out = torch.empty((nq, K), dtype=torch.float32, device=dev)
    iters = torch.empty(nq, dtype=torch.int32, device=dev)
    ndist = torch.empty(nq, dtype=torch.int32, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    placement = [None]

    def place(flags):
        if placement[0] != flags:
            ix.set_placement(flags)
            placement[0] = flags

    depth = [1]                       # prefetch depth of the form being measured

    def search(L, mode, with_stats=False, phase=None, tsrc=0, lz=None):
        p = bang.make_params(bloom_log2=lz or args.bloom_log2, mode=mode, table_source=tsrc,
                             out_iters=iters if with_stats else None,
                             out_ndist=ndist if with_stats else None, out_phase_cycles=phase,
                             prefetch_depth=depth[0])
        ix.search(q_dev, K, L, ids, dist_out, p, stream=sptr)

    def operating_point(mode, tsrc=0, lz=None):
        """Smallest L of the sweep with recall@k >= 0.9 (or --L)."""
        sweep = []
        if args.L is not None:
            return args.L, sweep
        for Lc in sweep_values():
            search(Lc, mode, tsrc=tsrc, lz=lz)
            stream.synchronize()
            rc = recall(ids.cpu().numpy().view(np.uint32), w["gt_ids"])
            sweep.append({"L": Lc, "recall@%d" % K: round(rc, 4)})
            if rc >= TARGET_RECALL:
                return Lc, sweep
        return sweep_values()[-1], sweep

    def timed(L, mode, steps, tsrc=0, lz=None):
        for _ in range(args.warmup):
            search(L, mode, tsrc=tsrc, lz=lz)
        stream.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        barrier()
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter()
        for s in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(s & 0xFF)
                starts[s].record(stream)
            search(L, mode, tsrc=tsrc, lz=lz)
            ends[s].record(stream)
        stream.synchronize()
        t_wall = time.perf_counter() - t_wall
        torch.cuda.synchronize(dev)
        barrier()
        step_ms = [starts[s].elapsed_time(ends[s]) for s in range(steps)]
        _, total_ms = job_throughput(nq, steps, sum(step_ms), world, dist, dev)
        return total_ms, step_ms, t_wall

    def measure(name, steps, tune=None):
        depth[0] = tune.get("prefetch_depth", 1) if tune is not None else 1
        if tune is None:
            mode, flags, what = FORMS[name]
            tsrc = 1 if name.endswith("_tc") else 0
            lz = args.bloom_log2
            if args.packed and not flags:
                flags = bang.BANG_GRAPH_PACKED
                what += "; graph rows packed"
            if args.records and not flags & (bang.BANG_GRAPH_IN_HBM | bang.BANG_VECTORS_IN_HBM):
                flags |= bang.BANG_NODE_RECORDS
                what += "; each node's row and vector as one host record"
            place(flags)
            L, sweep = operating_point(mode, tsrc)
        else:                       # settings chosen by bang_autotune
            mode, tsrc, lz, L, sweep = (tune["mode"], tune["table_source"], tune["bloom_log2"],
                                        tune["L"], [])
            flags = (tune.get("placement", 0) | (bang.BANG_GRAPH_PACKED if tune["graph_packed"] else 0)
                     | (bang.BANG_NEIGHBOR_CODES if tune["neighbor_codes"] else 0))
            if tune.get("node_records") and not tune.get("placement", 0):   # host memory only
                flags |= bang.BANG_NODE_RECORDS
            what = ("autotuned (bang_autotune): %s table%s, Bloom filter 2^%d bits, smallest L "
                    "reaching recall@%d 0.9%s" % ({0: "FP32", 1: "BF16", 3: "8-bit"}[mode],
                                                  " from the tensor cores" if tsrc else "", lz, K,
                                                  (", graph rows packed to %d-bit ids" % tune["adj_bits"]
                                                   if tune["graph_packed"] else "") +
                                                  (", neighbours' codes side by side in HBM"
                                                   if tune["neighbor_codes"] else "") +
                                                  (", each node's row and vector side by side"
                                                   if flags & bang.BANG_NODE_RECORDS else "")))
            if flags & bang.BANG_GRAPH_IN_HBM:
                what = "In-memory variant (§5.1), graph and vectors in HBM, with the " + what
            elif flags & bang.BANG_VECTORS_IN_HBM:
                what = ("vectors in HBM, graph rows read in place from host memory (between the "
                        "base method and the In-memory variant, §5.1), with the " + what)
            place(flags)
        search(L, mode, with_stats=True, tsrc=tsrc, lz=lz)
        stream.synchronize()
        rec = recall(ids.cpu().numpy().view(np.uint32), w["gt_ids"])
        derr = dist_error(ids.cpu().numpy().view(np.uint32), dist_out.cpu().numpy(), w["base"],
                          w["queries"])
        it = iters.cpu().numpy().astype(np.int64)
        nd = ndist.cpu().numpy().astype(np.int64)
        total_ms, step_ms, t_wall = timed(L, mode, steps, tsrc, lz)
        return dict(form=name, what=what, mode=mode, placement=flags, L=L, tsrc=tsrc, lz=lz,
                    depth=depth[0],
                    dist_error=derr,
                    recall=round(rec, 4), sweep=sweep, iters=it, ndist=nd,
                    value=nq * world * steps / (total_ms / 1e3), ms_per_step=total_ms / steps,
                    launch_s=statistics.mean(step_ms) / 1e3, t_wall=t_wall)

    # ---- the two forms of the paper's base method (host graph): time both,
    # report the fastest at recall@k >= 0.9 with the plain form beside it
    with ClockSampler(local) as clk:
        res = {f: measure(f, args.steps) for f in ("fp32", "bf16", "bf16_tc", "q8")}
        tune = None
        if args.L is None:
            place(0)
            t0 = time.perf_counter()
            try:
                tune = ix.autotune(q_dev, K, 0, truth=np.ascontiguousarray(w["gt_ids"][:, :K]),
                                   target_recall=TARGET_RECALL, bloom_min=14, bloom_max=19,
                                   try_packed_graph=1, try_neighbor_codes=1, try_prefetch_depth=1,
                                   try_node_records=1, stream=sptr)
                tune["adj_bits"] = int(np.ceil(np.log2(w["base"].shape[0] + 1)))
            except bang.BangError as e:        # no setting reaches the target within L <= 1024
                tune = {"failed": str(e)}
            tune["seconds"] = round(time.perf_counter() - t0, 2)
            if "failed" not in tune:
                res["autotuned"] = measure("autotuned", args.steps, tune)
    ok = [f for f in ("autotuned", "q8", "bf16_tc", "bf16", "fp32")
          if f in res and res[f]["recall"] >= TARGET_RECALL]
    head = res[max(ok, key=lambda f: res[f]["value"])] if ok else res["fp32"]
    variants = {f: measure(f, max(5, args.steps // 5)) for f in ("in_memory", "exact")}
    if tune is not None and "failed" not in tune:
        variants["in_memory_autotuned"] = measure("in_memory_autotuned", max(5, args.steps // 5),
                                                  dict(tune, placement=3))
        variants["hbm_vectors_autotuned"] = measure("hbm_vectors_autotuned", max(5, args.steps // 5),
                                                    dict(tune, placement=bang.BANG_VECTORS_IN_HBM))
    place(head["placement"])
    depth[0] = head["depth"]
    L, mode, tsrc, lz = head["L"], head["mode"], head["tsrc"], head["lz"]
    it, nd = head["iters"], head["ndist"]

    # ---- per-phase SM cycles of the fused kernel (one untimed launch): the
    # counterpart of the paper's per-kernel share of GPU time
    phase = torch.zeros((nq, len(bang.PHASES)), dtype=torch.int64, device=dev)
    search(L, mode, phase=phase, tsrc=tsrc, lz=lz)
    stream.synchronize()
    ph = phase.cpu().numpy().astype(np.float64).sum(0)
    phases = {name: round(float(ph[i] / ph[-1]), 4) for i, name in enumerate(bang.PHASES[:-1])}
    phases["cycles_per_expansion"] = round(float(ph[-1] / max(1, it.sum())), 1)

    # ---- algorithmic bytes per launch (one launch = the whole batch)
    esz = w["base"].dtype.itemsize
    row_bytes = R * 4
    if head["placement"] & bang.BANG_GRAPH_PACKED:          # ids packed to the fewest bits
        b = int(np.ceil(np.log2(w["base"].shape[0] + 1)))
        row_bytes = ((R * b + 31) // 32 + 7) // 8 * 8 * 4
    host_bytes = int(it.sum()) * (row_bytes + d * esz)     # neighbour row + full vector per expansion
    hbm_bytes = int(nd.sum()) * M + nq * d * esz + nq * K * 8 + 256 * d * 4
    launch_s = head["launch_s"]

    # ---- batched form: per-query k in {1, 10, 100} and L in {32, 64, 128, 256}
    # (at least k), the whole batch in one persistent launch replayed from a
    # CUDA graph, with the head's table, filter and graph layout
    batched = None
    if K == 10 and w["gt_ids"].shape[1] >= 100:
        rng = np.random.default_rng(44)
        kq = rng.choice([1, 10, 100], size=nq).astype(np.uint32)
        Lq = np.maximum(rng.choice([32, 64, 128, 256], size=nq), kq).astype(np.uint32)
        kd = torch.from_numpy(kq.view(np.int32)).to(dev)
        Ld = torch.from_numpy(Lq.view(np.int32)).to(dev)
        bids = torch.empty((nq, 100), dtype=torch.int32, device=dev)
        bdist = torch.empty((nq, 100), dtype=torch.float32, device=dev)
        bp = bang.make_params(bloom_log2=lz, mode=mode, prefetch_depth=depth[0])
        ix.search_batched(q_dev, kd, Ld, 100, 256, bids, bdist, bp, stream=sptr)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            ix.search_batched(q_dev, kd, Ld, 100, 256, bids, bdist, bp, stream=sptr)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize(dev)
        bsteps = max(3, min(args.steps, 20))
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(bsteps)]
        for a_, b_ in evs:
            with torch.cuda.stream(stream):
                flush.fill_(3)
                a_.record(stream)
                graph.replay()
                b_.record(stream)
        stream.synchronize()
        bms = statistics.mean(a_.elapsed_time(b_) for a_, b_ in evs)
        got = bids.cpu().numpy().view(np.uint32)
        rec = {}
        for kk in (1, 10, 100):
            sel = np.where(kq == kk)[0]
            rec["recall@%d" % kk] = round(recall(got[sel, :kk], w["gt_ids"][sel], kk), 4)
        batched = {"value": nq / (bms / 1e3), "unit": "queries/s", "ms_per_step": bms,
                   "launch": "one persistent launch (bang_search_batched) replayed from a CUDA graph",
                   "k_mix": "uniform over {1, 10, 100}", "L_mix": "uniform over {32, 64, 128, 256}, "
                   "at least k", "mean_L": float(Lq.mean()), **rec}

    # ---- end to end through the C ABI: pinned host queries and results
    q_host = torch.from_numpy(w["queries"]).pin_memory()
    ids_h = torch.empty((nq, K), dtype=torch.int32).pin_memory()
    dist_h = torch.empty((nq, K), dtype=torch.float32).pin_memory()
    hp = bang.make_params(bloom_log2=lz, mode=mode, table_source=tsrc, prefetch_depth=depth[0])
    for _ in range(2):
        ix.search(q_host, K, L, ids_h, dist_h, hp, stream=sptr)
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ix.search(q_host, K, L, ids_h, dist_h, hp, stream=sptr)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    search(L, mode, tsrc=tsrc, lz=lz)
    stream.synchronize()
    assert (ids_h.numpy() == ids.cpu().numpy()).all()

    records = bool(head["placement"] & bang.BANG_NODE_RECORDS)   # row and vector in one record
    gather = (row_bytes + d * esz + 31) // 32 * 32 if records else row_bytes
    link = bang.bang_probe_host_link(local, 1 << 30, gather)      # the head's own request size
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_gbs = hbm_bytes / launch_s / 1e9

    def brief(r):
        return {"what": r["what"], "value": r["value"], "ms_per_step": r["ms_per_step"],
                "L": r["L"], "recall@%d" % K: r["recall"], "sweep": r["sweep"],
                "mean_iterations": float(r["iters"].mean()),
                "dist_error_vs_fp64": r["dist_error"]}

    line = {
        "metric": metric_name(), "value": head["value"], "unit": "queries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {1: "bf16-table/f32", 3: "u8-table/int32"}.get(mode, "f32"), "data": "synthetic",
        "config": {"workload": workload_name(args), "form": head["form"], "form_what": head["what"],
                   "L": L, "recall@%d" % K: head["recall"], "k": K,
                   "bloom_log2": lz, "sweep": head["sweep"], "autotune": tune,
                   "mean_iterations": float(it.mean()), "mean_pq_distances": float(nd.mean()),
                   "phase_share": phases,
                   "parallelism": "replica per GPU" if world > 1 else "single GPU",
                   "l2": "512 MB flush written between timed steps",
                   "n": int(w["base"].shape[0]), "nq": nq,
                   "index_build": w.get("index_build", "host generator (workload/)"),
                   "ground_truth": w.get("truth", "host generator (workload/), exact")},
        "plain_form": brief(res["fp32"]),
        "forms": {f: brief(r) for f, r in list(res.items()) + list(variants.items())},
        # the binding roofline of this path is the host link (neighbour rows
        # and full vectors read in place from page-locked host memory); its
        # peak is measured in this run, HBM's comes from MEASURED_PEAKS.json
        "roofline": {"bound": "host_link", "achieved": host_bytes / launch_s / 1e9,
                     "peak": link["gather_gbs"], "unit": "GB/s",
                     "frac": host_bytes / launch_s / 1e9 / link["gather_gbs"],
                     "traffic": NCU_HOST_TRAFFIC.get((mode, lz, L, head["placement"])) if args.n is None
                     else None,
                     "traffic_note": "host sectors x 32 B from the capture of this head's settings"
                                     if args.n is None and (mode, lz, L, head["placement"]) in NCU_HOST_TRAFFIC
                                     else "no capture of this head's settings (mode %d, 2^%d bits, L %d, "
                                          "placement %d)" % (mode, lz, L, head["placement"]),
                     "peak_source": "measured in this run: random %d-byte row gathers in place "
                                    "from mapped host memory over NVLink-C2C" % link["gather_row_bytes"],
                     "algorithmic_bytes_per_launch": host_bytes,
                     "per_unit": "%d B per expansion (%sneighbour row %d B + vector %d B)" % (
                         row_bytes + d * esz, "one record: " if records else "", row_bytes, d * esz),
                     "units_per_launch": int(it.sum())},
        "hbm_roofline": {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": hbm_gbs / hbm_peak,
                         "traffic": NCU_TRAFFIC.get((mode, lz, L, head["placement"])) if args.n is None
                         else None,
                         "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                         "algorithmic_bytes_per_launch": hbm_bytes},
        "host_link": {"copy_engine_gbs": link["h2d_copy_gbs"],
                      "host_threads_gather_gbs": link["cpu_gather_gbs"],
                      "host_threads": link["cpu_threads"],
                      "load_latency_ns": link["latency_ns"],
                      "note": "the paper's path (host threads gather rows, copy engine moves "
                              "them) is bounded by host_threads_gather_gbs"},
        "e2e": {"value": nq / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": nq * d * esz,
                "d2h_bytes_per_step": nq * K * 8},
        "gpu_launches": args.steps * (2 if tsrc else 1),
        "clocks": clk.summary(),
        "wall_s_timed_region": sum(r["t_wall"] for r in res.values()),
    }
    if batched is not None:
        line["batched_form"] = batched
    if not args.no_serving:
        line["serving"] = serving(bang, ix, w, L, mode, head["value"], lz)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, res["fp32"]["L"], min(args.cpu_sample, nq),
                                            args.bloom_log2)
    ix.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
