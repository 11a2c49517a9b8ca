/*
 * bang.h -- C ABI of the GB300 implementation of BANG's search path
 * (Karthik V. et al., "BANG: Billion-Scale Approximate Nearest Neighbor
 * Search using a Single GPU", arXiv 2401.11324).
 *
 * The paper states the problem as: given a graph index G, its medoid s, the
 * PQ distance table of a batch of queries Q and a worklist size t >= k,
 * return k approximate nearest neighbours of every query (Alg. 2).  The data
 * placement follows the paper's schema (§4, first figure): PQ codes on the
 * GPU; graph and full-precision vectors in host memory.  This ABI loads the
 * PQ data, registers the host-resident graph and vectors, and searches.
 *
 * Conventions for every call:
 *  - The return value is a bang_status; BANG_OK (0) on success.  On any
 *    other value, bang_last_error() returns a message for the calling thread
 *    (valid until that thread's next call into the library).
 *  - Pointers are plain host or device addresses.  Arguments documented as
 *    "host or device" are detected with cudaPointerGetAttributes; device
 *    memory must belong to the GPU the call works on (the index's, or the
 *    `device` argument), otherwise the call returns BANG_EINVAL.
 *  - Outputs are allocated by the caller.
 *  - A bang_index is not thread-safe: serialise calls on one index.
 *  - Ids are uint32; 0xFFFFFFFF marks an absent id.  n < 2^31.
 */
#ifndef BANG_H
#define BANG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bang_index bang_index;

typedef enum { BANG_U8 = 0, BANG_I8 = 1, BANG_F32 = 2 } bang_dtype;

typedef enum {
    BANG_OK = 0,
    BANG_EINVAL = -1,   /* an argument is out of range or inconsistent */
    BANG_ENOMEM = -2,   /* a device or pinned-host allocation failed */
    BANG_ECUDA = -3,    /* a CUDA call failed (message names it) */
    BANG_ETIMEOUT = -4, /* a bounded device-side wait gave up */
    BANG_ESTATE = -5    /* the index is missing a step (PQ, graph or vectors) */
} bang_status;

#define BANG_NONE 0xFFFFFFFFu

/* Optional search settings and statistics.  Zero-initialise, then set what
 * you need; a NULL pointer to the struct means all defaults. */
typedef struct bang_search_params {
    /* Bloom filter size z = 2^bloom_log2 bits per query (§4.3; the paper's
     * z is a tuned size, §6.3).  10..20; 0 selects 16. */
    uint32_t bloom_log2;
    /* Safety cap on expansions per query; 0 selects 8*L + 64.  A query that
     * reaches it stops, keeps its re-ranked candidates, and reports status
     * 1 in out_status. */
    uint32_t iter_cap;
    /* Optional per-query outputs (nq entries each), host or device:
     * expansions (the paper's iteration count I, §7.7), status (0 = converged,
     * 1 = stopped by iter_cap, 2 = its tensor-core table could not be built,
     * -1 = its k or L out of range in the batched form), and PQ distances
     * computed (§4.4). */
    uint32_t *out_iters;
    int32_t *out_status;
    uint32_t *out_ndist;
    /* Optional visit trace: the expanded node of every iteration, nq rows
     * of trace_cap entries (host or device); rows are not padded. */
    uint32_t *trace;
    uint32_t trace_cap;
    /* Optional per-query profile, nq rows of 10 SM-cycle counts (host or
     * device): PQ table (§4.1), choice of u*, seen filter (§4.3), PQ
     * distances (§4.4), next-node choice and prefetch (§4.5), re-rank
     * candidate (§4.8), merge remainder, merge ranking of the new keys and
     * merge shifting of the worklist (§4.6-§4.7), and the query's total: the
     * paper's per-kernel GPU-time breakdown (§7.3) for the fused kernel. */
    unsigned long long *out_phase_cycles;
    /* Distance mode (bang_mode): PQ distances from an FP32 table (0, the
     * default, bit-exact with the reference order), from a BF16 table summed
     * in FP32 (1, the reduced-precision form: half the table's shared memory;
     * entries rounded to nearest, ties to even, so also deterministic),
     * or exact distances in the loop without table or re-rank (2, the
     * paper's Exact-distance variant, §5.2; results are the first k entries
     * of the final worklist), or from an 8-bit table summed exactly in
     * integers (3; not in the paper, whose table is FP32: from the FP32
     * table T of a query, lo_s = min_c T[s][c], g = the widest subspace's
     * max - min, entry = min(255, rint((T - lo_s) * (255 / g))), all in FP32;
     * a quarter of the FP32 table's shared memory; bit-exact with the
     * reference order like mode 0). */
    uint32_t mode;
    /* bang_search_batched only: the persistent grid is grid_mult times the
     * CTAs that fit on the device at once (0 or 1: exactly that many). */
    uint32_t grid_mult;
    /* Where the PQ tables of modes 0 and 1 come from: 0 = built by each
     * query's warp on CUDA cores (mode 0: bit-exact); 1 = built for the whole
     * batch by the tensor-core kernel of bang_pq_tables (three-way BF16
     * splits, about FP32-accurate) into per-stream device scratch owned by the
     * index (nq*M*256 entries of 4 bytes in mode 0, 2 in mode 1), then read by
     * the search; 2 = the same with both operands rounded to TF32 (the
     * numerics of a TF32 GEMM with FP32 accumulation: the TF32 table form);
     * 3 = no table (mode 0 only): each FP32 entry a PQ distance needs is
     * computed from the query and the codebook (read through the L1 cache)
     * in the table build's own order, so results are bit-exact with
     * table_source 0, while a query holds no M*256*4-byte table in shared
     * memory and more queries are resident per SM (table_subspaces below
     * keeps part of the table).  Also accepted by bang_search_batched_noalloc. */
    uint32_t table_source;
    /* How many candidates for the next node are requested per iteration: 0
     * or 1 = the chosen one only, after the distances (§4.5's eager choice);
     * 2 = also the first unvisited worklist entry after u*, at the start of
     * the iteration (used when it is chosen, wasted otherwise).  Results do
     * not depend on it. */
    uint32_t prefetch_depth;
    /* When the new neighbours' PQ code rows are requested: 0 = after the seen
     * filter, only the new ones; 1 = every neighbour's row as soon as the
     * expanded node's row arrives, so that the filter runs while they are in
     * flight (used when R <= 64, d <= 128 and M <= 32, and without
     * BANG_NEIGHBOR_CODES; otherwise ignored).  Results do not depend on it. */
    uint32_t early_codes;
    /* How the re-rank of §4.8 runs (modes 0, 1 and 3; mode 2 has none):
     * 0 = fused into the loop (each expanded node's vector arrives with its
     * row and its exact distance enters the top-k at once); 1 = staged, as the
     * paper structures it: the search fetches no vectors and records every
     * expanded node (the candidate set) in device scratch owned by the index,
     * one list per query as long as the iteration cap (nq * iter_cap * 4
     * bytes per stream; iter_cap 0 counts as 8*L + 64), then a separate
     * kernel computes the candidates' exact distances and keeps the k
     * nearest.  Both return the k smallest (distance, id) keys of the same
     * candidates in the same arithmetic: the results are identical; 2 =
     * staged over the final worklist only (its L entries, ordered by PQ
     * distance, including entries a capped search left unexpanded): the
     * reading of §4.8's candidates as the top-L, fewer candidates and so
     * possibly lower recall than 0 and 1.  Not accepted by
     * bang_search_batched_noalloc.  Any other value: BANG_EINVAL. */
    uint32_t rerank;
    /* Preferred share of each SM's unified L1/shared storage given to shared
     * memory, in percent (1..100; 0 = the CUDA driver's choice; above 100:
     * BANG_EINVAL).  A hint that trades resident queries against L1 capacity
     * (the codebook, for table_source 3); results do not depend on it. */
    uint32_t smem_carveout;
    /* With table_source 3: how many subspaces, the first ones, keep their
     * FP32 entries in shared memory (table_subspaces*256*4 bytes per query);
     * the others are computed when needed.  0 = none; M or more = all (the
     * table form's memory, computed the same way).  Results do not depend
     * on it (bit-exact with mode 0). */
    uint32_t table_subspaces;
} bang_search_params;

typedef enum { BANG_MODE_PQ_F32 = 0, BANG_MODE_PQ_BF16 = 1, BANG_MODE_EXACT = 2,
               BANG_MODE_PQ_Q8 = 3 } bang_mode;

/* Placement flags for bang_set_placement. */
enum { BANG_GRAPH_IN_HBM = 1, BANG_VECTORS_IN_HBM = 2, BANG_GRAPH_PACKED = 4, BANG_NEIGHBOR_CODES = 8,
       BANG_NODE_RECORDS = 16 };

/* Create an empty index bound to CUDA device `device`.  *out receives an
 * opaque handle owned by the library; free it with bang_destroy. */
int bang_create(int device, bang_index **out);

/* Load the PQ codebooks and codes (§4: m subspaces of the d dimensions,
 * 256 centroids each; a point is stored as its m centroid ids) to the device.
 *   d, M      dimensions and subspaces, 1 <= M <= min(d, 128), d <= 512.
 *             Subspace s covers dimensions [off_s, off_(s+1)) with
 *             off_s = s*(d/M) + min(s, d%M): the first d%M subspaces take one
 *             extra dimension.
 *   codebook  host, 256*d floats: subspace s occupies the 256*dsub_s floats
 *             starting at 256*off_s, centroid c at offset c*dsub_s in it.
 *   codes     host, n*M bytes, row-major.
 *   n         points, 1 <= n < 2^31.
 * The library copies both; the caller may free them on return.  Replaces
 * earlier PQ data and requires graph and vectors to be registered again. */
int bang_load_pq(bang_index *ix, uint32_t d, uint32_t M, const float *codebook,
                 const uint8_t *codes, uint64_t n);

/* Register the graph (the Vamana index of §2.2, kept in host memory as in
 * Alg. 2, where the CPU serves the neighbour lists).
 *   adj     host, n*R ids (n from bang_load_pq), row i = out-neighbours of i;
 *           unused slots hold 0xFFFFFFFF.  Ids must be < n, distinct within
 *           a row and differ from the row's own id.
 *   R       row width, 1..128.
 *   medoid  entry point s of the search (§6.3), < n.
 * Not copied when `adj` starts on a 128-byte boundary: the memory must then
 * stay valid and unchanged until bang_destroy or the next
 * bang_register_graph; the library page-locks it with cudaHostRegister
 * unless it is already page-locked, and the GPU reads it in place.  A
 * pointer off that boundary (numpy places large arrays 16 bytes past a page)
 * is copied once into aligned page-locked memory owned by the index, since a
 * misaligned 256-byte row costs 9 32-byte sectors on the host link instead
 * of 8; the caller may then free its copy.  BANG_ENOMEM if that copy cannot
 * be allocated.  Invalid ids return BANG_EINVAL (checked here, not at
 * search). */
int bang_register_graph(bang_index *ix, const uint32_t *adj, uint32_t R, uint32_t medoid);

/* Register the full-precision vectors used by the re-rank (§4.8), host
 * memory, n*d elements of `dtype`, row-major.  Same ownership and alignment
 * rule as the graph.  Queries passed to bang_search have the same element
 * type. */
int bang_register_vectors(bang_index *ix, const void *base, bang_dtype dtype);

/* Search a batch of nq queries (Alg. 2; one query per warp): PQ distance
 * table (§4.1), greedy search from the medoid with a Bloom-filter seen set
 * (§4.3), PQ distances of new neighbours (§4.4), eager choice of the next
 * node (§4.5), sorted merge into the worklist of L entries (§4.6, §4.7),
 * and re-rank of every expanded node by exact squared L2 distance (§4.8).
 *   queries   host or device, nq*d elements of the registered dtype.
 *   k, L      1 <= k <= 256, k <= L <= 1024 (L is the paper's t).
 *   params    may be NULL.
 *   out_ids   host or device, nq*k ids sorted by (distance, id); padded
 *             with 0xFFFFFFFF when fewer than k nodes were expanded.
 *   out_dist  host or device, nq*k squared L2 distances (+inf padding).
 *   stream    a cudaStream_t (NULL = the legacy default stream).
 * Work is ordered on `stream`.  If every pointer argument is device memory
 * the call returns after enqueueing; otherwise it copies through device
 * staging buffers and returns after the stream has finished.
 * Ties: distances are compared first, then ids. */
int bang_search(bang_index *ix, const void *queries, uint32_t nq, uint32_t k, uint32_t L,
                const bang_search_params *params, uint32_t *out_ids, float *out_dist,
                void *stream);

/* Batched form: queries with their own k and L in one persistent launch.
 *   k_per_q, L_per_q  host or device, nq entries each; query i needs
 *                     1 <= k_i <= k_max and k_i <= L_i <= L_max (otherwise its
 *                     row is padded and out_status[i] = -1).
 *   k_max, L_max      bounds (as bang_search's k, L); they size the shared
 *                     memory and the output rows: out_ids and out_dist are
 *                     nq*k_max, row i holding k_i results then padding.
 * A grid of resident CTAs pulls queries from a device work counter; when
 * L_per_q is host memory the queries are handed out by decreasing L.  With
 * every pointer argument in device memory the call only enqueues work
 * (cudaMemsetAsync + one kernel) and can be captured in a CUDA graph; make one
 * call with the same stream outside the capture first, since the first call
 * on a stream allocates its 256-byte work counter.  Calls in flight on
 * different streams use separate counters. */
int bang_search_batched(bang_index *ix, const void *queries, uint32_t nq, const uint32_t *k_per_q,
                        const uint32_t *L_per_q, uint32_t k_max, uint32_t L_max,
                        const bang_search_params *params, uint32_t *out_ids, float *out_dist,
                        void *stream);

/* Allocation-free batched search (the paper has no counterpart).  Same
 * arguments, results and per-query rules as bang_search_batched, for callers
 * that cannot let a library allocate device memory: a serving loop that must
 * not stall on the device-wide synchronisation cudaMalloc/cudaFree can cause,
 * work recorded into a CUDA graph under global stream capture (allocations
 * are refused there), or a framework that owns the whole memory budget.
 *   - Allocates nothing (no cudaMalloc/cudaFree, no pinned or staging
 *     buffers): every pointer argument must already be device memory,
 *     otherwise BANG_EINVAL.
 *   - Its scratch (the persistent launch's work counter and the
 *     longest-L-first query order, computed on the device) is a file-scope
 *     device array of about 270 KB that every GPU loading the library keeps
 *     until exit; nq above 65536 (its capacity) returns BANG_EINVAL.
 *   - The first call on a device looks up that array's device address; make
 *     it before any stream capture.  The address is kept for the life of the
 *     process: it does not survive cudaDeviceReset on that device (the
 *     reset destroys the context the array lives in), so a process that
 *     resets a device must not call this entry point on it afterwards.
 *   - Every pointer must be device memory of the index's GPU (or managed
 *     memory); device memory of another GPU returns BANG_EINVAL.
 *   - All calls share the array: calls that overlap on the GPU (on different
 *     streams, or different indexes at once) race and must not be issued.
 *     Each call clears the counter it needs and rewrites the order.
 * Enqueues two kernels on `stream` and returns. */
int bang_search_batched_noalloc(bang_index *ix, const void *queries, uint32_t nq,
                                const uint32_t *k_per_q, const uint32_t *L_per_q, uint32_t k_max,
                                uint32_t L_max, const bang_search_params *params,
                                uint32_t *out_ids, float *out_dist, void *stream);

/* Choose where the search reads the graph and the full vectors: 0 keeps
 * both in host memory, read in place (Alg. 2); BANG_GRAPH_IN_HBM and/or
 * BANG_VECTORS_IN_HBM copy the registered arrays into device memory once
 * (the paper's In-memory variant, §5.1; BANG_MODE_EXACT usually wants the
 * vectors there too).  The copies are owned by the library and dropped when
 * the corresponding array is registered again or the flag is cleared.
 * BANG_GRAPH_PACKED (not in the paper, whose rows hold 32-bit ids) makes the
 * search read a copy of the graph with every id packed into b bits, b the
 * fewest with 2^b - 1 >= n (the all-ones value marks an empty slot), rows
 * padded to 32 bytes: 160 bytes instead of 256 per row at n = 1M, R = 64, so
 * fewer bytes cross the host link per expansion (in HBM with
 * BANG_GRAPH_IN_HBM).  The copy is page-locked host memory owned by the
 * index, built once from the registered rows; results are unchanged.
 * BANG_NEIGHBOR_CODES (not in the paper) keeps in HBM, for every node, the PQ
 * code rows of its R neighbours side by side (n*R*32 bytes: 2 GB at n = 1M,
 * R = 64), so that the codes of the next node's neighbours are requested
 * together with its row instead of after it; needs R <= 64, d <= 128 and
 * M <= 32; results are unchanged.
 * BANG_NODE_RECORDS (not in the paper) makes the search read a page-locked
 * copy, owned by the index, in which each node's neighbour row (packed when
 * BANG_GRAPH_PACKED is also set) and its full vector lie side by side, the
 * record padded to 32 bytes: one expansion then reads one contiguous record
 * (288 bytes at n = 1M, R = 64, d = 128 u8 with packed rows) instead of a row
 * and a vector at two places.  Not with BANG_GRAPH_IN_HBM or
 * BANG_VECTORS_IN_HBM (BANG_EINVAL); results are unchanged.
 * Blocks until the copies are done.  BANG_ENOMEM if the device or the host
 * memory is full. */
int bang_set_placement(bang_index *ix, uint32_t flags);

/* PQ distance tables of nq queries on the tensor cores (§4.1 as a dense
 * queries x centroids contraction: tcgen05 MMAs with BF16 high/low operand
 * splits and FP32 accumulation, about FP32-accurate):
 * out[q][s][c] = ||q_s - C_s[c]||^2, M x 256 per query, FP32 or (bit 0 of
 * out_bf16) BF16; bit 1 of out_bf16 rounds both operands to TF32 first (a
 * TF32 value is two exact BF16 parts, so the products are those of a TF32
 * GEMM).  queries and out are device memory; waits for the stream.  Needs the
 * vectors registered (for the element type); BANG_EINVAL if a subspace
 * spans more than 4 blocks of 16 dimensions; BANG_ETIMEOUT if a bounded
 * tensor-core wait gave up. */
int bang_pq_tables(bang_index *ix, const void *queries, uint32_t nq, void *out, uint32_t out_bf16,
                   void *stream);

/* Sizes of a loaded index (any pointer may be NULL); dtype is a bang_dtype,
 * -1 before bang_register_vectors. */
int bang_index_info(const bang_index *ix, uint64_t *n, uint32_t *d, uint32_t *M, uint32_t *R,
                    int32_t *dtype);

/* ---- Index build on the GPU.  The paper searches an index built
 * beforehand (its graph comes from DiskANN, §1; PQ with 256 centroids per
 * subspace, §4); these calls build the same kinds of arrays on the device.
 *
 * Clustered graph: for every cluster (members listed in ascending id, local
 * position b = index within the cluster):
 *   1. candidates of member a: the K = min(2 Rin, m - 1) other members
 *      nearest to a by (distance, b), with Rin = R - nx;
 *   2. RobustPrune (Vamana, §2.2): in (distance, b) order a live candidate is
 *      kept (at most Rin) and removes every later candidate j with
 *      alpha^2 * d(kept, j) <= d(a, j), alpha^2 and the product in FP32;
 *   3. the kept list plus every member that kept a, pruned again;
 *   4. repair, members in ascending b: a member nobody links to (with
 *      neighbours of its own) is appended to the first of its neighbours with
 *      room, or replaces that neighbour's last entry when that entry's target
 *      keeps another in-link;
 *   5. row of member a: its list (a cluster medoid keeps at most R - nh),
 *      then medoids[xclu[a][t]] for t < nx (for a cluster medoid
 *      medoids[hclu[g][t]], t < nh), skipping its own cluster, ids >= ng and
 *      medoids 0xFFFFFFFF; repeated ids dropped keeping the first; padding
 *      0xFFFFFFFF.
 * Distances are squared L2 rounded to FP32: integer data summed exactly then
 * converted; f32 summed in ascending dimension order, each difference,
 * product and sum rounded (no fused multiply-add).  Deterministic: the same
 * inputs give the same bytes on any run.
 *   base     n*d elements of dtype, host or device.
 *   members  host, n ids: a permutation of 0..n-1 grouped by cluster, each
 *            cluster in ascending id; gstart host, ng+1 offsets from 0 to n.
 *   medoids  host, ng ids (< n, or 0xFFFFFFFF for none).
 *   xclu     host, n*nx cluster ids (row = point id); hclu host, ng*nh.
 *   adj      n*R output, host or device.
 * Limits: R <= 128, nx < R, nh < R, rows of at most 2048 bytes.  Allocates
 * its own device scratch (about n*(d*elem + 12*Rin + 40) bytes) and blocks
 * until done on `stream`.  BANG_EINVAL for inconsistent index arrays. */
int bang_build_cluster_graph(int device, const void *base, bang_dtype dtype, uint64_t n, uint32_t d,
                             const uint32_t *members, const uint64_t *gstart, uint32_t ng,
                             const uint32_t *medoids, uint32_t R, float alpha, uint32_t nx,
                             const uint32_t *xclu, uint32_t nh, const uint32_t *hclu,
                             uint32_t *adj, void *stream);

/* Overlapping-shard graph (§2.2: the paper's Vamana index is built by
 * splitting the dataset into smaller overlapping clusters, building a
 * directed subgraph on each with GreedySearch and RobustPrune, and merging
 * the subgraphs' edges), in a batched form whose result does not depend on
 * thread scheduling:
 *   1. point i joins the shards of its ell nearest centres (FP32 squared
 *      distance over ascending dimensions, each difference, product and sum
 *      rounded; ties to the smaller centre index);
 *   2. shard g lists its members in ascending id; its entry is the member
 *      nearest its centre (same distance; ties to the smaller id); it
 *      inserts the entry first, then the other members in ascending id
 *      (callers whose ids follow the data's structure shuffle the rows);
 *   3. two passes, pruning parameter 1 then alpha; a pass cuts every shard's
 *      insertion order into batches (pass 1: 1, 1, 2, 4, ... up to
 *      cap = max(1, floor(batch_frac * m)), pass 2: cap each) and batch r of
 *      every shard forms round r.  In a round, against the graph as it stood
 *      at the round's start, every member runs GreedySearch from its shard's
 *      entry (Alg. 1 with exact distances as in BANG_MODE_EXACT, worklist Lb,
 *      a 2^log2z-bit Bloom seen set, at most iter_cap expansions); its list
 *      becomes RobustPrune(member, expanded nodes U its current list); then
 *      every node named by a new list takes the members that named it: the
 *      union sorted by distance when it fits in R, else RobustPrune'd;
 *   4. point i's row is the union of its shard lists, sorted when it fits
 *      in R, else RobustPrune'd with alpha.
 * Distances are the exact squared L2 of the search's Exact-distance mode
 * rounded to FP32; lists are sorted by (distance, id) without repeats or the
 * owner and cut to their 750 nearest (the bound DiskANN puts on the
 * candidate pool; only reverse edges into hub nodes reach it).  RobustPrune
 * keeps, in that order, each live candidate (at most R)
 * and removes every later candidate c with a^2 * d(kept, c) <= d(owner, c),
 * a^2 and the product in FP32.  Rows are written sorted, 0xFFFFFFFF padding.
 *   base      n*d elements of dtype, host or device; n*ell < 2^31 - 1.
 *   centres   host, S*d floats; ell in 1..min(4, S).
 *   R         multiple of 4 in 4..128, ell*R <= 512.  Lb 1..1024; log2z
 *             10..20; iter_cap 0 selects 2*Lb + 64, and iter_cap + R <= 512;
 *             alpha >= 1; 0 < batch_frac <= 1.
 *   adj       n*R output, host or device.  shard_of: host, n*ell, may be NULL
 *             (each point's shards, nearest centre first).
 * Device memory: about n*ell*(R*4 + d*elem rounded to 16, then to 32 bytes
 * per record) plus per-round scratch (about 40*R bytes per member of the
 * largest round, and 8 bytes per candidate of the longest reverse-edge
 * lists).  Blocks until done. */
int bang_build_shard_graph(int device, const void *base, bang_dtype dtype, uint64_t n, uint32_t d,
                           const float *centres, uint32_t S, uint32_t ell, uint32_t R, uint32_t Lb,
                           float alpha, float batch_frac, uint32_t log2z, uint32_t iter_cap,
                           uint32_t *adj, uint32_t *shard_of, void *stream);

/* PQ codebook and codes on the GPU (§4): M contiguous subspaces, the first
 * d mod M one dimension wider (§6.3); 256 centroids per subspace by k-means:
 * centroids start at the points init[s*256 + c]; each of `iters` Lloyd
 * iterations assigns every training point (rows `sample`) to its nearest
 * centroid (FP64 distance in ascending dimension order, each difference,
 * product and sum rounded; ties to the smaller centroid) and moves each
 * centroid to the FP64 mean of its points summed in sample order (no points:
 * it stays).  The FP32 codebook (256*d floats; subspace s at 256*off[s],
 * centroid c at +c*dsub_s) then encodes all n points the same way (codes
 * n*M).  Deterministic.  base host or device; sample (ns ids) and init
 * (M*256 ids) host, all < n; codebook and codes host or device.  Subspaces
 * of at most 16 dimensions.  Blocks until done. */
int bang_build_pq(int device, const void *base, bang_dtype dtype, uint64_t n, uint32_t d, uint32_t M,
                  const uint64_t *sample, uint64_t ns, const uint64_t *init, uint32_t iters,
                  float *codebook, uint8_t *codes, void *stream);

/* Exact k nearest neighbours of nq queries among n points on the GPU: the
 * ground truth of k-recall@k (§6.3).  Squared L2; integer data exact; f32 in
 * FP64, summed in ascending dimension order with each difference, product and
 * sum rounded; sorted by (distance, id), padded with 0xFFFFFFFF / +inf when
 * n < k.  base (n*d) and queries (nq*d) host or device, of dtype; out_ids and
 * out_dist (nq*k) both host or both device.  k <= 256, d <= 4096.  Allocates
 * device scratch (about nq*k*24*ceil(n/262144) bytes plus copies of host
 * inputs) and blocks until done. */
int bang_ground_truth(int device, const void *base, const void *queries, bang_dtype dtype, uint64_t n,
                      uint32_t nq, uint32_t d, uint32_t k, uint32_t *out_ids, double *out_dist,
                      void *stream);

/* ---- Autotuner (not in the paper).  Picks, for this GPU and index, the
 * settings that change speed but not the method: the PQ table's precision
 * (bang_mode; bit m of `modes` admits mode m), whether mode 1's tables come
 * from the tensor cores (table_source), the Bloom filter size 2^bloom_log2
 * (the paper's z, §4.3), for the batched form the persistent grid
 * multiple, and optionally the graph layout (BANG_GRAPH_PACKED,
 * BANG_NEIGHBOR_CODES; the index's placement is restored on return).  Every candidate searches the given queries on `stream`; its
 * accuracy is recall@k against `truth` (host, nq*k ids; 0xFFFFFFFF entries
 * are skipped) or, when truth is NULL, against an FP32 search with worklist
 * 2L (at most 1024) and a 2^18-bit filter.  Speed is the mean of `reps`
 * CUDA-event-timed launches after one warm-up.
 *   target_recall 0: L is fixed (k <= L <= 1024); a candidate qualifies when
 *                 its recall is at least the FP32 form's (mode 0, 2^16 bits)
 *                 minus recall_tolerance (default 0.005).
 *   target_recall in (0, 1]: every candidate takes the smallest worklist of
 *                 {16, 24, 32, 48, 64, 80, 96, 112, 128, 160, 192, 224, 256,
 *                 288, 320, 384, 512, 768, 1024} (at least k, at most L unless
 *                 L is 0) whose
 *                 recall reaches the target.
 * The fastest qualifying candidate is returned in *out with its L, time and
 * recall, beside the FP32 form's (ref_ms, ref_recall at its own L).  With
 * cache_path set, a decision is looked up first (JSON lines keyed by GPU
 * name and SM count, index shape, placement, nq, k, L and the options) and
 * appended after tuning.  Defaults (0): modes 0, 1 and 3; Bloom 2^13..2^17;
 * reps 3.  Allocates its own scratch; blocks until done.  BANG_EINVAL when
 * no candidate qualifies. */
typedef struct bang_autotune_opts {
    uint32_t modes;              /* bit mask over bang_mode; 0 = modes 0, 1, 3 */
    uint32_t bloom_min, bloom_max;   /* log2 filter sizes tried; 0 = 13, 17 */
    uint32_t try_tensor_tables;  /* also try table_source 1 with mode 1 */
    uint32_t batched;            /* tune bang_search_batched (grid_mult 1, 2, 4) */
    uint32_t reps;               /* timed launches per candidate; 0 = 3 */
    float target_recall;         /* 0: fixed L; else the recall to reach */
    float recall_tolerance;      /* fixed L: allowed recall loss; 0 = 0.005 */
    const char *cache_path;      /* JSON-lines decision cache, or NULL */
    uint32_t try_packed_graph;   /* also try BANG_GRAPH_PACKED rows */
    uint32_t try_neighbor_codes; /* also try BANG_NEIGHBOR_CODES (where the index allows it) */
    uint32_t try_prefetch_depth; /* also time the winner with prefetch_depth 2 */
    uint32_t try_node_records;   /* also time the winner with BANG_NODE_RECORDS (host placement only) */
    uint32_t try_structure;      /* also time the winner with early code rows, then with the
                                    re-rank staged (rerank 1): both leave the results unchanged */
} bang_autotune_opts;

typedef struct bang_autotune_result {
    uint32_t mode, bloom_log2, table_source, grid_mult, L;
    float ms, recall;            /* chosen settings: ms per batch, recall@k */
    float ref_ms, ref_recall;    /* FP32 form, 2^16-bit filter */
    uint32_t candidates;         /* candidates evaluated */
    uint32_t from_cache;         /* 1 when read from cache_path */
    uint32_t graph_packed;       /* 1: the choice reads packed rows (set the flag) */
    uint32_t neighbor_codes;     /* 1: the choice uses the neighbour-code layout (set the flag) */
    uint32_t prefetch_depth;     /* 1 or 2 (bang_search_params.prefetch_depth) */
    uint32_t node_records;       /* 1: the choice reads node records (set BANG_NODE_RECORDS) */
    uint32_t early_codes;        /* bang_search_params.early_codes of the choice */
    uint32_t rerank;             /* bang_search_params.rerank of the choice (0 or 1) */
} bang_autotune_result;

int bang_autotune(bang_index *ix, const void *queries, uint32_t nq, uint32_t k, uint32_t L,
                  const uint32_t *truth, const bang_autotune_opts *opts, bang_autotune_result *out,
                  void *stream);

/* ---- Serving: continuous batching (north of the paper's batch-at-a-time
 * evaluation, §6.2 runs one batch of 10,000 queries).  Admission is by device
 * memory: a server owns a device arena of mem_bytes (and a page-locked host
 * mirror of it) allocated at start; a dispatcher thread packs pending
 * requests, in arrival order, into one bang_search_batched launch (at most
 * max_batch queries) as soon as one of `streams` streams is free and the
 * arena has room for the batch's queries and results; a request that does
 * not fit waits until earlier launches release their memory (first in,
 * first out).  Launches on different streams overlap on the GPU.  Results
 * are identical to searching each request alone with the same k, L and
 * settings. */
typedef struct bang_server bang_server;
typedef struct bang_server_config {
    uint32_t k_max, L_max;   /* bounds of every request's k and L */
    uint32_t max_batch;      /* queries per launch, and per request, at most */
    uint32_t streams;        /* slots (launches in flight at once), 1..16 */
    uint32_t mode;           /* bang_mode of the searches */
    uint32_t bloom_log2;     /* as bang_search_params (0 = 16) */
    uint64_t mem_bytes;      /* device bytes for batches in flight (0: room for `streams`
                                full batches); a batch of nq queries takes about
                                nq * (d * elem + 8 + 8 * k_max) bytes */
    uint32_t early_codes;    /* as bang_search_params (0 or 1) */
} bang_server_config;

/* Start a server on the calling thread's current device for a fully loaded
 * index (which must outlive the server).  While the server runs, its
 * dispatcher thread is the index's caller: make no other call on that index
 * until bang_server_stop returns.  BANG_ENOMEM if the arena does not fit. */
int bang_server_start(bang_index *ix, const bang_server_config *cfg, bang_server **out);
/* Queue nq (1..max_batch) host queries with their k and L (host arrays,
 * copied before return); *ticket identifies the request.  BANG_EINVAL if the
 * request alone needs more than mem_bytes. */
int bang_server_submit(bang_server *s, const void *queries, uint32_t nq, const uint32_t *k_per_q,
                       const uint32_t *L_per_q, uint64_t *ticket);
/* Wait up to timeout_ms (negative: no limit) for a request, copy its results
 * (nq*k_max ids and distances, rows padded as bang_search_batched) to host
 * memory and release the ticket; *latency_ms = submit to results in host
 * memory.  BANG_ETIMEOUT leaves the ticket valid. */
int bang_server_wait(bang_server *s, uint64_t ticket, int32_t timeout_ms, uint32_t *out_ids,
                     float *out_dist, double *latency_ms);
/* Finish queued and running requests, then free the server. */
int bang_server_stop(bang_server *s);

/* Release device memory, unregister host memory registered by the library
 * and free the handle.  NULL is accepted. */
int bang_destroy(bang_index *ix);

/* Host memory for the graph and the vectors that the paper keeps in host
 * memory (§4, schema figure): an anonymous mapping of `bytes` (> 0), aligned
 * to the system's transparent-huge-page size and advised for huge pages
 * before it is first touched, so that where the system allows it (Linux
 * transparent huge pages in "madvise" or "always" mode) the GPU's reads of
 * the registered memory need far fewer address translations and reach far
 * more host memory at full speed (the host-placement search of 60M and 200M
 * points ran 2.0x and 2.2x as fast).  The library's own host copies (packed
 * rows, node records, aligned copies) use the same memory.  Fill it, then
 * pass it to bang_register_graph / bang_register_vectors as usual.  *out
 * receives the memory (zero-filled); BANG_ENOMEM if the mapping fails.  The
 * paper has no counterpart: it says where its host arrays should live. */
int bang_host_alloc(uint64_t bytes, void **out);
/* Unmap memory from bang_host_alloc, after every index that registered it
 * has been destroyed.  NULL is accepted; any other pointer is BANG_EINVAL. */
int bang_host_free(void *p);

/* Measured figures of the link between the GPU and host memory (the paper's
 * PCIe 4.0 link, 32 GB/s peak, §6.1; NVLink-C2C on a Grace-hosted GB300). */
typedef struct bang_link_probe {
    double h2d_copy_gbs;        /* copy engine: page-locked host -> device, best of 3 */
    double gather_gbs;          /* kernel reads of random rows in place from mapped host memory */
    double latency_ns;          /* one dependent 4-byte load from mapped host memory */
    uint32_t gather_row_bytes;  /* row size used for gather_gbs */
    double cpu_gather_gbs;      /* host threads gathering random rows into a page-locked
                                   staging buffer: the paper's FetchNeighbors path (Alg. 2),
                                   whose rows would then cross by copy engine */
    uint32_t cpu_threads;       /* threads used for cpu_gather_gbs */
} bang_link_probe;

/* Measure the host link of `device` with a page-locked buffer of `bytes`
 * (>= 1 MiB) that the call allocates and frees; `row_bytes` (16..512, a
 * multiple of 16) is the gathered row size, e.g. R*4 for a neighbour row.
 * Blocks until done; takes about bytes/10 GB/s plus a few milliseconds. */
int bang_probe_host_link(int device, uint64_t bytes, uint32_t row_bytes, bang_link_probe *out);

/* Message for the last non-OK status returned to the calling thread. */
const char *bang_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BANG_H */
