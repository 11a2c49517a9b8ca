/*
 * CPU oracle for the BANG search path (arXiv 2401.11324).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct
 * restatement of what the search path computes, one query at a time, written
 * from the paper.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  The product path never links, imports or
 * calls it, and it shares no code, header, table or constant generator with
 * the CUDA implementation.
 *
 * Precision: the graph search decides integers (which node is expanded next)
 * from floating-point comparisons, so those decisions are taken in FP32, the
 * precision of the GPU kernel, with the summation orders stated below.  Ground
 * truth (brute force) is FP64, or exact integers for integer data.
 *
 * Build with -ffp-contract=off: every fused multiply-add below is an explicit
 * fmaf(); nothing else may be contracted.
 *
 * Functions, and the passage of the paper each one follows:
 *   orc_chunk_offsets        §4 (PQ splits d into m contiguous subspaces)
 *   orc_pq_train             §4 (independent k-means per subspace, 256 centroids)
 *   orc_pq_encode            §4 (a point is the list of its per-subspace cluster ids)
 *   orc_medoid               §6.3 (the search starts from the medoid)
 *   orc_robust_prune         §2.2 (Vamana RobustPrune with the pruning parameter)
 *   orc_vamana_build         §2.2, §6.3 (R, L, pruning parameter): two passes
 *                            (parameter 1, then alpha) of GreedySearch +
 *                            RobustPrune + reverse edges; pinned by hand-worked
 *                            builds (a chain, a reverse-edge overflow, an edge
 *                            the second pass restores) and invariants
 *   orc_shard_graph          §2.2 (the index is built on overlapping clusters
 *                            with GreedySearch and RobustPrune and the subgraphs'
 *                            edges merged), in a batched form
 *   orc_cluster_graph        the clustered construction of the large synthetic
 *                            indexes (per-cluster candidates, RobustPrune of §2.2,
 *                            reverse edges, medoid links); not from the paper
 *   orc_adc_table_f32        §4.1 (PQDistTable: squared distance of each query
 *                            sub-vector to each centroid)
 *   orc_adc_dist_f32         §4.4 (asymmetric distance = sum of table entries)
 *   orc_adc_table_bf16       the table rounded to BF16 (not in the paper)
 *   orc_adc_table_q8/_dist_q8 an 8-bit form of the §4.1 table that the paper
 *                            does not have (its table is FP32): per-subspace
 *                            offset, one scale per query, integer sums
 *   orc_fnv1a32/_fnv1a64     §4.3, §6.3 (two FNV-1a hash functions)
 *   orc_bloom_*              §4.3 (per-query Bloom filter of visited nodes)
 *   orc_exact_dist           §4.8 (exact distance used by the re-rank)
 *   orc_search               Alg. 1, Alg. 2, §4.3-§4.8; mode 1: the Exact-distance
 *                            variant of §5.2 (exact distances, no table, no re-rank);
 *                            mode 2: mode 0 with the 8-bit table; mode 3: with the
 *                            BF16 table; orc_search_rr: the re-rank candidates
 *                            are the expanded nodes (§4.8) or the final worklist
 *   orc_bruteforce_knn       §6.3 (ground truth S for k-recall@k)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "bang_oracle.h"

#define ORC_NONE 0xFFFFFFFFu

/* ---------------------------------------------------------------------- */
/* element access                                                          */
/* ---------------------------------------------------------------------- */

static float elem_f(const void *v, int dtype, uint64_t i)
{
    if (dtype == ORC_U8) return (float)((const uint8_t *)v)[i];
    if (dtype == ORC_I8) return (float)((const int8_t *)v)[i];
    return ((const float *)v)[i];
}

static int32_t elem_i(const void *v, int dtype, uint64_t i)
{
    if (dtype == ORC_U8) return (int32_t)((const uint8_t *)v)[i];
    return (int32_t)((const int8_t *)v)[i];
}

/* ---------------------------------------------------------------------- */
/* PQ layout (§4): d dimensions split into M contiguous subspaces.  When M  */
/* does not divide d (the paper's m=74 with d=128), the first d%M           */
/* subspaces take one extra dimension.                                      */
/* ---------------------------------------------------------------------- */

void orc_chunk_offsets(uint32_t d, uint32_t M, uint32_t *off)
{
    uint32_t base = d / M, extra = d % M, s;
    off[0] = 0;
    for (s = 0; s < M; s++) off[s + 1] = off[s] + base + (s < extra ? 1u : 0u);
}

/* Codebook layout: subspace s owns the 256 * dsub_s floats starting at
 * 256 * off[s]; centroid c of subspace s starts at 256*off[s] + c*dsub_s. */
static const float *centroid(const float *cb, const uint32_t *off, uint32_t s, uint32_t c)
{
    uint32_t ds = off[s + 1] - off[s];
    return cb + (size_t)256 * off[s] + (size_t)c * ds;
}

/* ---------------------------------------------------------------------- */
/* PQ training (§4): k-means with 256 centroids in every subspace.          */
/* The seeded choices (training sample, initial centroids) are inputs.     */
/* Lloyd iterations with FP64 sums; an empty cluster keeps its centroid;   */
/* assignment ties go to the smaller centroid id.  obj_trace (optional,    */
/* M*iters entries) receives, for every subspace and iteration, the       */
/* objective sum_i min_c ||x_i - c||^2 of the assignment step.            */
/* ---------------------------------------------------------------------- */

int orc_pq_train(const float *X, uint32_t d, uint32_t M, const uint32_t *off,
                 const uint64_t *sample, uint64_t ns, const uint64_t *init,
                 uint32_t iters, float *codebook, double *obj_trace)
{
    uint32_t s, it, c, j;
    uint64_t i;
    for (s = 0; s < M; s++) {
        uint32_t o = off[s], ds = off[s + 1] - off[s];
        double *cent = (double *)malloc(sizeof(double) * 256 * ds);
        double *sums = (double *)malloc(sizeof(double) * 256 * ds);
        uint64_t *cnt = (uint64_t *)malloc(sizeof(uint64_t) * 256);
        if (!cent || !sums || !cnt) { free(cent); free(sums); free(cnt); return -1; }
        for (c = 0; c < 256; c++)
            for (j = 0; j < ds; j++)
                cent[c * ds + j] = (double)X[init[c] * (uint64_t)d + o + j];
        for (it = 0; it < iters; it++) {
            double obj = 0.0;
            memset(sums, 0, sizeof(double) * 256 * ds);
            memset(cnt, 0, sizeof(uint64_t) * 256);
            for (i = 0; i < ns; i++) {
                const float *x = X + sample[i] * (uint64_t)d + o;
                double best = INFINITY;
                uint32_t bc = 0;
                for (c = 0; c < 256; c++) {
                    double acc = 0.0;
                    for (j = 0; j < ds; j++) {
                        double t = (double)x[j] - cent[c * ds + j];
                        acc += t * t;
                    }
                    if (acc < best) { best = acc; bc = c; }
                }
                obj += best;
                cnt[bc]++;
                for (j = 0; j < ds; j++) sums[bc * ds + j] += (double)x[j];
            }
            if (obj_trace) obj_trace[(size_t)s * iters + it] = obj;
            for (c = 0; c < 256; c++)
                if (cnt[c])
                    for (j = 0; j < ds; j++) cent[c * ds + j] = sums[c * ds + j] / (double)cnt[c];
        }
        for (c = 0; c < 256; c++)
            for (j = 0; j < ds; j++)
                codebook[(size_t)256 * o + (size_t)c * ds + j] = (float)cent[c * ds + j];
        free(cent); free(sums); free(cnt);
        init += 256;
    }
    return 0;
}

/* PQ encoding (§4): code[i][s] = argmin_c ||x_s - C[s][c]||^2 in FP64,
 * ties to the smaller c. */
void orc_pq_encode(const void *X, int dtype, uint64_t n, uint32_t d, uint32_t M,
                   const uint32_t *off, const float *codebook, uint8_t *codes)
{
    uint64_t i;
    uint32_t s, c, j;
    for (i = 0; i < n; i++) {
        for (s = 0; s < M; s++) {
            uint32_t o = off[s], ds = off[s + 1] - off[s];
            double best = INFINITY;
            uint32_t bc = 0;
            for (c = 0; c < 256; c++) {
                const float *cc = centroid(codebook, off, s, c);
                double acc = 0.0;
                for (j = 0; j < ds; j++) {
                    double t = (double)elem_f(X, dtype, i * d + o + j) - (double)cc[j];
                    acc += t * t;
                }
                if (acc < best) { best = acc; bc = c; }
            }
            codes[i * M + s] = (uint8_t)bc;
        }
    }
}

/* Medoid (§6.3: the entry point fixed at construction): the point nearest,
 * in FP64, to the mean of all points; ties to the smaller id. */
uint32_t orc_medoid(const void *X, int dtype, uint64_t n, uint32_t d)
{
    double *mean = (double *)calloc(d, sizeof(double));
    double best = INFINITY;
    uint32_t bi = 0, j;
    uint64_t i;
    if (!mean) return ORC_NONE;
    for (i = 0; i < n; i++)
        for (j = 0; j < d; j++) mean[j] += (double)elem_f(X, dtype, i * d + j);
    for (j = 0; j < d; j++) mean[j] /= (double)n;
    for (i = 0; i < n; i++) {
        double acc = 0.0;
        for (j = 0; j < d; j++) {
            double t = (double)elem_f(X, dtype, i * d + j) - mean[j];
            acc += t * t;
        }
        if (acc < best) { best = acc; bi = (uint32_t)i; }
    }
    free(mean);
    return bi;
}

/* ---------------------------------------------------------------------- */
/* Vamana construction (§2.2; parameters in §6.3).                          */
/* ---------------------------------------------------------------------- */

static double sqdist_f64(const float *X, uint32_t d, uint64_t a, const float *y)
{
    const float *x = X + a * d;
    double acc = 0.0;
    uint32_t j;
    for (j = 0; j < d; j++) {
        double t = (double)x[j] - (double)y[j];
        acc += t * t;
    }
    return acc;
}

typedef struct { double dist; uint32_t id; } orc_dpair;

static int dpair_cmp(const void *pa, const void *pb)
{
    const orc_dpair *a = (const orc_dpair *)pa, *b = (const orc_dpair *)pb;
    if (a->dist < b->dist) return -1;
    if (a->dist > b->dist) return 1;
    return (a->id < b->id) ? -1 : (a->id > b->id);
}

/* RobustPrune(p, V, alpha, R): repeatedly keep the nearest remaining
 * candidate p* and drop every candidate p' with alpha*d(p*,p') <= d(p,p')
 * (Euclidean distances, compared here as alpha^2 * squared distances).
 * cand may contain p itself and duplicates; both are ignored.  Returns the
 * number of kept neighbours, written to out[0..R). */
uint32_t orc_robust_prune(const float *X, uint32_t d, uint32_t p, const uint32_t *cand,
                          uint32_t nc, float alpha, uint32_t R, uint32_t *out)
{
    orc_dpair *v = (orc_dpair *)malloc(sizeof(orc_dpair) * (nc ? nc : 1));
    unsigned char *alive = (unsigned char *)malloc(nc ? nc : 1);
    uint32_t nv = 0, i, j, nout = 0;
    double a2 = (double)alpha * (double)alpha;
    const float *xp = X + (uint64_t)p * d;
    for (i = 0; i < nc; i++) {
        uint32_t c = cand[i], dup = 0;
        if (c == p || c == ORC_NONE) continue;
        for (j = 0; j < nv; j++) if (v[j].id == c) { dup = 1; break; }
        if (dup) continue;
        v[nv].id = c;
        v[nv].dist = sqdist_f64(X, d, c, xp);
        nv++;
    }
    qsort(v, nv, sizeof(orc_dpair), dpair_cmp);
    for (i = 0; i < nv; i++) alive[i] = 1;
    for (i = 0; i < nv && nout < R; i++) {
        if (!alive[i]) continue;
        out[nout++] = v[i].id;
        for (j = i + 1; j < nv; j++) {
            if (!alive[j]) continue;
            if (a2 * sqdist_f64(X, d, v[j].id, X + (uint64_t)v[i].id * d) <= v[j].dist) alive[j] = 0;
        }
    }
    free(v); free(alive);
    return nout;
}

/* GreedySearch used during construction (exact FP64 distances, worklist of
 * Lb entries, every node inserted at most once).  Writes the expanded nodes
 * to V and returns their number. */
static uint32_t build_greedy(const float *X, uint32_t d, const uint32_t *adj, uint32_t R,
                             uint32_t s, const float *xq, uint32_t Lb, unsigned char *seen,
                             uint32_t *touched, uint32_t *ntouched, orc_dpair *Lst,
                             unsigned char *exp, uint32_t *V, uint32_t vcap)
{
    uint32_t nl = 1, nv = 0, i, r;
    Lst[0].id = s; Lst[0].dist = sqdist_f64(X, d, s, xq); exp[0] = 0;
    seen[s] = 1; touched[(*ntouched)++] = s;
    for (;;) {
        uint32_t u = ORC_NONE;
        for (i = 0; i < nl; i++) if (!exp[i]) { u = i; break; }
        if (u == ORC_NONE || nv >= vcap) break;
        exp[u] = 1;
        {
            uint32_t p = Lst[u].id;
            V[nv++] = p;
            for (r = 0; r < R; r++) {
                uint32_t nb = adj[(uint64_t)p * R + r];
                orc_dpair e;
                uint32_t pos;
                if (nb == ORC_NONE || seen[nb]) continue;
                seen[nb] = 1; touched[(*ntouched)++] = nb;
                e.id = nb; e.dist = sqdist_f64(X, d, nb, xq);
                /* insert into the sorted worklist, keep Lb entries */
                pos = nl;
                while (pos > 0 && dpair_cmp(&Lst[pos - 1], &e) > 0) pos--;
                if (pos >= Lb) continue;
                if (nl < Lb) nl++;
                for (i = nl - 1; i > pos; i--) { Lst[i] = Lst[i - 1]; exp[i] = exp[i - 1]; }
                Lst[pos] = e; exp[pos] = 0;
            }
        }
    }
    return nv;
}

/* Vamana build: two passes over the points in the given order, pruning
 * parameter 1 then alpha.  For every p: GreedySearch from the medoid,
 * RobustPrune(p, visited U N_out(p)), then add p to every new neighbour's
 * list, re-pruning a list that would exceed R.  The seeded random initial
 * graph (n*R, unused slots 0xFFFFFFFF) and the visiting order are inputs. */
int orc_vamana_build(const float *X, uint64_t n, uint32_t d, uint32_t R, uint32_t Lb,
                     float alpha, uint32_t medoid, const uint32_t *init_adj,
                     const uint32_t *order, uint32_t *adj)
{
    uint32_t vcap = 4 * Lb + 64;
    unsigned char *seen = (unsigned char *)calloc(n, 1);
    uint32_t *touched = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)vcap * R + Lb + 1));
    orc_dpair *Lst = (orc_dpair *)malloc(sizeof(orc_dpair) * (Lb + 1));
    unsigned char *exp = (unsigned char *)malloc(Lb + 1);
    uint32_t *V = (uint32_t *)malloc(sizeof(uint32_t) * vcap);
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (vcap + R + 1));
    uint32_t *pr = (uint32_t *)malloc(sizeof(uint32_t) * (R + 1));
    int pass;
    uint64_t t;
    if (!seen || !touched || !Lst || !exp || !V || !cand || !pr) return -1;
    memcpy(adj, init_adj, sizeof(uint32_t) * n * R);
    for (pass = 0; pass < 2; pass++) {
        float a = pass == 0 ? 1.0f : alpha;
        for (t = 0; t < n; t++) {
            uint32_t p = order[t], nv, nt = 0, nc = 0, r, np, i;
            nv = build_greedy(X, d, adj, R, medoid, X + (uint64_t)p * d, Lb, seen, touched, &nt,
                              Lst, exp, V, vcap);
            for (i = 0; i < nt; i++) seen[touched[i]] = 0;
            for (i = 0; i < nv; i++) cand[nc++] = V[i];
            for (r = 0; r < R; r++) cand[nc++] = adj[(uint64_t)p * R + r];
            np = orc_robust_prune(X, d, p, cand, nc, a, R, pr);
            for (r = 0; r < R; r++) adj[(uint64_t)p * R + r] = r < np ? pr[r] : ORC_NONE;
            for (i = 0; i < np; i++) {
                uint32_t j = pr[i], deg = 0, has = 0;
                uint32_t *lj = adj + (uint64_t)j * R;
                for (r = 0; r < R; r++) {
                    if (lj[r] == ORC_NONE) continue;
                    deg++;
                    if (lj[r] == p) has = 1;
                }
                if (has) continue;
                if (deg < R) {
                    for (r = 0; r < R; r++) if (lj[r] == ORC_NONE) { lj[r] = p; break; }
                } else {
                    uint32_t c2[1024], k2 = 0, nk;
                    uint32_t kept[1024];
                    for (r = 0; r < R; r++) c2[k2++] = lj[r];
                    c2[k2++] = p;
                    nk = orc_robust_prune(X, d, j, c2, k2, a, R, kept);
                    for (r = 0; r < R; r++) lj[r] = r < nk ? kept[r] : ORC_NONE;
                }
            }
        }
    }
    free(seen); free(touched); free(Lst); free(exp); free(V); free(cand); free(pr);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Clustered graph.  The paper searches a graph it takes from DiskANN (§1)  */
/* and gives no construction; the large synthetic indexes here use this    */
/* one, restated plainly so that the GPU builder can be checked against it. */
/* For each cluster (members given in ascending id; b = local position):   */
/*  1. candidates of member a: the K = min(2 Rin, m - 1) other members      */
/*     nearest to a, by (distance, b), Rin = R - nx;                        */
/*  2. RobustPrune (Vamana, §2.2): walk the candidates in (distance, b)     */
/*     order; a candidate still alive is kept (up to Rin) and removes every */
/*     later candidate j with alpha^2 * d(kept, j) <= d(a, j), alpha^2 and  */
/*     the product rounded to FP32;                                         */
/*  3. reverse edges: the kept list plus every member that kept a, without  */
/*     repeats, pruned again the same way;                                  */
/*  4. repair, members in ascending b: a member nobody links to (and that   */
/*     has neighbours) is appended to the first of its neighbours that has  */
/*     room, or replaces that neighbour's last entry when the entry's       */
/*     target keeps another in-link; in-degrees are updated as it goes;     */
/*  5. the global row of a member: its list (a cluster medoid keeps at most */
/*     R - nh), then the medoids of the clusters in xclu (nx per point) or, */
/*     for a cluster medoid, hclu (nh per cluster), skipping its own        */
/*     cluster and out-of-range ids; repeated ids are dropped keeping the   */
/*     first; the rest of the row is 0xFFFFFFFF.                            */
/* Distances are squared L2: exact integers for u8/i8; for f32 the sum in   */
/* ascending j of (x_j - y_j)^2, each difference, product and sum rounded   */
/* to FP32.                                                                 */
/* ---------------------------------------------------------------------- */

static float cg_dist(const void *X, int dtype, uint32_t d, uint64_t a, uint64_t b)
{
    uint32_t j;
    if (dtype == ORC_F32) {
        const float *x = (const float *)X + a * d, *y = (const float *)X + b * d;
        float acc = 0.0f;
        for (j = 0; j < d; j++) {
            float t = x[j] - y[j];
            float sq = t * t;
            acc = acc + sq;
        }
        return acc;
    } else {
        int64_t acc = 0;
        for (j = 0; j < d; j++) {
            int64_t t = (int64_t)elem_i(X, dtype, a * d + j) - (int64_t)elem_i(X, dtype, b * d + j);
            acc += t * t;
        }
        return (float)acc;
    }
}

typedef struct { float dist; uint32_t b; } cg_cand;

static int cg_cmp(const void *pa, const void *pb)
{
    const cg_cand *x = (const cg_cand *)pa, *y = (const cg_cand *)pb;
    if (x->dist < y->dist) return -1;
    if (x->dist > y->dist) return 1;
    return (x->b < y->b) ? -1 : (x->b > y->b);
}

/* RobustPrune of step 2 over nc candidates (sorted here); P maps local
 * positions to point ids.  Returns the number kept (written to out). */
static uint32_t cg_prune(const void *X, int dtype, uint32_t d, const uint32_t *P, cg_cand *c,
                         uint32_t nc, float alpha, uint32_t Rin, uint32_t *out)
{
    uint32_t i, j, nout = 0;
    float a2 = alpha * alpha;
    unsigned char *dead = (unsigned char *)calloc(nc ? nc : 1, 1);
    qsort(c, nc, sizeof(cg_cand), cg_cmp);
    for (i = 0; i < nc && nout < Rin; i++) {
        if (dead[i]) continue;
        out[nout++] = c[i].b;
        for (j = i + 1; j < nc; j++) {
            if (dead[j]) continue;
            float lhs = a2 * cg_dist(X, dtype, d, P[c[i].b], P[c[j].b]);
            if (lhs <= c[j].dist) dead[j] = 1;
        }
    }
    free(dead);
    return nout;
}

int orc_cluster_graph(const void *X, int dtype, uint32_t d, uint64_t n, const uint32_t *members,
                      const uint64_t *gstart, uint32_t ng, const uint32_t *medoids, uint32_t R,
                      float alpha, uint32_t nx, const uint32_t *xclu, uint32_t nh,
                      const uint32_t *hclu, uint32_t *adj)
{
    uint32_t g, Rin;
    uint64_t i;
    if (nx >= R || nh >= R) return -1;
    Rin = R - nx;
    for (i = 0; i < n * (uint64_t)R; i++) adj[i] = ORC_NONE;
    for (g = 0; g < ng; g++) {
        uint32_t m = (uint32_t)(gstart[g + 1] - gstart[g]), a, b, t, K;
        const uint32_t *P = members + gstart[g];
        uint32_t *fwd, *fwd2, *deg, *deg2, *indeg;
        cg_cand *cand;
        if (m == 0) continue;
        K = 2 * Rin < m - 1 ? 2 * Rin : m - 1;
        fwd = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * Rin);
        fwd2 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * Rin);
        deg = (uint32_t *)calloc(m, sizeof(uint32_t));
        deg2 = (uint32_t *)calloc(m, sizeof(uint32_t));
        indeg = (uint32_t *)calloc(m, sizeof(uint32_t));
        cand = (cg_cand *)malloc(sizeof(cg_cand) * (m + Rin + 1));
        if (!fwd || !fwd2 || !deg || !deg2 || !indeg || !cand) {
            free(fwd); free(fwd2); free(deg); free(deg2); free(indeg); free(cand);
            return -2;
        }
        /* steps 1-2 */
        for (a = 0; a < m; a++) {
            uint32_t nc = 0;
            for (b = 0; b < m; b++) {
                if (b == a) continue;
                cand[nc].dist = cg_dist(X, dtype, d, P[a], P[b]);
                cand[nc].b = b;
                nc++;
            }
            qsort(cand, nc, sizeof(cg_cand), cg_cmp);
            deg[a] = cg_prune(X, dtype, d, P, cand, K, alpha, Rin, fwd + (size_t)a * Rin);
        }
        /* step 3 */
        for (a = 0; a < m; a++) {
            uint32_t nc = 0;
            for (t = 0; t < deg[a]; t++) {
                cand[nc].b = fwd[(size_t)a * Rin + t];
                cand[nc].dist = cg_dist(X, dtype, d, P[a], P[cand[nc].b]);
                nc++;
            }
            for (b = 0; b < m; b++) {
                int chose = 0, have = 0;
                for (t = 0; t < deg[b]; t++) if (fwd[(size_t)b * Rin + t] == a) chose = 1;
                if (!chose) continue;
                for (t = 0; t < deg[a]; t++) if (fwd[(size_t)a * Rin + t] == b) have = 1;
                if (have) continue;
                cand[nc].b = b;
                cand[nc].dist = cg_dist(X, dtype, d, P[a], P[b]);
                nc++;
            }
            deg2[a] = cg_prune(X, dtype, d, P, cand, nc, alpha, Rin, fwd2 + (size_t)a * Rin);
        }
        /* step 4 */
        for (a = 0; a < m; a++)
            for (t = 0; t < deg2[a]; t++) indeg[fwd2[(size_t)a * Rin + t]]++;
        for (a = 0; a < m; a++) {
            if (indeg[a] != 0 || deg2[a] == 0) continue;
            for (t = 0; t < deg2[a]; t++) {
                uint32_t j = fwd2[(size_t)a * Rin + t];
                uint32_t *lj = fwd2 + (size_t)j * Rin;
                if (deg2[j] < Rin) {
                    lj[deg2[j]] = a;
                    deg2[j]++;
                    indeg[a]++;
                    break;
                }
                if (indeg[lj[deg2[j] - 1]] > 1) {
                    indeg[lj[deg2[j] - 1]]--;
                    lj[deg2[j] - 1] = a;
                    indeg[a]++;
                    break;
                }
            }
        }
        /* step 5 */
        for (a = 0; a < m; a++) {
            uint32_t *row = adj + (uint64_t)P[a] * R, w = 0, r, q;
            int is_med = P[a] == medoids[g];
            uint32_t keep = deg2[a];
            if (is_med && keep > R - nh) keep = R - nh;
            for (t = 0; t < keep; t++) row[w++] = P[fwd2[(size_t)a * Rin + t]];
            for (t = 0; t < (is_med ? nh : nx); t++) {
                uint32_t c2 = is_med ? hclu[(size_t)g * nh + t] : xclu[(uint64_t)P[a] * nx + t];
                if (c2 >= ng || c2 == g || medoids[c2] == ORC_NONE) continue;
                row[w++] = medoids[c2];
            }
            for (r = 0; r < w; r++)
                for (q = 0; q < r; q++)
                    if (row[q] != ORC_NONE && row[q] == row[r]) { row[r] = ORC_NONE; break; }
            q = 0;
            for (r = 0; r < w; r++) if (row[r] != ORC_NONE) row[q++] = row[r];
            for (r = q; r < R; r++) row[r] = ORC_NONE;
        }
        free(fwd); free(fwd2); free(deg); free(deg2); free(indeg); free(cand);
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* PQDistTable (§4.1), FP32 form: T[s][c] = sum over the dimensions j of    */
/* subspace s, in ascending j, of (q_j - C[s][c][j])^2, accumulated as      */
/* acc = fmaf(diff, diff, acc) from acc = 0, diff rounded to FP32.          */
/* ---------------------------------------------------------------------- */

void orc_adc_table_f32(const float *q, uint32_t M, const uint32_t *off,
                       const float *codebook, float *T)
{
    uint32_t s, c, j;
    for (s = 0; s < M; s++) {
        uint32_t o = off[s], ds = off[s + 1] - off[s];
        for (c = 0; c < 256; c++) {
            const float *cc = centroid(codebook, off, s, c);
            float acc = 0.0f;
            for (j = 0; j < ds; j++) {
                float diff = q[o + j] - cc[j];
                acc = fmaf(diff, diff, acc);
            }
            T[s * 256 + c] = acc;
        }
    }
}

/* Asymmetric distance (§4.4): the sum over subspaces of T[s][code[s]].
 * The paper leaves the summation order to the reduction it uses; the order
 * fixed here is: eight partial sums p_r over the subspaces s = r (mod 8),
 * each added in ascending s from 0, then three butterfly rounds
 * p_r += p_(r xor 4), p_r += p_(r xor 2), p_r += p_(r xor 1); result p_0. */
float orc_adc_dist_f32(const float *T, uint32_t M, const uint8_t *code)
{
    float p[8], nx[8];
    uint32_t s, r, h;
    for (r = 0; r < 8; r++) p[r] = 0.0f;
    for (s = 0; s < M; s++) p[s & 7] = p[s & 7] + T[s * 256 + code[s]];
    for (h = 4; h >= 1; h >>= 1) {
        for (r = 0; r < 8; r++) nx[r] = p[r] + p[r ^ h];
        for (r = 0; r < 8; r++) p[r] = nx[r];
    }
    return p[0];
}

/* ---------------------------------------------------------------------- */
/* BF16 table.  Not in the paper, whose table is FP32 (§4.1); added as a    */
/* reduced form with half the table: every FP32 entry is rounded to the     */
/* nearest BF16 value (8 significant bits; halfway cases to the value whose */
/* last kept bit is 0), and distances sum the BF16 values, widened back to  */
/* FP32, in the order of orc_adc_dist_f32.                                  */
/* ---------------------------------------------------------------------- */

float orc_round_bf16(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) {
        if (u & 0x007FFFFFu) u |= 0x00400000u;        /* NaN stays NaN */
    } else {
        uint32_t keep_lsb = (u >> 16) & 1u;
        u += 0x7FFFu + keep_lsb;                      /* may carry into the exponent */
    }
    u &= 0xFFFF0000u;
    memcpy(&x, &u, 4);
    return x;
}

void orc_adc_table_bf16(const float *T, uint32_t M, float *Tb)
{
    uint32_t i;
    for (i = 0; i < M * 256u; i++) Tb[i] = orc_round_bf16(T[i]);
}

/* ---------------------------------------------------------------------- */
/* 8-bit table.  Not in the paper, whose table is FP32 (§4.1); added as a   */
/* reduced form whose table is a quarter of the FP32 one.  From the FP32    */
/* table T of one query:                                                    */
/*   lo_s = min_c T[s][c],  w_s = max_c T[s][c] - lo_s  (FP32 subtraction), */
/*   g = max_s w_s;  if g == 0 every entry is 0; otherwise                  */
/*   inv = 255 / g (FP32 division) and                                      */
/*   Q[s][c] = min(255, rint((T[s][c] - lo_s) * inv)),                      */
/* the subtraction and the product each rounded to FP32, rint rounding      */
/* halves to even.  Q[s][c] * g / 255 + lo_s approximates T[s][c] within    */
/* g / 510 plus rounding.  The per-subspace offsets add the same constant   */
/* to every candidate of the query, so the integer sum of Q ranks the       */
/* candidates as the dequantised sum does.                                  */
/* ---------------------------------------------------------------------- */

void orc_adc_table_q8(const float *T, uint32_t M, uint8_t *Q)
{
    uint32_t s, c;
    float g = 0.0f;
    float *lo = (float *)malloc(sizeof(float) * (M ? M : 1));
    for (s = 0; s < M; s++) {
        float mn = T[s * 256], mx = T[s * 256], w;
        for (c = 1; c < 256; c++) {
            if (T[s * 256 + c] < mn) mn = T[s * 256 + c];
            if (T[s * 256 + c] > mx) mx = T[s * 256 + c];
        }
        lo[s] = mn;
        w = mx - mn;
        if (w > g) g = w;
    }
    for (s = 0; s < M; s++) {
        for (c = 0; c < 256; c++) {
            uint32_t v = 0;
            if (g > 0.0f) {
                float inv = 255.0f / g;
                float x = (T[s * 256 + c] - lo[s]) * inv;
                v = (uint32_t)rintf(x);
                if (v > 255u) v = 255u;
            }
            Q[s * 256 + c] = (uint8_t)v;
        }
    }
    free(lo);
}

/* Asymmetric distance on the 8-bit table: the exact integer sum over the
 * subspaces of Q[s][code[s]]. */
uint32_t orc_adc_dist_q8(const uint8_t *Q, uint32_t M, const uint8_t *code)
{
    uint32_t s, acc = 0;
    for (s = 0; s < M; s++) acc += Q[s * 256 + code[s]];
    return acc;
}

/* ---------------------------------------------------------------------- */
/* Exact distance for the re-rank (§4.8).                                   */
/* Integer data: exact integer sum of squared differences.                  */
/* FP32 data: 32 partial sums p_r over the dimensions j with                */
/* (j/4) mod 32 = r, each accumulated in ascending j with                   */
/* fmaf(diff, diff, p_r) from 0; then five butterfly rounds                 */
/* p_r += p_(r xor h) for h = 16, 8, 4, 2, 1; result p_0.                   */
/* The returned key is exact in double (integer, or the FP32 value).       */
/* ---------------------------------------------------------------------- */

double orc_exact_dist(const void *q, const void *x, int dtype, uint32_t d)
{
    uint32_t j;
    if (dtype != ORC_F32) {
        int64_t acc = 0;
        for (j = 0; j < d; j++) {
            int64_t t = (int64_t)elem_i(q, dtype, j) - (int64_t)elem_i(x, dtype, j);
            acc += t * t;
        }
        return (double)acc;
    } else {
        const float *qf = (const float *)q, *xf = (const float *)x;
        float p[32], nx[32];
        uint32_t r, h;
        for (r = 0; r < 32; r++) p[r] = 0.0f;
        for (j = 0; j < d; j++) {
            float diff = qf[j] - xf[j];
            r = (j >> 2) & 31u;
            p[r] = fmaf(diff, diff, p[r]);
        }
        for (h = 16; h >= 1; h >>= 1) {
            for (r = 0; r < 32; r++) nx[r] = p[r] + p[r ^ h];
            for (r = 0; r < 32; r++) p[r] = nx[r];
        }
        return (double)p[0];
    }
}

/* ---------------------------------------------------------------------- */
/* Bloom filter of seen nodes (§4.3; two FNV-1a hashes, §6.3).              */
/* z = 2^log2z bits.  h1 = FNV-1a 32-bit over the 4 little-endian bytes of  */
/* the id; h2 = FNV-1a 64-bit over the same bytes, folded to 32 bits as     */
/* (h >> 32) xor (h & 0xffffffff).  Bit positions: h1 mod z and h2 mod z.   */
/* ---------------------------------------------------------------------- */

uint32_t orc_fnv1a32_bytes(const unsigned char *b, uint32_t len)
{
    uint32_t h = 2166136261u, i;
    for (i = 0; i < len; i++) { h ^= b[i]; h *= 16777619u; }
    return h;
}

uint64_t orc_fnv1a64_bytes(const unsigned char *b, uint32_t len)
{
    uint64_t h = 14695981039346656037ull;
    uint32_t i;
    for (i = 0; i < len; i++) { h ^= b[i]; h *= 1099511628211ull; }
    return h;
}

static void id_bytes(uint32_t id, unsigned char *b)
{
    b[0] = (unsigned char)(id & 0xff);
    b[1] = (unsigned char)((id >> 8) & 0xff);
    b[2] = (unsigned char)((id >> 16) & 0xff);
    b[3] = (unsigned char)((id >> 24) & 0xff);
}

void orc_bloom_positions(uint32_t id, uint32_t log2z, uint32_t *pos2)
{
    unsigned char b[4];
    uint64_t h2;
    uint32_t mask = (log2z >= 32) ? 0xFFFFFFFFu : ((1u << log2z) - 1u);
    id_bytes(id, b);
    h2 = orc_fnv1a64_bytes(b, 4);
    pos2[0] = orc_fnv1a32_bytes(b, 4) & mask;
    pos2[1] = ((uint32_t)(h2 >> 32) ^ (uint32_t)(h2 & 0xFFFFFFFFu)) & mask;
}

int orc_bloom_test(const uint32_t *bits, uint32_t log2z, uint32_t id)
{
    uint32_t p[2];
    orc_bloom_positions(id, log2z, p);
    return ((bits[p[0] >> 5] >> (p[0] & 31)) & 1u) && ((bits[p[1] >> 5] >> (p[1] & 31)) & 1u);
}

void orc_bloom_insert(uint32_t *bits, uint32_t log2z, uint32_t id)
{
    uint32_t p[2];
    orc_bloom_positions(id, log2z, p);
    bits[p[0] >> 5] |= 1u << (p[0] & 31);
    bits[p[1] >> 5] |= 1u << (p[1] & 31);
}

/* ---------------------------------------------------------------------- */
/* Search (Alg. 1 run for each query of the batch as in Alg. 2).            */
/* ---------------------------------------------------------------------- */

typedef struct { float dist; uint32_t id; int visited; } orc_entry;

static int entry_cmp(const void *pa, const void *pb)
{
    const orc_entry *a = (const orc_entry *)pa, *b = (const orc_entry *)pb;
    if (a->dist < b->dist) return -1;
    if (a->dist > b->dist) return 1;
    return (a->id < b->id) ? -1 : (a->id > b->id);
}

static int dpair_cmp_stable(const void *pa, const void *pb) { return dpair_cmp(pa, pb); }

/* Distance of node v in the search loop: mode 0 the FP32 PQ distance
 * (§4.4), mode 1 the exact distance (§5.2), mode 2 the 8-bit table's integer
 * sum (exact in FP32: at most 255 * M). */
static float search_dist(const orc_index *ix, int mode, const float *T, const uint8_t *Q,
                         const void *q, uint32_t v)
{
    size_t esz = ix->dtype == ORC_F32 ? 4 : 1;
    if (mode == 0 || mode == 3) return orc_adc_dist_f32(T, ix->M, ix->codes + (uint64_t)v * ix->M);
    if (mode == 2) return (float)orc_adc_dist_q8(Q, ix->M, ix->codes + (uint64_t)v * ix->M);
    return (float)orc_exact_dist(q, (const unsigned char *)ix->base + (uint64_t)v * ix->d * esz,
                                 ix->dtype, ix->d);
}

/* One query.  Steps, in the order of Alg. 2 and §4:
 *  - T <- PQDistTable row of the query (§4.1); the query is converted to FP32.
 *  - worklist L <- [(ADC(s), s, unvisited)], s inserted into the Bloom filter.
 *  - loop: u* <- first unvisited entry of L (L is kept sorted by (distance,
 *    id)); stop when there is none, or after iter_cap expansions (status 1).
 *    Mark u* visited; record it as a re-rank candidate with its exact
 *    distance (§4.2, §4.8: the candidates' full vectors are fetched as they
 *    are visited).  N <- adj(u*) in stored order, skipping 0xFFFFFFFF.
 *    N' <- the ids of N whose Bloom test fails, all tested against the
 *    filter as it was before this iteration; then insert all of N' (§4.3).
 *    D[n] <- ADC(n) for n in N' (§4.4).  L <- the first L entries of
 *    L u {(D[n], n, unvisited)} sorted by (distance, id) (§4.6, §4.7).
 *  - re-rank (§4.8): sort the candidates by (exact distance, id); output
 *    the first k; pad with id 0xFFFFFFFF and distance +inf.
 * The eager choice of the next candidate (§4.5) is the first unvisited
 * entry after the merge, so it does not appear as a separate step. */
static void search_one(const orc_index *ix, const void *q, int mode, uint32_t k, uint32_t Lsz,
                       uint32_t log2z, uint32_t iter_cap, uint32_t *out_ids, float *out_dist,
                       uint32_t *out_iters, int32_t *out_status, uint64_t *out_ndist,
                       uint32_t *trace, uint32_t trace_cap, int rerank_list)
{
    uint32_t d = ix->d, M = ix->M, R = ix->R, i, r;
    float *qf = (float *)malloc(sizeof(float) * d);
    float *T = (float *)malloc(sizeof(float) * (size_t)M * 256);
    uint8_t *Q = (uint8_t *)malloc((size_t)M * 256);
    uint32_t nwords = (log2z >= 5) ? (1u << (log2z - 5)) : 1u;
    uint32_t *bits = (uint32_t *)calloc(nwords, sizeof(uint32_t));
    orc_entry *Lst = (orc_entry *)malloc(sizeof(orc_entry) * (Lsz + R + 1));
    uint32_t *Np = (uint32_t *)malloc(sizeof(uint32_t) * (R + 1));
    uint32_t ccap = iter_cap + 1, nc = 0, nl, iters = 0;
    orc_dpair *C = (orc_dpair *)malloc(sizeof(orc_dpair) * (ccap > Lsz + R + 1 ? ccap : Lsz + R + 1));
    uint64_t ndist = 0;
    int32_t status = 0;
    size_t esz = ix->dtype == ORC_F32 ? 4 : 1;

    for (i = 0; i < d; i++) qf[i] = elem_f(q, ix->dtype, i);
    if (mode != 1) orc_adc_table_f32(qf, M, ix->off, ix->codebook, T);
    if (mode == 2) orc_adc_table_q8(T, M, Q);
    if (mode == 3) orc_adc_table_bf16(T, M, T);

    Lst[0].id = ix->medoid;
    Lst[0].dist = search_dist(ix, mode, T, Q, q, ix->medoid);
    Lst[0].visited = 0;
    ndist++;
    nl = 1;
    orc_bloom_insert(bits, log2z, ix->medoid);

    for (;;) {
        uint32_t u = ORC_NONE, nn = 0, nadd;
        for (i = 0; i < nl; i++) if (!Lst[i].visited) { u = i; break; }
        if (u == ORC_NONE) break;
        if (iters >= iter_cap) { status = 1; break; }
        Lst[u].visited = 1;
        {
            uint32_t us = Lst[u].id;
            if (trace && iters < trace_cap) trace[iters] = us;
            iters++;
            if (mode != 1) {
                C[nc].id = us;
                C[nc].dist = orc_exact_dist(q, (const unsigned char *)ix->base + (uint64_t)us * d * esz,
                                            ix->dtype, d);
                nc++;
            }
            for (r = 0; r < R; r++) {
                uint32_t nb = ix->adj[(uint64_t)us * R + r];
                if (nb == ORC_NONE) continue;
                if (!orc_bloom_test(bits, log2z, nb)) Np[nn++] = nb;
            }
        }
        for (i = 0; i < nn; i++) orc_bloom_insert(bits, log2z, Np[i]);
        nadd = 0;
        for (i = 0; i < nn; i++) {
            Lst[nl + nadd].id = Np[i];
            Lst[nl + nadd].dist = search_dist(ix, mode, T, Q, q, Np[i]);
            Lst[nl + nadd].visited = 0;
            nadd++;
        }
        ndist += nn;
        qsort(Lst, nl + nadd, sizeof(orc_entry), entry_cmp);
        nl = (nl + nadd < Lsz) ? nl + nadd : Lsz;
    }

    if (mode == 1) {                    /* Alg. 1: the k nearest entries of the worklist */
        nc = 0;
        for (i = 0; i < nl; i++) { C[nc].id = Lst[i].id; C[nc].dist = (double)Lst[i].dist; nc++; }
    } else if (rerank_list) {           /* re-rank the final worklist only (reading c9's option) */
        nc = 0;
        for (i = 0; i < nl; i++) {
            C[nc].id = Lst[i].id;
            C[nc].dist = orc_exact_dist(q, (const unsigned char *)ix->base + (uint64_t)Lst[i].id * d * esz,
                                        ix->dtype, d);
            nc++;
        }
    }
    qsort(C, nc, sizeof(orc_dpair), dpair_cmp_stable);
    for (i = 0; i < k; i++) {
        if (i < nc) { out_ids[i] = C[i].id; out_dist[i] = (float)C[i].dist; }
        else { out_ids[i] = ORC_NONE; out_dist[i] = INFINITY; }
    }
    if (out_iters) *out_iters = iters;
    if (out_status) *out_status = status;
    if (out_ndist) *out_ndist = ndist;
    free(qf); free(T); free(Q); free(bits); free(Lst); free(Np); free(C);
}

int orc_search(const orc_index *ix, const void *queries, int mode, uint32_t nq, uint32_t k,
               uint32_t L, uint32_t log2z, uint32_t iter_cap, uint32_t *out_ids, float *out_dist,
               uint32_t *out_iters, int32_t *out_status, uint64_t *out_ndist,
               uint32_t *trace, uint32_t trace_cap, int nthreads)
{
    return orc_search_rr(ix, queries, mode, nq, k, L, log2z, iter_cap, out_ids, out_dist, out_iters,
                         out_status, out_ndist, trace, trace_cap, nthreads, 0);
}

int orc_search_rr(const orc_index *ix, const void *queries, int mode, uint32_t nq, uint32_t k,
                  uint32_t L, uint32_t log2z, uint32_t iter_cap, uint32_t *out_ids, float *out_dist,
                  uint32_t *out_iters, int32_t *out_status, uint64_t *out_ndist,
                  uint32_t *trace, uint32_t trace_cap, int nthreads, int rerank_list)
{
    int64_t qi;
    size_t esz = ix->dtype == ORC_F32 ? 4 : 1;
    if (k == 0 || L < k || ix->M == 0 || ix->d == 0 || mode < 0 || mode > 3) return -1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#else
    (void)nthreads;
#endif
    for (qi = 0; qi < (int64_t)nq; qi++) {
        search_one(ix, (const unsigned char *)queries + (uint64_t)qi * ix->d * esz, mode, k, L, log2z,
                   iter_cap, out_ids + (uint64_t)qi * k, out_dist + (uint64_t)qi * k,
                   out_iters ? out_iters + qi : NULL, out_status ? out_status + qi : NULL,
                   out_ndist ? out_ndist + qi : NULL,
                   trace ? trace + (uint64_t)qi * trace_cap : NULL, trace_cap, rerank_list);
    }
    return 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Overlapping-shard graph (§2.2): the paper's Vamana index is built by     */
/* splitting the dataset into smaller overlapping clusters, building a      */
/* directed subgraph on each with GreedySearch and RobustPrune, and merging */
/* the subgraphs' edges.  Restated in a batched form a GPU can also run:    */
/*  1. assignment: point i joins the shards of its ell nearest centres      */
/*     (FP32 squared distance over ascending dimensions, each difference,   */
/*     product and sum rounded; ties to the smaller centre index);          */
/*  2. shard g lists its members in ascending point id; its entry e_g is    */
/*     the member nearest its centre (same distance, ties to the smaller    */
/*     id); it inserts e_g first, then the other members in ascending id;   */
/*  3. two passes, pruning parameter 1 then alpha.  A pass cuts each        */
/*     shard's insertion order into batches (pass 1: 1, 1, 2, 4, ... up to  */
/*     cap_g = max(1, floor(batch_frac * m_g)); pass 2: cap_g each); batch  */
/*     r of every shard forms round r.  In a round, against the graph as it */
/*     stood at the round's start, each member p runs GreedySearch from e_g */
/*     (Alg. 1 with exact distances, worklist Lb, a Bloom seen set of       */
/*     2^log2z bits, at most iter_cap expansions): V_p = its expanded       */
/*     nodes.  Then p's list becomes RobustPrune(p, V_p U N(p)).  Then each */
/*     q named by a new list takes the members that named it: N(q) U In(q) */
/*     sorted when it fits in R, else RobustPrune(q, N(q) U In(q));         */
/*  4. merge: point i's row is the union of its shard lists (as point ids), */
/*     sorted when it fits in R, else RobustPrune(i, union) with alpha.     */
/* Distances are orc_exact_dist rounded to FP32; candidate lists are sorted */
/* by (distance, id) with repeats and the point itself removed, and cut to  */
/* their 750 nearest (DiskANN's bound on the candidate pool; only reverse   */
/* edges into hubs reach it); every row is kept in that order.  RobustPrune:*/
/* in that order, a live candidate is kept (at most R) and removes each     */
/* later candidate c with a^2 * d(kept, c) <= d(p, c), a^2 and the product  */
/* rounded to FP32.                                                         */
/* ---------------------------------------------------------------------- */

typedef struct { float dist; uint32_t id; } sg_cand;

#define SG_CAND_CAP 750       /* RobustPrune considers the 750 nearest candidates (DiskANN's bound) */

static int sg_cmp(const void *pa, const void *pb)
{
    const sg_cand *a = (const sg_cand *)pa, *b = (const sg_cand *)pb;
    if (a->dist < b->dist) return -1;
    if (a->dist > b->dist) return 1;
    return (a->id < b->id) ? -1 : (a->id > b->id);
}

static float sg_dist(const void *V, int dtype, uint32_t d, uint64_t a, uint64_t b)
{
    size_t esz = dtype == ORC_F32 ? 4 : 1;
    return (float)orc_exact_dist((const unsigned char *)V + a * d * esz,
                                 (const unsigned char *)V + b * d * esz, dtype, d);
}

/* FP32 squared distance of point i to centre c (step 1). */
static float sg_centre_dist(const void *X, int dtype, uint32_t d, uint64_t i, const float *c)
{
    float acc = 0.0f;
    uint32_t j;
    for (j = 0; j < d; j++) {
        float t = elem_f(X, dtype, i * d + j) - c[j];
        float sq = t * t;
        acc = acc + sq;
    }
    return acc;
}

/* The list of p from nc candidate ids (any order, repeats allowed): drop p
 * and NONE, sort by (distance to p, id), drop repeats, then keep all (at
 * most R) or RobustPrune.  V holds the vectors the ids index.  Returns the
 * row length; out has R slots, padded with NONE. */
static uint32_t sg_list(const void *V, int dtype, uint32_t d, uint32_t p, const uint32_t *ids,
                        uint32_t nc, float alpha, uint32_t R, int always_prune, uint32_t *out)
{
    sg_cand *c = (sg_cand *)malloc(sizeof(sg_cand) * (nc ? nc : 1));
    unsigned char *dead = (unsigned char *)calloc(nc ? nc : 1, 1);
    uint32_t m = 0, u = 0, i, j, nout = 0;
    float a2 = alpha * alpha;
    for (i = 0; i < nc; i++) {
        if (ids[i] == p || ids[i] == ORC_NONE) continue;
        c[m].id = ids[i];
        c[m].dist = sg_dist(V, dtype, d, p, ids[i]);
        m++;
    }
    qsort(c, m, sizeof(sg_cand), sg_cmp);
    for (i = 0; i < m; i++)
        if (u == 0 || c[i].id != c[u - 1].id) c[u++] = c[i];
    if (u > SG_CAND_CAP) u = SG_CAND_CAP;
    if (u <= R && !always_prune) {
        for (i = 0; i < u; i++) out[nout++] = c[i].id;
    } else {
        for (i = 0; i < u && nout < R; i++) {
            if (dead[i]) continue;
            out[nout++] = c[i].id;
            for (j = i + 1; j < u; j++) {
                float lhs;
                if (dead[j]) continue;
                lhs = a2 * sg_dist(V, dtype, d, c[i].id, c[j].id);
                if (lhs <= c[j].dist) dead[j] = 1;
            }
        }
    }
    for (i = nout; i < R; i++) out[i] = ORC_NONE;
    free(c); free(dead);
    return nout;
}

typedef struct { uint32_t q, p; } sg_pair;

static int sg_pair_cmp(const void *pa, const void *pb)
{
    const sg_pair *a = (const sg_pair *)pa, *b = (const sg_pair *)pb;
    if (a->q != b->q) return a->q < b->q ? -1 : 1;
    return (a->p < b->p) ? -1 : (a->p > b->p);
}

int orc_shard_graph(const void *X, int dtype, uint64_t n, uint32_t d, const float *centres,
                    uint32_t S, uint32_t ell, uint32_t R, uint32_t Lb, float alpha,
                    float batch_frac, uint32_t log2z, uint32_t iter_cap, uint32_t *adj,
                    uint32_t *shard_of, int nthreads)
{
    size_t esz = dtype == ORC_F32 ? 4 : 1;
    uint64_t nv = n * ell, i, v;
    uint32_t g, t, pass;
    uint32_t *sh, *cnt, *vpt, *vadj, *entry, *epos, *cap, *vid;
    uint64_t *gstart, *cur;
    unsigned char *vbase;
    int rc = 0;
    if (n == 0 || d == 0 || S == 0 || ell == 0 || ell > S || R == 0 || Lb == 0 || iter_cap == 0 ||
        log2z < 5 || log2z > 24 || nv >= ORC_NONE || !(batch_frac > 0.0f))
        return -1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    (void)nthreads;
#endif
    sh = (uint32_t *)malloc(sizeof(uint32_t) * nv);
    vid = (uint32_t *)malloc(sizeof(uint32_t) * nv);
    cnt = (uint32_t *)calloc(S, sizeof(uint32_t));
    gstart = (uint64_t *)calloc(S + 1, sizeof(uint64_t));
    cur = (uint64_t *)calloc(S, sizeof(uint64_t));
    vpt = (uint32_t *)malloc(sizeof(uint32_t) * nv);
    vadj = (uint32_t *)malloc(sizeof(uint32_t) * nv * R);
    entry = (uint32_t *)malloc(sizeof(uint32_t) * S);
    epos = (uint32_t *)malloc(sizeof(uint32_t) * S);
    cap = (uint32_t *)malloc(sizeof(uint32_t) * S);
    vbase = (unsigned char *)malloc(nv * d * esz);
    if (!sh || !vid || !cnt || !gstart || !cur || !vpt || !vadj || !entry || !epos || !cap || !vbase) {
        rc = -2;
        goto done;
    }
    /* 1. assignment */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int64_t ii = 0; ii < (int64_t)n; ii++) {
        sg_cand *best = (sg_cand *)malloc(sizeof(sg_cand) * S);
        uint32_t gg;
        for (gg = 0; gg < S; gg++) {
            best[gg].dist = sg_centre_dist(X, dtype, d, (uint64_t)ii, centres + (uint64_t)gg * d);
            best[gg].id = gg;
        }
        qsort(best, S, sizeof(sg_cand), sg_cmp);
        for (gg = 0; gg < ell; gg++) sh[(uint64_t)ii * ell + gg] = best[gg].id;
        free(best);
    }
    /* 2. members in ascending point id, entries, virtual vectors */
    for (i = 0; i < nv; i++) cnt[sh[i]]++;
    for (g = 0; g < S; g++) gstart[g + 1] = gstart[g] + cnt[g];
    for (g = 0; g < S; g++) cur[g] = gstart[g];
    for (i = 0; i < n; i++)
        for (t = 0; t < ell; t++) {
            g = sh[i * ell + t];
            vid[i * ell + t] = (uint32_t)cur[g];
            vpt[cur[g]++] = (uint32_t)i;
        }
    for (g = 0; g < S; g++) {
        float bd = INFINITY;
        entry[g] = ORC_NONE;
        epos[g] = 0;
        for (v = gstart[g]; v < gstart[g + 1]; v++) {
            float dd = sg_centre_dist(X, dtype, d, vpt[v], centres + (uint64_t)g * d);
            if (entry[g] == ORC_NONE || dd < bd) { bd = dd; entry[g] = (uint32_t)v; }
        }
        if (entry[g] != ORC_NONE) epos[g] = (uint32_t)(entry[g] - gstart[g]);
        cap[g] = (uint32_t)(batch_frac * (float)cnt[g]);
        if (cap[g] < 1) cap[g] = 1;
    }
    for (v = 0; v < nv; v++)
        memcpy(vbase + v * d * esz, (const unsigned char *)X + (uint64_t)vpt[v] * d * esz, d * esz);
    for (i = 0; i < nv * R; i++) vadj[i] = ORC_NONE;

    /* 3. two passes of batched insertion */
    for (pass = 0; pass < 2; pass++) {
        float a = pass == 0 ? 1.0f : alpha;
        uint32_t *start = (uint32_t *)calloc(S, sizeof(uint32_t));   /* next position per shard */
        uint32_t round;
        for (round = 0;; round++) {
            uint64_t nb = 0, b, npairs = 0, q0;
            uint32_t *mem, *V, *nvis;
            sg_pair *pairs;
            for (g = 0; g < S; g++) {
                uint32_t size = pass == 0 ? (round == 0 ? 1u : (round - 1 < 31 ? 1u << (round - 1) : cap[g])) : cap[g];
                if (size > cap[g]) size = cap[g];
                if (start[g] < cnt[g]) nb += (cnt[g] - start[g] < size) ? cnt[g] - start[g] : size;
            }
            if (nb == 0) { free(start); break; }
            mem = (uint32_t *)malloc(sizeof(uint32_t) * nb);
            V = (uint32_t *)malloc(sizeof(uint32_t) * nb * iter_cap);
            nvis = (uint32_t *)malloc(sizeof(uint32_t) * nb);
            pairs = (sg_pair *)malloc(sizeof(sg_pair) * nb * R);
            nb = 0;
            for (g = 0; g < S; g++) {
                uint32_t size = pass == 0 ? (round == 0 ? 1u : (round - 1 < 31 ? 1u << (round - 1) : cap[g])) : cap[g];
                uint32_t e;
                if (size > cap[g]) size = cap[g];
                for (e = 0; e < size && start[g] < cnt[g]; e++, start[g]++) {
                    uint32_t pos = start[g];       /* insertion position -> member index */
                    uint32_t idx = pos == 0 ? epos[g] : (pos - 1 < epos[g] ? pos - 1 : pos);
                    mem[nb++] = (uint32_t)(gstart[g] + idx);
                }
            }
            /* GreedySearch of every member against the round's starting graph */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
            for (int64_t bb = 0; bb < (int64_t)nb; bb++) {
                uint32_t p = mem[bb], gg = sh[0], k1;
                float d1;
                int32_t st;
                uint64_t nd;
                orc_index ix;
                uint32_t lo = 0, hi = S;
                while (hi - lo > 1) {              /* shard of virtual node p */
                    uint32_t mid = (lo + hi) / 2;
                    if (gstart[mid] <= p) lo = mid; else hi = mid;
                }
                while (lo + 1 < S && gstart[lo + 1] <= p) lo++;
                gg = lo;
                memset(&ix, 0, sizeof ix);
                ix.d = d; ix.M = 1; ix.R = R; ix.medoid = entry[gg]; ix.n = nv; ix.dtype = dtype;
                ix.adj = vadj; ix.base = vbase;
                search_one(&ix, vbase + (uint64_t)p * d * esz, 1, 1, Lb, log2z, iter_cap, &k1, &d1,
                           &nvis[bb], &st, &nd, V + (uint64_t)bb * iter_cap, iter_cap, 0);
                if (nvis[bb] > iter_cap) nvis[bb] = iter_cap;
            }
            /* RobustPrune of every member's visited set and current list */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
            for (int64_t bb = 0; bb < (int64_t)nb; bb++) {
                uint32_t p = mem[bb], r;
                uint32_t *c = (uint32_t *)malloc(sizeof(uint32_t) * (iter_cap + R));
                uint32_t nc = 0;
                for (r = 0; r < nvis[bb]; r++) c[nc++] = V[(uint64_t)bb * iter_cap + r];
                for (r = 0; r < R; r++) c[nc++] = vadj[(uint64_t)p * R + r];
                sg_list(vbase, dtype, d, p, c, nc, a, R, 1, vadj + (uint64_t)p * R);
                free(c);
            }
            /* reverse edges */
            for (b = 0; b < nb; b++) {
                uint32_t p = mem[b], r;
                for (r = 0; r < R; r++) {
                    uint32_t q = vadj[(uint64_t)p * R + r];
                    if (q == ORC_NONE) break;
                    pairs[npairs].q = q;
                    pairs[npairs].p = p;
                    npairs++;
                }
            }
            qsort(pairs, npairs, sizeof(sg_pair), sg_pair_cmp);
            {
                uint64_t *segs = (uint64_t *)malloc(sizeof(uint64_t) * (npairs + 1));
                uint64_t ns = 0;
                for (q0 = 0; q0 < npairs; q0++)
                    if (q0 == 0 || pairs[q0].q != pairs[q0 - 1].q) segs[ns++] = q0;
                segs[ns] = npairs;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
                for (int64_t sgi = 0; sgi < (int64_t)ns; sgi++) {
                    uint64_t lo = segs[sgi], hi = segs[sgi + 1], e;
                    uint32_t q = pairs[lo].q, r, nc = 0;
                    uint32_t *c = (uint32_t *)malloc(sizeof(uint32_t) * (R + (hi - lo)));
                    for (r = 0; r < R; r++) c[nc++] = vadj[(uint64_t)q * R + r];
                    for (e = lo; e < hi; e++) c[nc++] = pairs[e].p;
                    sg_list(vbase, dtype, d, q, c, nc, a, R, 0, vadj + (uint64_t)q * R);
                    free(c);
                }
                free(segs);
            }
            free(mem); free(V); free(nvis); free(pairs);
        }
    }
    /* 4. merge the shard lists of every point */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
#endif
    for (int64_t ii = 0; ii < (int64_t)n; ii++) {
        uint32_t *c = (uint32_t *)malloc(sizeof(uint32_t) * ell * R);
        uint32_t nc = 0, tt, r;
        for (tt = 0; tt < ell; tt++) {
            uint32_t vv = vid[(uint64_t)ii * ell + tt];
            for (r = 0; r < R; r++) {
                uint32_t q = vadj[(uint64_t)vv * R + r];
                if (q != ORC_NONE) c[nc++] = vpt[q];
            }
        }
        sg_list(X, dtype, d, (uint32_t)ii, c, nc, alpha, R, 0, adj + (uint64_t)ii * R);
        free(c);
    }
    if (shard_of) memcpy(shard_of, sh, sizeof(uint32_t) * nv);
done:
    free(sh); free(vid); free(cnt); free(gstart); free(cur); free(vpt); free(vadj); free(entry);
    free(epos); free(cap); free(vbase);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Brute-force ground truth (§6.3, k-recall@k): exact distances in FP64    */
/* (exact integers for integer data) to every point, sorted by             */
/* (distance, id), first k.                                                */
/* ---------------------------------------------------------------------- */

void orc_bruteforce_knn(const void *base, const void *queries, int dtype, uint64_t n,
                        uint32_t nq, uint32_t d, uint32_t k, uint32_t *ids, double *dists,
                        int nthreads)
{
    int64_t qi;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#else
    (void)nthreads;
#endif
    for (qi = 0; qi < (int64_t)nq; qi++) {
        orc_dpair *top = (orc_dpair *)malloc(sizeof(orc_dpair) * (k + 1));
        uint32_t nt = 0, j, t;
        uint64_t i;
        for (i = 0; i < n; i++) {
            orc_dpair e;
            double acc = 0.0;
            if (dtype == ORC_F32) {
                const float *qf = (const float *)queries + (uint64_t)qi * d;
                const float *xf = (const float *)base + i * d;
                for (j = 0; j < d; j++) {
                    double t2 = (double)qf[j] - (double)xf[j];
                    acc += t2 * t2;
                }
            } else {
                int64_t ia = 0;
                for (j = 0; j < d; j++) {
                    int64_t t2 = (int64_t)elem_i(queries, dtype, (uint64_t)qi * d + j) -
                                 (int64_t)elem_i(base, dtype, i * d + j);
                    ia += t2 * t2;
                }
                acc = (double)ia;
            }
            e.dist = acc; e.id = (uint32_t)i;
            if (nt == k && dpair_cmp(&e, &top[k - 1]) >= 0) continue;
            t = (nt < k) ? nt++ : k - 1;
            while (t > 0 && dpair_cmp(&top[t - 1], &e) > 0) { top[t] = top[t - 1]; t--; }
            top[t] = e;
        }
        for (j = 0; j < k; j++) {
            ids[(uint64_t)qi * k + j] = j < nt ? top[j].id : ORC_NONE;
            dists[(uint64_t)qi * k + j] = j < nt ? top[j].dist : INFINITY;
        }
        free(top);
    }
}
