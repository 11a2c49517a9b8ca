/*
 * Synthetic-workload index builder: the stand-in for the prebuilt DiskANN
 * index and the ground-truth files that the paper's datasets ship with.
 *
 * The paper searches an index it does not build (§1: the graph is taken from
 * DiskANN; §6.3: R=64, L=200, pruning parameter 1.2; PQ with 256 centroids per
 * subspace).  This file builds such an index quickly and deterministically
 * (any thread count gives the same bytes) for the large synthetic
 * configurations, with OpenMP across points and clusters:
 *   wl_pq_train      k-means codebooks, 256 centroids per subspace
 *   wl_pq_encode     nearest centroid per subspace
 *   wl_medoids       nearest point to the mean of each group of points
 *   wl_cluster_graph clustered graph: per cluster, exact k-nearest candidates
 *                    pruned by the Vamana RobustPrune rule, reverse edges,
 *                    plus links to other clusters' medoids
 *   wl_bruteforce    exact k nearest neighbours (ground truth)
 * Nothing here is on the search path; the search reads only the arrays this
 * file writes.  Floating-point accumulation orders are fixed; partial sums
 * are combined in a fixed chunk order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define WL_NONE 0xFFFFFFFFu
enum { WL_U8 = 0, WL_I8 = 1, WL_F32 = 2 };

static inline float wl_elem(const void *v, int dt, uint64_t i)
{
    if (dt == WL_U8) return (float)((const uint8_t *)v)[i];
    if (dt == WL_I8) return (float)((const int8_t *)v)[i];
    return ((const float *)v)[i];
}

/* squared distance between rows a and b of X (same dtype); integer data is
 * exact (returned as float; exact below 2^24), float data is summed in
 * ascending j. */
static inline float wl_dist(const void *X, int dt, uint32_t d, uint64_t a, uint64_t b)
{
    uint32_t j;
    if (dt == WL_U8) {
        const uint8_t *x = (const uint8_t *)X + a * d, *y = (const uint8_t *)X + b * d;
        int32_t acc = 0;
        for (j = 0; j < d; j++) { int32_t t = (int32_t)x[j] - (int32_t)y[j]; acc += t * t; }
        return (float)acc;
    } else if (dt == WL_I8) {
        const int8_t *x = (const int8_t *)X + a * d, *y = (const int8_t *)X + b * d;
        int32_t acc = 0;
        for (j = 0; j < d; j++) { int32_t t = (int32_t)x[j] - (int32_t)y[j]; acc += t * t; }
        return (float)acc;
    } else {
        const float *x = (const float *)X + a * d, *y = (const float *)X + b * d;
        float acc = 0.0f;
        for (j = 0; j < d; j++) { float t = x[j] - y[j]; acc += t * t; }
        return acc;
    }
}

/* ---------------------------------------------------------------------- */
/* PQ codebooks: k-means (256 centroids) per subspace on a float sample.   */
/* ---------------------------------------------------------------------- */
#define WL_NCHUNK 64

static uint32_t wl_nearest256(const float *x, const float *cT, uint32_t ds, float *dist)
{
    uint32_t c, j, bc = 0;
    float best;
    for (c = 0; c < 256; c++) dist[c] = 0.0f;
    for (j = 0; j < ds; j++) {
        float xj = x[j];
        const float *row = cT + (size_t)j * 256;
        for (c = 0; c < 256; c++) { float t = xj - row[c]; dist[c] = dist[c] + t * t; }
    }
    best = dist[0];
    for (c = 1; c < 256; c++) if (dist[c] < best) { best = dist[c]; bc = c; }
    return bc;
}

void wl_pq_train(const float *Xs, uint64_t ns, uint32_t d, uint32_t M, const uint32_t *off,
                 const uint64_t *init, uint32_t iters, float *codebook)
{
    uint32_t s;
    for (s = 0; s < M; s++) {
        uint32_t o = off[s], ds = off[s + 1] - off[s], it, c, j;
        float *cent = (float *)malloc(sizeof(float) * 256 * ds);
        float *cT = (float *)malloc(sizeof(float) * 256 * ds);
        double *sums = (double *)malloc(sizeof(double) * WL_NCHUNK * 256 * ds);
        uint64_t *cnt = (uint64_t *)malloc(sizeof(uint64_t) * WL_NCHUNK * 256);
        for (c = 0; c < 256; c++)
            for (j = 0; j < ds; j++) cent[c * ds + j] = Xs[init[(size_t)s * 256 + c] * d + o + j];
        for (it = 0; it < iters; it++) {
            int64_t ch;
            for (c = 0; c < 256; c++)
                for (j = 0; j < ds; j++) cT[(size_t)j * 256 + c] = cent[c * ds + j];
            memset(sums, 0, sizeof(double) * WL_NCHUNK * 256 * ds);
            memset(cnt, 0, sizeof(uint64_t) * WL_NCHUNK * 256);
#pragma omp parallel for schedule(dynamic, 1)
            for (ch = 0; ch < WL_NCHUNK; ch++) {
                uint64_t lo = ns * (uint64_t)ch / WL_NCHUNK, hi = ns * (uint64_t)(ch + 1) / WL_NCHUNK, i;
                double *cs = sums + (size_t)ch * 256 * ds;
                uint64_t *cc = cnt + (size_t)ch * 256;
                float dist[256];
                for (i = lo; i < hi; i++) {
                    const float *x = Xs + i * d + o;
                    uint32_t bc = wl_nearest256(x, cT, ds, dist), jj;
                    cc[bc]++;
                    for (jj = 0; jj < ds; jj++) cs[bc * ds + jj] += (double)x[jj];
                }
            }
            for (c = 0; c < 256; c++) {
                uint64_t tot = 0;
                int ch2;
                for (ch2 = 0; ch2 < WL_NCHUNK; ch2++) tot += cnt[(size_t)ch2 * 256 + c];
                if (!tot) continue;
                for (j = 0; j < ds; j++) {
                    double a = 0.0;
                    for (ch2 = 0; ch2 < WL_NCHUNK; ch2++) a += sums[((size_t)ch2 * 256 + c) * ds + j];
                    cent[c * ds + j] = (float)(a / (double)tot);
                }
            }
        }
        memcpy(codebook + (size_t)256 * o, cent, sizeof(float) * 256 * ds);
        free(cent); free(cT); free(sums); free(cnt);
    }
}

void wl_pq_encode(const void *X, int dt, uint64_t n, uint32_t d, uint32_t M, const uint32_t *off,
                  const float *codebook, uint8_t *codes)
{
    float *cT = (float *)malloc(sizeof(float) * 256 * d);
    int64_t i;
    uint32_t s0;
    for (s0 = 0; s0 < M; s0++) {
        uint32_t o = off[s0], ds = off[s0 + 1] - off[s0], c, j;
        for (c = 0; c < 256; c++)
            for (j = 0; j < ds; j++)
                cT[(size_t)256 * o + (size_t)j * 256 + c] = codebook[(size_t)256 * o + c * ds + j];
    }
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)n; i++) {
        uint32_t s, j;
        float x[1024], dist[256];
        for (j = 0; j < d && j < 1024; j++) x[j] = wl_elem(X, dt, (uint64_t)i * d + j);
        for (s = 0; s < M; s++) {
            uint32_t o = off[s], ds = off[s + 1] - off[s];
            codes[(uint64_t)i * M + s] = (uint8_t)wl_nearest256(x + o, cT + (size_t)256 * o, ds, dist);
        }
    }
    free(cT);
}

/* For each group g (members[gstart[g] .. gstart[g+1])), the member nearest
 * (FP64) to the group mean; ties to the smaller id. */
void wl_medoids(const void *X, int dt, uint32_t d, const uint32_t *members,
                const uint64_t *gstart, uint32_t ng, uint32_t *out)
{
    int64_t g;
#pragma omp parallel for schedule(dynamic, 1)
    for (g = 0; g < (int64_t)ng; g++) {
        uint64_t lo = gstart[g], hi = gstart[g + 1], i;
        double *mean = (double *)calloc(d, sizeof(double));
        double best = INFINITY;
        uint32_t bi = WL_NONE, j;
        for (i = lo; i < hi; i++)
            for (j = 0; j < d; j++) mean[j] += (double)wl_elem(X, dt, (uint64_t)members[i] * d + j);
        for (j = 0; j < d; j++) mean[j] /= (double)(hi > lo ? hi - lo : 1);
        for (i = lo; i < hi; i++) {
            double acc = 0.0;
            for (j = 0; j < d; j++) {
                double t = (double)wl_elem(X, dt, (uint64_t)members[i] * d + j) - mean[j];
                acc += t * t;
            }
            if (acc < best || (acc == best && members[i] < bi)) { best = acc; bi = members[i]; }
        }
        out[g] = bi;
        free(mean);
    }
}

/* ---------------------------------------------------------------------- */
/* Clustered graph.                                                        */
/* ---------------------------------------------------------------------- */

typedef struct { float d; uint32_t i; } wl_pair;

static int wl_pair_cmp(const void *a, const void *b)
{
    const wl_pair *x = (const wl_pair *)a, *y = (const wl_pair *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->i < y->i) ? -1 : (x->i > y->i);
}

/* Deterministic quickselect: afterwards a[0..k) hold the k smallest pairs
 * (in no particular order).  Keys are unique (ids differ). */
static void wl_select(wl_pair *a, uint32_t n, uint32_t k)
{
    uint32_t lo = 0, hi = n;
    if (k >= n) return;
    while (hi - lo > 1) {
        wl_pair piv = a[lo + (hi - lo) / 2], t;
        uint32_t i = lo, lt = lo, gt = hi;
        while (i < gt) {
            int c = wl_pair_cmp(&a[i], &piv);
            if (c < 0) { t = a[lt]; a[lt] = a[i]; a[i] = t; lt++; i++; }
            else if (c > 0) { gt--; t = a[gt]; a[gt] = a[i]; a[i] = t; }
            else i++;
        }
        if (k <= lt) hi = lt;
        else if (k >= gt) lo = gt;
        else return;
    }
}

/* RobustPrune (Vamana, §2.2 of the paper): keep the nearest remaining
 * candidate, drop every candidate c with alpha^2 * d(kept, c) <= d(p, c).
 * Candidates carry their distance to p; distances between candidates are
 * computed on demand.  P maps local indices to point ids. */
static uint32_t wl_prune(const void *X, int dt, uint32_t d, const uint32_t *P, wl_pair *cand,
                         uint32_t nc, float alpha, uint32_t R, uint32_t *out, unsigned char *alive)
{
    uint32_t i, j, nout = 0;
    float a2 = alpha * alpha;
    qsort(cand, nc, sizeof(wl_pair), wl_pair_cmp);
    for (i = 0; i < nc; i++) alive[i] = 1;
    for (i = 0; i < nc && nout < R; i++) {
        if (!alive[i]) continue;
        out[nout++] = cand[i].i;
        for (j = i + 1; j < nc; j++)
            if (alive[j] && a2 * wl_dist(X, dt, d, P[cand[i].i], P[cand[j].i]) <= cand[j].d)
                alive[j] = 0;
    }
    return nout;
}

/* members/gstart: points of each cluster (sorted ids).  For every point:
 * Rin = R - nx in-cluster neighbours (K = 2*Rin exact nearest candidates,
 * RobustPrune, then reverse edges with re-pruning), followed by nx links to
 * the medoids of the clusters listed in xclu (n*nx cluster ids, drawn by the
 * caller's seeded generator).  A cluster medoid instead keeps R - nh
 * in-cluster neighbours followed by nh links to the medoids listed in
 * hclu (ng*nh cluster ids).  adj: n*R, unused slots 0xFFFFFFFF. */
int wl_cluster_graph(const void *X, int dt, uint32_t d, uint64_t n, const uint32_t *members,
                     const uint64_t *gstart, uint32_t ng, const uint32_t *medoids, uint32_t R,
                     float alpha, uint32_t nx, const uint32_t *xclu, uint32_t nh,
                     const uint32_t *hclu, uint32_t *adj)
{
    uint32_t Rin = R - nx;
    int64_t g;
    int err = 0;
    if (nx >= R || nh >= R || Rin > 1000) return -1;
    for (uint64_t i = 0; i < n * (uint64_t)R; i++) adj[i] = WL_NONE;
#pragma omp parallel for schedule(dynamic, 1)
    for (g = 0; g < (int64_t)ng; g++) {
        uint64_t lo = gstart[g], hi = gstart[g + 1];
        uint32_t m = (uint32_t)(hi - lo), a, b, K = 2 * Rin;
        const uint32_t *P = members + lo;
        uint32_t *nb, *deg, *tmp;
        wl_pair *cand;
        unsigned char *alive;
        if (m == 0) continue;
        if (K > m - 1) K = m - 1;
        nb = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * Rin);
        deg = (uint32_t *)calloc(m, sizeof(uint32_t));
        cand = (wl_pair *)malloc(sizeof(wl_pair) * (m + Rin + 2));
        alive = (unsigned char *)malloc(m + Rin + 2);
        tmp = (uint32_t *)malloc(sizeof(uint32_t) * (Rin + 1));
        if (!nb || !deg || !cand || !alive || !tmp) {
#pragma omp atomic write
            err = -2;
            free(nb); free(deg); free(cand); free(alive); free(tmp);
            continue;
        }
        /* forward lists: K exact nearest, pruned */
        for (a = 0; a < m; a++) {
            uint32_t nc = 0;
            for (b = 0; b < m; b++)
                if (b != a) { cand[nc].d = wl_dist(X, dt, d, P[a], P[b]); cand[nc].i = b; nc++; }
            wl_select(cand, nc, K);
            if (nc > K) nc = K;
            deg[a] = wl_prune(X, dt, d, P, cand, nc, alpha, Rin, nb + (size_t)a * Rin, alive);
        }
        /* reverse edges: every node's candidates become its forward list
         * plus the nodes that chose it; one more RobustPrune over that union */
        {
            uint32_t *rcnt = (uint32_t *)calloc(m + 1, sizeof(uint32_t));
            uint32_t *rsrc, *fill, t;
            for (a = 0; a < m; a++)
                for (t = 0; t < deg[a]; t++) rcnt[nb[(size_t)a * Rin + t] + 1]++;
            for (a = 0; a < m; a++) rcnt[a + 1] += rcnt[a];
            rsrc = (uint32_t *)malloc(sizeof(uint32_t) * (rcnt[m] + 1));
            fill = (uint32_t *)calloc(m, sizeof(uint32_t));
            for (a = 0; a < m; a++)
                for (t = 0; t < deg[a]; t++) {
                    uint32_t j = nb[(size_t)a * Rin + t];
                    rsrc[rcnt[j] + fill[j]++] = a;
                }
            {
                uint32_t *nb2 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * Rin);
                uint32_t *deg2 = (uint32_t *)calloc(m, sizeof(uint32_t));
                wl_pair *c2 = (wl_pair *)malloc(sizeof(wl_pair) * (Rin + 1));
                for (a = 0; a < m; a++) {
                    uint32_t nc = 0, nr = rcnt[a + 1] - rcnt[a], r, q2, dup;
                    wl_pair *cc = cand;
                    if (nr + deg[a] + 1 > m + Rin + 2) nr = m + Rin + 1 - deg[a];
                    for (t = 0; t < deg[a]; t++) {
                        uint32_t j = nb[(size_t)a * Rin + t];
                        cc[nc].i = j; cc[nc].d = wl_dist(X, dt, d, P[a], P[j]); nc++;
                    }
                    for (r = 0; r < nr; r++) {
                        uint32_t j = rsrc[rcnt[a] + r];
                        dup = 0;
                        for (q2 = 0; q2 < deg[a]; q2++) if (nb[(size_t)a * Rin + q2] == j) { dup = 1; break; }
                        if (dup) continue;
                        cc[nc].i = j; cc[nc].d = wl_dist(X, dt, d, P[a], P[j]); nc++;
                    }
                    deg2[a] = wl_prune(X, dt, d, P, cc, nc, alpha, Rin, nb2 + (size_t)a * Rin, alive);
                }
                memcpy(nb, nb2, sizeof(uint32_t) * (size_t)m * Rin);
                memcpy(deg, deg2, sizeof(uint32_t) * m);
                free(nb2); free(deg2); free(c2);
            }
            /* repair: a node nobody links to gets an edge from the nearest of
             * its own neighbours that has room, or that can give up its
             * farthest edge without orphaning that edge's target */
            {
                uint32_t *indeg = (uint32_t *)calloc(m, sizeof(uint32_t));
                for (a = 0; a < m; a++)
                    for (t = 0; t < deg[a]; t++) indeg[nb[(size_t)a * Rin + t]]++;
                for (a = 0; a < m; a++) {
                    if (indeg[a] || !deg[a]) continue;
                    for (t = 0; t < deg[a]; t++) {
                        uint32_t j = nb[(size_t)a * Rin + t];
                        uint32_t *lj = nb + (size_t)j * Rin;
                        if (deg[j] < Rin) { lj[deg[j]++] = a; indeg[a]++; break; }
                        if (indeg[lj[deg[j] - 1]] > 1) {
                            indeg[lj[deg[j] - 1]]--;
                            lj[deg[j] - 1] = a;
                            indeg[a]++;
                            break;
                        }
                    }
                }
                free(indeg);
            }
            free(rcnt); free(rsrc); free(fill);
        }
        /* write global adjacency */
        for (a = 0; a < m; a++) {
            uint32_t p = P[a], r, w = 0;
            uint32_t *out = adj + (uint64_t)p * R;
            int is_med = (p == medoids[g]);
            uint32_t keep = is_med ? (R - nh < deg[a] ? R - nh : deg[a]) : deg[a];
            for (r = 0; r < keep; r++) out[w++] = P[nb[(size_t)a * Rin + r]];
            if (is_med) {
                for (r = 0; r < nh; r++) {
                    uint32_t c2 = hclu[(size_t)g * nh + r];
                    if (c2 < ng && c2 != (uint32_t)g && medoids[c2] != WL_NONE) out[w++] = medoids[c2];
                }
            } else {
                for (r = 0; r < nx; r++) {
                    uint32_t c2 = xclu[(uint64_t)p * nx + r];
                    if (c2 < ng && c2 != (uint32_t)g && medoids[c2] != WL_NONE) out[w++] = medoids[c2];
                }
            }
            /* drop duplicates (two links to the same medoid) */
            for (r = 0; r < w; r++) {
                uint32_t q2;
                for (q2 = 0; q2 < r; q2++) if (out[q2] == out[r]) { out[r] = WL_NONE; break; }
            }
            {
                uint32_t w2 = 0;
                for (r = 0; r < w; r++) if (out[r] != WL_NONE) out[w2++] = out[r];
                for (r = w2; r < R; r++) out[r] = WL_NONE;
            }
        }
        free(nb); free(deg); free(cand); free(alive); free(tmp);
    }
    return err;
}

/* ---------------------------------------------------------------------- */
/* Exact k nearest neighbours, sorted by (distance, id).  Distances are      */
/* exact integers for integer data and FP64 for float data.                */
/* ---------------------------------------------------------------------- */
void wl_bruteforce(const void *base, const void *queries, int dt, uint64_t n, uint32_t nq,
                   uint32_t d, uint32_t k, uint32_t *ids, double *dists)
{
    const uint32_t QB = 16, XB = 2048;
    int64_t qb;
    int64_t nqb = ((int64_t)nq + QB - 1) / QB;
#pragma omp parallel for schedule(dynamic, 1)
    for (qb = 0; qb < nqb; qb++) {
        uint32_t q0 = (uint32_t)qb * QB, q1 = q0 + QB < nq ? q0 + QB : nq, qi;
        double *topd = (double *)malloc(sizeof(double) * QB * (k + 1));
        uint32_t *topi = (uint32_t *)malloc(sizeof(uint32_t) * QB * (k + 1));
        uint32_t nt[64];
        uint64_t x0;
        for (qi = 0; qi < QB; qi++) nt[qi] = 0;
        for (x0 = 0; x0 < n; x0 += XB) {
            uint64_t x1 = x0 + XB < n ? x0 + XB : n, x;
            for (qi = q0; qi < q1; qi++) {
                double *td = topd + (size_t)(qi - q0) * (k + 1);
                uint32_t *ti = topi + (size_t)(qi - q0) * (k + 1);
                uint32_t *cnt = &nt[qi - q0];
                for (x = x0; x < x1; x++) {
                    double dv;
                    uint32_t j, t;
                    if (dt == WL_U8) {
                        const uint8_t *a = (const uint8_t *)queries + (uint64_t)qi * d;
                        const uint8_t *b = (const uint8_t *)base + x * d;
                        int32_t acc = 0;
                        for (j = 0; j < d; j++) { int32_t u = (int32_t)a[j] - (int32_t)b[j]; acc += u * u; }
                        dv = (double)acc;
                    } else if (dt == WL_I8) {
                        const int8_t *a = (const int8_t *)queries + (uint64_t)qi * d;
                        const int8_t *b = (const int8_t *)base + x * d;
                        int32_t acc = 0;
                        for (j = 0; j < d; j++) { int32_t u = (int32_t)a[j] - (int32_t)b[j]; acc += u * u; }
                        dv = (double)acc;
                    } else {
                        const float *a = (const float *)queries + (uint64_t)qi * d;
                        const float *b = (const float *)base + x * d;
                        double acc = 0.0;
                        for (j = 0; j < d; j++) { double u = (double)a[j] - (double)b[j]; acc += u * u; }
                        dv = acc;
                    }
                    if (*cnt == k && !(dv < td[k - 1] || (dv == td[k - 1] && x < ti[k - 1]))) continue;
                    t = (*cnt < k) ? (*cnt)++ : k - 1;
                    while (t > 0 && (td[t - 1] > dv || (td[t - 1] == dv && ti[t - 1] > x))) {
                        td[t] = td[t - 1]; ti[t] = ti[t - 1]; t--;
                    }
                    td[t] = dv; ti[t] = (uint32_t)x;
                }
            }
        }
        for (qi = q0; qi < q1; qi++) {
            uint32_t j;
            for (j = 0; j < k; j++) {
                int ok = j < nt[qi - q0];
                ids[(uint64_t)qi * k + j] = ok ? topi[(size_t)(qi - q0) * (k + 1) + j] : WL_NONE;
                dists[(uint64_t)qi * k + j] = ok ? topd[(size_t)(qi - q0) * (k + 1) + j] : INFINITY;
            }
        }
        free(topd); free(topi);
    }
}

/* ---------------------------------------------------------------------- */
/* Index for checks at full size, without nearest-neighbour work: seeded    */
/* values from a counter-based hash (SplitMix64 finaliser), so any thread   */
/* count writes the same bytes.  Points fall into ng contiguous id ranges   */
/* ("clusters"); member a of a cluster of m members links to the members    */
/* (a + 1 + (s_a + r) mod (m - 1)) mod m, r < R - nx, s_a drawn per point    */
/* (distinct, never itself), then to the first member of nx other clusters  */
/* (repeats dropped, 0xFFFFFFFF padding).  Vectors, queries and codes are   */
/* uniform; the codebook covers the element range.                          */
/* ---------------------------------------------------------------------- */

static inline uint64_t wl_mix(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

static void wl_fill_rows(void *X, int dt, uint64_t rows, uint32_t d, uint64_t seed)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)rows; i++) {
        uint32_t j;
        for (j = 0; j < d; j++) {
            uint64_t h = wl_mix(seed ^ wl_mix((uint64_t)i * d + j));
            if (dt == WL_U8) ((uint8_t *)X)[(uint64_t)i * d + j] = (uint8_t)(h >> 56);
            else if (dt == WL_I8) ((int8_t *)X)[(uint64_t)i * d + j] = (int8_t)(uint8_t)(h >> 56);
            else ((float *)X)[(uint64_t)i * d + j] = (float)((int64_t)(h >> 40) - (1ll << 23)) / (float)(1 << 23);
        }
    }
}

int wl_scale_index(int dt, uint64_t n, uint32_t d, uint32_t M, uint32_t R, uint32_t nx, uint32_t ng,
                   uint32_t nq, uint64_t seed, void *base, void *queries, float *codebook,
                   uint8_t *codes, uint32_t *adj)
{
    uint64_t per = (n + ng - 1) / ng;
    uint32_t Rin = R - nx, j;
    int64_t i;
    if (nx >= R || ng < 2 || per < (uint64_t)Rin + 1) return -1;
    wl_fill_rows(base, dt, n, d, seed * 4 + 0);
    wl_fill_rows(queries, dt, nq, d, seed * 4 + 1);
    for (j = 0; j < 256 * d; j++) {
        uint64_t h = wl_mix((seed * 4 + 2) ^ wl_mix(j));
        float u = (float)(h >> 40) / (float)(1 << 24);        /* [0, 1) */
        codebook[j] = dt == WL_U8 ? 255.0f * u : dt == WL_I8 ? 255.0f * u - 128.0f : 2.0f * u - 1.0f;
    }
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)n; i++) {
        uint64_t g = (uint64_t)i / per, lo = g * per, hi = lo + per < n ? lo + per : n;
        uint64_t m = hi - lo, a = (uint64_t)i - lo, s;
        uint32_t r, w = 0, q;
        uint32_t *row = adj + (uint64_t)i * R;
        for (s = 0; s < M; s++) codes[(uint64_t)i * M + s] = (uint8_t)(wl_mix((seed * 4 + 3) ^ wl_mix((uint64_t)i * M + s)) >> 56);
        if (m < (uint64_t)Rin + 1) {             /* a short last cluster: link to everyone */
            for (s = 0; s < m; s++) if (s != a && w < Rin) row[w++] = (uint32_t)(lo + s);
        } else {
            uint64_t st = wl_mix(seed ^ (0xABCDull << 40) ^ (uint64_t)i) % (m - 1);
            for (r = 0; r < Rin; r++) row[w++] = (uint32_t)(lo + (a + 1 + (st + r) % (m - 1)) % m);
        }
        for (r = 0; r < nx; r++) {
            uint64_t g2 = (g + 1 + wl_mix(seed ^ (0x5151ull << 40) ^ ((uint64_t)i * nx + r)) % (ng - 1)) % ng;
            uint32_t t = (uint32_t)(g2 * per);
            int dup = 0;
            if ((uint64_t)t >= n) continue;
            for (q = 0; q < w; q++) if (row[q] == t) dup = 1;
            if (!dup) row[w++] = t;
        }
        for (; w < R; w++) row[w] = WL_NONE;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Equal-weight Gaussian mixture with low-rank components, counter-based so */
/* that any thread count writes the same bytes (the large configurations): */
/* point i takes component c_i = h(seed, i, 0) mod ncomp and               */
/*   x = centre[c_i] + A[c_i] z + noise * e,  z ~ N(0, I_rank), e ~ N(0, I_d) */
/* (A[c] stored rank-major, d values per rank; x_j summed over the rank in  */
/* ascending order)                                                          */
/* with every normal drawn as the sum of twelve uniforms minus 6 (Irwin-    */
/* Hall: mean 0, variance 1; the uniforms are 16-bit pieces of SplitMix64   */
/* counters, so every sum is exact in FP32 and no libm call is made: x86   */
/* and Arm hosts write the same bytes); the sum over the rank in ascending  */
/* order in FP32 (no fused multiply-add); integers rounded half to even and */
/* clipped to the element range.                                            */
/* ---------------------------------------------------------------------- */

static inline float wl_normal(uint64_t seed, uint64_t i, uint64_t k)
{
    float s = 0.0f;
    int t, q;
    for (t = 0; t < 3; t++) {
        uint64_t h = wl_mix((seed << 48) ^ (i * 0x100000001B3ull + k * 3 + (uint64_t)t + 1));
        for (q = 0; q < 4; q++) s = s + ((float)((h >> (16 * q)) & 0xFFFFu) + 0.5f) / 65536.0f;
    }
    return s - 6.0f;
}

int wl_mixture(void *X, int dt, uint64_t n, uint32_t d, const float *centres, uint32_t ncomp,
               const float *factors, uint32_t rank, float noise, uint64_t seed, uint32_t *labels)
{
    int64_t i;
    if (rank > 64 || ncomp == 0 || d > 512) return -1;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)n; i++) {
        float z[64], x[512], e[512];
        uint32_t c = (uint32_t)(wl_mix((seed << 48) ^ ((uint64_t)i * 0x100000001B3ull)) % ncomp), r, j;
        const float *cen = centres + (uint64_t)c * d, *A = factors + (uint64_t)c * d * rank;
        for (r = 0; r < rank; r++) z[r] = wl_normal(seed, (uint64_t)i, r);
        for (j = 0; j < d; j++) e[j] = wl_normal(seed, (uint64_t)i, 64 + j);
        for (j = 0; j < d; j++) x[j] = cen[j];
        for (r = 0; r < rank; r++)              /* factors stored rank-major: A[r][j] */
            for (j = 0; j < d; j++) x[j] = x[j] + A[(uint64_t)r * d + j] * z[r];
        for (j = 0; j < d; j++) {
            float v;
            x[j] = x[j] + noise * e[j];
            v = rintf(x[j]);
            if (dt == WL_U8) ((uint8_t *)X)[(uint64_t)i * d + j] = (uint8_t)(v < 0.f ? 0.f : v > 255.f ? 255.f : v);
            else if (dt == WL_I8) ((int8_t *)X)[(uint64_t)i * d + j] = (int8_t)(v < -128.f ? -128.f : v > 127.f ? 127.f : v);
            else ((float *)X)[(uint64_t)i * d + j] = x[j];
        }
        if (labels) labels[i] = c;
    }
    return 0;
}

int wl_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
