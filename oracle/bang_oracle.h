/*
 * CPU oracle for the BANG search path (arXiv 2401.11324).
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the product path.
 */
#ifndef BANG_ORACLE_H
#define BANG_ORACLE_H

#include <stdint.h>

/* Element types of base vectors and queries (queries share the base type). */
enum { ORC_U8 = 0, ORC_I8 = 1, ORC_F32 = 2 };

/* Everything one search reads.  All arrays are host memory owned by the
 * caller:
 *   off       M+1 subspace offsets (orc_chunk_offsets)
 *   codebook  256*d floats; subspace s at 256*off[s], centroid c at +c*dsub_s
 *   codes     n*M bytes
 *   adj       n*R ids, unused slots 0xFFFFFFFF
 *   base      n*d elements of dtype */
typedef struct {
    uint32_t d, M, R, medoid;
    uint64_t n;
    int dtype;
    const uint32_t *off;
    const float *codebook;
    const uint8_t *codes;
    const uint32_t *adj;
    const void *base;
} orc_index;

void orc_chunk_offsets(uint32_t d, uint32_t M, uint32_t *off);
int orc_pq_train(const float *X, uint32_t d, uint32_t M, const uint32_t *off,
                 const uint64_t *sample, uint64_t ns, const uint64_t *init,
                 uint32_t iters, float *codebook, double *obj_trace);
void orc_pq_encode(const void *X, int dtype, uint64_t n, uint32_t d, uint32_t M,
                   const uint32_t *off, const float *codebook, uint8_t *codes);
uint32_t orc_medoid(const void *X, int dtype, uint64_t n, uint32_t d);
uint32_t orc_robust_prune(const float *X, uint32_t d, uint32_t p, const uint32_t *cand,
                          uint32_t nc, float alpha, uint32_t R, uint32_t *out);
int orc_vamana_build(const float *X, uint64_t n, uint32_t d, uint32_t R, uint32_t Lb,
                     float alpha, uint32_t medoid, const uint32_t *init_adj,
                     const uint32_t *order, uint32_t *adj);
int orc_cluster_graph(const void *X, int dtype, uint32_t d, uint64_t n, const uint32_t *members,
                      const uint64_t *gstart, uint32_t ng, const uint32_t *medoids, uint32_t R,
                      float alpha, uint32_t nx, const uint32_t *xclu, uint32_t nh,
                      const uint32_t *hclu, uint32_t *adj);
/* Overlapping-shard graph (§2.2): see the C file for the steps.  centres is
 * S*d floats; adj is n*R (rows sorted by (distance, id), NONE padding);
 * shard_of (n*ell, may be NULL) receives each point's shards, nearest first. */
int orc_shard_graph(const void *X, int dtype, uint64_t n, uint32_t d, const float *centres,
                    uint32_t S, uint32_t ell, uint32_t R, uint32_t Lb, float alpha,
                    float batch_frac, uint32_t log2z, uint32_t iter_cap, uint32_t *adj,
                    uint32_t *shard_of, int nthreads);
void orc_adc_table_f32(const float *q, uint32_t M, const uint32_t *off,
                       const float *codebook, float *T);
float orc_adc_dist_f32(const float *T, uint32_t M, const uint8_t *code);
float orc_round_bf16(float x);
void orc_adc_table_bf16(const float *T, uint32_t M, float *Tb);
void orc_adc_table_q8(const float *T, uint32_t M, uint8_t *Q);
uint32_t orc_adc_dist_q8(const uint8_t *Q, uint32_t M, const uint8_t *code);
double orc_exact_dist(const void *q, const void *x, int dtype, uint32_t d);
uint32_t orc_fnv1a32_bytes(const unsigned char *b, uint32_t len);
uint64_t orc_fnv1a64_bytes(const unsigned char *b, uint32_t len);
void orc_bloom_positions(uint32_t id, uint32_t log2z, uint32_t *pos2);
int orc_bloom_test(const uint32_t *bits, uint32_t log2z, uint32_t id);
void orc_bloom_insert(uint32_t *bits, uint32_t log2z, uint32_t id);
/* mode 0: PQ distances + re-rank of the expanded nodes (§4); mode 1: exact
 * distances in the loop, no re-rank, result = the worklist's first k (§5.2);
 * mode 2: as mode 0 with the 8-bit table (orc_adc_table_q8); mode 3: as mode 0
 * with the table rounded to BF16 (orc_adc_table_bf16). */
int orc_search(const orc_index *ix, const void *queries, int mode, uint32_t nq, uint32_t k,
               uint32_t L, uint32_t log2z, uint32_t iter_cap, uint32_t *out_ids, float *out_dist,
               uint32_t *out_iters, int32_t *out_status, uint64_t *out_ndist,
               uint32_t *trace, uint32_t trace_cap, int nthreads);
/* orc_search with the choice of re-rank candidates in the PQ modes: 0 = the
 * expanded nodes (§4.8, as orc_search); 1 = the final worklist only (the
 * exact re-rank of the top-L, including entries a capped search left
 * unexpanded). */
int orc_search_rr(const orc_index *ix, const void *queries, int mode, uint32_t nq, uint32_t k,
                  uint32_t L, uint32_t log2z, uint32_t iter_cap, uint32_t *out_ids, float *out_dist,
                  uint32_t *out_iters, int32_t *out_status, uint64_t *out_ndist,
                  uint32_t *trace, uint32_t trace_cap, int nthreads, int rerank_list);
int orc_max_threads(void);
void orc_bruteforce_knn(const void *base, const void *queries, int dtype, uint64_t n,
                        uint32_t nq, uint32_t d, uint32_t k, uint32_t *ids, double *dists,
                        int nthreads);

#endif
