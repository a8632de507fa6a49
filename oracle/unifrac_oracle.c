/*
 * FP64 CPU oracle for the all-pairs UniFrac distance matrix.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg load it; the product library never
 * links, calls or falls back to it, and it shares no code with the CUDA path.
 *
 * What it computes (paper, Section II): UniFrac, a phylogenetic measure of
 * beta diversity between every pair of samples of a feature x sample table,
 * giving an N x N distance matrix, in the unweighted and the weighted
 * normalized variants.  The paper states the measure in words only; the
 * formulas are the standard published definitions, written out here:
 *
 *   w[b,i] = (sum of counts of sample i on the tips below branch b) / C_i,
 *            C_i = total count of sample i              (relative abundance)
 *   p[b,i] = 1 if any tip below branch b is present in sample i, else 0
 *
 *   unweighted (Lozupone & Knight 2005):
 *       d_ij = sum_b len_b * (p_bi XOR p_bj) / sum_b len_b * (p_bi OR p_bj)
 *   weighted normalized (Lozupone et al. 2007):
 *       d_ij = sum_b len_b * |w_bi - w_bj| / sum_b len_b * (w_bi + w_bj)
 *
 * sums run over every non-root branch b of the tree.  Readings where the
 * paper is silent: the root branch is ignored (length treated as 0); a zero
 * denominator (both samples empty, only zero-length branches, i == j) gives
 * d = 0; explicit zero counts are absent features; a duplicate (feature,
 * sample) entry or two features on one tip make the table invalid (rejected,
 * not summed).
 *
 * Steps, in the order of the definition:
 *   1. per sample, place each feature's count on its tip node;
 *   2. walk the nodes in postorder and add every node's total into its parent,
 *      so each node holds the count below its branch (FP64, exact for
 *      integer totals below 2^53), then divide by C_i and test for > 0;
 *   3. for every requested pair, loop over the non-root branches and form the
 *      two sums above in FP64, then divide.
 *
 * parity pinned: the tests check this file against brute-force ancestor
 * walks, closed forms on star trees (Jaccard, Bray-Curtis), Faith's PD, the
 * tip-depth identity and metric invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_E_ARG (-1)
#define ORACLE_E_TREE (-2)
#define ORACLE_E_TABLE (-3)
#define ORACLE_E_OOM (-4)

typedef struct {
  int32_t n_nodes;
  const int32_t *parent;
  const double *length;
  int32_t n_samples;
  /* per-sample (transposed) view of the table: features and counts */
  int64_t *s_ptr;   /* n_samples + 1 */
  int32_t *s_node;  /* tip node of each entry */
  double *s_count;  /* count of each entry */
  double *total;    /* C_i */
} oracle_input;

static void oracle_free(oracle_input *in) {
  free(in->s_ptr);
  free(in->s_node);
  free(in->s_count);
  free(in->total);
}

/* Validate the tree and table and build the per-sample view. */
static int oracle_prepare(int32_t n_nodes, const int32_t *parent,
                          const double *length, int32_t n_features,
                          const int32_t *feature_node, int32_t n_samples,
                          const int64_t *indptr, const int32_t *indices,
                          const int32_t *counts, oracle_input *in) {
  memset(in, 0, sizeof(*in));
  if (n_nodes < 1 || n_features < 0 || n_samples < 0 || !parent || !length)
    return ORACLE_E_ARG;
  for (int32_t k = 0; k < n_nodes - 1; ++k)
    if (parent[k] <= k || parent[k] >= n_nodes) return ORACLE_E_TREE;
  if (parent[n_nodes - 1] != -1) return ORACLE_E_TREE;
  char *is_internal = (char *)calloc((size_t)n_nodes, 1);
  if (!is_internal) return ORACLE_E_OOM;
  for (int32_t k = 0; k < n_nodes - 1; ++k) is_internal[parent[k]] = 1;
  for (int32_t f = 0; f < n_features; ++f) {
    int32_t t = feature_node[f];
    if (t < 0 || t >= n_nodes || is_internal[t]) {
      free(is_internal);
      return ORACLE_E_TREE;
    }
  }
  free(is_internal);
  if (indptr[0] != 0) return ORACLE_E_TABLE;
  for (int32_t f = 0; f < n_features; ++f)
    if (indptr[f + 1] < indptr[f]) return ORACLE_E_TABLE;
  int64_t nnz = indptr[n_features];
  /* A (feature, sample) cell appears at most once, and a tip carries at most
   * one feature (a tip is one taxon): a second entry for the same cell, or a
   * second feature on the same tip, is a malformed table, not a sum. */
  {
    int32_t *last_feature = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n_samples + 1));
    char *tip_used = (char *)calloc((size_t)n_nodes, 1);
    if (!last_feature || !tip_used) {
      free(last_feature);
      free(tip_used);
      return ORACLE_E_OOM;
    }
    for (int32_t s = 0; s < n_samples; ++s) last_feature[s] = -1;
    int bad = 0;
    for (int32_t f = 0; f < n_features && !bad; ++f) {
      if (tip_used[feature_node[f]]) bad = 1;
      tip_used[feature_node[f]] = 1;
      for (int64_t e = indptr[f]; e < indptr[f + 1] && !bad; ++e) {
        int32_t s = indices[e];
        if (s < 0 || s >= n_samples || last_feature[s] == f) bad = 1;
        else last_feature[s] = f;
      }
    }
    free(last_feature);
    free(tip_used);
    if (bad) return ORACLE_E_TABLE;
  }
  in->n_nodes = n_nodes;
  in->parent = parent;
  in->length = length;
  in->n_samples = n_samples;
  in->s_ptr = (int64_t *)calloc((size_t)n_samples + 1, sizeof(int64_t));
  in->s_node = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  in->s_count = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  in->total = (double *)calloc((size_t)n_samples + 1, sizeof(double));
  if (!in->s_ptr || !in->s_node || !in->s_count || !in->total) {
    oracle_free(in);
    return ORACLE_E_OOM;
  }
  for (int64_t e = 0; e < nnz; ++e) {
    int32_t s = indices[e];
    if (s < 0 || s >= n_samples || counts[e] < 0) {
      oracle_free(in);
      return ORACLE_E_TABLE;
    }
    in->s_ptr[s + 1]++;
  }
  for (int32_t s = 0; s < n_samples; ++s) in->s_ptr[s + 1] += in->s_ptr[s];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n_samples + 1));
  if (!fill) {
    oracle_free(in);
    return ORACLE_E_OOM;
  }
  memcpy(fill, in->s_ptr, sizeof(int64_t) * ((size_t)n_samples + 1));
  for (int32_t f = 0; f < n_features; ++f) {
    for (int64_t e = indptr[f]; e < indptr[f + 1]; ++e) {
      int32_t s = indices[e];
      int64_t at = fill[s]++;
      in->s_node[at] = feature_node[f];
      in->s_count[at] = (double)counts[e];
      in->total[s] += (double)counts[e];
    }
  }
  free(fill);
  return ORACLE_OK;
}

/* Steps 1-2 for one sample: w[k] (relative abundance below branch k) and
 * p[k] (presence below branch k) for every node k.  acc is scratch [n]. */
static void oracle_embed_one(const oracle_input *in, int32_t s, double *acc,
                             double *w, unsigned char *p) {
  const int32_t n = in->n_nodes;
  for (int32_t k = 0; k < n; ++k) acc[k] = 0.0;
  for (int64_t e = in->s_ptr[s]; e < in->s_ptr[s + 1]; ++e)
    acc[in->s_node[e]] += in->s_count[e];
  for (int32_t k = 0; k < n - 1; ++k) acc[in->parent[k]] += acc[k];
  const double C = in->total[s];
  for (int32_t k = 0; k < n; ++k) {
    w[k] = C > 0.0 ? acc[k] / C : 0.0;
    p[k] = acc[k] > 0.0 ? 1 : 0;
  }
}

/* Step 3 for one pair, from the two samples' embeddings. */
static double oracle_distance(const oracle_input *in, int variant,
                              const double *wi, const unsigned char *pi,
                              const double *wj, const unsigned char *pj) {
  double num = 0.0, den = 0.0;
  const int32_t n = in->n_nodes;
  for (int32_t b = 0; b < n - 1; ++b) { /* every non-root branch */
    const double len = in->length[b];
    if (variant == 0) {
      num += len * (double)(pi[b] ^ pj[b]);
      den += len * (double)(pi[b] | pj[b]);
    } else {
      num += len * fabs(wi[b] - wj[b]);
      den += len * (wi[b] + wj[b]);
    }
  }
  return den > 0.0 ? num / den : 0.0;
}

/* Embedding of one sample: w_out[n_nodes], p_out[n_nodes]. */
int oracle_embedding(int32_t n_nodes, const int32_t *parent,
                     const double *length, int32_t n_features,
                     const int32_t *feature_node, int32_t n_samples,
                     const int64_t *indptr, const int32_t *indices,
                     const int32_t *counts, int32_t sample, double *w_out,
                     unsigned char *p_out) {
  oracle_input in;
  int rc = oracle_prepare(n_nodes, parent, length, n_features, feature_node,
                          n_samples, indptr, indices, counts, &in);
  if (rc) return rc;
  if (sample < 0 || sample >= n_samples) {
    oracle_free(&in);
    return ORACLE_E_ARG;
  }
  double *acc = (double *)malloc(sizeof(double) * (size_t)n_nodes);
  if (!acc) {
    oracle_free(&in);
    return ORACLE_E_OOM;
  }
  oracle_embed_one(&in, sample, acc, w_out, p_out);
  free(acc);
  oracle_free(&in);
  return ORACLE_OK;
}

/* Distances of the given rows against every sample:
 * out[r * n_samples + j] = d(rows[r], j), variant 0 = unweighted,
 * 1 = weighted normalized.  Parallel over j when built with OpenMP;
 * *threads_used receives the thread count (may be NULL). */
int oracle_unifrac_rows(int32_t n_nodes, const int32_t *parent,
                        const double *length, int32_t n_features,
                        const int32_t *feature_node, int32_t n_samples,
                        const int64_t *indptr, const int32_t *indices,
                        const int32_t *counts, int variant, int32_t n_rows,
                        const int32_t *rows, double *out, int n_threads,
                        int32_t *threads_used) {
  if (variant != 0 && variant != 1) return ORACLE_E_ARG;
  oracle_input in;
  int rc = oracle_prepare(n_nodes, parent, length, n_features, feature_node,
                          n_samples, indptr, indices, counts, &in);
  if (rc) return rc;
  for (int32_t r = 0; r < n_rows; ++r)
    if (rows[r] < 0 || rows[r] >= n_samples) {
      oracle_free(&in);
      return ORACLE_E_ARG;
    }
  const size_t n = (size_t)n_nodes;
  double *rw = (double *)malloc(sizeof(double) * n * (size_t)(n_rows > 0 ? n_rows : 1));
  unsigned char *rp = (unsigned char *)malloc(n * (size_t)(n_rows > 0 ? n_rows : 1));
  double *acc0 = (double *)malloc(sizeof(double) * n);
  if (!rw || !rp || !acc0) {
    free(rw);
    free(rp);
    free(acc0);
    oracle_free(&in);
    return ORACLE_E_OOM;
  }
  for (int32_t r = 0; r < n_rows; ++r)
    oracle_embed_one(&in, rows[r], acc0, rw + n * (size_t)r, rp + n * (size_t)r);
  free(acc0);
  int used = 1;
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#else
  n_threads = 1;
#endif
  int failed = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
  {
    double *acc = (double *)malloc(sizeof(double) * n);
    double *wj = (double *)malloc(sizeof(double) * n);
    unsigned char *pj = (unsigned char *)malloc(n);
#ifdef _OPENMP
#pragma omp single
    used = omp_get_num_threads();
#endif
    if (!acc || !wj || !pj) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      failed = 1;
    } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
      for (int32_t j = 0; j < n_samples; ++j) {
        oracle_embed_one(&in, j, acc, wj, pj);
        for (int32_t r = 0; r < n_rows; ++r)
          out[(size_t)r * (size_t)n_samples + (size_t)j] =
              oracle_distance(&in, variant, rw + n * (size_t)r,
                              rp + n * (size_t)r, wj, pj);
      }
    }
    free(acc);
    free(wj);
    free(pj);
  }
  free(rw);
  free(rp);
  oracle_free(&in);
  if (threads_used) *threads_used = used;
  return failed ? ORACLE_E_OOM : ORACLE_OK;
}

/* Distances of an explicit list of pairs: out[k] = d(pi[k], pj[k]). */
int oracle_unifrac_pairs(int32_t n_nodes, const int32_t *parent,
                         const double *length, int32_t n_features,
                         const int32_t *feature_node, int32_t n_samples,
                         const int64_t *indptr, const int32_t *indices,
                         const int32_t *counts, int variant, int64_t n_pairs,
                         const int32_t *pi, const int32_t *pj, double *out) {
  if (variant != 0 && variant != 1) return ORACLE_E_ARG;
  oracle_input in;
  int rc = oracle_prepare(n_nodes, parent, length, n_features, feature_node,
                          n_samples, indptr, indices, counts, &in);
  if (rc) return rc;
  const size_t n = (size_t)n_nodes;
  double *acc = (double *)malloc(sizeof(double) * n);
  double *wa = (double *)malloc(sizeof(double) * n);
  double *wb = (double *)malloc(sizeof(double) * n);
  unsigned char *pa = (unsigned char *)malloc(n);
  unsigned char *pb = (unsigned char *)malloc(n);
  int status = ORACLE_OK;
  if (!acc || !wa || !wb || !pa || !pb) status = ORACLE_E_OOM;
  for (int64_t k = 0; status == ORACLE_OK && k < n_pairs; ++k) {
    if (pi[k] < 0 || pi[k] >= n_samples || pj[k] < 0 || pj[k] >= n_samples) {
      status = ORACLE_E_ARG;
      break;
    }
    oracle_embed_one(&in, pi[k], acc, wa, pa);
    oracle_embed_one(&in, pj[k], acc, wb, pb);
    out[k] = oracle_distance(&in, variant, wa, pa, wb, pb);
  }
  free(acc);
  free(wa);
  free(wb);
  free(pa);
  free(pb);
  oracle_free(&in);
  return status;
}
