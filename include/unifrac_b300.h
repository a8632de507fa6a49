/*
 * unifrac_b300 -- all-pairs UniFrac distance matrices on one NVIDIA B300.
 *
 * C ABI of the library.  The operation is the one the paper (Section II)
 * names as the core of microbiome beta-diversity analysis: for N samples of a
 * feature x sample count table placed on a rooted phylogenetic tree, compute
 * the N x N matrix of UniFrac distances, unweighted or weighted normalized,
 * optionally split into stripes of the matrix that are computed separately
 * and merged (Section II divides the matrix into stripes for that purpose).
 * With, for every non-root branch b and sample i,
 *
 *   w[b,i] = (count of sample i on the tips below b) / (total count of i)
 *   p[b,i] = 1 if w[b,i] > 0 else 0
 *
 *   unweighted          d_ij = sum_b len_b (p_bi XOR p_bj) / sum_b len_b (p_bi OR p_bj)
 *   weighted normalized d_ij = sum_b len_b |w_bi - w_bj|  / sum_b len_b (w_bi + w_bj)
 *
 * (standard definitions; a zero denominator gives 0, the root branch is
 * ignored).  Every call returns 0 on success or a negative UNIFRAC_E_* code;
 * no call aborts, throws or prints.  A context is not thread-safe: use one
 * context per host thread / stream.
 */
#ifndef UNIFRAC_B300_H
#define UNIFRAC_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct unifrac_ctx unifrac_ctx; /* opaque */

/* Which distance (Section II covers the unweighted and the weighted normalized
 * variants).
 * UNIFRAC_BOTH computes the two from one embedding pass; `out` then holds the
 * unweighted result followed by the weighted one, each of
 * unifrac_output_bytes(...) bytes. */
enum unifrac_variant {
  UNIFRAC_UNWEIGHTED = 0,
  UNIFRAC_WEIGHTED_NORMALIZED = 1,
  UNIFRAC_BOTH = 2
};

/* Arithmetic (Section II adds single-precision arithmetic to the method).
 * UNIFRAC_FP64:  double output; every sum in FP64 (max abs error vs an FP64
 *                reference <= 1e-12).
 * UNIFRAC_MIXED: float output; FP32 arithmetic with two-level FP32 sums
 *                (weighted) or an exact integer-digit BF16 tensor-core Gram
 *                with an exact integer epilogue (unweighted); one FP32
 *                quotient per distance (max abs error vs FP64 <= 2e-6). */
enum unifrac_precision { UNIFRAC_FP64 = 0, UNIFRAC_MIXED = 1 };

/* Output layouts.  Element type is double (FP64) or float (MIXED).
 * STRIPES:   rows [stripe_start, stripe_stop) of the stripe form: stripe s in
 *            [0, ceil((N-1)/2)), element k in [0, N) holds d(k, (k+s+1) mod N);
 *            out is [(stripe_stop-stripe_start) x N] row-major.  The union of
 *            all stripes covers every unordered pair (for even N the last
 *            stripe holds each of its pairs twice).
 * CONDENSED: upper triangle i<j, row-major, N(N-1)/2 elements.
 * FULL:      N x N row-major, symmetric, zero diagonal.
 * For CONDENSED and FULL the stripe range selects which pairs are computed
 * and written; other elements of the caller's buffer are left untouched, so
 * runs over disjoint stripe ranges merge into the full result. */
enum unifrac_layout {
  UNIFRAC_OUT_STRIPES = 0,
  UNIFRAC_OUT_CONDENSED = 1,
  UNIFRAC_OUT_FULL = 2
};

enum unifrac_status {
  UNIFRAC_OK = 0,
  UNIFRAC_E_INVALID_ARG = -1,    /* NULL pointer, bad enum, bad size */
  UNIFRAC_E_BAD_TREE = -2,       /* not postorder, several roots, negative/NaN length,
                                    feature on an internal node */
  UNIFRAC_E_BAD_TABLE = -3,      /* CSR malformed, sample id out of range, negative
                                    count, duplicate (feature, sample), two features
                                    on one tip, a sample total >= 2^32 */
  UNIFRAC_E_STRIPE_RANGE = -4,   /* stripe range outside [0, n_stripes] or reversed */
  UNIFRAC_E_BUFFER_TOO_SMALL = -5,
  UNIFRAC_E_CUDA = -6,           /* a CUDA runtime call failed */
  UNIFRAC_E_OOM = -7,            /* device or host allocation failed */
  UNIFRAC_E_DEVICE_TIMEOUT = -8, /* a bounded device-side wait gave up */
  UNIFRAC_E_UNSUPPORTED = -9     /* combination not supported (message explains) */
};

/*
 * unifrac_create -- validate and upload one problem: a tree, a table and the
 * studies the samples belong to.  Section II: the input is a table of
 * microbiome profiles (sparse: most features absent from most samples) and the
 * tree of evolutionary relationships between its features.
 *
 *  n_nodes        nodes of the rooted tree, >= 1.
 *  parent[n]      postorder parent array: parent[k] > k for k < n-1 and
 *                 parent[n-1] = -1 (the root is the last node).  Host memory.
 *  length[n]      FP64 branch length above each node (>= 0, finite); the
 *                 root's is ignored.  Host memory.
 *  n_features     rows of the table, >= 0.
 *  feature_node[F] tip node of each feature (a node with no children; at
 *                 most one feature per tip).  Host memory.
 *  n_samples      columns of the table, >= 0.
 *  indptr[F+1], indices[nnz], counts[nnz]
 *                 CSR table, rows = features, indices = sample ids in
 *                 [0, n_samples), counts >= 0 (0 means absent), no duplicate
 *                 (feature, sample).  int64 / int32 / int32, host memory.
 *  n_studies      >= 1.  With n_studies > 1 the samples are the concatenation
 *                 of independent studies that share the tree; distances are
 *                 formed only within a study.
 *  study_offsets  [n_studies+1] sample offsets (0 ... n_samples, non-decreasing),
 *                 or NULL when n_studies == 1.  Host memory.
 *  cuda_stream    cudaStream_t on which every later device operation of this
 *                 context is enqueued (NULL = legacy default stream).  The
 *                 current CUDA device at create time is the context's device.
 *  out            receives the new context.
 *
 * Every input is copied; the caller keeps ownership and may free its buffers
 * when the call returns.  Work: validation and per-sample totals (host
 * threads, O(n + nnz)); the tree, its levels and the table uploaded (a
 * canonical table -- rows strictly increasing, no explicit zeros -- as
 * passed); per-branch presence counts per study (which samples reach each
 * branch) from device bitsets (O(n x samples / 64) words); the branch order,
 * tensor-core length digits and per-sample weighted sums on the host.
 * Allocates, besides the uploaded inputs, the per-run presence masks of the
 * embedding: 16 bytes per (node, 128-column tile).
 * Synchronous; uses the current device.
 */
int unifrac_create(int32_t n_nodes, const int32_t *parent, const double *length,
                   int32_t n_features, const int32_t *feature_node,
                   int32_t n_samples, const int64_t *indptr,
                   const int32_t *indices, const int32_t *counts,
                   int32_t n_studies, const int32_t *study_offsets,
                   void *cuda_stream, unifrac_ctx **out);

/*
 * unifrac_run -- compute distances into `out`.
 *
 *  variant        enum unifrac_variant (UNIFRAC_BOTH: two results, one after
 *                 the other in `out`).
 *  precision      enum unifrac_precision.
 *  stripe_start, stripe_stop
 *                 stripe range [start, stop); stop = -1 means "to the last
 *                 stripe".  With n_studies > 1 only the whole range (0, -1) is
 *                 accepted and layout must be CONDENSED or FULL; the output is
 *                 each study's block in study order.
 *  layout         enum unifrac_layout.
 *  out            device pointer (enqueued on the context's stream, returns
 *                 before completion) or host pointer (staged through device
 *                 memory; the call returns after the copy has completed).
 *  out_bytes      capacity of `out`; must be >= unifrac_output_bytes(...)
 *                 (twice that for UNIFRAC_BOTH).
 *
 * Pipeline (all on the device): embedding of every branch (level-synchronous
 * postorder sums, skipping all-zero branch tiles, with a presence mask per
 * non-zero tile), packing for the chosen kernel, the pair kernel, and the
 * epilogue writing `out`.  Work buffers are allocated on first use and kept
 * in the context.
 */
int unifrac_run(unifrac_ctx *ctx, int variant, int precision,
                int32_t stripe_start, int32_t stripe_stop, int layout,
                void *out, size_t out_bytes);

/*
 * unifrac_run_streamed -- the whole matrix into HOST memory, computed in
 * chunks of `chunk_stripes` stripes so that only two chunks live on the device
 * (for sample counts whose matrix exceeds device memory).  Section II of the
 * paper: the matrix is computed as a set of stripes that are merged into the
 * final matrix afterwards.
 *
 *   layout   UNIFRAC_OUT_CONDENSED or UNIFRAC_OUT_FULL (as unifrac_run; with
 *            UNIFRAC_BOTH the unweighted matrix first, then the weighted one)
 *   host_out caller-owned host buffer of >= unifrac_output_bytes(layout)
 *            (x2 for UNIFRAC_BOTH) bytes; pinned or pageable
 *
 * The first chunk computes the embedding and packs the operands; later chunks
 * reuse them and run only the pair kernels of their stripes.  Each chunk's
 * stripes are computed into a device buffer and rewritten there as the row
 * runs of the matrix (in row i, the columns i + s and i - s of the chunk's
 * stripes s), which a copy stream moves while the next chunk computes:
 * page-locked host_out in the full layout takes them directly (2D copies of
 * the rows whose runs do not wrap past the last column; host threads place
 * the few that do); otherwise they go to a pinned buffer and host threads
 * copy each run into host_out (UNIFRAC_OPT_HOST_THREADS).  The values are
 * those of unifrac_run.
 * Single-study contexts only (UNIFRAC_E_UNSUPPORTED otherwise).  Synchronous:
 * returns when host_out is complete.  Keeps two device chunk buffers, two
 * device row-run buffers (twice a chunk each) and two pinned host buffers
 * (twice a chunk each; for page-locked full output only the wrapping runs,
 * 2 (L - 1) L elements per variant for chunks of L stripes) in the context
 * until it is destroyed.
 */
int unifrac_run_streamed(unifrac_ctx *ctx, int variant, int precision, int layout,
                         void *host_out, size_t out_bytes, int32_t chunk_stripes);

/* Frees the context and its device buffers (synchronises the device first).
 * Buffers of 64 MiB and more go to the library's cache of device blocks
 * (unifrac_set_memory_cache) rather than back to the driver.  NULL-safe. */
void unifrac_destroy(unifrac_ctx *ctx);

/* Static message for a status code (never NULL).  The most recent failure of a
 * context has a detailed message in unifrac_last_error(ctx). */
const char *unifrac_strerror(int status);
const char *unifrac_last_error(const unifrac_ctx *ctx);

/* Number of stripes ceil((n-1)/2) of study `study` (n = its sample count). */
int unifrac_n_stripes(const unifrac_ctx *ctx, int32_t study, int32_t *out);

/* Bytes `out` must hold for the given layout / precision / stripe range. */
int unifrac_output_bytes(const unifrac_ctx *ctx, int precision, int layout,
                         int32_t stripe_start, int32_t stripe_stop,
                         size_t *out);

/* Tuning options (the autotuner sets these; defaults are chosen per shape).
 * Values are validated; a bad key or value returns UNIFRAC_E_INVALID_ARG. */
enum unifrac_option {
  UNIFRAC_OPT_UNWEIGHTED_MIXED_KERNEL = 0, /* 0 auto (tensor core), 1 tensor core,
                                              2 bit-packed lookup (FP64 sums) */
  UNIFRAC_OPT_WEIGHTED_FLUSH = 1,         /* weighted mixed kernel: selected branches summed
                                              in registers before each add into the FP32
                                              running totals (shared memory), 16..4096 */
  /* 2, 3: unused */
  UNIFRAC_OPT_USE_GRAPH = 4,              /* 1 = capture a run (all its launches) in a CUDA
                                              graph and replay it while nothing changes */
  UNIFRAC_OPT_SPARSE_THRESHOLD = 5,       /* weighted mixed kernel: branches present in fewer
                                              samples than this run through the sparse phase;
                                              -1 auto (largest study / 4), 0 all dense */
  UNIFRAC_OPT_UNWEIGHTED_SPARSE_THRESHOLD = 6, /* unweighted tensor-core kernel: same split;
                                              -1 auto (largest study / 16 above 8,192
                                              samples in total, else all tensor core),
                                              0 all tensor */
  UNIFRAC_OPT_OVERLAP_VARIANTS = 7, /* UNIFRAC_BOTH: 1 (default) runs the two variants'
                                       packing and pair kernels on two streams after the
                                       shared embedding; 0 one after the other */
  UNIFRAC_OPT_SPARSE_LANE_PAIRS = 8, /* weighted sparse pair kernel: a branch whose rows in
                                        the two tiles give at most this many pairs is walked
                                        by one lane, a larger one by a whole warp; 0 .. 4096,
                                        default 128 (unweighted 64) */
  UNIFRAC_OPT_UNWEIGHTED_SPARSE_LANE_PAIRS = 9, /* the same for the unweighted sparse kernel */
  UNIFRAC_OPT_PERSISTENT = 10, /* 1 (default): each mixed-precision pair kernel runs as one
                                  persistent launch, as many CTAs as fit on the GPU at once,
                                  each pulling (study, tile pair) work items from a device
                                  counter in the order of the work list (largest studies
                                  first); 0: one CTA per work item */
  UNIFRAC_OPT_RARE_LIST = 11,  /* weighted mixed kernel: branches of the sparse part present
                                  in at most this many samples (all studies together) are
                                  taken branch by branch -- every pair of the samples
                                  holding one -- instead of by the sparse kernel's walk of
                                  each tile pair's bitmap words; 0 .. 4096, 0 off, default
                                  256; the sums are the same exact integers */
  UNIFRAC_OPT_UNWEIGHTED_RARE_LIST = 12, /* the same for the unweighted sparse part */
  UNIFRAC_OPT_COPY_RANGES = 13, /* output in pinned host memory, one study's whole matrix
                                  (layout FULL or CONDENSED, range (0, -1)): the weighted
                                  variant's dense pair kernel runs as this many launches
                                  over consecutive row blocks of the work list, and the
                                  part of the matrix each one completes is copied to host
                                  memory while the next computes; 1 .. 64, default 32
                                  (at most one per block row of 12 tiles);
                                  1 copies the whole matrix after the last kernel.  The
                                  results are the same for every value. */
  UNIFRAC_OPT_HOST_THREADS = 14 /* host threads of unifrac_run_streamed's stripe merge:
                                   0 (default) = the CPUs this process may run on
                                   (its affinity mask and cgroup CPU quota), at
                                   most 32; 1 .. 256 = that many.  The results are
                                   the same for every value. */
};
int unifrac_set_option(unifrac_ctx *ctx, int option, int64_t value);
int unifrac_get_option(const unifrac_ctx *ctx, int option, int64_t *value);

/*
 * unifrac_autotune -- pick the kernel settings of one (variant, precision)
 * for this context by timing candidates on the device, and keep the fastest
 * as the context's options.  One option at a time, the others held at their
 * current values: the dense / sparse split (UNIFRAC_OPT_SPARSE_THRESHOLD at
 * 1/16 .. 3/4 of the largest study, weighted; UNIFRAC_OPT_UNWEIGHTED_SPARSE_
 * THRESHOLD all tensor core or 1/32 .. 1/4, unweighted; then 3/4 and 3/2 of
 * the best), the single-lane incidence bound of the sparse kernels
 * (UNIFRAC_OPT_SPARSE_LANE_PAIRS / UNIFRAC_OPT_UNWEIGHTED_SPARSE_LANE_PAIRS
 * 32, 64, 128, 256, when the split has a sparse part), the per-branch list
 * bound (UNIFRAC_OPT_RARE_LIST / UNIFRAC_OPT_UNWEIGHTED_RARE_LIST 0, 64, 256,
 * 1024, likewise; both then 3/4 and 3/2 of the best) and, weighted, the
 * register flush length (UNIFRAC_OPT_WEIGHTED_FLUSH 128, 256, 512).  Each candidate runs `repeats` times (>= 1, after one
 * warm-up run) into `out`, a DEVICE buffer of at least
 * unifrac_output_bytes(ctx, precision, UNIFRAC_OUT_CONDENSED, 0, -1) bytes
 * whose contents are overwritten; the time compared is embedding + packing +
 * pair kernels (CUDA events).  A candidate whose work buffers do not fit in
 * device memory is skipped; the variant's work buffers are released at the
 * end (the next run allocates what the chosen settings need).  Synchronises
 * the context's stream.  FP64 has nothing to tune (returns 0).
 */
int unifrac_autotune(unifrac_ctx *ctx, int variant, int precision, void *out,
                     size_t out_bytes, int repeats);

/*
 * unifrac_pcoa -- principal coordinates analysis of a distance matrix, the
 * ordination the UniFrac matrix feeds (the paper, Sections I and II).
 * Classical PCoA: A = -1/2 (D o D), B = J A J with J = I - 11^T / n; returns
 * the k largest eigenvalues of B (descending) and the coordinates
 * U_k sqrt(max(lambda_k, 0)).
 *
 *   dist       DEVICE pointer, the full n x n matrix (unifrac_run with
 *              UNIFRAC_OUT_FULL), float (UNIFRAC_MIXED) or double (UNIFRAC_FP64),
 *              symmetric, 16-byte aligned; not modified
 *   k          1 <= k <= min(n, UNIFRAC_PCOA_MAX_K) components
 *   iters      subspace iterations (>= 0; 12 is ample for the leading
 *              components of UniFrac matrices)
 *   seed       seed of the random start (results are reproducible)
 *   eigvals    HOST double[k]
 *   coords     HOST double[n * k], row-major (sample i: coords[i * k .. + k))
 *   cuda_stream  stream for the device work (NULL = legacy default stream)
 *
 * Method: subspace iteration with m = min(n, 2k + 16) columns, all products
 * on the device in the library's own kernels.  A is never stored: each
 * product A Q streams D once (its column panels, A being symmetric) and forms
 * -1/2 d^2 on the fly, FP32 sums within chunks of rows and FP64 across
 * chunks; the centring terms, the CholeskyQR2 orthonormalisation (Gram
 * matrices and products with R^-1) and the Ritz products in FP64.  Only m x m
 * work (Cholesky factors and their inverses, the Jacobi eigensolver of the
 * Ritz matrix) runs on the host.  Allocates O(n m) device memory while it
 * runs (about 4 n m (c + 2) + 40 n m bytes, c <= 16 chunks; UNIFRAC_E_OOM if
 * that fails).  Synchronous.  Errors: UNIFRAC_E_INVALID_ARG (sizes, k,
 * precision, NULL or misaligned pointers), UNIFRAC_E_OOM, UNIFRAC_E_CUDA.
 * No context needed.
 */
#define UNIFRAC_PCOA_MAX_K 384
int unifrac_pcoa(const void *dist, int precision, int32_t n, int32_t k, int32_t iters,
                 uint64_t seed, double *eigvals, double *coords, void *cuda_stream);

/*
 * unifrac_mantel -- the Mantel test between two distance matrices (the paper,
 * Section III): the correlation of the pair distances of x and y, Pearson or
 * Spearman (Pearson on average ranks, ties sharing the mean of their
 * positions), and its two-sided permutation p-value.  Over the pairs i < j:
 *   r = sum (x - mean x)(y - mean y) / sqrt(sum (x - mean x)^2 sum (y - mean y)^2);
 * permutation pi gives r_pi with y(pi(i), pi(j)) in place of y(i, j);
 *   p = (1 + #{m : |r_m| >= |r|}) / (n_perms + 1).
 *
 *   x, y       DEVICE pointers, full n x n matrices (unifrac_run with
 *              UNIFRAC_OUT_FULL layout), float (UNIFRAC_MIXED) or double
 *              (UNIFRAC_FP64), 16-byte aligned, not modified; only the strict
 *              upper triangle of x is read, and y must be symmetric (whole
 *              rows of y are read).  Values finite.
 *   n          3 <= n <= UNIFRAC_MANTEL_MAX_SAMPLES
 *   perms      HOST int32 [n_perms x n], row m a permutation of 0 .. n-1
 *              (validated; the caller draws them, so results are reproducible
 *              and comparable across implementations); NULL if n_perms == 0
 *   method     enum unifrac_mantel_method
 *   r          HOST double: the statistic (NaN if either matrix is constant)
 *   perm_stats HOST double[n_perms] (may be NULL): r_m of each permutation
 *   p_value    HOST double: the p-value (NaN if n_perms == 0 or r is NaN)
 *   cuda_stream  stream for the device work (NULL = legacy default stream)
 *
 * Sums are FP64 (UNIFRAC_MIXED: FP32 products, summed in FP32 per thread
 * over at most ceil(n / 128) pairs and then over the 32 lanes of a warp,
 * FP64 beyond).  Each row of y is staged in shared
 * memory once per batch of 16 permutations while (n + 8) sizeof(T) <= 220 KB,
 * else read from global memory; the environment variable
 * UNIFRAC_MANTEL_SMEM_BYTES lowers that 220 KB budget.  Allocates device memory while it runs:
 * about 12 n_perms n bytes, plus for Spearman two rank matrices of the input
 * type and about 16 n^2 bytes of sort buffers.  Synchronous.  Errors:
 * UNIFRAC_E_INVALID_ARG (bad size, enum, pointer, alignment or permutation),
 * UNIFRAC_E_OOM, UNIFRAC_E_CUDA.  No context needed.
 */
enum unifrac_mantel_method { UNIFRAC_MANTEL_PEARSON = 0, UNIFRAC_MANTEL_SPEARMAN = 1 };
#define UNIFRAC_MANTEL_MAX_SAMPLES 92682 /* n (n - 1) / 2 < 2^32 */
int unifrac_mantel(const void *x, const void *y, int precision, int32_t n, const int32_t *perms,
                   int32_t n_perms, int method, double *r, double *perm_stats, double *p_value,
                   void *cuda_stream);

/*
 * unifrac_check_bounded_wait -- runs the library's bounded device-side wait
 * (the one every mbarrier wait of the tensor-core kernel uses, there with a
 * 1 s limit) on an mbarrier that nothing arrives at, with a limit of
 * `limit_us` microseconds (1 .. 1,000,000), so that the wait runs out; one
 * thread of one CTA, no copies or tensor memory involved.  *status receives
 * the code the kernel recorded: UNIFRAC_E_DEVICE_TIMEOUT when the bound works.
 * The call returns UNIFRAC_OK when the kernel ran to its end (the device stays
 * usable), UNIFRAC_E_INVALID_ARG, UNIFRAC_E_OOM or UNIFRAC_E_CUDA otherwise.
 * Synchronous.  No context needed.
 */
int unifrac_check_bounded_wait(uint32_t limit_us, int32_t *status, void *cuda_stream);

/*
 * unifrac_measure_peak -- the measured issue rate of one arithmetic pipe of
 * the current device, the ceiling against which the pair kernels' work is
 * reported (the paper names no hardware model; the weighted kernel is bound
 * by FP32 operations, the plain FP64 kernels by FP64 operations, Section II).
 * A full-occupancy grid (a multiple of the SM count) runs chains of fused
 * multiply-adds on eight independent accumulators per thread for about 20 ms;
 * *ops_per_s receives FMA instructions per second (one FMA = one operation),
 * best of three timed launches (CUDA events on `cuda_stream`).  Allocates a
 * few KB of device memory while it runs.  Synchronous.  Errors:
 * UNIFRAC_E_INVALID_ARG (unknown pipe, NULL output), UNIFRAC_E_OOM,
 * UNIFRAC_E_CUDA.  No context needed.
 */
enum unifrac_peak_pipe { UNIFRAC_PEAK_FP32_FMA = 0, UNIFRAC_PEAK_FP64_FMA = 1 };
int unifrac_measure_peak(int pipe, double *ops_per_s, void *cuda_stream);

/* Statistics of the context / its last run. */
enum unifrac_stat {
  UNIFRAC_STAT_KERNEL_LAUNCHES = 0, /* kernels launched by the last run */
  UNIFRAC_STAT_PAIR_BRANCH = 1,     /* sum over studies of C(n_s,2) * B_s */
  UNIFRAC_STAT_USEFUL = 2,          /* sum over studies and branches of C(n_b,2) */
  UNIFRAC_STAT_BRANCHES_KEPT = 3,   /* branches with a sample below and length > 0 */
  UNIFRAC_STAT_LEVELS = 4,          /* levels of the postorder embedding */
  UNIFRAC_STAT_TILE_PAIRS = 5,      /* 128 x 128 pair tiles of the last run */
  UNIFRAC_STAT_SELECTED_UPDATES = 6,/* pair-branch updates the last pair kernel did
                                       (after skipping all-zero branch tiles) */
  UNIFRAC_STAT_PAIR_KERNEL_MS = 7,  /* device time of the last pair kernel (ms); after an
                                       overlapped UNIFRAC_BOTH run: everything after the
                                       embedding */
  UNIFRAC_STAT_EMBED_MS = 8,        /* device time of the last embedding + pack (ms); after
                                       an overlapped UNIFRAC_BOTH run: the embedding */
  UNIFRAC_STAT_DEVICE_BYTES = 9,    /* device memory held by the context */
  UNIFRAC_STAT_PAIR_MS_UNWEIGHTED = 10, /* device time of the pair kernel of the last */
  UNIFRAC_STAT_PAIR_MS_WEIGHTED = 11,   /*   unweighted / weighted run (ms)          */
  UNIFRAC_STAT_DEVICE_ERROR = 12,   /* 0, or the UNIFRAC_E_* code a kernel of the last run
                                       raised (synchronises the context's stream) */
  UNIFRAC_STAT_SELECTED_UNWEIGHTED = 13, /* UNIFRAC_STAT_SELECTED_UPDATES of the last */
  UNIFRAC_STAT_SELECTED_WEIGHTED = 14,   /*   unweighted / weighted run (dense part)  */
  UNIFRAC_STAT_SPARSE_MS_UNWEIGHTED = 15, /* device time of the sparse pair kernel of */
  UNIFRAC_STAT_SPARSE_MS_WEIGHTED = 16,   /*   the last run of each variant (ms), the
                                             per-branch lists excluded              */
  UNIFRAC_STAT_SPARSE_UPDATES_UNWEIGHTED = 17, /* pair updates it did (co-present      */
  UNIFRAC_STAT_SPARSE_UPDATES_WEIGHTED = 18,   /*   (pair, branch) of the sparse part) */
  UNIFRAC_STAT_CREATE_HOST_MS = 19,   /* unifrac_create: validation and host preparation (ms) */
  UNIFRAC_STAT_CREATE_DEVICE_MS = 20, /* unifrac_create: device set-up and uploads (ms) */
  UNIFRAC_STAT_MAX_REACH = 21,        /* most non-root branches one sample reaches: exact
                                         when the tree has >= 65,793 of them, else that
                                         count (an upper bound; the tensor-core path
                                         needs < 65,793) */
  UNIFRAC_STAT_LIST_MS_UNWEIGHTED = 22, /* device time of the per-branch list pairs (the     */
  UNIFRAC_STAT_LIST_MS_WEIGHTED = 23,   /*   very rarely present branches) of the last run  */
  UNIFRAC_STAT_LIST_UPDATES_UNWEIGHTED = 24, /* co-present (pair, branch) updates they made */
  UNIFRAC_STAT_LIST_UPDATES_WEIGHTED = 25
};
int unifrac_get_stat(const unifrac_ctx *ctx, int stat, double *value);

/*
 * unifrac_dense_noalloc -- the full N x N FP64 matrix of a small problem,
 * computed without allocating anything.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc (a real-time or
 * embedded pipeline that reserves all device memory at start-up, a plug-in
 * running inside an application that owns the memory pool, code that must not
 * risk the device-wide synchronisation an allocation can cause).
 * unifrac_create allocates, so those callers use this call instead.
 *
 *  variant      enum unifrac_variant.
 *  n_nodes      nodes of the tree; parent[n_nodes] (int32) and length[n_nodes]
 *               (FP64) are DEVICE arrays in the postorder form of
 *               unifrac_create (parent[k] > k, root last; root length ignored).
 *  n_samples    samples, 0 .. UNIFRAC_NOALLOC_MAX_SAMPLES.
 *  tip_counts   DEVICE array [n_nodes x n_samples] (node-major, u32): the count
 *               of each sample on each tip; rows of internal nodes must be 0.
 *               Each sample total must stay below 2^32.
 *  out          DEVICE array [n_samples x n_samples] FP64, row-major; receives
 *               the symmetric matrix with a zero diagonal.
 *  cuda_stream  stream the two kernels are enqueued on (asynchronous).
 *
 * Work space: one fixed device array of UNIFRAC_NOALLOC_MAX_CELLS 32-bit
 * counts inside the library (4 MB, held by every GPU that loads the library
 * until the process exits).  n_nodes * n_samples above that, or n_samples above
 * UNIFRAC_NOALLOC_MAX_SAMPLES, returns UNIFRAC_E_UNSUPPORTED.  Every call made
 * outside stream capture looks up that array's device address
 * (cudaGetSymbolAddress) with the current device; a call on a capturing stream
 * uses the address of the last earlier call on that device, and is refused
 * with UNIFRAC_E_UNSUPPORTED when there was none: make one call on each device
 * before any stream capture.  All calls share the array: calls that overlap
 * on the GPU race and corrupt each other's results -- serialise them (one
 * stream, or events).  Nothing carries over between calls.  Allocates no
 * device or host memory.  Returns UNIFRAC_E_CUDA when a launch fails (that
 * launch's own status; an error left pending by earlier unrelated work is not
 * reported or cleared).
 */
#define UNIFRAC_NOALLOC_MAX_CELLS (1u << 20)
#define UNIFRAC_NOALLOC_MAX_SAMPLES 4096
int unifrac_dense_noalloc(int variant, int32_t n_nodes, const int32_t *parent,
                          const double *length, int32_t n_samples,
                          const uint32_t *tip_counts, double *out,
                          void *cuda_stream);

/*
 * The library's cache of device blocks.  A context's work buffers at large
 * sizes run to tens of GB (about 65 GB at 50,000 samples on a 400,000-node
 * tree, with the full output staged for host memory); giving
 * them back to the driver and taking them again costs tens of milliseconds
 * per context.  Buffers of 64 MiB and more that a context frees (on
 * unifrac_destroy, or when a run needs a larger one) are kept, per device,
 * and a later context or run takes one of about the same size (at most 1/8
 * larger) back.  A taken block holds whatever its last user left; the
 * library never reads device memory it has not written.  When the driver
 * cannot satisfy an allocation, the library releases the device's cache and
 * tries once more.  Memory of other users of the device (for instance a
 * framework's own allocator) is not covered by that retry: release the cache
 * before large allocations of your own.
 *
 * unifrac_set_memory_cache -- most bytes the cache may hold on `device`
 *   (-1 as `device`: the current device): max_bytes >= 0 (0 turns caching
 *   off; blocks over the new cap are freed at once) or -1 for the default,
 *   half the device's memory.  UNIFRAC_E_INVALID_ARG for max_bytes < -1 or a
 *   device that cannot be selected.
 * unifrac_release_cached_memory -- frees every cached block of `device`
 *   (-1: of every device).  Contexts that exist keep their own buffers.
 * unifrac_cached_memory -- bytes the cache holds on `device` (-1: current)
 *   into *bytes.
 * All three are thread-safe and leave the caller's current device as it was.
 */
int unifrac_set_memory_cache(int device, int64_t max_bytes);
int unifrac_release_cached_memory(int device);
int unifrac_cached_memory(int device, int64_t *bytes);

#ifdef __cplusplus
}
#endif

#endif /* UNIFRAC_B300_H */
