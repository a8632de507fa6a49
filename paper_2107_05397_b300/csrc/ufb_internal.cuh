// Internal declarations of the unifrac_b300 library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "unifrac_b300.h"

namespace ufb {

// Samples per pair tile and per column tile of the embedding.  Every study's
// columns start on a multiple of TILE so that no tile straddles two studies.
constexpr int TILE = 128;
// Branches per 32-bit word of the (tile, branch) nonzero bitmaps.
constexpr int WORD = 32;
// Positions per window of the weighted kernel's sparse phase (32 bitmap words).
constexpr int kRareWin = 1024;

// Counts of the embedding are held only for the (node, column tile) pairs
// that have a non-zero count: slot[node * n_tiles + t] is the tile's row of
// TILE u32 counts in the compact array, kNoSlot where the node has no count in
// the tile (fixed at create from the table's presence; the embedding never
// writes or reads there).  count_tile returns the tile's counts, or nullptr
// for kNoSlot: every caller skips the tile then (or reads zeros), so a tile
// without a slot is never addressed.
constexpr uint32_t kNoSlot = 0xffffffffu;
__device__ __forceinline__ uint32_t *count_tile(uint32_t *cnt, const uint32_t *slot,
                                                int64_t node, int64_t t, int32_t n_tiles) {
  const uint32_t s = slot[node * n_tiles + t];
  return s == kNoSlot ? nullptr : cnt + (int64_t)s * TILE;
}
__device__ __forceinline__ const uint32_t *count_tile(const uint32_t *cnt, const uint32_t *slot,
                                                      int64_t node, int64_t t, int32_t n_tiles) {
  const uint32_t s = slot[node * n_tiles + t];
  return s == kNoSlot ? nullptr : cnt + (int64_t)s * TILE;
}

// One 128 x 128 block of sample pairs, I-tile <= J-tile, both in one study.
struct WorkItem {
  int32_t tile_i;  // global column tile of the rows
  int32_t tile_j;  // global column tile of the columns
  int32_t study;
  int32_t pad;
};

// Where a study's samples live in the embedding and its block in `out`.
struct StudyDev {
  int64_t out_off;  // element offset of the study's output block
  int32_t n;        // samples
  int32_t col0;     // first embedding column (multiple of TILE)
};

// Epilogue parameters shared by every pair kernel.
struct OutSpec {
  void *out;
  const StudyDev *studies;
  int32_t layout;  // enum unifrac_layout
  int32_t s0, s1;  // stripe range [s0, s1)
  int32_t is_f64;
};

// Device buffers that only grow; released by the context.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

// Work buffers of one variant's packing and pair kernels.  Each variant slot
// (0 unweighted, 1 weighted normalized) has its own set, so the two variants
// of one call can run concurrently on two streams.
struct VarBufs {
  DevBuf vals, vals2, bits, persample, partial, rc, bsize, boff, blocks, cpre, spart, rbits;
  DevBuf vlist, voff;  // very rarely present positions: lists, offsets
  DevBuf trec, tidx;   // their tile-major records; per-tile offsets, counts, cursors
  int32_t voff_pv = -1;  // first listed position the offsets in voff were made for
  unsigned long long list_entries = 0;  // entries of the lists of the last plan
};

// Device counters: slot s (variant) owns the work queues 4 s + {0: dense /
// tensor-core / lookup pair kernel, 1: sparse pair kernel} (read as 32-bit
// counters) and kCounterBase + 4 s + {0: selected units, 1: error code,
// 2: sparse updates}; all are cleared at the start of the slot's run.
constexpr int kCounterBase = 8;
constexpr int kCounters = kCounterBase + 8;

}  // namespace ufb

struct unifrac_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  std::string last_error;

  // ---- problem shape
  int32_t n_nodes = 0, n_features = 0, n_samples = 0, n_studies = 1;
  int64_t nnz = 0;
  std::vector<int32_t> study_off;   // [S+1] sample offsets
  std::vector<int32_t> study_col0;  // [S] first embedding column
  int32_t n_cols = 0;               // embedding columns (multiple of TILE)
  int32_t n_tiles = 0;              // n_cols / TILE
  std::vector<int32_t> col_of_sample;  // [N]

  // ---- tree levels (host) and device copies
  int32_t n_levels = 0;               // levels above the tips (root excluded)
  std::vector<int32_t> level_ptr;     // [n_levels+1] into d_level_nodes
  int32_t *d_level_nodes = nullptr;   // internal non-root nodes grouped by level
  int32_t *d_level_ptr = nullptr;     // device copy of level_ptr
  int32_t *d_child_ptr = nullptr;     // [n_nodes+1]
  int32_t *d_child_idx = nullptr;     // [n_nodes-1]

  // ---- table on the device (rows = features that sit on a tip, non-empty)
  int32_t n_frows = 0;
  int32_t *d_frow_tip = nullptr;      // [n_frows] tip node of the row
  int64_t *d_frow_ptr = nullptr;      // [n_frows+1]
  // tip rows cut into chunks of at most tip_chunk entries, one warp each
  // (a common feature has an entry in nearly every sample)
  int64_t n_tchunks = 0, tip_chunk = 256;
  int32_t *d_tchunk_row = nullptr;    // [n_tchunks] row of the chunk
  int64_t *d_tchunk_lo = nullptr;     // [n_tchunks] its first entry
  // [n_nodes][n_tiles] presence masks written by the embedding beside the
  // counts, valid where the tile is flagged: word w has bit l set when
  // column 4 l + w of the tile holds a non-zero count
  uint4 *d_pmask = nullptr;
  // [n_nodes][n_tiles] slot of each (node, tile) in the compact counts array
  // (kNoSlot: no count there), and the number of slots; set at create
  uint32_t *d_slot = nullptr;
  int64_t n_slots = 0;
  int32_t *d_fent_col = nullptr;      // [nnz'] embedding column (sorted per row)
  uint32_t *d_fent_cnt = nullptr;     // [nnz'] count (> 0)
  double *d_inv_total = nullptr;      // [n_cols] 1 / C_i (0 for empty or padding)
  double *d_S = nullptr;              // [n_cols] weighted sums S_col (FP64), set at create

  // ---- kept branches (postorder ids), ordered by presence count descending
  int32_t K = 0;                      // kept branches
  int32_t K_pad = 0;                  // K rounded up to 64
  int32_t *d_perm = nullptr;          // [K_pad] node of each position (-1 padding)
  double *d_len_perm = nullptr;       // [K_pad] FP64 length (0 padding)
  uint8_t *d_digits = nullptr;        // [3][K_pad] base-256 digits of len / sigma
  uint32_t *d_qperm = nullptr;        // [K_pad] 24-bit fixed-point length q_k
  double tc_scale = 0.0;              // sigma * 2^-24
  std::vector<int64_t> nb;            // presence count per node (all studies)
  std::vector<int64_t> nb_perm;       // presence count of each kept position
  int32_t max_study_n = 0;            // largest study
  int64_t max_reach = 0;              // most branches reached by one sample

  // ---- statistics
  double stat_pair_branch = 0, stat_useful = 0;
  double stat_launches = 0, stat_tile_pairs = 0;
  unsigned long long *d_counter = nullptr;  // [kCounters] device counters
  double sel_unit = 1.0;                    // branches per counted selection unit
  double sel_unit_v[2] = {1.0, 1.0};        // same, last run of each variant
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  bool ev_valid = false;
  // pair-kernel events of the last run of each variant, and of its sparse kernel
  cudaEvent_t ev_pair[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaEvent_t ev_sp[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaEvent_t ev_list[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // per-branch list pairs
  bool ev_pair_valid[2] = {false, false};

  // ---- options
  int opt_uw_kernel = 0;
  int opt_flush = 256;
  int opt_persistent = 1;  // pair kernels: persistent grid over a device work queue
  // branches present in at most this many samples (slot 0 unweighted, 1
  // weighted) are summed from per-branch lists instead of the sparse kernel
  int64_t opt_rare_list[2] = {256, 256};
  int opt_copy_ranges = 32;  // launches of the weighted dense kernel into pinned host output
  int opt_host_threads = 0;  // threads of the streamed merge (0: the CPUs this process may use)
  // sparse kernels (slot 0 unweighted, 1 weighted): incidences of at most
  // this many pairs are walked by one lane
  int opt_lane_pairs[2] = {64, 128};
  double create_host_ms = 0.0;        // unifrac_create: validation and host preparation
  double create_device_ms = 0.0;      // unifrac_create: device set-up and uploads
  int opt_use_graph = 0;
  int opt_overlap = 1;                // both variants of one call on two streams
  int64_t opt_sparse_threshold = -1;  // presence count below which a branch runs sparse
  int64_t opt_uw_sparse_threshold = -1;  // same, unweighted tensor-core form
  float sp_scale = 1.0f;              // fixed-point scale of the sparse sums (power of 2)

  // ---- cached work list (depends on layout and stripe range only)
  bool items_valid = false;
  int items_layout = -1;
  int32_t items_s0 = 0, items_s1 = 0, n_items = 0;

  // ---- CUDA graph of the last run (UNIFRAC_OPT_USE_GRAPH)
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // second stream of an overlapped two-variant run ([0] normal priority,
  // [1] the device's highest), and its fork / join
  cudaStream_t stream2[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;
  int cur_slot = 0;                   // variant slot being enqueued
  // unifrac_run_streamed: copy stream, its events, and the chunk buffers
  // (two on the device, two pinned on the host), kept between calls
  cudaStream_t copy_stream = nullptr;
  // host output of UNIFRAC_BOTH: the first result's copy to host_part0
  // (bytes, from dev_part0) starts on copy_stream as soon as its kernels end,
  // while the second variant computes
  void *early_host = nullptr;
  const void *early_dev = nullptr;
  size_t early_bytes = 0;
  cudaEvent_t ev_first_done = nullptr;
  // host output of one study's whole matrix (full or condensed): the weighted
  // variant's pair kernel runs as cc_n launches over consecutive ranges of
  // work items, [cc_items[c], cc_items[c+1]), each completing the rows of
  // tile rows [cc_tiles[c], cc_tiles[c+1]); the parts of the matrix a range
  // completes go to host memory on copy_stream while the next computes.
  // cc_variant < 0: off.
  int cc_variant = -1;
  int cc_n = 0;
  std::vector<int32_t> cc_items, cc_tiles;
  std::vector<cudaEvent_t> cc_ev;
  char *cc_host = nullptr;      // the variant's matrix in host memory
  const char *cc_dev = nullptr;  // ... and on the device
  size_t cc_elem = 4;
  int cc_layout = 0;
  int64_t cc_samples = 0;
  std::vector<ufb::WorkItem> h_items;  // host copy of the work list (tile-row order per study)
  cudaEvent_t ev_chunk_done[2] = {nullptr, nullptr}, ev_chunk_copied[2] = {nullptr, nullptr};
  void *chunk_host[2] = {nullptr, nullptr};
  size_t chunk_host_bytes = 0;
  cudaGraphExec_t graph_exec = nullptr;
  int gk_variant = -1, gk_precision = -1, gk_layout = -1;
  int32_t gk_s0 = 0, gk_s1 = 0;
  void *gk_dst = nullptr;
  int64_t gk_opts = -1, opt_generation = 0, gk_bufs = -1, buf_generation = 0;
  // set by the streamed run for its later chunks: the embedding and every
  // variant's packed operands from the chunk before are still valid, so a run
  // enqueues only the pair kernels of its stripe range
  bool reuse_prepared = false;
  uint64_t prep_sig = 0;  // addresses and sizes of those buffers when prepared
  double graph_launches = 0;
  bool capturing = false;

  // ---- work buffers (grown on demand)
  ufb::DevBuf cnt, flag, items, studies, stage, tables, chunk_dev[2];
  ufb::DevBuf chunk_rows[2];  // streamed output: each chunk's stripes as row runs
  ufb::DevBuf item_of;  // [n_tiles x n_tiles] work item of each tile pair, -1 if none
  // [n_tiles] int4 per row tile: the column tiles [x, y) and [z, w) that hold
  // its work items (disjoint runs of item_of's row; [0, n_tiles) if more)
  ufb::DevBuf jrange;
  ufb::VarBufs vb[2];
  size_t device_bytes = 0;
};

namespace ufb {
// buffers and counters of the variant slot being enqueued
inline VarBufs &cur_bufs(unifrac_ctx *ctx) { return ctx->vb[ctx->cur_slot]; }
inline unsigned long long *cur_counters(unifrac_ctx *ctx) {
  return ctx->d_counter + kCounterBase + 4 * ctx->cur_slot;
}
// work queue k of the slot being enqueued, or nullptr when the pair kernels
// run one CTA per work item (UNIFRAC_OPT_PERSISTENT = 0)
inline unsigned int *cur_queue(unifrac_ctx *ctx, int k) {
  return ctx->opt_persistent ? reinterpret_cast<unsigned int *>(ctx->d_counter + 4 * ctx->cur_slot + k)
                             : nullptr;
}
// CTAs of a pair kernel launch: one per work unit, or (persistent) as many as
// are resident at once, at most one per unit
template <typename K>
inline int pair_grid(unifrac_ctx *ctx, K kernel, int threads, size_t smem, int64_t units) {
  if (!ctx->opt_persistent) return (int)units;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return (int)std::min<int64_t>(units, (int64_t)per_sm * ctx->sm_count);
}
}  // namespace ufb

namespace ufb {

int fail(unifrac_ctx *ctx, int code, const std::string &msg);
// Device blocks of the contexts, through the process-wide cache of large
// blocks (devcache.cu): dev_alloc takes a cached block of about the size or
// allocates one (releasing the cache and retrying once when the device is
// full); dev_free returns a block of dev_alloc -- only when no device work can
// still use it -- to the cache, or frees it.
cudaError_t dev_alloc(void **p, size_t bytes);
void dev_free(void *p);
// cudaMalloc for a call's own temporaries (freed with cudaFree), releasing the
// cache and retrying once when the device is full.
cudaError_t dev_malloc_retry(void **p, size_t bytes);
// After launch range c of the chunked variant: the rows that range completed
// are copied to host memory on the copy stream, ordered after the launch.
int enqueue_range_copy(unifrac_ctx *ctx, int c);
// Event record on the context's stream; while a CUDA graph is being captured
// the record becomes a graph node (external event record), so replays
// record the event too and it can be queried afterwards.
void record_event(unifrac_ctx *ctx, cudaEvent_t ev);
int cuda_fail(unifrac_ctx *ctx, cudaError_t e, const char *what);
int grow(unifrac_ctx *ctx, DevBuf &b, size_t bytes);

// embedding (K1) ------------------------------------------------------------
// Fills the counts below each branch (u32, the 128 of a (node, column tile)
// at its slot of the compact array, count_tile) and flag[node][tile] (1 if
// any column of the tile is non-zero) for every node.
// Per node and study, the samples with a non-zero count below the node
// (acc[s * n_nodes + v], v < root), from device bitsets, and from the same
// bitsets the slot map of the compact counts (ctx->d_slot, n_slots); with count_reach
// also the most nodes one column reaches (*max_reach).  Needs the tree, level
// and table rows on the device; synchronises the context's stream.
int presence_counts(unifrac_ctx *ctx, const std::vector<int32_t> &sw, bool count_reach,
                    std::vector<int32_t> &acc, int64_t *max_reach);
int embed_counts(unifrac_ctx *ctx, uint32_t *cnt, uint8_t *flag);

// packing ---------------------------------------------------------------------
// Branch-major values v[k][col] = len_k * cnt / C_col (float or double) and the
// (tile, k) nonzero bitmap words of the positions k < k_end (k_end: K, or a
// multiple of 32).
int pack_weighted(unifrac_ctx *ctx, const uint32_t *cnt, const uint8_t *flag,
                  bool f64, void *vals, uint32_t *bits, int32_t k_end);
// Sparse blocks of positions [32 * kf_words, k_end), one per (tile, window of
// kRareWin positions): sizes, byte offsets boff[n_tiles * n_win + 1] and fill.
// values: weighted blocks (fixed-point values round(v * sp_scale)) from the
// counts; else presence blocks from the presence masks.
// cpre: [n_tiles * n_win][kRareWin / 32 + 1] (rows, entries) before each
// chunk of 32 positions of a block, totals last.
int build_rare_blocks(unifrac_ctx *ctx, bool values, const uint32_t *cnt, const uint32_t *bits,
                      const uint8_t *rc, int32_t kf_words, int32_t k_end, int32_t n_win,
                      uint32_t *bsize, unsigned long long *boff, uint2 *cpre, uint8_t *blocks);
// Packing of positions >= 32 * kf_words for the sparse kernels: bitmap words,
// row non-zero counts and, when aq is given, aq[col] += q_k.
int pack_rare(unifrac_ctx *ctx, const uint32_t *cnt, const uint8_t *flag, int32_t kf_words,
              uint32_t *bits, uint8_t *rc, unsigned long long *aq);
// Exclusive scan of n u32 sizes into u64 offsets, offs[n] = total (one CTA).
int scan_sizes(unifrac_ctx *ctx, int64_t n, const uint32_t *sizes, unsigned long long *offs);
// Buffers of the per-branch lists (see list_fill below).
struct ListBufs {
  unsigned long long *ents = nullptr;  // entries, voff order
  uint2 *trec = nullptr;               // tile-major records
  unsigned long long *toff = nullptr;  // [n_tiles + 1] record offsets per tile
  uint32_t *tcnt = nullptr;            // [n_tiles] records per tile
  uint32_t *tcur = nullptr;            // [n_tiles] fill cursors
  unsigned long long n_ent = 0;        // entries of all lists
};
// Unweighted sparse pairs (u64 per pair) of positions [32 kf_words,
// 32 vr_words), then the listed ones.
int pairs_sparse_presence(unifrac_ctx *ctx, const uint32_t *bits, int32_t kf_words,
                          int32_t vr_words, const uint8_t *blocks, const unsigned long long *boff,
                          const uint2 *cpre, int32_t n_win, ListBufs list,
                          unsigned long long *spart, const WorkItem *items, int32_t n_items);
// Very rarely present positions [pv, K), one list per position (voff: host
// prefix sums of their presence counts): u64 (value << 32) | column for every
// column where the position is present, value = the fixed-point value of the
// sparse blocks (values) or the 24-bit length q_k; a tile-major record per
// entry (entry index, end of its list) with per-tile offsets; the pairs of
// each list added into the sparse partial sums of their tile pairs
// (ctx->item_of), records taken in tile order.
int list_fill(unifrac_ctx *ctx, bool values, const uint32_t *cnt, const uint8_t *flag,
              const uint32_t *bits, const uint8_t *rc, int32_t pv, const long long *voff,
              ListBufs L);
int pairs_list(unifrac_ctx *ctx, bool presence, int32_t pv, ListBufs L, void *spart);
// Bit-packed presence bytes [K_pad/8][n_cols], per-group length tables
// [K_pad/8][256] (FP64), group bitmaps and a_col = sum_k len_k p[k][col].
int pack_lookup(unifrac_ctx *ctx, const uint32_t *cnt, const uint8_t *flag,
                uint8_t *bytes, double *tables, uint32_t *gbits, double *a);
// Sample-major BF16 operands for the tensor-core Gram: X[col][k] in {0,1} and
// three digit planes D_p[col][k] = digit_p(k) * X[col][k]; K-tile bitmaps;
// a_col = tc_scale * sum_k q_k p[k][col] (exact).
// Positions [0, k_tc) (a multiple of 64): X and D have rows of k_tc elements.
// aq (u64 per column) must be zeroed by the caller; finish_tc_a turns it into a.
int pack_tc(unifrac_ctx *ctx, const uint32_t *cnt, const uint8_t *flag, int32_t k_tc,
            uint16_t *X, uint16_t *D, uint32_t *kbits, unsigned long long *aq);
int finish_tc_a(unifrac_ctx *ctx, const unsigned long long *aq, double *a);

// pair kernels ------------------------------------------------------------
// spart: [sp_parts][n_items][TILE * TILE] u32 partial sums of the sparse
// kernel (part p sums the bitmap words 32 p + warp modulo 32 sp_parts),
// 1 <= sp_parts <= kMaxSparseParts.
constexpr int kMaxSparseParts = 8;
int pairs_weighted(unifrac_ctx *ctx, bool f64, const void *vals,
                   const uint32_t *bits, int32_t kf_words, int32_t vr_words,
                   const uint8_t *blocks, const unsigned long long *boff, const uint2 *cpre,
                   int32_t n_win, ListBufs list, uint32_t *spart,
                   int32_t sp_parts, const double *S, const WorkItem *items,
                   int32_t n_items, const OutSpec &o);
int pairs_lookup(unifrac_ctx *ctx, const uint8_t *bytes, const double *tables,
                 const uint32_t *gbits, const double *a, const WorkItem *items,
                 int32_t n_items, const OutSpec &o);
size_t tc_smem_bytes();
// spart: null, or [n_items][TILE * TILE] u64 sums of q over the sparse positions.
// aq: per-sample sums of the 24-bit lengths of the branches present (exact).
int pairs_tc(unifrac_ctx *ctx, int32_t k_tc, const uint16_t *X, const uint16_t *D,
             const uint32_t *kbits, const unsigned long long *aq,
             const unsigned long long *spart, const WorkItem *items, int32_t n_items,
             const OutSpec &o);

}  // namespace ufb
