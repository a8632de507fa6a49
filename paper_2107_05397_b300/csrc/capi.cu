// C ABI of unifrac_b300: context creation (host-side validation and tree /
// table preparation), the run pipeline and the small helper calls.
//
// Section II of the paper frames the problem: a table of microbiome profiles
// that is sparse, a phylogenetic tree over its features, and the all-pairs
// UniFrac distance matrix, computable in stripes that merge into the whole.
#include <sched.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <future>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "ufb_internal.cuh"

namespace ufb {

int fail(unifrac_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->last_error = msg;
  return code;
}

void record_event(unifrac_ctx *ctx, cudaEvent_t ev) {
  if (ctx->capturing)
    cudaEventRecordWithFlags(ev, ctx->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(ev, ctx->stream);
}

int cuda_fail(unifrac_ctx *ctx, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(ctx, UNIFRAC_E_OOM, m);
  return fail(ctx, UNIFRAC_E_CUDA, m);
}

int grow(unifrac_ctx *ctx, DevBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (b.bytes >= bytes) return UNIFRAC_OK;
  if (b.p) {
    // no work of this context (any of its streams) may still use the block
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise before reallocation");
    dev_free(b.p);
    ctx->device_bytes -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
  }
  cudaError_t e = dev_alloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return cuda_fail(ctx, e, "device allocation");
  }
  b.bytes = bytes;
  ctx->buf_generation++;  // a captured graph may hold the old address
  ctx->device_bytes += bytes;
  return UNIFRAC_OK;
}

namespace {

constexpr int32_t kWinWordsHost = kRareWin / WORD;

// Keeps the caller's current device unchanged across a library call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

template <typename T, typename A>
int upload(unifrac_ctx *ctx, T **dst, const std::vector<T, A> &src) {
  size_t bytes = std::max<size_t>(src.size() * sizeof(T), 16);
  cudaError_t e = dev_alloc(reinterpret_cast<void **>(dst), bytes);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "device allocation (inputs)");
  ctx->device_bytes += bytes;
  if (!src.empty()) {
    e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upload inputs");
  }
  return UNIFRAC_OK;
}

// Upload of `count` elements straight from the caller's array.
template <typename T>
int upload_raw(unifrac_ctx *ctx, T **dst, const T *src, size_t count) {
  const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = dev_alloc(reinterpret_cast<void **>(dst), bytes);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "device allocation (inputs)");
  ctx->device_bytes += bytes;
  if (count) {
    e = cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upload inputs");
  }
  return UNIFRAC_OK;
}

// Sample indices of the table entries to embedding columns, in place.
__global__ void k_map_columns(int32_t *ent, int64_t n, const int32_t *__restrict__ col_of_sample) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    ent[e] = col_of_sample[ent[e]];
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Host threads for the O(entries) preparation: one below ~64k entries, else
// up to the hardware's count (at most 32).
// CPUs this process may run on: its affinity mask, lowered to a cgroup CPU
// quota where one is set (cgroup v2 cpu.max, else v1 cfs_quota_us /
// cfs_period_us).  More threads than that only queue behind each other.
static int usable_cpus() {
  static const int n = [] {
    int c = 0;
    cpu_set_t set;
    if (sched_getaffinity(0, sizeof(set), &set) == 0) c = CPU_COUNT(&set);
    if (c <= 0) c = (int)std::max(1u, std::thread::hardware_concurrency());
    long long quota = -1, period = 0;
    if (FILE *f = std::fopen("/sys/fs/cgroup/cpu.max", "r")) {
      char q[32] = {0};
      if (std::fscanf(f, "%31s %lld", q, &period) == 2 && std::strcmp(q, "max") != 0)
        quota = std::atoll(q);
      std::fclose(f);
    } else if (FILE *fq = std::fopen("/sys/fs/cgroup/cpu/cpu.cfs_quota_us", "r")) {
      if (std::fscanf(fq, "%lld", &quota) != 1) quota = -1;
      std::fclose(fq);
      if (FILE *fp = std::fopen("/sys/fs/cgroup/cpu/cpu.cfs_period_us", "r")) {
        if (std::fscanf(fp, "%lld", &period) != 1) period = 0;
        std::fclose(fp);
      }
    }
    if (quota > 0 && period > 0) c = std::min<long long>(c, std::max(1LL, (quota + period - 1) / period));
    return c;
  }();
  return n;
}

int host_threads(int64_t work) {
  if (work < (1 << 16)) return 1;
  return std::max(1, std::min(32, usable_cpus()));
}

// Runs fn(0) .. fn(T-1) on T threads (fn(0) on the calling thread).
template <typename F>
void run_threads(int T, F &&fn) {
  std::vector<std::thread> th;
  th.reserve(T > 1 ? T - 1 : 0);
  for (int t = 1; t < T; ++t) th.emplace_back(fn, t);
  fn(0);
  for (auto &x : th) x.join();
}

void free_ctx(unifrac_ctx *ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  // every stream of the context idle before its blocks go back to the cache
  cudaDeviceSynchronize();
  void *ptrs[] = {ctx->d_level_nodes, ctx->d_level_ptr, ctx->d_child_ptr, ctx->d_child_idx, ctx->d_frow_tip,
                  ctx->d_frow_ptr,    ctx->d_tchunk_row, ctx->d_tchunk_lo, ctx->d_pmask,
                  ctx->d_fent_col,  ctx->d_fent_cnt,  ctx->d_inv_total,
                  ctx->d_S,           ctx->d_perm,
                  ctx->d_len_perm,    ctx->d_digits,    ctx->d_counter,   ctx->d_qperm,
                  ctx->d_slot};
  for (void *p : ptrs)
    if (p) dev_free(p);
  ufb::DevBuf *bufs[] = {&ctx->cnt,   &ctx->flag,   &ctx->items,        &ctx->studies,
                         &ctx->stage, &ctx->tables, &ctx->chunk_dev[0], &ctx->chunk_dev[1],
                         &ctx->chunk_rows[0], &ctx->chunk_rows[1], &ctx->item_of,
                         &ctx->jrange};
  for (auto *b : bufs)
    if (b->p) dev_free(b->p);
  for (auto &V : ctx->vb) {
    ufb::DevBuf *vbufs[] = {&V.vals, &V.vals2, &V.bits,   &V.persample, &V.partial, &V.rc,
                            &V.bsize, &V.boff, &V.blocks, &V.cpre,      &V.spart,   &V.rbits,
                            &V.vlist, &V.voff,  &V.trec,    &V.tidx};
    for (auto *b : vbufs)
      if (b->p) dev_free(b->p);
  }
  for (cudaStream_t s : ctx->stream2)
    if (s) cudaStreamDestroy(s);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  for (cudaEvent_t ev : ctx->cc_ev)
    if (ev) cudaEventDestroy(ev);
  for (int b = 0; b < 2; ++b) {
    if (ctx->ev_chunk_done[b]) cudaEventDestroy(ctx->ev_chunk_done[b]);
    if (ctx->ev_chunk_copied[b]) cudaEventDestroy(ctx->ev_chunk_copied[b]);
    if (ctx->chunk_host[b]) cudaFreeHost(ctx->chunk_host[b]);
  }
  if (ctx->ev_first_done) cudaEventDestroy(ctx->ev_first_done);
  if (ctx->ev_fork2) cudaEventDestroy(ctx->ev_fork2);
  if (ctx->ev_join2) cudaEventDestroy(ctx->ev_join2);
  for (auto &e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (auto &pr : ctx->ev_pair)
    for (auto &e : pr)
      if (e) cudaEventDestroy(e);
  for (auto *set : {&ctx->ev_sp, &ctx->ev_list})
    for (auto &pr : *set)
      for (auto &e : pr)
        if (e) cudaEventDestroy(e);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

int64_t n_pairs_layout(int layout, int64_t n, int32_t s0, int32_t s1) {
  if (layout == UNIFRAC_OUT_FULL) return n * n;
  if (layout == UNIFRAC_OUT_CONDENSED) return n * (n - 1) / 2;
  return (int64_t)(s1 - s0) * n;
}

// Tile pairs (I <= J) of a study that hold at least one pair of the stripe
// range, plus the diagonal tiles when the layout writes a diagonal.
void study_items(int32_t study, int32_t n, int32_t tile0, int layout, int32_t s0, int32_t s1,
                 std::vector<WorkItem> &items) {
  if (n <= 0) return;
  if (n == 1 && layout != UNIFRAC_OUT_FULL) return;
  const int32_t T = (n + TILE - 1) / TILE;
  // Tile pairs in blocks of kOrderBlock x kOrderBlock tiles: the CTAs resident
  // at one time (about one block) then share their row tiles and their column
  // tiles, so each operand slice comes from DRAM once per block and is reused
  // from L2 (row by row, every CTA of a wave would stream its own column
  // tile).  The set of pairs is the same in any order.
  constexpr int32_t kOrderBlock = 12;
  for (int32_t BI = 0; BI < T; BI += kOrderBlock)
  for (int32_t BJ = BI; BJ < T; BJ += kOrderBlock)
  for (int32_t I = BI; I < std::min(T, BI + kOrderBlock); ++I) {
    for (int32_t J = std::max(I, BJ); J < std::min(T, BJ + kOrderBlock); ++J) {
      bool need = (I == J && layout == UNIFRAC_OUT_FULL);
      if (!need) {
        // differences delta = lj - li of pairs li < lj in the tile pair
        const int64_t i0 = (int64_t)I * TILE, i1 = std::min<int64_t>(i0 + TILE, n) - 1;
        const int64_t j0 = (int64_t)J * TILE, j1 = std::min<int64_t>(j0 + TILE, n) - 1;
        const int64_t dlo = std::max<int64_t>(1, j0 - i1), dhi = j1 - i0;
        if (dlo <= dhi) {
          // stripe of delta: min(delta-1, n-delta-1) in [s0, s1)
          //   delta in [s0+1, s1]  or  delta in [n-s1, n-s0-1]
          const int64_t a0 = std::max<int64_t>(dlo, s0 + 1), a1 = std::min<int64_t>(dhi, s1);
          const int64_t b0 = std::max<int64_t>(dlo, (int64_t)n - s1),
                        b1 = std::min<int64_t>(dhi, (int64_t)n - s0 - 1);
          need = (a0 <= a1) || (b0 <= b1);
        }
      }
      if (need) items.push_back(WorkItem{tile0 + I, tile0 + J, study, 0});
    }
  }
}

}  // namespace
}  // namespace ufb

using namespace ufb;

extern "C" {

const char *unifrac_strerror(int status) {
  switch (status) {
    case UNIFRAC_OK: return "success";
    case UNIFRAC_E_INVALID_ARG: return "invalid argument";
    case UNIFRAC_E_BAD_TREE: return "malformed tree";
    case UNIFRAC_E_BAD_TABLE: return "malformed table";
    case UNIFRAC_E_STRIPE_RANGE: return "stripe range out of bounds";
    case UNIFRAC_E_BUFFER_TOO_SMALL: return "output buffer too small";
    case UNIFRAC_E_CUDA: return "CUDA error";
    case UNIFRAC_E_OOM: return "out of memory";
    case UNIFRAC_E_DEVICE_TIMEOUT: return "device-side wait timed out";
    case UNIFRAC_E_UNSUPPORTED: return "unsupported combination";
    default: return "unknown status";
  }
}

const char *unifrac_last_error(const unifrac_ctx *ctx) {
  return ctx ? ctx->last_error.c_str() : "no context";
}

static int create_impl(int32_t n_nodes, const int32_t *parent, const double *length,
                       int32_t n_features, const int32_t *feature_node, int32_t n_samples,
                       const int64_t *indptr, const int32_t *indices, const int32_t *counts,
                       int32_t n_studies, const int32_t *study_offsets, void *cuda_stream,
                       unifrac_ctx *ctx) {
  const auto t_create0 = std::chrono::steady_clock::now();
  // ---------------------------------------------------------------- arguments
  if (n_nodes < 1 || !parent || !length) return fail(ctx, UNIFRAC_E_INVALID_ARG, "tree arrays");
  if (n_features < 0 || n_samples < 0 || !indptr)
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "table sizes / indptr");
  if (n_features > 0 && !feature_node)
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "feature_node is NULL");
  if (n_studies < 1) return fail(ctx, UNIFRAC_E_INVALID_ARG, "n_studies < 1");
  if (n_studies > 1 && !study_offsets)
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "study_offsets is NULL with several studies");
  const int64_t nnz = indptr[n_features];
  if (indptr[0] != 0 || nnz < 0) return fail(ctx, UNIFRAC_E_BAD_TABLE, "indptr[0] != 0");
  if (nnz > 0 && (!indices || !counts))
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "indices / counts NULL");
  if (n_samples > (INT32_MAX / 2)) return fail(ctx, UNIFRAC_E_INVALID_ARG, "too many samples");

  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->n_nodes = n_nodes;
  ctx->n_features = n_features;
  ctx->n_samples = n_samples;
  ctx->n_studies = n_studies;
  ctx->nnz = nnz;
  const int32_t root = n_nodes - 1;

  // ---------------------------------------------------------------- tree
  for (int32_t k = 0; k < root; ++k) {
    if (parent[k] <= k || parent[k] >= n_nodes)
      return fail(ctx, UNIFRAC_E_BAD_TREE,
                  "parent[" + std::to_string(k) + "] is not a later node (postorder required)");
    if (!std::isfinite(length[k]) || length[k] < 0.0)
      return fail(ctx, UNIFRAC_E_BAD_TREE,
                  "length[" + std::to_string(k) + "] is negative or not finite");
  }
  if (parent[root] != -1) return fail(ctx, UNIFRAC_E_BAD_TREE, "the last node must be the root");
  std::vector<int32_t> child_ptr(n_nodes + 1, 0), child_idx(std::max(root, 1));
  for (int32_t k = 0; k < root; ++k) child_ptr[parent[k] + 1]++;
  for (int32_t v = 0; v < n_nodes; ++v) child_ptr[v + 1] += child_ptr[v];
  {
    std::vector<int32_t> fill(child_ptr.begin(), child_ptr.end() - 1);
    for (int32_t k = 0; k < root; ++k) child_idx[fill[parent[k]]++] = k;
  }
  // levels: tips 0, internal nodes 1 + highest child
  std::vector<int32_t> level(n_nodes, 0);
  for (int32_t k = 0; k < root; ++k) level[parent[k]] = std::max(level[parent[k]], level[k] + 1);
  int32_t max_level = 0;
  for (int32_t k = 0; k < root; ++k) max_level = std::max(max_level, level[k]);
  ctx->n_levels = max_level;
  ctx->level_ptr.assign(max_level + 1, 0);
  for (int32_t k = 0; k < root; ++k)
    if (level[k] >= 1) ctx->level_ptr[level[k]]++;
  for (int32_t L = 0; L < max_level; ++L) ctx->level_ptr[L + 1] += ctx->level_ptr[L];
  std::vector<int32_t> level_nodes(ctx->level_ptr[max_level]);
  {
    std::vector<int32_t> fill(ctx->level_ptr.begin(), ctx->level_ptr.end());
    for (int32_t k = 0; k < root; ++k)
      if (level[k] >= 1) level_nodes[fill[level[k] - 1]++] = k;
  }
  // root-to-node path length (root branch excluded), parents before children
  std::vector<double> depth(n_nodes, 0.0);
  for (int32_t k = root - 1; k >= 0; --k) depth[k] = depth[parent[k]] + length[k];

  // ---------------------------------------------------------------- studies
  std::vector<int32_t> soff(n_studies + 1, 0);
  if (study_offsets) {
    for (int32_t s = 0; s <= n_studies; ++s) soff[s] = study_offsets[s];
  } else {
    soff[1] = n_samples;
  }
  if (soff[0] != 0 || soff[n_studies] != n_samples)
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "study_offsets must run from 0 to n_samples");
  for (int32_t s = 0; s < n_studies; ++s)
    if (soff[s + 1] < soff[s]) return fail(ctx, UNIFRAC_E_INVALID_ARG, "study_offsets decrease");
  ctx->study_off = soff;
  ctx->study_col0.assign(n_studies, 0);
  int64_t cols = 0;
  for (int32_t s = 0; s < n_studies; ++s) {
    ctx->study_col0[s] = (int32_t)cols;
    cols += ((int64_t)(soff[s + 1] - soff[s]) + TILE - 1) / TILE * TILE;
  }
  if (cols > INT32_MAX / 2) return fail(ctx, UNIFRAC_E_INVALID_ARG, "too many samples");
  ctx->n_cols = (int32_t)cols;
  ctx->n_tiles = ctx->n_cols / TILE;
  ctx->col_of_sample.assign(n_samples, 0);
  std::vector<int32_t> study_of(n_samples, 0);
  for (int32_t s = 0; s < n_studies; ++s)
    for (int32_t i = soff[s]; i < soff[s + 1]; ++i) {
      ctx->col_of_sample[i] = ctx->study_col0[s] + (i - soff[s]);
      study_of[i] = s;
    }

  // ---------------------------------------------------------------- table
  std::vector<char> tip_used(n_nodes, 0);
  for (int32_t f = 0; f < n_features; ++f) {
    const int32_t t = feature_node[f];
    if (t < 0 || t >= n_nodes)
      return fail(ctx, UNIFRAC_E_BAD_TREE, "feature_node[" + std::to_string(f) + "] out of range");
    if (child_ptr[t + 1] != child_ptr[t])
      return fail(ctx, UNIFRAC_E_BAD_TREE,
                  "feature " + std::to_string(f) + " sits on an internal node");
    if (tip_used[t])
      return fail(ctx, UNIFRAC_E_BAD_TABLE, "two features on tip " + std::to_string(t));
    tip_used[t] = 1;
  }
  std::vector<int64_t> total(n_samples, 0);
  std::vector<int32_t> frow_tip;
  std::vector<int64_t> frow_ptr(1, 0);
  std::vector<int32_t> fent_col;   // entry columns and counts, unless `direct`
  std::vector<uint32_t> fent_cnt;
  std::vector<std::pair<int32_t, int32_t>> row;  // (sample, count)
  // Parallel pass for the usual table: every row's sample indices strictly
  // increasing and in range, counts >= 0.  Threads check their rows (reading
  // only) and add per-thread sample totals, summed in thread order
  // (integers).  Without explicit zeros the caller's indices and counts are
  // the entry arrays themselves (`direct`: uploaded as they are, sample
  // indices mapped to embedding columns on the device); with zeros they are
  // copied without them.  Any other table takes the sequential pass below,
  // which reports what is wrong.
  bool table_done = false, direct = false;
  {
    const int T = host_threads(nnz);
    std::vector<uint8_t> bad(T, 0);
    std::vector<int64_t> zeros(T, 0);
    std::vector<std::vector<int64_t>> tot(T);
    run_threads(T, [&](int t) {
      std::vector<int64_t> &tt = tot[t];
      tt.assign(n_samples, 0);
      int64_t z = 0;  // local: one shared counter per thread would share a cache line
      for (int32_t f = (int32_t)((int64_t)n_features * t / T);
           f < (int32_t)((int64_t)n_features * (t + 1) / T); ++f) {
        const int64_t lo = indptr[f], hi = indptr[f + 1];
        if (hi < lo || lo < 0 || hi > nnz) {
          bad[t] = 1;
          return;
        }
        for (int64_t e = lo; e < hi; ++e) {
          const int32_t i = indices[e];
          if (i < 0 || i >= n_samples || counts[e] < 0 || (e > lo && i <= indices[e - 1])) {
            bad[t] = 1;
            return;
          }
          tt[i] += counts[e];
          z += counts[e] == 0;
        }
      }
      zeros[t] = z;
    });
    if (std::find(bad.begin(), bad.end(), 1) == bad.end() && indptr[0] == 0 &&
        indptr[n_features] == nnz) {
      const bool has_zeros = std::accumulate(zeros.begin(), zeros.end(), (int64_t)0) > 0;
      direct = !has_zeros;
      int64_t out = 0;
      if (has_zeros) {
        fent_col.reserve((size_t)nnz);
        fent_cnt.reserve((size_t)nnz);
      }
      for (int32_t f = 0; f < n_features; ++f) {
        const int64_t start_f = out;
        if (has_zeros) {
          for (int64_t e = indptr[f]; e < indptr[f + 1]; ++e)
            if (counts[e] != 0) {
              fent_col.push_back(ctx->col_of_sample[indices[e]]);
              fent_cnt.push_back((uint32_t)counts[e]);
              ++out;
            }
        } else {
          out = indptr[f + 1];
        }
        if (out > start_f) {
          frow_tip.push_back(feature_node[f]);
          frow_ptr.push_back(out);
        }
      }
      for (int t = 0; t < T; ++t)
        for (int32_t i = 0; i < n_samples; ++i) total[i] += tot[t][i];
      table_done = true;
    }
  }
  if (!table_done) {
  frow_tip.reserve(n_features);
  frow_ptr.reserve((size_t)n_features + 1);
  fent_col.reserve((size_t)nnz);
  fent_cnt.reserve((size_t)nnz);
  for (int32_t f = 0; f < n_features; ++f) {
    const int64_t lo = indptr[f], hi = indptr[f + 1];
    if (hi < lo || hi > nnz) return fail(ctx, UNIFRAC_E_BAD_TABLE, "indptr not monotone");
    // fast path: sample indices strictly increasing and in range (no sort,
    // no duplicates possible)
    bool ordered = true;
    for (int64_t e = lo; e < hi && ordered; ++e)
      ordered = indices[e] >= 0 && indices[e] < n_samples && counts[e] >= 0 &&
                (e == lo || indices[e] > indices[e - 1]);
    if (ordered) {
      const size_t before = fent_col.size();
      for (int64_t e = lo; e < hi; ++e) {
        if (counts[e] == 0) continue;
        const int32_t i = indices[e];
        fent_col.push_back(ctx->col_of_sample[i]);
        fent_cnt.push_back((uint32_t)counts[e]);
        total[i] += counts[e];
      }
      if (fent_col.size() == before) continue;
      frow_tip.push_back(feature_node[f]);
      frow_ptr.push_back((int64_t)fent_col.size());
      continue;
    }
    row.clear();
    for (int64_t e = lo; e < hi; ++e) {
      const int32_t s = indices[e];
      if (s < 0 || s >= n_samples)
        return fail(ctx, UNIFRAC_E_BAD_TABLE, "sample index out of range in row " + std::to_string(f));
      if (counts[e] < 0) return fail(ctx, UNIFRAC_E_BAD_TABLE, "negative count");
      if (counts[e] > 0) row.emplace_back(s, counts[e]);
    }
    if (!std::is_sorted(row.begin(), row.end())) std::sort(row.begin(), row.end());
    for (size_t q = 1; q < row.size(); ++q)
      if (row[q].first == row[q - 1].first)
        return fail(ctx, UNIFRAC_E_BAD_TABLE,
                    "duplicate (feature, sample) entry in row " + std::to_string(f));
    // explicit zeros are absent features, but duplicates including zeros are still malformed
    for (int64_t e = lo + 1; e < hi; ++e)
      if (indices[e] == indices[e - 1])
        return fail(ctx, UNIFRAC_E_BAD_TABLE,
                    "duplicate (feature, sample) entry in row " + std::to_string(f));
    if (row.empty()) continue;
    frow_tip.push_back(feature_node[f]);
    for (auto &pr : row) {
      fent_col.push_back(ctx->col_of_sample[pr.first]);
      fent_cnt.push_back((uint32_t)pr.second);
      total[pr.first] += pr.second;
    }
    frow_ptr.push_back((int64_t)fent_col.size());
  }
  }  // sequential pass
  for (int32_t i = 0; i < n_samples; ++i)
    if (total[i] > (int64_t)UINT32_MAX)
      return fail(ctx, UNIFRAC_E_BAD_TABLE,
                  "sample " + std::to_string(i) + " has a total count >= 2^32");
  ctx->n_frows = (int32_t)frow_tip.size();
  std::vector<int32_t> tchunk_row;
  std::vector<int64_t> tchunk_lo;
  tchunk_row.reserve(frow_tip.size() + (size_t)(frow_ptr.back() / ctx->tip_chunk) + 1);
  tchunk_lo.reserve(tchunk_row.capacity());
  for (int32_t r = 0; r < ctx->n_frows; ++r)
    for (int64_t lo = frow_ptr[r]; lo < frow_ptr[r + 1]; lo += ctx->tip_chunk) {
      tchunk_row.push_back(r);
      tchunk_lo.push_back(lo);
    }
  ctx->n_tchunks = (int64_t)tchunk_row.size();
  // Per-column weighted sums S_col = sum_b v[b][col] through the tip-depth
  // identity (every count below a branch is a tip count, and a tip's count
  // appears once for every branch on its root path):
  // S_i = (1 / C_i) * sum_f c_fi * depth(tip_f), FP64, entries in row order;
  // fixed for the context, so computed once here -- on a background task
  // while the device phase below runs (it reads only the table rows and the
  // tip depths, which nothing changes meanwhile).
  // (64 fixed chunks of rows, summed in chunk order: the same result
  // whatever the number of host threads)
  auto s_task = std::async(std::launch::async, [&]() {
    std::vector<double> S(ctx->n_cols, 0.0);
    const int32_t R = ctx->n_frows;
    const int kChunks = R >= 4096 ? 64 : 1;
    std::vector<std::vector<double>> part(kChunks);
    std::atomic<int> next_chunk{0};
    const int64_t n_ent = direct ? nnz : (int64_t)fent_col.size();
    run_threads(std::min(kChunks, host_threads(n_ent)), [&](int) {
      for (int c; (c = next_chunk.fetch_add(1)) < kChunks;) {
        std::vector<double> &P = part[c];
        P.assign(ctx->n_cols, 0.0);
        for (int32_t r = (int32_t)((int64_t)R * c / kChunks);
             r < (int32_t)((int64_t)R * (c + 1) / kChunks); ++r) {
          const double dep = depth[frow_tip[r]];
          for (int64_t e = frow_ptr[r]; e < frow_ptr[r + 1]; ++e)
            if (direct)
              P[ctx->col_of_sample[indices[e]]] += (double)counts[e] * dep;
            else
              P[fent_col[e]] += (double)fent_cnt[e] * dep;
        }
      }
    });
    for (int c = 0; c < kChunks; ++c)
      for (int32_t col = 0; col < ctx->n_cols; ++col) S[col] += part[c][col];
    return S;
  });

  // ------------------------------------------- presence counts and pruning
  // n_b: the samples with a non-zero count below branch b, per study, from
  // per-node sample bitsets built on the device (tips from their table rows,
  // internal nodes as the OR of their children, level by level), popcounted
  // over each study's columns; with the tree's size above the tensor-core
  // exactness bound, also the most branches one sample reaches.  The device
  // needs the tree, its levels and the table rows for this, so they are
  // uploaded here.
  double dev_ms = 0.0;
  ctx->nb.assign(n_nodes, 0);
  double pair_branch = 0.0, useful = 0.0;
  int rc;
  {
    const auto t_dev0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&ctx->device) != cudaSuccess)
      return fail(ctx, UNIFRAC_E_CUDA, "no CUDA device");
    const cudaError_t e =
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device attribute");
    if ((rc = upload(ctx, &ctx->d_level_nodes, level_nodes))) return rc;
    if ((rc = upload(ctx, &ctx->d_level_ptr, ctx->level_ptr))) return rc;
    if ((rc = upload(ctx, &ctx->d_child_ptr, child_ptr))) return rc;
    if ((rc = upload(ctx, &ctx->d_child_idx, child_idx))) return rc;
    if ((rc = upload(ctx, &ctx->d_frow_tip, frow_tip))) return rc;
    if ((rc = upload(ctx, &ctx->d_frow_ptr, frow_ptr))) return rc;
    if ((rc = upload(ctx, &ctx->d_tchunk_row, tchunk_row))) return rc;
    if ((rc = upload(ctx, &ctx->d_tchunk_lo, tchunk_lo))) return rc;
    {
      const size_t pm_bytes = std::max<size_t>((size_t)ctx->n_nodes * ctx->n_tiles * 16, 16);
      const cudaError_t em = dev_alloc(reinterpret_cast<void **>(&ctx->d_pmask), pm_bytes);
      if (em != cudaSuccess) return cuda_fail(ctx, em, "device allocation (presence masks)");
      ctx->device_bytes += pm_bytes;
    }
    if (!direct) {
      if ((rc = upload(ctx, &ctx->d_fent_col, fent_col))) return rc;
    } else {  // the caller's sample indices, mapped to columns when studies add padding
      if ((rc = upload_raw(ctx, &ctx->d_fent_col, indices, (size_t)nnz))) return rc;
      if (n_studies > 1 && nnz > 0) {
        int32_t *d_map = nullptr;
        if ((rc = upload_raw(ctx, &d_map, ctx->col_of_sample.data(), ctx->col_of_sample.size())))
          return rc;
        k_map_columns<<<(unsigned)std::min<int64_t>((nnz + 255) / 256, 148 * 32), 256>>>(
            ctx->d_fent_col, nnz, d_map);
        cudaError_t e2 = cudaGetLastError();
        if (e2 == cudaSuccess) e2 = cudaDeviceSynchronize();
        dev_free(d_map);
        ctx->device_bytes -= std::max<size_t>(ctx->col_of_sample.size() * 4, 16);
        if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "column map");
      }
    }
    // a sample reaches at most root branches: count exactly only when that
    // bound does not already settle the tensor-core exactness test
    const bool count_reach = (int64_t)root >= 65793;
    if (!count_reach) ctx->max_reach = root;
    std::vector<int32_t> sw(2 * (size_t)n_studies);  // 64-bit word range of each study
    for (int32_t st = 0; st < n_studies; ++st) {
      sw[2 * st] = ctx->study_col0[st] / 64;
      sw[2 * st + 1] =
          sw[2 * st] + (int32_t)(((int64_t)(soff[st + 1] - soff[st]) + TILE - 1) / TILE * 2);
    }
    std::vector<int32_t> acc;
    int64_t reach = 0;
    if ((rc = presence_counts(ctx, sw, count_reach, acc, &reach))) return rc;
    if (count_reach) ctx->max_reach = reach;
    for (int32_t st = 0; st < n_studies; ++st) {  // statistics in study order
      const int32_t *a = acc.data() + (size_t)st * n_nodes;
      int64_t B_s = 0;
      for (int32_t v = 0; v < root; ++v) {
        ctx->nb[v] += a[v];
        if (a[v] > 0 && length[v] > 0.0) {
          B_s++;
          useful += 0.5 * (double)a[v] * (double)(a[v] - 1);
        }
      }
      const double n_s = (double)(soff[st + 1] - soff[st]);
      pair_branch += 0.5 * n_s * (n_s - 1.0) * (double)B_s;
    }
    dev_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_dev0).count();
  }
  ctx->stat_pair_branch = pair_branch;
  ctx->stat_useful = useful;
  // kept branches by presence count, descending, ties in node order: a
  // stable counting sort (counts are at most n_samples)
  std::vector<int32_t> perm;
  {
    std::vector<int64_t> start((size_t)n_samples + 2, 0);
    int64_t kept = 0;
    for (int32_t v = 0; v < root; ++v)
      if (ctx->nb[v] > 0 && length[v] > 0.0) {
        start[(size_t)(n_samples - ctx->nb[v]) + 1]++;  // bucket n_samples - nb: larger counts first
        kept++;
      }
    for (size_t b = 1; b < start.size(); ++b) start[b] += start[b - 1];
    perm.resize((size_t)kept);
    for (int32_t v = 0; v < root; ++v)
      if (ctx->nb[v] > 0 && length[v] > 0.0) perm[(size_t)start[(size_t)(n_samples - ctx->nb[v])]++] = v;
  }
  ctx->K = (int32_t)perm.size();
  ctx->nb_perm.resize(perm.size());
  for (size_t k = 0; k < perm.size(); ++k) ctx->nb_perm[k] = ctx->nb[perm[k]];
  for (int32_t s = 0; s < n_studies; ++s)
    ctx->max_study_n = std::max(ctx->max_study_n, soff[s + 1] - soff[s]);
  // fixed-point scale of the sparse weighted sums: every pair sum is at most
  // the deepest tip's depth D < 2^ed, so scale = 2^(30 - ed) keeps each u32
  // sum (plus at most half a unit per term) below 2^31
  {
    double dmax = 0.0;
    for (int32_t f = 0; f < n_features; ++f) dmax = std::max(dmax, depth[feature_node[f]]);
    int ed = 0;
    if (dmax > 0.0) std::frexp(dmax, &ed);  // dmax < 2^ed
    ctx->sp_scale = std::ldexp(1.0f, std::max(-100, std::min(100, 30 - ed)));
  }
  ctx->K_pad = std::max<int32_t>(64, (ctx->K + 63) / 64 * 64);
  std::vector<double> len_perm(ctx->K_pad, 0.0);
  for (int32_t k = 0; k < ctx->K; ++k) len_perm[k] = length[perm[k]];
  perm.resize(ctx->K_pad, -1);
  // base-256 digits of len / sigma for the tensor-core Gram (24-bit fixed
  // point, sigma the power of two just above the longest kept branch)
  double maxlen = 0.0;
  for (int32_t k = 0; k < ctx->K; ++k) maxlen = std::max(maxlen, len_perm[k]);
  int ex = 0;
  if (maxlen > 0.0) std::frexp(maxlen, &ex);  // maxlen < 2^ex
  const double sigma = std::ldexp(1.0, ex);
  ctx->tc_scale = std::ldexp(sigma, -24);
  std::vector<uint8_t> digits(3 * (size_t)ctx->K_pad, 0);
  for (int32_t k = 0; k < ctx->K; ++k) {
    int64_t q = std::llround(std::ldexp(len_perm[k] / sigma, 24));
    q = std::min<int64_t>(std::max<int64_t>(q, 0), (1 << 24) - 1);
    digits[k] = (uint8_t)(q >> 16);
    digits[ctx->K_pad + k] = (uint8_t)((q >> 8) & 255);
    digits[2 * (size_t)ctx->K_pad + k] = (uint8_t)(q & 255);
  }

  // per-column reciprocal totals and the column-sorted table
  std::vector<double> inv_total(ctx->n_cols, 0.0);
  for (int32_t i = 0; i < n_samples; ++i)
    if (total[i] > 0) inv_total[ctx->col_of_sample[i]] = 1.0 / (double)total[i];
  std::vector<double> S = s_task.get();  // the sums of the task above, times 1 / C_i here
  for (int32_t c = 0; c < ctx->n_cols; ++c) S[c] *= inv_total[c];
  ctx->create_host_ms = ms_since(t_create0) - dev_ms;

  // ---------------------------------------------------------------- device
  cudaError_t e;
  if (!direct) {
    if ((rc = upload(ctx, &ctx->d_fent_cnt, fent_cnt))) return rc;
  } else if ((rc = upload_raw(ctx, &ctx->d_fent_cnt, reinterpret_cast<const uint32_t *>(counts),
                              (size_t)nnz))) {  // counts >= 0: the same bits as u32
    return rc;
  }
  if ((rc = upload(ctx, &ctx->d_inv_total, inv_total))) return rc;
  if ((rc = upload(ctx, &ctx->d_S, S))) return rc;
  if ((rc = upload(ctx, &ctx->d_perm, perm))) return rc;
  if ((rc = upload(ctx, &ctx->d_len_perm, len_perm))) return rc;
  if ((rc = upload(ctx, &ctx->d_digits, digits))) return rc;
  {
    std::vector<uint32_t> qperm(ctx->K_pad, 0u);
    for (int32_t k = 0; k < ctx->K; ++k)
      qperm[k] = ((uint32_t)digits[k] << 16) | ((uint32_t)digits[ctx->K_pad + k] << 8) |
                 (uint32_t)digits[2 * (size_t)ctx->K_pad + k];
    if ((rc = upload(ctx, &ctx->d_qperm, qperm))) return rc;
  }
  std::vector<unsigned long long> zero_counters(kCounters, 0ull);
  if ((rc = upload(ctx, &ctx->d_counter, zero_counters))) return rc;
  for (auto &ev : ctx->ev) {
    e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event");
  }
  for (auto &pr : ctx->ev_pair)
    for (auto &ev : pr) {
      e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "event");
    }
  for (auto *set : {&ctx->ev_sp, &ctx->ev_list})
    for (auto &pr : *set)
      for (auto &ev : pr) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "event");
      }
  ctx->create_device_ms = ms_since(t_create0) - ctx->create_host_ms;
  return UNIFRAC_OK;
}

int unifrac_create(int32_t n_nodes, const int32_t *parent, const double *length,
                   int32_t n_features, const int32_t *feature_node, int32_t n_samples,
                   const int64_t *indptr, const int32_t *indices, const int32_t *counts,
                   int32_t n_studies, const int32_t *study_offsets, void *cuda_stream,
                   unifrac_ctx **out) {
  if (!out) return UNIFRAC_E_INVALID_ARG;
  *out = nullptr;
  unifrac_ctx *ctx = new (std::nothrow) unifrac_ctx();
  if (!ctx) return UNIFRAC_E_OOM;
  int rc;
  try {
    rc = create_impl(n_nodes, parent, length, n_features, feature_node, n_samples, indptr,
                     indices, counts, n_studies, study_offsets, cuda_stream, ctx);
  } catch (const std::bad_alloc &) {
    rc = UNIFRAC_E_OOM;
  } catch (...) {
    rc = UNIFRAC_E_INVALID_ARG;
  }
  if (rc != UNIFRAC_OK) {
    free_ctx(ctx);
    return rc;
  }
  *out = ctx;
  return UNIFRAC_OK;
}

void unifrac_destroy(unifrac_ctx *ctx) { free_ctx(ctx); }

int unifrac_n_stripes(const unifrac_ctx *ctx, int32_t study, int32_t *out) {
  if (!ctx || !out || study < 0 || study >= ctx->n_studies) return UNIFRAC_E_INVALID_ARG;
  *out = (ctx->study_off[study + 1] - ctx->study_off[study]) / 2;
  return UNIFRAC_OK;
}

static int resolve_range(const unifrac_ctx *ctx, int layout, int32_t s0, int32_t s1,
                         int32_t *r0, int32_t *r1) {
  if (ctx->n_studies > 1) {
    if (layout == UNIFRAC_OUT_STRIPES || s0 != 0 || s1 != -1) return UNIFRAC_E_UNSUPPORTED;
    *r0 = 0;
    *r1 = INT32_MAX;
    return UNIFRAC_OK;
  }
  const int32_t nst = ctx->n_samples / 2;
  if (s1 == -1) s1 = nst;
  if (s0 < 0 || s1 < s0 || s1 > nst) return UNIFRAC_E_STRIPE_RANGE;
  *r0 = s0;
  *r1 = s1;
  return UNIFRAC_OK;
}

int unifrac_output_bytes(const unifrac_ctx *ctx, int precision, int layout,
                         int32_t stripe_start, int32_t stripe_stop, size_t *out) {
  if (!ctx || !out) return UNIFRAC_E_INVALID_ARG;
  if (precision != UNIFRAC_FP64 && precision != UNIFRAC_MIXED) return UNIFRAC_E_INVALID_ARG;
  if (layout < UNIFRAC_OUT_STRIPES || layout > UNIFRAC_OUT_FULL) return UNIFRAC_E_INVALID_ARG;
  int32_t s0, s1;
  int rc = resolve_range(ctx, layout, stripe_start, stripe_stop, &s0, &s1);
  if (rc) return rc;
  int64_t elems = 0;
  for (int32_t s = 0; s < ctx->n_studies; ++s)
    elems += n_pairs_layout(layout, ctx->study_off[s + 1] - ctx->study_off[s], s0, s1);
  *out = (size_t)elems * (precision == UNIFRAC_FP64 ? 8 : 4);
  return UNIFRAC_OK;
}

// Everything a run needs that is decided on the host.  Buffers are grown and
// the work list uploaded before any device work is enqueued, so the enqueue
// step issues only kernels, memsets, device-to-device copies and event
// records -- the form a CUDA graph can capture.
struct RunPlan {
  int variant, precision, layout;
  int32_t s0, s1;
  bool f64;
  enum Kind { WEIGHTED, TENSOR, LOOKUP } kind;
  int32_t kf_words = 0, n_win = 0;
  int32_t vr_words = 0;  // positions from 32 vr_words on are listed per branch (if < K)
  int32_t k_tc = 0;  // tensor-core positions (TENSOR)
  int32_t sp_parts = 1;  // parts of each tile pair's sparse sums (WEIGHTED)
  bool shares_gpu = false;  // runs beside the other variant on a second stream
  void *dst = nullptr;
  int32_t n_items = 0;
};

// Parts per tile pair of the weighted sparse kernel (one CTA per SM): the
// fewest that fill the last wave of tile pairs x parts, each part costing
// about 1% extra (its own accumulator set-up and partial sums).
static int32_t sparse_parts(int32_t n_items, int sms) {
  if (n_items <= 0 || sms <= 0) return 1;
  int32_t best = 1;
  double best_t = 1e300;
  for (int32_t p = 1; p <= kMaxSparseParts; ++p) {
    const double waves = std::ceil((double)n_items * p / sms);
    const double t = waves / p * (1.0 + 0.01 * p);
    if (t < best_t - 1e-9) {
      best_t = t;
      best = p;
    }
  }
  return best;
}

static int plan_items(unifrac_ctx *ctx, int layout, int32_t s0, int32_t s1) {
  // the work list depends only on (layout, stripe range): rebuild when it changes
  if (ctx->items_valid && ctx->items_layout == layout && ctx->items_s0 == s0 &&
      ctx->items_s1 == s1)
    return UNIFRAC_OK;
  std::vector<WorkItem> items;
  std::vector<StudyDev> studies(ctx->n_studies);
  int64_t off = 0;
  for (int32_t s = 0; s < ctx->n_studies; ++s) {
    const int32_t n = ctx->study_off[s + 1] - ctx->study_off[s];
    studies[s] = StudyDev{off, n, ctx->study_col0[s]};
    off += n_pairs_layout(layout, n, s0, s1);
  }
  // items of the largest studies first (their tile pairs are full, the small
  // studies' partial ones fill the last wave); outputs are placed by study,
  // so the order changes nothing else
  std::vector<int32_t> order(ctx->n_studies);
  for (int32_t s = 0; s < ctx->n_studies; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return ctx->study_off[a + 1] - ctx->study_off[a] > ctx->study_off[b + 1] - ctx->study_off[b];
  });
  for (int32_t s : order)
    study_items(s, ctx->study_off[s + 1] - ctx->study_off[s], ctx->study_col0[s] / TILE, layout,
                s0, s1, items);
  int rc;
  if ((rc = grow(ctx, ctx->items, items.size() * sizeof(WorkItem)))) return rc;
  if ((rc = grow(ctx, ctx->studies, studies.size() * sizeof(StudyDev)))) return rc;
  // the work item of each (row tile, column tile), for the per-branch pairs
  // of the very rarely present positions
  std::vector<int32_t> item_of((size_t)ctx->n_tiles * ctx->n_tiles, -1);
  for (size_t x = 0; x < items.size(); ++x)
    item_of[(size_t)items[x].tile_i * ctx->n_tiles + items[x].tile_j] = (int32_t)x;
  if ((rc = grow(ctx, ctx->item_of, std::max<size_t>(item_of.size(), 1) * sizeof(int32_t)))) return rc;
  // per row tile, the runs of column tiles with a work item: at most two
  // (a stripe range gives a band and its wrapped part), else the whole row
  std::vector<int4> jrange((size_t)ctx->n_tiles, make_int4(0, 0, 0, 0));
  for (int32_t r = 0; r < ctx->n_tiles; ++r) {
    const int32_t *row = item_of.data() + (size_t)r * ctx->n_tiles;
    int32_t runs[4] = {0, 0, 0, 0}, n_runs = 0;
    for (int32_t c = 0; c < ctx->n_tiles;) {
      if (row[c] < 0) { ++c; continue; }
      int32_t d = c;
      while (d < ctx->n_tiles && row[d] >= 0) ++d;
      if (n_runs < 2) { runs[2 * n_runs] = c; runs[2 * n_runs + 1] = d; }
      ++n_runs;
      c = d;
    }
    jrange[(size_t)r] = n_runs <= 2 ? make_int4(runs[0], runs[1], runs[2], runs[3])
                                    : make_int4(0, ctx->n_tiles, 0, 0);
  }
  if ((rc = grow(ctx, ctx->jrange, std::max<size_t>(jrange.size(), 1) * sizeof(int4)))) return rc;
  cudaError_t e;
  if (!items.empty()) {
    e = cudaMemcpyAsync(ctx->items.p, items.data(), items.size() * sizeof(WorkItem),
                        cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upload work items");
  }
  e = cudaMemcpyAsync(ctx->studies.p, studies.data(), studies.size() * sizeof(StudyDev),
                      cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "upload studies");
  if (!item_of.empty()) {
    e = cudaMemcpyAsync(ctx->item_of.p, item_of.data(), item_of.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->jrange.p, jrange.data(), jrange.size() * sizeof(int4),
                          cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upload item table");
  }
  // pageable sources: the copies above are staged before returning
  ctx->n_items = (int32_t)items.size();
  ctx->h_items = std::move(items);
  ctx->items_valid = true;
  ctx->items_layout = layout;
  ctx->items_s0 = s0;
  ctx->items_s1 = s1;
  return UNIFRAC_OK;
}

// The sparse range [32 kf_words, K) splits at 32 vr_words: positions present
// in at most the variant's rare-list bound of samples (all studies; they are last, positions go
// by presence count descending) from the first such word on are listed per
// branch.  Grows the lists and uploads their offsets (prefix sums of the
// presence counts) when the split moved.  Returns the entries listed.
static int plan_lists(unifrac_ctx *ctx, RunPlan &P, VarBufs &V, size_t entry_bytes) {
  const int32_t k_words = (ctx->K + WORD - 1) / WORD;
  P.vr_words = k_words;
  const int64_t bound = ctx->opt_rare_list[P.variant == UNIFRAC_WEIGHTED_NORMALIZED ? 1 : 0];
  if (bound > 0) {
    int32_t pv = ctx->K;
    while (pv > P.kf_words * WORD && ctx->nb_perm[pv - 1] <= bound) --pv;
    P.vr_words = std::max(P.kf_words, (pv + WORD - 1) / WORD);
  }
  const int32_t p_list = P.vr_words * WORD;
  if (p_list >= ctx->K) return UNIFRAC_OK;
  std::vector<long long> voff((size_t)(ctx->K - p_list) + 1, 0);
  for (int32_t k = p_list; k < ctx->K; ++k)
    voff[(size_t)(k - p_list) + 1] = voff[(size_t)(k - p_list)] + ctx->nb_perm[k];
  if (voff.back() >= (1ll << 32)) {  // records hold 32-bit entry indices: no lists
    P.vr_words = k_words;
    return UNIFRAC_OK;
  }
  int rc;
  const int64_t old_bytes = (int64_t)V.voff.bytes;
  const size_t n_ent = std::max<size_t>((size_t)voff.back(), 1);
  V.list_entries = (unsigned long long)voff.back();
  if ((rc = grow(ctx, V.vlist, n_ent * entry_bytes))) return rc;
  if ((rc = grow(ctx, V.trec, n_ent * 8))) return rc;
  // per tile: record offsets (u64, n_tiles + 1), counts and cursors (u32)
  if ((rc = grow(ctx, V.tidx, ((size_t)ctx->n_tiles + 1) * 8 + (size_t)ctx->n_tiles * 8))) return rc;
  if ((rc = grow(ctx, V.voff, voff.size() * sizeof(long long)))) return rc;
  if (V.voff_pv != p_list || (int64_t)V.voff.bytes != old_bytes) {
    // on the context's stream, after earlier work that may read the old
    // offsets (a pageable source: staged before the call returns)
    cudaError_t e = cudaMemcpyAsync(V.voff.p, voff.data(), voff.size() * sizeof(long long),
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upload list offsets");
    V.voff_pv = p_list;
  }
  return UNIFRAC_OK;
}

// Grow every buffer the plan touches (may synchronise / allocate).
static int plan_buffers(unifrac_ctx *ctx, RunPlan &P) {
  int rc;
  VarBufs &V = ctx->vb[P.variant];
  // counts only where a node has some in a column tile (the create-time slots)
  if ((rc = grow(ctx, ctx->cnt, (size_t)std::max<int64_t>(ctx->n_slots, 1) * TILE * sizeof(uint32_t))))
    return rc;
  if ((rc = grow(ctx, ctx->flag, (size_t)ctx->n_nodes * ctx->n_tiles))) return rc;
  if (P.kind == RunPlan::WEIGHTED) {
    const size_t elem = P.f64 ? 8 : 4;
    const int32_t n_words = ctx->K_pad / WORD;
    if ((rc = grow(ctx, V.bits, (size_t)ctx->n_tiles * n_words * 4))) return rc;
    if ((rc = grow(ctx, V.persample, (size_t)ctx->n_cols * 8))) return rc;
    P.kf_words = n_words;
    if (!P.f64 && ctx->opt_sparse_threshold != 0) {
      // dense / sparse split at a multiple of 32 positions (FP32 form only)
      const int64_t th = ctx->opt_sparse_threshold > 0
                             ? ctx->opt_sparse_threshold
                             : std::max<int64_t>(32, ctx->max_study_n / 4);
      int32_t kf = 0;
      while (kf < ctx->K && ctx->nb_perm[kf] >= th) ++kf;
      P.kf_words = kf / WORD;
    }
    P.vr_words = (ctx->K + WORD - 1) / WORD;
    const bool has_sparse = P.kf_words < n_words && P.kf_words * WORD < ctx->K;
    if (has_sparse && (rc = plan_lists(ctx, P, V, 8))) return rc;
    P.n_win = (P.vr_words - P.kf_words + kWinWordsHost - 1) / kWinWordsHost;
    if (!has_sparse) P.n_win = (n_words - P.kf_words + kWinWordsHost - 1) / kWinWordsHost;
    const bool listed = P.vr_words * WORD < ctx->K;
    // dense values for the positions below the split only (all of them when
    // there is no sparse part)
    const size_t dense_rows =
        (P.n_win > 0 || listed) ? (size_t)P.kf_words * WORD : (size_t)ctx->K_pad;
    if ((rc = grow(ctx, V.vals, std::max<size_t>(dense_rows, 1) * ctx->n_cols * elem))) return rc;
    if (P.n_win > 0 || listed) {
      // upper bound of the sparse blocks: every sample is in one tile, so a
      // branch has at most n_b entries and min(n_b, tiles) flagged rows
      uint64_t rows = 0, ents = 0;
      for (int32_t k = P.kf_words * WORD; k < std::min(ctx->K, P.vr_words * WORD); ++k) {
        rows += (uint64_t)std::min<int64_t>(ctx->nb_perm[k], ctx->n_tiles);
        ents += (uint64_t)ctx->nb_perm[k];
      }
      // per block: 16-byte header, rowstart, two 16-byte alignments (<= 80 in
      // all); 8 bytes per (value, row) entry
      const uint64_t nblk = (uint64_t)ctx->n_tiles * P.n_win;
      const uint64_t bound = nblk * 80 + 4 * rows + 8 * ents + 64;
      if ((rc = grow(ctx, V.rc, (size_t)ctx->n_tiles * ctx->K_pad))) return rc;
      if ((rc = grow(ctx, V.bsize, nblk * 4))) return rc;
      if ((rc = grow(ctx, V.cpre, nblk * (kRareWin / WORD + 1) * 8))) return rc;
      if ((rc = grow(ctx, V.boff, (nblk + 1) * 8))) return rc;
      if ((rc = grow(ctx, V.blocks, bound))) return rc;
      // beside the other variant, whose kernels fill the last wave anyway,
      // parts would only add their fixed costs
      P.sp_parts = P.shares_gpu ? 1 : sparse_parts(P.n_items, ctx->sm_count);
      if ((rc = grow(ctx, V.spart, (size_t)std::max(P.n_items, 1) * P.sp_parts * TILE * TILE * 4)))
        return rc;
    }
  } else if (P.kind == RunPlan::TENSOR) {
    // positions [0, k_tc) on the tensor cores, the rarely present rest sparse
    int64_t th = ctx->opt_uw_sparse_threshold;
    if (th < 0)  // split once the operands grow large (many samples in total)
      th = ctx->n_cols > 8192 ? std::max<int64_t>(32, ctx->max_study_n / 16) : 0;
    int32_t kf = ctx->K;
    if (th > 0) {
      kf = 0;
      while (kf < ctx->K && ctx->nb_perm[kf] >= th) ++kf;
    }
    P.k_tc = std::min<int32_t>(ctx->K_pad, std::max<int32_t>(64, (kf + 63) / 64 * 64));
    // the sparse kernel sums 12-bit halves of q in 32-bit counters: exact
    // while fewer than 2^20 positions are sparse
    constexpr int32_t kMaxSparsePositions = (1 << 20) - 64;
    if (ctx->K - P.k_tc > kMaxSparsePositions)
      P.k_tc = std::min<int32_t>(ctx->K_pad, (ctx->K - kMaxSparsePositions + 63) / 64 * 64);
    const int32_t n_words = ctx->K_pad / WORD;
    P.kf_words = P.k_tc / WORD;
    P.vr_words = (ctx->K + WORD - 1) / WORD;
    if (P.k_tc < ctx->K && (rc = plan_lists(ctx, P, V, 8))) return rc;
    const bool listed = P.vr_words * WORD < ctx->K;
    P.n_win = P.k_tc >= ctx->K ? 0 : (P.vr_words - P.kf_words + kWinWordsHost - 1) / kWinWordsHost;
    (void)n_words;
    const int32_t n_kt = P.k_tc / 64;
    const int32_t k_words = (n_kt + 31) / 32;
    const size_t plane = (size_t)ctx->n_cols * P.k_tc * 2;
    if ((rc = grow(ctx, V.vals, plane))) return rc;
    if ((rc = grow(ctx, V.vals2, 3 * plane))) return rc;
    if ((rc = grow(ctx, V.bits, (size_t)ctx->n_tiles * k_words * 4))) return rc;
    if ((rc = grow(ctx, V.partial, (size_t)ctx->n_cols * 8))) return rc;
    if ((rc = grow(ctx, V.persample, (size_t)ctx->n_cols * 8))) return rc;
    if (P.n_win > 0 || listed) {
      uint64_t rows = 0, ents = 0;
      for (int32_t k = P.kf_words * WORD; k < std::min(ctx->K, P.vr_words * WORD); ++k) {
        rows += (uint64_t)std::min<int64_t>(ctx->nb_perm[k], ctx->n_tiles);
        ents += (uint64_t)ctx->nb_perm[k];
      }
      // per block: 16-byte header, rowstart, two 16-byte alignments (<= 80 in
      // all); 1 byte per row entry
      const uint64_t nblk = (uint64_t)ctx->n_tiles * P.n_win;
      const uint64_t bound = nblk * 80 + 4 * rows + ents + 64;
      if ((rc = grow(ctx, V.rbits, (size_t)ctx->n_tiles * n_words * 4))) return rc;
      if ((rc = grow(ctx, V.rc, (size_t)ctx->n_tiles * ctx->K_pad))) return rc;
      if ((rc = grow(ctx, V.bsize, nblk * 4))) return rc;
      if ((rc = grow(ctx, V.cpre, nblk * (kRareWin / WORD + 1) * 8))) return rc;
      if ((rc = grow(ctx, V.boff, (nblk + 1) * 8))) return rc;
      if ((rc = grow(ctx, V.blocks, bound))) return rc;
      if ((rc = grow(ctx, V.spart, (size_t)std::max(P.n_items, 1) * TILE * TILE * 8))) return rc;
    }
  } else {
    const int32_t G = ctx->K_pad / 8;
    const int32_t g_words = (G + WORD - 1) / WORD;
    if ((rc = grow(ctx, V.vals, (size_t)G * ctx->n_cols))) return rc;
    if ((rc = grow(ctx, ctx->tables, (size_t)G * 256 * 8))) return rc;
    if ((rc = grow(ctx, V.bits, (size_t)ctx->n_tiles * g_words * 4))) return rc;
    if ((rc = grow(ctx, V.partial, (size_t)((G + 31) / 32) * ctx->n_cols * 8))) return rc;
    if ((rc = grow(ctx, V.persample, (size_t)ctx->n_cols * 8))) return rc;
  }
  return UNIFRAC_OK;
}

static ListBufs list_bufs(const unifrac_ctx *ctx, VarBufs &V) {
  ListBufs L;
  L.ents = static_cast<unsigned long long *>(V.vlist.p);
  L.trec = static_cast<uint2 *>(V.trec.p);
  char *ti = static_cast<char *>(V.tidx.p);
  L.toff = reinterpret_cast<unsigned long long *>(ti);
  L.tcnt = reinterpret_cast<uint32_t *>(ti + ((size_t)ctx->n_tiles + 1) * 8);
  L.tcur = L.tcnt + ctx->n_tiles;
  L.n_ent = V.list_entries;
  return L;
}

// Device work of one variant after the embedding (no allocation, no host copy,
// no sync).
static int enqueue_variant(unifrac_ctx *ctx, const RunPlan &P, bool overlapped) {
  int rc;
  ctx->cur_slot = P.variant;
  VarBufs &V = ctx->vb[P.variant];
  cudaError_t e =
      cudaMemsetAsync(cur_counters(ctx), 0, 4 * sizeof(unsigned long long), ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(ctx->d_counter + 4 * ctx->cur_slot, 0, 4 * sizeof(unsigned long long),
                        ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reset counters");
  OutSpec o;
  o.out = P.dst;
  o.studies = static_cast<const StudyDev *>(ctx->studies.p);
  o.layout = P.layout;
  o.s0 = P.s0;
  o.s1 = P.s1;
  o.is_f64 = P.f64 ? 1 : 0;
  uint32_t *cnt = static_cast<uint32_t *>(ctx->cnt.p);
  uint8_t *flag = static_cast<uint8_t *>(ctx->flag.p);
  const WorkItem *d_items = static_cast<const WorkItem *>(ctx->items.p);
  const int32_t n_items = P.n_items;
  const int variant = P.variant;
  if (P.kind == RunPlan::WEIGHTED) {
    const double *S = ctx->d_S;
    uint32_t *bits = static_cast<uint32_t *>(V.bits.p);
    // dense values for the frequently present positions, sparse blocks built
    // from the counts for the rest
    // positions [32 vr_words, K) are listed per branch
    const bool listed = !P.f64 && P.vr_words * WORD < ctx->K;
    const bool sparse = P.n_win > 0 || listed;
    const int32_t k_end = sparse ? P.kf_words * WORD : ctx->K;
    if (!ctx->reuse_prepared &&
        (rc = pack_weighted(ctx, cnt, flag, P.f64, V.vals.p, bits, k_end)))
      return rc;
    if (sparse && !ctx->reuse_prepared) {
      uint8_t *rcb = static_cast<uint8_t *>(V.rc.p);
      if ((rc = pack_rare(ctx, cnt, flag, P.kf_words, bits, rcb, nullptr))) return rc;
      if (P.n_win > 0 &&
          (rc = build_rare_blocks(ctx, true, cnt, bits, rcb, P.kf_words,
                                  std::min(ctx->K, P.vr_words * WORD), P.n_win,
                                  static_cast<uint32_t *>(V.bsize.p),
                                  static_cast<unsigned long long *>(V.boff.p),
                                  static_cast<uint2 *>(V.cpre.p),
                                  static_cast<uint8_t *>(V.blocks.p))))
        return rc;
      if (listed &&
          (rc = list_fill(ctx, true, cnt, flag, bits, rcb, P.vr_words * WORD,
                          static_cast<const long long *>(V.voff.p), list_bufs(ctx, V))))
        return rc;
    }
    if (!overlapped) record_event(ctx, ctx->ev[1]);
    record_event(ctx, ctx->ev_pair[variant][0]);
    ctx->sel_unit = 1.0;
    if ((rc = pairs_weighted(ctx, P.f64, V.vals.p, bits, P.kf_words, P.vr_words,
                             static_cast<const uint8_t *>(V.blocks.p),
                             static_cast<const unsigned long long *>(V.boff.p),
                             static_cast<const uint2 *>(V.cpre.p), P.n_win,
                             listed ? list_bufs(ctx, V) : ListBufs(),
                             sparse ? static_cast<uint32_t *>(V.spart.p) : nullptr,
                             P.sp_parts, S, d_items, n_items, o)))
      return rc;
  } else if (P.kind == RunPlan::TENSOR) {
    uint16_t *X = static_cast<uint16_t *>(V.vals.p);
    uint16_t *D = static_cast<uint16_t *>(V.vals2.p);
    uint32_t *kbits = static_cast<uint32_t *>(V.bits.p);
    double *a = static_cast<double *>(V.persample.p);
    unsigned long long *aq = static_cast<unsigned long long *>(V.partial.p);
    const bool listed = P.vr_words * WORD < ctx->K && P.k_tc < ctx->K;
    const bool sparse = P.n_win > 0 || listed;
    unsigned long long *spart = sparse ? static_cast<unsigned long long *>(V.spart.p) : nullptr;
    if (!ctx->reuse_prepared) {
      e = cudaMemsetAsync(aq, 0, (size_t)ctx->n_cols * 8, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "clear per-sample sums");
      if ((rc = pack_tc(ctx, cnt, flag, P.k_tc, X, D, kbits, aq))) return rc;
      if (sparse) {
        uint32_t *rbits = static_cast<uint32_t *>(V.rbits.p);
        uint8_t *rcb = static_cast<uint8_t *>(V.rc.p);
        // presence sums a_col over every sparse position, listed ones included
        if ((rc = pack_rare(ctx, cnt, flag, P.kf_words, rbits, rcb, aq))) return rc;
        if (P.n_win > 0 &&
            (rc = build_rare_blocks(ctx, false, cnt, rbits, rcb, P.kf_words,
                                    std::min(ctx->K, P.vr_words * WORD), P.n_win,
                                    static_cast<uint32_t *>(V.bsize.p),
                                    static_cast<unsigned long long *>(V.boff.p),
                                    static_cast<uint2 *>(V.cpre.p),
                                    static_cast<uint8_t *>(V.blocks.p))))
          return rc;
        if (listed &&
            (rc = list_fill(ctx, false, cnt, flag, rbits, rcb, P.vr_words * WORD,
                            static_cast<const long long *>(V.voff.p), list_bufs(ctx, V))))
          return rc;
      }
      if ((rc = finish_tc_a(ctx, aq, a))) return rc;
    }
    if (!overlapped) record_event(ctx, ctx->ev[1]);
    record_event(ctx, ctx->ev_pair[variant][0]);
    ctx->sel_unit = 64.0;
    record_event(ctx, ctx->ev_sp[0][0]);
    if (!spart) {  // an empty list phase
      record_event(ctx, ctx->ev_list[0][0]);
      record_event(ctx, ctx->ev_list[0][1]);
    }
    if (spart &&
        (rc = pairs_sparse_presence(ctx, static_cast<const uint32_t *>(V.rbits.p), P.kf_words,
                                    P.vr_words, static_cast<const uint8_t *>(V.blocks.p),
                                    static_cast<const unsigned long long *>(V.boff.p),
                                    static_cast<const uint2 *>(V.cpre.p), P.n_win,
                                    listed ? list_bufs(ctx, V) : ListBufs(), spart, d_items,
                                    n_items)))
      return rc;
    record_event(ctx, ctx->ev_sp[0][1]);
    if ((rc = pairs_tc(ctx, P.k_tc, X, D, kbits, aq, spart, d_items, n_items, o))) return rc;
  } else {
    double *a = static_cast<double *>(V.persample.p);
    uint8_t *bytes = static_cast<uint8_t *>(V.vals.p);
    double *tables = static_cast<double *>(ctx->tables.p);
    uint32_t *gbits = static_cast<uint32_t *>(V.bits.p);
    if (!ctx->reuse_prepared && (rc = pack_lookup(ctx, cnt, flag, bytes, tables, gbits, a)))
      return rc;
    if (!overlapped) record_event(ctx, ctx->ev[1]);
    record_event(ctx, ctx->ev_pair[variant][0]);
    ctx->sel_unit = 8.0;
    if ((rc = pairs_lookup(ctx, bytes, tables, gbits, a, d_items, n_items, o))) return rc;
  }
  if (!overlapped) record_event(ctx, ctx->ev[2]);
  record_event(ctx, ctx->ev_pair[variant][1]);
  ctx->sel_unit_v[variant] = ctx->sel_unit;
  return UNIFRAC_OK;
}

// The first result's copy to host memory, ordered after its kernels on the
// context's (current) stream, run on the copy stream (see
// unifrac_ctx::early_host).
static int enqueue_early_copy(unifrac_ctx *ctx) {
  if (!ctx->early_host) return UNIFRAC_OK;
  cudaError_t e = cudaEventRecord(ctx->ev_first_done, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_first_done, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->early_host, ctx->early_dev, ctx->early_bytes, cudaMemcpyDeviceToHost,
                        ctx->copy_stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy first result to host");
  return UNIFRAC_OK;
}

// The embedding once, then each variant's packing and pair kernels.
// With two plans and UNIFRAC_OPT_OVERLAP_VARIANTS, the first plan runs on a
// second stream forked after the embedding and joined at the end, the
// second on the context's stream (both are captured into the same
// graph); the variants have separate buffers and counters, and share only the
// read-only embedding and the output buffer, which they write in disjoint
// halves.
static int enqueue_run(unifrac_ctx *ctx, const RunPlan *plans, int n_plans) {
  int rc;
  record_event(ctx, ctx->ev[0]);
  if (!ctx->reuse_prepared &&
      (rc = embed_counts(ctx, static_cast<uint32_t *>(ctx->cnt.p),
                         static_cast<uint8_t *>(ctx->flag.p))))
    return rc;
  const bool overlap = n_plans == 2 && ctx->opt_overlap;
  if (!overlap) {
    for (int i = 0; i < n_plans; ++i) {
      if ((rc = enqueue_variant(ctx, plans[i], false))) return rc;
      if (i == 0 && (rc = enqueue_early_copy(ctx))) return rc;
    }
    return UNIFRAC_OK;
  }
  cudaError_t e = cudaSuccess;
  // The first plan (the unweighted variant of UNIFRAC_BOTH, the shorter) runs
  // on the second stream.  When its result is copied to host memory while the
  // second plan computes, that stream has the highest priority, so that the
  // first plan finishes early and the copy hides behind the second.  Otherwise
  // both streams have the same priority: the hardware then fills each
  // variant's idle tails with the other's blocks, which a priority order
  // prevents (about 20 ms of 820 on the 50,000-sample matrix).
  const int pri = ctx->early_host ? 1 : 0;
  if (!ctx->stream2[pri]) {
    int lo_pri = 0, hi_pri = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri);
    if (e == cudaSuccess)
      e = cudaStreamCreateWithPriority(&ctx->stream2[pri], cudaStreamNonBlocking,
                                       pri ? hi_pri : lo_pri);
  }
  if (e == cudaSuccess && !ctx->ev_fork2) e = cudaEventCreateWithFlags(&ctx->ev_fork2, cudaEventDisableTiming);
  if (e == cudaSuccess && !ctx->ev_join2) e = cudaEventCreateWithFlags(&ctx->ev_join2, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "second stream");
  cudaStream_t s2 = ctx->stream2[pri];
  record_event(ctx, ctx->ev[1]);  // the embedding alone
  e = cudaEventRecord(ctx->ev_fork2, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, ctx->ev_fork2, 0);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fork");
  cudaStream_t main_stream = ctx->stream;
  ctx->stream = s2;
  rc = enqueue_variant(ctx, plans[0], true);
  if (!rc) rc = enqueue_early_copy(ctx);
  ctx->stream = main_stream;
  if (!rc) rc = enqueue_variant(ctx, plans[1], true);
  e = cudaEventRecord(ctx->ev_join2, s2);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join2, 0);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "join");
  if (rc) return rc;
  record_event(ctx, ctx->ev[2]);
  return UNIFRAC_OK;
}

// Graph replay of a captured run.  The legacy default stream cannot be
// captured, so capture and replay use the context's private stream, ordered
// after / before the caller's stream with events.
static int graph_key_matches(const unifrac_ctx *ctx, const RunPlan &P, int variant_arg) {
  return ctx->graph_exec && ctx->gk_variant == variant_arg && ctx->gk_precision == P.precision &&
         ctx->gk_layout == P.layout && ctx->gk_s0 == P.s0 && ctx->gk_s1 == P.s1 &&
         ctx->gk_dst == P.dst && ctx->gk_opts == ctx->opt_generation &&
         ctx->gk_bufs == ctx->buf_generation;
}

static int graph_launch(unifrac_ctx *ctx) {
  cudaError_t e = cudaEventRecord(ctx->ev_fork, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cap_stream, ctx->ev_fork, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(ctx->graph_exec, ctx->cap_stream);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_join, ctx->cap_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
  return UNIFRAC_OK;
}

static int graph_capture(unifrac_ctx *ctx, const RunPlan *plans, int n_plans, int variant_arg) {
  const RunPlan &P = plans[0];
  cudaError_t e;
  if (!ctx->cap_stream) {
    e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph stream");
  }
  if (ctx->graph_exec) {
    cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
  }
  cudaStream_t user = ctx->stream;
  const double launches = ctx->stat_launches;
  ctx->stream = ctx->cap_stream;
  e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
  int rc = UNIFRAC_OK;
  ctx->capturing = true;
  if (e == cudaSuccess) rc = enqueue_run(ctx, plans, n_plans);
  ctx->capturing = false;
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &graph);
  ctx->stream = user;
  ctx->stat_launches = launches;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "begin capture");
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "end capture");
  e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    ctx->graph_exec = nullptr;
    return cuda_fail(ctx, e, "graph instantiate");
  }
  ctx->gk_variant = variant_arg;
  ctx->gk_precision = P.precision;
  ctx->gk_layout = P.layout;
  ctx->gk_s0 = P.s0;
  ctx->gk_s1 = P.s1;
  ctx->gk_dst = P.dst;
  ctx->gk_opts = ctx->opt_generation;
  ctx->gk_bufs = ctx->buf_generation;
  return UNIFRAC_OK;
}

extern "C++" {
namespace ufb {
int enqueue_range_copy(unifrac_ctx *ctx, int c) {
  cudaStream_t cs = ctx->copy_stream;
  cudaError_t e = cudaEventRecord(ctx->cc_ev[(size_t)c], ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->cc_ev[(size_t)c], 0);
  const int64_t n = ctx->cc_samples;
  const int64_t r0 = std::min<int64_t>(n, (int64_t)ctx->cc_tiles[(size_t)c] * TILE);
  const int64_t r1 = std::min<int64_t>(n, (int64_t)ctx->cc_tiles[(size_t)c + 1] * TILE);
  const size_t el = ctx->cc_elem;
  if (e == cudaSuccess && r1 > r0) {
    if (ctx->cc_layout == UNIFRAC_OUT_FULL) {
      // rows [r0, r1) from column r0 on, and their mirror: rows [r1, n) of
      // columns [r0, r1); the columns before r0 came with earlier ranges
      const size_t pitch = (size_t)n * el, at = ((size_t)r0 * n + r0) * el;
      e = cudaMemcpy2DAsync(ctx->cc_host + at, pitch, ctx->cc_dev + at, pitch,
                            (size_t)(n - r0) * el, (size_t)(r1 - r0), cudaMemcpyDeviceToHost, cs);
      if (e == cudaSuccess && n > r1) {
        const size_t at2 = ((size_t)r1 * n + r0) * el;
        e = cudaMemcpy2DAsync(ctx->cc_host + at2, pitch, ctx->cc_dev + at2, pitch,
                              (size_t)(r1 - r0) * el, (size_t)(n - r1), cudaMemcpyDeviceToHost, cs);
      }
    } else {  // condensed: row i of the upper triangle starts at i n - i (i + 1) / 2
      auto row_at = [n](int64_t i) { return (size_t)(i * n - i * (i + 1) / 2); };
      const size_t a = row_at(r0), b = row_at(r1);
      if (b > a)
        e = cudaMemcpyAsync(ctx->cc_host + a * el, ctx->cc_dev + a * el, (b - a) * el,
                            cudaMemcpyDeviceToHost, cs);
    }
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy a row range to host");
  return UNIFRAC_OK;
}
}  // namespace ufb
}  // extern "C++"

// The item ranges of a chunked host copy.  A range may end before item x
// when no item from x on has a smaller row tile than item x (then every tile
// row above item x's is complete once the items before x are done); the
// work list goes by block rows of tiles, so these cuts are the starts of its
// block rows.  Of them, those nearest to equal shares of the items.
static void plan_copy_ranges(unifrac_ctx *ctx, int ranges) {
  ctx->cc_items.assign(1, 0);
  ctx->cc_tiles.assign(1, 0);
  const std::vector<WorkItem> &it = ctx->h_items;
  const int64_t n = (int64_t)it.size();
  std::vector<int32_t> suffix_min((size_t)n + 1, INT32_MAX);
  for (int64_t x = n - 1; x >= 0; --x)
    suffix_min[(size_t)x] = std::min(suffix_min[(size_t)x + 1], it[(size_t)x].tile_i);
  std::vector<int32_t> cuts;  // valid cuts, ascending
  for (int64_t x = 1; x < n; ++x)
    if (it[(size_t)x].tile_i > it[(size_t)x - 1].tile_i && suffix_min[(size_t)x] == it[(size_t)x].tile_i)
      cuts.push_back((int32_t)x);
  const int32_t tile0 = ctx->study_col0[0] / TILE;
  size_t v = 0;
  for (int c = 1; c < ranges && v < cuts.size(); ++c) {
    const int64_t target = (int64_t)c * n / ranges;
    while (v + 1 < cuts.size() && cuts[v + 1] <= target) ++v;
    // the nearer of the cuts around the target
    size_t pick = v;
    if (v + 1 < cuts.size() && cuts[v + 1] - target < target - cuts[v]) pick = v + 1;
    const int32_t x = cuts[pick];
    if (x <= ctx->cc_items.back()) continue;
    ctx->cc_items.push_back(x);
    ctx->cc_tiles.push_back(it[(size_t)x].tile_i - tile0);
  }
  ctx->cc_items.push_back((int32_t)n);
  ctx->cc_tiles.push_back((int32_t)((ctx->cc_samples + TILE - 1) / TILE));
  ctx->cc_n = (int)ctx->cc_items.size() - 1;
}

// Addresses and sizes of the buffers a run prepares before its pair kernels
// (the embedding and every variant's packed operands): equal signatures mean
// none of them was reallocated since.
static uint64_t prep_signature(const unifrac_ctx *ctx) {
  uint64_t h = 1469598103934665603ull;  // FNV-1a over (address, size) pairs
  auto mix = [&](const ufb::DevBuf &b) {
    h = (h ^ (uint64_t)(uintptr_t)b.p) * 1099511628211ull;
    h = (h ^ (uint64_t)b.bytes) * 1099511628211ull;
  };
  mix(ctx->cnt);
  mix(ctx->flag);
  mix(ctx->tables);
  for (const ufb::VarBufs &V : ctx->vb)
    for (const ufb::DevBuf *b : {&V.vals, &V.vals2, &V.bits, &V.persample, &V.partial, &V.rc, &V.bsize,
                                 &V.boff, &V.blocks, &V.cpre, &V.rbits, &V.vlist, &V.voff,
                                 &V.trec, &V.tidx})
      mix(*b);
  return h;
}

static int run_impl(unifrac_ctx *ctx, int variant, int precision, int32_t stripe_start,
                    int32_t stripe_stop, int layout, void *out, size_t out_bytes) {
  if (variant != UNIFRAC_UNWEIGHTED && variant != UNIFRAC_WEIGHTED_NORMALIZED &&
      variant != UNIFRAC_BOTH)
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "variant");
  if (precision != UNIFRAC_FP64 && precision != UNIFRAC_MIXED)
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "precision");
  if (layout < UNIFRAC_OUT_STRIPES || layout > UNIFRAC_OUT_FULL)
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "layout");
  const int n_plans = variant == UNIFRAC_BOTH ? 2 : 1;
  int32_t s0, s1;
  int rc = resolve_range(ctx, layout, stripe_start, stripe_stop, &s0, &s1);
  if (rc == UNIFRAC_E_UNSUPPORTED)
    return fail(ctx, rc, "several studies need layout CONDENSED or FULL and the range (0, -1)");
  if (rc) return fail(ctx, rc, "stripe range");
  size_t one = 0;
  unifrac_output_bytes(ctx, precision, layout, stripe_start, stripe_stop, &one);
  const size_t need = one * n_plans;
  if (need > 0 && !out) return fail(ctx, UNIFRAC_E_INVALID_ARG, "out is NULL");
  if (out_bytes < need)
    return fail(ctx, UNIFRAC_E_BUFFER_TOO_SMALL,
                "out holds " + std::to_string(out_bytes) + " bytes, needs " + std::to_string(need));
  RunPlan plans[2];
  for (int i = 0; i < n_plans; ++i) {
    RunPlan &P = plans[i];
    P.variant = variant == UNIFRAC_BOTH ? i : variant;
    P.precision = precision;
    P.layout = layout;
    P.s0 = s0;
    P.s1 = s1;
    P.f64 = precision == UNIFRAC_FP64;
    if (P.variant == UNIFRAC_WEIGHTED_NORMALIZED)
      P.kind = RunPlan::WEIGHTED;
    else if (!P.f64 && ctx->opt_uw_kernel != 2 && ctx->max_reach < 65793)
      // tensor-core Gram: exact while every plane sum stays below 2^24, i.e.
      // while no sample reaches 65,793 branches (255 * 65,793 >= 2^24)
      P.kind = RunPlan::TENSOR;
    else
      P.kind = RunPlan::LOOKUP;
  }
  RunPlan &P = plans[0];

  // where does `out` live?
  bool device_out = false, pinned_out = false;
  if (need > 0) {
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, out);
    if (e != cudaSuccess) {
      cudaGetLastError();
      attr.type = cudaMemoryTypeUnregistered;
    }
    device_out = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
    pinned_out = attr.type == cudaMemoryTypeHost;
  }
  const bool whole = (layout == UNIFRAC_OUT_STRIPES) ||
                     (s0 == 0 && (ctx->n_studies > 1 || s1 == ctx->n_samples / 2));
  void *dst = out;
  if (!device_out && need > 0) {
    if ((rc = grow(ctx, ctx->stage, need))) return rc;
    dst = ctx->stage.p;
  }
  if ((rc = plan_items(ctx, layout, s0, s1))) return rc;
  ctx->stat_tile_pairs = (double)ctx->n_items;
  for (int i = 0; i < n_plans; ++i) {
    plans[i].dst = static_cast<char *>(dst) + (size_t)i * one;
    plans[i].n_items = ctx->n_items;
    plans[i].shares_gpu = n_plans == 2 && ctx->opt_overlap;
    if ((rc = plan_buffers(ctx, plans[i]))) return rc;
  }
  if (ctx->reuse_prepared && prep_signature(ctx) != ctx->prep_sig) ctx->reuse_prepared = false;
  if (!device_out && need > 0 && !whole) {  // untouched elements keep the caller's values
    cudaError_t e = cudaMemcpyAsync(dst, out, need, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stage output");
  }

  const bool use_graph = ctx->opt_use_graph && device_out;
  size_t copied = 0;  // bytes of the result already on their way to host memory
  bool ranged = false;  // the last variant's bytes go out range by range
  if (use_graph && graph_key_matches(ctx, P, variant)) {
    if ((rc = graph_launch(ctx))) return rc;
    ctx->stat_launches = ctx->graph_launches;
  } else {
    ctx->stat_launches = 0;
    // into pinned host memory, the first of two results is copied while the
    // second computes
    const bool early = !device_out && pinned_out && n_plans == 2 && one > 0;
    if (early) {
      cudaError_t e = cudaSuccess;
      if (!ctx->copy_stream) e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
      if (e == cudaSuccess && !ctx->ev_first_done)
        e = cudaEventCreateWithFlags(&ctx->ev_first_done, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "copy stream");
      ctx->early_host = out;
      ctx->early_dev = dst;
      ctx->early_bytes = one;
    }
    // into pinned host memory, one study's whole matrix: the weighted
    // variant's dense kernel in ranges of rows, each range's rows copied out
    // while the next computes
    const RunPlan &last = plans[n_plans - 1];
    ranged = !device_out && pinned_out && one > 0 && ctx->opt_copy_ranges > 1 && whole &&
             ctx->n_studies == 1 && last.kind == RunPlan::WEIGHTED &&
             (layout == UNIFRAC_OUT_FULL || layout == UNIFRAC_OUT_CONDENSED);
    if (ranged) {
      cudaError_t e = cudaSuccess;
      if (!ctx->copy_stream) e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "copy stream");
      ctx->cc_samples = ctx->n_samples;
      plan_copy_ranges(ctx, ctx->opt_copy_ranges);
      while (ctx->cc_ev.size() < (size_t)ctx->cc_n) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy range events");
        ctx->cc_ev.push_back(ev);
      }
      ctx->cc_variant = last.variant;
      ctx->cc_host = static_cast<char *>(out) + (size_t)(n_plans - 1) * one;
      ctx->cc_dev = static_cast<const char *>(dst) + (size_t)(n_plans - 1) * one;
      ctx->cc_elem = precision == UNIFRAC_FP64 ? sizeof(double) : sizeof(float);
      ctx->cc_layout = layout;
    }
    rc = enqueue_run(ctx, plans, n_plans);
    ctx->early_host = nullptr;
    ctx->cc_variant = -1;
    if (rc) {
      if (early || ranged) cudaStreamSynchronize(ctx->copy_stream);
      return rc;
    }
    if (early) copied = one;
    if (use_graph) {  // this run executed eagerly; later identical runs replay the graph
      ctx->graph_launches = ctx->stat_launches;
      if ((rc = graph_capture(ctx, plans, n_plans, variant))) return rc;
    }
  }
  for (int i = 0; i < n_plans; ++i) {
    ctx->sel_unit_v[plans[i].variant] = plans[i].kind == RunPlan::WEIGHTED ? 1.0
                                        : plans[i].kind == RunPlan::TENSOR ? 64.0
                                                                           : 8.0;
    ctx->ev_pair_valid[plans[i].variant] = true;
  }
  ctx->ev_valid = true;

  cudaError_t e;
  if (!device_out && need > 0) {
    const size_t end = need - (ranged ? one : 0);  // the rest is on its way already
    if (end > copied) {
      e = cudaMemcpyAsync(static_cast<char *>(out) + copied,
                          static_cast<const char *>(dst) + copied, end - copied,
                          cudaMemcpyDeviceToHost, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "copy result to host");
    }
    e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && (copied || ranged)) e = cudaStreamSynchronize(ctx->copy_stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise");
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "run");
  return UNIFRAC_OK;
}

int unifrac_run(unifrac_ctx *ctx, int variant, int precision, int32_t stripe_start,
                int32_t stripe_stop, int layout, void *out, size_t out_bytes) {
  if (!ctx) return UNIFRAC_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, UNIFRAC_E_CUDA, "cannot select the context's device");
  try {
    return run_impl(ctx, variant, precision, stripe_start, stripe_stop, layout, out, out_bytes);
  } catch (const std::bad_alloc &) {
    return fail(ctx, UNIFRAC_E_OOM, "host allocation");
  } catch (...) {
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "unexpected failure");
  }
}

int unifrac_set_option(unifrac_ctx *ctx, int option, int64_t value) {
  if (!ctx) return UNIFRAC_E_INVALID_ARG;
  ctx->opt_generation++;  // invalidates a captured graph
  switch (option) {
    case UNIFRAC_OPT_UNWEIGHTED_MIXED_KERNEL:
      if (value < 0 || value > 2) return UNIFRAC_E_INVALID_ARG;
      ctx->opt_uw_kernel = (int)value;
      return UNIFRAC_OK;
    case UNIFRAC_OPT_WEIGHTED_FLUSH:
      if (value < 16 || value > 4096) return UNIFRAC_E_INVALID_ARG;
      ctx->opt_flush = (int)value;
      return UNIFRAC_OK;
    case UNIFRAC_OPT_USE_GRAPH:
      if (value < 0 || value > 1) return UNIFRAC_E_INVALID_ARG;
      ctx->opt_use_graph = (int)value;
      return UNIFRAC_OK;
    case UNIFRAC_OPT_OVERLAP_VARIANTS:
      if (value < 0 || value > 1) return UNIFRAC_E_INVALID_ARG;
      ctx->opt_overlap = (int)value;
      return UNIFRAC_OK;
    case UNIFRAC_OPT_SPARSE_THRESHOLD:
      if (value < -1) return UNIFRAC_E_INVALID_ARG;
      ctx->opt_sparse_threshold = value;
      return UNIFRAC_OK;
    case UNIFRAC_OPT_PERSISTENT:
      if (value < 0 || value > 1) return UNIFRAC_E_INVALID_ARG;
      ctx->opt_persistent = (int)value;
      return UNIFRAC_OK;
    case UNIFRAC_OPT_RARE_LIST:
    case UNIFRAC_OPT_UNWEIGHTED_RARE_LIST:
      if (value < 0 || value > 4096) return UNIFRAC_E_INVALID_ARG;
      ctx->opt_rare_list[option == UNIFRAC_OPT_RARE_LIST ? 1 : 0] = value;
      return UNIFRAC_OK;
    case UNIFRAC_OPT_SPARSE_LANE_PAIRS:
    case UNIFRAC_OPT_UNWEIGHTED_SPARSE_LANE_PAIRS:
      if (value < 0 || value > 4096) return UNIFRAC_E_INVALID_ARG;
      ctx->opt_lane_pairs[option == UNIFRAC_OPT_SPARSE_LANE_PAIRS ? 1 : 0] = (int)value;
      return UNIFRAC_OK;
    case UNIFRAC_OPT_UNWEIGHTED_SPARSE_THRESHOLD:
      if (value < -1) return UNIFRAC_E_INVALID_ARG;
      ctx->opt_uw_sparse_threshold = value;
      return UNIFRAC_OK;
    case UNIFRAC_OPT_COPY_RANGES:
      if (value < 1 || value > 64) return UNIFRAC_E_INVALID_ARG;
      ctx->opt_copy_ranges = (int)value;
      return UNIFRAC_OK;
    case UNIFRAC_OPT_HOST_THREADS:
      if (value < 0 || value > 256) return UNIFRAC_E_INVALID_ARG;
      ctx->opt_host_threads = (int)value;
      ctx->opt_generation--;  // host-side only: a captured graph stays valid
      return UNIFRAC_OK;
    default:
      return UNIFRAC_E_INVALID_ARG;
  }
}

int unifrac_get_option(const unifrac_ctx *ctx, int option, int64_t *value) {
  if (!ctx || !value) return UNIFRAC_E_INVALID_ARG;
  switch (option) {
    case UNIFRAC_OPT_UNWEIGHTED_MIXED_KERNEL: *value = ctx->opt_uw_kernel; return UNIFRAC_OK;
    case UNIFRAC_OPT_WEIGHTED_FLUSH: *value = ctx->opt_flush; return UNIFRAC_OK;
    case UNIFRAC_OPT_USE_GRAPH: *value = ctx->opt_use_graph; return UNIFRAC_OK;
    case UNIFRAC_OPT_OVERLAP_VARIANTS: *value = ctx->opt_overlap; return UNIFRAC_OK;
    case UNIFRAC_OPT_SPARSE_THRESHOLD: *value = ctx->opt_sparse_threshold; return UNIFRAC_OK;
    case UNIFRAC_OPT_SPARSE_LANE_PAIRS: *value = ctx->opt_lane_pairs[1]; return UNIFRAC_OK;
    case UNIFRAC_OPT_PERSISTENT: *value = ctx->opt_persistent; return UNIFRAC_OK;
    case UNIFRAC_OPT_RARE_LIST: *value = ctx->opt_rare_list[1]; return UNIFRAC_OK;
    case UNIFRAC_OPT_UNWEIGHTED_RARE_LIST: *value = ctx->opt_rare_list[0]; return UNIFRAC_OK;
    case UNIFRAC_OPT_UNWEIGHTED_SPARSE_LANE_PAIRS: *value = ctx->opt_lane_pairs[0]; return UNIFRAC_OK;
    case UNIFRAC_OPT_UNWEIGHTED_SPARSE_THRESHOLD:
      *value = ctx->opt_uw_sparse_threshold;
      return UNIFRAC_OK;
    case UNIFRAC_OPT_COPY_RANGES: *value = ctx->opt_copy_ranges; return UNIFRAC_OK;
    case UNIFRAC_OPT_HOST_THREADS: *value = ctx->opt_host_threads; return UNIFRAC_OK;
    default: return UNIFRAC_E_INVALID_ARG;
  }
}

extern "C++" namespace ufb {
// The chunk of L stripes [s0, s0 + L) (nv variants, one after the other, L x n
// elements each) rewritten as the row runs of the matrix,
// up[v][i][t] = d(i, (i + s0 + 1 + t) mod n) and
// down[v][i][t] = d(i, (i - s0 - L + t) mod n), on the context's stream
// (stripe_rows.cu).
int stripe_rows(unifrac_ctx *ctx, const void *chunk, int32_t n, int32_t L, int32_t s0, int nv,
                bool f64, void *up, void *down);
}  // namespace ufb

// Streamed output: stripes [s0, s1) per chunk into one of two device buffers
// (the kernels of the next chunk overlap the copy of this one on a copy
// stream), copied to pinned host memory and merged into the caller's
// condensed or full matrix by host threads while the GPU computes on.
static int run_streamed_impl(unifrac_ctx *ctx, int variant, int precision, int layout,
                             void *host_out, size_t out_bytes, int32_t chunk_stripes) {
  if (!host_out || chunk_stripes < 1) return fail(ctx, UNIFRAC_E_INVALID_ARG, "output / chunk");
  if (variant < UNIFRAC_UNWEIGHTED || variant > UNIFRAC_BOTH)
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "variant");
  if (precision != UNIFRAC_FP64 && precision != UNIFRAC_MIXED)
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "precision");
  if (layout != UNIFRAC_OUT_CONDENSED && layout != UNIFRAC_OUT_FULL)
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "streamed output is condensed or full");
  if (ctx->n_studies != 1)
    return fail(ctx, UNIFRAC_E_UNSUPPORTED, "streamed output needs a single study");
  bool pinned = false;  // page-locked host memory: the copy engines can write it
  {  // host threads write the result: it must be host memory
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, host_out) == cudaSuccess) {
      if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged)
        return fail(ctx, UNIFRAC_E_INVALID_ARG, "streamed output must be host memory");
      pinned = attr.type == cudaMemoryTypeHost;
    }
    cudaGetLastError();
  }
  const int nv = variant == UNIFRAC_BOTH ? 2 : 1;
  const int64_t n = ctx->n_samples;
  const size_t elem = precision == UNIFRAC_FP64 ? 8 : 4;
  const int64_t per_matrix = n_pairs_layout(layout, n, 0, 0);
  if (out_bytes < (size_t)(per_matrix * nv) * elem)
    return fail(ctx, UNIFRAC_E_BUFFER_TOO_SMALL, "output buffer");
  if (layout == UNIFRAC_OUT_FULL)  // the zero diagonal (stripes hold no i == i pairs)
    for (int v = 0; v < nv; ++v)
      for (int64_t i = 0; i < n; ++i) {
        if (elem == 8)
          static_cast<double *>(host_out)[v * per_matrix + i * n + i] = 0.0;
        else
          static_cast<float *>(host_out)[v * per_matrix + i * n + i] = 0.f;
      }
  const int32_t nst = (int32_t)(n / 2);
  if (nst == 0) return UNIFRAC_OK;
  const int32_t chunk = std::min(chunk_stripes, nst);
  const size_t chunk_bytes = (size_t)chunk * n * elem * nv;
  cudaError_t e = cudaSuccess;
  if (!ctx->copy_stream) {
    e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaEventCreateWithFlags(&ctx->ev_chunk_done[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_chunk_copied[b], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy stream");
  }
  int rc;
  for (int b = 0; b < 2; ++b)
    if ((rc = grow(ctx, ctx->chunk_dev[b], chunk_bytes)) ||
        (rc = grow(ctx, ctx->chunk_rows[b], 2 * chunk_bytes)))
      return rc;
  // pinned buffers: the whole row runs of a chunk, or (page-locked full
  // output, written by the copy engines) only the runs that wrap
  const bool direct = pinned && layout == UNIFRAC_OUT_FULL;
  const size_t host_bytes =
      direct ? std::max<size_t>(16, (size_t)nv * 2 * (chunk - 1) * chunk * elem) : 2 * chunk_bytes;
  if (ctx->chunk_host_bytes < host_bytes) {
    for (int b = 0; b < 2; ++b) {
      if (ctx->chunk_host[b]) cudaFreeHost(ctx->chunk_host[b]);
      ctx->chunk_host[b] = nullptr;
    }
    ctx->chunk_host_bytes = 0;
    for (int b = 0; b < 2; ++b) {
      e = cudaMallocHost(&ctx->chunk_host[b], host_bytes);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "pinned host buffer");
    }
    ctx->chunk_host_bytes = host_bytes;
  }
  // Place the row runs of the chunk of stripes [s0, s0 + L) held in pinned
  // buffer b (up runs of every variant, then down runs; see stripe_rows) into
  // the output.  Row i of the full matrix takes its up run at the cyclic
  // columns i + s0 + 1 + t and its down run at i - s0 - L + t (mod n); a
  // condensed row i keeps the columns above i: the up run's up to n - 1, the
  // down run's that wrapped past n.  Host threads take blocks of rows; every
  // piece is one contiguous copy.
  // Full layout into page-locked memory: the copy engines write the runs
  // straight into host_out.  Consecutive rows' runs start n + 1 elements
  // apart, so the rows whose runs do not wrap past column n form four
  // rectangles per variant with that pitch (up runs of rows [0, n - s1) and
  // [n - s0 - 1, n), down runs of rows [s1, n) and [0, s0 + 1)); the runs of
  // the L - 1 rows that wrap (up: rows [n - s1, n - s0 - 1), down: rows
  // [s0 + 1, s1)) go to the pinned buffer and the host places them.
  auto direct_copies = [&](int b, int32_t s0, int32_t L, const char *rows_dev) -> cudaError_t {
    const int64_t s1 = s0 + L;
    const size_t run = (size_t)L * elem, dpitch = (size_t)(n + 1) * elem;
    char *stage = static_cast<char *>(ctx->chunk_host[b]);
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < nv && e == cudaSuccess; ++v) {
      char *out = static_cast<char *>(host_out) + (size_t)v * per_matrix * elem;
      const char *U = rows_dev + (size_t)v * n * run;
      const char *D = rows_dev + (size_t)(nv + v) * n * run;
      struct Rect { int64_t row0, rows, col0; const char *src; };
      const Rect rects[4] = {{0, n - s1, s0 + 1, U},
                             {n - s0 - 1, s0 + 1, s0 + 1 - n, U},
                             {s1, n - s1, -s1, D},
                             {0, s0 + 1, n - s1, D}};
      for (const Rect &r : rects) {
        if (r.rows <= 0 || e != cudaSuccess) continue;
        // row i's run starts at element i (n + 1) + col0
        e = cudaMemcpy2DAsync(out + (size_t)(r.row0 * (n + 1) + r.col0) * elem, dpitch,
                              r.src + (size_t)r.row0 * run, run, run, (size_t)r.rows,
                              cudaMemcpyDeviceToHost, ctx->copy_stream);
      }
      if (L > 1 && e == cudaSuccess)
        e = cudaMemcpyAsync(stage + (size_t)(2 * v) * (L - 1) * run, U + (size_t)(n - s1) * run,
                            (size_t)(L - 1) * run, cudaMemcpyDeviceToHost, ctx->copy_stream);
      if (L > 1 && e == cudaSuccess)
        e = cudaMemcpyAsync(stage + (size_t)(2 * v + 1) * (L - 1) * run, D + (size_t)(s0 + 1) * run,
                            (size_t)(L - 1) * run, cudaMemcpyDeviceToHost, ctx->copy_stream);
    }
    return e;
  };
  auto place_wrapped = [&](int b, int32_t s0, int32_t L) {
    if (L <= 1) return;
    const size_t run = (size_t)L * elem;
    const char *stage = static_cast<const char *>(ctx->chunk_host[b]);
    for (int v = 0; v < nv; ++v)
      for (int side = 0; side < 2; ++side)
        for (int64_t r = 0; r < L - 1; ++r) {
          const int64_t i = side == 0 ? n - (s0 + L) + r : s0 + 1 + r;
          const int64_t c0 = side == 0 ? (i + s0 + 1) % n : ((i - s0 - L) % n + n) % n;
          const char *src = stage + ((size_t)(2 * v + side) * (L - 1) + (size_t)r) * run;
          char *row = static_cast<char *>(host_out) + ((size_t)v * per_matrix + (size_t)i * n) * elem;
          const int64_t first = std::min<int64_t>(L, n - c0);
          std::memcpy(row + c0 * elem, src, first * elem);
          if (first < L) std::memcpy(row, src + first * elem, (L - first) * elem);
        }
  };
  auto merge = [&](int b, int32_t s0, int32_t L) {
    if (direct) return place_wrapped(b, s0, L);
    const char *up = static_cast<const char *>(ctx->chunk_host[b]);
    const char *down = up + (size_t)nv * n * L * elem;
    char *dst = static_cast<char *>(host_out);
    const int T = ctx->opt_host_threads > 0 ? ctx->opt_host_threads : host_threads((int64_t)L * n);
    const int64_t rows_per = (n + T - 1) / T;
    run_threads(T, [&](int t) {
      const int64_t i_lo = std::min<int64_t>(n, (int64_t)t * rows_per);
      const int64_t i_hi = std::min<int64_t>(n, i_lo + rows_per);
      for (int v = 0; v < nv; ++v)
        for (int64_t i = i_lo; i < i_hi; ++i) {
          const char *ur = up + ((size_t)v * n + i) * L * elem;
          const char *dr = down + ((size_t)v * n + i) * L * elem;
          if (layout == UNIFRAC_OUT_FULL) {
            char *row = dst + ((size_t)v * per_matrix + (size_t)i * n) * elem;
            auto place = [&](int64_t c0, const char *src) {  // cyclic run from column c0
              const int64_t first = std::min<int64_t>(L, n - c0);
              std::memcpy(row + c0 * elem, src, first * elem);
              if (first < L) std::memcpy(row, src + first * elem, (L - first) * elem);
            };
            place((i + s0 + 1) % n, ur);
            place(((i - s0 - L) % n + n) % n, dr);
          } else {
            // (i, hi) sits at base + hi in the condensed matrix
            const int64_t base = (int64_t)v * per_matrix + i * n - i * (i + 1) / 2 - i - 1;
            const int64_t nu = std::min<int64_t>(L, std::max<int64_t>(0, n - i - s0 - 1));
            if (nu > 0) std::memcpy(dst + (base + i + s0 + 1) * elem, ur, nu * elem);
            const int64_t nd = std::min<int64_t>(L, std::max<int64_t>(0, s0 + L - i));
            if (nd > 0) std::memcpy(dst + (base + i - s0 - L + n) * elem, dr, nd * elem);
          }
        }
    });
  };
  const int saved_graph = ctx->opt_use_graph;
  ctx->opt_use_graph = 0;  // every chunk has its own stripe range
  const int32_t n_chunks = (nst + chunk - 1) / chunk;
  rc = UNIFRAC_OK;
  for (int32_t c = 0; c <= n_chunks && rc == UNIFRAC_OK; ++c) {
    if (c < n_chunks) {
      const int b = c & 1;
      const int32_t s0 = c * chunk, s1 = std::min(nst, s0 + chunk);
      const size_t bytes = (size_t)(s1 - s0) * n * elem * nv;
      if (c >= 2 && (e = cudaStreamWaitEvent(ctx->stream, ctx->ev_chunk_copied[b], 0)) != cudaSuccess) {
        rc = cuda_fail(ctx, e, "chunk order");
        break;
      }
      // the first chunk embeds and packs; later ones reuse that (the pair
      // kernels only read it), unless one of its buffers was reallocated
      ctx->reuse_prepared = c > 0;
      rc = run_impl(ctx, variant, precision, s0, s1, UNIFRAC_OUT_STRIPES, ctx->chunk_dev[b].p, bytes);
      ctx->reuse_prepared = false;
      if (rc) break;
      if (c == 0) ctx->prep_sig = prep_signature(ctx);
      char *rows_dev = static_cast<char *>(ctx->chunk_rows[b].p);
      if ((rc = stripe_rows(ctx, ctx->chunk_dev[b].p, (int32_t)n, s1 - s0, s0, nv, elem == 8,
                            rows_dev, rows_dev + bytes)))
        break;
      e = cudaEventRecord(ctx->ev_chunk_done[b], ctx->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_chunk_done[b], 0);
      if (e == cudaSuccess)
        e = direct ? direct_copies(b, s0, s1 - s0, rows_dev)
                   : cudaMemcpyAsync(ctx->chunk_host[b], rows_dev, 2 * bytes,
                                     cudaMemcpyDeviceToHost, ctx->copy_stream);
      if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_chunk_copied[b], ctx->copy_stream);
      if (e != cudaSuccess) {
        rc = cuda_fail(ctx, e, "chunk copy");
        break;
      }
    }
    if (c >= 1) {  // merge the previous chunk while this one computes
      const int pb = (c - 1) & 1;
      if ((e = cudaEventSynchronize(ctx->ev_chunk_copied[pb])) != cudaSuccess) {
        rc = cuda_fail(ctx, e, "chunk wait");
        break;
      }
      const int32_t p0 = (c - 1) * chunk;
      merge(pb, p0, std::min(nst, p0 + chunk) - p0);
    }
  }
  if (rc) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamSynchronize(ctx->stream);
  }
  ctx->opt_use_graph = saved_graph;
  return rc;
}

int unifrac_run_streamed(unifrac_ctx *ctx, int variant, int precision, int layout,
                         void *host_out, size_t out_bytes, int32_t chunk_stripes) {
  if (!ctx) return UNIFRAC_E_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return fail(ctx, UNIFRAC_E_CUDA, "cannot select the context's device");
  try {
    return run_streamed_impl(ctx, variant, precision, layout, host_out, out_bytes, chunk_stripes);
  } catch (const std::bad_alloc &) {
    return fail(ctx, UNIFRAC_E_OOM, "host allocation");
  } catch (...) {
    return fail(ctx, UNIFRAC_E_INVALID_ARG, "unexpected failure");
  }
}

// Frees the packing and pair-kernel work buffers of one variant slot (they
// are allocated again, at the size the next run needs, on first use).
static void release_variant_buffers(unifrac_ctx *ctx, int slot) {
  cudaDeviceSynchronize();
  VarBufs &V = ctx->vb[slot];
  DevBuf *vbufs[] = {&V.vals, &V.vals2, &V.bits,   &V.persample, &V.partial, &V.rc,
                     &V.bsize, &V.boff, &V.blocks, &V.cpre,      &V.spart,   &V.rbits,
                     &V.vlist, &V.voff,  &V.trec,    &V.tidx};
  for (DevBuf *b : vbufs)
    if (b->p) {
      dev_free(b->p);
      ctx->device_bytes -= b->bytes;
      b->p = nullptr;
      b->bytes = 0;
    }
  V.voff_pv = -1;
  ctx->buf_generation++;  // a captured graph holds the old addresses
  ctx->reuse_prepared = false;
}

int unifrac_autotune(unifrac_ctx *ctx, int variant, int precision, void *out, size_t out_bytes,
                     int repeats) {
  if (!ctx || !out || repeats < 1) return UNIFRAC_E_INVALID_ARG;
  if (variant != UNIFRAC_UNWEIGHTED && variant != UNIFRAC_WEIGHTED_NORMALIZED)
    return UNIFRAC_E_INVALID_ARG;
  if (precision != UNIFRAC_FP64 && precision != UNIFRAC_MIXED) return UNIFRAC_E_INVALID_ARG;
  if (precision == UNIFRAC_FP64) return UNIFRAC_OK;
  DeviceGuard g(ctx->device);
  const bool weighted = variant == UNIFRAC_WEIGHTED_NORMALIZED;
  const int split_opt = weighted ? UNIFRAC_OPT_SPARSE_THRESHOLD : UNIFRAC_OPT_UNWEIGHTED_SPARSE_THRESHOLD;
  const int64_t n = std::max<int32_t>(ctx->max_study_n, 1);
  const int saved_graph = ctx->opt_use_graph;
  ctx->opt_use_graph = 0;
  // time one setting of one option (best of `repeats` runs after a warm-up
  // run); a setting whose buffers do not fit in device memory is skipped
  auto timed = [&](int option, int64_t v, double *t) -> int {
    *t = 1e300;
    int rc = unifrac_set_option(ctx, option, v);
    if (rc) return rc;
    for (int r = 0; r <= repeats; ++r) {
      rc = unifrac_run(ctx, variant, precision, 0, -1, UNIFRAC_OUT_CONDENSED, out, out_bytes);
      if (rc == UNIFRAC_E_OOM) {
        cudaGetLastError();
        release_variant_buffers(ctx, variant);
        *t = 1e300;
        return UNIFRAC_OK;
      }
      if (rc) return rc;
      cudaError_t e = cudaEventSynchronize(ctx->ev[2]);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[2]);
      if (r > 0) *t = std::min(*t, (double)ms);  // first run is the warm-up
    }
    return UNIFRAC_OK;
  };
  // one option at a time, the others held at their current (tuned) values
  auto tune = [&](int option, std::vector<int64_t> vals, bool refine) -> int {
    double best = 1e300;
    int64_t best_v = vals[0];
    std::vector<int64_t> tried;
    auto one = [&](int64_t v) -> int {
      if (std::find(tried.begin(), tried.end(), v) != tried.end()) return UNIFRAC_OK;
      tried.push_back(v);
      double t;
      int rc = timed(option, v, &t);
      if (!rc && t < best) {
        best = t;
        best_v = v;
      }
      return rc;
    };
    int rc = UNIFRAC_OK;
    for (int64_t v : vals)
      if ((rc = one(v))) return rc;
    if (refine && best_v > 0) {  // then 3/4 and 3/2 of the best coarse value
      const int64_t coarse = best_v;
      if ((rc = one(std::max<int64_t>(2, coarse * 3 / 4)))) return rc;
      if ((rc = one(coarse * 3 / 2))) return rc;
    }
    if (best >= 1e300) return fail(ctx, UNIFRAC_E_OOM, "autotune: no candidate fits in device memory");
    return unifrac_set_option(ctx, option, best_v);
  };
  std::vector<int64_t> split;
  if (weighted) {
    for (int64_t num : {1, 2, 4, 8, 12}) split.push_back(std::max<int64_t>(2, n * num / 16));
  } else {
    split.push_back(0);  // everything on the tensor cores
    for (int64_t num : {1, 2, 4, 8}) split.push_back(std::max<int64_t>(2, n * num / 32));
  }
  int rc = tune(split_opt, split, true);
  int64_t th = 0;
  if (!rc) rc = unifrac_get_option(ctx, split_opt, &th);
  // incidences a lane walks alone (when the chosen split has a sparse part)
  if (!rc && th != 0)
    rc = tune(weighted ? UNIFRAC_OPT_SPARSE_LANE_PAIRS : UNIFRAC_OPT_UNWEIGHTED_SPARSE_LANE_PAIRS,
              {32, 64, 128, 256}, true);
  // presence bound of the per-branch lists of the very rarely present positions
  if (!rc && th != 0)
    rc = tune(weighted ? UNIFRAC_OPT_RARE_LIST : UNIFRAC_OPT_UNWEIGHTED_RARE_LIST,
              {0, 64, 256, 1024}, true);
  // branches summed in registers before each FP32 running-total update
  if (!rc && weighted) rc = tune(UNIFRAC_OPT_WEIGHTED_FLUSH, {128, 256, 512}, false);
  ctx->opt_use_graph = saved_graph;
  // the candidates' buffers were sized for the largest of them: release them,
  // the next run allocates what the chosen settings need
  release_variant_buffers(ctx, variant);
  return rc;
}

int unifrac_get_stat(const unifrac_ctx *ctx_c, int stat, double *value) {
  if (!ctx_c || !value) return UNIFRAC_E_INVALID_ARG;
  unifrac_ctx *ctx = const_cast<unifrac_ctx *>(ctx_c);
  switch (stat) {
    case UNIFRAC_STAT_KERNEL_LAUNCHES: *value = ctx->stat_launches; return UNIFRAC_OK;
    case UNIFRAC_STAT_PAIR_BRANCH: *value = ctx->stat_pair_branch; return UNIFRAC_OK;
    case UNIFRAC_STAT_USEFUL: *value = ctx->stat_useful; return UNIFRAC_OK;
    case UNIFRAC_STAT_BRANCHES_KEPT: *value = ctx->K; return UNIFRAC_OK;
    case UNIFRAC_STAT_LEVELS: *value = ctx->n_levels; return UNIFRAC_OK;
    case UNIFRAC_STAT_TILE_PAIRS: *value = ctx->stat_tile_pairs; return UNIFRAC_OK;
    case UNIFRAC_STAT_DEVICE_BYTES: *value = (double)ctx->device_bytes; return UNIFRAC_OK;
    case UNIFRAC_STAT_SELECTED_UPDATES:
    case UNIFRAC_STAT_PAIR_KERNEL_MS:
    case UNIFRAC_STAT_EMBED_MS: {
      if (!ctx->ev_valid) return fail(ctx, UNIFRAC_E_INVALID_ARG, "no run yet");
      DeviceGuard g(ctx->device);
      cudaError_t e = cudaEventSynchronize(ctx->ev[2]);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "event");
      if (stat == UNIFRAC_STAT_SELECTED_UPDATES) {
        unsigned long long c = 0;
        e = cudaMemcpy(&c, ctx->d_counter + kCounterBase + 4 * ctx->cur_slot, sizeof(c),
                       cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "counter");
        *value = (double)c * ctx->sel_unit * (double)TILE * (double)TILE;
        return UNIFRAC_OK;
      }
      float ms = 0.f;
      if (stat == UNIFRAC_STAT_PAIR_KERNEL_MS)
        e = cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[2]);
      else
        e = cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "elapsed time");
      *value = ms;
      return UNIFRAC_OK;
    }
    case UNIFRAC_STAT_PAIR_MS_UNWEIGHTED:
    case UNIFRAC_STAT_PAIR_MS_WEIGHTED: {
      const int v = stat == UNIFRAC_STAT_PAIR_MS_UNWEIGHTED ? 0 : 1;
      if (!ctx->ev_pair_valid[v]) return fail(ctx, UNIFRAC_E_INVALID_ARG, "no run of that variant");
      DeviceGuard g(ctx->device);
      cudaError_t e = cudaEventSynchronize(ctx->ev_pair[v][1]);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "event");
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ctx->ev_pair[v][0], ctx->ev_pair[v][1]);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "elapsed time");
      *value = ms;
      return UNIFRAC_OK;
    }
    case UNIFRAC_STAT_SELECTED_UNWEIGHTED:
    case UNIFRAC_STAT_SELECTED_WEIGHTED: {
      const int v = stat == UNIFRAC_STAT_SELECTED_UNWEIGHTED ? 0 : 1;
      if (!ctx->ev_pair_valid[v]) return fail(ctx, UNIFRAC_E_INVALID_ARG, "no run of that variant");
      DeviceGuard g(ctx->device);
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise");
      unsigned long long c = 0;
      e = cudaMemcpy(&c, ctx->d_counter + kCounterBase + 4 * v, sizeof(c), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "counter");
      *value = (double)c * ctx->sel_unit_v[v] * (double)TILE * (double)TILE;
      return UNIFRAC_OK;
    }
    case UNIFRAC_STAT_CREATE_HOST_MS: *value = ctx->create_host_ms; return UNIFRAC_OK;
    case UNIFRAC_STAT_CREATE_DEVICE_MS: *value = ctx->create_device_ms; return UNIFRAC_OK;
    case UNIFRAC_STAT_MAX_REACH: *value = (double)ctx->max_reach; return UNIFRAC_OK;
    case UNIFRAC_STAT_SPARSE_MS_UNWEIGHTED:
    case UNIFRAC_STAT_SPARSE_MS_WEIGHTED:
    case UNIFRAC_STAT_SPARSE_UPDATES_UNWEIGHTED:
    case UNIFRAC_STAT_SPARSE_UPDATES_WEIGHTED:
    case UNIFRAC_STAT_LIST_MS_UNWEIGHTED:
    case UNIFRAC_STAT_LIST_MS_WEIGHTED:
    case UNIFRAC_STAT_LIST_UPDATES_UNWEIGHTED:
    case UNIFRAC_STAT_LIST_UPDATES_WEIGHTED: {
      const int v = (stat == UNIFRAC_STAT_SPARSE_MS_UNWEIGHTED ||
                     stat == UNIFRAC_STAT_SPARSE_UPDATES_UNWEIGHTED ||
                     stat == UNIFRAC_STAT_LIST_MS_UNWEIGHTED ||
                     stat == UNIFRAC_STAT_LIST_UPDATES_UNWEIGHTED) ? 0 : 1;
      const bool list = stat >= UNIFRAC_STAT_LIST_MS_UNWEIGHTED;
      if (!ctx->ev_pair_valid[v]) return fail(ctx, UNIFRAC_E_INVALID_ARG, "no run of that variant");
      DeviceGuard g(ctx->device);
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise");
      if (stat == UNIFRAC_STAT_SPARSE_UPDATES_UNWEIGHTED ||
          stat == UNIFRAC_STAT_SPARSE_UPDATES_WEIGHTED ||
          stat == UNIFRAC_STAT_LIST_UPDATES_UNWEIGHTED ||
          stat == UNIFRAC_STAT_LIST_UPDATES_WEIGHTED) {
        unsigned long long c = 0;
        e = cudaMemcpy(&c, ctx->d_counter + kCounterBase + 4 * v + (list ? 3 : 2), sizeof(c),
                       cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "counter");
        *value = (double)c;
        return UNIFRAC_OK;
      }
      float ms = 0.f;
      cudaEvent_t (&ev)[2] = list ? ctx->ev_list[v] : ctx->ev_sp[v];
      if (cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) {
        cudaGetLastError();
        ms = 0.f;  // no such phase in that run
      }
      // the sparse phase's window holds the list kernel: report the two apart
      if (!list) {
        float lm = 0.f;
        if (cudaEventElapsedTime(&lm, ctx->ev_list[v][0], ctx->ev_list[v][1]) != cudaSuccess) {
          cudaGetLastError();
          lm = 0.f;
        }
        ms = std::max(0.f, ms - lm);
      }
      *value = ms;
      return UNIFRAC_OK;
    }
    case UNIFRAC_STAT_DEVICE_ERROR: {
      DeviceGuard g(ctx->device);
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise");
      unsigned long long c[kCounters] = {0};
      e = cudaMemcpy(c, ctx->d_counter, sizeof(c), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "counter");
      // the error codes of both variant slots (a run of both may raise in either)
      const unsigned long long err =
          c[kCounterBase + 1] ? c[kCounterBase + 1] : c[kCounterBase + 4 + 1];
      *value = -(double)err;
      return UNIFRAC_OK;
    }
    default:
      return UNIFRAC_E_INVALID_ARG;
  }
}

}  // extern "C"
