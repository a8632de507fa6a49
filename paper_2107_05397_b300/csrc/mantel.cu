// unifrac_mantel: the Mantel test between two distance matrices on the GPU
// (the paper, Section III: the correlation of two distance matrices, Pearson
// or Spearman, assessed by permuting the samples of one of them).
//
// Over the P = n(n-1)/2 pairs i < j, with dx = x - mean x, dy = y - mean y:
//   r = sum dx dy / sqrt(sum dx^2 sum dy^2)
// (Spearman: Pearson on the average ranks of the pair values).  A permutation
// pi relabels the samples of y; the means and sums of squares stay the same,
// so a permuted statistic needs only the cross sum
//   c_pi = sum_{i<j} dx(i, j) dy(pi(i), pi(j)).
//
// Kernel layout (k_mantel_cross, y-row-stationary): one block per (row a of
// y, batch of kMantelBatch permutations).  The block stages row a of y in
// shared memory once; for each permutation p of the batch it takes the row
// i = pi_p^-1(a) of x, whose pairs (i, j > i) map to the y pairs
// (a, pi_p(j)), and streams x(i, j > i) and pi_p(j) with coalesced loads
// while gathering y(a, pi_p(j)) from shared memory.  Each permutation reads
// every pair of x once (HBM) and every row of y once per batch; the
// random gather that would otherwise hit one 32-byte sector per value is a
// shared-memory access instead.  Rows too long for shared memory are read
// from global memory (the batch keeps the row in L2).  Per (permutation,
// row) block sums go to `partial`, summed per permutation in a fixed order
// (k_sum_rows), so results do not depend on scheduling.  Two-sided
// p = (1 + #{|r_pi| >= |r|}) / (M + 1).
//
// Spearman ranks are computed on the device: the upper-triangle values are
// sorted with their pair index (CUB radix sort), run heads found by a
// max-scan of head positions, each run's average rank written at its head,
// and the centred ranks scattered into a symmetric n x n matrix of the input
// precision, which then goes through the Pearson kernels.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <memory>
#include <thread>
#include <vector>

#include "ufb_internal.cuh"

namespace ufb {
namespace {

constexpr int kMantelBatch = 16;          // permutations per block
constexpr int kShortRowBytes = 24 * 1024;  // rows up to this: short-row launch shape
constexpr int kShortRowThreads = 128;
constexpr int kMantelUnroll = 4;          // loads in flight per thread and round (even)
constexpr int kMomentBlocks = 592;
constexpr size_t kSmemBudget = 220 * 1024;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

// Stage row `a` of the n x n matrix y into `buf`: element k of the row lands
// at buf[k + s], s = (a n) mod (16 / sizeof(T)), so that global and shared
// 16-byte chunks line up.  Chunks that would reach past the matrix end are
// copied element by element.
template <typename T>
__device__ __forceinline__ int stage_row(T *buf, const T *__restrict__ y, int64_t a, int32_t n) {
  constexpr int kVec = 16 / sizeof(T);
  const int64_t start = a * n;
  const int s = (int)(start % kVec);
  const int64_t first = start - s;  // 16-byte aligned element index
  const int nchunk = (n + s + kVec - 1) / kVec;
  const int64_t total = (int64_t)n * n;
  for (int c = threadIdx.x; c < nchunk; c += blockDim.x) {
    const int64_t g = first + (int64_t)c * kVec;
    if (g + kVec <= total) {
      cp_async16(buf + (size_t)c * kVec, y + g);
    } else {
      for (int e = 0; e < kVec; ++e)
        if (g + e < total) buf[(size_t)c * kVec + e] = y[g + e];
    }
  }
  return s;
}

// y-row-stationary cross sums.  Block (a, batch): row a of y is staged once
// (NBUF = 1; NBUF = 0 reads it from global memory, where it stays in L2 for
// the batch), then for each permutation p of the batch, with i = pi_p^-1(a),
//   partial[p][a] = sum_{j > i} (x(i, j) - mx) (y(a, pi_p(j)) - my),
// i.e. the pairs (i, j) of x whose relabelled y pair has a as its first
// sample.  Over a = 0 .. n-1 the rows i = pi_p^-1(a) run over every row once,
// so the partials of one permutation sum to its cross sum.  x(i, j > i) and
// pi_p(j) are coalesced loads (x from HBM, each pair once per permutation;
// the batch's permutation rows stay in L2); y(a, .) is a shared-memory
// gather.  No barrier between permutations: per-warp sums go to red[][] and
// are reduced once at the end.  P: permutation entry type (uint16_t while
// n <= 65,536, else int32_t).
template <typename T, typename P, int NBUF, int MINB, int NT>
__global__ void __launch_bounds__(NT, MINB) k_mantel_cross(
    const T *__restrict__ x, const T *__restrict__ y, int32_t n, T mx, T my,
    const P *__restrict__ perms, const P *__restrict__ inv, int32_t n_perms,
    double *__restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kMantelBatch][NT / 32];
  const int64_t a = blockIdx.x;
  const int p0 = blockIdx.y * kMantelBatch;
  const int nb = min(kMantelBatch, n_perms - p0);
  // staged rows are centred once here (y - my), rows read from global memory
  // are centred in the loop
  const T *yv;
  T yc = my;
  if (NBUF > 0) {
    T *buf = reinterpret_cast<T *>(smem_raw);
    const int s = stage_row(buf, y, a, n);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += NT) buf[s + k] -= my;
    __syncthreads();
    yv = buf + s;
    yc = T(0);
  } else {
    yv = y + a * n;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int b = 0; b < nb; ++b) {
    const int64_t p = p0 + b;
    const P *prow = perms + p * n;
    const int i = (int)inv[p * n + a];
    const T *xrow = x + (int64_t)i * n;
    // kMantelUnroll independent (permutation entry, x) loads in flight per
    // thread each round; slots past the row end load nothing and add 0
    T acc0 = T(0), acc1 = T(0);
    for (int j = i + 1 + threadIdx.x; j < n; j += kMantelUnroll * NT) {
      int q[kMantelUnroll];
      T xv[kMantelUnroll];
#pragma unroll
      for (int u = 0; u < kMantelUnroll; ++u) {
        const int jj = j + u * NT;
        q[u] = jj < n ? (int)prow[jj] : 0;
        xv[u] = jj < n ? __ldg(xrow + jj) : mx;
      }
#pragma unroll
      for (int u = 0; u < kMantelUnroll; u += 2) {
        acc0 = fma_t(xv[u] - mx, NBUF > 0 ? yv[q[u]] : yv[q[u]] - yc, acc0);
        acc1 = fma_t(xv[u + 1] - mx, NBUF > 0 ? yv[q[u + 1]] : yv[q[u + 1]] - yc, acc1);
      }
    }
    // warp sum in T (B300's FP64 pipe is narrow: FP64 here would bound the
    // FP32 kernel), FP64 from the per-warp sums on
    T v = acc0 + acc1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[b][warp] = (double)v;
  }
  __syncthreads();
  for (int b = warp; b < nb; b += NT / 32) {
    double v = 0.0;
    for (int w = lane; w < NT / 32; w += 32) v += red[b][w];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) partial[(int64_t)(p0 + b) * n + a] = v;
  }
}

// out[p] = sum_i partial[p][i], fixed order (block per permutation).
__global__ void __launch_bounds__(256) k_sum_rows(const double *__restrict__ partial, int32_t n,
                                                  double *__restrict__ out) {
  __shared__ double red[8];
  const double *row = partial + (int64_t)blockIdx.x * n;
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) v += row[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

// Per-block sums of (v - c) and (v - c)^2 over the strict upper triangle of an
// n x n matrix (FP64); blocks stride over rows.
template <typename T>
__global__ void __launch_bounds__(256) k_moments(const T *__restrict__ m, int32_t n, double c,
                                                 double *__restrict__ out) {
  __shared__ double r1[8], r2[8];
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
    for (int64_t j = i + 1 + threadIdx.x; j < n; j += 256) {
      const double d = (double)m[i * n + j] - c;
      s1 += d;
      s2 += d * d;
    }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = s1;
    r2[threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) {
      a += r1[w];
      b += r2[w];
    }
    out[2 * blockIdx.x] = a;
    out[2 * blockIdx.x + 1] = b;
  }
}

// ---- Spearman ranks ------------------------------------------------------

// keys[t] = m(i, j), idx[t] = t for the condensed index t of pair i < j.
template <typename T>
__global__ void k_upper_keys(const T *__restrict__ m, int32_t n, T *__restrict__ keys,
                             uint32_t *__restrict__ idx) {
  const int64_t i = blockIdx.x;
  const int64_t row = i * n - i * (i + 1) / 2 - i - 1;
  for (int64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x) {
    keys[row + j] = m[i * n + j];
    idx[row + j] = (uint32_t)(row + j);
  }
}

// head[t] = t at the first element of a run of equal sorted keys, else 0.
template <typename T>
__global__ void k_run_heads(const T *__restrict__ keys, int64_t P, uint32_t *__restrict__ head) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P;
       t += (int64_t)gridDim.x * blockDim.x)
    head[t] = (t == 0 || keys[t] != keys[t - 1]) ? (uint32_t)t : 0u;
}

// At the last element of each run: runval[head] = its average 1-based rank
// minus the mean rank (P + 1) / 2.
template <typename T>
__global__ void k_run_values(const T *__restrict__ keys, const uint32_t *__restrict__ head,
                             int64_t P, double *__restrict__ runval) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P;
       t += (int64_t)gridDim.x * blockDim.x)
    if (t == P - 1 || keys[t + 1] != keys[t]) {
      const uint32_t h = head[t];
      runval[h] = 0.5 * ((double)h + (double)t) + 1.0 - 0.5 * ((double)P + 1.0);
    }
}

// R(i, j) = R(j, i) = centred rank of pair (i, j).  rowbase[i] is the
// condensed index of pair (i, j) minus j.
template <typename T>
__global__ void k_scatter_ranks(const uint32_t *__restrict__ idx, const uint32_t *__restrict__ head,
                                const double *__restrict__ runval, const int64_t *__restrict__ rowbase,
                                int32_t n, int64_t P, T *__restrict__ R) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx[t];
    // row i: the largest i with rowbase[i] + i + 1 <= c (its first pair)
    int lo = 0, hi = n - 2;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (rowbase[mid] + mid + 1 <= c) lo = mid;
      else hi = mid - 1;
    }
    const int64_t i = lo, j = c - rowbase[lo];
    const T v = (T)runval[head[t]];
    R[i * n + j] = v;
    R[j * n + i] = v;
  }
}

template <typename T>
__global__ void k_zero_diag(T *R, int32_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    R[i * n + i] = T(0);
}

// fn(lo, hi) over [0, n) in contiguous ranges on host threads (one thread
// below 64 rows).
template <typename F>
void host_parallel(int64_t n, F &&fn) {
  const unsigned hw = std::thread::hardware_concurrency();
  const int T = n < 64 ? 1 : (int)std::max<int64_t>(1, std::min<int64_t>(std::min(32u, hw ? hw : 1u), n));
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) th.emplace_back(fn, n * t / T, n * (t + 1) / T);
  fn((int64_t)0, n / T);
  for (auto &x : th) x.join();
}

// Device allocations released together when the call returns.
struct Cuda {
  std::vector<void *> ptrs;
  ~Cuda() {
    for (void *p : ptrs) cudaFree(p);
  }
  template <typename U>
  bool alloc(U **p, size_t count) {
    void *q = nullptr;
    if (dev_malloc_retry(&q, std::max<size_t>(count, 1) * sizeof(U)) != cudaSuccess) return false;
    ptrs.push_back(q);
    *p = static_cast<U *>(q);
    return true;
  }
};

// Centred-rank matrix R (n x n, type T) of the upper triangle of m.
template <typename T>
int spearman_ranks(const T *m, int32_t n, T *R, cudaStream_t st, Cuda &mem) {
  const int64_t P = (int64_t)n * (n - 1) / 2;
  T *k_in, *k_out;
  uint32_t *i_in, *i_out, *head;
  double *runval;
  int64_t *rowbase;
  if (!mem.alloc(&k_in, P) || !mem.alloc(&k_out, P) || !mem.alloc(&i_in, P) ||
      !mem.alloc(&i_out, P) || !mem.alloc(&head, P) || !mem.alloc(&runval, P) ||
      !mem.alloc(&rowbase, n))
    return UNIFRAC_E_OOM;
  std::vector<int64_t> rb(n);
  for (int64_t i = 0; i < n; ++i) rb[i] = i * n - i * (i + 1) / 2 - i - 1;
  if (cudaMemcpyAsync(rowbase, rb.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return UNIFRAC_E_CUDA;
  k_upper_keys<T><<<n, 256, 0, st>>>(m, n, k_in, i_in);
  size_t tmp_sort = 0, tmp_scan = 0;
  if (cub::DeviceRadixSort::SortPairs(nullptr, tmp_sort, k_in, k_out, i_in, i_out, P, 0,
                                      (int)(8 * sizeof(T)), st) != cudaSuccess ||
      cub::DeviceScan::InclusiveScan(nullptr, tmp_scan, head, head, ::cuda::maximum<>{}, P, st) !=
          cudaSuccess)
    return UNIFRAC_E_CUDA;
  unsigned char *tmp;
  if (!mem.alloc(&tmp, std::max(tmp_sort, tmp_scan))) return UNIFRAC_E_OOM;
  size_t t1 = tmp_sort, t2 = tmp_scan;
  if (cub::DeviceRadixSort::SortPairs(tmp, t1, k_in, k_out, i_in, i_out, P, 0, (int)(8 * sizeof(T)),
                                      st) != cudaSuccess)
    return UNIFRAC_E_CUDA;
  const int g = 148 * 8;
  k_run_heads<T><<<g, 256, 0, st>>>(k_out, P, head);
  if (cub::DeviceScan::InclusiveScan(tmp, t2, head, head, ::cuda::maximum<>{}, P, st) != cudaSuccess)
    return UNIFRAC_E_CUDA;
  k_run_values<T><<<g, 256, 0, st>>>(k_out, head, P, runval);
  k_scatter_ranks<T><<<g, 256, 0, st>>>(i_out, head, runval, rowbase, n, P, R);
  k_zero_diag<T><<<(n + 255) / 256, 256, 0, st>>>(R, n);
  return cudaGetLastError() == cudaSuccess ? UNIFRAC_OK : UNIFRAC_E_CUDA;
}

// Shared memory the y-row staging may use per block: kSmemBudget, or less
// when UNIFRAC_MANTEL_SMEM_BYTES is set (to leave room for other work on the
// SMs; 0 gathers y from global memory).
size_t smem_budget() {
  const char *v = std::getenv("UNIFRAC_MANTEL_SMEM_BYTES");
  if (!v || !*v) return kSmemBudget;
  char *end = nullptr;
  const long long b = std::strtoll(v, &end, 10);
  if (end == v || b < 0) return kSmemBudget;
  return std::min<size_t>((size_t)b, kSmemBudget);
}

template <typename T, typename P, int NBUF, int MINB, int NT>
cudaError_t launch_cross(int32_t M, size_t smem, cudaStream_t st, const T *x, const T *y, int32_t n,
                         T mx, T my, const P *perms, const P *inv, double *partial) {
  if (smem > 0) {
    const cudaError_t e = cudaFuncSetAttribute(k_mantel_cross<T, P, NBUF, MINB, NT>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // gridDim.y is at most 65,535: batches beyond that in further launches
  const int64_t batches = (M + kMantelBatch - 1) / kMantelBatch;
  for (int64_t b0 = 0; b0 < batches; b0 += 65535) {
    const int64_t nbat = std::min<int64_t>(65535, batches - b0);
    const int64_t first = b0 * kMantelBatch;
    const int32_t cnt = (int32_t)std::min<int64_t>(M - first, nbat * kMantelBatch);
    k_mantel_cross<T, P, NBUF, MINB, NT><<<dim3(n, (unsigned)nbat), NT, smem, st>>>(
        x, y, n, mx, my, perms + first * n, inv + first * n, cnt, partial + first * n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Launch shape by row length (buf_bytes per staged row of y): short rows,
// kShortRowThreads threads (several blocks per SM); long rows, 1,024
// threads, two blocks per SM while two rows fit; rows longer than the
// shared-memory budget are read from global memory (L2).
template <typename T, typename P>
cudaError_t cross_sums(int32_t n, int32_t M, cudaStream_t st, const T *x, const T *y, T mx, T my,
                       const P *perms, const P *inv, double *partial) {
  const size_t buf_bytes = (((size_t)n + 16 / sizeof(T) + 3) & ~(size_t)3) * sizeof(T);
  const size_t budget = smem_budget();
  if (buf_bytes <= kShortRowBytes && buf_bytes <= budget)
    return launch_cross<T, P, 1, 1, kShortRowThreads>(M, buf_bytes, st, x, y, n, mx, my, perms, inv, partial);
  if (2 * buf_bytes <= budget)
    return launch_cross<T, P, 1, 2, 1024>(M, buf_bytes, st, x, y, n, mx, my, perms, inv, partial);
  if (buf_bytes <= budget)
    return launch_cross<T, P, 1, 1, 1024>(M, buf_bytes, st, x, y, n, mx, my, perms, inv, partial);
  return launch_cross<T, P, 0, 1, 1024>(M, 0, st, x, y, n, mx, my, perms, inv, partial);
}

template <typename T>
int mantel_pearson(const T *x, const T *y, int32_t n, const int32_t *perms_host, int32_t n_perms,
                   double *r_out, double *stats_out, double *p_out, cudaStream_t st, Cuda &mem) {
  const int64_t P = (int64_t)n * (n - 1) / 2;
  double *mom;
  if (!mem.alloc(&mom, 2 * kMomentBlocks)) return UNIFRAC_E_OOM;
  std::vector<double> h(2 * kMomentBlocks);
  auto moments = [&](const T *v, double c, double &s1, double &s2) -> int {
    k_moments<T><<<kMomentBlocks, 256, 0, st>>>(v, n, c, mom);
    if (cudaMemcpyAsync(h.data(), mom, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return UNIFRAC_E_CUDA;
    s1 = s2 = 0.0;
    for (int b = 0; b < kMomentBlocks; ++b) {
      s1 += h[2 * b];
      s2 += h[2 * b + 1];
    }
    return UNIFRAC_OK;
  };
  double sx, sxx, sy, syy;
  int rc;
  if ((rc = moments(x, 0.0, sx, sxx)) || (rc = moments(y, 0.0, sy, syy))) return rc;
  const double mx = sx / (double)P, my = sy / (double)P;
  if ((rc = moments(x, mx, sx, sxx)) || (rc = moments(y, my, sy, syy))) return rc;
  // the second pass is taken about the first mean; its residual sum corrects
  // the sum of squares to the exact mean: sum (v - m)^2 = sum (v - c)^2 - (sum (v - c))^2 / P
  sxx -= sx * sx / (double)P;
  syy -= sy * sy / (double)P;
  const double norm = std::sqrt(sxx * syy);
  // the identity first, then the caller's permutations, and their inverses
  // (16-bit entries while every sample index fits)
  const int32_t M = n_perms + 1;
  const bool narrow = n <= 65536;
  const size_t esz = narrow ? 2 : 4;
  unsigned char *d_pi;
  double *partial, *cross;
  if (!mem.alloc(&d_pi, 2 * (size_t)M * n * esz) || !mem.alloc(&partial, (size_t)M * n) ||
      !mem.alloc(&cross, (size_t)M))
    return UNIFRAC_E_OOM;
  const size_t hp_bytes = 2 * (size_t)M * n * esz;
  std::unique_ptr<unsigned char[]> hp(new unsigned char[hp_bytes]);  // every byte written below
  const int64_t half = (int64_t)M * n;
  auto put = [&](int64_t t, int32_t v) {
    if (narrow) reinterpret_cast<uint16_t *>(hp.get())[t] = (uint16_t)v;
    else reinterpret_cast<int32_t *>(hp.get())[t] = v;
  };
  host_parallel(M, [&](int64_t p0, int64_t p1) {  // permutation rows and their inverses
    for (int64_t p = p0; p < p1; ++p)
      for (int32_t i = 0; i < n; ++i) {
        const int32_t v = p == 0 ? i : perms_host[(p - 1) * n + i];
        put(p * n + i, v);
        put(half + p * n + v, i);
      }
  });
  if (cudaMemcpyAsync(d_pi, hp.get(), hp_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return UNIFRAC_E_CUDA;
  const T mxt = (T)mx, myt = (T)my;
  const cudaError_t e =
      narrow ? cross_sums<T, uint16_t>(n, M, st, x, y, mxt, myt, reinterpret_cast<const uint16_t *>(d_pi),
                                       reinterpret_cast<const uint16_t *>(d_pi) + half, partial)
             : cross_sums<T, int32_t>(n, M, st, x, y, mxt, myt, reinterpret_cast<const int32_t *>(d_pi),
                                      reinterpret_cast<const int32_t *>(d_pi) + half, partial);
  if (e != cudaSuccess) return UNIFRAC_E_CUDA;
  k_sum_rows<<<M, 256, 0, st>>>(partial, n, cross);
  std::vector<double> c(M);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(c.data(), cross, M * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return UNIFRAC_E_CUDA;
  // The kernel centres with the means rounded to T.  Over the P pairs,
  // sum (v - m_T) = P (m - m_T) for either matrix and any permutation, so the
  // cross sum about the exact means is c - P (mx - mx_T)(my - my_T).
  const double corr = (double)P * (mx - (double)mxt) * (my - (double)myt);
  const bool defined = norm > 0.0 && std::isfinite(norm);
  for (int32_t p = 0; p < M; ++p) c[p] = defined ? (c[p] - corr) / norm : NAN;
  *r_out = c[0];
  int64_t hits = 0;
  for (int32_t p = 1; p < M; ++p) {
    if (stats_out) stats_out[p - 1] = c[p];
    if (std::fabs(c[p]) >= std::fabs(c[0])) ++hits;
  }
  *p_out = (defined && n_perms > 0) ? (1.0 + (double)hits) / (double)M : NAN;
  return UNIFRAC_OK;
}

template <typename T>
int mantel_impl(const T *x, const T *y, int32_t n, const int32_t *perms, int32_t n_perms, int method,
                double *r, double *stats, double *p, cudaStream_t st) {
  Cuda mem;
  if (method == UNIFRAC_MANTEL_PEARSON)
    return mantel_pearson<T>(x, y, n, perms, n_perms, r, stats, p, st, mem);
  T *rx, *ry;
  if (!mem.alloc(&rx, (size_t)n * n) || !mem.alloc(&ry, (size_t)n * n)) return UNIFRAC_E_OOM;
  int rc;
  {
    Cuda scratch;  // sort buffers, released before the permutation pass
    if ((rc = spearman_ranks<T>(x, n, rx, st, scratch))) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess) return UNIFRAC_E_CUDA;
  }
  {
    Cuda scratch;
    if ((rc = spearman_ranks<T>(y, n, ry, st, scratch))) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess) return UNIFRAC_E_CUDA;
  }
  return mantel_pearson<T>(rx, ry, n, perms, n_perms, r, stats, p, st, mem);
}

}  // namespace
}  // namespace ufb

extern "C" int unifrac_mantel(const void *x, const void *y, int precision, int32_t n,
                              const int32_t *perms, int32_t n_perms, int method, double *r,
                              double *perm_stats, double *p_value, void *cuda_stream) {
  using namespace ufb;
  if (!x || !y || !r || !p_value || n < 3 || n > UNIFRAC_MANTEL_MAX_SAMPLES || n_perms < 0 ||
      (n_perms > 0 && !perms))
    return UNIFRAC_E_INVALID_ARG;
  if (precision != UNIFRAC_FP64 && precision != UNIFRAC_MIXED) return UNIFRAC_E_INVALID_ARG;
  if (method != UNIFRAC_MANTEL_PEARSON && method != UNIFRAC_MANTEL_SPEARMAN)
    return UNIFRAC_E_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) % 16 != 0)
    return UNIFRAC_E_INVALID_ARG;
  cudaPointerAttributes ax{}, ay{};
  if (cudaPointerGetAttributes(&ax, x) != cudaSuccess || cudaPointerGetAttributes(&ay, y) != cudaSuccess ||
      (ax.type != cudaMemoryTypeDevice && ax.type != cudaMemoryTypeManaged) ||
      (ay.type != cudaMemoryTypeDevice && ay.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return UNIFRAC_E_INVALID_ARG;
  }
  try {
    std::atomic<bool> bad{false};  // every row a permutation of 0 .. n-1
    host_parallel(n_perms, [&](int64_t p0, int64_t p1) {
      std::vector<uint8_t> seen(n);
      for (int64_t p = p0; p < p1 && !bad.load(std::memory_order_relaxed); ++p) {
        std::fill(seen.begin(), seen.end(), 0);
        for (int32_t i = 0; i < n; ++i) {
          const int32_t v = perms[p * n + i];
          if (v < 0 || v >= n || seen[v]) {
            bad = true;
            return;
          }
          seen[v] = 1;
        }
      }
    });
    if (bad) return UNIFRAC_E_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == UNIFRAC_FP64)
      return mantel_impl<double>(static_cast<const double *>(x), static_cast<const double *>(y), n,
                                 perms, n_perms, method, r, perm_stats, p_value, st);
    return mantel_impl<float>(static_cast<const float *>(x), static_cast<const float *>(y), n, perms,
                              n_perms, method, r, perm_stats, p_value, st);
  } catch (const std::bad_alloc &) {
    return UNIFRAC_E_OOM;
  }
}
