// unifrac_dense_noalloc: the whole-matrix FP64 computation for small problems
// without any allocation, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not wanted
// after start-up -- a real-time or embedded pipeline that reserves all memory
// at initialisation, a plug-in living inside a host application that owns
// the device memory pool, or work enqueued from a context that must not
// synchronise the device (cudaMalloc/cudaFree can).  unifrac_create allocates
// device buffers for its inputs and work space, so such callers cannot use it.
//
// This entry point allocates nothing: its only work space is the file-scope
// array `g_noalloc_scratch` below (UNIFRAC_NOALLOC_MAX_CELLS u32 counts, 4 MB),
// which every GPU that loads this library holds until the process exits.  Its
// device address is looked up with the device current on every call made
// outside stream capture; a call enqueued on a capturing stream uses the
// address found by the last earlier call on that device (and is refused if
// there was none), so make one call on each device before any stream
// capture.  All calls share the array: calls that overlap on the GPU
// (different streams, or the same stream from several host threads without
// ordering) race and corrupt each other's results.  Nothing needs clearing
// between calls: the first kernel overwrites every cell it later reads.
#include <mutex>

#include "ufb_internal.cuh"

namespace ufb {
namespace {

constexpr size_t kMaxCells = UNIFRAC_NOALLOC_MAX_CELLS;
constexpr int kMaxSamples = UNIFRAC_NOALLOC_MAX_SAMPLES;
constexpr int kMaxDevices = 64;

// counts below each branch, node-major [n_nodes][n_samples] (4 MB)
static __device__ __align__(256) uint32_t g_noalloc_scratch[kMaxCells];

std::mutex g_setup_mutex;
uint32_t *g_scratch_ptr[kMaxDevices] = {nullptr};

// Sequential postorder accumulation, one thread per sample: copy the sample's
// column of counts (only tips may be non-zero), then add every node into its
// parent in postorder, so each node holds the count below its branch and the
// root holds the sample total.  A parent entry that is not a later node is
// skipped, so a malformed array gives wrong numbers but no stray access.
__global__ void k_noalloc_embed(int32_t n_nodes, const int32_t *__restrict__ parent,
                                int32_t n_samples, const uint32_t *__restrict__ tip_counts,
                                uint32_t *__restrict__ scratch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_samples) return;
  for (int32_t k = 0; k < n_nodes; ++k)
    scratch[(size_t)k * n_samples + i] = tip_counts[(size_t)k * n_samples + i];
  for (int32_t k = 0; k < n_nodes - 1; ++k) {
    const int32_t p = parent[k];
    if (p > k && p < n_nodes)
      scratch[(size_t)p * n_samples + i] += scratch[(size_t)k * n_samples + i];
  }
}

// One warp per pair i <= j of the upper triangle, diagonal included: warp t
// of the N (N + 1) / 2 takes row i, the largest with
// off(i) = i N - i (i - 1) / 2 <= t, and j = i + t - off(i).  FP64 sums over
// the non-root branches of the definition, warp-reduced; writes d into both
// halves of the full matrix, 0 on the diagonal.
__device__ __forceinline__ int64_t tri_offset(int64_t i, int64_t N) { return i * N - i * (i - 1) / 2; }

__global__ void k_noalloc_pairs(int variant, int32_t n_nodes, const double *__restrict__ length,
                                int32_t n_samples, const uint32_t *__restrict__ scratch,
                                double *__restrict__ out) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t N = n_samples;
  if (t >= N * (N + 1) / 2) return;
  // closed-form row (a root of i^2 - (2N + 1) i + 2t = 0), then exact
  // integer correction of the rounding
  const double b = 2.0 * (double)N + 1.0;
  int64_t i = (int64_t)((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
  i = i < 0 ? 0 : (i >= N ? N - 1 : i);
  while (i > 0 && tri_offset(i, N) > t) --i;
  while (i + 1 < N && tri_offset(i + 1, N) <= t) ++i;
  const int64_t j = i + (t - tri_offset(i, N));
  if (i == j) {
    if (lane == 0) out[i * N + i] = 0.0;
    return;
  }
  const uint32_t *root = scratch + (size_t)(n_nodes - 1) * n_samples;
  const double ci = (double)root[i], cj = (double)root[j];
  double num = 0.0, den = 0.0;
  for (int32_t br = lane; br < n_nodes - 1; br += 32) {
    const double L = length[br];
    const uint32_t xi = scratch[(size_t)br * n_samples + i];
    const uint32_t xj = scratch[(size_t)br * n_samples + j];
    if (variant == UNIFRAC_UNWEIGHTED) {
      const bool pi = xi != 0u, pj = xj != 0u;
      num += (pi != pj) ? L : 0.0;
      den += (pi || pj) ? L : 0.0;
    } else {
      const double wi = ci > 0.0 ? (double)xi / ci : 0.0;
      const double wj = cj > 0.0 ? (double)xj / cj : 0.0;
      num += L * fabs(wi - wj);
      den += L * (wi + wj);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, off);
    den += __shfl_xor_sync(0xffffffffu, den, off);
  }
  if (lane == 0) {
    const double d = den > 0.0 ? fmin(1.0, fmax(0.0, num / den)) : 0.0;
    out[i * N + j] = d;
    out[j * N + i] = d;
  }
}

}  // namespace
}  // namespace ufb

extern "C" int unifrac_dense_noalloc(int variant, int32_t n_nodes, const int32_t *parent,
                                     const double *length, int32_t n_samples,
                                     const uint32_t *tip_counts, double *out,
                                     void *cuda_stream) {
  using namespace ufb;
  if (variant != UNIFRAC_UNWEIGHTED && variant != UNIFRAC_WEIGHTED_NORMALIZED)
    return UNIFRAC_E_INVALID_ARG;
  if (n_nodes < 1 || n_samples < 0 || !parent || !length) return UNIFRAC_E_INVALID_ARG;
  if (n_samples == 0) return UNIFRAC_OK;
  if (!tip_counts || !out) return UNIFRAC_E_INVALID_ARG;
  if (n_samples > kMaxSamples || (size_t)n_nodes * (size_t)n_samples > kMaxCells)
    return UNIFRAC_E_UNSUPPORTED;  // beyond the fixed work space of this entry point
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return UNIFRAC_E_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // The array's device address: looked up again on every call made outside
  // stream capture (a device reset loads the module again, possibly at
  // another address), the cached value used while the stream is capturing.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return UNIFRAC_E_CUDA;
  uint32_t *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
      if (cap != cudaStreamCaptureStatusNone) return UNIFRAC_E_UNSUPPORTED;  // see the header
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
        return UNIFRAC_E_CUDA;
      g_scratch_ptr[dev] = static_cast<uint32_t *>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  // each launch's own status (cudaLaunchKernel returns it): an error left
  // pending by unrelated earlier work is neither reported nor cleared here,
  // and the second kernel is not launched when the first one failed
  {
    void *args[] = {&n_nodes, (void *)&parent, &n_samples, (void *)&tip_counts, &scratch};
    if (cudaLaunchKernel((const void *)k_noalloc_embed, dim3((n_samples + 127) / 128), dim3(128),
                         args, 0, st) != cudaSuccess)
      return UNIFRAC_E_CUDA;
  }
  const int64_t warps = (int64_t)n_samples * (n_samples + 1) / 2;
  void *args[] = {&variant, &n_nodes, (void *)&length, &n_samples, &scratch, &out};
  if (cudaLaunchKernel((const void *)k_noalloc_pairs, dim3((unsigned)((warps * 32 + 255) / 256)),
                       dim3(256), args, 0, st) != cudaSuccess)
    return UNIFRAC_E_CUDA;
  return UNIFRAC_OK;
}
