// unifrac_measure_peak: measured issue rate of one arithmetic pipe on this
// GPU, the ceiling the pair kernels' work is compared against.
//
// The weighted pair kernel does two FP32 operations per pair-branch update
// (a min and an add), the plain FP64 kernels one or two FP64 operations; the
// ceilings of those kernels are the FP32 and FP64 pipe rates at the clock the
// GPU actually runs.  Nominal unit counts do not give the FP64 rate of this
// chip, so it is measured: every thread of a full-occupancy grid (a multiple
// of the SM count) runs a long chain of fused multiply-adds on eight
// independent accumulators (enough independent work to cover the pipe's
// latency), and the rate is the number of FMA instructions per second between
// two CUDA events.  One FMA counts as one operation.
#include <algorithm>

#include "ufb_internal.cuh"

namespace ufb {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakAcc = 8;

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_chain(int32_t iters, T b, T c, T *__restrict__ sink) {
  T a[kPeakAcc];
#pragma unroll
  for (int q = 0; q < kPeakAcc; ++q) a[q] = (T)(threadIdx.x + q);
  for (int32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kPeakAcc; ++q) a[q] = fma_rn(a[q], b, c);
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < kPeakAcc; ++q) s += a[q];
  // b is 1 and c is 0 at run time, so s is a small integer: the store never
  // happens, but the compiler cannot know that and keeps the chain
  if (s == (T)-1) sink[blockIdx.x] = s;
}

template <typename T>
int time_chain(int32_t iters, int blocks, cudaStream_t st, T *sink, float *ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    k_fma_chain<T><<<blocks, kPeakThreads, 0, st>>>(iters, (T)1, (T)0, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e == cudaSuccess ? UNIFRAC_OK : UNIFRAC_E_CUDA;
}

template <typename T>
int measure(cudaStream_t st, double *ops_per_s) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chain<T>, kPeakThreads, 0) !=
          cudaSuccess)
    return UNIFRAC_E_CUDA;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  T *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T) * blocks) != cudaSuccess) return UNIFRAC_E_OOM;
  // a short run to size the timed one to about 20 ms, a warm-up, then the
  // best of three
  int rc;
  float ms = 0.f;
  int32_t iters = 256;
  if ((rc = time_chain<T>(iters, blocks, st, sink, &ms)) == UNIFRAC_OK) {
    const double scale = ms > 0.f ? 20.0 / ms : 64.0;
    iters = (int32_t)std::min(1.0e8, std::max(256.0, iters * scale));
    rc = time_chain<T>(iters, blocks, st, sink, &ms);
  }
  float best = 1e30f;
  for (int rep = 0; rc == UNIFRAC_OK && rep < 3; ++rep) {
    rc = time_chain<T>(iters, blocks, st, sink, &ms);
    if (ms > 0.f) best = std::min(best, ms);
  }
  cudaFree(sink);
  if (rc != UNIFRAC_OK) return rc;
  *ops_per_s = (double)blocks * kPeakThreads * kPeakAcc * (double)iters / (best * 1e-3);
  return UNIFRAC_OK;
}

}  // namespace
}  // namespace ufb

extern "C" int unifrac_measure_peak(int pipe, double *ops_per_s, void *cuda_stream) {
  using namespace ufb;
  if (!ops_per_s) return UNIFRAC_E_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (pipe == UNIFRAC_PEAK_FP32_FMA) return measure<float>(st, ops_per_s);
  if (pipe == UNIFRAC_PEAK_FP64_FMA) return measure<double>(st, ops_per_s);
  return UNIFRAC_E_INVALID_ARG;
}
