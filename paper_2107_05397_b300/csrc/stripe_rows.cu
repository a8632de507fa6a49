// Stripes to row runs, for the streamed output (the paper, Section II: the
// matrix is computed as stripes that are merged into the whole afterwards).
//
// Stripe s holds d(k, (k + s + 1) mod n) at element k.  A chunk of L stripes
// [s0, s0 + L) covers, in row i of the full matrix, the cyclic diagonals
// i + d and i - d for d in [s0 + 1, s0 + L]: two cyclic runs of L columns,
//   up run:   columns (i + s0 + 1 + t) mod n,    t = 0 .. L-1,  value C[t][i]
//   down run: columns (i - s0 - L + t') mod n,   t' = 0 .. L-1,
//             value C[u][(i - s0 - 1 - u) mod n] with u = L - 1 - t'
// (C[u][k]: element k of the chunk's stripe u).  This kernel writes both
// runs of every row, row-major (up[i][t], down[i][t']), so that the host
// places whole contiguous runs (at most four per row) instead of single
// elements read down the chunk's columns.
//
// The up runs are a transpose of the chunk, the down runs a sheared one:
// a block stages a 32 x 64 window of the chunk in shared memory, read along
// its rows (coalesced) and written along the output rows (coalesced).
#include "ufb_internal.cuh"

namespace ufb {
namespace {

constexpr int kTileR = 32;  // output rows per block
constexpr int kTileS = 32;  // stripes per block
constexpr int kRowsPerPass = 8;

// blockIdx.z = 2 v + (0: up runs, 1: down runs)
template <typename T>
__global__ void __launch_bounds__(kTileS * kRowsPerPass)
    k_stripe_rows(const T *__restrict__ chunk, int32_t n, int32_t L, int32_t s0,
                  T *__restrict__ up, T *__restrict__ down) {
  // up: [stripe][32 rows], row stride 33; down: [stripe][64-wide window], row
  // stride 66: both read across stripes hit 32 different banks
  constexpr int kUpLd = kTileR + 1, kDownLd = 2 * kTileR + 2;
  __shared__ T tile[kTileS * kDownLd];
  const int v = blockIdx.z >> 1;
  const bool is_down = (blockIdx.z & 1) != 0;
  const int64_t i0 = (int64_t)blockIdx.x * kTileR;
  const int u0 = blockIdx.y * kTileS;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const T *C = chunk + (int64_t)v * L * n;
  if (!is_down) {
    for (int uu = ty; uu < kTileS; uu += kRowsPerPass) {
      const int u = u0 + uu;
      const int64_t k = i0 + tx;
      if (u < L && k < n) tile[uu * kUpLd + tx] = C[(int64_t)u * n + k];
    }
    __syncthreads();
    T *U = up + (int64_t)v * n * L;
    for (int ii = ty; ii < kTileR; ii += kRowsPerPass) {
      const int64_t i = i0 + ii;
      const int u = u0 + tx;
      if (i < n && u < L) U[i * L + u] = tile[tx * kUpLd + ii];
    }
  } else {
    // window element m of stripe u0 + uu is C[u0 + uu][(kb + m) mod n],
    // kb = i0 - s0 - 1 - u0 - 31; output (i0 + ii, u0 + uu) reads m = ii - uu + 31
    const int64_t kb = i0 - s0 - 1 - u0 - (kTileS - 1);
    for (int uu = ty; uu < kTileS; uu += kRowsPerPass) {
      const int u = u0 + uu;
      if (u >= L) continue;
      for (int m = tx; m < 2 * kTileR - 1; m += kTileS) {
        int64_t k = (kb + m) % n;
        if (k < 0) k += n;
        tile[uu * kDownLd + m] = C[(int64_t)u * n + k];
      }
    }
    __syncthreads();
    T *D = down + (int64_t)v * n * L;
    for (int ii = ty; ii < kTileR; ii += kRowsPerPass) {
      const int64_t i = i0 + ii;
      const int u = u0 + tx;
      if (i < n && u < L) D[i * L + (L - 1 - u)] = tile[tx * kDownLd + ii - tx + (kTileS - 1)];
    }
  }
}

}  // namespace

int stripe_rows(unifrac_ctx *ctx, const void *chunk, int32_t n, int32_t L, int32_t s0, int nv,
                bool f64, void *up, void *down) {
  if (n <= 0 || L <= 0) return UNIFRAC_OK;
  const dim3 grid((unsigned)((n + kTileR - 1) / kTileR), (unsigned)((L + kTileS - 1) / kTileS),
                  (unsigned)(2 * nv));
  const dim3 block(kTileS, kRowsPerPass);
  if (f64)
    k_stripe_rows<double><<<grid, block, 0, ctx->stream>>>(
        static_cast<const double *>(chunk), n, L, s0, static_cast<double *>(up),
        static_cast<double *>(down));
  else
    k_stripe_rows<float><<<grid, block, 0, ctx->stream>>>(
        static_cast<const float *>(chunk), n, L, s0, static_cast<float *>(up),
        static_cast<float *>(down));
  ctx->stat_launches += 1;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stripe rows");
  return UNIFRAC_OK;
}

}  // namespace ufb
