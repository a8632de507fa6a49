// unifrac_pcoa: principal coordinates analysis of a full distance matrix on
// the GPU -- the ordination the UniFrac matrix feeds (the paper, Sections I
// and II, places the matrix in that pipeline).
//
// Classical PCoA: A = -1/2 (D o D), B = J A J with J = I - 11^T/n, the k
// largest eigenpairs of B, coordinates U_k sqrt(max(lambda_k, 0)).  B is never
// formed: with r the row means of A (A is symmetric) and g their mean,
//   B Q = A Q - r (1^T Q) - 1 (r^T Q) + g 1 (1^T Q).
// The eigenpairs come from subspace iteration with a seeded random start of
// m = 2k + 16 columns: Y = B Q, Q = orth(Y), repeated; then the
// Rayleigh-Ritz step T = Q^T B Q, T = W diag(theta) W^T, U = Q W.
//
// Device: the n x n work -- A = -1/2 D o D in FP32 with FP64 row sums (one
// pass over D), and every A Q product (cuBLAS SGEMM, the one plain GEMM of
// the path).  Host threads: the n x m work in FP64 -- the centring terms,
// orthonormalisation by shifted CholeskyQR2 (a Cholesky factor of the Gram
// matrix Y^T Y, twice; the first shifted by a tiny multiple of its trace so
// that a rank-deficient Y still factors), and the m x m eigenproblem by the
// cyclic Jacobi method.
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "ufb_internal.cuh"

namespace ufb {
namespace {

// A = -1/2 D o D (FP32) and the row means of A (FP64), one CTA per row.
template <typename TD>
__global__ void __launch_bounds__(256) k_pcoa_square(const TD *__restrict__ D, int64_t n,
                                                     float *__restrict__ A,
                                                     double *__restrict__ rowmean) {
  __shared__ double red[8];
  const int64_t i = blockIdx.x;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double d = (double)D[i * n + j];
    const double a = -0.5 * d * d;
    A[i * n + j] = (float)a;
    s += a;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    rowmean[i] = t / (double)n;
  }
}

// SplitMix64 (Steele, Lea and Flood 2014): the counter-based generator of the
// random start, uniform in [-1, 1).
uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

template <typename F>
void parallel_rows(int64_t n, F &&fn) {  // fn(lo, hi, thread) over row ranges
  const unsigned hw = std::thread::hardware_concurrency();
  const int T = n < 4096 ? 1 : (int)std::max(1u, std::min(32u, hw ? hw : 1u));
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) th.emplace_back(fn, n * t / T, n * (t + 1) / T, t);
  fn((int64_t)0, n / T, 0);
  for (auto &x : th) x.join();
}

// Gram matrix G = Y^T Y of the column-major n x m matrix Y (FP64).
std::vector<double> gram(const std::vector<double> &Y, int64_t n, int m) {
  const unsigned hw = std::thread::hardware_concurrency();
  const int T = n < 4096 ? 1 : (int)std::max(1u, std::min(32u, hw ? hw : 1u));
  std::vector<std::vector<double>> part(T, std::vector<double>((size_t)m * m, 0.0));
  parallel_rows(n, [&](int64_t lo, int64_t hi, int t) {
    std::vector<double> &P = part[t];
    for (int a = 0; a < m; ++a)
      for (int b = a; b < m; ++b) {
        double s = 0.0;
        const double *ya = &Y[(size_t)a * n], *yb = &Y[(size_t)b * n];
        for (int64_t i = lo; i < hi; ++i) s += ya[i] * yb[i];
        P[(size_t)a * m + b] += s;
      }
  });
  std::vector<double> G((size_t)m * m, 0.0);
  for (int t = 0; t < T; ++t)
    for (int a = 0; a < m; ++a)
      for (int b = a; b < m; ++b) G[(size_t)a * m + b] += part[t][(size_t)a * m + b];
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < a; ++b) G[(size_t)a * m + b] = G[(size_t)b * m + a];
  return G;
}

// One CholeskyQR step: G = R^T R, Y <- Y R^{-1}.  shift > 0 adds
// shift * trace(G) / m to the diagonal first.  Pivots that are not positive
// (an exactly dependent column) become 1, leaving that column's remainder.
void cholesky_qr(std::vector<double> &Y, int64_t n, int m, double shift) {
  std::vector<double> G = gram(Y, n, m);
  double tr = 0.0;
  for (int a = 0; a < m; ++a) tr += G[(size_t)a * m + a];
  if (shift > 0.0)
    for (int a = 0; a < m; ++a) G[(size_t)a * m + a] += shift * tr / m + 1e-300;
  std::vector<double> R((size_t)m * m, 0.0);  // upper triangular, row-major
  for (int j = 0; j < m; ++j) {
    double d = G[(size_t)j * m + j];
    for (int l = 0; l < j; ++l) d -= R[(size_t)l * m + j] * R[(size_t)l * m + j];
    const double rjj = d > 0.0 ? std::sqrt(d) : 1.0;
    R[(size_t)j * m + j] = rjj;
    for (int c = j + 1; c < m; ++c) {
      double v = G[(size_t)j * m + c];
      for (int l = 0; l < j; ++l) v -= R[(size_t)l * m + j] * R[(size_t)l * m + c];
      R[(size_t)j * m + c] = v / rjj;
    }
  }
  // rows of Y solve x R = y (forward substitution)
  parallel_rows(n, [&](int64_t lo, int64_t hi, int) {
    std::vector<double> x(m);
    for (int64_t i = lo; i < hi; ++i) {
      for (int j = 0; j < m; ++j) {
        double v = Y[(size_t)j * n + i];
        for (int l = 0; l < j; ++l) v -= x[l] * R[(size_t)l * m + j];
        x[j] = v / R[(size_t)j * m + j];
      }
      for (int j = 0; j < m; ++j) Y[(size_t)j * n + i] = x[j];
    }
  });
}

void orthonormalise(std::vector<double> &Y, int64_t n, int m) {
  cholesky_qr(Y, n, m, 1e-13);
  cholesky_qr(Y, n, m, 0.0);
}

// Cyclic Jacobi eigenvalue method (rotations zeroing each off-diagonal entry
// in turn; Golub and Van Loan, Matrix Computations, 8.5) for the symmetric
// m x m matrix T (row-major, destroyed).  Returns eigenvalues; V (row-major,
// columns = eigenvectors).
std::vector<double> jacobi_eigen(std::vector<double> &T, int m, std::vector<double> &V) {
  V.assign((size_t)m * m, 0.0);
  for (int a = 0; a < m; ++a) V[(size_t)a * m + a] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        const double x = T[(size_t)a * m + b] * T[(size_t)a * m + b];
        tot += x;
        if (a != b) off += x;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = T[(size_t)p * m + q];
        if (apq == 0.0) continue;
        const double app = T[(size_t)p * m + p], aqq = T[(size_t)q * m + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {  // T <- J^T T J
          const double tkp = T[(size_t)k * m + p], tkq = T[(size_t)k * m + q];
          T[(size_t)k * m + p] = c * tkp - s * tkq;
          T[(size_t)k * m + q] = s * tkp + c * tkq;
        }
        for (int k = 0; k < m; ++k) {
          const double tpk = T[(size_t)p * m + k], tqk = T[(size_t)q * m + k];
          T[(size_t)p * m + k] = c * tpk - s * tqk;
          T[(size_t)q * m + k] = s * tpk + c * tqk;
        }
        for (int k = 0; k < m; ++k) {  // V <- V J
          const double vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
          V[(size_t)k * m + p] = c * vkp - s * vkq;
          V[(size_t)k * m + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<double> w(m);
  for (int a = 0; a < m; ++a) w[a] = T[(size_t)a * m + a];
  return w;
}

struct PcoaDev {
  float *A = nullptr, *Q = nullptr, *Y = nullptr;
  double *rowmean = nullptr;
  cublasHandle_t h = nullptr;
  ~PcoaDev() {
    if (A) cudaFree(A);
    if (Q) cudaFree(Q);
    if (Y) cudaFree(Y);
    if (rowmean) cudaFree(rowmean);
    if (h) cublasDestroy(h);
  }
};

}  // namespace
}  // namespace ufb

extern "C" int unifrac_pcoa(const void *dist, int precision, int32_t n, int32_t k, int32_t iters,
                            uint64_t seed, double *eigvals, double *coords, void *cuda_stream) {
  using namespace ufb;
  if (!dist || !eigvals || !coords || n < 1 || k < 1 || k > n || iters < 0)
    return UNIFRAC_E_INVALID_ARG;
  if (precision != UNIFRAC_FP64 && precision != UNIFRAC_MIXED) return UNIFRAC_E_INVALID_ARG;
  // oversampled subspace: component c converges as (lambda_{m+1} / lambda_c)^iters,
  // and UniFrac spectra decay slowly, so the subspace is wide (the products
  // with A cost about the same for any m of this size: they stream A)
  const int m = std::min<int>(n, 2 * k + 16);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  PcoaDev dv;
  const size_t nn = (size_t)n * n;
  if (cudaMalloc(&dv.A, nn * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&dv.Q, (size_t)n * m * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&dv.Y, (size_t)n * m * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&dv.rowmean, (size_t)n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return UNIFRAC_E_OOM;
  }
  if (cublasCreate(&dv.h) != CUBLAS_STATUS_SUCCESS || cublasSetStream(dv.h, st) != CUBLAS_STATUS_SUCCESS)
    return UNIFRAC_E_CUDA;
  if (precision == UNIFRAC_FP64)
    k_pcoa_square<double><<<n, 256, 0, st>>>(static_cast<const double *>(dist), n, dv.A, dv.rowmean);
  else
    k_pcoa_square<float><<<n, 256, 0, st>>>(static_cast<const float *>(dist), n, dv.A, dv.rowmean);
  if (cudaGetLastError() != cudaSuccess) return UNIFRAC_E_CUDA;
  std::vector<double> r(n);
  if (cudaMemcpyAsync(r.data(), dv.rowmean, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return UNIFRAC_E_CUDA;
  double g = 0.0;
  for (int32_t i = 0; i < n; ++i) g += r[i];
  g /= (double)n;

  // random start, orthonormal columns (column-major n x m)
  std::vector<double> Q((size_t)n * m), Y((size_t)n * m);
  for (size_t x = 0; x < Q.size(); ++x)
    Q[x] = (double)(splitmix64(seed ^ splitmix64(x)) >> 11) * 0x1.0p-52 - 1.0;
  orthonormalise(Q, n, m);
  std::vector<float> buf((size_t)n * m);
  // Y = B Q: device product A Q, host centring terms
  auto apply_B = [&]() -> int {
    for (size_t x = 0; x < buf.size(); ++x) buf[x] = (float)Q[x];
    if (cudaMemcpyAsync(dv.Q, buf.data(), buf.size() * sizeof(float), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return UNIFRAC_E_CUDA;
    const float one = 1.f, zero = 0.f;
    if (cublasSgemm(dv.h, CUBLAS_OP_N, CUBLAS_OP_N, n, m, n, &one, dv.A, n, dv.Q, n, &zero, dv.Y, n) !=
        CUBLAS_STATUS_SUCCESS)
      return UNIFRAC_E_CUDA;
    if (cudaMemcpyAsync(buf.data(), dv.Y, buf.size() * sizeof(float), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return UNIFRAC_E_CUDA;
    std::vector<double> s(m, 0.0), t(m, 0.0);  // 1^T Q and r^T Q
    for (int j = 0; j < m; ++j)
      for (int32_t i = 0; i < n; ++i) {
        s[j] += Q[(size_t)j * n + i];
        t[j] += r[i] * Q[(size_t)j * n + i];
      }
    parallel_rows(n, [&](int64_t lo, int64_t hi, int) {
      for (int j = 0; j < m; ++j)
        for (int64_t i = lo; i < hi; ++i)
          Y[(size_t)j * n + i] = (double)buf[(size_t)j * n + i] - r[i] * s[j] - t[j] + g * s[j];
    });
    return UNIFRAC_OK;
  };
  int rc;
  for (int it = 0; it < iters; ++it) {
    if ((rc = apply_B())) return rc;
    Q.swap(Y);
    orthonormalise(Q, n, m);
  }
  // Rayleigh-Ritz: T = Q^T B Q (symmetrised), eigenpairs, U = Q W
  if ((rc = apply_B())) return rc;
  std::vector<double> T((size_t)m * m, 0.0);
  for (int a = 0; a < m; ++a)
    for (int b = a; b < m; ++b) {
      double v = 0.0;
      for (int32_t i = 0; i < n; ++i) v += 0.5 * (Q[(size_t)a * n + i] * Y[(size_t)b * n + i] +
                                                  Q[(size_t)b * n + i] * Y[(size_t)a * n + i]);
      T[(size_t)a * m + b] = T[(size_t)b * m + a] = v;
    }
  std::vector<double> W;
  std::vector<double> theta = jacobi_eigen(T, m, W);
  std::vector<int> order(m);
  for (int a = 0; a < m; ++a) order[a] = a;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return theta[a] > theta[b]; });
  for (int c = 0; c < k; ++c) eigvals[c] = theta[order[c]];
  parallel_rows(n, [&](int64_t lo, int64_t hi, int) {
    for (int64_t i = lo; i < hi; ++i)
      for (int c = 0; c < k; ++c) {
        const int col = order[c];
        double u = 0.0;
        for (int a = 0; a < m; ++a) u += Q[(size_t)a * n + i] * W[(size_t)a * m + col];
        coords[(size_t)i * k + c] = u * std::sqrt(std::max(theta[col], 0.0));
      }
  });
  return UNIFRAC_OK;
}
