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
// Device: A = -1/2 D o D in FP32 with FP64 row sums (one pass over D), every
// A Q product (cuBLAS SGEMM, the pass over A that bounds the iteration), and
// the n x m FP64 work -- the centring terms, orthonormalisation by shifted
// CholeskyQR2 (the Gram matrix Y^T Y and Y R^-1 by DGEMM, the m x m Cholesky
// factor R and its inverse on the host; twice, the first factor shifted by a tiny
// multiple of the trace so that a rank-deficient Y still factors) and the
// Ritz products.  Host: only m x m work (Cholesky, the eigenproblem of
// Q^T B Q by the cyclic Jacobi method).
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
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

// Y = Yf - r s^T - 1 t^T + g 1 s^T in FP64 (column-major n x m): the
// double-centring terms of B Q = J A J Q added to the product A Q.
__global__ void k_centre(const float *__restrict__ Yf, const double *__restrict__ r,
                         const double *__restrict__ st, double g, int64_t n, int m,
                         double *__restrict__ Y) {
  const int64_t total = n * m;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = x % n;
    const int j = (int)(x / n);
    const double sj = st[j], tj = st[m + j];
    Y[x] = (double)Yf[x] - r[i] * sj - tj + g * sj;
  }
}

__global__ void k_to_float(const double *__restrict__ a, int64_t len, float *__restrict__ b) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < len;
       x += (int64_t)gridDim.x * blockDim.x)
    b[x] = (float)a[x];
}

// Upper Cholesky factor of the m x m FP64 matrix G (column-major): G = R^T R.
// shift > 0 adds shift * trace(G) / m to the diagonal first.  Pivots that are
// not positive (an exactly dependent column) become 1, leaving that column's
// remainder.  Output R column-major, zero below the diagonal.
std::vector<double> cholesky_upper(std::vector<double> G, int m, double shift) {
  double tr = 0.0;
  for (int a = 0; a < m; ++a) tr += G[(size_t)a * m + a];
  if (shift > 0.0)
    for (int a = 0; a < m; ++a) G[(size_t)a * m + a] += shift * tr / m + 1e-300;
  std::vector<double> R((size_t)m * m, 0.0);
  auto at = [m](std::vector<double> &M, int row, int col) -> double & { return M[(size_t)col * m + row]; };
  for (int j = 0; j < m; ++j) {
    double d = at(G, j, j);
    for (int l = 0; l < j; ++l) d -= at(R, l, j) * at(R, l, j);
    const double rjj = d > 0.0 ? std::sqrt(d) : 1.0;
    at(R, j, j) = rjj;
    for (int c = j + 1; c < m; ++c) {
      double v = at(G, j, c);
      for (int l = 0; l < j; ++l) v -= at(R, l, j) * at(R, l, c);
      at(R, j, c) = v / rjj;
    }
  }
  return R;
}

// Inverse of the upper triangular m x m matrix R (column-major), by back
// substitution column by column: R X = I.
std::vector<double> upper_inverse(const std::vector<double> &R, int m) {
  std::vector<double> X((size_t)m * m, 0.0);
  for (int c = 0; c < m; ++c) {
    for (int i = c; i >= 0; --i) {
      double v = i == c ? 1.0 : 0.0;
      for (int l = i + 1; l <= c; ++l) v -= R[(size_t)l * m + i] * X[(size_t)c * m + l];
      X[(size_t)c * m + i] = v / R[(size_t)i * m + i];
    }
  }
  return X;
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
  float *A = nullptr, *Qf = nullptr, *Yf = nullptr;
  double *Q = nullptr, *Y = nullptr, *W = nullptr, *r = nullptr, *ones = nullptr, *st = nullptr,
         *G = nullptr, *U = nullptr;
  cublasHandle_t h = nullptr;
  ~PcoaDev() {
    for (void *p : {(void *)A, (void *)Qf, (void *)Yf, (void *)Q, (void *)Y, (void *)W, (void *)r,
                    (void *)ones, (void *)st, (void *)G, (void *)U})
      if (p) cudaFree(p);
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
  const size_t nn = (size_t)n * n, nm = (size_t)n * m;
  if (cudaMalloc(&dv.A, nn * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&dv.Qf, nm * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&dv.Yf, nm * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&dv.Q, nm * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dv.Y, nm * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dv.W, nm * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dv.U, (size_t)n * k * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dv.r, (size_t)n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dv.ones, (size_t)n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dv.st, 2 * (size_t)m * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dv.G, (size_t)m * m * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return UNIFRAC_E_OOM;
  }
  if (cublasCreate(&dv.h) != CUBLAS_STATUS_SUCCESS || cublasSetStream(dv.h, st) != CUBLAS_STATUS_SUCCESS)
    return UNIFRAC_E_CUDA;
  if (precision == UNIFRAC_FP64)
    k_pcoa_square<double><<<n, 256, 0, st>>>(static_cast<const double *>(dist), n, dv.A, dv.r);
  else
    k_pcoa_square<float><<<n, 256, 0, st>>>(static_cast<const float *>(dist), n, dv.A, dv.r);
  if (cudaGetLastError() != cudaSuccess) return UNIFRAC_E_CUDA;
  std::vector<double> r(n), ones(n, 1.0);
  if (cudaMemcpyAsync(r.data(), dv.r, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(dv.ones, ones.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return UNIFRAC_E_CUDA;
  double g = 0.0;
  for (int32_t i = 0; i < n; ++i) g += r[i];
  g /= (double)n;
  const int grid = 148 * 8;
  const double d1 = 1.0, d0 = 0.0;

  // M <- M R^-1 with M^T M = R^T R (CholeskyQR): the Gram matrix and the
  // product with R^-1 are DGEMMs (their long dimension n parallelises; the
  // triangular routines only parallelise over the m x m output), the factor
  // and its inverse are m x m host work
  std::vector<double> Gh((size_t)m * m);
  auto cholqr = [&](double *&M, double shift) -> int {
    if (cublasDgemm(dv.h, CUBLAS_OP_T, CUBLAS_OP_N, m, m, n, &d1, M, n, M, n, &d0, dv.G, m) !=
        CUBLAS_STATUS_SUCCESS)
      return UNIFRAC_E_CUDA;
    if (cudaMemcpyAsync(Gh.data(), dv.G, Gh.size() * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return UNIFRAC_E_CUDA;
    for (int a = 0; a < m; ++a)  // exact symmetry
      for (int b = a + 1; b < m; ++b) Gh[(size_t)b * m + a] = Gh[(size_t)a * m + b];
    const std::vector<double> Rinv = upper_inverse(cholesky_upper(Gh, m, shift), m);
    if (cudaMemcpyAsync(dv.G, Rinv.data(), Rinv.size() * sizeof(double), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cublasDgemm(dv.h, CUBLAS_OP_N, CUBLAS_OP_N, n, m, m, &d1, M, n, dv.G, m, &d0, dv.W, n) !=
            CUBLAS_STATUS_SUCCESS ||
        cudaStreamSynchronize(st) != cudaSuccess)  // Rinv (host) is copied before it goes out of scope
      return UNIFRAC_E_CUDA;
    std::swap(M, dv.W);
    return UNIFRAC_OK;
  };
  auto orthonormalise = [&](double *&M) -> int {
    int rc = cholqr(M, 1e-13);  // shifted first pass: factors even a rank-deficient M
    return rc ? rc : cholqr(M, 0.0);
  };
  // Y = B Q = A Q - r (1^T Q) - 1 (r^T Q) + g 1 (1^T Q): the product in FP32
  // (SGEMM), the centring terms in FP64
  auto apply_B = [&]() -> int {
    k_to_float<<<grid, 256, 0, st>>>(dv.Q, (int64_t)nm, dv.Qf);
    const float one = 1.f, zero = 0.f;
    if (cublasSgemm(dv.h, CUBLAS_OP_N, CUBLAS_OP_N, n, m, n, &one, dv.A, n, dv.Qf, n, &zero, dv.Yf, n) !=
            CUBLAS_STATUS_SUCCESS ||
        cublasDgemv(dv.h, CUBLAS_OP_T, n, m, &d1, dv.Q, n, dv.ones, 1, &d0, dv.st, 1) !=
            CUBLAS_STATUS_SUCCESS ||
        cublasDgemv(dv.h, CUBLAS_OP_T, n, m, &d1, dv.Q, n, dv.r, 1, &d0, dv.st + m, 1) !=
            CUBLAS_STATUS_SUCCESS)
      return UNIFRAC_E_CUDA;
    k_centre<<<grid, 256, 0, st>>>(dv.Yf, dv.r, dv.st, g, n, m, dv.Y);
    return cudaGetLastError() == cudaSuccess ? UNIFRAC_OK : UNIFRAC_E_CUDA;
  };

  // random start (SplitMix64 stream from the seed), orthonormal columns
  {
    std::vector<double> Q0(nm);
    for (size_t x = 0; x < nm; ++x)
      Q0[x] = (double)(splitmix64(seed ^ splitmix64(x)) >> 11) * 0x1.0p-52 - 1.0;
    if (cudaMemcpyAsync(dv.Q, Q0.data(), nm * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return UNIFRAC_E_CUDA;
  }
  int rc;
  if ((rc = orthonormalise(dv.Q))) return rc;
  for (int it = 0; it < iters; ++it) {
    if ((rc = apply_B())) return rc;
    std::swap(dv.Q, dv.Y);
    if ((rc = orthonormalise(dv.Q))) return rc;
  }
  // Rayleigh-Ritz: T = Q^T B Q (symmetrised), eigenpairs, U = Q W
  if ((rc = apply_B())) return rc;
  if (cublasDgemm(dv.h, CUBLAS_OP_T, CUBLAS_OP_N, m, m, n, &d1, dv.Q, n, dv.Y, n, &d0, dv.G, m) !=
      CUBLAS_STATUS_SUCCESS)
    return UNIFRAC_E_CUDA;
  std::vector<double> Th((size_t)m * m);
  if (cudaMemcpyAsync(Th.data(), dv.G, Th.size() * sizeof(double), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return UNIFRAC_E_CUDA;
  std::vector<double> T((size_t)m * m);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b)
      T[(size_t)a * m + b] = 0.5 * (Th[(size_t)b * m + a] + Th[(size_t)a * m + b]);
  std::vector<double> W;
  std::vector<double> theta = jacobi_eigen(T, m, W);
  std::vector<int> order(m);
  for (int a = 0; a < m; ++a) order[a] = a;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return theta[a] > theta[b]; });
  // U = Q W_k (device), coordinates U sqrt(max(theta, 0)) (host)
  std::vector<double> Wk((size_t)m * k);  // column-major m x k
  for (int c = 0; c < k; ++c)
    for (int a = 0; a < m; ++a) Wk[(size_t)c * m + a] = W[(size_t)a * m + order[c]];
  std::vector<double> Uh((size_t)n * k);
  if (cudaMemcpyAsync(dv.G, Wk.data(), Wk.size() * sizeof(double), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cublasDgemm(dv.h, CUBLAS_OP_N, CUBLAS_OP_N, n, k, m, &d1, dv.Q, n, dv.G, m, &d0, dv.U, n) !=
          CUBLAS_STATUS_SUCCESS ||
      cudaMemcpyAsync(Uh.data(), dv.U, Uh.size() * sizeof(double), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return UNIFRAC_E_CUDA;
  for (int c = 0; c < k; ++c) {
    eigvals[c] = theta[order[c]];
    const double sc = std::sqrt(std::max(theta[order[c]], 0.0));
    for (int32_t i = 0; i < n; ++i) coords[(size_t)i * k + c] = Uh[(size_t)c * n + i] * sc;
  }
  return UNIFRAC_OK;
}
