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
// Neither A nor B is stored: the product A Q reads D itself and forms each
// a = -1/2 d^2 as it goes (k_pcoa_dq), so each iteration is one pass over D
// (4 n^2 bytes in FP32) and the call holds only O(n m) device memory.  A is
// symmetric, so row i of A Q is the sum over j of A[j][i] Q[j][.]: a CTA
// owning 128 output rows streams the 128-wide column panel of D, each row j
// of the panel a contiguous, coalesced 512-byte segment.  Sums are FP32
// within a chunk of j and FP64 across chunks (k_pcoa_reduce, which also adds
// the centring terms).  The n x m FP64 work is on the device too: Gram
// products X^T Z (k_xtz_partial / k_xtz_reduce: CholeskyQR2's Y^T Y, the
// centring's Q^T 1 and Q^T r, the Ritz matrix Q^T Y) and products with small
// m x q matrices (k_x_times_s: Y R^-1, Q W).  Host: only m x m work (the
// Cholesky factor and its inverse, the eigenproblem of Q^T B Q by the cyclic
// Jacobi method).
#include <algorithm>
#include <cmath>
#include <vector>

#include "ufb_internal.cuh"

namespace ufb {
namespace {

// Row means of A = -1/2 D o D (FP64), one CTA per row.
template <typename TD>
__global__ void __launch_bounds__(256) k_pcoa_rowmean(const TD *__restrict__ D, int64_t n,
                                                      double *__restrict__ rowmean) {
  __shared__ double red[8];
  const int64_t i = blockIdx.x;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double d = (double)D[i * n + j];
    s += -0.5 * d * d;
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

// ---- Y = A Q from D (the pass over D of every iteration)
//
// CTA = 4 warps over a 128-row output panel [i0, i0 + 128) and 4 CW columns
// [c0, c0 + 4 CW) of Q: lane l of warp w accumulates rows i0 + 4l .. 4l + 3
// and columns c0 + w CW .. + CW - 1 in FP32 registers, over the rows j of
// one chunk [j0, j1) of D.  Per step of kBJ rows j, the CTA stages
// a = -1/2 d^2 of D[j][i0 .. i0 + 127] (the panel row, contiguous) and
// Qt[j][c0 .. c0 + 4 CW) in shared memory; a lane then reads its 4 a values
// as one 16-byte load and its CW values of Qt by broadcast, and issues 4 CW
// FMAs per j.  The partial sums of chunk kc go to Yp[kc][i][c] (FP32, rows
// padded to mp columns).
__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

constexpr int kDqRows = 128;
constexpr int kDqThreads = 128;
constexpr int kBJ = 32;

template <typename TD>
__device__ __forceinline__ float a_of(TD d) {
  const float f = (float)d;
  return -0.5f * f * f;
}

// four consecutive values (16-byte aligned FP32, two 16-byte FP64 loads)
__device__ __forceinline__ void load4(const float *p, float (&v)[4]) {
  const float4 x = __ldg(reinterpret_cast<const float4 *>(p));
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void load4(const double *p, double (&v)[4]) {
  const double2 x = __ldg(reinterpret_cast<const double2 *>(p));
  const double2 y = __ldg(reinterpret_cast<const double2 *>(p + 2));
  v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

template <typename TD, int CW>
__global__ void __launch_bounds__(kDqThreads) k_pcoa_dq(const TD *__restrict__ D, int32_t n,
                                                        const float *__restrict__ Qt, int32_t mp,
                                                        int32_t m, int32_t chunk,
                                                        float *__restrict__ Yp) {
  __shared__ __align__(16) float sA[kBJ][kDqRows];
  __shared__ __align__(16) float sQ[kBJ][4 * CW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * kDqRows;
  const int64_t j0 = (int64_t)blockIdx.y * chunk;
  const int64_t j1 = min64(j0 + chunk, n);
  const int c0 = blockIdx.z * 4 * CW;
  // vector loads need every row start aligned: n a multiple of 4 (the base
  // pointer is checked on the host)
  const bool vec_ok = (n & 3) == 0;
  float acc[4][CW];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < CW; ++c) acc[q][c] = 0.f;
  for (int64_t jb = j0; jb < j1; jb += kBJ) {
    // stage the panel rows: thread t takes columns 4 (t % 32) .. + 3 of rows
    // t / 32, t / 32 + 4, ... (a warp reads one 512-byte row segment)
    {
      constexpr int kRowsPerThread = kBJ / (kDqThreads / 32);
      const int cq = (threadIdx.x & 31) * 4;
      const int rbase = threadIdx.x >> 5;
      // every row's load issued before the first store (one round trip)
      TD v[kRowsPerThread][4];
#pragma unroll
      for (int u = 0; u < kRowsPerThread; ++u) {
        const int64_t j = jb + rbase + u * (kDqThreads / 32);
        const TD *row = D + j * (int64_t)n + i0 + cq;
        if (j < j1 && vec_ok && i0 + cq + 3 < n) {
          load4(row, v[u]);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) v[u][e] = (j < j1 && i0 + cq + e < n) ? row[e] : (TD)0;
        }
      }
#pragma unroll
      for (int u = 0; u < kRowsPerThread; ++u)
        *reinterpret_cast<float4 *>(&sA[rbase + u * (kDqThreads / 32)][cq]) =
            make_float4(a_of(v[u][0]), a_of(v[u][1]), a_of(v[u][2]), a_of(v[u][3]));
    }
    for (int x = threadIdx.x; x < kBJ * 4 * CW; x += kDqThreads) {
      const int r = x / (4 * CW), c = x % (4 * CW);
      const int64_t j = jb + r;
      sQ[r][c] = (j < j1 && c0 + c < m) ? Qt[j * mp + c0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < kBJ; ++r) {
      const float4 a4 = *reinterpret_cast<const float4 *>(&sA[r][lane * 4]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        const float qv = sQ[r][warp * CW + c];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q][c] = __fmaf_rn(av[q], qv, acc[q][c]);
      }
    }
    __syncthreads();
  }
  float *dst = Yp + (int64_t)blockIdx.y * n * mp;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + lane * 4 + q;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      const int col = c0 + warp * CW + c;
      if (col < m) dst[(int64_t)i * mp + col] = acc[q][c];
    }
  }
}

// Y[i + c n] = sum_kc Yp[kc][i][c] (FP64, chunk order) - r_i s_c - t_c + g s_c:
// the chunks' partial products of A Q summed, plus the double-centring terms
// of B Q (s = Q^T 1, t = Q^T r).  Y column-major n x m, FP64.
__global__ void k_pcoa_reduce(const float *__restrict__ Yp, int32_t kc, int64_t n, int32_t mp,
                              int32_t m, const double *__restrict__ r,
                              const double *__restrict__ s, const double *__restrict__ t,
                              double g, double *__restrict__ Y) {
  const int64_t total = n * m;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = x / m;
    const int c = (int)(x % m);
    double v = 0.0;
    for (int k = 0; k < kc; ++k) v += (double)Yp[((int64_t)k * n + i) * mp + c];
    Y[(int64_t)c * n + i] = v - r[i] * s[c] - t[c] + g * s[c];
  }
}

// Qt[i][c] = (float)Q[i + c n]: the FP32, row-major copy of Q that k_pcoa_dq
// reads (rows padded to mp columns, zeros beyond m).
__global__ void k_pcoa_qt(const double *__restrict__ Q, int64_t n, int32_t m, int32_t mp,
                          float *__restrict__ Qt) {
  const int64_t total = n * mp;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = x / mp;
    const int c = (int)(x % mp);
    Qt[x] = c < m ? (float)Q[(int64_t)c * n + i] : 0.f;
  }
}

// ---- FP64 products of tall n x m matrices (column-major)
//
// C = X^T Z, X n x p, Z n x q: CTA (x, y) sums rows [x R, (x + 1) R) for the
// entries e = y 2048 + tid + 256 u (u < 8) of the p x q result (entry e is
// (e % p, e / p)), staging kXtzRows rows of X and Z at a time in shared
// memory; partials P[x][e], summed over x in order by k_xtz_reduce.
constexpr int kXtzThreads = 256;
constexpr int kXtzPer = 8;
constexpr int kXtzRows = 16;

__global__ void __launch_bounds__(kXtzThreads) k_xtz_partial(const double *__restrict__ X,
                                                             const double *__restrict__ Z,
                                                             int64_t n, int32_t p, int32_t q,
                                                             int64_t rows_per_cta,
                                                             double *__restrict__ P) {
  extern __shared__ __align__(16) double xz[];  // [kXtzRows][p], then [kXtzRows][q]
  double *sX = xz, *sZ = xz + (size_t)kXtzRows * p;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = min64(r0 + rows_per_cta, n);
  const int64_t pq = (int64_t)p * q;
  int ea[kXtzPer], eb[kXtzPer];
  double acc[kXtzPer];
#pragma unroll
  for (int u = 0; u < kXtzPer; ++u) {
    const int64_t e = (int64_t)blockIdx.y * kXtzThreads * kXtzPer + threadIdx.x + u * kXtzThreads;
    ea[u] = e < pq ? (int)(e % p) : -1;
    eb[u] = e < pq ? (int)(e / p) : 0;
    acc[u] = 0.0;
  }
  for (int64_t rb = r0; rb < r1; rb += kXtzRows) {
    const int nr = (int)min64(kXtzRows, r1 - rb);
    for (int x = threadIdx.x; x < kXtzRows * p; x += kXtzThreads) {
      const int rr = x % kXtzRows, a = x / kXtzRows;  // consecutive threads: consecutive rows
      sX[rr * p + a] = rr < nr ? X[(int64_t)a * n + rb + rr] : 0.0;
    }
    for (int x = threadIdx.x; x < kXtzRows * q; x += kXtzThreads) {
      const int rr = x % kXtzRows, b = x / kXtzRows;
      sZ[rr * q + b] = rr < nr ? Z[(int64_t)b * n + rb + rr] : 0.0;
    }
    __syncthreads();
    for (int rr = 0; rr < nr; ++rr) {
#pragma unroll
      for (int u = 0; u < kXtzPer; ++u)
        if (ea[u] >= 0) acc[u] = fma(sX[rr * p + ea[u]], sZ[rr * q + eb[u]], acc[u]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < kXtzPer; ++u)
    if (ea[u] >= 0) P[(int64_t)blockIdx.x * pq + (int64_t)eb[u] * p + ea[u]] = acc[u];
}

// C[e] = sum over the row blocks x of P[x][e] (in order); C column-major p x q.
__global__ void k_xtz_reduce(const double *__restrict__ P, int32_t blocks, int64_t pq,
                             double *__restrict__ C) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < pq;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int x = 0; x < blocks; ++x) v += P[(int64_t)x * pq + e];
    C[e] = v;
  }
}

// Out = X S: X n x p, S p x q (column-major FP64), Out n x q.  Thread = one
// row i and 32 columns [32 y, 32 y + 32) of S (blockIdx.y); S's columns of
// the tile are staged in shared memory, X's row is read one element at a
// time (consecutive threads, consecutive rows: coalesced).
constexpr int kXsCols = 32;

__global__ void __launch_bounds__(256) k_x_times_s(const double *__restrict__ X, int64_t n,
                                                   int32_t p, const double *__restrict__ S,
                                                   int32_t q, double *__restrict__ Out) {
  extern __shared__ __align__(16) double sS[];  // [kXsCols][p]
  const int c0 = blockIdx.y * kXsCols;
  const int nc = min(kXsCols, q - c0);
  for (int x = threadIdx.x; x < nc * p; x += blockDim.x) sS[x] = S[(int64_t)c0 * p + x];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc[kXsCols];
#pragma unroll
  for (int c = 0; c < kXsCols; ++c) acc[c] = 0.0;
  for (int a = 0; a < p; ++a) {
    const double x = X[(int64_t)a * n + i];
#pragma unroll
    for (int c = 0; c < kXsCols; ++c)
      if (c < nc) acc[c] = fma(x, sS[c * p + a], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < kXsCols; ++c)
    if (c < nc) Out[(int64_t)(c0 + c) * n + i] = acc[c];
}

// SplitMix64 (Steele, Lea and Flood 2014): the counter-based generator of the
// random start, uniform in [-1, 1).
uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
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
  float *Qt = nullptr, *Yp = nullptr;
  double *Q = nullptr, *Y = nullptr, *W = nullptr, *r = nullptr, *R2 = nullptr, *st = nullptr,
         *G = nullptr, *P = nullptr, *U = nullptr;
  ~PcoaDev() {
    for (void *p : {(void *)Qt, (void *)Yp, (void *)Q, (void *)Y, (void *)W, (void *)r,
                    (void *)R2, (void *)st, (void *)G, (void *)P, (void *)U})
      if (p) cudaFree(p);
  }
};

// Launch shape of the Gram products: row blocks of at least 256 rows, about
// two CTAs per SM over all entry tiles.
struct XtzShape {
  int32_t blocks, tiles;
  int64_t rows;
};
XtzShape xtz_shape(int64_t n, int32_t p, int32_t q, int sms) {
  XtzShape sh;
  sh.tiles = (int32_t)(((int64_t)p * q + kXtzThreads * kXtzPer - 1) / (kXtzThreads * kXtzPer));
  const int64_t want = std::max<int64_t>(1, (int64_t)2 * sms / sh.tiles);
  sh.rows = std::max<int64_t>(256, (n + want - 1) / want);
  sh.blocks = (int32_t)((n + sh.rows - 1) / sh.rows);
  return sh;
}

// C (p x q, column-major, device) = X^T Z over n rows; P is scratch of at least
// xtz_shape(...).blocks * p * q doubles.
int xtz(const double *X, const double *Z, int64_t n, int32_t p, int32_t q, double *P, double *C,
        int sms, cudaStream_t st) {
  const XtzShape sh = xtz_shape(n, p, q, sms);
  const size_t smem = (size_t)kXtzRows * (p + q) * sizeof(double);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_xtz_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    return UNIFRAC_E_CUDA;
  k_xtz_partial<<<dim3(sh.blocks, sh.tiles), kXtzThreads, smem, st>>>(X, Z, n, p, q, sh.rows, P);
  const int64_t pq = (int64_t)p * q;
  k_xtz_reduce<<<(unsigned)std::min<int64_t>((pq + 255) / 256, 4096), 256, 0, st>>>(P, sh.blocks,
                                                                                    pq, C);
  return cudaGetLastError() == cudaSuccess ? UNIFRAC_OK : UNIFRAC_E_CUDA;
}

// Out (n x q) = X (n x p) S (p x q), all column-major on the device.
int x_times_s(const double *X, int64_t n, int32_t p, const double *S, int32_t q, double *Out,
              cudaStream_t st) {
  const size_t smem = (size_t)kXsCols * p * sizeof(double);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_x_times_s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    return UNIFRAC_E_CUDA;
  k_x_times_s<<<dim3((unsigned)((n + 255) / 256), (q + kXsCols - 1) / kXsCols), 256, smem, st>>>(
      X, n, p, S, q, Out);
  return cudaGetLastError() == cudaSuccess ? UNIFRAC_OK : UNIFRAC_E_CUDA;
}

// Columns per warp of k_pcoa_dq for m columns (one launch covers 4 CW).
int dq_cw(int m) { return m <= 16 ? 4 : m <= 32 ? 8 : m <= 36 ? 9 : m <= 48 ? 12 : 16; }

template <typename TD>
int launch_dq(int cw, const TD *D, int32_t n, const float *Qt, int32_t mp, int32_t m,
              int32_t chunk, int32_t kc, float *Yp, cudaStream_t st) {
  const dim3 grid((n + kDqRows - 1) / kDqRows, kc, (m + 4 * cw - 1) / (4 * cw));
  switch (cw) {
    case 4: k_pcoa_dq<TD, 4><<<grid, kDqThreads, 0, st>>>(D, n, Qt, mp, m, chunk, Yp); break;
    case 8: k_pcoa_dq<TD, 8><<<grid, kDqThreads, 0, st>>>(D, n, Qt, mp, m, chunk, Yp); break;
    case 9: k_pcoa_dq<TD, 9><<<grid, kDqThreads, 0, st>>>(D, n, Qt, mp, m, chunk, Yp); break;
    case 12: k_pcoa_dq<TD, 12><<<grid, kDqThreads, 0, st>>>(D, n, Qt, mp, m, chunk, Yp); break;
    default: k_pcoa_dq<TD, 16><<<grid, kDqThreads, 0, st>>>(D, n, Qt, mp, m, chunk, Yp); break;
  }
  return cudaGetLastError() == cudaSuccess ? UNIFRAC_OK : UNIFRAC_E_CUDA;
}

}  // namespace
}  // namespace ufb

extern "C" int unifrac_pcoa(const void *dist, int precision, int32_t n, int32_t k, int32_t iters,
                            uint64_t seed, double *eigvals, double *coords, void *cuda_stream) {
  using namespace ufb;
  if (!dist || !eigvals || !coords || n < 1 || k < 1 || k > n || k > UNIFRAC_PCOA_MAX_K ||
      iters < 0)
    return UNIFRAC_E_INVALID_ARG;
  if (precision != UNIFRAC_FP64 && precision != UNIFRAC_MIXED) return UNIFRAC_E_INVALID_ARG;
  // 16-byte row loads of D need a 16-byte aligned base
  if (reinterpret_cast<uintptr_t>(dist) % 16 != 0) return UNIFRAC_E_INVALID_ARG;
  // oversampled subspace: component c converges as (lambda_{m+1} / lambda_c)^iters,
  // and UniFrac spectra decay slowly, so the subspace is wide (the product
  // with A costs about the same for any m of this size: it streams D)
  const int m = std::min<int>(n, 2 * k + 16);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return UNIFRAC_E_CUDA;
  const int cw = dq_cw(m);
  const int mp = (m + 3) / 4 * 4;
  // chunks of D's rows j: enough CTAs for several waves, at most 16 chunks
  // (FP32 sums within a chunk, FP64 across chunks)
  const int64_t panels = (n + kDqRows - 1) / kDqRows;
  const int64_t cblocks = (m + 4 * cw - 1) / (4 * cw);
  const int64_t want =
      std::min<int64_t>(16, std::max<int64_t>(1, (int64_t)sms * 16 / (panels * cblocks)));
  int32_t chunk = (int32_t)std::max<int64_t>(kBJ, ((n + want - 1) / want + kBJ - 1) / kBJ * kBJ);
  const int32_t kc = (int32_t)((n + chunk - 1) / chunk);
  PcoaDev dv;
  const size_t nm = (size_t)n * m;
  const XtzShape g_mm = xtz_shape(n, m, m, sms), g_m2 = xtz_shape(n, m, 2, sms);
  const size_t p_len = std::max((size_t)g_mm.blocks * m * m, (size_t)g_m2.blocks * m * 2);
  if (dev_malloc_retry((void **)&dv.Qt, (size_t)n * mp * sizeof(float)) != cudaSuccess ||
      dev_malloc_retry((void **)&dv.Yp, (size_t)kc * n * mp * sizeof(float)) != cudaSuccess ||
      dev_malloc_retry((void **)&dv.Q, nm * sizeof(double)) != cudaSuccess ||
      dev_malloc_retry((void **)&dv.Y, nm * sizeof(double)) != cudaSuccess ||
      dev_malloc_retry((void **)&dv.W, nm * sizeof(double)) != cudaSuccess ||
      dev_malloc_retry((void **)&dv.U, (size_t)n * k * sizeof(double)) != cudaSuccess ||
      dev_malloc_retry((void **)&dv.r, (size_t)n * sizeof(double)) != cudaSuccess ||
      dev_malloc_retry((void **)&dv.R2, 2 * (size_t)n * sizeof(double)) != cudaSuccess ||
      dev_malloc_retry((void **)&dv.st, 2 * (size_t)m * sizeof(double)) != cudaSuccess ||
      dev_malloc_retry((void **)&dv.G, (size_t)m * m * sizeof(double)) != cudaSuccess ||
      dev_malloc_retry((void **)&dv.P, p_len * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return UNIFRAC_E_OOM;
  }
  if (precision == UNIFRAC_FP64)
    k_pcoa_rowmean<double><<<n, 256, 0, st>>>(static_cast<const double *>(dist), n, dv.r);
  else
    k_pcoa_rowmean<float><<<n, 256, 0, st>>>(static_cast<const float *>(dist), n, dv.r);
  if (cudaGetLastError() != cudaSuccess) return UNIFRAC_E_CUDA;
  std::vector<double> r(n), ones(n, 1.0);
  if (cudaMemcpyAsync(r.data(), dv.r, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return UNIFRAC_E_CUDA;
  double g = 0.0;
  for (int32_t i = 0; i < n; ++i) g += r[i];
  g /= (double)n;
  // [1 r] as an n x 2 column-major matrix: Q^T [1 r] gives the centring terms
  if (cudaMemcpyAsync(dv.R2, ones.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(dv.R2 + n, dv.r, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)  // ones (host) is copied before it goes out of scope
    return UNIFRAC_E_CUDA;
  const int grid = sms * 8;

  // M <- M R^-1 with M^T M = R^T R (CholeskyQR): the Gram matrix and the
  // product with R^-1 on the device (their long dimension n parallelises),
  // the factor and its inverse are m x m host work
  std::vector<double> Gh((size_t)m * m);
  auto cholqr = [&](double *&M, double shift) -> int {
    int rc = xtz(M, M, n, m, m, dv.P, dv.G, sms, st);
    if (rc) return rc;
    if (cudaMemcpyAsync(Gh.data(), dv.G, Gh.size() * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return UNIFRAC_E_CUDA;
    for (int a = 0; a < m; ++a)  // exact symmetry
      for (int b = a + 1; b < m; ++b) Gh[(size_t)b * m + a] = Gh[(size_t)a * m + b];
    const std::vector<double> Rinv = upper_inverse(cholesky_upper(Gh, m, shift), m);
    if (cudaMemcpyAsync(dv.G, Rinv.data(), Rinv.size() * sizeof(double), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return UNIFRAC_E_CUDA;
    if ((rc = x_times_s(M, n, m, dv.G, m, dv.W, st))) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess)  // Rinv (host) is copied before it goes out of scope
      return UNIFRAC_E_CUDA;
    std::swap(M, dv.W);
    return UNIFRAC_OK;
  };
  auto orthonormalise = [&](double *&M) -> int {
    int rc = cholqr(M, 1e-13);  // shifted first pass: factors even a rank-deficient M
    return rc ? rc : cholqr(M, 0.0);
  };
  // Y = B Q = A Q - r (1^T Q) - 1 (r^T Q) + g 1 (1^T Q): the product from D
  // (FP32 sums within a chunk, FP64 across), the centring terms in FP64
  auto apply_B = [&]() -> int {
    k_pcoa_qt<<<grid, 256, 0, st>>>(dv.Q, n, m, mp, dv.Qt);
    int rc = (precision == UNIFRAC_FP64)
                 ? launch_dq<double>(cw, static_cast<const double *>(dist), n, dv.Qt, mp, m, chunk,
                                     kc, dv.Yp, st)
                 : launch_dq<float>(cw, static_cast<const float *>(dist), n, dv.Qt, mp, m, chunk,
                                    kc, dv.Yp, st);
    if (rc) return rc;
    if ((rc = xtz(dv.Q, dv.R2, n, m, 2, dv.P, dv.st, sms, st))) return rc;
    k_pcoa_reduce<<<grid, 256, 0, st>>>(dv.Yp, kc, n, mp, m, dv.r, dv.st, dv.st + m, g, dv.Y);
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
  if ((rc = xtz(dv.Q, dv.Y, n, m, m, dv.P, dv.G, sms, st))) return rc;
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
      cudaSuccess)
    return UNIFRAC_E_CUDA;
  if ((rc = x_times_s(dv.Q, n, m, dv.G, k, dv.U, st))) return rc;
  if (cudaMemcpyAsync(Uh.data(), dv.U, Uh.size() * sizeof(double), cudaMemcpyDeviceToHost, st) !=
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
