// Pair kernels on the CUDA cores: weighted normalized UniFrac (FP32 with a
// two-level sum, or all-FP64) and the bit-packed lookup form of unweighted UniFrac.
//
// Section II of the paper: the distance is formed for every pair of samples,
// giving an N x N matrix, in a weighted normalized and an unweighted variant.
// Both kernels compute a 128 x 128 block of pairs per CTA (thread micro-tile
// 8 x 8 in registers) and sweep the branch dimension in windows of 1024
// branches.  A branch enters the sweep only if it is non-zero somewhere in the
// row tile AND somewhere in the column tile (AND of the two tiles' bitmaps),
// which is the sparse-aware skipping of Hybrid UniFrac: both kernels only need
// branches that the two samples share (see the identities below).  Selected
// rows are staged into shared memory with cp.async in a two-stage pipeline.
//
// Weighted normalized, with v[b,i] = len_b * w[b,i] and S_i = sum_b v[b,i]:
//   sum_b len_b |w_bi - w_bj| = S_i + S_j - 2 * sum_b min(v_bi, v_bj)
//   sum_b len_b (w_bi + w_bj) = S_i + S_j
// (|x - y| = x + y - 2 min(x, y)), so only co-present branches contribute to the
// pair sum M_ij = sum_b min(v_bi, v_bj); S comes from the embedding.
// Unweighted, with a_i = sum_b len_b p_bi and G_ij = sum_b len_b p_bi p_bj:
//   sum_b len_b (p_bi XOR p_bj) = a_i + a_j - 2 G_ij
//   sum_b len_b (p_bi OR p_bj)  = a_i + a_j - G_ij
// and the lookup form evaluates G_ij 8 branches at a time from a byte of
// presence bits: G_ij = sum_g T_g[x_gi AND x_gj], T_g[m] = sum of the lengths
// of the branches whose bits are set in m.
#include <type_traits>

#include "epilogue.cuh"

namespace ufb {

namespace {

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kThreads = 256;
constexpr int kWinWords = 32;  // bitmap words per window (1024 branches)

// Warp 0 turns the AND of the two tiles' bitmap words [w0, w0+32) into an
// ascending list of selected indices; returns the count through *list_n.
__device__ __forceinline__ void build_window(const uint32_t *__restrict__ bI,
                                             const uint32_t *__restrict__ bJ, int n_words,
                                             int w0, int32_t *list, int32_t *list_n) {
  const int lane = threadIdx.x;
  const int w = w0 + lane;
  uint32_t m = (w < n_words) ? (bI[w] & bJ[w]) : 0u;
  const int c = __popc(m);
  int incl = c;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  int pos = incl - c;
  while (m) {
    const int b = __ffs(m) - 1;
    m &= m - 1;
    list[pos++] = w * WORD + b;
  }
  if (lane == 31) *list_n = incl;
}

// Rows owned by thread (ty, tx) of the 16 x 16 thread grid: 4 consecutive
// rows in each half of the tile, so the operand loads are 16-byte vectors.
__device__ __forceinline__ int own_row(int t16, int q) { return (q < 4) ? t16 * 4 + q : 64 + t16 * 4 + (q - 4); }

// ----------------------------------------------------------------------------
// weighted normalized

constexpr int BK = 16;  // branches per pipeline stage

template <typename T>
__device__ __forceinline__ void load8(const T *row, int t16, T (&x)[8]);

template <>
__device__ __forceinline__ void load8<float>(const float *row, int t16, float (&x)[8]) {
  const float4 lo = *reinterpret_cast<const float4 *>(row + t16 * 4);
  const float4 hi = *reinterpret_cast<const float4 *>(row + 64 + t16 * 4);
  x[0] = lo.x; x[1] = lo.y; x[2] = lo.z; x[3] = lo.w;
  x[4] = hi.x; x[5] = hi.y; x[6] = hi.z; x[7] = hi.w;
}

template <>
__device__ __forceinline__ void load8<double>(const double *row, int t16, double (&x)[8]) {
  const double2 a = *reinterpret_cast<const double2 *>(row + t16 * 4);
  const double2 b = *reinterpret_cast<const double2 *>(row + t16 * 4 + 2);
  const double2 c = *reinterpret_cast<const double2 *>(row + 64 + t16 * 4);
  const double2 d = *reinterpret_cast<const double2 *>(row + 64 + t16 * 4 + 2);
  x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
  x[4] = c.x; x[5] = c.y; x[6] = d.x; x[7] = d.y;
}

// Register micro-tile of min-sums.  FP32: FMNMX per pair and packed two-wide
// adds (add.f32x2), the min on the ALU pipe, the adds on the FMA pipe.
// FP64: fmin + add.
template <typename T>
struct MinAcc;

template <>
struct MinAcc<float> {
  float2 p[8][4];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) p[i][j] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void add(const float (&a)[8], const float (&b)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        p[i][j] = __fadd2_rn(p[i][j], make_float2(fminf(a[i], b[2 * j]), fminf(a[i], b[2 * j + 1])));
  }
  __device__ __forceinline__ double get(int i, int j) const {
    return (j & 1) ? (double)p[i][j >> 1].y : (double)p[i][j >> 1].x;
  }
  // tot[row][col] += p for the 8 x 8 pairs this thread owns (own_row layout:
  // columns 4 tx .. 4 tx + 3 and 64 + 4 tx .. 64 + 4 tx + 3, 16-byte vectors),
  // then p = 0.  Only the owning thread touches these elements.
  __device__ __forceinline__ void flush_to(float *tot, int ty, int tx) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
      float4 *lo = reinterpret_cast<float4 *>(tot + row * 128 + tx * 4);
      float4 *hi = reinterpret_cast<float4 *>(tot + row * 128 + 64 + tx * 4);
      float4 a = *lo, b = *hi;
      a.x += p[i][0].x; a.y += p[i][0].y; a.z += p[i][1].x; a.w += p[i][1].y;
      b.x += p[i][2].x; b.y += p[i][2].y; b.z += p[i][3].x; b.w += p[i][3].y;
      *lo = a;
      *hi = b;
    }
    zero();
  }
};

template <>
struct MinAcc<double> {
  double p[8][8];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) p[i][j] = 0.0;
  }
  __device__ __forceinline__ void add(const double (&a)[8], const double (&b)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) p[i][j] += fmin(a[i], b[j]);
  }
  __device__ __forceinline__ double get(int i, int j) const { return p[i][j]; }
};

// T = float: FP32 partial sums in registers, added every `flush` selected
// branches into an FP32 running total in shared memory (two-level summation:
// each level sums at most max(flush, K / flush) terms, so the rounding error
// stays near that of a sum of ~sqrt(K) terms); FP32 epilogue.  Keeping the
// total out of registers lets two CTAs share an SM.
// T = double: FP64 throughout.
//
// Hybrid split (FP32 form): positions [0, 32*kf_words) are the frequently
// present branches and run through the dense register tile here; the rest,
// present in few samples, were summed by k_pairs_sparse<false> into spart
// (sp_parts partial sums per tile pair, 32-bit fixed point, scale 1 / sp_inv),
// added in the epilogue.
template <typename T>
__global__ void __launch_bounds__(kThreads, (sizeof(T) == 4) ? 2 : 1)
    k_pairs_weighted(const WorkItem *__restrict__ items, int32_t n_items, int32_t item0,
                     int32_t item1, unsigned int *__restrict__ queue, const T *__restrict__ vals,
                     int64_t ldv, const uint32_t *__restrict__ bits, int32_t n_words,
                     int32_t kf_words, const uint32_t *__restrict__ spart, int32_t sp_parts,
                     double sp_inv, const double *__restrict__ S,
                     int32_t flush, OutSpec o, unsigned long long *__restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sbuf = reinterpret_cast<T *>(smem_raw);  // [2 stages][BK][2 sides][TILE]
  int32_t *list = reinterpret_cast<int32_t *>(smem_raw + sizeof(T) * 2 * BK * 2 * TILE);
  // FP32 form: running totals [TILE][TILE] after the list
  float *tot = reinterpret_cast<float *>(smem_raw + sizeof(T) * 2 * BK * 2 * TILE +
                                         sizeof(int32_t) * kWinWords * WORD);
  __shared__ int32_t list_n;
  __shared__ int32_t s_item;
  const bool sparse = (sizeof(T) == 4) && spart != nullptr;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  unsigned long long nsel = 0;

  // work items [item0, item1) (n_items in all: the stride of the sparse
  // partial sums): the next tile pair from the device queue (persistent
  // grid), or this CTA's own (one CTA per item)
  for (int iter = 0;; ++iter) {
  if (tid == 0)
    s_item = item0 + (queue ? (int32_t)atomicAdd(queue, 1u)
                            : (iter == 0 ? (int32_t)blockIdx.x : item1 - item0));
  __syncthreads();
  const int32_t item = s_item;
  if (item >= item1) break;
  const WorkItem it = items[item];
  const StudyDev sd = o.studies[it.study];
  const uint32_t *bI = bits + (int64_t)it.tile_i * n_words;
  const uint32_t *bJ = bits + (int64_t)it.tile_j * n_words;
  const int64_t colI = (int64_t)it.tile_i * TILE, colJ = (int64_t)it.tile_j * TILE;
  constexpr int CPR = TILE * sizeof(T) / 16;  // 16-byte chunks per row
  constexpr int kEl = 16 / sizeof(T);

  // FP32 form: part (registers, current chunk) + tot (shared memory).  FP64
  // form: part only.
  MinAcc<T> part;
  part.zero();
  if constexpr (sizeof(T) == 4) {
    // tot = 0 on the elements this thread owns
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = own_row(ty, i);
      *reinterpret_cast<float4 *>(tot + row * TILE + tx * 4) = make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4 *>(tot + row * TILE + 64 + tx * 4) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  // warps start their flush counters staggered, so the flushes of one warp
  // overlap the min / add work of the others
  int since_flush = (sizeof(T) == 4) ? (tid >> 5) * (flush / (kThreads / 32)) : 0;

  auto load_stage = [&](int s, int buf, int n) {
    for (int c = tid; c < BK * 2 * CPR; c += kThreads) {
      const int r = c / (2 * CPR);
      const int side = (c / CPR) & 1;
      const int q = c % CPR;
      const int li = s * BK + r;
      if (li < n) {
        const int32_t k = list[li];
        const T *src = vals + (int64_t)k * ldv + (side ? colJ : colI) + q * kEl;
        T *dst = sbuf + ((int64_t)(buf * BK + r) * 2 + side) * TILE + q * kEl;
        cp_async16(dst, src);
      }
    }
  };
  auto flush_part = [&]() {
    if constexpr (sizeof(T) == 4) part.flush_to(tot, ty, tx);
  };

  for (int w0 = 0; w0 < kf_words; w0 += kWinWords) {
    if (tid < 32) build_window(bI, bJ, kf_words, w0, list, &list_n);
    __syncthreads();
    const int n = list_n;
    nsel += (unsigned long long)n;
    const int ns = (n + BK - 1) / BK;
    if (ns > 0) {
      load_stage(0, 0, n);
      cp_commit();
      for (int s = 0; s < ns; ++s) {
        if (s + 1 < ns) {
          load_stage(s + 1, (s + 1) & 1, n);
          cp_commit();
          cp_wait<1>();
        } else {
          cp_wait<0>();
        }
        __syncthreads();
        const int rows = min(BK, n - s * BK);
        const T *base = sbuf + (int64_t)((s & 1) * BK) * 2 * TILE;
        if (rows == BK) {
          // full stage: operands of the next branch are loaded before the
          // current one is accumulated, so shared-memory latency overlaps math
          T a[2][8], b[2][8];
          load8<T>(base, ty, a[0]);
          load8<T>(base + TILE, tx, b[0]);
#pragma unroll
          for (int r = 0; r < BK; ++r) {
            if (r + 1 < BK) {
              load8<T>(base + ((r + 1) * 2 + 0) * TILE, ty, a[(r + 1) & 1]);
              load8<T>(base + ((r + 1) * 2 + 1) * TILE, tx, b[(r + 1) & 1]);
            }
            part.add(a[r & 1], b[r & 1]);
          }
        } else {
          for (int r = 0; r < rows; ++r) {
            T a[8], b[8];
            load8<T>(base + (r * 2 + 0) * TILE, ty, a);
            load8<T>(base + (r * 2 + 1) * TILE, tx, b);
            part.add(a, b);
          }
        }
        if constexpr (sizeof(T) == 4) {
          since_flush += rows;
          if (since_flush >= flush) {
            flush_part();
            since_flush = 0;
          }
        }
        __syncthreads();
      }
    }
    __syncthreads();
  }
  flush_part();

  // epilogue: d = (S_i + S_j - 2 M) / (S_i + S_j); FP32 in the FP32 form
  // (each term is within a few roundings of its exact value and the
  // difference is taken once, so the error stays a few units of 2^-24 of
  // S_i + S_j), FP64 in the FP64 form
  const float sp_inv_f = (float)sp_inv;
  float Sj_f[8];  // this thread's column sums, converted once
#pragma unroll
  for (int qj = 0; qj < 8; ++qj) Sj_f[qj] = (sizeof(T) == 4) ? (float)S[colJ + own_row(tx, qj)] : 0.f;
#pragma unroll
  for (int qi = 0; qi < 8; ++qi) {
    const int i = own_row(ty, qi);
    const int li = (int)(colI + i) - sd.col0;
    if (li >= sd.n) continue;
    const double Si = S[colI + i];
#pragma unroll
    for (int qj = 0; qj < 8; ++qj) {
      const int j = own_row(tx, qj);
      const int lj = (int)(colJ + j) - sd.col0;
      if (lj >= sd.n) continue;
      if (li < lj) {
        if constexpr (sizeof(T) == 4) {
          const float den = (float)Si + Sj_f[qj];
          float M = tot[i * TILE + j];
          if (sparse) {
            // the parts' integer sums add exactly (their total is below 2^31)
            const uint32_t *sp = spart + (int64_t)item * TILE * TILE + i * TILE + j;
            uint32_t q = 0;
#pragma unroll
            for (int p = 0; p < kMaxSparseParts; ++p)  // loads issued together
              if (p < sp_parts) q += sp[(int64_t)p * n_items * TILE * TILE];
            M = __fmaf_rn((float)q, sp_inv_f, M);
          }
          put_pair(o, sd, li, lj, ratio01_f32(__fmaf_rn(-2.f, M, den), den));
        } else {
          const double den = Si + S[colJ + j];
          put_pair(o, sd, li, lj, ratio01(den - 2.0 * part.get(qi, qj), den));
        }
      } else if (li == lj) {
        put_diag(o, sd, li);
      }
    }
  }
  __syncthreads();  // shared memory and s_item free for the next item
  }  // work items
  if (tid == 0 && counter) atomicAdd(counter, nsel);
}

// ----------------------------------------------------------------------------
// rarely present branches: weighted normalized (FP32 form) and unweighted
//
// For every tile pair, the branches at positions >= 32*kf_words present in both
// tiles contribute only for the rows that hold them: min(V_bi, V_bj) (weighted)
// or the 24-bit length q_b (unweighted) for every pair of a row of tile I and
// a row of tile J holding b.  The compact blocks (one per tile and window of
// kRareWin positions) list each flagged row's entries; the weighted blocks hold
// V = round(v * 2^s), and rounding is monotone, so
// min(V_bi, V_bj) = round(min(v_bi, v_bj) * 2^s); 2^s keeps every pair sum
// below 2^31.  Sums go into a 128 x 128 shared accumulator of integers (exact,
// independent of the order of the atomics), rows padded to TILE + 1 words so
// that lanes on one column of different rows use different banks; it is
// copied to spart at the end.
//
// A CTA of 32 warps per (tile pair, part): part p of n_parts takes the bitmap
// words kf_words + 32 p + warp, + 32 n_parts, ... (each warp its own, with no
// CTA-wide barrier in the loop) and writes its own partial sums, so that the
// tile pairs x parts fill the SMs' waves evenly.  For a
// word, the rank of its first flagged row in the window's block is the
// popcount of the block's earlier words; lane l takes the branch of bit l when
// it is flagged in both tiles.  A weighted entry is one 8-byte (value, row)
// word.  An incidence of at most lane_pairs pairs (an option) is walked by its lane alone,
// reading the blocks (read-only loads through L1).  A larger one is walked by
// the whole warp: one tile's rows (the "lane side") are held in registers,
// lane (g, b) = (lane / nL, lane % nL) holding row b, and the other tile's
// entries, copied by the warp into its own shared scratch, are swept
// a = g, g + G, ... with G = 32 / nL groups (rows beyond 32 on the lane side
// in further passes), so each update is one broadcast shared load, a min and
// one shared atomic.  The lane side is the tile whose row count fills more
// lanes.

constexpr int kSpThreads = 1024;
static_assert(kRareWin == kWinWords * WORD, "sparse blocks: one window is kWinWords bitmap words");
constexpr int kSpWarps = kSpThreads / 32;
constexpr int kAccLd = TILE + 1;   // padded accumulator row

// PRES = false: weighted form, entries carry V; 32-bit accumulators (spart u32).
// PRES = true:  unweighted form, entries are presences; adds the 24-bit q[k]
//               as two 12-bit halves into two 32-bit shared planes (32-bit
//               shared atomics are native; a half-sum stays below 2^32 while
//               fewer than 2^20 branches are summed), combined into 64-bit
//               spart at the end, exact -- the tensor-core epilogue adds it to
//               its digit sums.
template <bool PRES>
struct SparseCfg {
  using Acc = typename std::conditional<PRES, unsigned long long, uint32_t>::type;
  static constexpr size_t kAccBytes = ((size_t)TILE * kAccLd * 4 * (PRES ? 2 : 1) + 15) / 16 * 16;
  // the swept side of one incidence per warp: TILE entries of 1 byte
  // (unweighted), or of 8 bytes (weighted) at interleaved positions, the
  // largest 150 (k_pairs_sparse: two entries per 16-byte load)
  static constexpr size_t kScratch = PRES ? (size_t)TILE : (size_t)152 * 8;
  static constexpr size_t kSmem = kAccBytes + (size_t)kSpWarps * kScratch;
};

template <bool PRES>
__global__ void __launch_bounds__(kSpThreads, 1)
    k_pairs_sparse(const WorkItem *__restrict__ items, int32_t n_items,
                   unsigned int *__restrict__ queue, const uint32_t *__restrict__ bits,
                   int32_t n_words, int32_t kf_words, int32_t k_words, int32_t n_win,
                   const uint8_t *__restrict__ blocks, const unsigned long long *__restrict__ boff,
                   unsigned long long blocks_cap, int32_t n_tiles,
                   const uint2 *__restrict__ cpre,
                   const uint32_t *__restrict__ qlen, int32_t n_parts, int32_t lane_pairs,
                   typename SparseCfg<PRES>::Acc *__restrict__ spart,
                   unsigned long long *__restrict__ n_updates) {
  using Acc = typename SparseCfg<PRES>::Acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t *sacc = reinterpret_cast<uint32_t *>(smem_raw);  // [TILE][kAccLd] (PRES: low halves)
  uint32_t *sacc_hi = sacc + TILE * kAccLd;                 // PRES: high halves
  // (p / n, p % n) for lanes p < 32 and n = 1..32: group and row of a lane when
  // the lane side has n rows; gtab[n-1] = 32 / n groups; fillv[n-1] = lanes a
  // lane side of n rows keeps busy (n > 32: n / passes) -- no divisions later
  __shared__ uint16_t divtab[32][32];
  __shared__ uint8_t gtab[32];
  // gmul[G-1] = ceil(2^16 / G): a / G = (a gmul) >> 16 exactly for a < 128
  __shared__ uint32_t gmul[32];
  __shared__ uint8_t fillv[TILE];

  __shared__ int32_t s_unit;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *scr = smem_raw + SparseCfg<PRES>::kAccBytes + warp * SparseCfg<PRES>::kScratch;
  unsigned long long *eS = reinterpret_cast<unsigned long long *>(scr);  // weighted
  uint8_t *rS = scr;                                                     // unweighted
  unsigned long long my_updates = 0;
  {
    const int n = tid / 32 + 1, p = tid % 32;  // kSpThreads == 32 * 32
    divtab[n - 1][p] = (uint16_t)(((p / n) << 8) | (p % n));
    if (tid < 32) {
      gtab[tid] = (uint8_t)(32 / (tid + 1));
      gmul[tid] = (65536u + (uint32_t)tid) / (uint32_t)(tid + 1);  // ceil(2^16 / G)
    }
    if (tid < TILE) {
      const int m = tid + 1;
      fillv[tid] = (uint8_t)(m <= 32 ? (32 / m) * m : m / ((m + 31) / 32));
    }
  }
  // work units (tile pair, part), unit u = part * n_items + item: the next
  // from the device queue (persistent grid), or this CTA's own
  const int32_t n_units = n_items * n_parts;
  for (int iter = 0;; ++iter) {
  if (tid == 0)
    s_unit = queue ? (int32_t)atomicAdd(queue, 1u)
                   : (iter == 0 ? (int32_t)(blockIdx.y * n_items + blockIdx.x) : n_units);
  for (int x = tid; x < TILE * kAccLd * (PRES ? 2 : 1); x += kSpThreads) sacc[x] = 0u;
  __syncthreads();
  const int32_t unit = s_unit;
  if (unit >= n_units) break;
  const int32_t item = unit % n_items, part = unit / n_items;
  const WorkItem it = items[item];
  const int64_t tI = it.tile_i, tJ = it.tile_j;
  const uint32_t *bI = bits + tI * n_words;
  const uint32_t *bJ = bits + tJ * n_words;
  const uint32_t below = (1u << lane) - 1u;
  // blocks that did not fit their buffer were not written (the fill reported
  // it): read none of them
  const int w_end = boff[(int64_t)n_tiles * n_win] > blocks_cap ? kf_words : k_words;
  // Per word with a branch present in both tiles, what its incidences need
  // comes from loads that depend only on the word: the rows of the window's
  // block before the word and the block's total rows (cpre, written when the
  // blocks were sized) and the block's byte offset.  A flagged row's rank is
  // then that base plus a popcount; its row start and entries follow in two
  // more loads.  The next word's bitmap words are loaded before this word's
  // incidences are walked.
  const int w_step = kSpWarps * n_parts;
  int w = kf_words + part * kSpWarps + warp;
  uint32_t nmI = 0, nmJ = 0;
  if (w < w_end) {
    nmI = __ldg(bI + w);
    nmJ = __ldg(bJ + w);
  }
  for (; w < w_end; w += w_step) {
    const uint32_t mI = nmI, mJ = nmJ;
    if (w + w_step < w_end) {
      nmI = __ldg(bI + w + w_step);
      nmJ = __ldg(bJ + w + w_step);
    }
    const uint32_t both = mI & mJ;
    if (both == 0u) continue;  // warp-uniform
    const int jw = (w - kf_words) / kWinWords;
    const int wq = (w - kf_words) - jw * kWinWords;
    const int64_t itI = tI * n_win + jw, itJ = tJ * n_win + jw;
    const uint32_t cI = __ldg(&cpre[itI * (kWinWords + 1) + wq].x);
    const uint32_t cJ = __ldg(&cpre[itJ * (kWinWords + 1) + wq].x);
    const uint32_t nrI = __ldg(&cpre[itI * (kWinWords + 1) + kWinWords].x);
    const uint32_t nrJ = __ldg(&cpre[itJ * (kWinWords + 1) + kWinWords].x);
    // block layout: 16-byte header, rowstart[rows + 1], entries at a 16-byte
    // aligned offset
    const uint8_t *blkI = blocks + __ldg(boff + itI);
    const uint8_t *blkJ = blocks + __ldg(boff + itJ);
    const uint32_t *rsI = reinterpret_cast<const uint32_t *>(blkI) + 4;
    const uint32_t *rsJ = reinterpret_cast<const uint32_t *>(blkJ) + 4;
    const uint32_t offI = (16u + 4u * (nrI + 1u) + 15u) & ~15u;
    const uint32_t offJ = (16u + 4u * (nrJ + 1u) + 15u) & ~15u;
    const uint8_t *riI = blkI + offI, *riJ = blkJ + offJ;  // presence entries
    const unsigned long long *eI = reinterpret_cast<const unsigned long long *>(blkI + offI);
    const unsigned long long *eJ = reinterpret_cast<const unsigned long long *>(blkJ + offJ);
    struct { uint32_t x; } hI{nrI}, hJ{nrJ};

    int nI = 0, nJ = 0;
    uint32_t sI = 0, sJ = 0;
    uint32_t qk = 0;
    if ((both >> lane) & 1u) {
      const int rI = cI + __popc(mI & below);
      const int rJ = cJ + __popc(mJ & below);
      if (rI < (int)hI.x && rJ < (int)hJ.x) {  // defensive: the rows must exist
        sI = __ldg(rsI + rI);
        sJ = __ldg(rsJ + rJ);
        nI = (int)(__ldg(rsI + rI + 1) - sI);
        nJ = (int)(__ldg(rsJ + rJ + 1) - sJ);
        // a row of a tile has 1..TILE entries; anything else is skipped
        if (nI < 1 || nI > TILE || nJ < 1 || nJ > TILE) nI = nJ = 0;
      }
      if constexpr (PRES) qk = __ldg(qlen + 32 * w + lane);
    }
    const int total = nI * nJ;
    my_updates += (unsigned long long)total;
    if (total > 0 && total <= lane_pairs) {
      for (int a = 0; a < nI; ++a) {
        if constexpr (PRES) {
          const int ra = (int)__ldg(riI + sI + a) * kAccLd;
          for (int b = 0; b < nJ; ++b) {
            const int idx = ra + (int)__ldg(riJ + sJ + b);
            atomicAdd(&sacc[idx], qk & 0xfffu);
            atomicAdd(&sacc_hi[idx], qk >> 12);
          }
        } else {
          const unsigned long long ea = __ldg(eI + sI + a);
          const int ra = (int)(uint32_t)(ea & 0xffu) * kAccLd;
          const uint32_t va = (uint32_t)(ea >> 32);
          for (int b = 0; b < nJ; ++b) {
            const unsigned long long eb = __ldg(eJ + sJ + b);
            atomicAdd(&sacc[ra + (int)(uint32_t)(eb & 0xffu)], min(va, (uint32_t)(eb >> 32)));
          }
        }
      }
    }
    // warp-walked incidences: the owning lane picks the lane side (the tile
    // whose row count fills more lanes) and packs the descriptor
    const bool is_big = total > lane_pairs;
    uint32_t desc = 0, sL = 0, sT = 0;
    if (is_big) {
      const bool lJ = fillv[nJ - 1] >= fillv[nI - 1];
      desc = lJ ? ((uint32_t)nJ | ((uint32_t)nI << 8) | (1u << 16))
                : ((uint32_t)nI | ((uint32_t)nJ << 8));
      sL = lJ ? sJ : sI;
      sT = lJ ? sI : sJ;
    }
    uint32_t big = __ballot_sync(0xffffffffu, is_big);
    while (big) {
      const int src = __ffs(big) - 1;
      big &= big - 1;
      const uint32_t d = __shfl_sync(0xffffffffu, desc, src);
      const uint32_t bsL = __shfl_sync(0xffffffffu, sL, src);
      const uint32_t bsT = __shfl_sync(0xffffffffu, sT, src);
      uint32_t bq = 0;
      if constexpr (PRES) bq = __shfl_sync(0xffffffffu, qk, src);
      const int nL = (int)(d & 0xffu), nT = (int)((d >> 8) & 0xffu);
      const bool laneJ = (d >> 16) != 0u;
      const int mL = laneJ ? 1 : kAccLd, mT = laneJ ? kAccLd : 1;  // accumulator strides
      // lane (g, b) of the sweep: one divtab / gtab read, before the scratch
      // stores (which would force a re-read)
      int g = 0, G = 1, b = lane;
      if (nL <= 32) {
        const uint32_t t0 = divtab[nL - 1][lane];
        g = (int)(t0 >> 8);
        b = (int)(t0 & 0xffu);
        G = gtab[nL - 1];
      }
      // copy the swept side into the scratch: every load issued before the
      // first store (one memory round trip, not one per 32 entries), the
      // lane side's first entry alongside; entries past 32 behind
      // warp-uniform branches (most swept sides have at most 32)
      unsigned long long eb0 = 0;
      if constexpr (PRES) {
        const uint8_t *rT = (laneJ ? riI : riJ) + bsT;
        if (b < nL) eb0 = __ldg((laneJ ? riJ : riI) + bsL + b);
        if (nT <= 32) {
          if (lane < nT) rS[lane] = __ldg(rT + lane);
        } else {
          uint8_t r0 = __ldg(rT + lane), r1 = 0, r2 = 0, r3 = 0;
          if (lane + 32 < nT) r1 = __ldg(rT + lane + 32);
          if (lane + 64 < nT) r2 = __ldg(rT + lane + 64);
          if (lane + 96 < nT) r3 = __ldg(rT + lane + 96);
          rS[lane] = r0;
          if (lane + 32 < nT) rS[lane + 32] = r1;
          if (lane + 64 < nT) rS[lane + 64] = r2;
          if (lane + 96 < nT) rS[lane + 96] = r3;
        }
      } else {
        const unsigned long long *qT = (laneJ ? eI : eJ) + bsT;
        if (b < nL) eb0 = __ldg((laneJ ? eJ : eI) + bsL + b);
        // stored ready for the sweep: (accumulator offset of the row, value)
        uint2 *eS2 = reinterpret_cast<uint2 *>(eS);
        auto prep = [mT](unsigned long long e) {
          return make_uint2((uint32_t)(e & 0xffu) * (uint32_t)mT, (uint32_t)(e >> 32));
        };
        // entry a goes to position 2 ((k / 2) G + a - k G) + k % 2, k = a / G:
        // sweep group g's entries g + 2 m G and g + (2 m + 1) G side by side
        const uint32_t gm = gmul[G - 1];
        auto pos = [G, gm](int a) {
          const int k = (int)(((uint32_t)a * gm) >> 16);
          return 2 * ((k >> 1) * G + a - k * G) + (k & 1);
        };
        if (nT <= 32) {
          if (lane < nT) eS2[pos(lane)] = prep(__ldg(qT + lane));
        } else {
          unsigned long long t0 = __ldg(qT + lane), t1 = 0, t2 = 0, t3 = 0;
          if (lane + 32 < nT) t1 = __ldg(qT + lane + 32);
          if (lane + 64 < nT) t2 = __ldg(qT + lane + 64);
          if (lane + 96 < nT) t3 = __ldg(qT + lane + 96);
          eS2[pos(lane)] = prep(t0);
          if (lane + 32 < nT) eS2[pos(lane + 32)] = prep(t1);
          if (lane + 64 < nT) eS2[pos(lane + 64)] = prep(t2);
          if (lane + 96 < nT) eS2[pos(lane + 96)] = prep(t3);
        }
      }
      __syncwarp();
      for (; b < nL; b += 32) {  // one pass when nL <= 32
        if (g < G) {
          if constexpr (PRES) {
            const int base = (int)(b < 32 ? eb0 : __ldg((laneJ ? riJ : riI) + bsL + b)) * mL;
#pragma unroll 2
            for (int a = g; a < nT; a += G) {
              const int idx = base + (int)rS[a] * mT;
              atomicAdd(&sacc[idx], bq & 0xfffu);
              atomicAdd(&sacc_hi[idx], bq >> 12);
            }
          } else {
            const unsigned long long eb = b < 32 ? eb0 : __ldg((laneJ ? eJ : eI) + bsL + b);
            uint32_t *row = sacc + (uint32_t)(eb & 0xffu) * (uint32_t)mL;
            const uint32_t vb = (uint32_t)(eb >> 32);
            // entries a and a + G of this group in one 16-byte shared load
            // (the shared-memory pipe is the bound): pair q = m G + g holds
            // entries 2 m G + g and (2 m + 1) G + g
            const uint4 *eS4 = reinterpret_cast<const uint4 *>(eS);
#pragma unroll 1
            for (int a = g, q = g; a < nT; a += 2 * G, q += G) {
              const uint4 e = eS4[q];
              atomicAdd(row + e.x, min(vb, e.y));
              if (a + G < nT) atomicAdd(row + e.z, min(vb, e.w));
            }
          }
        }
        if (nL <= 32) break;
      }
      __syncwarp();  // the scratch is rewritten by the next incidence
    }
  }
  __syncthreads();
  Acc *dst = spart + (int64_t)unit * TILE * TILE;
  for (int x = tid; x < TILE * TILE; x += kSpThreads) {
    const int q = (x / TILE) * kAccLd + x % TILE;
    if constexpr (PRES)
      dst[x] = ((unsigned long long)sacc_hi[q] << 12) + (unsigned long long)sacc[q];
    else
      dst[x] = sacc[q];
  }
  __syncthreads();  // the accumulator is cleared for the next unit
  }  // work units
  // pair updates done (statistics)
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) my_updates += __shfl_xor_sync(0xffffffffu, my_updates, off);
  if (lane == 0 && n_updates && my_updates) atomicAdd(n_updates, my_updates);
}

// ----------------------------------------------------------------------------
// very rarely present branches: one list per branch, all pairs of its samples
//
// Positions [pv, K) hold branches present in so few samples (at most the
// UNIFRAC_OPT_RARE_LIST bound, all studies together) that walking their bitmap
// words for every tile pair costs far more than their few co-present pairs.
// They are taken branch by branch instead.  k_list_fill writes, for position
// k, one entry per sample where the branch is present, ascending by column:
// u64 (value << 32) | column, the value being V = round(v * 2^s) (weighted,
// the value the sparse blocks carry) or the 24-bit length q_k (unweighted), at
// offsets voff[k - pv] (host prefix sums of the presence counts).  Beside it,
// a tile-major index: one record (entry, end of its branch's list) per entry,
// grouped by the entry's column tile (offsets toff from the row counts rc of
// the sparse packing, which cover these positions too, taken where the tile's
// bitmap flags the position).  k_pairs_list walks
// the records in that order: for the entry p of a record, every later entry q
// of its branch (a larger column) gives the pair (p, q), whose
// min(V_p, V_q) (weighted) or q_k (unweighted) is added into the partial sums
// of the tile pair (tile of p, tile of q) with a global atomic (item_of maps a
// tile pair to its work item, -1 when this run does not compute it).  Records
// are taken in order by a grid sized so that the records in flight span a few
// column tiles (kListBlocksPerSm, kListGrab): the atomics then land in
// partial sums that stay in L2.  The integer sums are those the sparse kernel
// would have made, so the result is unchanged.

constexpr int kListWarps = 8;
// CTAs of the persistent list kernel per SM, and records a warp takes at a
// time.  Its atomics land in the partial sums of the tile pairs of the
// records in flight (in column-tile order); with as many CTAs as fit (8 per
// SM) and 32 records per warp those span a dozen column tiles at 50,000
// samples, whose partial sums (hundreds of MB) overflow L2 and make the list
// kernels DRAM-bound.  4 x 8 warps x 16 records per SM keep about three
// column tiles in flight (measured on B300: 2x faster at 50,000 samples,
// the same at 4,096 and 25,000), with warps enough to cover the loads'
// latency.
constexpr int kListBlocksPerSm = 4;
constexpr uint32_t kListGrab = 16;

// Entries of the listed positions in each column tile: tcnt[t] = sum over
// k in [pv, K) of rc[t][k] (the tile's non-zero columns of position k), taken
// only where the tile's bitmap flags k: the packing writes rc nowhere else.
__global__ void __launch_bounds__(256) k_list_tile_counts(int32_t pv, int32_t K, int32_t k_pad,
                                                          const uint32_t *__restrict__ bits,
                                                          int32_t n_words,
                                                          const uint8_t *__restrict__ rc,
                                                          uint32_t *__restrict__ tcnt) {
  __shared__ uint32_t red[8];
  const int64_t t = blockIdx.x;
  uint32_t s = 0;
  for (int32_t k = pv + threadIdx.x; k < K; k += blockDim.x)
    if ((bits[t * n_words + k / WORD] >> (k % WORD)) & 1u) s += rc[t * k_pad + k];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < 8; ++w) tot += red[w];
    tcnt[t] = tot;
  }
}

template <bool VALUES>
__global__ void __launch_bounds__(kListWarps * 32)
    k_list_fill(int32_t pv, int32_t K, const int32_t *__restrict__ perm,
                const uint8_t *__restrict__ flag, const uint4 *__restrict__ pmask, int32_t n_tiles,
                const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ cslot,
                const double *__restrict__ len_perm,
                const double *__restrict__ inv_total, float scale,
                const uint32_t *__restrict__ qlen, const long long *__restrict__ voff,
                unsigned long long *__restrict__ ents, const unsigned long long *__restrict__ toff,
                uint32_t *__restrict__ tcur, uint2 *__restrict__ trec, unsigned long long n_ent) {
  const int64_t k = pv + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= K) return;
  const int32_t b = perm[k];
  const long long base = voff[k - pv], cap = voff[k - pv + 1] - base;
  const uint32_t end = (uint32_t)(base + cap);
  float L = 0.f;
  uint32_t q = 0;
  if constexpr (VALUES)
    L = (float)len_perm[k];
  else
    q = qlen[k];
  long long n = 0;  // entries written so far (warp-uniform)
  for (int t0 = 0; t0 < n_tiles; t0 += 32) {
    // lane l: tile t0 + l -- its presence mask, its entries, and (one atomic
    // per tile, all the chunk's at once) their place among the tile's records
    const int t = t0 + lane;
    const bool fl = t < n_tiles && flag[(int64_t)b * n_tiles + t];
    uint4 my_pm = make_uint4(0u, 0u, 0u, 0u);
    uint32_t my_slot = 0;
    unsigned long long my_tbase = 0, my_tend = 0;
    if (fl) {
      my_pm = pmask[(int64_t)b * n_tiles + t];
      const uint32_t cnt_t = __popc(my_pm.x) + __popc(my_pm.y) + __popc(my_pm.z) + __popc(my_pm.w);
      if (cnt_t) my_slot = atomicAdd(&tcur[t], cnt_t);
      my_tbase = toff[t];
      my_tend = toff[t + 1];
    }
    uint32_t m = __ballot_sync(0xffffffffu, fl);
    while (m) {
      const int src = __ffs(m) - 1;
      const int tt = t0 + src;
      m &= m - 1;
      // bit l of word w of the mask: column 4 l + w of the tile
      const uint32_t wv[4] = {__shfl_sync(0xffffffffu, my_pm.x, src),
                              __shfl_sync(0xffffffffu, my_pm.y, src),
                              __shfl_sync(0xffffffffu, my_pm.z, src),
                              __shfl_sync(0xffffffffu, my_pm.w, src)};
      uint32_t mine = 0;
#pragma unroll
      for (int w = 0; w < 4; ++w) mine += (wv[w] >> lane) & 1u;
      uint32_t before = mine;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, before, off);
        if (lane >= off) before += y;
      }
      const uint32_t total = __shfl_sync(0xffffffffu, before, 31);
      before -= mine;
      // this (branch, tile) chunk's place among the tile's records
      const uint32_t slot = __shfl_sync(0xffffffffu, my_slot, src);
      const unsigned long long tbase = __shfl_sync(0xffffffffu, my_tbase, src);
      const unsigned long long tend = __shfl_sync(0xffffffffu, my_tend, src);
      uint32_t j = 0;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        if (!((wv[w] >> lane) & 1u)) continue;
        const uint32_t r = before + j++;
        const long long at = n + r;
        if (at >= cap) continue;  // defensive: never past the branch's share
        const int64_t col = (int64_t)tt * TILE + 4 * lane + w;
        uint32_t val;
        if constexpr (VALUES) {
          const float inv = (float)inv_total[col];
          const uint32_t *pc = count_tile(cnt, cslot, b, tt, n_tiles);
          const float v = pc ? L * ((float)pc[col % TILE] * inv) : 0.f;
          val = __float2uint_rn(v * scale);
        } else {
          val = q;
        }
        ents[base + at] = ((unsigned long long)val << 32) | (unsigned long long)(uint32_t)col;
        const unsigned long long rp = tbase + slot + r;
        if (rp < tend && rp < n_ent) trec[rp] = make_uint2((uint32_t)(base + at), end);
      }
      n += total;
    }
  }
}

// First index in [lo, hi] of a branch's (column-sorted) list entries whose
// column is >= target, by the whole warp: each round the 32 lanes probe
// evenly spaced entries and the ballot of "below" (a prefix, the entries
// being sorted) narrows the range to one gap, so a list of up to 1,024
// entries takes two rounds.  Warp-uniform arguments.
__device__ __forceinline__ uint32_t list_lower(const unsigned long long *__restrict__ ents,
                                               uint32_t lo, uint32_t hi, uint32_t target,
                                               int lane) {
  while (hi - lo > 32u) {
    const uint32_t step = (hi - lo + 31u) / 32u;
    const uint32_t idx = lo + (uint32_t)lane * step;
    const bool below = idx < hi && (uint32_t)__ldg(ents + idx) < target;
    const uint32_t c = (uint32_t)__popc(__ballot_sync(0xffffffffu, below));
    if (c == 0u) return lo;
    const uint32_t nhi = min(hi, lo + c * step);
    lo = lo + (c - 1u) * step + 1u;
    hi = nhi;
  }
  const bool below = lo + (uint32_t)lane < hi && (uint32_t)__ldg(ents + lo + lane) < target;
  return lo + (uint32_t)__popc(__ballot_sync(0xffffffffu, below));
}

// Persistent: each warp takes kListGrab records at a time from the queue, in
// record (column tile) order, and walks each record's later entries with its
// lanes.
template <bool PRES>
__global__ void __launch_bounds__(kListWarps * 32)
    k_pairs_list(const unsigned long long *__restrict__ toff, int32_t n_tiles,
                 const uint2 *__restrict__ trec, const unsigned long long *__restrict__ ents,
                 unsigned long long n_ent, const int32_t *__restrict__ item_of,
                 const int4 *__restrict__ jrange,
                 typename SparseCfg<PRES>::Acc *__restrict__ spart, unsigned int *__restrict__ queue,
                 unsigned long long *__restrict__ n_updates) {
  const int lane = threadIdx.x & 31;
  // defensive: never past the records written (one per entry)
  const unsigned long long n_rec = min(toff[n_tiles], n_ent);
  const uint32_t cols = (uint32_t)n_tiles * TILE;
  unsigned long long done = 0;
  for (;;) {
    unsigned long long r0 = 0;
    if (lane == 0) r0 = (unsigned long long)kListGrab * atomicAdd(queue, 1u);
    r0 = __shfl_sync(0xffffffffu, r0, 0);
    if (r0 >= n_rec) break;
    const uint32_t n_here = (uint32_t)min((unsigned long long)kListGrab, n_rec - r0);
    const uint2 mine = lane < (int)n_here ? trec[r0 + lane] : make_uint2(0u, 0u);
    for (uint32_t x = 0; x < n_here; ++x) {
      const uint32_t g = __shfl_sync(0xffffffffu, mine.x, x);
      const uint32_t end = __shfl_sync(0xffffffffu, mine.y, x);
      if (g >= end || end > n_ent) continue;  // defensive: a record must lie in the lists
      const unsigned long long ep = __ldg(ents + g);
      const uint32_t cp = (uint32_t)ep, vp = (uint32_t)(ep >> 32);
      if (cp >= cols) continue;  // defensive: a column must exist
      const int64_t row = (int64_t)(cp / TILE) * n_tiles;
      const uint32_t a = (cp % TILE) * TILE;
      // the run computes, in this row of tiles, the column tiles [x, y) and
      // [z, w) (from the work list; [0, n_tiles) when it has more runs): the
      // later entries of the branch in those columns, found by search
      const int4 jr = __ldg(jrange + cp / TILE);
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        const uint32_t c0 = (uint32_t)(part == 0 ? jr.x : jr.z) * TILE;
        const uint32_t c1 = (uint32_t)(part == 0 ? jr.y : jr.w) * TILE;
        if (c1 <= c0 || c1 <= cp + 1) continue;
        // a whole-row run (the whole matrix) needs no search
        const uint32_t q0 = c0 <= cp + 1 ? g + 1 : list_lower(ents, g + 1, end, c0, lane);
        const uint32_t q1 = c1 >= cols ? end : list_lower(ents, q0, end, c1, lane);
        for (uint32_t q = q0 + lane; q < q1; q += 32) {
          const unsigned long long eq = __ldg(ents + q);
          const uint32_t cq = (uint32_t)eq;
          if (cq >= cols) continue;
          const int32_t item = item_of[row + cq / TILE];
          if (item < 0) continue;
          const int64_t at = (int64_t)item * TILE * TILE + a + cq % TILE;
          if constexpr (PRES)
            atomicAdd(&spart[at], (unsigned long long)vp);
          else
            atomicAdd(&spart[at], min(vp, (uint32_t)(eq >> 32)));
          ++done;
        }
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) done += __shfl_xor_sync(0xffffffffu, done, off);
  if (lane == 0 && n_updates && done) atomicAdd(n_updates, done);
}

// ----------------------------------------------------------------------------
// unweighted, bit-packed lookup (FP64 sums)

constexpr int BG = 8;                              // groups per stage
constexpr int kGroupBytes = 256 * 8 + 2 * TILE;    // table + I bytes + J bytes

__global__ void __launch_bounds__(kThreads, 1)
    k_pairs_lookup(const WorkItem *__restrict__ items, const uint8_t *__restrict__ bytes,
                   int64_t ldb, const double *__restrict__ tables,
                   const uint32_t *__restrict__ gbits, int32_t g_words,
                   const double *__restrict__ a, OutSpec o,
                   unsigned long long *__restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char *sbuf = smem_raw;  // [2][BG][kGroupBytes]
  int32_t *list = reinterpret_cast<int32_t *>(smem_raw + 2 * BG * kGroupBytes);
  __shared__ int32_t list_n;

  const WorkItem it = items[blockIdx.x];
  const StudyDev sd = o.studies[it.study];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const uint32_t *bI = gbits + (int64_t)it.tile_i * g_words;
  const uint32_t *bJ = gbits + (int64_t)it.tile_j * g_words;
  const int64_t colI = (int64_t)it.tile_i * TILE, colJ = (int64_t)it.tile_j * TILE;
  constexpr int kTabChunks = 256 * 8 / 16;  // 128
  constexpr int kByteChunks = TILE / 16;    // 8
  constexpr int kChunks = kTabChunks + 2 * kByteChunks;

  double acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
  unsigned long long nsel = 0;

  auto load_stage = [&](int s, int buf, int n) {
    for (int c = tid; c < BG * kChunks; c += kThreads) {
      const int r = c / kChunks;
      const int q = c % kChunks;
      const int li = s * BG + r;
      if (li < n) {
        const int32_t g = list[li];
        unsigned char *dst = sbuf + (buf * BG + r) * kGroupBytes;
        const void *src;
        if (q < kTabChunks) {
          src = tables + (int64_t)g * 256 + q * 2;
          dst += q * 16;
        } else if (q < kTabChunks + kByteChunks) {
          src = bytes + (int64_t)g * ldb + colI + (q - kTabChunks) * 16;
          dst += 2048 + (q - kTabChunks) * 16;
        } else {
          src = bytes + (int64_t)g * ldb + colJ + (q - kTabChunks - kByteChunks) * 16;
          dst += 2048 + TILE + (q - kTabChunks - kByteChunks) * 16;
        }
        cp_async16(dst, src);
      }
    }
  };

  for (int w0 = 0; w0 < g_words; w0 += kWinWords) {
    if (tid < 32) build_window(bI, bJ, g_words, w0, list, &list_n);
    __syncthreads();
    const int n = list_n;
    nsel += (unsigned long long)n;
    const int ns = (n + BG - 1) / BG;
    if (ns > 0) {
      load_stage(0, 0, n);
      cp_commit();
      for (int s = 0; s < ns; ++s) {
        if (s + 1 < ns) {
          load_stage(s + 1, (s + 1) & 1, n);
          cp_commit();
          cp_wait<1>();
        } else {
          cp_wait<0>();
        }
        __syncthreads();
        const int rows = min(BG, n - s * BG);
        for (int r = 0; r < rows; ++r) {
          const unsigned char *grp = sbuf + ((s & 1) * BG + r) * kGroupBytes;
          const double *T = reinterpret_cast<const double *>(grp);
          const uint32_t xi0 = *reinterpret_cast<const uint32_t *>(grp + 2048 + ty * 4);
          const uint32_t xi1 = *reinterpret_cast<const uint32_t *>(grp + 2048 + 64 + ty * 4);
          const uint32_t xj0 = *reinterpret_cast<const uint32_t *>(grp + 2048 + TILE + tx * 4);
          const uint32_t xj1 = *reinterpret_cast<const uint32_t *>(grp + 2048 + TILE + 64 + tx * 4);
#pragma unroll
          for (int qj = 0; qj < 8; ++qj) {
            const uint32_t xj = (qj < 4) ? xj0 : xj1;
            const uint32_t rep = ((xj >> (8 * (qj & 3))) & 0xffu) * 0x01010101u;
            const uint32_t m0 = xi0 & rep, m1 = xi1 & rep;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              acc[q][qj] += T[(m0 >> (8 * q)) & 0xffu];
              acc[4 + q][qj] += T[(m1 >> (8 * q)) & 0xffu];
            }
          }
        }
        __syncthreads();
      }
    }
    __syncthreads();
  }
  if (tid == 0 && counter) atomicAdd(counter, nsel);

  // epilogue: d = (a_i + a_j - 2 G) / (a_i + a_j - G)
#pragma unroll
  for (int qi = 0; qi < 8; ++qi) {
    const int i = own_row(ty, qi);
    const int li = (int)(colI + i) - sd.col0;
    if (li >= sd.n) continue;
    const double ai = a[colI + i];
#pragma unroll
    for (int qj = 0; qj < 8; ++qj) {
      const int j = own_row(tx, qj);
      const int lj = (int)(colJ + j) - sd.col0;
      if (lj >= sd.n) continue;
      if (li < lj) {
        const double A = ai + a[colJ + j];
        const double G = acc[qi][qj];
        put_pair(o, sd, li, lj, ratio01(A - 2.0 * G, A - G));
      } else if (li == lj) {
        put_diag(o, sd, li);
      }
    }
  }
}

// The dense weighted kernel over all work items: one launch, or, when this
// variant's matrix goes to host memory range by range (unifrac_ctx::cc_*),
// one launch per range of items, each followed by the copy of what it
// completed.  launch(a, b) enqueues the kernel over items [a, b).
template <typename L>
int dense_ranges(unifrac_ctx *ctx, int32_t n_items, L launch) {
  const bool ranges = ctx->cc_variant == ctx->cur_slot && ctx->cc_n > 0 && !ctx->capturing &&
                      ctx->cc_items.size() == (size_t)ctx->cc_n + 1 &&
                      ctx->cc_items.back() == n_items;
  const int n = ranges ? ctx->cc_n : 1;
  for (int c = 0; c < n; ++c) {
    const int32_t a = ranges ? ctx->cc_items[c] : 0, b = ranges ? ctx->cc_items[c + 1] : n_items;
    if (b > a) {
      const cudaError_t e = launch(a, b);
      ctx->stat_launches += 1;
      if (e != cudaSuccess) return cuda_fail(ctx, e, "weighted kernel");
    }
    if (ranges) {
      const int rc = enqueue_range_copy(ctx, c);
      if (rc) return rc;
    }
  }
  return UNIFRAC_OK;
}

}  // namespace

int pairs_weighted(unifrac_ctx *ctx, bool f64, const void *vals, const uint32_t *bits,
                   int32_t kf_words, int32_t vr_words, const uint8_t *blocks,
                   const unsigned long long *boff, const uint2 *cpre, int32_t n_win,
                   ListBufs list, uint32_t *spart, int32_t sp_parts, const double *S,
                   const WorkItem *items, int32_t n_items, const OutSpec &o) {
  if (n_items <= 0) return UNIFRAC_OK;
  const int32_t n_words = ctx->K_pad / WORD;
  const size_t elem = f64 ? sizeof(double) : sizeof(float);
  const size_t smem = elem * 2 * BK * 2 * TILE + sizeof(int32_t) * kWinWords * WORD +
                      (f64 ? 0 : sizeof(float) * TILE * TILE);  // FP32 running totals
  cudaError_t e;
  if (f64) {
    // no sparse or list phase in FP64: empty windows
    for (cudaEvent_t ev : {ctx->ev_sp[1][0], ctx->ev_list[1][0], ctx->ev_list[1][1], ctx->ev_sp[1][1]})
      record_event(ctx, ev);
    e = cudaFuncSetAttribute(k_pairs_weighted<double>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "weighted kernel attribute");
    return dense_ranges(ctx, n_items, [&](int32_t a, int32_t b) {
      k_pairs_weighted<double><<<b - a, kThreads, smem, ctx->stream>>>(
          items, n_items, a, b, nullptr, static_cast<const double *>(vals), ctx->n_cols, bits,
          n_words, n_words, nullptr, 1, 1.0, S, 0, o, cur_counters(ctx));
      return cudaGetLastError();
    });
  } else {
    // a sparse part exists when some positions are neither dense nor listed
    // (n_win > 0) or some are listed; the listed ones add into the sparse
    // kernel's partial sums (part 0), so those are written or cleared first
    const bool listed = list.ents != nullptr && vr_words * WORD < ctx->K;
    const bool sparse = n_win > 0 || listed;
    record_event(ctx, ctx->ev_sp[1][0]);
    if (sparse && n_win <= 0) {
      e = cudaMemsetAsync(spart, 0, (size_t)n_items * sp_parts * TILE * TILE * sizeof(uint32_t),
                          ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "clear sparse sums");
    }
    if (n_win > 0) {
      constexpr size_t kSm = SparseCfg<false>::kSmem;
      e = cudaFuncSetAttribute(k_pairs_sparse<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kSm);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "sparse weighted kernel attribute");
      unsigned int *q = cur_queue(ctx, 1);
      const dim3 grid = q ? dim3(pair_grid(ctx, k_pairs_sparse<false>, kSpThreads, kSm,
                                           (int64_t)n_items * sp_parts))
                          : dim3(n_items, sp_parts);
      k_pairs_sparse<false><<<grid, kSpThreads, kSm, ctx->stream>>>(
          items, n_items, q, bits, n_words, kf_words, vr_words, n_win, blocks, boff,
          cur_bufs(ctx).blocks.bytes, ctx->n_tiles, cpre, nullptr, sp_parts, ctx->opt_lane_pairs[1],
          spart,
          cur_counters(ctx) + 2);
      ctx->stat_launches += 1;
    }
    record_event(ctx, ctx->ev_list[1][0]);
    if (listed) {
      int rc = pairs_list(ctx, false, vr_words * WORD, list, spart);
      if (rc) return rc;
    }
    record_event(ctx, ctx->ev_list[1][1]);
    record_event(ctx, ctx->ev_sp[1][1]);
    e = cudaFuncSetAttribute(k_pairs_weighted<float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "weighted kernel attribute");
    unsigned int *q = cur_queue(ctx, 0);
    return dense_ranges(ctx, n_items, [&](int32_t a, int32_t b) {
      // each range's queue starts at 0 (the first was cleared with the others)
      if (q && a > 0) {
        const cudaError_t m = cudaMemsetAsync(q, 0, sizeof(unsigned int), ctx->stream);
        if (m != cudaSuccess) return m;
      }
      k_pairs_weighted<float><<<pair_grid(ctx, k_pairs_weighted<float>, kThreads, smem, b - a),
                                kThreads, smem, ctx->stream>>>(
          items, n_items, a, b, q, static_cast<const float *>(vals), ctx->n_cols, bits, n_words,
          kf_words, sparse ? spart : nullptr, sp_parts, 1.0 / (double)ctx->sp_scale, S,
          ctx->opt_flush, o, cur_counters(ctx));
      return cudaGetLastError();
    });
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "weighted pair kernel");
  return UNIFRAC_OK;
}

int pairs_sparse_presence(unifrac_ctx *ctx, const uint32_t *bits, int32_t kf_words,
                          int32_t vr_words, const uint8_t *blocks, const unsigned long long *boff,
                          const uint2 *cpre, int32_t n_win, ListBufs list,
                          unsigned long long *spart, const WorkItem *items, int32_t n_items) {
  const bool listed = list.ents != nullptr && vr_words * WORD < ctx->K;
  if (n_items <= 0 || (n_win <= 0 && !listed)) {
    record_event(ctx, ctx->ev_list[0][0]);  // an empty list phase
    record_event(ctx, ctx->ev_list[0][1]);
    return UNIFRAC_OK;
  }
  auto run_list = [&]() -> int {
    record_event(ctx, ctx->ev_list[0][0]);
    if (listed) {
      int rc = pairs_list(ctx, true, vr_words * WORD, list, spart);
      if (rc) return rc;
    }
    record_event(ctx, ctx->ev_list[0][1]);
    return UNIFRAC_OK;
  };
  if (n_win <= 0) {  // only listed positions: their sums start from zero
    cudaError_t e = cudaMemsetAsync(spart, 0, (size_t)n_items * TILE * TILE * 8, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "clear sparse sums");
    return run_list();
  }
  const int32_t n_words = ctx->K_pad / WORD;
  constexpr size_t kSm = SparseCfg<true>::kSmem;
  cudaError_t e =
      cudaFuncSetAttribute(k_pairs_sparse<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSm);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sparse unweighted kernel attribute");
  unsigned int *q = cur_queue(ctx, 1);
  k_pairs_sparse<true><<<pair_grid(ctx, k_pairs_sparse<true>, kSpThreads, kSm, n_items),
                         kSpThreads, kSm, ctx->stream>>>(
      items, n_items, q, bits, n_words, kf_words, vr_words, n_win, blocks, boff,
      cur_bufs(ctx).blocks.bytes, ctx->n_tiles, cpre, ctx->d_qperm, 1, ctx->opt_lane_pairs[0],
      spart,
      cur_counters(ctx) + 2);
  ctx->stat_launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sparse unweighted kernel");
  return run_list();
}

int list_fill(unifrac_ctx *ctx, bool values, const uint32_t *cnt, const uint8_t *flag,
              const uint32_t *bits, const uint8_t *rc, int32_t pv, const long long *voff,
              ListBufs L) {
  const int64_t n = (int64_t)ctx->K - pv;
  if (n <= 0 || ctx->n_tiles <= 0) return UNIFRAC_OK;
  cudaStream_t st = ctx->stream;
  // records per column tile (from the sparse packing's row counts), their
  // offsets, and zeroed fill cursors
  k_list_tile_counts<<<ctx->n_tiles, 256, 0, st>>>(pv, ctx->K, ctx->K_pad, bits,
                                                   ctx->K_pad / WORD, rc, L.tcnt);
  int rc_ = scan_sizes(ctx, ctx->n_tiles, L.tcnt, L.toff);
  if (rc_) return rc_;
  cudaError_t e = cudaMemsetAsync(L.tcur, 0, (size_t)ctx->n_tiles * sizeof(uint32_t), st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "clear list cursors");
  const unsigned grid = (unsigned)((n + kListWarps - 1) / kListWarps);
  if (values)
    k_list_fill<true><<<grid, kListWarps * 32, 0, st>>>(
        pv, ctx->K, ctx->d_perm, flag, reinterpret_cast<const uint4 *>(ctx->d_pmask),
        ctx->n_tiles, cnt, ctx->d_slot, ctx->d_len_perm, ctx->d_inv_total, ctx->sp_scale, nullptr,
        voff, L.ents, L.toff, L.tcur, L.trec, L.n_ent);
  else
    k_list_fill<false><<<grid, kListWarps * 32, 0, st>>>(
        pv, ctx->K, ctx->d_perm, flag, reinterpret_cast<const uint4 *>(ctx->d_pmask),
        ctx->n_tiles, cnt, ctx->d_slot, nullptr, nullptr, 1.f, ctx->d_qperm, voff, L.ents, L.toff,
        L.tcur, L.trec, L.n_ent);
  ctx->stat_launches += 2;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rare branch lists");
  return UNIFRAC_OK;
}

int pairs_list(unifrac_ctx *ctx, bool presence, int32_t pv, ListBufs L, void *spart) {
  const int64_t n = (int64_t)ctx->K - pv;
  if (n <= 0 || ctx->n_tiles <= 0) return UNIFRAC_OK;
  const int32_t *item_of = static_cast<const int32_t *>(ctx->item_of.p);
  const int4 *jrange = static_cast<const int4 *>(ctx->jrange.p);
  // the list queue: the slot's third 32-bit queue counter (cleared with the others)
  unsigned int *queue = reinterpret_cast<unsigned int *>(ctx->d_counter + 4 * ctx->cur_slot + 2);
  // kListBlocksPerSm CTAs per SM: the records in flight (kListGrab per warp)
  // then span a few column tiles, whose partial sums stay in L2
  const unsigned grid = (unsigned)(kListBlocksPerSm * ctx->sm_count);
  if (presence)
    k_pairs_list<true><<<grid, kListWarps * 32, 0, ctx->stream>>>(
        L.toff, ctx->n_tiles, L.trec, L.ents, L.n_ent, item_of, jrange,
        static_cast<unsigned long long *>(spart), queue, cur_counters(ctx) + 3);
  else
    k_pairs_list<false><<<grid, kListWarps * 32, 0, ctx->stream>>>(
        L.toff, ctx->n_tiles, L.trec, L.ents, L.n_ent, item_of, jrange,
        static_cast<uint32_t *>(spart), queue, cur_counters(ctx) + 3);
  ctx->stat_launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rare branch pairs");
  return UNIFRAC_OK;
}

int pairs_lookup(unifrac_ctx *ctx, const uint8_t *bytes, const double *tables,
                 const uint32_t *gbits, const double *a, const WorkItem *items, int32_t n_items,
                 const OutSpec &o) {
  if (n_items <= 0) return UNIFRAC_OK;
  const int32_t G = ctx->K_pad / 8;
  const int32_t g_words = (G + WORD - 1) / WORD;
  const size_t smem = 2 * BG * kGroupBytes + sizeof(int32_t) * kWinWords * WORD;
  cudaError_t e = cudaFuncSetAttribute(k_pairs_lookup,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lookup kernel attribute");
  k_pairs_lookup<<<n_items, kThreads, smem, ctx->stream>>>(items, bytes, ctx->n_cols, tables,
                                                           gbits, g_words, a, o, cur_counters(ctx));
  ctx->stat_launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lookup pair kernel");
  return UNIFRAC_OK;
}

}  // namespace ufb
