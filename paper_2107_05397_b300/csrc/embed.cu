// K1: per-branch embedding of every sample, and the packing kernels that turn
// it into the operand layout of each pair kernel.
//
// Section II of the paper: UniFrac accounts for the evolutionary relationships
// between microbes -- a sample's abundance below a branch counts toward that
// branch.  For branch b and sample i the embedding is the count of sample i on
// the tips below b; the relative abundance is that count over the sample total.
//
// The tree is in postorder, so a node's children are finished before it.  The
// kernels here are level-synchronous: level 0 holds the tips, level L the nodes
// whose highest child is on level L-1, and one launch sums the children of all
// nodes of one level.  Counts are held per (node, 128-column tile) for the
// tiles where the node has a non-zero count (the create-time slot map gives
// each such tile its row of 128 u32 in a compact array; 22 % of the tiles at
// 50,000 samples on a 400,000-node tree), processed by one warp per tile
// (16-byte loads); a (node, tile) flag records whether the tile has any
// non-zero count, and tiles whose children are all zero are neither read nor
// written (the sparse-aware step: most features are absent from most
// samples).  Counts are summed as
// exact integers; the division by the sample total happens once, in packing.
#include <algorithm>

#include "ufb_internal.cuh"

namespace ufb {

namespace {

constexpr int kWarpsPerBlock = 8;

// Presence mask of a 128-column tile row held as one uint4 per lane (lane l:
// columns 4 l .. 4 l + 3): word w has bit l set when column 4 l + w is
// non-zero.  Every lane of the warp must call it.
__device__ __forceinline__ uint4 nonzero_mask(const uint4 &v) {
  return make_uint4(__ballot_sync(0xffffffffu, v.x != 0u), __ballot_sync(0xffffffffu, v.y != 0u),
                    __ballot_sync(0xffffffffu, v.z != 0u), __ballot_sync(0xffffffffu, v.w != 0u));
}

// Tip rows, in chunks of at most `chunk` entries of one table row (a feature
// on a tip), one warp per chunk: rows are uneven (a common feature has an
// entry in nearly every sample), chunks are not.  Two launches: k_tip_zero
// zeroes and flags every 128-column tile a row touches, each tile by the
// chunk that holds the row's first entry in it, then k_tip_scatter writes
// the counts (two chunks of a row can share a tile, so every zeroing must
// come before any count).
__global__ void k_tip_zero(int64_t n_chunks, const int32_t *__restrict__ chunk_row,
                           const int64_t *__restrict__ chunk_lo, int64_t chunk,
                           const int32_t *__restrict__ frow_tip,
                           const int64_t *__restrict__ frow_ptr,
                           const int32_t *__restrict__ ent_col, uint32_t *cnt,
                           const uint32_t *__restrict__ slot, uint8_t *flag, uint4 *pmask,
                           int32_t n_tiles) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n_chunks) return;
  const int32_t r = chunk_row[warp];
  const int64_t lo = chunk_lo[warp], rlo = frow_ptr[r], hi = min(frow_ptr[r + 1], lo + chunk);
  const int32_t tip = frow_tip[r];
  // the whole warp writes one tile (32 lanes x 16 bytes) per step, tiles
  // found by a ballot over 32 entries
  for (int64_t base = lo; base < hi; base += 32) {
    const int64_t e = base + lane;
    int32_t t = -1;
    bool first = false;
    if (e < hi) {
      t = ent_col[e] / TILE;
      first = e == rlo || ent_col[e - 1] / TILE != t;
    }
    for (uint32_t m = __ballot_sync(0xffffffffu, first); m; m &= m - 1) {
      const int32_t ts = __shfl_sync(0xffffffffu, t, __ffs(m) - 1);
      uint32_t *tr = count_tile(cnt, slot, tip, ts, n_tiles);
      if (tr) reinterpret_cast<uint4 *>(tr)[lane] = make_uint4(0u, 0u, 0u, 0u);
      if (lane == 0) {
        flag[(int64_t)tip * n_tiles + ts] = 1;
        pmask[(int64_t)tip * n_tiles + ts] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
  }
}

__global__ void k_tip_scatter(int64_t n_chunks, const int32_t *__restrict__ chunk_row,
                              const int64_t *__restrict__ chunk_lo, int64_t chunk,
                              const int32_t *__restrict__ frow_tip,
                              const int64_t *__restrict__ frow_ptr,
                              const int32_t *__restrict__ ent_col,
                              const uint32_t *__restrict__ ent_cnt, uint32_t *cnt,
                              const uint32_t *__restrict__ slot, uint32_t *pmask_w,
                              int32_t n_tiles) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n_chunks) return;
  const int32_t r = chunk_row[warp];
  const int64_t lo = chunk_lo[warp], hi = min(frow_ptr[r + 1], lo + chunk);
  const int32_t tip = frow_tip[r];
  uint32_t *pm = pmask_w + (int64_t)tip * n_tiles * 4;
#pragma unroll 4
  for (int64_t e = lo + lane; e < hi; e += 32) {
    const int32_t c = ent_col[e];
    const uint32_t v = ent_cnt[e];
    uint32_t *tr = count_tile(cnt, slot, tip, c / TILE, n_tiles);
    if (tr) tr[c % TILE] = v;
    // column 4 l + w of a tile is bit l of the tile's mask word w
    if (v) atomicOr(pm + (int64_t)(c / TILE) * 4 + (c & 3), 1u << ((c % TILE) >> 2));
  }
}

// One level: for every (node of the level, column tile), sum the flagged
// children's tiles.  A warp owns one node and 32 consecutive tiles: lane l
// ORs the children's flags of tile 32 g + l (and keeps which children had
// the tile, for nodes of at most 32 children), then the warp sums the rows of
// each flagged tile together (32 lanes x uint4 = 128 columns).  Sparse levels
// cost one warp per 32 tiles instead of one per tile.
__global__ void k_level(const int32_t *__restrict__ nodes, int32_t n_level,
                        const int32_t *__restrict__ child_ptr,
                        const int32_t *__restrict__ child_idx, uint32_t *cnt,
                        const uint32_t *__restrict__ slot, uint8_t *flag, uint4 *pmask,
                        int32_t n_tiles) {
  const int32_t n_groups = (n_tiles + 31) / 32;
  const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (item >= (int64_t)n_level * n_groups) return;  // whole warps
  const int32_t node = nodes[item / n_groups];
  const int32_t t = (int32_t)(item % n_groups) * 32 + lane;
  const int32_t c0 = child_ptr[node], c1 = child_ptr[node + 1];
  const bool few = c1 - c0 <= 32;
  uint32_t fmask = 0;  // children (by position) that have tile t
  if (t < n_tiles)
    for (int32_t c = c0; c < c1; ++c)
      if (flag[(int64_t)child_idx[c] * n_tiles + t]) fmask |= few ? 1u << (c - c0) : 1u;
  if (t < n_tiles) flag[(int64_t)node * n_tiles + t] = fmask ? 1 : 0;
  const int32_t gbase = (int32_t)(item % n_groups) * 32;
  uint32_t m = __ballot_sync(0xffffffffu, fmask != 0);
  if (c1 - c0 == 2) {
    // two children (nearly every node of a binary tree): two flagged tiles
    // per pass, the four child rows' loads issued before either store
    const int32_t ch0 = child_idx[c0], ch1 = child_idx[c0 + 1];
    // a child's tile, or nullptr when it has no counts there
    auto child = [&](int32_t ch, bool has, int32_t t) -> const uint4 * {
      const uint32_t *p = has ? count_tile(cnt, slot, ch, t, n_tiles) : nullptr;
      return p ? reinterpret_cast<const uint4 *>(p) + lane : nullptr;
    };
    while (m) {
      const int sa = __ffs(m) - 1;
      m &= m - 1;
      const int sb = m ? __ffs(m) - 1 : -1;
      if (m) m &= m - 1;
      const uint32_t fa = __shfl_sync(0xffffffffu, fmask, sa);
      const uint32_t fb = __shfl_sync(0xffffffffu, fmask, sb < 0 ? sa : sb);
      const int32_t ta = gbase + sa, tb = gbase + (sb < 0 ? sa : sb);
      const uint4 z = make_uint4(0u, 0u, 0u, 0u);
      const uint4 *pa0 = child(ch0, fa & 1u, ta), *pa1 = child(ch1, fa & 2u, ta);
      const uint4 *pb0 = child(ch0, sb >= 0 && (fb & 1u), tb);
      const uint4 *pb1 = child(ch1, sb >= 0 && (fb & 2u), tb);
      const uint4 a0 = pa0 ? __ldg(pa0) : z;
      const uint4 a1 = pa1 ? __ldg(pa1) : z;
      const uint4 b0 = pb0 ? __ldg(pb0) : z;
      const uint4 b1 = pb1 ? __ldg(pb1) : z;
      const uint4 sumA = make_uint4(a0.x + a1.x, a0.y + a1.y, a0.z + a1.z, a0.w + a1.w);
      const uint4 sumB = make_uint4(b0.x + b1.x, b0.y + b1.y, b0.z + b1.z, b0.w + b1.w);
      uint32_t *na = count_tile(cnt, slot, node, ta, n_tiles);
      if (na) reinterpret_cast<uint4 *>(na)[lane] = sumA;
      if (sb >= 0) {
        uint32_t *nb = count_tile(cnt, slot, node, tb, n_tiles);
        if (nb) reinterpret_cast<uint4 *>(nb)[lane] = sumB;
      }
      const uint4 ma = nonzero_mask(sumA);
      if (lane == 0) pmask[(int64_t)node * n_tiles + gbase + sa] = ma;
      if (sb >= 0) {  // warp-uniform
        const uint4 mb = nonzero_mask(sumB);
        if (lane == 0) pmask[(int64_t)node * n_tiles + gbase + sb] = mb;
      }
    }
    return;
  }
  for (; m; m &= m - 1) {
    const int src = __ffs(m) - 1;
    const int32_t ts = gbase + src;
    const uint32_t fm = __shfl_sync(0xffffffffu, fmask, src);
    uint4 s = make_uint4(0u, 0u, 0u, 0u);
    for (int32_t c = c0; c < c1; ++c) {
      const int32_t ch = child_idx[c];
      const uint32_t *ct = (few ? ((fm >> (c - c0)) & 1u) != 0u : flag[(int64_t)ch * n_tiles + ts] != 0)
                               ? count_tile(cnt, slot, ch, ts, n_tiles)
                               : nullptr;
      if (ct) {
        const uint4 v = reinterpret_cast<const uint4 *>(ct)[lane];
        s.x += v.x;
        s.y += v.y;
        s.z += v.z;
        s.w += v.w;
      }
    }
    uint32_t *nt = count_tile(cnt, slot, node, ts, n_tiles);
    if (nt) reinterpret_cast<uint4 *>(nt)[lane] = s;
    const uint4 ms = nonzero_mask(s);
    if (lane == 0) pmask[(int64_t)node * n_tiles + ts] = ms;
  }
}

// The upper levels hold few nodes each, too few to fill the GPU one launch per
// level.  k_levels_tail walks levels [L0, L1) in one launch: CTA (t, q) owns
// the 32 columns 128 t + 32 q .. +31, and each warp takes four nodes of a
// level at a time (eight lanes x 16 bytes per node); __syncthreads separates
// the levels, since a level reads only what earlier levels wrote for the same
// columns.  Global memory is read with plain (coherent) loads, and only the
// tiles of children that have counts there.  A node's
// flag is the same for the four quarters of its tile, so their stores agree;
// each quarter writes its own byte of every word of the presence mask.
constexpr int kTailThreads = 1024;

__global__ void __launch_bounds__(kTailThreads) k_levels_tail(
    const int32_t *__restrict__ nodes, const int32_t *__restrict__ level_ptr, int32_t L0,
    int32_t L1, const int32_t *__restrict__ child_ptr, const int32_t *__restrict__ child_idx,
    uint32_t *cnt, const uint32_t *__restrict__ slot, uint8_t *flag, uint8_t *pmask_b,
    int32_t n_tiles) {
  const int t = blockIdx.x >> 2, q = blockIdx.x & 3;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 3, l8 = lane & 7;
  const int off = q * 32 + l8 * 4;  // this lane's 4 columns within the tile
  for (int L = L0; L < L1; ++L) {
    const int32_t lo = level_ptr[L], hi = level_ptr[L + 1];
    // warp-uniform trip count (the mask ballots need every lane)
    for (int32_t i0 = lo + warp * 4; i0 < hi; i0 += (kTailThreads / 32) * 4) {
      const int32_t i = i0 + g;
      const bool act = i < hi;
      int32_t node = 0;
      uint4 s = make_uint4(0u, 0u, 0u, 0u);
      bool any = false;
      if (act) {
        node = nodes[i];
        const int32_t c0 = child_ptr[node], c1 = child_ptr[node + 1];
        if (c1 - c0 == 2) {
          // two children: both rows loaded beside their flags (near the root
          // both children nearly always hold the tile), then selected
          const int32_t ch0 = child_idx[c0], ch1 = child_idx[c0 + 1];
          const uint8_t f0 = flag[(int64_t)ch0 * n_tiles + t], f1 = flag[(int64_t)ch1 * n_tiles + t];
          const uint32_t *p0 = f0 ? count_tile(cnt, slot, ch0, t, n_tiles) : nullptr;
          const uint32_t *p1 = f1 ? count_tile(cnt, slot, ch1, t, n_tiles) : nullptr;
          const uint4 z = make_uint4(0u, 0u, 0u, 0u);
          const uint4 v0 = p0 ? *reinterpret_cast<const uint4 *>(p0 + off) : z;
          const uint4 v1 = p1 ? *reinterpret_cast<const uint4 *>(p1 + off) : z;
          any = (f0 | f1) != 0;
          s = make_uint4(v0.x + v1.x, v0.y + v1.y, v0.z + v1.z, v0.w + v1.w);
        } else {
          for (int32_t c = c0; c < c1; ++c) {
            const int32_t ch = child_idx[c];
            if (flag[(int64_t)ch * n_tiles + t]) {
              any = true;
              const uint32_t *pc = count_tile(cnt, slot, ch, t, n_tiles);
              if (!pc) continue;
              const uint4 v = *reinterpret_cast<const uint4 *>(pc + off);
              s.x += v.x;
              s.y += v.y;
              s.z += v.z;
              s.w += v.w;
            }
          }
        }
        if (l8 == 0) flag[(int64_t)node * n_tiles + t] = any ? 1 : 0;
        if (any) {
          uint32_t *pn = count_tile(cnt, slot, node, t, n_tiles);
          if (pn) *reinterpret_cast<uint4 *>(pn + off) = s;
        }
      }
      // this quarter's bits of the tile's presence mask: bits 8 q .. 8 q + 7
      // of each word, i.e. byte q (lanes of group g are ballot bits 8 g ..)
      const uint4 m = nonzero_mask(s);
      if (act && any && l8 == 0) {
        uint8_t *pb = pmask_b + ((int64_t)node * n_tiles + t) * 16 + q;
        pb[0] = (uint8_t)(m.x >> (8 * g));
        pb[4] = (uint8_t)(m.y >> (8 * g));
        pb[8] = (uint8_t)(m.z >> (8 * g));
        pb[12] = (uint8_t)(m.w >> (8 * g));
      }
    }
    __syncthreads();
  }
}

// Weighted packing of the positions [0, k_end) (all of them, or the frequently
// present ones when the rest go to the sparse blocks).  Block (column tile t,
// KR positions), warp w per bitmap word: lane l tests position 32 w + l and
// the ballot is the (t, word) bitmap word; the flagged rows are then read four
// at a time (16 bytes per lane) and written as
// v[k][col] = len_k * cnt[perm[k]][col] / C_col.  The mixed form computes v in
// FP32 (<= 3 roundings); the FP64 form in FP64.  k_end is K or a multiple of
// 32, so bitmap words never straddle it.
constexpr int KR = 256;

template <typename T>
__global__ void __launch_bounds__(256) k_pack_weighted(
    int32_t K, int32_t k_end, const int32_t *__restrict__ perm,
    const double *__restrict__ len_perm, const uint32_t *__restrict__ cnt,
    const uint8_t *__restrict__ flag, const uint32_t *__restrict__ slot, int32_t n_tiles,
    const double *__restrict__ inv_total, T *__restrict__ vals, int64_t ldv,
    uint32_t *__restrict__ bits, int32_t n_words) {
  const int t = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kw = blockIdx.y * KR + w * WORD;
  if (kw >= k_end) return;  // warp-uniform
  const int64_t col = (int64_t)t * TILE + lane * 4;
  const int k = kw + lane;
  const int k1 = min(K, k_end);
  const int32_t b = k < k1 ? perm[k] : 0;
  const bool fl = k < k1 && flag[(int64_t)b * n_tiles + t];
  const uint32_t word = __ballot_sync(0xffffffffu, fl);
  if (lane == 0 && kw / WORD < n_words) bits[(int64_t)t * n_words + kw / WORD] = word;
  T inv[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) inv[q] = (T)inv_total[col + q];
  uint32_t m = word;
  while (m) {
    constexpr int kU = 4;
    int src[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      src[u] = -1;
      if (m) {
        src[u] = __ffs(m) - 1;
        m &= m - 1;
      }
    }
    uint4 c[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      c[u] = make_uint4(0u, 0u, 0u, 0u);
      if (src[u] >= 0) {
        const int32_t bu = __shfl_sync(0xffffffffu, b, src[u]);
        const uint32_t *pc = count_tile(cnt, slot, bu, t, n_tiles);
        if (pc) c[u] = *reinterpret_cast<const uint4 *>(pc + lane * 4);
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (src[u] < 0) break;
      const int kk = kw + src[u];
      const T L = (T)len_perm[kk];
      if constexpr (sizeof(T) == 4) {
        float4 v;
        v.x = L * ((float)c[u].x * inv[0]);
        v.y = L * ((float)c[u].y * inv[1]);
        v.z = L * ((float)c[u].z * inv[2]);
        v.w = L * ((float)c[u].w * inv[3]);
        *reinterpret_cast<float4 *>(vals + (int64_t)kk * ldv + col) = v;
      } else {
        double2 v0, v1;
        v0.x = L * ((double)c[u].x * inv[0]);
        v0.y = L * ((double)c[u].y * inv[1]);
        v1.x = L * ((double)c[u].z * inv[2]);
        v1.y = L * ((double)c[u].w * inv[3]);
        double2 *dst = reinterpret_cast<double2 *>(vals + (int64_t)kk * ldv + col);
        dst[0] = v0;
        dst[1] = v1;
      }
    }
  }
}

// Lookup packing.  Block (column tile t, group block gb) of 128 threads, one
// column each, reading the presence masks of the flagged rows.  Group g holds
// positions 8g..8g+7; the byte of (g, col) has bit j set when branch 8g+j is
// present in col.  Also the (t, g) group bitmap and FP64 partial sums of
// a_col = sum_k len_k p[k][col] per group block.
constexpr int GR = 32;  // groups per block

__global__ void __launch_bounds__(128) k_pack_lookup(
    int32_t K, int32_t G, const int32_t *__restrict__ perm,
    const double *__restrict__ len_perm, const uint4 *__restrict__ pmask,
    const uint8_t *__restrict__ flag, int32_t n_cols, int32_t n_tiles,
    uint8_t *__restrict__ bytes, uint32_t *__restrict__ gbits, int32_t g_words,
    double *__restrict__ partial) {
  const int t = blockIdx.x;
  const int g0 = blockIdx.y * GR;
  const int64_t col = (int64_t)t * TILE + threadIdx.x;
  // this column in the presence masks: bit threadIdx.x / 4 of word threadIdx.x % 4
  const int mw = threadIdx.x & 3, mb = threadIdx.x >> 2;
  double a = 0.0;
  uint32_t gword = 0;
  for (int gi = 0; gi < GR; ++gi) {
    const int g = g0 + gi;
    if (g >= G) break;
    uint32_t byte = 0;
    bool anyflag = false;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = 8 * g + j;
      if (k < K) {
        const int32_t b = perm[k];
        if (flag[(int64_t)b * n_tiles + t]) {
          anyflag = true;
          const uint4 pm = pmask[(int64_t)b * n_tiles + t];
          const uint32_t word = mw == 0 ? pm.x : mw == 1 ? pm.y : mw == 2 ? pm.z : pm.w;
          if ((word >> mb) & 1u) {
            byte |= 1u << j;
            a += len_perm[k];
          }
        }
      }
    }
    bytes[(int64_t)g * n_cols + col] = (uint8_t)byte;
    if (anyflag) gword |= 1u << gi;
  }
  if (threadIdx.x == 0 && g0 / WORD < g_words) gbits[(int64_t)t * g_words + g0 / WORD] = gword;
  partial[(int64_t)blockIdx.y * n_cols + col] = a;
}

// T[g][m] = sum of len of the branches whose bit is set in m (FP64, bit order).
__global__ void k_lookup_tables(int32_t K, const double *__restrict__ len_perm,
                                double *__restrict__ tables) {
  const int g = blockIdx.x;
  const int m = threadIdx.x;  // 256 threads
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = 8 * g + j;
    if ((m >> j) & 1) s += (k < K) ? len_perm[k] : 0.0;
  }
  tables[(int64_t)g * 256 + m] = s;
}

// a_col = sum over blocks of the partials, in block order (deterministic).
__global__ void k_reduce_partials(int32_t n_cols, int32_t n_blocks,
                                  const double *__restrict__ partial, double *__restrict__ a) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n_cols) return;
  double s = 0.0;
  for (int b = 0; b < n_blocks; ++b) s += partial[(int64_t)b * n_cols + col];
  a[col] = s;
}

// ---------------------------------------------------------------------------
// Sparse blocks of the rarely present positions.  For every column tile t and
// window j of kRareWin positions starting at p0 (the first rarely present
// position), one block holds the tile's non-zero entries of the window's
// flagged rows:
//   u32 nrows, nent, off_ent, 0             (16-byte header)
//   u32 rowstart[nrows + 1]                 entry offset of each flagged row
//   entries at off_ent (16-byte aligned), one per non-zero column:
//     weighted blocks: u64 (V << 32) | r, V = round(v * 2^s) with
//                      v = len_k * cnt / C_col in FP32, r the row of the tile
//     presence blocks: u8 r
// An entry is a column with a non-zero count (its value may round to 0).
// Flagged rows appear in position order and a row's local index is the count
// of flagged positions of the tile before it in the window, so the pair kernel
// finds a branch's entries from the tile bitmap alone.

__device__ __forceinline__ uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// One warp per block: its size, and the rows / entries before each of its
// kChunks chunks of 32 positions, cpre[item][c] = (rows, entries), with the
// block's totals in cpre[item][kChunks].  VALUES: 8-byte entries, else 1 byte.
constexpr int kChunks = kRareWin / 32;

template <bool VALUES>
__global__ void k_rare_sizes(int32_t n_tiles, int32_t n_win, int32_t p0, int32_t K,
                             const uint32_t *__restrict__ bits, int32_t n_words,
                             const uint8_t *__restrict__ rc, int32_t k_pad,
                             uint32_t *__restrict__ bsize, uint2 *__restrict__ cpre) {
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (item >= (int64_t)n_tiles * n_win) return;
  const int64_t t = item / n_win;
  const int j = (int)(item % n_win);
  const int kb = p0 + kRareWin * j;
  uint32_t nrows = 0, nent = 0;
  for (int c = 0; c < kChunks; ++c) {
    const int k = kb + 32 * c + lane;
    const bool fl = k < K && ((bits[t * n_words + (k >> 5)] >> (k & 31)) & 1u);
    uint32_t e = fl ? rc[t * k_pad + k] : 0u;
    const uint32_t r = __popc(__ballot_sync(0xffffffffu, fl));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
    if (lane == 0) cpre[item * (kChunks + 1) + c] = make_uint2(nrows, nent);
    nrows += r;
    nent += e;
  }
  if (lane == 0) {
    cpre[item * (kChunks + 1) + kChunks] = make_uint2(nrows, nent);
    const uint32_t off_ent = align16(16u + 4u * (nrows + 1u));
    bsize[item] = align16(off_ent + (VALUES ? 8u : 1u) * nent);
  }
}

// Exclusive scan of the block sizes into byte offsets (one CTA of 1024 threads,
// contiguous chunks per thread); boff[n] receives the total.
__global__ void __launch_bounds__(1024) k_scan_sizes(int64_t n, const uint32_t *__restrict__ bsize,
                                                     unsigned long long *__restrict__ boff) {
  __shared__ unsigned long long part[1024];
  const int tid = threadIdx.x;
  const int64_t chunk = (n + 1023) / 1024;
  const int64_t lo = tid * chunk, hi = min(n, lo + chunk);
  unsigned long long sum = 0;
  for (int64_t i = lo; i < hi; ++i) sum += bsize[i];
  part[tid] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const unsigned long long v = tid >= off ? part[tid - off] : 0ull;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  unsigned long long run = part[tid] - sum;  // exclusive prefix of this chunk
  for (int64_t i = lo; i < hi; ++i) {
    boff[i] = run;
    run += bsize[i];
  }
  if (tid == 1023) boff[n] = part[1023];
}

// Fill: one warp per chunk of 32 positions of a block, at the offsets
// cpre gives; the chunk's flagged rows get their rowstart entries and their
// non-zero columns, compacted with four ballots (column 4l + w of lane l)
// over the counts cnt[perm[k]][col] (VALUES), or read as the row's presence
// mask, which holds those four ballots (presence).  VALUES: entries also carry
// round(v * scale) with v = len_k * (cnt * (1 / C_col)) in FP32, the same
// roundings as the dense packing; scale is a power of two.
template <bool VALUES>
__global__ void k_rare_fill(int32_t n_tiles, int32_t n_win, int32_t p0, int32_t K,
                            const uint32_t *__restrict__ bits, int32_t n_words,
                            const uint8_t *__restrict__ rc, int32_t k_pad,
                            const uint32_t *__restrict__ cnt,
                            const uint32_t *__restrict__ slot,
                            const uint4 *__restrict__ pmask,
                            const int32_t *__restrict__ perm,
                            const double *__restrict__ len_perm,
                            const double *__restrict__ inv_total, float scale,
                            const unsigned long long *__restrict__ boff,
                            const uint2 *__restrict__ cpre, uint8_t *__restrict__ blocks,
                            unsigned long long cap, unsigned long long *__restrict__ err) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t n_items = (int64_t)n_tiles * n_win;
  if (gw >= n_items * kChunks) return;
  // the host sizes the buffer from an upper bound; should the blocks ever
  // exceed it, nothing is written and the run reports the error
  if (boff[n_items] > cap) {
    if (gw == 0 && lane == 0 && err)
      atomicExch(err, (unsigned long long)(-UNIFRAC_E_BUFFER_TOO_SMALL));
    return;
  }
  const int64_t item = gw / kChunks;
  const int ch = (int)(gw % kChunks);
  const int64_t t = item / n_win;
  const int j = (int)(item % n_win);
  const int kc = p0 + kRareWin * j + 32 * ch;  // first position of the chunk
  const uint2 tot = cpre[item * (kChunks + 1) + kChunks];
  const uint2 pre = cpre[item * (kChunks + 1) + ch];
  const uint32_t nrows = tot.x, nent = tot.y;
  uint8_t *blk = blocks + boff[item];
  const uint32_t off_ent = align16(16u + 4u * (nrows + 1u));
  uint32_t *hdr = reinterpret_cast<uint32_t *>(blk);
  uint32_t *rowstart = hdr + 4;
  uint8_t *ri = blk + off_ent;                                                      // presence
  unsigned long long *ent = reinterpret_cast<unsigned long long *>(blk + off_ent);  // weighted
  if (ch == 0 && lane == 0) {
    hdr[0] = nrows;
    hdr[1] = nent;
    hdr[2] = off_ent;
    hdr[3] = 0u;
    rowstart[nrows] = nent;
  }
  const int k = kc + lane;
  const bool fl = k < K && ((bits[t * n_words + (k >> 5)] >> (k & 31)) & 1u);
  const uint32_t fb = __ballot_sync(0xffffffffu, fl);
  if (fb == 0u) return;
  const uint32_t c = fl ? rc[t * k_pad + k] : 0u;
  uint32_t incl = c;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t my_e = pre.y + incl - c;
  if (fl) rowstart[pre.x + __popc(fb & lt)] = my_e;
  float inv[4] = {0.f, 0.f, 0.f, 0.f};
  if constexpr (VALUES) {
#pragma unroll
    for (int q = 0; q < 4; ++q) inv[q] = (float)inv_total[t * TILE + 4 * lane + q];
  }
  // entries of each flagged row of the chunk, 8 rows in flight at a time
  uint32_t m = fb;
  while (m) {
    int src[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      src[g] = -1;
      if (m) {
        src[g] = __ffs(m) - 1;
        m &= m - 1;
      }
    }
    // VALUES: the counts (lane l: columns 4 l .. 4 l + 3); presence: the
    // row's mask alone (16 bytes, the same for every lane)
    uint4 cv[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      cv[g] = make_uint4(0u, 0u, 0u, 0u);
      if (src[g] >= 0) {
        if constexpr (VALUES) {
          const uint32_t *pc = count_tile(cnt, slot, perm[kc + src[g]], t, n_tiles);
          if (pc) cv[g] = *reinterpret_cast<const uint4 *>(pc + 4 * lane);
        } else
          cv[g] = pmask[(int64_t)perm[kc + src[g]] * n_tiles + t];
      }
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      if (src[g] < 0) break;
      const uint32_t base = __shfl_sync(0xffffffffu, my_e, src[g]);
      uint32_t cc[4] = {cv[g].x, cv[g].y, cv[g].z, cv[g].w};
      uint32_t B0, B1, B2, B3;
      if constexpr (VALUES) {
        B0 = __ballot_sync(0xffffffffu, cc[0] != 0u);
        B1 = __ballot_sync(0xffffffffu, cc[1] != 0u);
        B2 = __ballot_sync(0xffffffffu, cc[2] != 0u);
        B3 = __ballot_sync(0xffffffffu, cc[3] != 0u);
      } else {
        B0 = cc[0];
        B1 = cc[1];
        B2 = cc[2];
        B3 = cc[3];
#pragma unroll
        for (int w = 0; w < 4; ++w) cc[w] = (cc[w] >> lane) & 1u;
      }
      const uint32_t c0 = __popc(B0), c1 = __popc(B1), c2 = __popc(B2);
      const uint32_t pos[4] = {(uint32_t)__popc(B0 & lt), c0 + (uint32_t)__popc(B1 & lt),
                               c0 + c1 + (uint32_t)__popc(B2 & lt),
                               c0 + c1 + c2 + (uint32_t)__popc(B3 & lt)};
      float L = 0.f;
      if constexpr (VALUES) L = (float)len_perm[kc + src[g]];
#pragma unroll
      for (int w = 0; w < 4; ++w)
        if (cc[w] != 0u) {
          if constexpr (VALUES) {
            const float v = L * ((float)cc[w] * inv[w]);
            ent[base + pos[w]] = ((unsigned long long)__float2uint_rn(v * scale) << 32) |
                                 (unsigned long long)(4 * lane + w);
          } else {
            ri[base + pos[w]] = (uint8_t)(4 * lane + w);
          }
        }
    }
  }
}

// Packing of the rarely present positions [p0, K) for the sparse kernels.
// Block (column tile t, KR positions), warp w per bitmap word: lane l tests
// position 32 w + l, the ballot is the (t, word) bitmap word (p0 is a multiple
// of 32; words below it belong to the dense packing); then the flagged
// positions' presence masks (16 bytes each) are read four at a time for the
// row's count of non-zero columns rc and, when aq is given, aq[col] += q_k for
// every column where branch k is present.
__global__ void __launch_bounds__(256) k_pack_rare(
    int32_t K, int32_t p0, const int32_t *__restrict__ perm, const uint32_t *__restrict__ qperm,
    const uint4 *__restrict__ pmask, const uint8_t *__restrict__ flag,
    int32_t n_tiles, uint32_t *__restrict__ bits, int32_t n_words, uint8_t *__restrict__ rc,
    int32_t k_pad, unsigned long long *__restrict__ aq) {
  __shared__ unsigned long long red[kWarpsPerBlock][TILE];
  const int t = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kw = p0 + blockIdx.y * KR + w * WORD;  // first position of this warp's word
  const int k = kw + lane;
  const int32_t b = k < K ? perm[k] : 0;
  const bool fl = k < K && flag[(int64_t)b * n_tiles + t];
  const uint32_t word = __ballot_sync(0xffffffffu, fl);
  if (lane == 0 && kw / WORD < n_words) bits[(int64_t)t * n_words + kw / WORD] = word;
  unsigned long long acc[4] = {0ull, 0ull, 0ull, 0ull};
  uint32_t m = word;
  while (m) {
    constexpr int kU = 4;
    int src[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      src[u] = -1;
      if (m) {
        src[u] = __ffs(m) - 1;
        m &= m - 1;
      }
    }
    // the row's presence mask (16 bytes, the same for every lane) instead of
    // its 512 bytes of counts: bit lane of word w is column 4 lane + w
    uint4 c[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      c[u] = make_uint4(0u, 0u, 0u, 0u);
      if (src[u] >= 0) {
        const int32_t bu = __shfl_sync(0xffffffffu, b, src[u]);
        c[u] = pmask[(int64_t)bu * n_tiles + t];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (src[u] < 0) break;
      const int kk = kw + src[u];
      if (aq) {
        const unsigned long long q = qperm[kk];
        acc[0] += ((c[u].x >> lane) & 1u) ? q : 0ull;
        acc[1] += ((c[u].y >> lane) & 1u) ? q : 0ull;
        acc[2] += ((c[u].z >> lane) & 1u) ? q : 0ull;
        acc[3] += ((c[u].w >> lane) & 1u) ? q : 0ull;
      }
      const int nz = __popc(c[u].x) + __popc(c[u].y) + __popc(c[u].z) + __popc(c[u].w);
      if (lane == 0) rc[(int64_t)t * k_pad + kk] = (uint8_t)nz;
    }
  }
  if (!aq) return;  // block-uniform
#pragma unroll
  for (int q = 0; q < 4; ++q) red[w][lane * 4 + q] = acc[q];
  __syncthreads();
  if (threadIdx.x < TILE) {
    unsigned long long sum = 0;
    for (int ww = 0; ww < kWarpsPerBlock; ++ww) sum += red[ww][threadIdx.x];
    if (sum) atomicAdd(aq + (int64_t)t * TILE + threadIdx.x, sum);
  }
}

}  // namespace

int pack_rare(unifrac_ctx *ctx, const uint32_t *cnt, const uint8_t *flag, int32_t kf_words,
              uint32_t *bits, uint8_t *rc, unsigned long long *aq) {
  const int32_t p0 = kf_words * WORD;
  if (p0 >= ctx->K || ctx->n_tiles == 0) return UNIFRAC_OK;
  dim3 grid(ctx->n_tiles, (ctx->K - p0 + KR - 1) / KR);
  (void)cnt;  // the presence masks of the embedding stand in for the counts
  k_pack_rare<<<grid, 256, 0, ctx->stream>>>(ctx->K, p0, ctx->d_perm, ctx->d_qperm, ctx->d_pmask,
                                             flag, ctx->n_tiles, bits, ctx->K_pad / WORD, rc,
                                             ctx->K_pad, aq);
  ctx->stat_launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sparse packing");
  return UNIFRAC_OK;
}

int scan_sizes(unifrac_ctx *ctx, int64_t n, const uint32_t *sizes, unsigned long long *offs) {
  k_scan_sizes<<<1, 1024, 0, ctx->stream>>>(n, sizes, offs);
  ctx->stat_launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scan");
  return UNIFRAC_OK;
}

int build_rare_blocks(unifrac_ctx *ctx, bool values, const uint32_t *cnt, const uint32_t *bits,
                      const uint8_t *rc, int32_t kf_words, int32_t k_end, int32_t n_win,
                      uint32_t *bsize, unsigned long long *boff, uint2 *cpre, uint8_t *blocks) {
  cudaStream_t st = ctx->stream;
  const int64_t items = (int64_t)ctx->n_tiles * n_win;
  if (items <= 0) return UNIFRAC_OK;
  const int32_t n_words = ctx->K_pad / WORD;
  const int32_t p0 = kf_words * WORD;
  const unsigned grid = (unsigned)((items * 32 + 255) / 256);
  const unsigned grid_fill = (unsigned)((items * kChunks * 32 + 255) / 256);
  if (values) {
    k_rare_sizes<true><<<grid, 256, 0, st>>>(ctx->n_tiles, n_win, p0, k_end, bits, n_words, rc,
                                             ctx->K_pad, bsize, cpre);
    k_scan_sizes<<<1, 1024, 0, st>>>(items, bsize, boff);
    k_rare_fill<true><<<grid_fill, 256, 0, st>>>(
        ctx->n_tiles, n_win, p0, k_end, bits, n_words, rc, ctx->K_pad, cnt, ctx->d_slot,
        ctx->d_pmask, ctx->d_perm, ctx->d_len_perm, ctx->d_inv_total, ctx->sp_scale, boff, cpre,
        blocks,
        cur_bufs(ctx).blocks.bytes, cur_counters(ctx) + 1);
  } else {
    k_rare_sizes<false><<<grid, 256, 0, st>>>(ctx->n_tiles, n_win, p0, k_end, bits, n_words, rc,
                                              ctx->K_pad, bsize, cpre);
    k_scan_sizes<<<1, 1024, 0, st>>>(items, bsize, boff);
    k_rare_fill<false><<<grid_fill, 256, 0, st>>>(
        ctx->n_tiles, n_win, p0, k_end, bits, n_words, rc, ctx->K_pad, cnt, ctx->d_slot,
        ctx->d_pmask, ctx->d_perm, nullptr, nullptr, 1.f, boff, cpre, blocks,
        cur_bufs(ctx).blocks.bytes,
        cur_counters(ctx) + 1);
  }
  ctx->stat_launches += 3;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sparse blocks");
  return UNIFRAC_OK;
}

// ---------------------------------------------------------------------------
// Presence counts at create: bits[v][w] (u64, W words per node) has bit c of
// word w set when column 64 w + c has a non-zero count below node v.  Tips
// from their table rows, internal nodes as the OR of their children level by
// level (the embedding's level structure), then per node and study the
// popcount over the study's words, and per column the number of nodes it
// reaches.

namespace {

__global__ void k_pres_tips(int32_t n_frows, const int32_t *__restrict__ frow_tip,
                            const int64_t *__restrict__ frow_ptr,
                            const int32_t *__restrict__ fent_col, unsigned long long *bits,
                            int32_t W) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= n_frows) return;
  unsigned long long *row = bits + (int64_t)frow_tip[r] * W;
  for (int64_t e = frow_ptr[r] + lane; e < frow_ptr[r + 1]; e += 32) {
    const int32_t c = fent_col[e];
    atomicOr(row + (c >> 6), 1ull << (c & 63));
  }
}

__global__ void k_pres_level(const int32_t *__restrict__ nodes, int32_t n_level,
                             const int32_t *__restrict__ child_ptr,
                             const int32_t *__restrict__ child_idx, unsigned long long *bits,
                             int32_t W) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (int64_t)n_level * W) return;
  const int32_t node = nodes[x / W];
  const int32_t w = (int32_t)(x % W);
  unsigned long long s = 0ull;
  for (int32_t c = child_ptr[node]; c < child_ptr[node + 1]; ++c)
    s |= bits[(int64_t)child_idx[c] * W + w];
  bits[(int64_t)node * W + w] = s;
}

// Levels [L0, L1) in one launch: CTA b owns words [32 b, 32 b + 32) of every
// node and walks the levels in order, a barrier between levels (a level reads
// only what earlier levels wrote for the same words).  Plain loads: the data
// were written by this CTA.
__global__ void __launch_bounds__(1024) k_pres_levels_tail(
    const int32_t *__restrict__ nodes, const int32_t *__restrict__ level_ptr, int32_t L0,
    int32_t L1, const int32_t *__restrict__ child_ptr, const int32_t *__restrict__ child_idx,
    unsigned long long *bits, int32_t W) {
  const int32_t w0 = blockIdx.x * 32;
  for (int32_t L = L0; L < L1; ++L) {
    const int32_t lo = level_ptr[L], hi = level_ptr[L + 1];
    for (int64_t x = threadIdx.x; x < (int64_t)(hi - lo) * 32; x += blockDim.x) {
      const int32_t node = nodes[lo + (int32_t)(x >> 5)];
      const int32_t w = w0 + (int32_t)(x & 31);
      if (w >= W) continue;
      unsigned long long s = 0ull;
      for (int32_t c = child_ptr[node]; c < child_ptr[node + 1]; ++c)
        s |= bits[(int64_t)child_idx[c] * W + w];
      bits[(int64_t)node * W + w] = s;
    }
    __syncthreads();
  }
}

// acc[s][v] = samples of study s with a non-zero count below node v (one warp
// per node; sw[2 s], sw[2 s + 1]: the study's word range).
__global__ void k_pres_counts(const unsigned long long *__restrict__ bits, int32_t W,
                              int32_t n_count, int32_t n_studies, const int32_t *__restrict__ sw,
                              int32_t *__restrict__ acc, int32_t n_nodes) {
  const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (v >= n_count) return;
  const unsigned long long *row = bits + v * W;
  for (int32_t s = 0; s < n_studies; ++s) {
    int c = 0;
    for (int32_t w = sw[2 * s] + lane; w < sw[2 * s + 1]; w += 32) c += __popcll(row[w]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if (lane == 0) acc[(int64_t)s * n_nodes + v] = c;
  }
}

// reach[c] += nodes of [v0, v1) whose bitset has column c (blockIdx.y takes a
// slice of the nodes; a warp's 32 columns share one word).
__global__ void k_pres_reach(const unsigned long long *__restrict__ bits, int32_t W,
                             int32_t n_count, int32_t n_cols, int32_t *__restrict__ reach) {
  const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cols) return;
  const int32_t v0 = (int32_t)((int64_t)n_count * blockIdx.y / gridDim.y);
  const int32_t v1 = (int32_t)((int64_t)n_count * (blockIdx.y + 1) / gridDim.y);
  const int32_t w = c >> 6, b = c & 63;
  int32_t r = 0;
  for (int32_t v = v0; v < v1; ++v) r += (int32_t)((bits[(int64_t)v * W + w] >> b) & 1ull);
  if (r) atomicAdd(reach + c, r);
}

// Slot map of the compact counts: a (node, tile) has counts when its bitset
// has a sample in the tile's two 64-bit words.  One warp per node, 32 tiles
// at a time: k_slot_counts counts the node's tiles, and after a scan of those
// counts (the node's first slot), k_slot_fill numbers them in tile order.
__global__ void k_slot_counts(const unsigned long long *__restrict__ bits, int32_t W,
                              int32_t n_nodes, int32_t n_tiles, uint32_t *__restrict__ n_of) {
  const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (v >= n_nodes) return;
  const unsigned long long *row = bits + v * W;
  uint32_t c = 0;
  for (int32_t t0 = 0; t0 < n_tiles; t0 += 32) {
    const int32_t t = t0 + lane;
    const bool has = t < n_tiles && (row[2 * t] | row[2 * t + 1]) != 0ull;
    c += __popc(__ballot_sync(0xffffffffu, has));
  }
  if (lane == 0) n_of[v] = c;
}

__global__ void k_slot_fill(const unsigned long long *__restrict__ bits, int32_t W,
                            int32_t n_nodes, int32_t n_tiles,
                            const unsigned long long *__restrict__ first,
                            uint32_t *__restrict__ slot) {
  const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (v >= n_nodes) return;
  const unsigned long long *row = bits + v * W;
  unsigned long long next = first[v];
  for (int32_t t0 = 0; t0 < n_tiles; t0 += 32) {
    const int32_t t = t0 + lane;
    const bool has = t < n_tiles && (row[2 * t] | row[2 * t + 1]) != 0ull;
    const uint32_t m = __ballot_sync(0xffffffffu, has);
    if (t < n_tiles)
      slot[v * n_tiles + t] = has ? (uint32_t)(next + __popc(m & ((1u << lane) - 1u))) : kNoSlot;
    next += __popc(m);
  }
}

struct PresTemp {
  void *p[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  ~PresTemp() {
    for (void *q : p)
      if (q) cudaFree(q);
  }
};

}  // namespace

int presence_counts(unifrac_ctx *ctx, const std::vector<int32_t> &sw, bool count_reach,
                    std::vector<int32_t> &acc, int64_t *max_reach) {
  const int32_t n_nodes = ctx->n_nodes, root = n_nodes - 1, S = ctx->n_studies;
  const int32_t W = ctx->n_cols / 64;
  acc.assign((size_t)S * n_nodes, 0);
  // the slot map of the compact counts, [n_nodes][n_tiles]
  const int64_t cells = (int64_t)n_nodes * ctx->n_tiles;
  if (cells >= (int64_t)kNoSlot)
    return fail(ctx, UNIFRAC_E_UNSUPPORTED, "nodes x column tiles must stay below 2^32 - 1");
  {
    const cudaError_t ea = dev_alloc(reinterpret_cast<void **>(&ctx->d_slot),
                                     (size_t)std::max<int64_t>(cells, 4) * 4);
    if (ea != cudaSuccess) return cuda_fail(ctx, ea, "device allocation (count slots)");
    ctx->device_bytes += (size_t)std::max<int64_t>(cells, 4) * 4;
    ctx->n_slots = 0;
  }
  if (W == 0) return UNIFRAC_OK;
  cudaStream_t st = ctx->stream;
  PresTemp tmp;
  unsigned long long *bits;
  int32_t *d_sw, *d_acc, *d_reach;
  if (dev_malloc_retry(&tmp.p[0], (size_t)n_nodes * W * 8) != cudaSuccess ||
      dev_malloc_retry(&tmp.p[1], sw.size() * 4) != cudaSuccess ||
      dev_malloc_retry(&tmp.p[2], acc.size() * 4) != cudaSuccess ||
      dev_malloc_retry(&tmp.p[3], (size_t)ctx->n_cols * 4) != cudaSuccess ||
      dev_malloc_retry(&tmp.p[4], (size_t)n_nodes * 4) != cudaSuccess ||
      dev_malloc_retry(&tmp.p[5], ((size_t)n_nodes + 1) * 8) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, UNIFRAC_E_OOM, "presence bitsets");
  }
  bits = static_cast<unsigned long long *>(tmp.p[0]);
  d_sw = static_cast<int32_t *>(tmp.p[1]);
  d_acc = static_cast<int32_t *>(tmp.p[2]);
  d_reach = static_cast<int32_t *>(tmp.p[3]);
  cudaError_t e = cudaMemsetAsync(bits, 0, (size_t)n_nodes * W * 8, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_sw, sw.data(), sw.size() * 4, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "presence set-up");
  if (ctx->n_frows > 0)
    k_pres_tips<<<(unsigned)(((int64_t)ctx->n_frows * 32 + 255) / 256), 256, 0, st>>>(
        ctx->n_frows, ctx->d_frow_tip, ctx->d_frow_ptr, ctx->d_fent_col, bits, W);
  constexpr int32_t kTailNodes = 256;
  int32_t L0 = 0;
  while (L0 < ctx->n_levels && ctx->level_ptr[L0 + 1] - ctx->level_ptr[L0] > kTailNodes) ++L0;
  for (int L = 0; L < L0; ++L) {
    const int32_t lo = ctx->level_ptr[L], hi = ctx->level_ptr[L + 1];
    const int64_t items = (int64_t)(hi - lo) * W;
    if (items == 0) continue;
    k_pres_level<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(
        ctx->d_level_nodes + lo, hi - lo, ctx->d_child_ptr, ctx->d_child_idx, bits, W);
  }
  if (L0 < ctx->n_levels)
    k_pres_levels_tail<<<(unsigned)((W + 31) / 32), 1024, 0, st>>>(
        ctx->d_level_nodes, ctx->d_level_ptr, L0, ctx->n_levels, ctx->d_child_ptr,
        ctx->d_child_idx, bits, W);
  {
    uint32_t *n_of = static_cast<uint32_t *>(tmp.p[4]);
    unsigned long long *first = static_cast<unsigned long long *>(tmp.p[5]);
    const unsigned g = (unsigned)(((int64_t)n_nodes * 32 + 255) / 256);
    k_slot_counts<<<g, 256, 0, st>>>(bits, W, n_nodes, ctx->n_tiles, n_of);
    k_scan_sizes<<<1, 1024, 0, st>>>(n_nodes, n_of, first);
    k_slot_fill<<<g, 256, 0, st>>>(bits, W, n_nodes, ctx->n_tiles, first, ctx->d_slot);
  }
  if (root > 0)
    k_pres_counts<<<(unsigned)(((int64_t)root * 32 + 255) / 256), 256, 0, st>>>(
        bits, W, root, S, d_sw, d_acc, n_nodes);
  std::vector<int32_t> reach;
  if (count_reach && root > 0) {
    reach.assign(ctx->n_cols, 0);
    e = cudaMemsetAsync(d_reach, 0, (size_t)ctx->n_cols * 4, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "presence reach");
    const unsigned slices = (unsigned)std::max<int64_t>(1, std::min<int64_t>(64, root / 4096 + 1));
    k_pres_reach<<<dim3((unsigned)((ctx->n_cols + 255) / 256), slices), 256, 0, st>>>(
        bits, W, root, ctx->n_cols, d_reach);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(acc.data(), d_acc, acc.size() * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && count_reach && root > 0)
    e = cudaMemcpyAsync(reach.data(), d_reach, reach.size() * 4, cudaMemcpyDeviceToHost, st);
  unsigned long long n_slots = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&n_slots, static_cast<unsigned long long *>(tmp.p[5]) + n_nodes, 8,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "presence kernels");
  ctx->n_slots = (int64_t)n_slots;
  if (count_reach && root > 0)
    for (int32_t c = 0; c < ctx->n_cols; ++c) *max_reach = std::max<int64_t>(*max_reach, reach[c]);
  return UNIFRAC_OK;
}

int embed_counts(unifrac_ctx *ctx, uint32_t *cnt, uint8_t *flag) {
  cudaStream_t st = ctx->stream;
  const uint32_t *slot = ctx->d_slot;
  cudaError_t e = cudaMemsetAsync(flag, 0, (size_t)ctx->n_nodes * ctx->n_tiles, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "memset flags");
  ctx->stat_launches += 1;
  if (ctx->n_tchunks > 0 && ctx->n_tiles > 0) {
    const int64_t blocks = (ctx->n_tchunks * 32 + 255) / 256;
    k_tip_zero<<<(unsigned)blocks, 256, 0, st>>>(ctx->n_tchunks, ctx->d_tchunk_row,
                                                 ctx->d_tchunk_lo, ctx->tip_chunk, ctx->d_frow_tip,
                                                 ctx->d_frow_ptr, ctx->d_fent_col, cnt, slot,
                                                 flag, ctx->d_pmask, ctx->n_tiles);
    k_tip_scatter<<<(unsigned)blocks, 256, 0, st>>>(ctx->n_tchunks, ctx->d_tchunk_row,
                                                    ctx->d_tchunk_lo, ctx->tip_chunk,
                                                    ctx->d_frow_tip, ctx->d_frow_ptr,
                                                    ctx->d_fent_col, ctx->d_fent_cnt, cnt, slot,
                                                    reinterpret_cast<uint32_t *>(ctx->d_pmask),
                                                    ctx->n_tiles);
    ctx->stat_launches += 2;
  }
  // one launch per level while the levels are large, then the rest in one
  // launch (levels from the first with at most kTailNodes nodes)
  constexpr int32_t kTailNodes = 256;
  int32_t L0 = 0;
  while (L0 < ctx->n_levels && ctx->level_ptr[L0 + 1] - ctx->level_ptr[L0] > kTailNodes) ++L0;
  for (int L = 0; L < L0 && ctx->n_tiles > 0; ++L) {
    const int32_t lo = ctx->level_ptr[L], hi = ctx->level_ptr[L + 1];
    const int64_t items = (int64_t)(hi - lo) * ((ctx->n_tiles + 31) / 32);
    if (items == 0) continue;
    const int64_t blocks = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    k_level<<<(unsigned)blocks, 32 * kWarpsPerBlock, 0, st>>>(
        ctx->d_level_nodes + lo, hi - lo, ctx->d_child_ptr, ctx->d_child_idx, cnt, slot, flag,
        ctx->d_pmask, ctx->n_tiles);
    ctx->stat_launches += 1;
  }
  if (L0 < ctx->n_levels && ctx->n_tiles > 0) {
    k_levels_tail<<<(unsigned)ctx->n_tiles * 4, kTailThreads, 0, st>>>(
        ctx->d_level_nodes, ctx->d_level_ptr, L0, ctx->n_levels, ctx->d_child_ptr,
        ctx->d_child_idx, cnt, slot, flag, reinterpret_cast<uint8_t *>(ctx->d_pmask),
        ctx->n_tiles);
    ctx->stat_launches += 1;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "embedding kernels");
  return UNIFRAC_OK;
}

int pack_weighted(unifrac_ctx *ctx, const uint32_t *cnt, const uint8_t *flag, bool f64,
                  void *vals, uint32_t *bits, int32_t k_end) {
  cudaStream_t st = ctx->stream;
  const int32_t n_words = ctx->K_pad / WORD;
  k_end = min(k_end, ctx->K);
  if (k_end > 0 && ctx->n_tiles > 0) {
    dim3 grid(ctx->n_tiles, (k_end + KR - 1) / KR);
    if (f64)
      k_pack_weighted<double><<<grid, 256, 0, st>>>(
          ctx->K, k_end, ctx->d_perm, ctx->d_len_perm, cnt, flag, ctx->d_slot, ctx->n_tiles,
          ctx->d_inv_total, static_cast<double *>(vals), ctx->n_cols, bits, n_words);
    else
      k_pack_weighted<float><<<grid, 256, 0, st>>>(
          ctx->K, k_end, ctx->d_perm, ctx->d_len_perm, cnt, flag, ctx->d_slot, ctx->n_tiles,
          ctx->d_inv_total, static_cast<float *>(vals), ctx->n_cols, bits, n_words);
    ctx->stat_launches += 1;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "weighted packing");
  return UNIFRAC_OK;
}

int pack_lookup(unifrac_ctx *ctx, const uint32_t *cnt, const uint8_t *flag, uint8_t *bytes,
                double *tables, uint32_t *gbits, double *a) {
  (void)cnt;  // the embedding's presence masks stand in for the counts
  cudaStream_t st = ctx->stream;
  const int32_t G = ctx->K_pad / 8;
  const int32_t g_words = (G + WORD - 1) / WORD;
  const int32_t n_gblocks = (G + GR - 1) / GR;
  double *partial = static_cast<double *>(cur_bufs(ctx).partial.p);
  if (G > 0 && ctx->n_tiles > 0) {
    k_lookup_tables<<<G, 256, 0, st>>>(ctx->K, ctx->d_len_perm, tables);
    dim3 grid(ctx->n_tiles, n_gblocks);
    k_pack_lookup<<<grid, 128, 0, st>>>(ctx->K, G, ctx->d_perm, ctx->d_len_perm, ctx->d_pmask,
                                        flag, ctx->n_cols, ctx->n_tiles, bytes, gbits, g_words,
                                        partial);
    ctx->stat_launches += 2;
  }
  if (ctx->n_cols > 0) {
    k_reduce_partials<<<(ctx->n_cols + 255) / 256, 256, 0, st>>>(
        ctx->n_cols, G > 0 && ctx->n_tiles > 0 ? n_gblocks : 0, partial, a);
    ctx->stat_launches += 1;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lookup packing");
  return UNIFRAC_OK;
}

}  // namespace ufb
