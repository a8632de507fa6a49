// K3: unweighted UniFrac as a dense contraction on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators, TMA-staged operands).
//
// Section II of the paper: unweighted UniFrac over all pairs of samples, with
// GPU offload and fp32 compute.  With the 0/1 presence matrix X [samples x
// branches], branch lengths len and a_i = sum_b len_b X_ib:
//   G = X diag(len) X^T,   d_ij = (a_i + a_j - 2 G_ij) / (a_i + a_j - G_ij).
// Exactness: every kept length is written as a 24-bit fixed-point number
// q_b = round(len_b / sigma * 2^24) (sigma the power of two above the longest
// branch) and split into three base-256 digits q_b = 65536 d1 + 256 d2 + d3.
// Digits and 0/1 presences are exact in BF16, so each plane's Gram
// G_p = X diag(d_p) X^T is a sum of integers below 2^24 (as long as a sample
// reaches fewer than 65,793 branches) and is exact in the FP32 TMEM
// accumulator whatever its rounding.  The epilogue combines the planes in
// 64-bit integers, G = 65536 G_1 + 256 G_2 + G_3 in units of sigma 2^-24, and
// a_i uses the same q_b, so both sums of the ratio are exact; only the final
// quotient is rounded (FP32, the output precision).  The error is the 2^-25
// sigma quantisation of each length plus that last rounding.
//
// CTA = one 128 x 128 tile of sample pairs.  Warp 0 issues TMA loads (128B
// swizzle) of a 64-branch K-tile of X for the row tile and of the three digit
// planes D_p = X diag(d_p) for the column tile into a 3-stage ring; warp 1
// issues tcgen05.mma (M=128, N=128, K=16, BF16 -> FP32) into three TMEM
// accumulators of 128 columns; warps 2-5 read TMEM back (tcgen05.ld) and write
// the distances.  K-tiles where the row tile or the column tile has no
// presence at all are skipped (AND of the two tiles' K-tile bitmaps).  Only the
// frequently present branches (positions below k_tc) go through the tensor
// cores when a sparse split is set; the integer sums of the rest come from the
// sparse kernel (spart) and are added before scaling, still exactly.  Every
// wait on an mbarrier is bounded (1 s); a timeout records UNIFRAC_E_DEVICE_TIMEOUT,
// drains outstanding copies, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "epilogue.cuh"

namespace ufb {

namespace {

constexpr int TC_BM = 128;    // rows of a tile (UMMA M)
constexpr int TC_BN = 128;    // columns of a tile (UMMA N)
constexpr int TC_BK = 64;     // branches per K-tile (128 bytes of BF16: one swizzle row)
constexpr int TC_PLANES = 3;  // base-256 digits of the 24-bit lengths
constexpr int TC_STAGES = 3;
constexpr int TC_THREADS = 192;
constexpr uint32_t A_BYTES = TC_BM * TC_BK * 2;
constexpr uint32_t B_BYTES = TC_BN * TC_BK * 2;
constexpr uint32_t STAGE_BYTES = A_BYTES + TC_PLANES * B_BYTES;
constexpr uint32_t TMEM_COLS = 512;  // 3 x 128 used
constexpr uint64_t WAIT_NS = 1000000000ull;

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                           ((uint32_t)(TC_BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);

struct TcShared {
  uint8_t stage[TC_STAGES][STAGE_BYTES];  // A | B0 | B1 | B2, each 1024-aligned
  uint64_t full[TC_STAGES];
  uint64_t empty[TC_STAGES];
  uint64_t done;           // MMA -> epilogue: an item's accumulators are complete
  uint64_t tmem_free;      // epilogue -> MMA: the accumulators have been read back
  uint64_t item_full[2];   // producer -> MMA, epilogue: a work item is in the ring slot
  uint64_t item_empty[2];  // MMA + epilogue warps -> producer: the slot has been read
  int32_t item_ring[2];
  uint32_t tmem_base;
  int32_t abort;
  int32_t issued;
  int32_t consumed;
};
constexpr size_t TC_SMEM = sizeof(TcShared) + 1024;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase.  Returns false if the CTA is aborting or
// the wait exceeded limit_ns of %globaltimer (or, as a backstop, kWaitPolls
// polls): then it records the timeout and raises the abort.
constexpr uint64_t kWaitPolls = 1ull << 26;

__device__ bool mbar_wait_limit(uint64_t *bar, uint32_t parity, volatile int32_t *abort,
                                unsigned long long *err, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint64_t polls = 0;; ++polls) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (global_ns() - t0 > limit_ns || polls >= kWaitPolls) {
      *abort = 1;
      if (err) atomicExch(err, (unsigned long long)(-UNIFRAC_E_DEVICE_TIMEOUT));
      return false;
    }
  }
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int32_t *abort,
                                          unsigned long long *err) {
  return mbar_wait_limit(bar, parity, abort, err, WAIT_NS);
}

// The bounded wait run out on purpose: thread 0 waits on an mbarrier that
// nothing arrives at, with a short limit, and stores the status it recorded.
__global__ void k_wait_check(uint64_t limit_ns, unsigned long long *err) {
  __shared__ uint64_t bar;
  __shared__ int32_t abort;
  if (threadIdx.x == 0) {
    abort = 0;
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_wait_limit(&bar, 0, &abort, err, limit_ns);
  }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor for a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart (SBO),
// descriptor version 1, layout SWIZZLE_128B.  The leading offset is unused for
// swizzled K-major tiles.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Work items: with a device queue the grid is persistent (one CTA per SM)
// and each CTA pulls tile pairs until the queue runs dry; without one, the
// CTA takes item blockIdx.x only.  Warp 0 (producer) fetches each item into a
// two-slot ring in shared memory and streams its K-tiles through the stage
// ring, running ahead into the next item while the epilogue of the current
// one runs; warp 1 (MMA) waits for the epilogue to release the accumulators
// (tmem_free) before the first MMA of the next item.  The stage ring's
// sequence number runs on across items, so its phases stay consistent.
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_pairs_tc(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_d,
               const WorkItem *__restrict__ items, int32_t n_items, unsigned int *__restrict__ queue,
               const uint32_t *__restrict__ kbits, int32_t k_words, int32_t n_cols,
               const unsigned long long *__restrict__ aq,
               const unsigned long long *__restrict__ spart, OutSpec o,
               unsigned long long *__restrict__ counter) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  TcShared &sh = *reinterpret_cast<TcShared *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long *err = counter ? counter + 1 : nullptr;
  constexpr int kEpiWarps = TC_THREADS / 32 - 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    mbar_init(&sh.done, 1);
    mbar_init(&sh.tmem_free, kEpiWarps);
    for (int r = 0; r < 2; ++r) {
      mbar_init(&sh.item_full[r], 1);
      mbar_init(&sh.item_empty[r], 1 + kEpiWarps);
    }
    sh.abort = 0;
    sh.issued = 0;
    sh.consumed = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh.tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem_base;
  volatile int32_t *abort = &sh.abort;
  auto selected = [&](const WorkItem &it) {
    const uint32_t *bI = kbits + (int64_t)it.tile_i * k_words;
    const uint32_t *bJ = kbits + (int64_t)it.tile_j * k_words;
    int n = 0;
    for (int w = 0; w < k_words; ++w) n += __popc(bI[w] & bJ[w]);
    return n;
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int i = 0;  // stage-ring sequence number, across items
      for (int t = 0;; ++t) {
        const int slot = t & 1;
        if (t >= 2 && !mbar_wait(&sh.item_empty[slot], ((t >> 1) - 1) & 1, abort, err)) break;
        int32_t item = n_items;
        if (!*abort)
          item = queue ? (int32_t)atomicAdd(queue, 1u) : (t == 0 ? (int32_t)blockIdx.x : n_items);
        sh.item_ring[slot] = item;
        mbar_arrive(&sh.item_full[slot]);
        if (item >= n_items) break;
        const WorkItem it = items[item];
        const uint32_t *bI = kbits + (int64_t)it.tile_i * k_words;
        const uint32_t *bJ = kbits + (int64_t)it.tile_j * k_words;
        bool go = true;
        for (int w = 0; w < k_words && go; ++w) {
          uint32_t m = bI[w] & bJ[w];
          while (m && go) {
            const int kt = w * 32 + __ffs(m) - 1;
            m &= m - 1;
            const int s = i % TC_STAGES;
            if (i >= TC_STAGES &&
                !mbar_wait(&sh.empty[s], ((i / TC_STAGES) - 1) & 1, abort, err)) {
              go = false;
              break;
            }
            mbar_arrive_expect_tx(&sh.full[s], STAGE_BYTES);
            uint8_t *st = sh.stage[s];
            tma_load_2d(st, &map_x, kt * TC_BK, it.tile_i * TC_BM, &sh.full[s]);
#pragma unroll
            for (int p = 0; p < TC_PLANES; ++p)
              tma_load_2d(st + A_BYTES + p * B_BYTES, &map_d, kt * TC_BK,
                          p * n_cols + it.tile_j * TC_BN, &sh.full[s]);
            ++i;
            sh.issued = i;
          }
        }
        if (!go) break;
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int i = 0;         // stage-ring sequence number, across items
      int tc_items = 0;  // items with selected K-tiles so far
      for (int t = 0;; ++t) {
        const int slot = t & 1;
        if (!mbar_wait(&sh.item_full[slot], (t >> 1) & 1, abort, err)) break;
        const int32_t item = sh.item_ring[slot];
        mbar_arrive(&sh.item_empty[slot]);
        if (item >= n_items) break;
        const WorkItem it = items[item];
        const uint32_t *bI = kbits + (int64_t)it.tile_i * k_words;
        const uint32_t *bJ = kbits + (int64_t)it.tile_j * k_words;
        if (selected(it) == 0) continue;
        // the accumulators are free once the epilogue has read the last item's
        if (tc_items > 0 && !mbar_wait(&sh.tmem_free, (tc_items - 1) & 1, abort, err)) break;
        tc_fence_after();
        bool go = true;
        int first = 1;
        for (int w = 0; w < k_words && go; ++w) {
          uint32_t m = bI[w] & bJ[w];
          while (m && go) {
            m &= m - 1;
            const int s = i % TC_STAGES;
            if (!mbar_wait(&sh.full[s], (i / TC_STAGES) & 1, abort, err)) {
              go = false;
              break;
            }
            tc_fence_after();
            const uint32_t base = smem_u32(sh.stage[s]);
            const uint64_t da = sdesc_sw128(base);
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
#pragma unroll
              for (int p = 0; p < TC_PLANES; ++p) {
                const uint64_t db = sdesc_sw128(base + A_BYTES + p * B_BYTES);
                // +2 = 32 bytes (16 BF16) along K inside the swizzled row
                mma_bf16(tmem + p * TC_BN, da + 2 * kk, db + 2 * kk,
                         (first && kk == 0) ? 0u : 1u);
              }
            }
            first = 0;
            mma_commit(&sh.empty[s]);
            ++i;
            sh.consumed = i;
          }
        }
        if (!go) break;
        mma_commit(&sh.done);  // arrives when every MMA issued above has completed
        ++tc_items;
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lanes 32q .. 32q+31 are this warp's rows
    const int row = q * 32 + lane;
    int tc_items = 0;
    unsigned long long nsel = 0;
    for (int t = 0;; ++t) {
      const int slot = t & 1;
      const bool got = __all_sync(0xffffffffu,
                                  mbar_wait(&sh.item_full[slot], (t >> 1) & 1, abort, err));
      if (!got) break;
      const int32_t item = sh.item_ring[slot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.item_empty[slot]);
      if (item >= n_items) break;
      const WorkItem it = items[item];
      const int n_sel = selected(it);
      nsel += (unsigned long long)n_sel;
      bool ok = true;
      if (n_sel > 0) {
        ok = __all_sync(0xffffffffu, mbar_wait(&sh.done, tc_items & 1, abort, err));
        tc_fence_after();
        if (!ok) break;
      }
      const StudyDev sd = o.studies[it.study];
      const int64_t colI = (int64_t)it.tile_i * TC_BM, colJ = (int64_t)it.tile_j * TC_BN;
      const int li = (int)(colI + row) - sd.col0;
      const unsigned long long ai = aq[colI + row];
      for (int c = 0; c < TC_BN / 32; ++c) {
        uint32_t r0[32], r1[32], r2[32];
        if (n_sel > 0) {
          const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 32);
          tmem_ld32(tq, r0);
          tmem_ld32(tq + TC_BN, r1);
          tmem_ld32(tq + 2 * TC_BN, r2);
          tmem_ld_wait();
          if (c == TC_BN / 32 - 1) {
            // every accumulator column of this warp's rows is in registers:
            // the next item's MMAs may overwrite them
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.tmem_free);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) r0[j] = r1[j] = r2[j] = 0u;
        }
        if (li >= sd.n) continue;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = c * 32 + j;
          const int lj = (int)(colJ + col) - sd.col0;
          if (lj >= sd.n) continue;
          if (li < lj) {
            // all sums in units of the 24-bit lengths, exact 64-bit integers:
            // G = 65536 G1 + 256 G2 + G3 (+ sparse part), A = a_i + a_j
            unsigned long long g =
                ((unsigned long long)__float2uint_rn(__uint_as_float(r0[j])) << 16) +
                ((unsigned long long)__float2uint_rn(__uint_as_float(r1[j])) << 8) +
                (unsigned long long)__float2uint_rn(__uint_as_float(r2[j]));
            if (spart) g += spart[(int64_t)item * TC_BM * TC_BN + row * TC_BN + col];
            const unsigned long long A = ai + aq[colJ + col];
            const float d = ratio01_f32((float)(A - 2 * g), (float)(A - g));
            put_pair(o, sd, li, lj, d);
          } else if (li == lj) {
            put_diag(o, sd, li);
          }
        }
      }
      if (n_sel > 0) ++tc_items;
    }
    if (warp == 2 && lane == 0 && counter) atomicAdd(counter, nsel);
  }

  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort) {
    // drain TMA copies that were issued but never consumed (bounded)
    for (int i = sh.consumed; i < sh.issued; ++i) {
      const int s = i % TC_STAGES;
      const uint64_t t0 = global_ns();
      while (!mbar_try_wait(&sh.full[s], (i / TC_STAGES) & 1) && global_ns() - t0 < WAIT_NS) {
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// Packing for the tensor-core path.  Block (column tile t, 4 K-tiles) of 256
// threads: reads the presence masks of 64 branch rows x 128 columns per K-tile
// (16 bytes per row; word w, bit l is column 4 l + w), transposes through
// shared memory and writes sample-major BF16 rows of X (0/1) and of the
// three digit planes; K-tiles with no presence in the tile are not written
// (the pair kernel never reads them) and get a 0 bit in the K-tile bitmap.
// aq[col] += sum_k q_k p[k][col] (exact integers).
constexpr int PK_KT = 4;

__global__ void __launch_bounds__(256)
    k_pack_tc(int32_t K, int32_t K_pad, int32_t dig_ld, const int32_t *__restrict__ perm,
              const uint8_t *__restrict__ digits, const uint4 *__restrict__ pmask,
              const uint8_t *__restrict__ flag, int32_t n_cols, int32_t n_tiles,
              uint16_t *__restrict__ X, uint16_t *__restrict__ D, uint32_t *__restrict__ kbits,
              int32_t k_words, unsigned long long *__restrict__ aq) {
  __shared__ uint8_t pres[TC_BK][TILE + 16];
  __shared__ uint16_t dg[TC_PLANES][TC_BK];
  __shared__ uint32_t qv[TC_BK];
  __shared__ int any;
  const int t = blockIdx.x;
  const int tid = threadIdx.x;
  unsigned long long my_aq[4] = {0ull, 0ull, 0ull, 0ull};
  const int64_t plane = (int64_t)n_cols * K_pad;
  for (int g = 0; g < PK_KT; ++g) {
    const int kt = blockIdx.y * PK_KT + g;
    if (kt * TC_BK >= K_pad) break;
    if (tid == 0) any = 0;
    if (tid < TC_BK) {
      const int k = kt * TC_BK + tid;
      uint32_t q = 0;
#pragma unroll
      for (int p = 0; p < TC_PLANES; ++p) {
        const uint32_t dv = digits[(int64_t)p * dig_ld + k];
        dg[p][tid] = __bfloat16_as_ushort(__float2bfloat16_rn((float)dv));
        q = (q << 8) | dv;
      }
      qv[tid] = q;
    }
    __syncthreads();
    {
      const int r = tid >> 2, c0 = (tid & 3) * 32;
      const int k = kt * TC_BK + r;
      const int32_t b = (k < K) ? perm[k] : -1;
      const bool valid = b >= 0 && flag[(int64_t)b * n_tiles + t];
      uint4 pm = make_uint4(0u, 0u, 0u, 0u);
      if (valid) pm = pmask[(int64_t)b * n_tiles + t];
#pragma unroll
      for (int q = 0; q < 32; q += 4) {
        const int l = (c0 + q) >> 2;
        pres[r][c0 + q + 0] = (pm.x >> l) & 1u;
        pres[r][c0 + q + 1] = (pm.y >> l) & 1u;
        pres[r][c0 + q + 2] = (pm.z >> l) & 1u;
        pres[r][c0 + q + 3] = (pm.w >> l) & 1u;
      }
      if (pm.x | pm.y | pm.z | pm.w) any = 1;
    }
    __syncthreads();
    if (any) {
#pragma unroll
      for (int e4 = 0; e4 < 4; ++e4) {
        const int e = tid + 256 * e4;
        const int c = e >> 3, ch = e & 7;
        uint32_t xw[4], dw[TC_PLANES][4];
        unsigned long long qs = 0;
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) {
          uint32_t xx = 0, dd[TC_PLANES] = {0u, 0u, 0u};
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int kk = ch * 8 + j2 * 2 + h;
            if (pres[kk][c]) {
              xx |= 0x3F80u << (16 * h);
#pragma unroll
              for (int p = 0; p < TC_PLANES; ++p) dd[p] |= (uint32_t)dg[p][kk] << (16 * h);
              qs += qv[kk];
            }
          }
          xw[j2] = xx;
#pragma unroll
          for (int p = 0; p < TC_PLANES; ++p) dw[p][j2] = dd[p];
        }
        const int64_t off = ((int64_t)t * TILE + c) * K_pad + (int64_t)kt * TC_BK + ch * 8;
        *reinterpret_cast<uint4 *>(X + off) = make_uint4(xw[0], xw[1], xw[2], xw[3]);
#pragma unroll
        for (int p = 0; p < TC_PLANES; ++p)
          *reinterpret_cast<uint4 *>(D + p * plane + off) =
              make_uint4(dw[p][0], dw[p][1], dw[p][2], dw[p][3]);
        my_aq[e4] += qs;
      }
      if (tid == 0) atomicOr(kbits + (int64_t)t * k_words + kt / 32, 1u << (kt % 32));
    }
    __syncthreads();
  }
  // columns (tid >> 3) + 32 e4: reduce over the 8 threads (ch) sharing a column
#pragma unroll
  for (int e4 = 0; e4 < 4; ++e4) {
    unsigned long long v = my_aq[e4];
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    if ((tid & 7) == 0 && v) atomicAdd(aq + (int64_t)t * TILE + (tid >> 3) + 32 * e4, v);
  }
}

__global__ void k_aq_to_a(int32_t n_cols, const unsigned long long *__restrict__ aq, double scale,
                          double *__restrict__ a) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_cols) a[c] = (double)aq[c] * scale;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D BF16 tensor map: rows of `inner` elements, box 64 x 128, 128B swizzle.
bool make_map(CUtensorMap *m, void *base, uint64_t inner, uint64_t rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {TC_BK, TC_BM};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int pack_tc(unifrac_ctx *ctx, const uint32_t *cnt, const uint8_t *flag, int32_t k_tc,
            uint16_t *X, uint16_t *D, uint32_t *kbits, unsigned long long *aq) {
  cudaStream_t st = ctx->stream;
  const int32_t n_kt = k_tc / TC_BK;
  const int32_t k_words = (n_kt + 31) / 32;
  cudaError_t e = cudaMemsetAsync(kbits, 0, (size_t)ctx->n_tiles * k_words * 4, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "clear tensor-core packing");
  ctx->stat_launches += 1;
  if (ctx->n_tiles > 0 && n_kt > 0) {
    dim3 grid(ctx->n_tiles, (n_kt + PK_KT - 1) / PK_KT);
    (void)cnt;  // the embedding's presence masks stand in for the counts
    k_pack_tc<<<grid, 256, 0, st>>>(ctx->K, k_tc, ctx->K_pad, ctx->d_perm, ctx->d_digits,
                                    ctx->d_pmask, flag, ctx->n_cols, ctx->n_tiles, X, D, kbits,
                                    k_words, aq);
    ctx->stat_launches += 1;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-core packing");
  return UNIFRAC_OK;
}

int finish_tc_a(unifrac_ctx *ctx, const unsigned long long *aq, double *a) {
  if (ctx->n_cols <= 0) return UNIFRAC_OK;
  k_aq_to_a<<<(ctx->n_cols + 255) / 256, 256, 0, ctx->stream>>>(ctx->n_cols, aq, ctx->tc_scale, a);
  ctx->stat_launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-core per-sample sums");
  return UNIFRAC_OK;
}

size_t tc_smem_bytes() { return TC_SMEM; }

int pairs_tc(unifrac_ctx *ctx, int32_t k_tc, const uint16_t *X, const uint16_t *D,
             const uint32_t *kbits, const unsigned long long *aq,
             const unsigned long long *spart, const WorkItem *items, int32_t n_items,
             const OutSpec &o) {
  if (n_items <= 0) return UNIFRAC_OK;
  if (k_tc < TC_BK || k_tc % TC_BK) return fail(ctx, UNIFRAC_E_INVALID_ARG, "tensor-core K split");
  const int32_t n_kt = k_tc / TC_BK;
  const int32_t k_words = (n_kt + 31) / 32;
  CUtensorMap mx, md;
  if (!make_map(&mx, const_cast<uint16_t *>(X), k_tc, ctx->n_cols) ||
      !make_map(&md, const_cast<uint16_t *>(D), k_tc, (uint64_t)TC_PLANES * ctx->n_cols))
    return fail(ctx, UNIFRAC_E_CUDA, "cuTensorMapEncodeTiled failed");
  cudaError_t e =
      cudaFuncSetAttribute(k_pairs_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-core kernel attribute");
  unsigned int *q = cur_queue(ctx, 0);
  k_pairs_tc<<<pair_grid(ctx, k_pairs_tc, TC_THREADS, TC_SMEM, n_items), TC_THREADS, TC_SMEM,
               ctx->stream>>>(mx, md, items, n_items, q, kbits, k_words, ctx->n_cols, aq, spart,
                              o, cur_counters(ctx));
  ctx->stat_launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-core pair kernel");
  return UNIFRAC_OK;
}

}  // namespace ufb

extern "C" int unifrac_check_bounded_wait(uint32_t limit_us, int32_t *status, void *cuda_stream) {
  if (!status || limit_us == 0 || limit_us > 1000000u) return UNIFRAC_E_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned long long *d_err = nullptr;
  if (cudaMalloc(&d_err, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return UNIFRAC_E_OOM;
  }
  unsigned long long h = 0;
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(h), st);
  if (e == cudaSuccess) {
    ufb::k_wait_check<<<1, 32, 0, st>>>((uint64_t)limit_us * 1000ull, d_err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_err, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_err);
  if (e != cudaSuccess) return UNIFRAC_E_CUDA;
  *status = -(int32_t)h;
  return UNIFRAC_OK;
}

