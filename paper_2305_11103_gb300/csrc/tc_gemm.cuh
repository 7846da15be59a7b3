// Persistent, warp-specialised tcgen05 GEMM: D[M x N] = A[M x K] * B[N x K]^T
// with both operands K-major in global memory, fed by TMA into a 4-stage
// shared-memory ring (128-byte swizzle), accumulated by tcgen05.mma into one
// of two TMEM accumulators (128 lanes x 256 columns each), and handed to an
// epilogue functor that reads the accumulator with tcgen05.ld. The functor's
// apply_cols(row0, col, v, chunk, nchunks) receives column `col` of rows
// row0 .. row0 + 31 (v[r] = D[row0 + r][col]; the 32 lanes of a warp hold 32
// adjacent columns) for K-chunk `chunk` of `nchunks` (see chunk_kb).
//
//   warp 0, lane 0   TMA producer            (also allocates/frees TMEM)
//   warp 1, lane 0   MMA issuer
//   warps 2..9       epilogue: two warps per TMEM lane quarter, each taking
//                    half of the tile's columns (more loads in flight for
//                    the memory-bound epilogues)
//
// While the epilogue drains accumulator a, the MMA warp fills the other one,
// so the C traffic of one tile overlaps the loads and MMAs of the next.
// The K dimension can run over a list of operand "slice pairs" (for
// split-operand products): k-block kb belongs to pair i = kb / kb_per_pair
// and reads A columns pa[i] * slice_cols + kk * BK and B columns
// pb[i] * slice_cols + kk * BK, kk = kb - i * kb_per_pair. All pairs
// accumulate into the same FP32 accumulator. A plain GEMM has one pair (0, 0).
//
// Split stages (kSplit, for the hi/lo products of a split operand): a stage
// holds 64 bytes of K of four operand tiles, A slices pa[i] and pa[i] + 1 and
// B slices pb[i] and pb[i] + 1 (64-byte swizzle), and the MMA warp issues the
// three products hi*hi, hi*lo and lo*hi from it. Each slice is then loaded
// once instead of once per product it takes part in: two thirds of the bytes
// per unit of MMA work. Here k-block kb is 64 bytes of K of set i =
// kb / kb_per_pair.
//
// Every mbarrier wait is bounded; on timeout the status word gets
// BLOCKINV_ERR_TIMEOUT and the roles wind down.
//
// Single CTA (kPair false): each CTA owns whole 128 x 256 output tiles and
// loads both operand tiles of every k-block itself, by plain TMA tile loads
// into its own shared memory.
//
// CTA pair (kPair, clusters of two): the pair owns 256 x 256 tiles. Each CTA
// loads, by plain TMA tile loads into its own shared memory, the 128 rows of
// A that are its half of the tile and 128 of the 256 rows of B; all copies
// of a stage count on rank 0's barrier. Rank 0's MMA warp issues cta_group::2
// MMAs (M = 256) that read both CTAs' stages and write each CTA's 128 rows
// of the accumulator into that CTA's TMEM, and commits to the barriers of
// both; each CTA's epilogue drains its own TMEM and reports to rank 0.
//
// Consecutive items of a CTA and of its neighbours walk down a group of 16
// row tiles before the next column tile, so the B panel they share is read
// from L2.
#pragma once
#include <algorithm>

#include "internal.h"
#include "tc_common.cuh"

namespace blockinv {
namespace tc {

constexpr int kBM = 128;
constexpr int kBN = 256;
constexpr int kMaxStages = 6;
constexpr int kEpiWarps = 8;
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;

// The library's GEMMs run on CTA pairs (256 x 256 tiles, cta_group::2): per
// unit of MMA work a CTA loads two thirds of the operand bytes of a
// single-CTA 128 x 256 tile, which takes load off L2.
constexpr bool kPairTiles = true;

// B rows one CTA loads per tile: all kBN, or half of them in a CTA pair.
template <bool kPair>
__host__ __device__ constexpr int b_rows() { return kPair ? kBN / 2 : kBN; }
// Bytes of one operand stage in one CTA: kBM rows of A and b_rows() of B, 128
// bytes of K each (or, split, both slices of both at 64 bytes).
template <bool kPair>
__host__ __device__ constexpr int stage_bytes() { return (kBM + b_rows<kPair>()) * 128; }

constexpr int kMaxPairs = 48;
constexpr int kMaxChunks = 16;

struct KMap {
  int kblocks;            // k-blocks per output tile (= pairs * kb_per_pair)
  int kb_per_pair;        // k-blocks per slice pair
  int slice_cols;         // operand columns between consecutive slices
  int chunk_kb;           // k-blocks per accumulator hand-off (0 = the whole K); > 0 only for
                          // epilogues that add into their output (each chunk arrives separately)
  int chunk_end;          // chunks of chunk_kb cover k-blocks [0, chunk_end) (0 = all of K);
                          // the k-blocks after it form one more chunk
  int nbounds;            // > 0: instead, chunk c covers k-blocks [bounds[c], bounds[c + 1]), c < nbounds
  uint32_t group_starts;  // with nbounds: bit c set if chunk c starts a new group (bit 0 set)
  const int32_t* live_groups;  // with nbounds, may be null: only the chunks of groups below
                               // *live_groups run (read once at entry, written by an earlier kernel)
  int16_t bounds[kMaxChunks + 1];
  int8_t pa[kMaxPairs];   // A slice of pair i
  int8_t pb[kMaxPairs];   // B slice of pair i
};

// Group of chunk c under a group-start mask.
__host__ __device__ __forceinline__ int chunk_group(uint32_t group_starts, int c) {
#ifdef __CUDA_ARCH__
  return __popc(group_starts & ((2u << c) - 1u)) - 1;
#else
  return __builtin_popcount(group_starts & ((2u << c) - 1u)) - 1;
#endif
}

inline KMap plain_kmap(int kblocks) {
  KMap km{};
  km.kblocks = kblocks;
  km.kb_per_pair = kblocks;
  km.slice_cols = 0;
  return km;
}

struct GemmShared {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t cbar[2 * kEpiWarps];  // kTmaC epilogues: per warp, the TMA loads of its two C-block slots
  uint32_t tmem_base;
  uint32_t skip;  // pair: rank 0's reading of epi.skip(), taken by both CTAs
};

// Epilogue staging: each epilogue warp turns its 32 x 32 accumulator block
// (lane = row) around through shared memory (rows padded to 33 words, no bank
// conflicts), so that the functor's global accesses run along rows (lane =
// column) and every warp access covers whole cache lines.
constexpr int kStagePitch = 33;
constexpr size_t kSharedBytes = (sizeof(GemmShared) + 15) / 16 * 16;
constexpr size_t kEpiStageBytes = sizeof(float) * kEpiWarps * 32 * kStagePitch;

// kTmaC epilogues (the output moved by TMA in 32 x 32 FP32 blocks) keep two
// 4 KiB C-block slots per epilogue warp. The operand stages take what is left
// of the 227 KiB: 48 KiB stages (single CTA) 3 beside a kTmaC epilogue and 4
// beside the staging buffer of the others; 32 KiB stages (pair) 5 and 6.
constexpr size_t kTmaCBytes = (size_t)kEpiWarps * 2 * 4096;
template <bool kTmaC, bool kPair>
__host__ __device__ constexpr int gemm_stages() { return kPair ? (kTmaC ? 5 : 6) : (kTmaC ? 3 : 4); }
// Layout after the 1024-aligned base: the operand stages, the epilogue area
// (1024-aligned), then the barriers.
template <bool kTmaC, bool kPair>
constexpr size_t gemm_smem_bytes() {
  return (size_t)gemm_stages<kTmaC, kPair>() * stage_bytes<kPair>() + (kTmaC ? kTmaCBytes : kEpiStageBytes) +
         kSharedBytes + 1024;
}
static_assert(gemm_smem_bytes<false, false>() <= 227 * 1024 && gemm_smem_bytes<true, false>() <= 227 * 1024 &&
                  gemm_smem_bytes<false, true>() <= 227 * 1024 && gemm_smem_bytes<true, true>() <= 227 * 1024,
              "GEMM shared memory above the per-CTA limit");
static_assert(gemm_stages<false, true>() <= kMaxStages, "barrier arrays too short");

__device__ __forceinline__ void flag_timeout(int32_t* status) {
  if (status) atomicCAS(&status[0], 0, BLOCKINV_ERR_TIMEOUT);
}

// Work item t -> (row tile um, column tile tn), row tiles taken `group` at a
// time: consecutive items walk down a group's rows before the next column, so
// the items in flight together share A and B panels through L2 (a B tile is
// fetched once per group; the group's A panel is fetched again for later
// columns if it does not stay in L2).
constexpr int kGroupRows = 16;
__device__ __forceinline__ void item_coords(int t, int tiles_m, int tiles_n, int group, int& um, int& tn) {
  const int per_group = group * tiles_n;
  const int g = t / per_group;
  const int first = g * group;
  const int gsize = min(tiles_m - first, group);
  const int r = t - g * per_group;
  um = first + r % gsize;
  tn = r / gsize;
}

// The k-th (0-based) set bit of a 4-bit mask.
__device__ __forceinline__ int nth_set4(uint32_t mask, int k) {
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    if (mask & (1u << b)) {
      if (k == 0) return b;
      --k;
    }
  }
  return 0;
}

template <Kind K, class Epi, bool kSplit, bool kPair>
__global__ void __launch_bounds__(kGemmThreads, 1)
gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const __grid_constant__ CUtensorMap tmC, int tiles_m, int tiles_n, int m_base, int n_base, int dep_wait,
            int group, KMap km, Epi epi, int32_t* status) {
  constexpr int BK = (kSplit ? 64 : 128) / KindTraits<K>::elem_bytes;  // K elements per k-block
  constexpr int kS = gemm_stages<Epi::kTmaC, kPair>();                  // operand stages of this instance
  constexpr int kSB = stage_bytes<kPair>();                             // bytes of a stage in this CTA
  constexpr int kBR = b_rows<kPair>();                                  // B rows this CTA loads per tile
  constexpr int kTM = kPair ? 2 * kBM : kBM;                            // rows of an output tile
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* epi_area = smem + kS * kSB;
  GemmShared* sh = reinterpret_cast<GemmShared*>(epi_area + (Epi::kTmaC ? kTmaCBytes : kEpiStageBytes));
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // In a pair both CTAs walk the same tiles; rank 0 issues the MMAs and each
  // CTA loads, and runs the epilogue of, its own kBM rows of every tile.
  const int rank = kPair ? (int)cluster_rank() : 0;
  const int ntiles = tiles_m * tiles_n;
  const int first = kPair ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int stride = kPair ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  // Accumulator hand-offs: each of this CTA's tiles in nch K-chunks (kbc
  // k-blocks each up to kend, then the rest as one), every chunk accumulated
  // from zero and passed to the epilogue.
  const int kbc = (km.chunk_kb > 0 && km.chunk_kb < km.kblocks) ? km.chunk_kb : km.kblocks;
  const int kend = (km.chunk_end > 0 && km.chunk_end < km.kblocks) ? km.chunk_end : km.kblocks;
  const int nch_a = (kend + kbc - 1) / kbc;
  int nch = nch_a + (kend < km.kblocks ? 1 : 0);
  int kb_run = km.kblocks;  // k-blocks loaded per tile
  if (km.nbounds > 0) {     // explicit chunks, the trailing groups possibly switched off
    nch = km.nbounds;
    if (km.live_groups) {
      const int g = *(volatile const int32_t*)km.live_groups;
      nch = 0;
      while (nch < km.nbounds && chunk_group(km.group_starts, nch) < g) ++nch;
    }
    kb_run = km.bounds[nch];
  }
  const int my_tiles = first < ntiles ? (ntiles - first + stride - 1) / stride : 0;
  const int nitems = my_tiles * nch;
  // An earlier kernel of this computation failed: the status word it wrote is
  // the same for every CTA. A programmatic dependent runs to the end instead:
  // its predecessor may still be writing that word, and the dependent's
  // griddepcontrol.wait at the end is what keeps the stream order. The two
  // CTAs of a pair both take rank 0's reading (below): a timeout elsewhere in
  // this launch may set the word between their reads, and a CTA that left
  // alone would keep the other waiting at the cluster barrier.
  const bool skip_me = !dep_wait && epi.skip();
  if (!kPair && skip_me) return;

  if (threadIdx.x == 0) {
    sh->skip = skip_me ? 1u : 0u;
    for (int s = 0; s < kS; ++s) {
      mbar_init(&sh->full[s], 1);
      mbar_init(&sh->empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&sh->tfull[a], 1);
      mbar_init(&sh->tempty[a], kEpiWarps * (kPair ? 2 : 1));  // one arrival per epilogue warp
    }
    for (int w = 0; w < 2 * kEpiWarps; ++w) mbar_init(&sh->cbar[w], 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    if constexpr (kPair) {
      tmem_alloc_pair(&sh->tmem_base, 2 * kBN);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(&sh->tmem_base, 2 * kBN);
      tmem_relinquish();
    }
  }
  fence_before_sync();
  __syncthreads();
  // both CTAs' barriers initialised before either signals the other's
  if constexpr (kPair) cluster_sync_all();
  fence_after_sync();
  const uint32_t tmem = sh->tmem_base;
  bool skip_all = false;
  if constexpr (kPair) skip_all = ld_shared_cluster_u32(mapa_u32(smem_u32(&sh->skip), 0)) != 0;

  if (skip_all) {
    // the pair does no work and leaves through the common end below
  } else if (warp == 0 && lane == 0) {
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
    uint32_t it = 0;
    bool ok = true;
    for (int t = first; t < ntiles && ok; t += stride) {
      int um, tn;
      item_coords(t, tiles_m, tiles_n, group, um, tn);
      const int m0 = m_base + um * kTM + rank * kBM;  // this CTA's rows of A
      const int n0 = n_base + tn * kBN + rank * kBR;  // and of B
      for (int kb = 0; kb < kb_run; ++kb, ++it) {
        const int s = it % kS;
        const uint32_t ph = (it / kS) & 1;
        if (!mbar_wait(&sh->empty[s], ph ^ 1)) {
          ok = false;
          break;
        }
        unsigned char* sa = smem + s * kSB;
        // a pair's copies all count on rank 0's barrier, which rank 0 arms
        // for both CTAs' bytes
        const uint32_t fbar = kPair ? mapa_u32(smem_u32(&sh->full[s]), 0) : 0u;
        if (rank == 0) mbar_arrive_expect_tx(&sh->full[s], kSB * (kPair ? 2 : 1));
        auto load = [&](unsigned char* dst, const CUtensorMap* map, int x, int y) {
          if constexpr (kPair) tma_load_2d_pair(dst, map, fbar, x, y);
          else tma_load_2d(dst, map, &sh->full[s], x, y);
        };
        const int pair = kb / km.kb_per_pair;
        const int kk = kb - pair * km.kb_per_pair;
        const int xa = km.pa[pair] * km.slice_cols + kk * BK;
        const int xb = km.pb[pair] * km.slice_cols + kk * BK;
        if constexpr (kSplit) {  // [A hi | A lo | B hi | B lo], rows of 64 bytes
          load(sa, &tmA, xa, m0);
          load(sa + kBM * 64, &tmA, xa + km.slice_cols, m0);
          load(sa + 2 * kBM * 64, &tmB, xb, n0);
          load(sa + 2 * kBM * 64 + kBR * 64, &tmB, xb + km.slice_cols, n0);
        } else {
          load(sa, &tmA, xa, m0);
          load(sa + kBM * 128, &tmB, xb, n0);
        }
      }
    }
    if (!ok) {
      flag_timeout(status);
    } else if (it > 0) {
      // Let the last copies land before the CTA can leave (bounded): in a
      // pair, wait until the MMAs have consumed them.
      const uint32_t last = it - 1;
      if constexpr (kPair) mbar_wait(&sh->empty[last % kS], (last / kS) & 1);
      else mbar_wait(&sh->full[last % kS], (last / kS) & 1);
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    constexpr uint32_t id = idesc<K>(kTM, kBN);
    // arrive on the barrier at `bar` of every CTA of the tile once the MMAs
    // issued so far are done
    auto commit = [&](uint64_t* bar) {
      if constexpr (kPair) {
        mma_commit_pair(mapa_u32(smem_u32(bar), 0));
        mma_commit_pair(mapa_u32(smem_u32(bar), 1));
      } else {
        mma_commit(bar);
      }
    };
    auto wait = [&](uint64_t* bar, uint32_t parity) {
      return kPair ? mbar_wait_cluster(bar, parity) : mbar_wait(bar, parity);
    };
    auto issue = [&](uint32_t d, uint64_t da, uint64_t db, uint32_t acc) {
      if constexpr (kPair) mma_pair<K>(d, da, db, id, acc);
      else mma<K>(d, da, db, id, acc);
    };
    uint32_t it = 0, tl = 0;
    bool ok = true;
    for (int w = 0; w < nitems && ok; ++w, ++tl) {
      const int c = w % nch;
      const uint32_t a = tl & 1;
      const uint32_t aph = (tl >> 1) & 1;
      if (!wait(&sh->tempty[a], aph ^ 1)) {
        ok = false;
        break;
      }
      fence_after_sync();
      const uint32_t d = tmem + a * kBN;
      const int kb0 = km.nbounds > 0 ? km.bounds[c] : (c < nch_a ? c * kbc : kend);
      const int kb1 = km.nbounds > 0 ? km.bounds[c + 1] : (c < nch_a ? min(kend, kb0 + kbc) : km.kblocks);
      for (int kb = kb0; kb < kb1; ++kb, ++it) {
        const int s = it % kS;
        const uint32_t ph = (it / kS) & 1;
        if (!wait(&sh->full[s], ph)) {
          ok = false;
          break;
        }
        fence_after_sync();
        const uint32_t sa = smem_u32(smem + s * kSB);
        if constexpr (kSplit) {
          const uint64_t ah = sdesc_sw64(sa), al = sdesc_sw64(sa + kBM * 64);
          const uint64_t bh = sdesc_sw64(sa + 2 * kBM * 64), bl = sdesc_sw64(sa + 2 * kBM * 64 + kBR * 64);
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {  // 2 x 32 bytes of K per 64-byte row
            issue(d, ah + 2 * ks, bh + 2 * ks, ((kb - kb0) | ks) != 0 ? 1u : 0u);
            issue(d, ah + 2 * ks, bl + 2 * ks, 1u);
            issue(d, al + 2 * ks, bh + 2 * ks, 1u);
          }
        } else {
          const uint64_t da = sdesc_sw128(sa);
          const uint64_t db = sdesc_sw128(sa + kBM * 128);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)  // 4 x 32 bytes of K per 128-byte row
            issue(d, da + 2 * ks, db + 2 * ks, ((kb - kb0) | ks) != 0 ? 1u : 0u);
        }
        commit(&sh->empty[s]);
      }
      if (!ok) break;
      commit(&sh->tfull[a]);
    }
    if (!ok) flag_timeout(status);
  } else if (warp >= 2) {
    if constexpr (Epi::kTmaC) {
    // The C block of each 32 x 32 accumulator block comes in by TMA into one
    // of the warp's two slots (the tile's first two while its accumulator is
    // still being formed, each later one as soon as the block two before it
    // has gone out), is updated in place (lane = row of the block, as the
    // accumulator arrives from TMEM; the 128-byte swizzle makes the row's
    // float4 reads bank-conflict free) and goes back by TMA. Blocks in which
    // the epilogue changes no element (epi.block_live false) are neither
    // loaded nor stored; in the others, elements it must not change are
    // written back as loaded.
    constexpr int kWarpBlocks = kBN / 64;  // 32-column blocks per warp and tile
    static_assert(kWarpBlocks <= 4, "live-block mask holds 4 blocks");
    const int q = warp & 3;  // the TMEM lane quarter this warp may access
    const int half = (warp - 2) / 4;
    const int wi = warp - 2;
    const int cbeg = half * kWarpBlocks;
    uint32_t nload[2] = {0, 0};  // loads per slot: each slot barrier's phase
    bool ok = true;
    auto slot_buf = [&](int sl) { return epi_area + (wi * 2 + sl) * 4096; };
    auto request = [&](int sl, int x, int y) {  // lane 0
      mbar_arrive_expect_tx(&sh->cbar[wi * 2 + sl], 32 * 32 * 4);
      tma_load_2d(slot_buf(sl), &tmC, &sh->cbar[wi * 2 + sl], x, y);
    };
    uint32_t tl = 0;
    for (int w = 0; w < nitems && ok; ++w, ++tl) {
      const int t = first + (w / nch) * stride;
      const uint32_t a = tl & 1;
      const uint32_t aph = (tl >> 1) & 1;
      int um, tn;
      item_coords(t, tiles_m, tiles_n, group, um, tn);
      const int m0 = m_base + um * kTM + rank * kBM;  // this CTA's rows of the tile
      const int n0 = n_base + tn * kBN;
      const int row0 = m0 + q * 32;
      uint32_t live = 0;  // this warp's blocks that the epilogue changes
#pragma unroll
      for (int c = 0; c < kWarpBlocks; ++c)
        if (epi.block_live(row0, n0 + (cbeg + c) * 32)) live |= 1u << c;
      const int nl = __popc(live);
      auto col_of = [&](int i) { return n0 + (cbeg + nth_set4(live, i)) * 32; };
      if (lane == 0) {
        bulk_wait_read_all();  // the previous tile's last stores have left both slots
        if (nl > 0) request(0, col_of(0), row0);
        if (nl > 1) request(1, col_of(1), row0);
        // This warp's blocks of its next tile into L2 now, so that their loads
        // a tile later wait for L2 instead of DRAM.
        if (t + stride < ntiles) {
          int um2, tn2;
          item_coords(t + stride, tiles_m, tiles_n, group, um2, tn2);
          const int r2 = m_base + um2 * kTM + rank * kBM + q * 32;
          const int c2 = n_base + tn2 * kBN + cbeg * 32;
#pragma unroll
          for (int c = 0; c < kWarpBlocks; ++c)
            if (epi.block_live(r2, c2 + c * 32)) tma_prefetch_2d(&tmC, c2 + c * 32, r2);
        }
      }
      int pending = nl < 2 ? nl : 2;  // requested and not yet waited for, this tile
      int next = 0;                   // the live block waited for next (slot next & 1)
      if (!(kPair ? mbar_wait_cluster(&sh->tfull[a], aph) : mbar_wait(&sh->tfull[a], aph))) {
        flag_timeout(status);
        ok = false;
      }
      fence_after_sync();
#pragma unroll 1
      for (int i = 0; i < nl && ok; ++i) {
        const int sl = i & 1;
        unsigned char* cb = slot_buf(sl);
        const int col0 = col_of(i);
        uint32_t v[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + a * kBN + (col0 - n0), v);
        tmem_wait_ld();
        if (!mbar_wait(&sh->cbar[wi * 2 + sl], nload[sl] & 1)) {
          // the load is still in flight: the drain below waits for it again
          flag_timeout(status);
          ok = false;
          break;
        }
        ++nload[sl];
        --pending;
        ++next;
        const int row = row0 + lane;
        if (epi.block_simple(row0, col0)) {  // warp-uniform: x - v throughout
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float4* p = reinterpret_cast<float4*>(cb + lane * 128 + ((j ^ (lane & 7)) << 4));
            float4 x = *p;
            x.x -= __uint_as_float(v[4 * j + 0]);
            x.y -= __uint_as_float(v[4 * j + 1]);
            x.z -= __uint_as_float(v[4 * j + 2]);
            x.w -= __uint_as_float(v[4 * j + 3]);
            *p = x;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float4* p = reinterpret_cast<float4*>(cb + lane * 128 + ((j ^ (lane & 7)) << 4));
            float4 x = *p;
            x.x = epi.value(row, col0 + 4 * j + 0, x.x, __uint_as_float(v[4 * j + 0]));
            x.y = epi.value(row, col0 + 4 * j + 1, x.y, __uint_as_float(v[4 * j + 1]));
            x.z = epi.value(row, col0 + 4 * j + 2, x.z, __uint_as_float(v[4 * j + 2]));
            x.w = epi.value(row, col0 + 4 * j + 3, x.w, __uint_as_float(v[4 * j + 3]));
            *p = x;
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          tma_store_2d(&tmC, cb, col0, row0);
          bulk_commit();
          if (i + 2 < nl) {
            bulk_wait_read_all();  // the slot may be refilled
            request(sl, col_of(i + 2), row0);
          }
        }
        if (i + 2 < nl) ++pending;
        __syncwarp();
      }
      // after a failure, wait (bounded) for the copies still in flight
      for (int j = 0; j < pending; ++j) {
        const int sl = (next + j) & 1;
        mbar_wait(&sh->cbar[wi * 2 + sl], nload[sl] & 1);
        ++nload[sl];
      }
      if (!ok) break;
      fence_before_sync();
      __syncwarp();
      if (lane == 0) {  // this warp has read accumulator a (in a pair: on rank 0's barrier)
        if constexpr (kPair) mbar_arrive_cluster(mapa_u32(smem_u32(&sh->tempty[a]), 0));
        else mbar_arrive(&sh->tempty[a]);
      }
    }
    if (lane == 0) bulk_wait_all();  // every store complete before the CTA can leave
    } else {
    float* stage = reinterpret_cast<float*>(epi_area) + (warp - 2) * 32 * kStagePitch;
    const int q = warp & 3;  // the TMEM lane quarter this warp may access
    const int half = (warp - 2) / 4;
    uint32_t tl = 0;
    for (int w = 0; w < nitems; ++w, ++tl) {
      const int t = first + (w / nch) * stride;
      const uint32_t a = tl & 1;
      const uint32_t aph = (tl >> 1) & 1;
      if (!(kPair ? mbar_wait_cluster(&sh->tfull[a], aph) : mbar_wait(&sh->tfull[a], aph))) {
        flag_timeout(status);
        break;
      }
      fence_after_sync();
      int um, tn;
      item_coords(t, tiles_m, tiles_n, group, um, tn);
      const int m0 = m_base + um * kTM + rank * kBM;  // this CTA's rows of the tile
      const int n0 = n_base + tn * kBN;
      const int row0 = m0 + q * 32;
#pragma unroll 1
      for (int c = half * (kBN / 64); c < (half + 1) * (kBN / 64); ++c) {
        uint32_t v[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + a * kBN + c * 32, v);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) stage[lane * kStagePitch + j] = __uint_as_float(v[j]);
        __syncwarp();
        float col[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) col[r] = stage[r * kStagePitch + lane];
        __syncwarp();
        epi.apply_cols(row0, n0 + c * 32 + lane, col, w % nch, nch);
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) {  // this warp has read accumulator a (in a pair: on rank 0's barrier)
        if constexpr (kPair) mbar_arrive_cluster(mapa_u32(smem_u32(&sh->tempty[a]), 0));
        else mbar_arrive(&sh->tempty[a]);
      }
    }
    }
  }
  __syncthreads();
  // no CTA of a pair leaves while the other may still signal its barriers
  if constexpr (kPair) cluster_sync_all();
  if (warp == 0) {
    fence_after_sync();
    if constexpr (kPair) tmem_dealloc_pair(tmem, 2 * kBN);
    else tmem_dealloc(tmem, 2 * kBN);
  }
  // Launched as the programmatic dependent of the kernel before it: this grid
  // completes only after that one has, so the stream order after it holds.
  if (dep_wait && threadIdx.x == 0) asm volatile("griddepcontrol.wait;" ::: "memory");
}

int num_sms();

// A window of the output: the tiles of rows m_base .. m_base + M - 1 and
// columns n_base .. n_base + N - 1 (m_base a multiple of kBM, n_base a
// multiple of kBN), on at most max_ctas CTAs (0 = one per SM). The tiles are
// those of the whole product, so every output element is the same sum
// whichever window computes it.
//
// after_trigger: launch as the programmatic dependent of the previous kernel
// in the stream, which lets this grid start once every CTA of that kernel has
// executed griddepcontrol.launch_dependents (so both run at once on disjoint
// SMs). The caller guarantees that the two touch disjoint data; this grid
// still completes only after the previous one.
struct Window {
  int m_base = 0;
  int n_base = 0;
  int max_ctas = 0;
  int group_rows = 0;  // row tiles per group of the tile walk (0 = kGroupRows)
  bool after_trigger = false;
  const CUtensorMap* c_map = nullptr;  // the output for kTmaC epilogues: 32 x 32 FP32 boxes, 128-byte swizzle
};

// Most CTA pairs of this kernel resident at once (cached per instance).
template <class Kern>
int max_pairs(Kern kern, size_t smem) {
  static const int n = [&] {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(kGemmThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      c = 0;
    }
    return c;
  }();
  return n;
}

// tA: box {128 bytes of K, kBM rows}; tB: box {128 bytes of K, b_rows<kPair>()
// rows} (64 bytes of K and a 64-byte swizzle for kSplit). kPair: 256 x 256
// tiles on CTA pairs (clusters of two, cta_group::2 MMAs).
template <Kind K, class Epi, bool kSplit = false, bool kPair = false>
cudaError_t launch_gemm(const CUtensorMap& tA, const CUtensorMap& tB, int M, int N, KMap km, const Epi& epi,
                        int32_t* status, cudaStream_t s, const Window& win = Window{}) {
  if (win.m_base % kBM != 0 || win.n_base % kBN != 0 || win.max_ctas < 0) return cudaErrorInvalidValue;
  if (Epi::kTmaC && !win.c_map) return cudaErrorInvalidValue;
  // A kTmaC epilogue loads and stores each C block once per tile: K-chunked
  // hand-offs would reload a block whose store may not be visible yet.
  if (Epi::kTmaC && (km.chunk_kb > 0 || km.chunk_end > 0 || km.nbounds > 0)) return cudaErrorInvalidValue;
  const CUtensorMap tC = win.c_map ? *win.c_map : CUtensorMap{};
  const int group = win.group_rows > 0 ? win.group_rows : kGroupRows;
  int ctas = (win.max_ctas > 0 && win.max_ctas < num_sms()) ? win.max_ctas : num_sms();
  constexpr int kTM = kPair ? 2 * kBM : kBM;
  const int tiles_m = (M + kTM - 1) / kTM;
  const int tiles_n = (N + kBN - 1) / kBN;
  const int ntiles = tiles_m * tiles_n;
  if (ntiles == 0 || km.kblocks <= 0) return cudaSuccess;
  auto kern = gemm_kernel<K, Epi, kSplit, kPair>;
  const size_t smem = gemm_smem_bytes<Epi::kTmaC, kPair>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = ntiles < ctas ? ntiles : ctas;
  if constexpr (kPair) {
    // whole pairs, all resident at once (the tile walk is persistent)
    const int mp = max_pairs(kern, smem);
    const int pairs = std::min({ctas / 2, mp > 0 ? mp : ctas / 2, ntiles});
    if (pairs <= 0) return cudaErrorInvalidConfiguration;
    grid = 2 * pairs;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kGemmThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (kPair) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = 2;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  if (win.after_trigger) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, tA, tB, tC, tiles_m, tiles_n, win.m_base, win.n_base,
                            win.after_trigger ? 1 : 0, group, km, epi, status);
}

}  // namespace tc
}  // namespace blockinv
