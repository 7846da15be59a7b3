// K1: inverse of one pivot (diagonal) block, the paper's "diamond" operation
// (Table 3): P^-1 of the leading block A at the first elimination step, of the
// current Schur complement S_A = D - C A^-1 B afterwards (Eq. (a)).
//
// Gauss-Jordan elimination with partial pivoting, in place, FP64 (or FP32 for
// the mixed path). The b x b block is split by rows over a thread-block
// cluster of up to 16 CTAs; each CTA keeps its rows in shared memory and
// reads the other CTAs' candidates and the pivot row through distributed
// shared memory. One cluster barrier per eliminated column:
//
//   local argmax of |a[r][c]| over rows not yet used as pivots (warp 0)
//   -- cluster barrier --
//   every warp reduces the CTAs' candidates to the same pivot row p
//   (largest magnitude, lowest row index on ties); all CTAs read row p,
//   scale it (a[p][c] replaced by 1/piv) and eliminate column c from their
//   own rows (a[i][c] replaced by -a[i][c]/piv).
//
// Rows are not swapped; the pivot row of each column is recorded and the
// result is unscrambled on the way out: with p_c the pivot row of column c,
// inverse[c][p_j] = a[p_c][j]. The owner of a pivot row writes its scaled copy
// back only after the next barrier, when no other CTA can still be reading
// the unscaled row.
//
// Errors: a non-finite entry in the block gives BLOCKINV_ERR_NONFINITE; a
// column whose candidates are all exactly zero gives BLOCKINV_ERR_SINGULAR;
// the first error is kept in the device status word with the block index.
// The pivot row is scaled by multiplying with the correctly rounded
// reciprocal of the pivot (within an ulp of dividing; exact for unit pivots);
// the FP32 panel kernel of the mixed path uses a Newton-refined estimate.
#include <algorithm>
#include <climits>
#include <mutex>
#include <cooperative_groups.h>

#include "fp64_ops.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace blockinv {

namespace {

constexpr int kPivotThreads = 256;

template <bool kCluster>
__device__ __forceinline__ void cluster_or_block_sync() {
  if constexpr (kCluster) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

template <bool kCluster, typename P>
__device__ __forceinline__ P* peer(P* p, int rank) {
  if constexpr (kCluster) {
    return cg::this_cluster().map_shared_rank(p, rank);
  } else {
    return p;
  }
}

__device__ __forceinline__ void set_status(int32_t* status, int code, int block) {
  if (atomicCAS(&status[0], 0, code) == 0) status[1] = block;
}

// Correctly rounded reciprocal; a column is scaled by multiplying with it (a
// full IEEE division per element is a long instruction sequence).
__device__ __forceinline__ float recip(float v) { return __frcp_rn(v); }

// The FP32 panel kernel's reciprocal (on the critical path of every column;
// its result is refined later in the mixed path): the hardware estimate and
// one Newton-Raphson step r <- r (2 - v r), within about an ulp.
__device__ __forceinline__ float recip_newton(float v) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r * fmaf(-v, r, 2.0f);
}
__device__ __forceinline__ double recip(double v) { return __drcp_rn(v); }

template <typename T>
__device__ __forceinline__ void argmax_step(T& bv, int& bi, T ov, int oi) {
  if (ov > bv || (ov == bv && oi < bi)) {
    bv = ov;
    bi = oi;
  }
}

// T: arithmetic type; TIO: the type of P and of the output (FP32 blocks of the
// mixed path can be inverted in FP64).
template <typename T, typename TIO, bool kCluster>
__device__ __forceinline__ void pivot_gj_body(const TIO* __restrict__ P, int64_t ldp, int b, int R, int jlog,
                                              TIO* __restrict__ out, int64_t ldo, int32_t* status,
                                              int block_index) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* rows = reinterpret_cast<T*>(smem_raw);   // R x b, this CTA's rows
  T* prow = rows + (size_t)R * b;             // b: scaled pivot row
  T* fvec = prow + b;                         // R: multipliers a[r][c]
  T* pabs = fvec + R;                         // 2: candidate |pivot| by step parity
  int* pidx = reinterpret_cast<int*>(pabs + 2);  // 2: candidate row by step parity
  int* step_of_row = pidx + 2;                // R: column at which the row was pivot (-1 = not yet)
  int* perm = step_of_row + R;                // b: pivot row of each column
  int* flags = perm + b;                      // 1: non-finite entry seen by this CTA

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  int rank = 0, nranks = 1;
  if constexpr (kCluster) {
    rank = (int)cg::this_cluster().block_rank();
    nranks = (int)cg::this_cluster().num_blocks();
  }
  const int r0 = rank * R;
  const int nloc = max(0, min(b, r0 + R) - r0);
  const int jw = 1 << jlog;                   // threads along a row (power of two)
  const int jj = tid & (jw - 1);
  const int rr = tid >> jlog;
  const int rstep = kPivotThreads >> jlog;

  if (tid == 0) flags[0] = 0;
  for (int r = tid; r < R; r += kPivotThreads) step_of_row[r] = -1;
  __syncthreads();
  int bad = 0;
  for (int r = rr; r < nloc; r += rstep) {
    for (int j = jj; j < b; j += jw) {
      T v = static_cast<T>(P[(int64_t)(r0 + r) * ldp + j]);
      if (!isfinite(v)) bad = 1;
      rows[(size_t)r * b + j] = v;
    }
  }
  if (bad) atomicOr(&flags[0], 1);
  // Skip everything if an earlier kernel of this inversion already failed:
  // bit 2, OR-ed over the cluster with the rest, so that every CTA leaves
  // here or none does (each CTA reads the status word at its own time).
  if (tid == 0 && *(volatile int32_t*)&status[0] != 0) atomicOr(&flags[0], 2);
  cluster_or_block_sync<kCluster>();
  int anybad = 0;
  for (int q = 0; q < nranks; ++q) anybad |= *peer<kCluster>(&flags[0], q);
  if (anybad) {
    if (anybad == 1 && rank == 0 && tid == 0) set_status(status, BLOCKINV_ERR_NONFINITE, block_index);
    cluster_or_block_sync<kCluster>();
    return;
  }

  int prev_p = -1;
  int failed = 0;
  for (int c = 0; c < b; ++c) {
    if (tid < 32) {
      T bv = T(-1);
      int bi = INT_MAX;
      for (int r = lane; r < nloc; r += 32) {
        if (step_of_row[r] < 0) {
          T v = fabs(rows[(size_t)r * b + c]);
          if (v > bv) {
            bv = v;
            bi = r0 + r;
          }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, bv, off);
        int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        argmax_step(bv, bi, ov, oi);
      }
      if (lane == 0) {
        pabs[c & 1] = bv;
        pidx[c & 1] = bi;
      }
    }
    cluster_or_block_sync<kCluster>();
    // The previous pivot row can now be overwritten with its scaled copy.
    if (prev_p >= r0 && prev_p < r0 + nloc)
      for (int j = tid; j < b; j += kPivotThreads) rows[(size_t)(prev_p - r0) * b + j] = prow[j];
    T gv = T(-1);
    int gi = INT_MAX;
    if (lane < nranks) {
      gv = *peer<kCluster>(&pabs[c & 1], lane);
      gi = *peer<kCluster>(&pidx[c & 1], lane);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, gv, off);
      int oi = __shfl_xor_sync(0xffffffffu, gi, off);
      argmax_step(gv, gi, ov, oi);
    }
    __syncthreads();
    if (gi == INT_MAX || !(gv > T(0))) {
      failed = BLOCKINV_ERR_SINGULAR;
      break;
    }
    if (!isfinite(gv)) {
      failed = BLOCKINV_ERR_NONFINITE;
      break;
    }
    const int p = gi;
    const int owner = p / R;
    const T* prem = peer<kCluster>(rows, owner) + (size_t)(p - owner * R) * b;
    const T inv = recip(prem[c]);
    for (int j = tid; j < b; j += kPivotThreads) prow[j] = (j == c) ? inv : prem[j] * inv;
    for (int r = tid; r < nloc; r += kPivotThreads) fvec[r] = rows[(size_t)r * b + c];
    if (tid == 0) {
      perm[c] = p;
      if (owner == rank) step_of_row[p - r0] = c;
    }
    __syncthreads();
    for (int r = rr; r < nloc; r += rstep) {
      if (r0 + r == p) continue;
      const T f = fvec[r];
      T* row = rows + (size_t)r * b;
      for (int j = jj; j < b; j += jw) {
        const T v = (j == c) ? T(0) : row[j];
        row[j] = v - f * prow[j];
      }
    }
    __syncthreads();
    prev_p = p;
  }
  // After this barrier no CTA reads another CTA's shared memory any more.
  cluster_or_block_sync<kCluster>();
  if (failed) {
    if (rank == 0 && tid == 0) set_status(status, failed, block_index);
    return;
  }
  if (prev_p >= r0 && prev_p < r0 + nloc)
    for (int j = tid; j < b; j += kPivotThreads) rows[(size_t)(prev_p - r0) * b + j] = prow[j];
  __syncthreads();
  for (int r = rr; r < nloc; r += rstep) {
    const int i = step_of_row[r];
    const T* row = rows + (size_t)r * b;
    for (int j = jj; j < b; j += jw) out[(int64_t)i * ldo + perm[j]] = static_cast<TIO>(row[j]);
  }
}

// gate (may be null): the kernel runs only if *gate != 0 (read by every CTA
// before any cluster barrier, so the whole cluster leaves together).
template <typename T, typename TIO, bool kCluster>
__global__ void __launch_bounds__(kPivotThreads)
pivot_gj_kernel(const TIO* __restrict__ P, int64_t ldp, int b, int R, int jlog, TIO* __restrict__ out,
                int64_t ldo, int32_t* status, int block_index, const int32_t* gate) {
  // a kernel launched after this one as its programmatic dependent may start
  // now (it must not touch this block or its inverse)
  asm volatile("griddepcontrol.launch_dependents;");
  if (gate && *(volatile const int32_t*)gate == 0) return;
  pivot_gj_body<T, TIO, kCluster>(P, ldp, b, R, jlog, out, ldo, status, block_index);
}

// Condition estimate of an FP32 pivot block after its FP32 inverse:
// kappa = ||P||_inf ||P^-1||_inf. *gate = 1 when kappa > limit (or is not
// finite), and then *count is incremented; limit < 0 sets the gate always.
// One CTA of 1024 threads: a warp per row at a time, all of a lane's loads of
// both blocks in flight together (the kernel is latency-bound otherwise).
constexpr int kCondThreads = 1024;
__global__ void __launch_bounds__(kCondThreads)
pivot_cond_kernel(const float* __restrict__ P, int64_t ldp, const float* __restrict__ Pinv, int64_t ldo, int b,
                  float limit, int32_t* gate, int32_t* count, const int32_t* status) {
  // Launched as the programmatic dependent of the pivot inverse: let the
  // kernel after this one start, then wait for the inverse to be complete.
  asm volatile("griddepcontrol.launch_dependents;");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __shared__ float red[2][kCondThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float mp = 0.f, mi = 0.f;
  for (int r = warp; r < b; r += kCondThreads / 32) {
    float sp = 0.f, si = 0.f;
    for (int j = lane; j < b; j += 32) {
      sp += fabsf(P[(int64_t)r * ldp + j]);
      si += fabsf(Pinv[(int64_t)r * ldo + j]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sp += __shfl_xor_sync(0xffffffffu, sp, off);
      si += __shfl_xor_sync(0xffffffffu, si, off);
    }
    mp = fmaxf(mp, sp);
    mi = fmaxf(mi, si);
  }
  if (lane == 0) {
    red[0][warp] = mp;
    red[1][warp] = mi;
  }
  __syncthreads();
  if (tid == 0) {
    float a = 0.f, c = 0.f;
    for (int w = 0; w < kCondThreads / 32; ++w) {
      a = fmaxf(a, red[0][w]);
      c = fmaxf(c, red[1][w]);
    }
    const float kappa = a * c;
    const bool ill = limit < 0.f || !(kappa <= limit);
    const bool live = *(volatile const int32_t*)status == 0;
    *gate = (ill && live) ? 1 : 0;
    if (ill && live) atomicAdd(count, 1);
  }
}

// Grouped form for pivot blocks of order kWarpPivotMax + 1 .. kGroupedMaxB:
// one CTA per matrix of a batch, the block in shared memory. Per column: the
// pivot row (largest |x| among the rows not yet used, lowest row on ties,
// compared as integer keys: |x| as its bit pattern with a top bit marking a
// candidate), the scaled pivot row and the column's multipliers, then the
// whole block updated one element per thread and pass, so every lane works
// whatever b is. A warp's FP64 instruction holds the FP64 pipe for 16 clocks
// on this GPU: only the threads that scale the pivot row form its reciprocal,
// and no comparison runs on that pipe.
__host__ __device__ constexpr size_t grouped_pivot_smem(int b) {
  return sizeof(double) * ((size_t)b * b + 2 * (size_t)b) + sizeof(unsigned long long) * 8 +
         sizeof(int) * (8 + 2 * (size_t)b + 1) + 16;
}

__global__ void __launch_bounds__(kPivotThreads)
pivot_gj_grouped_kernel(const GroupStep* __restrict__ items, int count, int bmin) {
  const int m = blockIdx.x;
  if (m >= count) return;
  const GroupStep it = items[m];
  if (it.b > kGroupedMaxB || it.b <= bmin) return;  // the cluster kernel / the warp kernel
  const int b = it.b, bb = b * b;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* rows = reinterpret_cast<double*>(smem_raw);  // b x b
  double* prow = rows + bb;                            // b: scaled pivot row
  double* fvec = prow + b;                             // b: multipliers x[r][c]
  unsigned long long* wkey = reinterpret_cast<unsigned long long*>(fvec + b);  // per warp
  int* wrow = reinterpret_cast<int*>(wkey + kPivotThreads / 32);               // per warp
  int* perm = wrow + kPivotThreads / 32;               // b: pivot row of column c
  int* srow = perm + b;                                // b: column row r was pivot for (-1 = not yet)
  int* flag = srow + b;                                // non-finite entry seen
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* P = it.X + (int64_t)it.o * it.ldx + it.o;
  if (tid == 0) flag[0] = 0;
  for (int r = tid; r < b; r += kPivotThreads) srow[r] = -1;
  __syncthreads();
  int bad = 0;
  for (int e = tid; e < bb; e += kPivotThreads) {
    const int r = e / b, j = e - r * b;
    const double v = P[(int64_t)r * it.ldx + j];
    bad |= nonfinite_bits(v) ? 1 : 0;
    rows[e] = v;
  }
  if (bad) atomicOr(flag, 1);
  // an earlier kernel of this inversion failed: bit 2, read once for the
  // whole CTA, so that all threads leave here or none does
  if (tid == 0 && *(volatile const int32_t*)it.status != 0) atomicOr(flag, 2);
  __syncthreads();
  const int any = flag[0];
  if (any) {
    if (any == 1 && tid == 0) set_status(it.status, BLOCKINV_ERR_NONFINITE, it.k);
    return;
  }
  // flat walk e = tid + 256 i over the block, (r, j) stepped without division
  const int dr = kPivotThreads / b, dj = kPivotThreads - dr * b;
  const int r_first = tid / b, j_first = tid - r_first * b;
  int failed = 0;
  for (int c = 0; c < b; ++c) {
    unsigned long long key = 0ull;
    int row = INT_MAX;
    if (tid < b && srow[tid] < 0) {
      key = static_cast<unsigned long long>(__double_as_longlong(fabs(rows[tid * b + c]))) | (1ull << 63);
      row = tid;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, off);
      const int oi = __shfl_xor_sync(0xffffffffu, row, off);
      if (ok > key || (ok == key && oi < row)) {
        key = ok;
        row = oi;
      }
    }
    if (lane == 0) {
      wkey[warp] = key;
      wrow[warp] = row;
    }
    __syncthreads();
    key = wkey[0];
    row = wrow[0];
    for (int w = 1; w < kPivotThreads / 32; ++w) {
      const unsigned long long ok = wkey[w];
      const int oi = wrow[w];
      if (ok > key || (ok == key && oi < row)) {
        key = ok;
        row = oi;
      }
    }
    if (key == 0ull || key == (1ull << 63)) {  // no candidate, or all of them zero
      failed = BLOCKINV_ERR_SINGULAR;
      break;
    }
    if (((key >> 52) & 0x7FF) == 0x7FF) {
      failed = BLOCKINV_ERR_NONFINITE;
      break;
    }
    const int p = row;
    if (tid < b) {
      const double inv = recip(rows[p * b + c]);
      prow[tid] = (tid == c) ? inv : rows[p * b + tid] * inv;
      fvec[tid] = rows[tid * b + c];
    }
    if (tid == 0) {
      perm[c] = p;
      srow[p] = c;
    }
    __syncthreads();
    int r = r_first, j = j_first;
    for (int e = tid; e < bb; e += kPivotThreads) {
      const double pj = prow[j];
      rows[e] = (r == p) ? pj : ((j == c) ? 0.0 : rows[e]) - fvec[r] * pj;
      j += dj;
      r += dr;
      if (j >= b) {
        j -= b;
        ++r;
      }
    }
    __syncthreads();
  }
  if (failed) {
    if (tid == 0) set_status(it.status, failed, it.k);
    return;
  }
  // unscramble: row r holds row srow[r] of the inverse, column j at perm[j]
  int r = r_first, j = j_first;
  for (int e = tid; e < bb; e += kPivotThreads) {
    it.Pinv[(int64_t)srow[r] * b + perm[j]] = rows[e];
    j += dj;
    r += dr;
    if (j >= b) {
      j -= b;
      ++r;
    }
  }
}

// Grouped warp form for pivot blocks of order <= 32: one warp per matrix, a
// row per lane in registers, Gauss-Jordan with partial pivoting (largest |x|
// compared on its bit pattern, lowest row on ties), the pivot row broadcast
// by shuffles: no barriers at all. Rows are not swapped; the result is
// unscrambled on output (inverse[c][perm[j]] = row of pivot c, entry j).
constexpr int kWarpPivotMax = 32;
__global__ void __launch_bounds__(128)
pivot_warp_grouped_kernel(const GroupStep* __restrict__ items, int count) {
  const int m = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (m >= count) return;  // warp-uniform from here on
  const GroupStep it = items[m];
  if (it.b > kWarpPivotMax || *(volatile const int32_t*)it.status != 0) return;
  const int b = it.b;
  const double* P = it.X + (int64_t)it.o * it.ldx + it.o;
  double x[kWarpPivotMax];
  bool bad = false;
#pragma unroll
  for (int l = 0; l < kWarpPivotMax; ++l) {
    x[l] = (lane < b && l < b) ? P[(int64_t)lane * it.ldx + l] : 0.0;
    bad |= !isfinite(x[l]);
  }
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) set_status(it.status, BLOCKINV_ERR_NONFINITE, it.k);
    return;
  }
  bool used = false;
  int my_col = -1;
  int perm[kWarpPivotMax];
#pragma unroll
  for (int c = 0; c < kWarpPivotMax; ++c) {
    perm[c] = 0;
    if (c < b) {
      const bool cand = lane < b && !used;
      unsigned long long key = cand ? static_cast<unsigned long long>(__double_as_longlong(fabs(x[c]))) : 0ull;
      int idx = cand ? lane : kWarpPivotMax;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, off);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
        if (ok > key || (ok == key && oi < idx)) {
          key = ok;
          idx = oi;
        }
      }
      const int pr = idx < kWarpPivotMax ? idx : 0;
      const double pc = __shfl_sync(0xffffffffu, x[c], pr);
      if (idx >= kWarpPivotMax || pc == 0.0 || !isfinite(pc)) {
        if (lane == 0)
          set_status(it.status, (idx < kWarpPivotMax && pc != 0.0) ? BLOCKINV_ERR_NONFINITE : BLOCKINV_ERR_SINGULAR,
                     it.k);
        return;
      }
      perm[c] = pr;
      const double inv = 1.0 / pc;
      const bool is_pivot = lane == pr;
      const double alpha = is_pivot ? inv : -x[c] * inv;
#pragma unroll
      for (int l = 0; l < kWarpPivotMax; ++l) {
        const double pl = __shfl_sync(0xffffffffu, x[l], pr);
        if (l < b) x[l] = (l == c) ? alpha : fma(alpha, pl, is_pivot ? 0.0 : x[l]);
      }
      if (is_pivot) {
        used = true;
        my_col = c;
      }
    }
  }
  if (lane < b) {
#pragma unroll
    for (int j = 0; j < kWarpPivotMax; ++j)
      if (j < b) it.Pinv[(int64_t)my_col * b + perm[j]] = x[j];
  }
}

// ------------------------------------------------------------------------
// Look-ahead variant for FP64 blocks of order <= 256 (the FP64 path's pivot
// blocks). On this GPU the FP64 pipe retires 2 DFMA per clock and SM, and
// an FP64 warp instruction takes its full pipe slot whatever its active
// lanes (measured: one thread's 16 FMAs on a column cost about a
// microsecond). The 256-block (b^3 = 16.8 M DFMA) therefore spreads its rows
// over a cluster of up to 16 CTAs (at most kLaRows rows each, in shared
// memory), and the per-column critical path is built from few FP64
// instructions, every one of them with all its lanes busy, and from shared
// memory of the CTA itself:
//
//   1. every CTA waits on its own mbarrier until the records of column c of
//      all C CTAs have arrived in its slots (record = the CTA's candidate
//      key: |value| bits, row, reciprocal; and the candidate row);
//   2. warp 0 reduces the C keys (integer compares) to the pivot row, which
//      every CTA finds, unscaled, in the winner's slot; applies step c to
//      column c + 1 (lane = local row, one FMA), takes each lane's
//      reciprocal, and picks the local candidate of column c + 1 (largest
//      magnitude among rows not yet used as pivots, lowest row on ties) on
//      the integer pipe from the value's bit pattern;
//   3. every thread applies step c to the candidate row's element of its
//      column (one FMA); one warp packs the record of column c + 1 and sends
//      it to every CTA of the cluster as one bulk copy each (cp.async.bulk,
//      shared::cta to shared::cluster), completing on the receiver's
//      mbarrier;
//   4. step c on every other local row (the bulk of the FP64 work, b x rows
//      FMAs), started by the other warps at once, while the copies are in
//      flight.
//
// A record travels by DMA, so no thread waits for a remote store and no
// cluster barrier runs per column (a phase probe of the earlier form, with
// a cluster barrier and remote row loads, spent 3700 of 5970 clocks per
// column outside the bulk at b = 256). Slots, outgoing records and mbarriers
// alternate by column parity. A CTA sends the records of column c + 2 only
// after all records of column c + 1 have reached it, and each CTA sends
// those after it has finished reading its slots of column c: so a slot is
// rewritten only after its last reader is done with it.
//
// Each element gets x - f * (P[p][j] r) with r the pivot's reciprocal
// (3 FMAs from the hardware estimate, within an ulp; exact for powers of
// two), the same arithmetic as the row-split kernel except for that
// reciprocal.
constexpr int kLaRows = 16;             // local rows per CTA
constexpr int kLaMaxB = kPivotThreads;  // one column per thread

struct LaKey {
  unsigned long long vbits;  // |candidate| as FP64 bits (0 with no candidate)
  int row;                   // global row (INT_MAX with no candidate)
  int pad;
  double inv;                // reciprocal of the candidate
  double pad2;               // the record header is 32 bytes
};
static_assert(sizeof(LaKey) == 32, "record header");

// Bytes of one record (key, then the candidate row of b doubles), a multiple
// of 16 for the bulk copy.
__host__ __device__ __forceinline__ int la_rec_bytes(int b) { return (32 + 8 * b + 15) / 16 * 16; }

struct LaSmem {
  double* rows;            // [kLaRows][b]: this CTA's rows
  unsigned char* slot;     // [2][C] records by column parity and sending CTA
  unsigned char* out;      // [2] records this CTA sends, by column parity
  uint64_t* bar;           // [2] mbarriers: all C records of a column have arrived
  double* fbuf;            // [kLaRows]: multipliers of the current step (column c before it)
  double* win;             // [3]: the current pivot's reciprocal, then (as int32) its CTA, row, failure
  int* perm;               // [b]: pivot row of each column
  int* misc;               // [0] candidate local row (-1 none), [1] flags of this CTA, [2] wait failed
  int rec;                 // record bytes
  __device__ LaKey* key(int par, int q) const {
    return reinterpret_cast<LaKey*>(slot + ((size_t)par * 16 + q) * rec);
  }
  __device__ double* row_of(int par, int q) const {
    return reinterpret_cast<double*>(slot + ((size_t)par * 16 + q) * rec + 32);
  }
};

__device__ __forceinline__ LaSmem la_layout(unsigned char* raw, int b) {
  LaSmem m;
  m.rec = la_rec_bytes(b);
  m.rows = reinterpret_cast<double*>(raw);
  m.slot = reinterpret_cast<unsigned char*>(m.rows + (size_t)kLaRows * b);  // 16-byte aligned: 128 b bytes of rows
  m.out = m.slot + (size_t)2 * 16 * m.rec;
  m.bar = reinterpret_cast<uint64_t*>(m.out + (size_t)2 * m.rec);
  m.fbuf = reinterpret_cast<double*>(m.bar + 2);
  m.win = m.fbuf + kLaRows;
  m.perm = reinterpret_cast<int*>(m.win + 3);
  m.misc = m.perm + b;
  return m;
}

size_t la_smem_bytes(int b) {
  return sizeof(double) * (size_t)kLaRows * b + (size_t)(2 * 16 + 2) * la_rec_bytes(b) + 2 * sizeof(uint64_t) +
         sizeof(double) * (kLaRows + 3) + sizeof(int) * ((size_t)b + 4) + 16;
}

// Send this CTA's outgoing record of parity `par` into slot [par][rank] of
// CTA q, completing on q's mbarrier of that parity.
__device__ __forceinline__ void la_send(const LaSmem& m, int par, int rank, int q) {
  const uint32_t src = tc::smem_u32(m.out + (size_t)par * m.rec);
  const uint32_t dst = tc::mapa_u32(tc::smem_u32(m.slot + ((size_t)par * 16 + rank) * m.rec), (uint32_t)q);
  const uint32_t bar = tc::mapa_u32(tc::smem_u32(&m.bar[par]), (uint32_t)q);
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   dst),
               "r"(src), "r"(m.rec), "r"(bar)
               : "memory");
}

__device__ __forceinline__ bool key_better(const LaKey& a, const LaKey& b) {
  return a.vbits > b.vbits || (a.vbits == b.vbits && a.row < b.row);
}

// The reciprocal without the range check of recip64 (the caller checks the
// winner's exponent): estimate r, e = 1 - v r, r (1 + e + e^2).
__device__ __forceinline__ double recip_core(double v) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(v));
  const double e = fma(-v, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// Local candidate of column cn from warp 0 (lane = local row): key and
// reciprocal, and the candidate's value x, into this CTA's outgoing record
// of column cn; local row into m.misc[0]. x = the lane's updated value,
// valid = the lane holds a row not yet used as a pivot.
__device__ __forceinline__ void la_pick(const LaSmem& m, int lane, double x, bool valid, int r0, int cn) {
  const unsigned long long ab =
      valid ? (static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull) : 0ull;
  const unsigned hi = static_cast<unsigned>(ab >> 32), lo = static_cast<unsigned>(ab);
  const double rr = recip_core(x);
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  const unsigned win = __reduce_min_sync(0xffffffffu, (valid && hi == mhi && lo == mlo) ? (unsigned)lane : 64u);
  unsigned char* o = m.out + (size_t)(cn & 1) * m.rec;
  LaKey* key = reinterpret_cast<LaKey*>(o);
  if (lane == 0 && win == 64u) {
    LaKey k;
    k.vbits = 0ull;
    k.row = INT_MAX;
    k.pad = 0;
    k.inv = 0.0;
    k.pad2 = 0.0;
    *key = k;
    m.misc[0] = -1;
  }
  if ((unsigned)lane == win) {
    LaKey k;
    k.vbits = ab;
    k.row = r0 + lane;
    k.pad = 0;
    const int ef = exp_field(x);
    k.inv = (ef >= 1 && ef <= 2044) ? rr : 1.0 / x;  // outside the normal range: the division
    k.pad2 = 0.0;
    *key = k;
    reinterpret_cast<double*>(o + 32)[cn] = x;  // the candidate row's element of column cn
    m.misc[0] = lane;
  }
}

// RT: a compile-time bound on the rows per CTA (4, 8 or 16), so that the
// bulk update is unrolled with its multipliers in registers.
template <int RT>
__global__ void __launch_bounds__(kPivotThreads, 1)
pivot_la_f64_kernel(const double* __restrict__ P, int64_t ldp, int b, double* __restrict__ out, int64_t ldo,
                    int32_t* status, int block_index) {
  // a kernel launched after this one as its programmatic dependent may start
  // now (it must not touch this block or its inverse)
  asm volatile("griddepcontrol.launch_dependents;");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  LaSmem m = la_layout(smem_raw, b);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int R = (b + C - 1) / C;  // rows per CTA (<= RT)
  const int r0 = rank * R;
  const int nloc = max(0, min(b, r0 + R) - r0);
  const bool col = tid < b;       // this thread updates column tid

  int bad = 0;
  if (col)
    for (int r = 0; r < nloc; ++r) {
      const double v = P[(int64_t)(r0 + r) * ldp + tid];
      if (nonfinite_bits(v)) bad = 1;
      m.rows[(size_t)r * b + tid] = v;
    }
  if (tid == 0) {
    m.misc[1] = (*(volatile const int32_t*)&status[0] != 0) ? 2 : 0;
    m.misc[2] = 0;
    tc::mbar_init(&m.bar[0], 1);
    tc::mbar_init(&m.bar[1], 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (bad) atomicOr(&m.misc[1], 1);
  // every CTA of the cluster is running, its mbarriers are initialised (peers
  // may send from here on) and its flags are set
  cl.sync();
  int flags = 0;
  for (int q = 0; q < C; ++q) flags |= *cl.map_shared_rank(&m.misc[1], q);
  if (flags) {
    // the same decision in every CTA: non-finite input, or an earlier kernel failed
    if ((flags & 1) && !(flags & 2) && rank == 0 && tid == 0)
      set_status(status, BLOCKINV_ERR_NONFINITE, block_index);
    cl.sync();
    return;
  }

  uint32_t used = 0;  // local rows already used as pivots (the same in every thread)
  // this CTA's record of column cn to every CTA, one bulk copy each from the
  // last warp (the other warps go on with the bulk of the step). The record
  // (key, candidate row) is complete: every thread has written its part and
  // ordered it for the async proxy before the CTA barrier that precedes this.
  constexpr int kSendWarp = kPivotThreads / 32 - 1;
  auto send = [&](int cn) {
    if (warp == kSendWarp && lane < C) la_send(m, cn & 1, rank, lane);
  };

  // column 0: candidates from the input itself
  if (tid == 0) tc::mbar_arrive_expect_tx(&m.bar[0], (uint32_t)(C * m.rec));
  if (warp == 0) {
    const double x = lane < nloc ? m.rows[(size_t)lane * b] : 0.0;
    la_pick(m, lane, x, lane < nloc, r0, 0);
  }
  __syncthreads();
  {
    const int rs = m.misc[0];
    if (col && tid != 0 && rs >= 0) reinterpret_cast<double*>(m.out + 32)[tid] = m.rows[(size_t)rs * b + tid];
  }
  tc::fence_proxy_async_smem();
  __syncthreads();
  send(0);
  int failed = 0;
  int* wi = reinterpret_cast<int*>(m.win + 1);  // [0] CTA of the pivot row, [1] its row, [2] failure (win[1..2])
  for (int c = 0; c < b; ++c) {
    const int par = c & 1;
    const int cn = c + 1;
    const bool ahead = cn < b;
    // the records of column c from every CTA (bounded wait; the same outcome
    // in every thread of the CTA)
    const bool arrived = tc::mbar_wait_for(&m.bar[par], (uint32_t)((c >> 1) & 1), tc::kWaitLimitNs);
    if (__syncthreads_or(!arrived)) {
      failed = BLOCKINV_ERR_TIMEOUT;
      break;
    }
    if (tid == 0 && ahead) tc::mbar_arrive_expect_tx(&m.bar[cn & 1], (uint32_t)(C * m.rec));
    if (warp == 0) {
      // the pivot of column c: the best key in this CTA's slots (lane q holds
      // CTA q's), by three warp reductions on the integer pipe: the largest
      // |value| bits (high word, then low word), then among those the lowest
      // row, with (row, CTA) packed as row * 16 + CTA (rows < 2^20)
      unsigned long long kv = 0ull;
      unsigned kp = 0xFFFFFFFFu;
      double kinv = 0.0;
      if (lane < C) {
        const LaKey k = *m.key(par, lane);
        kv = k.vbits;
        kp = k.row == INT_MAX ? 0xFFFFFFFFu : (static_cast<unsigned>(k.row) << 4) | static_cast<unsigned>(lane);
        kinv = k.inv;
      }
      const unsigned vhi = static_cast<unsigned>(kv >> 32), vlo = static_cast<unsigned>(kv);
      const unsigned mhi = __reduce_max_sync(0xffffffffu, vhi);
      const unsigned mlo = __reduce_max_sync(0xffffffffu, vhi == mhi ? vlo : 0u);
      kp = __reduce_min_sync(0xffffffffu, (vhi == mhi && vlo == mlo) ? kp : 0xFFFFFFFFu);
      kv = (static_cast<unsigned long long>(mhi) << 32) | mlo;
      const int kr = kp == 0xFFFFFFFFu ? INT_MAX : static_cast<int>(kp >> 4);
      const int ks = static_cast<int>(kp & 15u);
      const double inv = __shfl_sync(0xffffffffu, kinv, ks);
      int fail = 0;
      if (kr == INT_MAX || kv == 0ull)
        fail = BLOCKINV_ERR_SINGULAR;
      else if ((kv >> 52) >= 0x7FFull || nonfinite_bits(inv))
        fail = BLOCKINV_ERR_NONFINITE;
      if (lane == 0) {
        m.win[0] = inv;
        wi[0] = ks;
        wi[1] = kr;
        wi[2] = fail;
        if (!fail) m.perm[c] = kr;
      }
      if (!fail) {
        const int pl = kr - r0;
        const bool mine = pl >= 0 && pl < nloc;
        if (mine) used |= 1u << pl;
        const double* prow = m.row_of(par, ks);
        // multipliers: column c of the local rows before step c
        const double fl = lane < nloc ? m.rows[(size_t)lane * b + c] : 0.0;
        if (lane < nloc) m.fbuf[lane] = fl;
        if (ahead) {
          // step c on column cn (lane = row), then this CTA's candidate of column cn
          double x = 0.0;
          bool valid = false;
          if (lane < nloc) {
            double* e = m.rows + (size_t)lane * b + cn;
            const double sj = prow[cn] * inv;
            x = (mine && lane == pl) ? sj : fma(-fl, sj, *e);
            *e = x;
            valid = !((used >> lane) & 1u);
          }
          la_pick(m, lane, x, valid, r0, cn);
        }
      }
    }
    __syncthreads();  // the pivot, column cn, the candidate and the multipliers are in shared memory
    failed = wi[2];
    if (failed) break;  // the same in every CTA (the same keys); no copies in flight
    const int who = wi[0], p = wi[1];
    const double inv = m.win[0];
    const int pl = p - r0;
    const bool mine = pl >= 0 && pl < nloc;
    if (warp != 0 && mine) used |= 1u << pl;
    const double* prow = m.row_of(par, who);
    const int rs = ahead ? m.misc[0] : -1;
    // step c on element (r, tid): the pivot row is scaled, column c takes
    // -f inv, every other element x - f (P[p][tid] inv)
    const double sj = col ? ((tid == c) ? inv : prow[tid] * inv) : 0.0;
    if (ahead) {
      if (col && tid != cn && rs >= 0) {
        double* e = m.rows + (size_t)rs * b + tid;
        const double v = fma(-m.fbuf[rs], sj, tid == c ? 0.0 : *e);  // rs is never the pivot row
        *e = v;
        reinterpret_cast<double*>(m.out + (size_t)(cn & 1) * m.rec + 32)[tid] = v;
      }
      tc::fence_proxy_async_smem();
      __syncthreads();  // the record of column cn is complete
      send(cn);         // the copies fly while the bulk below runs
    }
    if (col && tid != cn) {
      // every element of the column first (one load each, all in flight), then
      // the FMAs and stores (row rs was done above; its load is harmless)
      double f[RT], x[RT];
#pragma unroll
      for (int r = 0; r < RT; ++r) {
        f[r] = m.fbuf[r];
        x[r] = r < nloc ? m.rows[(size_t)r * b + tid] : 0.0;
      }
      const bool zc = tid == c;  // column c drops its old value
#pragma unroll
      for (int r = 0; r < RT; ++r)
        if (r < nloc && r != rs)
          m.rows[(size_t)r * b + tid] = (mine && r == pl) ? sj : fma(-f[r], sj, zc ? 0.0 : x[r]);
    }
    // the CTA barrier after the next wait orders the bulk of step c before
    // warp 0 reads column c + 2
  }
  // every CTA is done with every slot and no copy is in flight (a timed-out
  // CTA may leave copies in flight only after a failure)
  cl.sync();
  if (failed) {  // the same code in every CTA, or a timeout in some (the first report wins)
    if (tid == 0) set_status(status, failed, block_index);
    return;
  }
  // unscramble: inverse[c][p_j] = a[p_c][j] for the step c at which row p_c was pivot
  if (col) {
    const int pj = m.perm[tid];
    for (int c = 0; c < b; ++c) {
      const int l = m.perm[c] - r0;
      if (l >= 0 && l < nloc) out[(int64_t)c * ldo + pj] = m.rows[(size_t)l * b + tid];
    }
  }
}

// ------------------------------------------------------------------------
// Panel-blocked variant for FP32 blocks of order 65..512. The columns are cut
// into panels of 32, dealt round-robin to the CTAs of a cluster (each CTA
// keeps its columns for all rows, column-major). For panel k, its owner runs
// the 32 Gauss-Jordan steps restricted to the panel's columns (partial
// pivoting over all unused rows; CTA barriers only). After one cluster
// barrier every CTA copies the panel and its 32 pivot rows and applies the
// combined effect of the 32 steps to its own other columns as one rank-32
// update:
//
//   P[r, j] <- (r a pivot row of the panel ? 0 : P[r, j]) + sum_l Panel[r, l] P_old[R_l, j]
//
// which equals performing the 32 steps on those columns. So a 256-block takes
// 8 cluster barriers instead of 256; the sequential column steps run inside
// one CTA.
constexpr int kPanel = 32;

template <typename T>
struct BlockedSmem {
  T* cols;      // ncl x b, column-major
  T* panel;     // kPanel x b, column-major: copy of the current panel
  T* pr;        // ncl x kPanel: old pivot rows restricted to my columns
  T* cand;      // 2 x 8 x kPanel: each warp's candidate pivot row (double-buffered by column)
  unsigned long long* key;  // 2 x 8 warp pivot keys (value bits, ~row), double-buffered by column
  int* perm;    // b: pivot row of each global column
  int* srow;    // b: column at which each row was the pivot (-1: not yet)
  unsigned char* inpanel;  // b
  int* flags;   // [0] non-finite seen, [1] singular, [2] non-finite pivot
};

template <typename T>
__device__ __forceinline__ BlockedSmem<T> blocked_layout(unsigned char* raw, int b, int ncl) {
  BlockedSmem<T> m;
  m.cols = reinterpret_cast<T*>(raw);
  m.panel = m.cols + (size_t)ncl * b;
  m.pr = m.panel + (size_t)kPanel * b;
  m.cand = m.pr + (size_t)ncl * kPanel;
  m.key = reinterpret_cast<unsigned long long*>(m.cand + 16 * kPanel);
  m.perm = reinterpret_cast<int*>(m.key + 16);
  m.srow = m.perm + b;
  m.flags = m.srow + b;
  m.inpanel = reinterpret_cast<unsigned char*>(m.flags + 4);
  return m;
}

template <typename T, bool kCluster>
__global__ void __launch_bounds__(kPivotThreads, 1)
pivot_blocked_kernel(const T* __restrict__ P, int64_t ldp, int b, int ncl, T* __restrict__ out, int64_t ldo,
                     int32_t* status, int block_index) {
  static_assert(sizeof(T) == 4, "the blocked pivot kernel serves the FP32 mixed path");
  // a kernel launched after this one as its programmatic dependent may start
  // now (it must not touch this block or its inverse)
  asm volatile("griddepcontrol.launch_dependents;");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BlockedSmem<T> m = blocked_layout<T>(smem_raw, b, ncl);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int rank = 0, nranks = 1;
  if constexpr (kCluster) {
    rank = (int)cg::this_cluster().block_rank();
    nranks = (int)cg::this_cluster().num_blocks();
  }
  const int npanels = (b + kPanel - 1) / kPanel;
  // load my panels' columns (rows read coalesced, stored column-major)
  int bad = 0;
  for (int k = rank, slot = 0; k < npanels; k += nranks, ++slot) {
    const int w = min(kPanel, b - k * kPanel);
    for (int e = tid; e < kPanel * b; e += kPivotThreads) {
      const int r = e / kPanel, l = e - r * kPanel;
      if (l < w) {
        const T v = P[(int64_t)r * ldp + k * kPanel + l];
        if (!isfinite(v)) bad = 1;
        m.cols[(size_t)(slot * kPanel + l) * b + r] = v;
      }
    }
  }
  for (int r = tid; r < b; r += kPivotThreads) {
    m.srow[r] = -1;
    m.inpanel[r] = 0;
  }
  if (tid < 4) m.flags[tid] = 0;
  __syncthreads();
  if (bad) atomicOr(&m.flags[0], 1);
  // an earlier kernel failed: bit 2, OR-ed over the cluster with the rest, so
  // that every CTA leaves here or none does (each CTA reads the status word
  // at its own time)
  if (tid == 0 && *(volatile int32_t*)&status[0] != 0) atomicOr(&m.flags[0], 2);
  cluster_or_block_sync<kCluster>();
  int anybad = 0;
  for (int q = 0; q < nranks; ++q) anybad |= *peer<kCluster>(&m.flags[0], q);
  if (anybad) {
    if (anybad == 1 && rank == 0 && tid == 0) set_status(status, BLOCKINV_ERR_NONFINITE, block_index);
    cluster_or_block_sync<kCluster>();
    return;
  }
  const int r0 = tid, r1 = tid + kPivotThreads;  // rows of this thread (b <= 512)
  int failed = 0;
  for (int k = 0; k < npanels; ++k) {
    const int owner = k % nranks, kslot = k / nranks;
    const int w = min(kPanel, b - k * kPanel);
    if (rank == owner) {
      // Gauss-Jordan on the panel's w columns with this thread's rows in
      // registers (x0: row r0, x1: row r1); two CTA barriers per column.
      T* pc = m.cols + (size_t)kslot * kPanel * b;
      T x0[kPanel], x1[kPanel];
#pragma unroll
      for (int l = 0; l < kPanel; ++l) {
        x0[l] = (l < w && r0 < b) ? pc[(size_t)l * b + r0] : T(0);
        x1[l] = (l < w && r1 < b) ? pc[(size_t)l * b + r1] : T(0);
      }
      bool free0 = r0 < b && m.srow[r0] < 0;
      bool free1 = r1 < b && m.srow[r1] < 0;
      bool stop = false;
      const bool two = b > kPivotThreads;  // a second row per thread only above 256 rows
      // One CTA barrier per column. Pivot search: |x| of a free row as its
      // FP32 bit pattern (ordered like the value; NaN above infinity) and the
      // row index form a 64-bit key (value, ~row): the largest key is the
      // largest magnitude, lowest row on ties. Each warp reduces its keys with
      // two redux operations and publishes its key and its candidate row's raw
      // values; after the barrier every thread takes the largest of the 8 keys
      // and reads the pivot row from the winner's slot. Keys and slots
      // alternate by column, so nothing is rewritten before its readers pass
      // the next barrier. Columns are taken four at a time in registers 0..3,
      // then the registers rotate by four (eight rotations restore the order).
#pragma unroll 1
      for (int cb = 0; cb < kPanel; cb += 4) {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int c = cb + cc;
          if (c < w && !stop) {
            const int buf = c & 1;
            unsigned vb = free0 ? __float_as_uint(fabsf(x0[cc])) : 0u;
            unsigned vi = static_cast<unsigned>(r0);
            if (two && free1) {
              const unsigned v1 = __float_as_uint(fabsf(x1[cc]));
              if (v1 > vb) {
                vb = v1;
                vi = static_cast<unsigned>(r1);
              }
            }
            const unsigned wmax = __reduce_max_sync(0xffffffffu, vb);
            const unsigned wrow = __reduce_min_sync(0xffffffffu, vb == wmax ? vi : 0xffffffffu);
            if (static_cast<int>(wrow) == r0 || static_cast<int>(wrow) == r1) {  // the warp's candidate row
              const bool h = static_cast<int>(wrow) == r1;
              float4* slot = reinterpret_cast<float4*>(m.cand + (buf * 8 + warp) * kPanel);
#pragma unroll
              for (int q = 0; q < kPanel / 4; ++q)
                slot[q] = h ? make_float4(x1[4 * q], x1[4 * q + 1], x1[4 * q + 2], x1[4 * q + 3])
                            : make_float4(x0[4 * q], x0[4 * q + 1], x0[4 * q + 2], x0[4 * q + 3]);
            }
            if (lane == 0)
              m.key[buf * 8 + warp] = (static_cast<unsigned long long>(wmax) << 32) | static_cast<unsigned>(~wrow);
            __syncthreads();
            unsigned long long kk;
            {
              const ulonglong2* kp = reinterpret_cast<const ulonglong2*>(m.key + buf * 8);
              const ulonglong2 k01 = kp[0], k23 = kp[1], k45 = kp[2], k67 = kp[3];
              const unsigned long long a = k01.x > k01.y ? k01.x : k01.y;
              const unsigned long long b2 = k23.x > k23.y ? k23.x : k23.y;
              const unsigned long long c2 = k45.x > k45.y ? k45.x : k45.y;
              const unsigned long long d = k67.x > k67.y ? k67.x : k67.y;
              const unsigned long long ab = a > b2 ? a : b2, cd = c2 > d ? c2 : d;
              kk = ab > cd ? ab : cd;
            }
            const float gv = __uint_as_float(static_cast<unsigned>(kk >> 32));
            const int p = static_cast<int>(~static_cast<unsigned>(kk));
            if (!(gv > 0.f) || !isfinite(gv)) {
              if (tid == 0) m.flags[!(gv > 0.f) && !isnan(gv) ? 1 : 2] = 1;
              stop = true;
            } else {
              const float* prow = m.cand + (buf * 8 + ((p & (kPivotThreads - 1)) >> 5)) * kPanel;
              float pr[kPanel];
#pragma unroll
              for (int q = 0; q < kPanel / 4; ++q) {
                const float4 v = reinterpret_cast<const float4*>(prow)[q];
                pr[4 * q] = v.x;
                pr[4 * q + 1] = v.y;
                pr[4 * q + 2] = v.z;
                pr[4 * q + 3] = v.w;
              }
              const float inv = recip_newton(pr[cc]);
              // pivot row: P[p][l] * inv (l != c), inv at l = c; every other
              // row: x[l] - (x[c] inv) P[p][l] (l != c), -x[c] inv at l = c
              if (r0 == p) {
                m.perm[k * kPanel + c] = p;
                m.srow[p] = k * kPanel + c;
#pragma unroll
                for (int l = 0; l < kPanel; ++l) x0[l] = (l == cc) ? inv : pr[l] * inv;
              } else {
                const float f0 = x0[cc] * inv;
#pragma unroll
                for (int l = 0; l < kPanel; ++l) x0[l] = (l == cc) ? -f0 : x0[l] - f0 * pr[l];
              }
              if (two) {
                if (r1 == p) {
                  m.perm[k * kPanel + c] = p;
                  m.srow[p] = k * kPanel + c;
#pragma unroll
                  for (int l = 0; l < kPanel; ++l) x1[l] = (l == cc) ? inv : pr[l] * inv;
                } else {
                  const float f1 = x1[cc] * inv;
#pragma unroll
                  for (int l = 0; l < kPanel; ++l) x1[l] = (l == cc) ? -f1 : x1[l] - f1 * pr[l];
                }
              }
              free0 = free0 && r0 != p;
              free1 = free1 && r1 != p;
            }
          }
        }
        // rotate by four: the next four columns move into registers 0..3
        {
          float t0[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) t0[u] = x0[u];
#pragma unroll
          for (int l = 0; l < kPanel - 4; ++l) x0[l] = x0[l + 4];
#pragma unroll
          for (int u = 0; u < 4; ++u) x0[kPanel - 4 + u] = t0[u];
          if (two) {
            float t1[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) t1[u] = x1[u];
#pragma unroll
            for (int l = 0; l < kPanel - 4; ++l) x1[l] = x1[l + 4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x1[kPanel - 4 + u] = t1[u];
          }
        }
      }
#pragma unroll
      for (int l = 0; l < kPanel; ++l) {
        if (l < w && r0 < b) pc[(size_t)l * b + r0] = x0[l];
        if (l < w && r1 < b) pc[(size_t)l * b + r1] = x1[l];
      }
      __syncthreads();
      if constexpr (kCluster) {
        // publish the panel through L2 for the other CTAs (see below)
        float4* xg = reinterpret_cast<float4*>(out + (size_t)(k & 1) * kPanel * b);
        const float4* pc4 = reinterpret_cast<const float4*>(pc);
        for (int e4 = tid; e4 < (w * b) / 4; e4 += kPivotThreads) xg[e4] = pc4[e4];
        for (int e = (w * b) / 4 * 4 + tid; e < w * b; e += kPivotThreads) out[(size_t)(k & 1) * kPanel * b + e] = pc[e];
      }
    }
    cluster_or_block_sync<kCluster>();
    // everyone: pivot rows and panel of step k from the owner. The flags, the
    // panel's pivot rows and the first (for b <= 256 the only) batch of the
    // panel are loaded together, so the remote reads cost one round trip. The
    // other CTAs read the panel from the copy the owner left in global memory
    // (the output buffer, free until the end; two alternating panel slots, so
    // a slot is rewritten only after every CTA has passed the next cluster
    // barrier): seven CTAs pulling it from the owner's shared memory at once
    // would queue on that one SM. The cluster barrier orders those writes
    // before these reads; the loads bypass L1, which may hold an older panel.
    {
      const int* rflags = peer<kCluster>(m.flags, owner);
      const int* rperm = peer<kCluster>(m.perm, owner);
      const bool via_l2 = kCluster && rank != owner;
      const float4* rpanel4 = via_l2 ? reinterpret_cast<const float4*>(out + (size_t)(k & 1) * kPanel * b)
                                     : reinterpret_cast<const float4*>(m.cols + (size_t)kslot * kPanel * b);
      const int n4 = (w * b) / 4;  // float4 part; a remainder of w * b % 4 floats follows
      constexpr int kPer = 8;      // float4 loads in flight per thread
      float4 v[kPer];
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int e4 = tid + q * kPivotThreads;
        if (e4 < n4) v[q] = via_l2 ? __ldcg(rpanel4 + e4) : rpanel4[e4];
      }
      const int f1 = rflags[1], f2 = rflags[2];
      const int rr = (tid < w) ? rperm[k * kPanel + tid] : 0;
      if (f1 || f2) {
        failed = f1 ? BLOCKINV_ERR_SINGULAR : BLOCKINV_ERR_NONFINITE;
        break;
      }
      if (tid < w) {
        m.perm[k * kPanel + tid] = rr;
        m.srow[rr] = k * kPanel + tid;
        m.inpanel[rr] = 1;
      }
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int e4 = tid + q * kPivotThreads;
        if (e4 < n4) reinterpret_cast<float4*>(m.panel)[e4] = v[q];
      }
      for (int base = kPer * kPivotThreads; base < n4; base += kPer * kPivotThreads) {
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
          const int e4 = base + tid + q * kPivotThreads;
          if (e4 < n4) v[q] = via_l2 ? __ldcg(rpanel4 + e4) : rpanel4[e4];
        }
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
          const int e4 = base + tid + q * kPivotThreads;
          if (e4 < n4) reinterpret_cast<float4*>(m.panel)[e4] = v[q];
        }
      }
      const float* rpanel = reinterpret_cast<const float*>(rpanel4);
      for (int e = n4 * 4 + tid; e < w * b; e += kPivotThreads) m.panel[e] = via_l2 ? __ldcg(rpanel + e) : rpanel[e];
    }
    __syncthreads();
    // old pivot rows in my columns outside the panel
    const int my_cols = ncl;
    for (int e = tid; e < my_cols * kPanel; e += kPivotThreads) {
      const int lc = e / kPanel, l = e - lc * kPanel;
      m.pr[e] = (l < w) ? m.cols[(size_t)lc * b + m.perm[k * kPanel + l]] : T(0);
    }
    __syncthreads();
    // rank-w update of my columns (skipping the panel itself on the owner),
    // four columns per pass so that four accumulator chains run side by side
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int r = h ? r1 : r0;
      if (r >= b) continue;
      T pv[kPanel];
#pragma unroll
      for (int l = 0; l < kPanel; ++l) pv[l] = (l < w) ? m.panel[(size_t)l * b + r] : T(0);
      const bool piv_row = m.inpanel[r] != 0;
      for (int lp = 0; lp < ncl / kPanel; ++lp) {
        const int gk = lp * nranks + rank;  // global panel of my local panel lp
        if (gk >= npanels || (rank == owner && gk == k)) continue;
        const int wg = min(kPanel, b - gk * kPanel);
        for (int c0 = 0; c0 < wg; c0 += 4) {
          const int lc = lp * kPanel + c0;
          T acc[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            acc[u] = (piv_row || c0 + u >= wg) ? T(0) : m.cols[(size_t)(lc + u) * b + r];
          const T* prc = m.pr + (size_t)lc * kPanel;
          if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int q = 0; q < kPanel / 4; ++q) {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float4 v = reinterpret_cast<const float4*>(prc + u * kPanel)[q];
                acc[u] += pv[4 * q] * v.x + pv[4 * q + 1] * v.y + pv[4 * q + 2] * v.z + pv[4 * q + 3] * v.w;
              }
            }
          } else {
#pragma unroll
            for (int l = 0; l < kPanel; ++l)
#pragma unroll
              for (int u = 0; u < 4; ++u) acc[u] += pv[l] * prc[u * kPanel + l];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (c0 + u < wg) m.cols[(size_t)(lc + u) * b + r] = acc[u];
        }
      }
    }
    __syncthreads();
    if (tid < w) m.inpanel[m.perm[k * kPanel + tid]] = 0;
    __syncthreads();
  }
  // after this barrier nobody reads another CTA's shared memory
  cluster_or_block_sync<kCluster>();
  if (failed) {
    if (rank == 0 && tid == 0) set_status(status, failed, block_index);
    return;
  }
  for (int k = rank, slot = 0; k < npanels; k += nranks, ++slot) {
    const int w = min(kPanel, b - k * kPanel);
    for (int l = 0; l < w; ++l) {
      const int gc = k * kPanel + l;
      const T* col = m.cols + (size_t)(slot * kPanel + l) * b;
      for (int r = tid; r < b; r += kPivotThreads) out[(int64_t)m.srow[r] * ldo + m.perm[gc]] = col[r];
    }
  }
}

size_t blocked_smem_bytes(int b, int ncl, int elem) {
  return (size_t)elem * ((size_t)ncl * b + (size_t)kPanel * b + (size_t)ncl * kPanel + 16 * kPanel) +
         sizeof(unsigned long long) * 16 + sizeof(int) * (2 * (size_t)b + 4) + b + 64;
}

// Cluster size for the blocked kernel: one 32-column panel per CTA where
// possible (the rank updates of each panel step then run on as many SMs as
// there are panels), at most 8 CTAs, more panels per CTA only when needed;
// each CTA's columns must fit in 225 KiB of shared memory.
bool plan_blocked(int b, int elem, int* ctas, int* ncl, size_t* smem) {
  const int npanels = (b + kPanel - 1) / kPanel;
  int c0 = 1;
  while (c0 < npanels && c0 < 8) c0 *= 2;
  for (int c = c0; c <= 8; c *= 2) {
    const int per = (npanels + c - 1) / c;
    const size_t bytes = blocked_smem_bytes(b, per * kPanel, elem);
    if (bytes <= 225 * 1024) {
      *ctas = c;
      *ncl = per * kPanel;
      *smem = bytes;
      return true;
    }
  }
  return false;
}

size_t pivot_smem_bytes(int b, int R, int elem) {
  size_t t = (size_t)R * b + b + R + 2;            // T arrays
  size_t i = 2 + (size_t)R + b + 1;                // int arrays
  return t * elem + i * sizeof(int) + 16;
}

// Kernel attributes are per device; the largest shared-memory size set so far
// for each instantiation and device is remembered, so the attribute calls run
// only when a launch needs more.
template <typename T, typename TIO, bool kCluster>
cudaError_t configure(size_t smem) {
  static std::mutex mu;
  static size_t done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  if (dev >= 0 && dev < 64 && done[dev] >= smem) return cudaSuccess;
  auto k = pivot_gj_kernel<T, TIO, kCluster>;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if constexpr (kCluster) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = smem;
  return e;
}

}  // namespace

bool plan_pivot(int b, int elem_bytes, PivotPlan* plan) {
  if (b < 1 || b > BLOCKINV_MAX_BLOCK) return false;
  int R, C;
  if (b <= 64) {
    R = b;
    C = 1;
  } else {
    R = 32;
    C = (b + R - 1) / R;
    if (C > 16) {
      R = (b + 15) / 16;
      C = (b + R - 1) / R;
    }
  }
  size_t smem = pivot_smem_bytes(b, R, elem_bytes);
  if (smem > 227 * 1024) return false;
  plan->b = b;
  plan->rows = R;
  plan->ctas = C;
  plan->smem = smem;
  return true;
}

// The dynamic shared-memory attribute of kernel K, set only when a launch on
// this device needs more than was set before (one record per kernel).
template <auto K>
cudaError_t set_smem_once(size_t smem) {
  static std::mutex mu;
  static size_t done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  if (dev >= 0 && dev < 64 && done[dev] >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = smem;
  return e;
}

template <typename T>
cudaError_t launch_pivot_blocked(const T* P, int64_t ldp, int b, T* Pinv, int64_t ldo, int32_t* status,
                                 int block_index, cudaStream_t s, bool* done) {
  *done = false;
  int ctas = 0, ncl = 0;
  size_t smem = 0;
  if (!plan_blocked(b, (int)sizeof(T), &ctas, &ncl, &smem)) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas, 1, 1);
  cfg.blockDim = dim3(kPivotThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  cudaError_t e;
  if (ctas > 1) {
    auto k = pivot_blocked_kernel<T, true>;
    e = set_smem_once<pivot_blocked_kernel<T, true>>(smem);
    if (e != cudaSuccess) return e;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k, P, ldp, b, ncl, Pinv, ldo, status, block_index);
  } else {
    auto k = pivot_blocked_kernel<T, false>;
    e = set_smem_once<pivot_blocked_kernel<T, false>>(smem);
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernelEx(&cfg, k, P, ldp, b, ncl, Pinv, ldo, status, block_index);
  }
  *done = (e == cudaSuccess);
  return e;
}

// Row-distributed Gauss-Jordan (pivot_gj_kernel) in arithmetic T on blocks of
// type TIO, optionally gated.
template <typename T, typename TIO>
cudaError_t launch_gj(const TIO* P, int64_t ldp, int b, TIO* Pinv, int64_t ldo, int32_t* status, int block_index,
                      const int32_t* gate, cudaStream_t s) {
  PivotPlan plan;
  if (!plan_pivot(b, (int)sizeof(T), &plan)) return cudaErrorInvalidValue;
  int jw = 1, jlog = 0;
  while (jw < b && jw < kPivotThreads) {
    jw <<= 1;
    ++jlog;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(plan.ctas, 1, 1);
  cfg.blockDim = dim3(kPivotThreads, 1, 1);
  cfg.dynamicSmemBytes = plan.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (plan.ctas > 1) {
    cudaError_t e = configure<T, TIO, true>(plan.smem);
    if (e != cudaSuccess) return e;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan.ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pivot_gj_kernel<T, TIO, true>, P, ldp, b, plan.rows, jlog, Pinv, ldo, status,
                              block_index, gate);
  }
  cudaError_t e = configure<T, TIO, false>(plan.smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, pivot_gj_kernel<T, TIO, false>, P, ldp, b, plan.rows, jlog, Pinv, ldo, status,
                            block_index, gate);
}

// Cluster size of the look-ahead FP64 kernel: at most kLaRows rows per CTA,
// about 8 rows per CTA for small blocks (shorter column steps), at most 16.
int la_ctas(int b) {
  int c = (b + 7) / 8;
  if (c > 16) c = 16;
  while ((b + c - 1) / c > kLaRows) ++c;
  return c;
}

template <int RT>
cudaError_t launch_pivot_la_rt(const double* P, int64_t ldp, int b, int C, double* Pinv, int64_t ldo,
                               int32_t* status, int block_index, cudaStream_t s) {
  const size_t smem = la_smem_bytes(b);
  cudaError_t e = set_smem_once<pivot_la_f64_kernel<RT>>(smem);
  if (e != cudaSuccess) return e;
  if (C > 8) {  // clusters above the portable 8 CTAs, allowed once per device
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64 || !done[dev]) {
      e = cudaFuncSetAttribute(pivot_la_f64_kernel<RT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
      if (dev >= 0 && dev < 64) done[dev] = true;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(kPivotThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, pivot_la_f64_kernel<RT>, P, ldp, b, Pinv, ldo, status, block_index);
}

cudaError_t launch_pivot_la(const double* P, int64_t ldp, int b, double* Pinv, int64_t ldo, int32_t* status,
                            int block_index, cudaStream_t s) {
  const int C = la_ctas(b);
  if (C > 16 || b > kLaMaxB) return cudaErrorInvalidValue;
  const int R = (b + C - 1) / C;
  if (R <= 4) return launch_pivot_la_rt<4>(P, ldp, b, C, Pinv, ldo, status, block_index, s);
  if (R <= 8) return launch_pivot_la_rt<8>(P, ldp, b, C, Pinv, ldo, status, block_index, s);
  return launch_pivot_la_rt<16>(P, ldp, b, C, Pinv, ldo, status, block_index, s);
}

template <typename T>
cudaError_t launch_pivot_inverse(const T* P, int64_t ldp, int b, T* Pinv, int64_t ldo,
                                 int32_t* status, int block_index, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    if (b <= kLaMaxB) return launch_pivot_la(P, ldp, b, Pinv, ldo, status, block_index, s);
  }
  if constexpr (sizeof(T) == 4) {
    if (b > 64) {
      bool done = false;
      cudaError_t e = launch_pivot_blocked<T>(P, ldp, b, Pinv, ldo, status, block_index, s, &done);
      if (e != cudaSuccess || done) return e;
    }
  }
  return launch_gj<T, T>(P, ldp, b, Pinv, ldo, status, block_index, nullptr, s);
}

cudaError_t launch_pivot_cond(const float* P, int64_t ldp, int b, const float* Pinv, int64_t ldo,
                              const int32_t* status, float cond_limit, int32_t* gate, int32_t* count,
                              bool after_trigger, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1, 1, 1);
  cfg.blockDim = dim3(kCondThreads, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = after_trigger ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, pivot_cond_kernel, P, ldp, Pinv, ldo, b, cond_limit, gate, count, status);
}

cudaError_t launch_pivot_f64_gated(const float* P, int64_t ldp, int b, float* Pinv, int64_t ldo, int32_t* status,
                                   int block_index, const int32_t* gate, cudaStream_t s) {
  return launch_gj<double, float>(P, ldp, b, Pinv, ldo, status, block_index, gate, s);
}


int pivot_inverse_ctas(int b, int elem, bool f64_check) {
  int c = 1, ctas = 0, ncl = 0;
  size_t smem = 0;
  PivotPlan plan;
  if (elem == 8 && b <= kLaMaxB)
    c = la_ctas(b);
  else if (elem == 4 && b > 64 && plan_blocked(b, elem, &ctas, &ncl, &smem))
    c = ctas;
  else if (plan_pivot(b, elem, &plan))
    c = plan.ctas;
  if (f64_check && plan_pivot(b, (int)sizeof(double), &plan)) c = std::max(c, plan.ctas);
  return c;
}

cudaError_t launch_pivot_grouped(const GroupStep* items, int count, int bmax, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (bmax > kGroupedMaxB) return cudaErrorInvalidValue;
  const size_t smem = grouped_pivot_smem(bmax);
  // blocks of order <= 32: one warp each; larger ones: one CTA each
  pivot_warp_grouped_kernel<<<(count + 3) / 4, 128, 0, s>>>(items, count);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || bmax <= kWarpPivotMax) return e;
  e = cudaFuncSetAttribute(pivot_gj_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  pivot_gj_grouped_kernel<<<count, kPivotThreads, smem, s>>>(items, count, kWarpPivotMax);
  return cudaGetLastError();
}

template cudaError_t launch_pivot_inverse<double>(const double*, int64_t, int, double*, int64_t,
                                                  int32_t*, int, cudaStream_t);
template cudaError_t launch_pivot_inverse<float>(const float*, int64_t, int, float*, int64_t,
                                                 int32_t*, int, cudaStream_t);

}  // namespace blockinv
