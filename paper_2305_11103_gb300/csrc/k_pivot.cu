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
#include <climits>
#include <cooperative_groups.h>

#include "internal.h"

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

template <typename T>
__device__ __forceinline__ void argmax_step(T& bv, int& bi, T ov, int oi) {
  if (ov > bv || (ov == bv && oi < bi)) {
    bv = ov;
    bi = oi;
  }
}

template <typename T, bool kCluster>
__device__ __forceinline__ void pivot_gj_body(const T* __restrict__ P, int64_t ldp, int b, int R, int jlog,
                                              T* __restrict__ out, int64_t ldo, int32_t* status,
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
      T v = P[(int64_t)(r0 + r) * ldp + j];
      if (!isfinite(v)) bad = 1;
      rows[(size_t)r * b + j] = v;
    }
  }
  if (bad) atomicOr(&flags[0], 1);
  // Skip everything if an earlier kernel of this inversion already failed.
  const int prior = *(volatile int32_t*)&status[0];
  cluster_or_block_sync<kCluster>();
  int anybad = 0;
  for (int q = 0; q < nranks; ++q) anybad |= *peer<kCluster>(&flags[0], q);
  if (anybad || prior != 0) {
    if (anybad && prior == 0 && rank == 0 && tid == 0)
      set_status(status, BLOCKINV_ERR_NONFINITE, block_index);
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
    const T piv = prem[c];
    for (int j = tid; j < b; j += kPivotThreads) prow[j] = (j == c) ? T(1) / piv : prem[j] / piv;
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
    for (int j = jj; j < b; j += jw) out[(int64_t)i * ldo + perm[j]] = row[j];
  }
}

template <typename T, bool kCluster>
__global__ void __launch_bounds__(kPivotThreads)
pivot_gj_kernel(const T* __restrict__ P, int64_t ldp, int b, int R, int jlog, T* __restrict__ out, int64_t ldo,
                int32_t* status, int block_index) {
  pivot_gj_body<T, kCluster>(P, ldp, b, R, jlog, out, ldo, status, block_index);
}

// Grouped form: one CTA per matrix of a batch, block order <= kGroupedMaxB,
// every row of the pivot block in the CTA's shared memory.
__global__ void __launch_bounds__(kPivotThreads)
pivot_gj_grouped_kernel(const GroupStep* __restrict__ items, int count) {
  const int m = blockIdx.x;
  if (m >= count) return;
  const GroupStep it = items[m];
  if (it.b > kGroupedMaxB) return;  // handled by the cluster kernel
  int jw = 1, jlog = 0;
  while (jw < it.b && jw < kPivotThreads) {
    jw <<= 1;
    ++jlog;
  }
  pivot_gj_body<double, false>(it.X + (int64_t)it.o * it.ldx + it.o, it.ldx, it.b, it.b, jlog, it.Pinv, it.b,
                               it.status, it.k);
}

size_t pivot_smem_bytes(int b, int R, int elem) {
  size_t t = (size_t)R * b + b + R + 2;            // T arrays
  size_t i = 2 + (size_t)R + b + 1;                // int arrays
  return t * elem + i * sizeof(int) + 16;
}

template <typename T, bool kCluster>
cudaError_t configure(size_t smem) {
  auto k = pivot_gj_kernel<T, kCluster>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if constexpr (kCluster) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
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

template <typename T>
cudaError_t launch_pivot_inverse(const T* P, int64_t ldp, int b, T* Pinv, int64_t ldo,
                                 int32_t* status, int block_index, cudaStream_t s) {
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
    cudaError_t e = configure<T, true>(plan.smem);
    if (e != cudaSuccess) return e;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan.ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pivot_gj_kernel<T, true>, P, ldp, b, plan.rows, jlog, Pinv, ldo,
                              status, block_index);
  }
  cudaError_t e = configure<T, false>(plan.smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, pivot_gj_kernel<T, false>, P, ldp, b, plan.rows, jlog, Pinv, ldo,
                            status, block_index);
}

cudaError_t launch_pivot_grouped(const GroupStep* items, int count, int bmax, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (bmax > kGroupedMaxB) return cudaErrorInvalidValue;
  const size_t smem = pivot_smem_bytes(bmax, bmax, sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(pivot_gj_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  pivot_gj_grouped_kernel<<<count, kPivotThreads, smem, s>>>(items, count);
  return cudaGetLastError();
}

template cudaError_t launch_pivot_inverse<double>(const double*, int64_t, int, double*, int64_t,
                                                  int32_t*, int, cudaStream_t);
template cudaError_t launch_pivot_inverse<float>(const float*, int64_t, int, float*, int64_t,
                                                 int32_t*, int, cudaStream_t);

}  // namespace blockinv
