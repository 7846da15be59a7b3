// Batched inversion of many matrices of one order n <= 32 with one partition,
// FP64: the paper's motivating workload beyond 5 x 5 (Sec. 2: 11 x 11
// systematics matrices split into blocks of 5 and 6), and in general any order
// up to 32 with the paper's Table 2 partition or the caller's.
//
// A segment of NMAX lanes (16 or 32) holds one matrix, one row per lane in
// registers. Eq. (a) is applied one block at a time, in block order: the
// pivot block's Gauss-Jordan elimination, column by column with the pivot
// row searched among the block's rows only (partial pivoting inside the
// block), where each row operation is applied to whole rows. On the block's
// rows this forms P^-1 X[k, :] (the row panel); on every other row it forms
// the Schur complement S = D - C P^-1 B and the column panel -C P^-1. The
// pivot row is broadcast with warp shuffles of the segment. Rows are not
// swapped: each lane remembers the column it was pivot for, and the result
// is unscrambled on the way out.
//
// With BLOCKINV_BATCH_SPD the input is taken as symmetric positive definite:
// every pivot block and Schur complement is then SPD, so the diagonal pivots
// are used without a search, and the result is made exactly symmetric (the
// upper triangle is mirrored).
//
// Memory: a CTA of 128 threads stages its consecutive matrices through shared
// memory, so global loads and stores are coalesced. A matrix with a zero or
// non-finite pivot (or a non-finite entry) gets BLOCKINV_ERR_SINGULAR /
// BLOCKINV_ERR_NONFINITE in its status word and is left unchanged.
#include <climits>
#include <vector>

#include "internal.h"

namespace blockinv {

namespace {

constexpr int kTinyThreads = 128;
constexpr int kTinyMax = 32;

struct TinyPartition {
  int n;
  int col_o[kTinyMax];  // offset of the block that holds column c
  int col_b[kTinyMax];  // its order
};

template <int NMAX>
__global__ void __launch_bounds__(kTinyThreads)
tiny_batched_kernel(double* __restrict__ A, int64_t count, TinyPartition part, int spd, int32_t* __restrict__ status) {
  constexpr int MPC = kTinyThreads / NMAX;  // matrices per CTA
  extern __shared__ double stage[];          // MPC x n x n
  __shared__ int seg_state[MPC];             // 0 ok, else the error status
  const int n = part.n;
  const int nn = n * n;
  const int64_t m0 = (int64_t)blockIdx.x * MPC;
  const int tid = threadIdx.x;
  const int seg = tid / NMAX, lane = tid % NMAX;
  const int64_t nmat = min((int64_t)MPC, count - m0);
  const bool live = seg < nmat;
  const double* src = A + m0 * nn;
  for (int e = tid; e < nmat * nn; e += kTinyThreads) stage[e] = src[e];
  if (tid < MPC) seg_state[tid] = 0;
  __syncthreads();

  const bool row_ok = live && lane < n;
  double* mine = stage + (size_t)seg * nn;
  double x[NMAX];
  bool nonfinite = false;
#pragma unroll
  for (int l = 0; l < NMAX; ++l) {
    x[l] = (row_ok && l < n) ? mine[lane * n + l] : 0.0;
    nonfinite |= !isfinite(x[l]);
  }
  // a non-finite entry anywhere in this segment's matrix
  const unsigned bits = __ballot_sync(0xffffffffu, nonfinite);
  const unsigned segmask = (NMAX == 32) ? 0xffffffffu : (0xffffu << (tid & 16));
  int err = (bits & segmask) ? BLOCKINV_ERR_NONFINITE : 0;
  bool used = false;  // this lane's row has been a pivot row
  int my_col = -1;    // the column it was pivot for
  int perm[NMAX];     // pivot row of each column (the same in every lane of the segment)
#pragma unroll
  for (int c = 0; c < NMAX; ++c) {
    perm[c] = c;
    if (c < n) {
      const int o = part.col_o[c], b = part.col_b[c];
      int pr = c;  // SPD: the diagonal pivot
      bool found = true;
      if (!spd) {
        // pivot search among the block's rows not yet used: |x| as its bit
        // pattern (non-negative doubles order like their bits; NaN above
        // infinity), compared on the integer pipe, lowest row on ties
        const bool cand = row_ok && !used && lane >= o && lane < o + b;
        unsigned long long key = cand ? static_cast<unsigned long long>(__double_as_longlong(fabs(x[c]))) : 0ull;
        int idx = cand ? lane : NMAX;
#pragma unroll
        for (int off = NMAX / 2; off > 0; off >>= 1) {
          const unsigned long long ok2 = __shfl_xor_sync(0xffffffffu, key, off, NMAX);
          const int oi = __shfl_xor_sync(0xffffffffu, idx, off, NMAX);
          if (ok2 > key || (ok2 == key && oi < idx)) {
            key = ok2;
            idx = oi;
          }
        }
        found = idx < NMAX;
        pr = found ? idx : 0;
      }
      perm[c] = pr;
      const double pc = __shfl_sync(0xffffffffu, x[c], pr, NMAX);
      if (err == 0 && live) {
        if (!found || pc == 0.0) err = BLOCKINV_ERR_SINGULAR;
        else if (!isfinite(pc)) err = BLOCKINV_ERR_NONFINITE;
      }
      const double inv = (err == 0) ? 1.0 / pc : 0.0;
      const bool is_pivot = lane == pr;
      // every row: x[l] += alpha P[p][l] (l != c), with the pivot row first
      // cleared and alpha = inv there, alpha = -x[c] inv elsewhere; x[c] gets
      // inv on the pivot row and -x[c] inv elsewhere
      const double alpha = is_pivot ? inv : -x[c] * inv;
#pragma unroll
      for (int l = 0; l < NMAX; ++l) {
        const double pl = __shfl_sync(0xffffffffu, x[l], pr, NMAX);  // pivot row, before this column's update
        if (l < n) x[l] = (l == c) ? alpha : fma(alpha, pl, is_pivot ? 0.0 : x[l]);
      }
      if (is_pivot) {
        used = true;
        my_col = c;
      }
    }
  }
  if (err != 0 && live && lane == 0) seg_state[seg] = err;
  __syncthreads();
  const bool ok = live && seg_state[seg] == 0;
  // unscramble: row my_col of the inverse gets x[j] at column perm[j]
  if (ok && lane < n) {
#pragma unroll
    for (int j = 0; j < NMAX; ++j)
      if (j < n) mine[my_col * n + perm[j]] = x[j];
  }
  __syncthreads();
  if (spd && ok) {  // exact symmetry: the upper triangle wins
    for (int e = lane; e < nn; e += NMAX) {
      const int i = e / n, j = e - i * n;
      if (i > j) mine[e] = mine[j * n + i];
    }
  }
  __syncthreads();
  double* dst = A + m0 * nn;
  for (int e = tid; e < nmat * nn; e += kTinyThreads)
    if (seg_state[e / nn] == 0) dst[e] = stage[e];
  if (status && live && lane == 0) status[m0 + seg] = seg_state[seg];
}

template <int NMAX>
cudaError_t launch_tiny(const TinyPartition& part, bool spd, double* A, int64_t count, int32_t* status,
                        cudaStream_t s) {
  constexpr int MPC = kTinyThreads / NMAX;
  const int64_t blocks = (count + MPC - 1) / MPC;
  const size_t smem = sizeof(double) * MPC * part.n * part.n;
  tiny_batched_kernel<NMAX><<<(unsigned)blocks, kTinyThreads, smem, s>>>(A, count, part, spd ? 1 : 0, status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tiny_batched(int n, const std::vector<int>& sizes, bool spd, double* A, int64_t count,
                                int32_t* status, cudaStream_t s) {
  if (n < 1 || n > kTinyMax || count < 1 || count >= (int64_t)INT32_MAX * 4) return cudaErrorInvalidValue;
  TinyPartition part{};
  part.n = n;
  int o = 0;
  for (int b : sizes) {
    if (b < 1 || o + b > n) return cudaErrorInvalidValue;
    for (int c = o; c < o + b; ++c) {
      part.col_o[c] = o;
      part.col_b[c] = b;
    }
    o += b;
  }
  if (o != n) return cudaErrorInvalidValue;
  return n <= 16 ? launch_tiny<16>(part, spd, A, count, status, s) : launch_tiny<32>(part, spd, A, count, status, s);
}

}  // namespace blockinv
