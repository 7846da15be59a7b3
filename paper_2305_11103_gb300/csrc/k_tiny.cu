// Batched inversion of many matrices of one order n <= 32 with one partition,
// FP64: the paper's motivating workload beyond 5 x 5 (Sec. 2: 11 x 11
// systematics matrices split into blocks of 5 and 6), and in general any order
// up to 32 with the paper's Table 2 partition or the caller's.
//
// A group of L lanes holds one matrix, R rows per lane in registers (row
// r = lane + L s, s < R; L R >= n, chosen per order so that few slots idle:
// 11 x 11 is 4 lanes x 3 rows). Eq. (a) is applied one block at a time, in
// block order: the pivot block's Gauss-Jordan elimination, column by column
// with the pivot row searched among the block's rows only (partial pivoting
// inside the block), where each row operation is applied to whole rows. On the
// block's rows this forms P^-1 X[k, :] (the row panel); on every other row it
// forms the Schur complement S = D - C P^-1 B and the column panel -C P^-1.
// The pivot row is broadcast with warp shuffles inside the group. Rows are not
// swapped: each row remembers the column it was pivot for, and the result is
// unscrambled on the way out.
//
// Cost model: on this GPU a warp's FP64 instruction occupies the SM's FP64
// pipe for 16 clocks, so the kernel counts FP64 instructions: per column and
// lane R L-padded row updates of n fused multiply-adds, R products for the
// multipliers and one reciprocal of the pivot (a hardware estimate and one
// third-order correction, 3 FMAs, instead of a division). Finiteness and zero
// tests look at bit patterns on the integer pipe.
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

#include "fp64_ops.cuh"
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

template <int L, int R, bool kSPD>
__global__ void __launch_bounds__(kTinyThreads)
tiny_batched_kernel(double* __restrict__ A, int64_t count, TinyPartition part, int32_t* __restrict__ status) {
  constexpr int NC = L * R;                  // row slots (>= n)
  constexpr int MPC = kTinyThreads / L;      // matrices per CTA
  extern __shared__ double stage[];          // MPC x n x n
  __shared__ int seg_state[MPC];             // 0 ok, else the error status
  const int n = part.n;
  const int nn = n * n;
  const int64_t m0 = (int64_t)blockIdx.x * MPC;
  const int tid = threadIdx.x;
  const int seg = tid / L, gl = tid % L;
  const int wbase = (tid & 31) - gl;         // the group's first lane in the warp
  const int64_t nmat = min((int64_t)MPC, count - m0);
  const bool live = seg < nmat;
  const double* src = A + m0 * nn;
  for (int e = tid; e < nmat * nn; e += kTinyThreads) stage[e] = src[e];
  if (tid < MPC) seg_state[tid] = 0;
  __syncthreads();

  double* mine = stage + (size_t)seg * nn;
  double x[R][NC];
  bool nonfinite = false;
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int r = gl + L * s;
#pragma unroll
    for (int l = 0; l < NC; ++l) {
      x[s][l] = (live && r < n && l < n) ? mine[r * n + l] : 0.0;
      nonfinite |= exp_field(x[s][l]) == 0x7FF;
    }
  }
  // a non-finite entry anywhere in this group's matrix
  const unsigned bits = __ballot_sync(0xffffffffu, nonfinite);
  const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << wbase);
  int err = (bits & gmask) ? BLOCKINV_ERR_NONFINITE : 0;
  bool used[R];       // the row in slot s has been a pivot row
  int my_col[R];      // the column it was pivot for
#pragma unroll
  for (int s = 0; s < R; ++s) {
    used[s] = false;
    my_col[s] = -1;
  }
  int perm[NC];       // pivot row of each column (the same in every lane of the group)
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    perm[c] = c;
    if (c < n) {
      int pr = c;  // SPD: the diagonal pivot
      bool found = true;
      if constexpr (!kSPD) {
        // pivot search among the block's rows not yet used: candidates carry
        // the top bit above |x| as its bit pattern (non-negative doubles order
        // like their bits; NaN above infinity), lowest row on ties
        const int o = part.col_o[c], b = part.col_b[c];
        unsigned long long key = 0ull;
        int idx = NC;
#pragma unroll
        for (int s = 0; s < R; ++s) {
          const int r = gl + L * s;
          const bool cand = live && r < n && !used[s] && r >= o && r < o + b;
          const unsigned long long k =
              cand ? (static_cast<unsigned long long>(__double_as_longlong(fabs(x[s][c]))) | (1ull << 63)) : 0ull;
          if (k > key) {
            key = k;
            idx = r;
          }
        }
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1) {
          const unsigned long long ok2 = __shfl_xor_sync(0xffffffffu, key, off, L);
          const int oi = __shfl_xor_sync(0xffffffffu, idx, off, L);
          if (ok2 > key || (ok2 == key && oi < idx)) {
            key = ok2;
            idx = oi;
          }
        }
        found = (key >> 63) != 0;
        pr = found ? idx : c;
      }
      perm[c] = pr;
      const int owner = pr % L, slot = pr / L;
      double pv = x[0][c];
#pragma unroll
      for (int s = 1; s < R; ++s)
        if (slot == s) pv = x[s][c];
      const double pc = __shfl_sync(0xffffffffu, pv, wbase + owner);
      if (err == 0 && live) {  // compared on the integer pipe
        const unsigned long long pb = static_cast<unsigned long long>(__double_as_longlong(pc));
        if (!found || (pb << 1) == 0ull) err = BLOCKINV_ERR_SINGULAR;
        else if (exp_field(pc) == 0x7FF) err = BLOCKINV_ERR_NONFINITE;
      }
      const double inv = (err == 0) ? recip64(pc) : 0.0;
      // every row: x[l] += alpha P[p][l] (l != c), with the pivot row first
      // cleared and alpha = inv there, alpha = -x[c] inv elsewhere; x[c] gets
      // inv on the pivot row and -x[c] inv elsewhere
      bool piv[R];
      double alpha[R];
#pragma unroll
      for (int s = 0; s < R; ++s) {
        piv[s] = gl == owner && s == slot;
        alpha[s] = piv[s] ? inv : -x[s][c] * inv;
      }
      // columns past n: a uniform branch out, since predicated-off FP64
      // instructions still occupy this GPU's FP64 pipe (measured)
#pragma unroll
      for (int l = 0; l < NC; ++l) {
        if (l >= n) break;
        double v = x[0][l];
#pragma unroll
        for (int s = 1; s < R; ++s)
          if (slot == s) v = x[s][l];
        const double pl = __shfl_sync(0xffffffffu, v, wbase + owner);  // pivot row, before this column's update
#pragma unroll
        for (int s = 0; s < R; ++s) x[s][l] = (l == c) ? alpha[s] : fma(alpha[s], pl, piv[s] ? 0.0 : x[s][l]);
      }
#pragma unroll
      for (int s = 0; s < R; ++s)
        if (piv[s]) {
          used[s] = true;
          my_col[s] = c;
        }
    }
  }
  if (err != 0 && live && gl == 0) seg_state[seg] = err;
  __syncthreads();
  const bool ok = live && seg_state[seg] == 0;
  // unscramble: row my_col of the inverse gets x[j] at column perm[j]
  if (ok) {
#pragma unroll
    for (int s = 0; s < R; ++s) {
      if (gl + L * s >= n) continue;
#pragma unroll
      for (int j = 0; j < NC; ++j)
        if (j < n) mine[my_col[s] * n + perm[j]] = x[s][j];
    }
  }
  __syncthreads();
  if (kSPD && ok) {  // exact symmetry: the upper triangle wins
    for (int e = gl; e < nn; e += L) {
      const int i = e / n, j = e - i * n;
      if (i > j) mine[e] = mine[j * n + i];
    }
  }
  __syncthreads();
  double* dst = A + m0 * nn;
  for (int e = tid; e < nmat * nn; e += kTinyThreads)
    if (seg_state[e / nn] == 0) dst[e] = stage[e];
  if (status && live && gl == 0) status[m0 + seg] = seg_state[seg];
}

template <int L, int R, bool kSPD>
cudaError_t launch_tiny(const TinyPartition& part, double* A, int64_t count, int32_t* status, cudaStream_t s) {
  constexpr int MPC = kTinyThreads / L;
  const int64_t blocks = (count + MPC - 1) / MPC;
  const size_t smem = sizeof(double) * MPC * part.n * part.n;
  auto k = tiny_batched_kernel<L, R, kSPD>;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<(unsigned)blocks, kTinyThreads, smem, s>>>(A, count, part, status);
  return cudaGetLastError();
}

// (L, R) per order: L R >= n with few idle slots, at most 48 doubles of rows
// per lane.
template <bool kSPD>
cudaError_t launch_tiny_for(const TinyPartition& part, double* A, int64_t count, int32_t* status, cudaStream_t s) {
  const int n = part.n;
  if (n <= 8) return launch_tiny<1, 8, kSPD>(part, A, count, status, s);
  if (n <= 12) return launch_tiny<4, 3, kSPD>(part, A, count, status, s);
  if (n <= 16) return launch_tiny<8, 2, kSPD>(part, A, count, status, s);
  if (n <= 24) return launch_tiny<8, 3, kSPD>(part, A, count, status, s);
  return launch_tiny<16, 2, kSPD>(part, A, count, status, s);
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
  return spd ? launch_tiny_for<true>(part, A, count, status, s) : launch_tiny_for<false>(part, A, count, status, s);
}

}  // namespace blockinv
