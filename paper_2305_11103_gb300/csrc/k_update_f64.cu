// FP64 kernels of one elimination step (Eq. (a), block form; in-place
// assembly as in the paper's `invertor_inplace_by_a`, Sec. 4.2):
//
//  K2 row panel   X[k, j] <- P^-1 X[k, j] for every block column j != k
//                 (the paper's right-arrow op, -A^-1 B up to sign), and
//                 X[k, k] <- P^-1. The block column k (rows outside block k)
//                 is copied to U first, since K3 overwrites it.
//  K3 Schur update X[i, j] <- X[i, j] - U[i] X[k, j] for i, j != k (S_A =
//                 D - C A^-1 B for the trailing blocks, and the top-left
//                 update A^-1 + A^-1 B S_A^-1 C A^-1 for the rows already
//                 eliminated), fused with the column assembly
//                 X[i, k] <- -U[i] P^-1: block column k is treated as zero
//                 on input and row panel k holds P^-1 there.
//
// FP64 on GB300 issues at about 2 DFMA per clock per SM, so both kernels are
// bound by the FP64 pipe, not by memory: K3 moves 16 bytes of X per 2b flops.
// They are register-tiled SIMT kernels sized to keep that pipe busy.
#include "internal.h"

namespace blockinv {

namespace {

__device__ __forceinline__ bool failed(const int32_t* status) {
  return *(volatile const int32_t*)status != 0;
}

// ---------------------------------------------------------------- K2 ------
// One CTA owns a 32-column strip of row panel k (all b rows), so the strip
// can be read completely before it is overwritten in place. Thread (g, c)
// holds rows g, g + 8, g + 16, ... of column c.
constexpr int kPanelCols = 32;
constexpr int kPanelK = 8;

// Row panel for the 32-column strip starting at j0 (all b rows of block k).
// kFit (grouped batches, b often well below MAXB): a warp runs only the FMAs
// of its rows below b (its row count is warp-uniform), and the last k chunk
// only its b mod 8 values.
template <int MAXB, bool kFit = false>
__device__ __forceinline__ void row_panel_strip(double* __restrict__ X, int64_t ldx, int n, int o, int b,
                                                const double* __restrict__ Pinv, int j0) {
  constexpr int RPT = MAXB / 8;  // rows per thread
  __shared__ double Ps[kPanelK][MAXB];
  __shared__ double Xs[kPanelK][kPanelCols];
  const int tid = threadIdx.x;
  const int c = tid & 31;
  const int g = tid >> 5;
  const int j = j0 + c;
  double acc[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) acc[q] = 0.0;

  for (int kc = 0; kc < b; kc += kPanelK) {
    for (int e = tid; e < b * kPanelK; e += 256) {
      const int r = e / kPanelK;
      const int kk = e - r * kPanelK;
      Ps[kk][r] = (kc + kk < b) ? Pinv[(int64_t)r * b + kc + kk] : 0.0;
    }
    {
      const int kk = tid >> 5;  // 8 rows x 32 columns
      const int jj = j0 + (tid & 31);
      Xs[kk][tid & 31] = (kc + kk < b && jj < n) ? X[(int64_t)(o + kc + kk) * ldx + jj] : 0.0;
    }
    __syncthreads();
    if (!kFit) {
#pragma unroll
      for (int kk = 0; kk < kPanelK; ++kk) {
        const double x = Xs[kk][c];
#pragma unroll
        for (int q = 0; q < RPT; ++q) acc[q] = fma(Ps[kk][g + 8 * q], x, acc[q]);
      }
    } else {
      // Rows outside, k inside, with a warp-uniform branch around each row's
      // FMAs: predicated-off FP64 instructions still occupy this GPU's FP64
      // pipe (measured), so rows at or past b must be branched over.
      const int nq = b > g ? (b - g + 7) / 8 : 0;  // rows g + 8 q < b of this warp
      const int kn = min(kPanelK, b - kc);
      if (kn == kPanelK) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          if (q >= nq) break;
          double a = acc[q];
#pragma unroll
          for (int kk = 0; kk < kPanelK; ++kk) a = fma(Ps[kk][g + 8 * q], Xs[kk][c], a);
          acc[q] = a;
        }
      } else {
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          if (q >= nq) break;
          double a = acc[q];
          for (int kk = 0; kk < kn; ++kk) a = fma(Ps[kk][g + 8 * q], Xs[kk][c], a);
          acc[q] = a;
        }
      }
    }
    __syncthreads();
  }
  if (j >= n) return;
  const bool pivot_col = (j >= o && j < o + b);
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int r = g + 8 * q;
    if (r < b) X[(int64_t)(o + r) * ldx + j] = pivot_col ? Pinv[(int64_t)r * b + (j - o)] : acc[q];
  }
}

// Copy block column k (rows [r0, r1) outside block k) into U (n x b, ld b).
__device__ __forceinline__ void copy_column_panel(const double* __restrict__ X, int64_t ldx, int o, int b,
                                                  double* __restrict__ U, int r0, int r1, int part,
                                                  int nparts) {
  const int64_t total = (int64_t)(r1 - r0) * b;
  for (int64_t e = (int64_t)part * blockDim.x + threadIdx.x; e < total; e += (int64_t)nparts * blockDim.x) {
    const int i = r0 + (int)(e / b);
    const int l = (int)(e - (int64_t)(i - r0) * b);
    if (i >= o && i < o + b) continue;
    U[(int64_t)i * b + l] = X[(int64_t)i * ldx + o + l];
  }
}

// One CTA per 32-column strip of row panel k (all b rows), so the strip can
// be read completely before it is overwritten in place. Thread (g, c) holds
// rows g, g + 8, g + 16, ... of column c. Extra CTAs copy the column panel.
template <int MAXB>
__global__ void __launch_bounds__(256)
row_panel_f64_kernel(double* __restrict__ X, int64_t ldx, int n, int o, int b,
                     const double* __restrict__ Pinv, double* __restrict__ U,
                     const int32_t* status, int col_tiles) {
  if (failed(status)) return;
  if ((int)blockIdx.x >= col_tiles) {
    copy_column_panel(X, ldx, o, b, U, 0, n, blockIdx.x - col_tiles, gridDim.x - col_tiles);
    return;
  }
  row_panel_strip<MAXB>(X, ldx, n, o, b, Pinv, blockIdx.x * kPanelCols);
}

__device__ __forceinline__ int find_item(const int32_t* __restrict__ start, int count, int t) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Grouped row panel: strip t of the batch belongs to item m; the same CTA
// also copies its share of item m's column panel.
template <int MAXB>
__global__ void __launch_bounds__(256)
row_panel_grouped_kernel(const GroupStep* __restrict__ items, int count, const int32_t* __restrict__ col_start) {
  const int t = blockIdx.x;
  const int m = find_item(col_start, count, t);
  const GroupStep it = items[m];
  if (failed(it.status)) return;
  const int strips = col_start[m + 1] - col_start[m];
  const int s = t - col_start[m];
  const int rows_per = (it.n + strips - 1) / strips;
  const int r0 = min(it.n, s * rows_per), r1 = min(it.n, r0 + rows_per);
  copy_column_panel(it.X, it.ldx, it.o, it.b, it.U, r0, r1, 0, 1);
  row_panel_strip<MAXB, true>(it.X, it.ldx, it.n, it.o, it.b, it.Pinv, s * kPanelCols);
}

// ---------------------------------------------------------------- K3 ------
constexpr int kTile = 64;
constexpr int kTileK = 8;

// Write masks for the look-ahead split of one step's update (B1 = the rows /
// columns of the next pivot block [o1, o1 + b1)):
//   kAll   every element outside the pivot rows of this step
//   kRest  elements with row and column outside B1
//   kNextA elements with row in B1 or column in B1 (row tiles that meet B1)
//   kNextB elements with column in B1 (row tiles that miss B1)
enum WriteMask { kAll = 0, kRest = 1, kNextA = 2, kNextB = 3 };

__device__ __forceinline__ bool in_range(int v, int lo, int len) { return v >= lo && v < lo + len; }

// One TILE x TILE output tile (TILE = 64 or 32) by 256 threads, each holding
// (TILE / 16) x (TILE / 16) outputs.
// kCompact (grouped batches): i0 counts only the n - b rows outside the pivot
// block (row ic is ic, or ic + b from o on), so no tile computes pivot rows,
// and the last k chunk runs only its b mod 8 values.
template <int TILE = kTile, bool kCompact = false>
__device__ __forceinline__ void schur_tile(double* __restrict__ X, int64_t ldx, int n, int o, int b,
                                           const double* __restrict__ U, int i0, int j0, int o1 = 0, int b1 = 0,
                                           int mask = kAll) {
  constexpr int PT = TILE / 16;              // outputs per thread along each side
  constexpr int LOADS = TILE * kTileK / 256;  // tile elements per thread per k chunk
  __shared__ __align__(16) double Us[kTileK][TILE];
  __shared__ __align__(16) double Vs[kTileK][TILE];
  const int tid = threadIdx.x;
  const int tx = tid & 15;
  const int ty = tid >> 4;
  double acc[PT][PT];
#pragma unroll
  for (int a = 0; a < PT; ++a)
#pragma unroll
    for (int d = 0; d < PT; ++d) acc[a][d] = 0.0;

  for (int kc = 0; kc < b; kc += kTileK) {
#pragma unroll
    for (int h = 0; h < LOADS; ++h) {
      const int e = tid + h * 256;
      // U tile: TILE rows x 8 k
      const int ui = e >> 3, uk = e & 7;
      const int ic = i0 + ui;
      const bool iok = kCompact ? ic < n - b : ic < n;
      const int gi = (kCompact && ic >= o) ? ic + b : ic;
      Us[uk][ui] = (iok && kc + uk < b) ? U[(int64_t)gi * b + kc + uk] : 0.0;
      // V tile: 8 k x TILE columns of row panel k
      const int vk = e / TILE, vj = e % TILE;
      const int gj = j0 + vj;
      Vs[vk][vj] = (gj < n && kc + vk < b) ? X[(int64_t)(o + kc + vk) * ldx + gj] : 0.0;
    }
    __syncthreads();
    auto kstep = [&](int kk) {
      double u[PT], v[PT];
#pragma unroll
      for (int a = 0; a < PT; ++a) u[a] = Us[kk][ty * PT + a];
#pragma unroll
      for (int d = 0; d < PT; ++d) v[d] = Vs[kk][tx * PT + d];
#pragma unroll
      for (int a = 0; a < PT; ++a)
#pragma unroll
        for (int d = 0; d < PT; ++d) acc[a][d] = fma(u[a], v[d], acc[a][d]);
    };
    if (!kCompact || kc + kTileK <= b) {
#pragma unroll
      for (int kk = 0; kk < kTileK; ++kk) kstep(kk);
    } else {
      for (int kk = 0; kk < b - kc; ++kk) kstep(kk);  // the last, partial chunk
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < PT; ++a) {
    const int ic = i0 + ty * PT + a;
    if (kCompact ? ic >= n - b : (ic >= n || (ic >= o && ic < o + b))) continue;
    const int i = (kCompact && ic >= o) ? ic + b : ic;
    const bool ri = in_range(i, o1, b1);
    double* row = X + (int64_t)i * ldx;
#pragma unroll
    for (int d = 0; d < PT; ++d) {
      const int j = j0 + tx * PT + d;
      if (j >= n) continue;
      const bool cj = in_range(j, o1, b1);
      const bool write = mask == kAll || (mask == kRest && !ri && !cj) || (mask == kNextA && (ri || cj)) ||
                         (mask == kNextB && cj);
      if (!write) continue;
      const double base = (j >= o && j < o + b) ? 0.0 : row[j];
      row[j] = base - acc[a][d];
    }
  }
}

// Look-ahead part of step k: the elements of block row and block column
// B1 = [o1, o1 + b1). Tiles: row tiles meeting B1 x all column tiles, then
// the other row tiles x column tiles meeting B1 (disjoint element sets).
__global__ void __launch_bounds__(256)
schur_next_f64_kernel(double* __restrict__ X, int64_t ldx, int n, int o, int b, const double* __restrict__ U,
                      const int32_t* status, int o1, int b1) {
  if (failed(status)) return;
  const int tn = (n + kTile - 1) / kTile;
  const int r_lo = o1 / kTile, r_hi = (o1 + b1 + kTile - 1) / kTile;
  const int c_lo = r_lo, c_hi = r_hi;
  const int part1 = (r_hi - r_lo) * tn;
  int t = blockIdx.x;
  if (t < part1) {
    const int i0 = (r_lo + t / tn) * kTile, j0 = (t % tn) * kTile;
    schur_tile(X, ldx, n, o, b, U, i0, j0, o1, b1, kNextA);
    return;
  }
  t -= part1;
  const int cw = c_hi - c_lo;
  int rt = t / cw;
  if (rt >= r_lo) rt += r_hi - r_lo;  // skip the row tiles of part 1
  const int i0 = rt * kTile, j0 = (c_lo + t % cw) * kTile;
  if (i0 >= o && i0 + kTile <= o + b) return;
  schur_tile(X, ldx, n, o, b, U, i0, j0, o1, b1, kNextB);
}

// The rest of step k after the look-ahead part: elements outside B1.
__global__ void __launch_bounds__(256)
schur_rest_f64_kernel(double* __restrict__ X, int64_t ldx, int n, int o, int b, const double* __restrict__ U,
                      const int32_t* status, int o1, int b1) {
  const int i0 = blockIdx.y * kTile;
  const int j0 = blockIdx.x * kTile;
  if (i0 >= o && i0 + kTile <= o + b) return;
  if (i0 >= o1 && i0 + kTile <= o1 + b1) return;  // whole tile in the next pivot rows
  if (j0 >= o1 && j0 + kTile <= o1 + b1) return;  // whole tile in the next pivot columns
  if (failed(status)) return;
  schur_tile(X, ldx, n, o, b, U, i0, j0, o1, b1, kRest);
}

__global__ void __launch_bounds__(256)
schur_update_f64_kernel(double* __restrict__ X, int64_t ldx, int n, int o, int b,
                        const double* __restrict__ U, const int32_t* status) {
  const int i0 = blockIdx.y * kTile;
  const int j0 = blockIdx.x * kTile;
  if (i0 >= o && i0 + kTile <= o + b) return;  // tile lies inside the pivot rows
  if (failed(status)) return;
  schur_tile(X, ldx, n, o, b, U, i0, j0);
}

// Grouped Schur update: tile t of the batch belongs to item m (TILE x TILE
// tiles, TILE = 64 or 32, over the n - b rows outside the pivot block by the
// n columns: ceil((n - b) / TILE) x ceil(n / TILE) tiles per item).
template <int TILE>
__global__ void __launch_bounds__(256)
schur_update_grouped_kernel(const GroupStep* __restrict__ items, int count, const int32_t* __restrict__ tile_start) {
  const int t = blockIdx.x;
  const int m = find_item(tile_start, count, t);
  const GroupStep it = items[m];
  const int tiles_col = (it.n + TILE - 1) / TILE;
  const int local = t - tile_start[m];
  const int i0 = (local / tiles_col) * TILE;  // compact row: pivot rows skipped
  const int j0 = (local % tiles_col) * TILE;
  if (failed(it.status)) return;
  schur_tile<TILE, true>(it.X, it.ldx, it.n, it.o, it.b, it.U, i0, j0);
}

// --------------------------------------------------------- residual -------
// Partial sums of ||A X - I||_F^2 (sums3[0]), ||A||_F^2 (sums3[1]) and
// ||X||_F^2 (sums3[2]). The product tile is formed in FP64 and reduced in
// the epilogue, so no n x n temporary is needed.
__global__ void __launch_bounds__(256)
residual_f64_kernel(int n, const double* __restrict__ A, int64_t lda,
                    const double* __restrict__ X, int64_t ldx, double* sums3) {
  const int i0 = blockIdx.y * kTile;
  const int j0 = blockIdx.x * kTile;
  __shared__ __align__(16) double As[kTileK][kTile];
  __shared__ __align__(16) double Xs[kTileK][kTile];
  __shared__ double red[3][8];
  const int tid = threadIdx.x;
  const int tx = tid & 15;
  const int ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int d = 0; d < 4; ++d) acc[a][d] = 0.0;
  for (int kc = 0; kc < n; kc += kTileK) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + h * 256;
      const int ai = e >> 3, ak = e & 7;
      As[ak][ai] = (i0 + ai < n && kc + ak < n) ? A[(int64_t)(i0 + ai) * lda + kc + ak] : 0.0;
      const int xk = e >> 6, xj = e & 63;
      Xs[xk][xj] = (kc + xk < n && j0 + xj < n) ? X[(int64_t)(kc + xk) * ldx + j0 + xj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTileK; ++kk) {
      double u[4], v[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) u[a] = As[kk][ty * 4 + a];
#pragma unroll
      for (int d = 0; d < 4; ++d) v[d] = Xs[kk][tx * 4 + d];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int d = 0; d < 4; ++d) acc[a][d] = fma(u[a], v[d], acc[a][d]);
    }
    __syncthreads();
  }
  double r2 = 0.0, a2 = 0.0, x2 = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty * 4 + a;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int j = j0 + tx * 4 + d;
      if (i < n && j < n) {
        const double e = acc[a][d] - (i == j ? 1.0 : 0.0);
        r2 = fma(e, e, r2);
        const double av = A[(int64_t)i * lda + j];
        const double xv = X[(int64_t)i * ldx + j];
        a2 = fma(av, av, a2);
        x2 = fma(xv, xv, x2);
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, off);
    a2 += __shfl_xor_sync(0xffffffffu, a2, off);
    x2 += __shfl_xor_sync(0xffffffffu, x2, off);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = r2;
    red[1][tid >> 5] = a2;
    red[2][tid >> 5] = x2;
  }
  __syncthreads();
  if (tid < 3) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[tid][w];
    atomicAdd(&sums3[tid], s);
  }
}

}  // namespace

cudaError_t launch_row_panel_f64(double* X, int64_t ldx, int n, int o, int b,
                                 const double* Pinv, double* U, const int32_t* status,
                                 cudaStream_t s) {
  const int col_tiles = (n + kPanelCols - 1) / kPanelCols;
  const int copy_ctas = (n > b) ? 64 : 0;
  dim3 grid(col_tiles + copy_ctas);
  if (b <= 64)
    row_panel_f64_kernel<64><<<grid, 256, 0, s>>>(X, ldx, n, o, b, Pinv, U, status, col_tiles);
  else if (b <= 128)
    row_panel_f64_kernel<128><<<grid, 256, 0, s>>>(X, ldx, n, o, b, Pinv, U, status, col_tiles);
  else if (b <= 256)
    row_panel_f64_kernel<256><<<grid, 256, 0, s>>>(X, ldx, n, o, b, Pinv, U, status, col_tiles);
  else if (b <= 512)
    row_panel_f64_kernel<512><<<grid, 256, 0, s>>>(X, ldx, n, o, b, Pinv, U, status, col_tiles);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_schur_update_f64(double* X, int64_t ldx, int n, int o, int b,
                                    const double* U, const int32_t* status, cudaStream_t s) {
  if (n == b) return cudaSuccess;
  const int t = (n + kTile - 1) / kTile;
  schur_update_f64_kernel<<<dim3(t, t), 256, 0, s>>>(X, ldx, n, o, b, U, status);
  return cudaGetLastError();
}

cudaError_t launch_row_panel_grouped(const GroupStep* items, int count, const int32_t* col_start,
                                     int total_cols, int bmax, cudaStream_t s) {
  if (count <= 0 || total_cols <= 0) return cudaSuccess;
  if (bmax <= 64)
    row_panel_grouped_kernel<64><<<total_cols, 256, 0, s>>>(items, count, col_start);
  else if (bmax <= 128)
    row_panel_grouped_kernel<128><<<total_cols, 256, 0, s>>>(items, count, col_start);
  else if (bmax <= 256)
    row_panel_grouped_kernel<256><<<total_cols, 256, 0, s>>>(items, count, col_start);
  else if (bmax <= 512)
    row_panel_grouped_kernel<512><<<total_cols, 256, 0, s>>>(items, count, col_start);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_schur_update_grouped(const GroupStep* items, int count, const int32_t* tile_start,
                                        int total_tiles, int tile, cudaStream_t s) {
  if (count <= 0 || total_tiles <= 0) return cudaSuccess;
  if (tile == 32)
    schur_update_grouped_kernel<32><<<total_tiles, 256, 0, s>>>(items, count, tile_start);
  else if (tile == 64)
    schur_update_grouped_kernel<64><<<total_tiles, 256, 0, s>>>(items, count, tile_start);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_schur_split_f64(double* X, int64_t ldx, int n, int o, int b, const double* U,
                                   const int32_t* status, int o1, int b1, bool next_part, cudaStream_t s) {
  if (n == b) return cudaSuccess;
  const int t = (n + kTile - 1) / kTile;
  if (next_part) {
    const int r_lo = o1 / kTile, r_hi = (o1 + b1 + kTile - 1) / kTile;
    const int tiles = (r_hi - r_lo) * t + (t - (r_hi - r_lo)) * (r_hi - r_lo);
    schur_next_f64_kernel<<<tiles, 256, 0, s>>>(X, ldx, n, o, b, U, status, o1, b1);
  } else {
    schur_rest_f64_kernel<<<dim3(t, t), 256, 0, s>>>(X, ldx, n, o, b, U, status, o1, b1);
  }
  return cudaGetLastError();
}

cudaError_t launch_residual_f64(int n, const double* A, int64_t lda, const double* X,
                                int64_t ldx, double* sums3, cudaStream_t s) {
  const int t = (n + kTile - 1) / kTile;
  residual_f64_kernel<<<dim3(t, t), 256, 0, s>>>(n, A, lda, X, ldx, sums3);
  return cudaGetLastError();
}

}  // namespace blockinv
