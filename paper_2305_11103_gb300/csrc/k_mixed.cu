// Mixed-precision elimination: the same in-place block Gauss-Jordan steps as
// the FP64 path (Eq. (a) once per diagonal block), on an FP32 copy of the
// matrix, with the Schur update (the dominant 2 b (n - b) n flops per step)
// on the tensor cores:
//
//   X32[i, j] <- (j in pivot cols ? 0 : X32[i, j]) - sum_l U[i, l] Vt[j, l]
//
// U (block column k) and Vt (row panel k = P^-1 X[k, :], transposed) are
// packed K-major, rounded to TF32 or BF16, by the FP32 row-panel kernel,
// and multiplied by tcgen05.mma with an FP32 accumulator in TMEM. The pivot
// blocks are inverted in FP32 by the cluster Gauss-Jordan kernel. Accuracy is
// recovered afterwards by Newton-Schulz refinement against the FP64 input.
#include <cuda_bf16.h>

#include <algorithm>

#include "tc_gemm.cuh"

namespace blockinv {

namespace {

__device__ __forceinline__ bool failed(const int32_t* status) {
  return *(volatile const int32_t*)status != 0;
}

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

template <bool kBF16>
struct OpType;
template <>
struct OpType<false> {
  using T = float;
  static __device__ __forceinline__ T cvt(float x) { return round_tf32(x); }
};
template <>
struct OpType<true> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ T cvt(float x) { return __float2bfloat16_rn(x); }
};

// ------------------------------------------------------------- casts ------
// Row by row (a CTA per row at a time), so no element index is divided.
// kVec: A's rows start 16-byte aligned (aligned A, even lda), so four
// elements move per 2 x 16-byte load and one 16-byte store (X32 rows are
// multiples of 32 floats); otherwise one element at a time.
template <bool kVec>
__global__ void cast_f64_to_f32_kernel(const double* __restrict__ A, int64_t lda, float* __restrict__ X,
                                       int64_t ldx, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const double* a = A + (int64_t)i * lda;
    float* x = X + (int64_t)i * ldx;
    if constexpr (kVec) {
#pragma unroll 2
      for (int j = 4 * threadIdx.x; j < ldx; j += 4 * blockDim.x) {
        float4 v;
        if (j + 3 < n) {
          const double2 p = *reinterpret_cast<const double2*>(a + j);
          const double2 q = *reinterpret_cast<const double2*>(a + j + 2);
          v = make_float4((float)p.x, (float)p.y, (float)q.x, (float)q.y);
        } else {
          v = make_float4(j < n ? (float)a[j] : 0.f, j + 1 < n ? (float)a[j + 1] : 0.f,
                          j + 2 < n ? (float)a[j + 2] : 0.f, 0.f);
        }
        *reinterpret_cast<float4*>(x + j) = v;
      }
    } else {
#pragma unroll 4
      for (int j = threadIdx.x; j < ldx; j += blockDim.x) x[j] = (j < n) ? (float)a[j] : 0.f;
    }
  }
}

template <bool kVec>
__global__ void cast_f32_to_f64_kernel(const float* __restrict__ X, int64_t ldx, double* __restrict__ A,
                                       int64_t lda, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const float* x = X + (int64_t)i * ldx;
    double* a = A + (int64_t)i * lda;
    if constexpr (kVec) {
#pragma unroll 2
      for (int j = 4 * threadIdx.x; j < n; j += 4 * blockDim.x) {
        const float4 v = *reinterpret_cast<const float4*>(x + j);
        if (j + 3 < n) {
          *reinterpret_cast<double2*>(a + j) = make_double2((double)v.x, (double)v.y);
          *reinterpret_cast<double2*>(a + j + 2) = make_double2((double)v.z, (double)v.w);
        } else {
          a[j] = (double)v.x;
          if (j + 1 < n) a[j + 1] = (double)v.y;
          if (j + 2 < n) a[j + 2] = (double)v.z;
        }
      }
    } else {
#pragma unroll 4
      for (int j = threadIdx.x; j < n; j += blockDim.x) a[j] = (double)x[j];
    }
  }
}

bool rows_16b_aligned(const void* p, int64_t ld, int elem) {
  return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && (ld * elem) % 16 == 0;
}

// --------------------------------------------------------- row panel ------
// One CTA per 32-column strip of row panel k: V = P^-1 X32[k, strip] in FP32,
// written back to X32 (P^-1 itself in the pivot columns) and, transposed and
// rounded, to Vt[j][0..kpad) (zero beyond b). Extra CTAs pack
// U[i][l] = X32[i][o + l] for rows outside block k (zero elsewhere).
constexpr int kCols = 32;
constexpr int kKc = 16;  // k columns of P^-1 per shared-memory chunk (double-buffered)

// Operands are stored as `nsl` slices of kpad columns: slice 0 holds the
// rounded value (hi), slice 1 (if present) the rounded remainder (lo), so
// that hi*hi + hi*lo + lo*hi carries about twice the operand precision.
// Rows are ldop elements apart (two steps' slice sets side by side when the
// Schur updates of two steps run as one sweep).
template <int MAXB, bool kBF16>
__global__ void __launch_bounds__(256)
row_panel_mixed_kernel(float* __restrict__ X, int64_t ldx, int n, int o, int b, const float* __restrict__ Pinv,
                       typename OpType<kBF16>::T* __restrict__ U, typename OpType<kBF16>::T* __restrict__ Vt,
                       int kpad, int nsl, int64_t ldop, const int32_t* status, int col_tiles) {
  using Op = OpType<kBF16>;
  if (failed(status)) return;
  const int tid = threadIdx.x;
  if ((int)blockIdx.x >= col_tiles) {
    // U: four consecutive columns per thread and step (kpad is a multiple of 64)
    const int q4 = kpad / 4;
    const int64_t total = (int64_t)n * q4;
    const int64_t stride = (int64_t)(gridDim.x - col_tiles) * blockDim.x;
    for (int64_t e = (int64_t)(blockIdx.x - col_tiles) * blockDim.x + tid; e < total; e += stride) {
      const int i = (int)(e / q4);
      const int l0 = 4 * (int)(e - (int64_t)i * q4);
      const bool row_keep = !(i >= o && i < o + b);
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = (row_keep && l0 + u < b) ? X[(int64_t)i * ldx + o + l0 + u] : 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const auto hi = Op::cvt(v[u]);
        U[(int64_t)i * ldop + l0 + u] = hi;
        if (nsl > 1) U[(int64_t)i * ldop + kpad + l0 + u] = Op::cvt(v[u] - static_cast<float>(hi));
      }
    }
    return;
  }
  extern __shared__ __align__(16) float sm[];
  // two chunks of P^-1 columns (rows padded to MAXB + 4: the fill, k fastest,
  // hits 32 different banks) and of the strip's rows of X
  constexpr int PLD = MAXB + 4;
  float* Ps = sm;                        // [2][kKc][PLD]
  float* Xs = Ps + 2 * kKc * PLD;        // [2][kKc][kCols]
  float* Vs = Xs + 2 * kKc * kCols;      // [kCols][MAXB + 1]
  // thread (rg, cg): rows rg * RPT .. + RPT, columns 4 cg .. + 4 of the strip;
  // per k step RPT / 4 + 1 vector loads from shared memory feed 4 RPT FMAs
  // (rows of Ps at or past b are never written: their results are dropped)
  constexpr int RPT = MAXB / 32;
  constexpr int PF = MAXB * kKc / 256;   // P^-1 elements per thread per chunk
  const int cg = tid & 7;
  const int rg = tid >> 3;
  const int j0 = blockIdx.x * kCols;
  float acc[RPT][4];
#pragma unroll
  for (int r = 0; r < RPT; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
  // Two chunks in flight: chunk i + 2 is fetched into registers while chunk i
  // is used, and stashed in shared memory after chunk i + 1 (an L2 round trip
  // outlasts one chunk's FMAs).
  constexpr int XF = kKc * kCols / 256;  // strip elements per thread per chunk
  struct Regs {
    float p[PF];
    float x[XF];
  };
  auto fetch = [&](int kc, Regs& g) {  // global -> registers
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int e = tid + q * 256;
      const int r = e / kKc, kk = e - r * kKc;
      g.p[q] = (r < b && kc + kk < b) ? Pinv[(int64_t)r * b + kc + kk] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < XF; ++q) {
      const int kk = (tid >> 5) + 8 * q;
      const int jj = j0 + (tid & 31);
      g.x[q] = (kc + kk < b && jj < n) ? X[(int64_t)(o + kc + kk) * ldx + jj] : 0.f;
    }
  };
  auto stash = [&](int buf, const Regs& g) {  // registers -> shared chunk buf
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int e = tid + q * 256;
      const int r = e / kKc, kk = e - r * kKc;
      Ps[(buf * kKc + kk) * PLD + r] = g.p[q];
    }
#pragma unroll
    for (int q = 0; q < XF; ++q) Xs[(buf * kKc + (tid >> 5) + 8 * q) * kCols + (tid & 31)] = g.x[q];
  };
  auto compute = [&](int buf) {
    const float* P0 = Ps + buf * kKc * PLD;
    const float* X0 = Xs + buf * kKc * kCols;
#pragma unroll
    for (int kk = 0; kk < kKc; ++kk) {
      const float4 xv = *reinterpret_cast<const float4*>(&X0[kk * kCols + 4 * cg]);
      float pv[RPT];
      if constexpr (RPT % 4 == 0) {
#pragma unroll
        for (int r = 0; r < RPT; r += 4) {
          const float4 t = *reinterpret_cast<const float4*>(&P0[kk * PLD + rg * RPT + r]);
          pv[r] = t.x;
          pv[r + 1] = t.y;
          pv[r + 2] = t.z;
          pv[r + 3] = t.w;
        }
      } else {
#pragma unroll
        for (int r = 0; r < RPT; ++r) pv[r] = P0[kk * PLD + rg * RPT + r];
      }
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        acc[r][0] = fmaf(pv[r], xv.x, acc[r][0]);
        acc[r][1] = fmaf(pv[r], xv.y, acc[r][1]);
        acc[r][2] = fmaf(pv[r], xv.z, acc[r][2]);
        acc[r][3] = fmaf(pv[r], xv.w, acc[r][3]);
      }
    }
  };
  const int nch = (b + kKc - 1) / kKc;
  Regs ga, gb;
  fetch(0, ga);
  if (nch > 1) fetch(kKc, gb);
  stash(0, ga);
  __syncthreads();
  // chunk i uses buffer i & 1; ga / gb alternate as the landing registers
  for (int i = 0; i < nch; i += 2) {
    if (i + 2 < nch) fetch((i + 2) * kKc, ga);
    compute(0);
    if (i + 1 < nch) stash(1, gb);
    __syncthreads();
    if (i + 1 >= nch) break;
    if (i + 3 < nch) fetch((i + 3) * kKc, gb);
    compute(1);
    if (i + 2 < nch) stash(0, ga);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int row = rg * RPT + r;
    if (row >= b) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 4 * cg + q;
      const int j = j0 + c;
      const bool pivot_col = (j >= o && j < o + b);
      const float v = (j < n) ? (pivot_col ? Pinv[(int64_t)row * b + (j - o)] : acc[r][q]) : 0.f;
      if (j < n) X[(int64_t)(o + row) * ldx + j] = v;
      Vs[c * (MAXB + 1) + row] = v;
    }
  }
  __syncthreads();
  for (int cc = 0; cc < kCols; ++cc) {
    const int jj = j0 + cc;
    if (jj >= n) break;
    for (int r = tid; r < kpad; r += 256) {
      const float v = r < b ? Vs[cc * (MAXB + 1) + r] : 0.f;
      const auto hi = Op::cvt(v);
      Vt[(int64_t)jj * ldop + r] = hi;
      if (nsl > 1) Vt[(int64_t)jj * ldop + kpad + r] = Op::cvt(v - static_cast<float>(hi));
    }
  }
}

// ---------------------------------------------------- Schur epilogue ------
// The Schur update of one elimination step, or of two in one sweep:
//
//   X[i, j] <- (drop(i, j) ? 0 : X[i, j]) - sum_l U[i, l] Vt[j, l]
//
// for the rows i outside [s0, s1) (the newest pivot block, written by its
// row panel instead). drop(i, j): j in [d0, d1), or j in [g0, g1) with i
// outside [e0, e1). One step k: s = d = block k, g empty (block column k
// becomes -U P^-1, since Vt holds P^-1 there). Two steps k, k + 1 (U and Vt
// holding both steps' panels): s = d = block k + 1, g = e = block k (the rows
// of block k, which hold step k's row panel, keep their block-k columns).
// A launch writes only the elements of its part:
enum SchurPart {
  kWhole = 0,      // every row outside [s0, s1)
  kInside = 1,     // only the square [r0, r1) x [r0, r1) (the next pivot block)
  kOutside = 2,    // all but that square
  kCrossRows = 3,  // only the rows [r0, r1)
  kCrossCols = 4,  // only the columns [r0, r1), rows outside [r0, r1)
};

struct EpiSchurF32 {
  float* X;
  int64_t ldx;
  int n;
  const int32_t* status;
  int s0, s1;          // rows not written
  int d0, d1;          // columns whose old value is dropped in every written row
  int g0, g1, e0, e1;  // columns whose old value is dropped in rows outside [e0, e1)
  int part = kWhole;
  int r0 = 0, r1 = 0;
  // The GEMM moves X's 32 x 32 blocks by TMA and asks value() per element.
  static constexpr bool kTmaC = true;
  __device__ bool skip() const { return failed(status); }
  __device__ bool writes(int row, int col) const {
    if (row >= n || col >= n || (row >= s0 && row < s1)) return false;
    const bool rin = row >= r0 && row < r1, cin = col >= r0 && col < r1;
    switch (part) {
      case kInside: return rin && cin;
      case kOutside: return !(rin && cin);
      case kCrossRows: return rin;
      case kCrossCols: return cin && !rin;
      default: return true;
    }
  }
  // The new value of X[row][col] from its current value x and the product v
  // (x itself where this launch writes nothing).
  __device__ float value(int row, int col, float x, float v) const {
    if (!writes(row, col)) return x;
    const bool drop = (col >= d0 && col < d1) || (col >= g0 && col < g1 && !(row >= e0 && row < e1));
    return (drop ? 0.f : x) - v;
  }
  // Whether value() is x - v for every element of the 32 x 32 block at (row0,
  // col0) that lies inside the matrix (the block meets no row left alone, no
  // dropped column and no edge of its part); elements outside the matrix are
  // not stored. The GEMM then skips the per-element tests.
  __device__ bool block_simple(int row0, int col0) const {
    const int rend = row0 + 32, cend = col0 + 32;
    if ((row0 < s1 && rend > s0) || (col0 < d1 && cend > d0) || (col0 < g1 && cend > g0)) return false;
    const bool rows_in = row0 >= r0 && rend <= r1, rows_out = rend <= r0 || row0 >= r1;
    const bool cols_in = col0 >= r0 && cend <= r1, cols_out = cend <= r0 || col0 >= r1;
    switch (part) {
      case kInside: return rows_in && cols_in;
      case kOutside: return rows_out || cols_out;
      case kCrossRows: return rows_in;
      case kCrossCols: return cols_in && rows_out;
      default: return true;
    }
  }
  // Whether value() may change an element of the 32 x 32 block at (row0,
  // col0); blocks it leaves alone are neither loaded nor stored.
  __device__ bool block_live(int row0, int col0) const {
    if (row0 >= n || col0 >= n) return false;
    const int rend = min(row0 + 32, n), cend = min(col0 + 32, n);
    if (row0 >= s0 && rend <= s1) return false;
    const bool rows_meet = row0 < r1 && rend > r0, cols_meet = col0 < r1 && cend > r0;
    const bool rows_in = row0 >= r0 && rend <= r1, cols_in = col0 >= r0 && cend <= r1;
    switch (part) {
      case kInside: return rows_meet && cols_meet;
      case kOutside: return !(rows_in && cols_in);
      case kCrossRows: return rows_meet;
      case kCrossCols: return cols_meet && !rows_in;
      default: return true;
    }
  }
};

// The epilogue of step (o, b) alone.
EpiSchurF32 one_step_epi(float* X, int64_t ldx, int n, int o, int b, const int32_t* status) {
  EpiSchurF32 e{};
  e.X = X;
  e.ldx = ldx;
  e.n = n;
  e.status = status;
  e.s0 = o;
  e.s1 = o + b;
  e.d0 = o;
  e.d1 = o + b;
  e.g0 = e.g1 = e.e0 = e.e1 = 0;
  return e;
}

// The epilogue of steps (o, b) and (o1, b1) in one sweep.
EpiSchurF32 two_step_epi(float* X, int64_t ldx, int n, int o, int b, int o1, int b1, const int32_t* status) {
  EpiSchurF32 e = one_step_epi(X, ldx, n, o1, b1, status);
  e.g0 = e.e0 = o;
  e.g1 = e.e1 = o + b;
  return e;
}

template <int MAXB, bool kBF16>
cudaError_t launch_panel(float* X, int64_t ldx, int n, int o, int b, const float* Pinv, void* U, void* Vt,
                         int kpad, int nsl, int64_t ldop, const int32_t* status, cudaStream_t s) {
  using T = typename OpType<kBF16>::T;
  const int col_tiles = (n + kCols - 1) / kCols;
  // packing CTAs: about 16 columns of U per thread
  const int64_t pack_threads = ((int64_t)n * kpad / 16 + 255) / 256;
  const int grid = col_tiles + (int)std::max<int64_t>(8, std::min<int64_t>(pack_threads, 4096));
  const size_t smem = sizeof(float) * (2 * (size_t)kKc * (MAXB + 4) + 2 * kKc * kCols + (size_t)kCols * (MAXB + 1));
  auto k = row_panel_mixed_kernel<MAXB, kBF16>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, 256, smem, s>>>(X, ldx, n, o, b, Pinv, static_cast<T*>(U), static_cast<T*>(Vt), kpad, nsl, ldop,
                            status, col_tiles);
  return cudaGetLastError();
}

template <bool kBF16>
cudaError_t launch_panel_any(float* X, int64_t ldx, int n, int o, int b, const float* Pinv, void* U, void* Vt,
                             int kpad, int nsl, int64_t ldop, const int32_t* status, cudaStream_t s) {
  if (b <= 64) return launch_panel<64, kBF16>(X, ldx, n, o, b, Pinv, U, Vt, kpad, nsl, ldop, status, s);
  if (b <= 128) return launch_panel<128, kBF16>(X, ldx, n, o, b, Pinv, U, Vt, kpad, nsl, ldop, status, s);
  if (b <= 256) return launch_panel<256, kBF16>(X, ldx, n, o, b, Pinv, U, Vt, kpad, nsl, ldop, status, s);
  if (b <= 512) return launch_panel<512, kBF16>(X, ldx, n, o, b, Pinv, U, Vt, kpad, nsl, ldop, status, s);
  return cudaErrorInvalidValue;
}

// The Schur GEMM over the panels of `nsets` elimination steps (slice sets
// 0 .. nsets - 1 of U and Vt, nsl slices each: hi*hi, and hi*lo + lo*hi with
// the split, all three from split stages that hold both slices of both
// operands), kb k-blocks per set (64 bytes of K each with the split, else 128;
// tU and tV boxes to match), with the epilogue epi over the
// tiles of its part: the next pivot block's square (kInside), block row or
// column (kCrossRows, kCrossCols), or the whole matrix (kWhole, kOutside; the
// latter on at most max_ctas CTAs, with after_trigger as the programmatic
// dependent of the kernel before it).
template <tc::Kind K>
cudaError_t launch_schur_tc(const CUtensorMap& tU, const CUtensorMap& tV, const CUtensorMap& tX,
                            const EpiSchurF32& epi, int nsets, int nsl, int kb, int kpad, int32_t* status,
                            cudaStream_t s, int max_ctas = 0, bool after_trigger = false) {
  tc::KMap km{};
  km.kb_per_pair = kb;
  km.slice_cols = kpad;
  for (int t = 0; t < nsets; ++t) {
    km.pa[t] = (int8_t)(t * nsl);  // the first slice of set t
    km.pb[t] = (int8_t)(t * nsl);
  }
  km.kblocks = nsets * kb;
  tc::Window win;
  win.c_map = &tX;
  int M = epi.n, N = epi.n;
  switch (epi.part) {
    case kInside:
      win.m_base = epi.r0 / tc::kBM * tc::kBM;
      win.n_base = epi.r0 / tc::kBN * tc::kBN;
      M = epi.r1 - win.m_base;
      N = epi.r1 - win.n_base;
      break;
    case kCrossRows:
      win.m_base = epi.r0 / tc::kBM * tc::kBM;
      M = epi.r1 - win.m_base;
      break;
    case kCrossCols:
      win.n_base = epi.r0 / tc::kBN * tc::kBN;
      N = epi.r1 - win.n_base;
      break;
    case kOutside:
      win.max_ctas = max_ctas;
      win.after_trigger = after_trigger;
      break;
    default:
      break;
  }
  return nsl > 1 ? tc::launch_gemm<K, EpiSchurF32, true, tc::kPairTiles>(tU, tV, M, N, km, epi, status, s, win)
                 : tc::launch_gemm<K, EpiSchurF32, false, tc::kPairTiles>(tU, tV, M, N, km, epi, status, s, win);
}

}  // namespace

cudaError_t launch_cast_f64_to_f32(const double* A, int64_t lda, float* X, int64_t ldx, int n, cudaStream_t s) {
  if (rows_16b_aligned(A, lda, 8) && rows_16b_aligned(X, ldx, 4))
    cast_f64_to_f32_kernel<true><<<8 * tc::num_sms(), 256, 0, s>>>(A, lda, X, ldx, n);
  else
    cast_f64_to_f32_kernel<false><<<4 * tc::num_sms(), 256, 0, s>>>(A, lda, X, ldx, n);
  return cudaGetLastError();
}

cudaError_t launch_cast_f32_to_f64(const float* X, int64_t ldx, double* A, int64_t lda, int n, cudaStream_t s) {
  if (rows_16b_aligned(A, lda, 8) && rows_16b_aligned(X, ldx, 4))
    cast_f32_to_f64_kernel<true><<<8 * tc::num_sms(), 256, 0, s>>>(X, ldx, A, lda, n);
  else
    cast_f32_to_f64_kernel<false><<<4 * tc::num_sms(), 256, 0, s>>>(X, ldx, A, lda, n);
  return cudaGetLastError();
}

int mixed_kpad(int bmax) { return (bmax + 63) / 64 * 64; }

cudaError_t mixed_elimination(const Plan& mp, bool bf16, int nsl, float* X32, int64_t ld32, float* Pinv, void* U,
                              void* Vt, float pivot_cond_limit, int32_t* piv_words, int32_t* status, cudaStream_t s,
                              bool lookahead, bool fuse) {
  const int n = mp.n;
  const int p = (int)mp.sizes.size();
  const int kpad = mixed_kpad(mp.bmax);
  const int eb = bf16 ? 2 : 4;
  const CUtensorMapDataType dt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  // K elements per k-block of the Schur GEMM: 64 bytes in the split stages
  const int BK = (nsl > 1 ? 64 : 128) / eb;
  // U and Vt rows: two slice sets of nsl slices of kpad columns (the panels of
  // two consecutive steps; one step uses set 0)
  const int64_t ldop = 2ll * nsl * kpad;
  unsigned char* Uset[2] = {static_cast<unsigned char*>(U), static_cast<unsigned char*>(U) + (size_t)nsl * kpad * eb};
  unsigned char* Vset[2] = {static_cast<unsigned char*>(Vt), static_cast<unsigned char*>(Vt) + (size_t)nsl * kpad * eb};
  CUtensorMap tU, tV;
  // X32 itself in 32 x 32 blocks for the update's epilogue (rows of ld32
  // floats, a multiple of 128 bytes)
  CUtensorMap tX;
  if (!make_tmap_2d(&tU, U, dt, (uint64_t)ldop, n, (uint64_t)ldop * eb, BK, tc::kBM, nsl > 1) ||
      !make_tmap_2d(&tV, Vt, dt, (uint64_t)ldop, n, (uint64_t)ldop * eb, BK, tc::b_rows<tc::kPairTiles>(),
                    nsl > 1) ||
      !make_tmap_2d(&tX, X32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, n, n, (uint64_t)ld32 * 4, 32, 32))
    return cudaErrorInvalidValue;
  const bool check = pivot_cond_limit != 0.f && piv_words;
  auto pivot = [&](int k) -> cudaError_t {
    const int o = mp.offs[k], b = mp.sizes[k];
    const double bd = b;
    TraceScope t("pivot_inverse_f32", 2.0 * bd * bd * bd, 8.0 * bd * bd, s);
    return launch_pivot_inverse<float>(X32 + (int64_t)o * ld32 + o, ld32, b, Pinv, b, status, k, s);
  };
  // FP64 arithmetic for the pivot blocks that the condition estimate flags:
  // the estimate, then the gated FP64 inverse
  auto pivot_cond = [&](int k, bool after_trigger) -> cudaError_t {
    if (!check) return cudaSuccess;
    const int o = mp.offs[k], b = mp.sizes[k];
    const double bd = b;
    TraceScope t("pivot_cond_estimate", 0, 8.0 * bd * bd, s);
    return launch_pivot_cond(X32 + (int64_t)o * ld32 + o, ld32, b, Pinv, b, status, pivot_cond_limit, piv_words,
                             piv_words + 1, after_trigger, s);
  };
  auto pivot_gated = [&](int k) -> cudaError_t {
    if (!check) return cudaSuccess;
    const int o = mp.offs[k], b = mp.sizes[k];
    const double bd = b;
    TraceScope t("pivot_f64_if_ill", 0, 8.0 * bd * bd, s);
    return launch_pivot_f64_gated(X32 + (int64_t)o * ld32 + o, ld32, b, Pinv, b, status, k, piv_words, s);
  };
  auto panel = [&](int k, int set) -> cudaError_t {
    const int o = mp.offs[k], b = mp.sizes[k];
    const double bd = b, nd = n, rest = n - b;
    TraceScope t("row_panel_mixed", 2.0 * bd * bd * rest, 4.0 * (2.0 * bd * nd + bd * bd + rest * bd) + eb * 2.0 * nd * kpad, s);
    return bf16 ? launch_panel_any<true>(X32, ld32, n, o, b, Pinv, Uset[set], Vset[set], kpad, nsl, ldop, status, s)
                : launch_panel_any<false>(X32, ld32, n, o, b, Pinv, Uset[set], Vset[set], kpad, nsl, ldop, status, s);
  };
  // a Schur GEMM launch: `elems` updated elements, `kdepth` = b summed over its steps
  auto gemm = [&](const char* name, const EpiSchurF32& epi, int nsets, int kb, double elems, double kdepth,
                  int max_ctas, bool after_trigger) -> cudaError_t {
    TraceScope t(name, 2.0 * kdepth * elems * (nsl > 1 ? 3 : 1), 4.0 * 2.0 * elems + eb * 2.0 * n * kdepth * nsl, s);
    return bf16 ? launch_schur_tc<tc::Kind::BF16>(tU, tV, tX, epi, nsets, nsl, kb, kpad, status, s, max_ctas,
                                                  after_trigger)
                : launch_schur_tc<tc::Kind::TF32>(tU, tV, tX, epi, nsets, nsl, kb, kpad, status, s, max_ctas,
                                                  after_trigger);
  };
  auto kblocks = [&](int b) { return (b + BK - 1) / BK; };
  const char* nm_next = bf16 ? "schur_next_block_bf16_tc" : "schur_next_block_tf32_tc";
  const char* nm_rest = bf16 ? "schur_update_bf16_tc" : "schur_update_tf32_tc";
  const char* nm_cross = bf16 ? "schur_cross_bf16_tc" : "schur_cross_tf32_tc";
  // Step k's update over everything but the pivot rows with set `set`, or,
  // split around the next pivot block's square (look-ahead), its square, the
  // next FP32 pivot inverse and its condition estimate by programmatic
  // dependent launch beside the rest. The pivot reads the square and writes
  // Pinv, the estimate reads both and writes the gate; the rest of the update
  // neither loads nor stores the 32 x 32 blocks of X wholly inside the square,
  // and stores a block straddling its edge (orders not multiples of 32) with
  // the square's bytes as loaded, so the pivot reads the same values either
  // way. The gated FP64 inverse follows.
  auto sweep_then_pivot = [&](EpiSchurF32 epi, int nsets, int kb, double kdepth, int knext,
                              bool split) -> cudaError_t {
    const double nd = n, rows = n - (epi.s1 - epi.s0);
    cudaError_t e;
    if (!split) {
      epi.part = kWhole;
      e = gemm(nm_rest, epi, nsets, kb, rows * nd, kdepth, 0, false);
      if (e == cudaSuccess && knext < p) e = pivot(knext);
      if (e == cudaSuccess && knext < p) e = pivot_cond(knext, false);
    } else {
      const int o1 = mp.offs[knext], b1 = mp.sizes[knext];
      const double inside = (double)b1 * b1;
      epi.r0 = o1;
      epi.r1 = o1 + b1;
      epi.part = kInside;
      e = gemm(nm_next, epi, nsets, kb, inside, kdepth, 0, false);
      if (e == cudaSuccess) e = pivot(knext);
      if (e == cudaSuccess) e = pivot_cond(knext, true);
      const int reserve = pivot_inverse_ctas(b1, 4, false) + (check ? 1 : 0);
      epi.part = kOutside;
      if (e == cudaSuccess) e = gemm(nm_rest, epi, nsets, kb, rows * nd - inside, kdepth, tc::num_sms() - reserve, true);
    }
    if (e == cudaSuccess && knext < p) e = pivot_gated(knext);
    return e;
  };
  const bool ahead = lookahead && p >= 3;
  cudaError_t e = pivot(0);
  if (e == cudaSuccess) e = pivot_cond(0, false);
  if (e == cudaSuccess) e = pivot_gated(0);
  if (!(fuse && p >= 2)) {
    // one step per sweep over X
    for (int k = 0; k < p && e == cudaSuccess; ++k) {
      const int o = mp.offs[k], b = mp.sizes[k];
      e = panel(k, 0);
      if (e != cudaSuccess || n == b) continue;
      e = sweep_then_pivot(one_step_epi(X32, ld32, n, o, b, status), 1, kblocks(b), b, k + 1,
                           ahead && k + 1 < p);
    }
    return e;
  }
  // Two steps per sweep (steps k, k + 1 with K = block k, L = block k + 1):
  //   row panel k (set 0);
  //   step k on block row L and block column L only (two windowed launches);
  //   pivot inverse of L; Vt of set 0 zeroed in the rows of L; row panel
  //   k + 1 (set 1, from the updated block row and column L);
  //   one rank-(b_k + b_L) sweep over the rest of X with both sets:
  //     X <- (drop ? 0 : X) - U_k Vt_k^T - U_L Vt_L^T,
  //   dropping block columns K and L (only L in the rows of K, which hold
  //   row panel k) and leaving the rows of L (row panel k + 1) alone.
  // Every element of the rest gets the same two rank-b products as two
  // separate steps, summed in one FP32 accumulator instead of rounded to
  // X32 in between. With an odd block count the last step runs alone.
  for (int k = 0; k < p && e == cudaSuccess; k += 2) {
    const int o = mp.offs[k], b = mp.sizes[k];
    e = panel(k, 0);
    if (e != cudaSuccess) break;
    if (k + 1 == p) {
      if (n != b) e = sweep_then_pivot(one_step_epi(X32, ld32, n, o, b, status), 1, kblocks(b), b, p, false);
      break;
    }
    const int o1 = mp.offs[k + 1], b1 = mp.sizes[k + 1];
    const double nd = n, bd = b;
    EpiSchurF32 cross = one_step_epi(X32, ld32, n, o, b, status);
    cross.r0 = o1;
    cross.r1 = o1 + b1;
    cross.part = kCrossRows;
    e = gemm(nm_cross, cross, 1, kblocks(b), (double)b1 * nd, bd, 0, false);
    cross.part = kCrossCols;
    if (e == cudaSuccess) e = gemm(nm_cross, cross, 1, kblocks(b), (double)b1 * (nd - b1 - bd), bd, 0, false);
    if (e == cudaSuccess) e = pivot(k + 1);
    if (e == cudaSuccess) e = pivot_cond(k + 1, false);
    if (e == cudaSuccess) e = pivot_gated(k + 1);
    if (e == cudaSuccess)
      e = cudaMemset2DAsync(Vset[0] + (size_t)o1 * ldop * eb, (size_t)ldop * eb, 0, (size_t)nsl * kpad * eb, b1, s);
    if (e == cudaSuccess) e = panel(k + 1, 1);
    if (e != cudaSuccess) break;
    // (with two blocks only, the sweep still updates the rows of block k)
    e = sweep_then_pivot(two_step_epi(X32, ld32, n, o, b, o1, b1, status), 2, kblocks(std::max(b, b1)),
                         (double)b + b1, k + 2, ahead && k + 2 < p);
  }
  return e;
}

}  // namespace blockinv
