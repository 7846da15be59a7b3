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
__global__ void cast_f64_to_f32_kernel(const double* __restrict__ A, int64_t lda, float* __restrict__ X,
                                       int64_t ldx, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const double* a = A + (int64_t)i * lda;
    float* x = X + (int64_t)i * ldx;
#pragma unroll 4
    for (int j = threadIdx.x; j < ldx; j += blockDim.x) x[j] = (j < n) ? (float)a[j] : 0.f;
  }
}

__global__ void cast_f32_to_f64_kernel(const float* __restrict__ X, int64_t ldx, double* __restrict__ A,
                                       int64_t lda, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const float* x = X + (int64_t)i * ldx;
    double* a = A + (int64_t)i * lda;
#pragma unroll 4
    for (int j = threadIdx.x; j < n; j += blockDim.x) a[j] = (double)x[j];
  }
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
template <int MAXB, bool kBF16>
__global__ void __launch_bounds__(256)
row_panel_mixed_kernel(float* __restrict__ X, int64_t ldx, int n, int o, int b, const float* __restrict__ Pinv,
                       typename OpType<kBF16>::T* __restrict__ U, typename OpType<kBF16>::T* __restrict__ Vt,
                       int kpad, int nsl, const int32_t* status, int col_tiles) {
  using Op = OpType<kBF16>;
  if (failed(status)) return;
  const int tid = threadIdx.x;
  const int64_t ldop = (int64_t)nsl * kpad;
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
// Elements written: every row outside the pivot rows [o, o + b); with
// part = kInside only those of the square [r0, r1) x [r0, r1) (the next
// pivot block), with part = kOutside all but those.
enum SchurPart { kWhole = 0, kInside = 1, kOutside = 2 };

struct EpiSchurF32 {
  float* X;
  int64_t ldx;
  int n, o, b;
  const int32_t* status;
  int part = kWhole;
  int r0 = 0, r1 = 0;
  // The GEMM moves X's 32 x 32 blocks by TMA and asks value() per element.
  static constexpr bool kTmaC = true;
  __device__ bool skip() const { return failed(status); }
  // The new value of X[row][col] from its current value x and the product v
  // (x itself where this launch writes nothing).
  __device__ float value(int row, int col, float x, float v) const {
    if (col >= n) return x;
    const bool col_in = col >= r0 && col < r1;
    if (!writes(row, col_in)) return x;
    const bool pivot_col = col >= o && col < o + b;
    return (pivot_col ? 0.f : x) - v;
  }
  // Whether value() changes any element of the 32 x 32 block at (row0, col0):
  // blocks of pivot rows only, past the matrix, outside the square (kInside)
  // or wholly inside it (kOutside) are neither loaded nor stored.
  __device__ bool block_live(int row0, int col0) const {
    if (row0 >= n || col0 >= n) return false;
    const int rend = min(row0 + 32, n), cend = min(col0 + 32, n);
    if (row0 >= o && rend <= o + b) return false;
    if (part == kWhole) return true;
    const bool rows_meet = row0 < r1 && rend > r0, cols_meet = col0 < r1 && cend > r0;
    if (part == kInside) return rows_meet && cols_meet;
    return !(row0 >= r0 && rend <= r1 && col0 >= r0 && cend <= r1);
  }
  __device__ bool writes(int row, bool col_in) const {
    if (row >= n || (row >= o && row < o + b)) return false;
    if (part == kWhole) return true;
    const bool in = col_in && row >= r0 && row < r1;
    return part == kInside ? in : !in;
  }
  __device__ void apply_cols(int row0, int col, const float (&v)[32], int chunk, int nchunks) const {
    if (col >= n) return;
    const bool pivot_col = col >= o && col < o + b;
    const bool col_in = col >= r0 && col < r1;
    if (part == kInside && !col_in) return;
    float* p = X + (int64_t)row0 * ldx + col;
    // all loads before any store, so the 32 reads are in flight together
    float cur[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) cur[r] = (writes(row0 + r, col_in) && !pivot_col) ? p[(int64_t)r * ldx] : 0.f;
#pragma unroll
    for (int r = 0; r < 32; ++r)
      if (writes(row0 + r, col_in)) p[(int64_t)r * ldx] = cur[r] - v[r];
  }
};

template <int MAXB, bool kBF16>
cudaError_t launch_panel(float* X, int64_t ldx, int n, int o, int b, const float* Pinv, void* U, void* Vt,
                         int kpad, int nsl, const int32_t* status, cudaStream_t s) {
  using T = typename OpType<kBF16>::T;
  const int col_tiles = (n + kCols - 1) / kCols;
  // packing CTAs: about 16 columns of U per thread
  const int64_t pack_threads = ((int64_t)n * kpad / 16 + 255) / 256;
  const int grid = col_tiles + (int)std::max<int64_t>(8, std::min<int64_t>(pack_threads, 4096));
  const size_t smem = sizeof(float) * (2 * (size_t)kKc * (MAXB + 4) + 2 * kKc * kCols + (size_t)kCols * (MAXB + 1));
  auto k = row_panel_mixed_kernel<MAXB, kBF16>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, 256, smem, s>>>(X, ldx, n, o, b, Pinv, static_cast<T*>(U), static_cast<T*>(Vt), kpad, nsl, status,
                            col_tiles);
  return cudaGetLastError();
}

template <bool kBF16>
cudaError_t launch_panel_any(float* X, int64_t ldx, int n, int o, int b, const float* Pinv, void* U, void* Vt,
                             int kpad, int nsl, const int32_t* status, cudaStream_t s) {
  if (b <= 64) return launch_panel<64, kBF16>(X, ldx, n, o, b, Pinv, U, Vt, kpad, nsl, status, s);
  if (b <= 128) return launch_panel<128, kBF16>(X, ldx, n, o, b, Pinv, U, Vt, kpad, nsl, status, s);
  if (b <= 256) return launch_panel<256, kBF16>(X, ldx, n, o, b, Pinv, U, Vt, kpad, nsl, status, s);
  if (b <= 512) return launch_panel<512, kBF16>(X, ldx, n, o, b, Pinv, U, Vt, kpad, nsl, status, s);
  return cudaErrorInvalidValue;
}

// The Schur update of step (o, b): the whole of it (part = kWhole), or the
// square [o1, o1 + b1)^2 of the next pivot block (kInside: only the tiles
// that cover it), or everything else (kOutside, on at most max_ctas CTAs,
// with after_trigger as the programmatic dependent of the kernel before it).
template <tc::Kind K>
cudaError_t launch_schur_tc(const CUtensorMap& tU, const CUtensorMap& tV, const CUtensorMap& tX, float* X, int64_t ldx,
                            int n, int o, int b, int kpad, int nsl, int32_t* status, cudaStream_t s, int part = kWhole,
                            int o1 = 0, int b1 = 0, int max_ctas = 0, bool after_trigger = false) {
  constexpr int BK = 128 / tc::KindTraits<K>::elem_bytes;
  const int kb = (b + BK - 1) / BK;
  tc::KMap km = tc::plain_kmap(kb);
  if (nsl > 1) {  // hi*hi + hi*lo + lo*hi
    km.kb_per_pair = kb;
    km.slice_cols = kpad;
    km.kblocks = 3 * kb;
    km.pa[0] = 0; km.pb[0] = 0;
    km.pa[1] = 0; km.pb[1] = 1;
    km.pa[2] = 1; km.pb[2] = 0;
  }
  EpiSchurF32 epi{X, ldx, n, o, b, status, part, o1, o1 + b1};
  tc::Window win;
  win.c_map = &tX;
  int M = n, N = n;
  if (part == kInside) {
    win.m_base = o1 / tc::kBM * tc::kBM;
    win.n_base = o1 / tc::kBN * tc::kBN;
    M = o1 + b1 - win.m_base;
    N = o1 + b1 - win.n_base;
  } else if (part == kOutside) {
    win.max_ctas = max_ctas;
    win.after_trigger = after_trigger;
  }
  return tc::launch_gemm<K, EpiSchurF32>(tU, tV, M, N, km, epi, status, s, win);
}

}  // namespace

cudaError_t launch_cast_f64_to_f32(const double* A, int64_t lda, float* X, int64_t ldx, int n, cudaStream_t s) {
  cast_f64_to_f32_kernel<<<4 * tc::num_sms(), 256, 0, s>>>(A, lda, X, ldx, n);
  return cudaGetLastError();
}

cudaError_t launch_cast_f32_to_f64(const float* X, int64_t ldx, double* A, int64_t lda, int n, cudaStream_t s) {
  cast_f32_to_f64_kernel<<<4 * tc::num_sms(), 256, 0, s>>>(X, ldx, A, lda, n);
  return cudaGetLastError();
}

int mixed_kpad(int bmax) { return (bmax + 63) / 64 * 64; }

cudaError_t mixed_elimination(const Plan& mp, bool bf16, int nsl, float* X32, int64_t ld32, float* Pinv, void* U,
                              void* Vt, float pivot_cond_limit, int32_t* piv_words, int32_t* status, cudaStream_t s,
                              bool lookahead) {
  const int n = mp.n;
  const int p = (int)mp.sizes.size();
  const int kpad = mixed_kpad(mp.bmax);
  const int eb = bf16 ? 2 : 4;
  const CUtensorMapDataType dt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const uint32_t BK = 128 / eb;
  const uint64_t w = (uint64_t)nsl * kpad;
  CUtensorMap tU, tV;
  // X32 itself in 32 x 32 blocks for the update's epilogue (rows of ld32
  // floats, a multiple of 128 bytes)
  CUtensorMap tX;
  if (!make_tmap_2d(&tU, U, dt, w, n, w * eb, BK, tc::kBM) ||
      !make_tmap_2d(&tV, Vt, dt, w, n, w * eb, BK, tc::kBN) ||
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
  auto schur = [&](int k, int part, int k1, int max_ctas, bool after_trigger) -> cudaError_t {
    const int o = mp.offs[k], b = mp.sizes[k];
    const int o1 = k1 >= 0 ? mp.offs[k1] : 0, b1 = k1 >= 0 ? mp.sizes[k1] : 0;
    const double bd = b, nd = n, rest = n - b;
    const double inside = (double)b1 * b1, elems = part == kWhole ? rest * nd
                                                   : part == kInside ? inside : rest * nd - inside;
    const char* name = part == kInside ? (bf16 ? "schur_next_block_bf16_tc" : "schur_next_block_tf32_tc")
                                       : (bf16 ? "schur_update_bf16_tc" : "schur_update_tf32_tc");
    TraceScope t(name, 2.0 * bd * elems * (nsl > 1 ? 3 : 1), 4.0 * 2.0 * elems + eb * 2.0 * nd * bd * nsl, s);
    return bf16 ? launch_schur_tc<tc::Kind::BF16>(tU, tV, tX, X32, ld32, n, o, b, kpad, nsl, status, s, part, o1,
                                                  b1, max_ctas, after_trigger)
                : launch_schur_tc<tc::Kind::TF32>(tU, tV, tX, X32, ld32, n, o, b, kpad, nsl, status, s, part, o1,
                                                  b1, max_ctas, after_trigger);
  };
  // One-step look-ahead: step k's Schur update is split into the next pivot
  // block's square and the rest. The next FP32 pivot inverse follows the
  // square and starts its programmatic dependent, the condition estimate,
  // which starts its own, the rest of the update, at once: they share the GPU
  // (the update on as many fewer SMs as the other two take). The pivot reads
  // the square and writes Pinv, the estimate reads both and writes the gate.
  // The rest of the update neither loads nor stores the 32 x 32 blocks of X
  // that lie wholly inside the square; a block that straddles its edge (a
  // block order that is not a multiple of 32) is stored back with the
  // square's bytes as loaded, so the pivot reads the same values either way.
  // The gated FP64 inverse and the next row panel (which overwrites U and Vt)
  // follow.
  const bool ahead = lookahead && p >= 3;
  cudaError_t e = pivot(0);
  if (e == cudaSuccess) e = pivot_cond(0, false);
  if (e == cudaSuccess) e = pivot_gated(0);
  for (int k = 0; k < p && e == cudaSuccess; ++k) {
    const int o = mp.offs[k], b = mp.sizes[k];
    const double bd = b, nd = n, rest = n - b;
    {
      TraceScope t("row_panel_mixed", 2.0 * bd * bd * rest, 4.0 * (2.0 * bd * nd + bd * bd + rest * bd) + eb * 2.0 * nd * kpad, s);
      e = bf16 ? launch_panel_any<true>(X32, ld32, n, o, b, Pinv, U, Vt, kpad, nsl, status, s)
               : launch_panel_any<false>(X32, ld32, n, o, b, Pinv, U, Vt, kpad, nsl, status, s);
    }
    if (e != cudaSuccess || n == b) continue;
    if (!ahead || k + 1 == p) {
      e = schur(k, kWhole, -1, 0, false);
      if (e == cudaSuccess && k + 1 < p) e = pivot(k + 1);
      if (e == cudaSuccess && k + 1 < p) e = pivot_cond(k + 1, false);
    } else {
      e = schur(k, kInside, k + 1, 0, false);
      if (e == cudaSuccess) e = pivot(k + 1);
      if (e == cudaSuccess) e = pivot_cond(k + 1, true);
      const int reserve = pivot_inverse_ctas(mp.sizes[k + 1], 4, false) + (check ? 1 : 0);
      if (e == cudaSuccess) e = schur(k, kOutside, k + 1, tc::num_sms() - reserve, true);
    }
    if (e == cudaSuccess && k + 1 < p) e = pivot_gated(k + 1);
  }
  return e;
}

}  // namespace blockinv
