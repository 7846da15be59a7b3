// Newton-Schulz refinement of an approximate inverse, X <- X + X (I - A X)
// (the same step as X (2I - A X)), with the residual E = I - A X computed to
// FP64 accuracy on the FP8 tensor cores.
//
// FP64-accurate residual (error-free splitting, after Ozaki et al.'s scheme
// for accurate matrix products). The diagonals are split off first:
// A = D_A + O_A, X = D_X + O_X, and
//
//   A X = D_A X + O_A D_X + O_A O_X,
//
// where the first two terms are elementwise FP64 products (a_ii x_ij and
// a_ij x_jj) and only O_A O_X needs a matrix product. Scaling the rows of O_A
// and the columns of O_X by their own maxima, rather than by a dominant
// diagonal, keeps the bits of the off-diagonal entries. Every row i of O_A is
// scaled by a power of two 2^-e_i (e_i the smallest integer with
// max_k |a_ik| < 2^e_i, k != i) and every column j of O_X by 2^-f_j; the
// scaled values, as fixed-point numbers with F = 5S - 1 fraction bits, are cut
// into S signed base-32 digits (the leading digit in [-16, 16], the others in
// [-16, 15]); every digit is an integer of magnitude <= 16, exact in FP8 E4M3.
// Then
//
//   (O_A O_X)_ij ~= 2^(e_i + f_j - 2F) sum_g 32^(2S - 2 - g) G_g(i, j),
//   G_g = sum_{p + q = g} Adigits_p Xdigits_q^T      (g = 0 .. S - 1),
//
// where each digit product is at most 2^8 in magnitude, so a GEMM over P digit
// pairs with n <= 2^16 / P terms each keeps every partial sum below 2^24 and
// the FP32 tensor-core accumulator holds it exactly. Group g is one GEMM (or
// several, when g + 1 pairs exceed that bound); the epilogue adds its result
// << 5 (S - 1 - g) into an int64 accumulator, again exactly: with S <= 9 and
// n <= 16384 every sum stays below 2^(22 + 40 + 0.1) < 2^63. The finalize kernel converts to FP64, forms E = I - A X, its
// Frobenius norm and the operands of the update. Dropped groups (p + q >= S)
// and the rounding of the fixed-point values leave an error of order
// 2^(-F) S sqrt(K) relative to the row and column scales.
//
// Both products run on the persistent tcgen05 GEMM (one CTA per output tile).
// The update X += X E uses split TF32 operands (hi + lo for X and E, the
// three products hi*hi + hi*lo + lo*hi) with the FP32 accumulator added to
// the FP64 X in the epilogue, one K-chunk at a time; E is small, so the
// correction needs far fewer bits than X itself.
//
// The iteration is stream-ordered: after each residual a one-thread kernel
// computes rho = ||E||_F / (||A||_F ||X||_F), records it, and raises a device
// flag when rho <= tol, when rho fails to drop by 4x (no contraction), or at
// the iteration cap. Every later kernel of the refinement returns at once
// when the flag is up.
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <climits>
#include <cstddef>

#include "tc_gemm.cuh"

namespace blockinv {

namespace {

constexpr int kLog2Digit = 5;  // base-32 digits
constexpr int kHeadroom = 1;   // fraction bits F = 5 S - 1 keep the leading digit within [-16, 16]
constexpr int kUpdateChunkK = 2048;  // K elements per accumulator hand-off in the update
// Incremental residual E_new = E - A (X_new - X), used after a residual with
// ||E||_F <= kIncrMaxE: the change of X is cut into S base-32 digits like X,
// and only the leading G digit groups are multiplied. With D the smallest
// difference, over the columns, between the exponent bounds of X and of the
// change, dropping the groups after G = S - floor(D / 5) costs no more than
// the fresh residual's own rounding of X (2^(c - 5 S) for a column bound 2^c),
// so E_new has the fresh residual's error floor; a change 2^-18 of X leaves
// 6 groups (21 digit products instead of 45).
constexpr double kIncrMaxE = 1e-3;

struct Ctl {
  int32_t done;        // refinement finished (converged or gave up)
  int32_t updates;     // updates applied
  int32_t code;        // BLOCKINV_OK or BLOCKINV_ERR_NOT_CONVERGED once done
  int32_t last;        // index of the last residual computed
  int32_t inc;         // the next residual is incremental (E_new = E - A (X_new - X))
  int32_t incs;        // incremental residuals computed
  int32_t groups;      // digit groups of the last incremental residual
};
static_assert(sizeof(Ctl) <= sizeof(int32_t) * kRefineCtlWords, "refinement control words");

// Which residual a kernel belongs to: every one, the fresh one (all digits of
// X) or the incremental one (digits of the change of X).
enum Path { kAny = 0, kFresh = 1, kIncr = 2 };

__device__ __forceinline__ bool halted(const Ctl* ctl, const int32_t* status, int path = kAny) {
  if (*(volatile const int32_t*)&ctl->done != 0 || *(volatile const int32_t*)status != 0) return true;
  if (path == kAny) return false;
  const bool inc = *(volatile const int32_t*)&ctl->inc != 0;
  return path == kFresh ? inc : !inc;
}

// Smallest e with |v| < 2^e for normal v (from the exponent field); very
// negative for zero.
__device__ __forceinline__ int exp_bound(double v) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  return static_cast<int>((bits >> 52) & 0x7FF) - 1022;
}

// Fixed-point integer round(v * 2^(F - e)), F = 5S - 1, from the bit pattern,
// |v| < 2^e.
__device__ __forceinline__ long long fixed_point(double v, int e, int S) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  const int ef = static_cast<int>((bits >> 52) & 0x7FF);
  if (ef == 0) return 0;  // zero or subnormal: below every digit kept
  const long long m = static_cast<long long>((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  // v = m * 2^(ef - 1075); shift = ef - 1075 + F - e (always negative here)
  const int sh = ef - 1075 + kLog2Digit * S - kHeadroom - e;
  long long q;
  if (sh >= 0) {
    q = m << sh;
  } else if (sh <= -62) {
    q = 0;
  } else {
    q = (m + (1ll << (-sh - 1))) >> (-sh);
  }
  return (bits >> 63) ? -q : q;
}

// E4M3 byte of an integer |d| <= 16 (exact). The hardware conversion is
// faster here than assembling the byte on the integer pipe (measured).
__device__ __forceinline__ uint8_t e4m3(int d) {
  return static_cast<uint8_t>(__nv_cvt_float_to_fp8(static_cast<float>(d), __NV_SATFINITE, __NV_E4M3));
}

// Balanced base-32 digits of q (|q| <= 2^(5S - 1)), most significant first:
// d[1..S-1] in [-16, 15], and d[0] in [-16, 16] since the lower digits sum to
// less than half a unit of the leading one; q = sum_p d[p] 32^(S-1-p).
// Adding 16 at each of the S - 1 lower digit positions makes those digits
// plain 5-bit fields (d + 16 in [0, 31], no carries), read with 32-bit shifts;
// the top digit is what remains above them.
template <int S>
__device__ __forceinline__ void digits(long long q, int (&d)[S]) {
  constexpr long long kBias = 16 * (((1ll << (kLog2Digit * (S - 1))) - 1) / 31);  // 16 * sum_{p < S-1} 32^p
  const long long qb = q + kBias;
  const unsigned lo = static_cast<unsigned>(qb);
  const unsigned hi = static_cast<unsigned>(static_cast<unsigned long long>(qb) >> 32);
#pragma unroll
  for (int p = 0; p < S - 1; ++p) {  // field p (from the least significant) is digit S - 1 - p
    const int sh = kLog2Digit * p;
    unsigned f;
    if (sh + kLog2Digit <= 32)
      f = lo >> sh;
    else if (sh >= 32)
      f = hi >> (sh - 32);
    else
      f = __funnelshift_r(lo, hi, sh);
    d[S - 1 - p] = static_cast<int>(f & 31u) - 16;
  }
  d[0] = static_cast<int>(qb >> (kLog2Digit * (S - 1)));
}

// ---------------------------------------------------------- scales -------
// One warp per row: e_i = max exponent bound over the row, and sum of squares.
__global__ void row_scale_kernel(const double* __restrict__ M, int64_t ld, int n, int32_t* __restrict__ rexp,
                                 double* __restrict__ sumsq, const Ctl* ctl, const int32_t* status) {
  if (halted(ctl, status)) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = M + (int64_t)warp * ld;
  int e = -2000;
  double s2 = 0.0;
  for (int k = lane; k < n; k += 32) {
    const double v = row[k];
    if (k != warp) e = max(e, exp_bound(v));
    s2 = fma(v, v, s2);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  }
  if (lane == 0) {
    rexp[warp] = e;
    atomicAdd(sumsq, s2);
  }
}

// Column exponent bounds (atomicMax per column after a CTA reduction) and the
// sum of squares. cexp must hold a very negative value beforehand.
__global__ void col_scale_kernel(const double* __restrict__ X, int64_t ld, int n, int32_t* __restrict__ cexp,
                                 double* __restrict__ sumsq, const Ctl* ctl, const int32_t* status, int path) {
  if (halted(ctl, status, path)) return;
  __shared__ int se[8][32];
  __shared__ double ss[8];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + tx;
  const int r0 = blockIdx.y * 256;
  int e = -2000;
  double s2 = 0.0;
  if (j < n) {
    for (int r = r0 + ty; r < min(n, r0 + 256); r += 8) {
      const double v = X[(int64_t)r * ld + j];
      if (r != j) e = max(e, exp_bound(v));
      s2 = fma(v, v, s2);
    }
  }
  se[ty][tx] = e;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  if (tx == 0) ss[ty] = s2;
  __syncthreads();
  if (ty == 0) {
    int m = se[0][tx];
    for (int y = 1; y < 8; ++y) m = max(m, se[y][tx]);
    if (j < n) atomicMax(&cexp[j], m);
    if (tx == 0 && sumsq) {
      double t = 0.0;
      for (int y = 0; y < 8; ++y) t += ss[y];
      atomicAdd(sumsq, t);
    }
  }
}

// ---------------------------------------------------------- slicing ------
// Row slices: out[i][p * Kp + k] = digit p of A[i][k] / 2^e_i (k < n), 4 k per thread.
template <int S>
__global__ void slice_rows_kernel(const double* __restrict__ M, int64_t ld, int n, const int32_t* __restrict__ rexp,
                                  int Kp, uint8_t* __restrict__ out, const Ctl* ctl, const int32_t* status) {
  if (halted(ctl, status)) return;
  const int64_t quads = (int64_t)n * (Kp / 4);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < quads; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / (Kp / 4));
    const int k0 = (int)(t - (int64_t)i * (Kp / 4)) * 4;
    const int e = rexp[i];
    uint32_t w[S];
#pragma unroll
    for (int p = 0; p < S; ++p) w[p] = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int k = k0 + c;
      if (k < n) {
        int d[S];
        digits<S>(fixed_point(k == i ? 0.0 : M[(int64_t)i * ld + k], e, S), d);
#pragma unroll
        for (int p = 0; p < S; ++p) w[p] |= static_cast<uint32_t>(e4m3(d[p])) << (8 * c);
      }
    }
    uint8_t* base = out + (int64_t)i * S * Kp + k0;
#pragma unroll
    for (int p = 0; p < S; ++p) *reinterpret_cast<uint32_t*>(base + (int64_t)p * Kp) = w[p];
  }
}

// Transposed column slices: out[j][q * Kp + k] = digit q of X[k][j] / 2^f_j.
// Tiles of 64 k x 32 j through shared memory.
template <int S>
__global__ void __launch_bounds__(256)
slice_cols_t_kernel(const double* __restrict__ X, int64_t ld, int n, const int32_t* __restrict__ cexp, int Kp,
                    uint8_t* __restrict__ out, const Ctl* ctl, const int32_t* status, int path) {
  if (halted(ctl, status, path)) return;
  __shared__ uint8_t sd[S][32][68];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j0 = blockIdx.x * 32, k0 = blockIdx.y * 64;
  const int j = j0 + tx;
  const int f = (j < n) ? cexp[j] : 0;
  for (int kk = ty; kk < 64; kk += 8) {
    const int k = k0 + kk;
    int d[S];
    const double v = (j < n && k < n && k != j) ? X[(int64_t)k * ld + j] : 0.0;
    digits<S>(fixed_point(v, f, S), d);
#pragma unroll
    for (int p = 0; p < S; ++p) sd[p][tx][kk] = e4m3(d[p]);
  }
  __syncthreads();
  // write: each (p, jj) row segment of 64 bytes = 16 words; 256 threads -> 16 (p, jj) per pass
  for (int t = threadIdx.x; t < S * 32 * 16; t += 256) {
    const int w = t & 15;
    const int jj = (t >> 4) & 31;
    const int p = t >> 9;
    const int jg = j0 + jj;
    if (jg < n) {
      const uint32_t word = *reinterpret_cast<const uint32_t*>(&sd[p][jj][w * 4]);
      *reinterpret_cast<uint32_t*>(out + (int64_t)jg * S * Kp + (int64_t)p * Kp + k0 + w * 4) = word;
    }
  }
}

// -------------------------------------------------------- epilogues ------
// T (int64) gets every digit group of a residual, each exact in the FP32
// accumulator: chunk c of a tile belongs to group g = chunk_group(starts, c)
// and is added shifted left by 5 (groups - 1 - g) bits; chunk 0 overwrites.
struct EpiAccumI64 {
  static constexpr bool kTmaC = false;  // updated through apply_cols
  long long* T;
  int64_t ldt;
  int n;
  int groups;
  uint32_t group_starts;
  const Ctl* ctl;
  const int32_t* status;
  int path;
  __device__ bool skip() const { return halted(ctl, status, path); }
  __device__ void apply_cols(int row0, int col, const float (&v)[32], int chunk, int nchunks) const {
    if (col >= n) return;
    const int shift = kLog2Digit * (groups - 1 - tc::chunk_group(group_starts, chunk));
    const bool first = chunk == 0;
    long long* p = T + (int64_t)row0 * ldt + col;
    // two halves of 16 rows: all loads of a half before its stores
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
      long long cur[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) cur[r] = (!first && row0 + h + r < n) ? p[(int64_t)(h + r) * ldt] : 0;
#pragma unroll
      for (int r = 0; r < 16; ++r)
        if (row0 + h + r < n) p[(int64_t)(h + r) * ldt] = cur[r] + (static_cast<long long>(__float2ll_rn(v[h + r])) << shift);
    }
  }
};

// X += the chunk's product. With an incremental residual to follow, D gets
// the change of X: the first chunk leaves X_old in D, the last one X_new - D
// (one FP64 rounding of the change).
struct EpiAddF64 {
  static constexpr bool kTmaC = false;  // updated through apply_cols
  double* X;
  int64_t ldx;
  int n;
  const Ctl* ctl;
  const int32_t* status;
  double* D;  // may be null
  int64_t ldd;
  __device__ bool skip() const { return halted(ctl, status); }
  __device__ void apply_cols(int row0, int col, const float (&v)[32], int chunk, int nchunks) const {
    if (col >= n) return;
    const bool keep = D && *(volatile const int32_t*)&ctl->inc != 0;
    const bool first = chunk == 0, last = chunk == nchunks - 1;
    double* p = X + (int64_t)row0 * ldx + col;
    double* d = keep ? D + (int64_t)row0 * ldd + col : nullptr;
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
      double cur[16], old[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const bool in = row0 + h + r < n;
        cur[r] = in ? p[(int64_t)(h + r) * ldx] : 0.0;
        old[r] = (in && keep && last && !first) ? d[(int64_t)(h + r) * ldd] : cur[r];
      }
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if (row0 + h + r >= n) continue;
        const double xn = cur[r] + static_cast<double>(v[h + r]);
        p[(int64_t)(h + r) * ldx] = xn;
        if (keep && last) d[(int64_t)(h + r) * ldd] = xn - old[r];
        else if (keep && first) d[(int64_t)(h + r) * ldd] = cur[r];
      }
    }
  }
};

// Digit groups of an incremental residual: G = S - floor(D / 5), D the
// smallest cx[j] - cd[j] over the columns whose change is not zero (cx: X's
// exponent bounds, cd: the change's), at least 1 and at most S.
__global__ void incr_groups_kernel(const int32_t* __restrict__ cx, const int32_t* __restrict__ cd, int n, int S,
                                   Ctl* ctl, const int32_t* status, int path) {
  if (halted(ctl, status, path)) return;
  __shared__ int red[32];
  int dmin = INT_MAX;
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    if (cd[j] > -2000) dmin = min(dmin, cx[j] - cd[j]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) dmin = min(dmin, __shfl_xor_sync(0xffffffffu, dmin, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dmin;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) dmin = min(dmin, red[w]);
    int g = S;
    if (dmin == INT_MAX) g = 1;                 // no change at all
    else if (dmin > 0) g = max(1, S - dmin / kLog2Digit);
    ctl->groups = g;
  }
}

// x rounded to TF32 (10 explicit mantissa bits), nearest with ties away from
// zero, on the integer pipe: half a unit added at bit 12 of the magnitude and
// the 13 bits below cleared (a carry into the exponent is the round-up).
// Inf and NaN are returned as they are.
__device__ __forceinline__ float tf32_rn(float x) {
  const uint32_t u = __float_as_uint(x);
  if ((u & 0x7F800000u) == 0x7F800000u) return x;
  return __uint_as_float((u + 0x1000u) & ~0x1FFFu);
}

// 2^e for -1022 <= e <= 1023 from its bit pattern (exact); 0 below.
__device__ __forceinline__ double pow2(int e) {
  if (e < -1022) return 0.0;
  return __longlong_as_double(static_cast<long long>(e + 1023) << 52);
}

// t 2^ex in FP64, rounded to nearest (ties to even), built from t's bits on
// the integer pipe (this GPU's FP64 pipe is the finalize kernel's bound): the
// magnitude's leading one gives the exponent, the next 52 bits the fraction,
// the 11 bits below decide the rounding. The same value as the FP64
// conversion times 2^ex; that product is the fallback where the result
// would leave the normal range.
// The out-of-range case of scaled_i64, kept out of line so that the compiler
// does not evaluate it (an int64 conversion and a multiply on the FP64 pipe)
// for every element.
__device__ __noinline__ double scaled_i64_slow(long long t, int ex) { return static_cast<double>(t) * pow2(ex); }

__device__ __forceinline__ double scaled_i64(long long t, int ex) {
  if (t == 0) return 0.0;
  const unsigned long long sign = t < 0 ? (1ull << 63) : 0ull;
  unsigned long long u = t < 0 ? 0ull - static_cast<unsigned long long>(t) : static_cast<unsigned long long>(t);
  const int lz = __clzll(static_cast<long long>(u));
  u <<= lz;  // leading one at bit 63
  int e = 63 - lz + ex;
  unsigned long long m = u >> 11;  // 53 bits with the leading one
  const unsigned long long rest = u & 0x7FFull;
  if (rest > 0x400ull || (rest == 0x400ull && (m & 1ull))) {
    ++m;
    if (m >> 53) {
      m >>= 1;
      ++e;
    }
  }
  const int be = e + 1023;
  if (be <= 0 || be >= 2047) return scaled_i64_slow(t, ex);
  return __longlong_as_double(static_cast<long long>(sign | (static_cast<unsigned long long>(be) << 52) |
                                                     (m & 0xFFFFFFFFFFFFFull)));
}

// v in FP32 with the fraction truncated, on the integer pipe: magnitudes
// below the FP32 normal range become zero, above it infinity (NaN stays NaN).
// Used where 22 bits or fewer are kept (the norm sum, the TF32 hi/lo split).
__device__ __forceinline__ float f32_trunc(double v) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned sign = static_cast<unsigned>(bits >> 32) & 0x80000000u;
  const int ef = static_cast<int>((bits >> 52) & 0x7FF);
  const int e = ef - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) {
    const bool nan = ef == 0x7FF && (bits & 0xFFFFFFFFFFFFFull) != 0;
    return __uint_as_float(sign | 0x7F800000u | (nan ? 0x400000u : 0u));
  }
  return __uint_as_float(sign | (static_cast<unsigned>(e) << 23) | static_cast<unsigned>((bits >> 29) & 0x7FFFFFull));
}

// E = I - a_ii x_ij - [i != j] a_ij x_jj - 2^(e_i + f_j + 2 - 5 (S + 1)) T
// (S = the digit groups summed in T: 2^(-2F) 32^(2S' - 1 - S) with F = 5S' - 1);
// ||E||^2; E^T split into TF32 hi/lo (rows j of Eop, columns i and Kp + i);
// optionally E itself in FP64.
// kBase: Ebase is given (the incremental residual); a template argument so
// that the compiler does not evaluate both forms for every element.
template <bool kBase>
__global__ void __launch_bounds__(256)
finalize_kernel(const long long* __restrict__ T, int64_t ldt, int n, const double* __restrict__ A,
                int64_t lda, const double* __restrict__ X, int64_t ldx, const int32_t* __restrict__ rexp,
                const int32_t* __restrict__ cexp, int S, double* __restrict__ e2sum, float* __restrict__ Eop,
                int Kp, double* Eout, int64_t lde, const double* Ebase, int64_t ldb, const Ctl* ctl,
                const int32_t* status, int path) {
  // Without kBase: E = I - A X. With it (incremental residual, X = the change
  // of the iterate): E = Ebase - A X; Ebase and Eout may be the same matrix.
  if (halted(ctl, status, path)) return;
  __shared__ double tile[32][33];
  __shared__ double red[8];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int j = j0 + tx;
  float s2 = 0.f;  // ||E||^2 needs a few digits only: FP32 keeps the FP64 pipe for E itself
  // all loads of this thread's four elements first (Eout may be Ebase, so a
  // store would otherwise hold back the next element's loads)
  constexpr int kR = 4;
  long long tv[kR];
  double aii[kR], aij[kR], xij[kR], bv[kR];
  int exv[kR];
  const bool jin = j < n;
  const double xjj = jin ? X[(int64_t)j * ldx + j] : 0.0;
  const int cj = jin ? cexp[j] : 0;
#pragma unroll
  for (int q = 0; q < kR; ++q) {
    const int i = i0 + ty + 8 * q;
    const bool in = i < n && jin;
    tv[q] = in ? T[(int64_t)i * ldt + j] : 0;
    aii[q] = in ? A[(int64_t)i * lda + i] : 0.0;
    aij[q] = in ? A[(int64_t)i * lda + j] : 0.0;
    xij[q] = in ? X[(int64_t)i * ldx + j] : 0.0;
    bv[q] = (kBase && in) ? Ebase[(int64_t)i * ldb + j] : 0.0;
    exv[q] = in ? rexp[i] : 0;
  }
  // Tiles off the diagonal (all but one in 32 of them) take the
  // off-diagonal formula alone: a select between the two would have the
  // FP64 pipe evaluate both for every element.
  const bool diag_tile = i0 == j0;
#pragma unroll
  for (int q = 0; q < kR; ++q) {
    const int ii = ty + 8 * q;
    const int i = i0 + ii;
    double e = 0.0;
    if (i < n && jin) {
      const int ex = exv[q] + cj + 2 * kHeadroom - kLog2Digit * (S + 1);
      const double r = scaled_i64(tv[q], ex);
      const double dx = aii[q] * xij[q];  // (D_A X)_ij
      if (!diag_tile) {
        if constexpr (kBase) e = (bv[q] - fma(aij[q], xjj, dx)) - r;
        else e = -fma(aij[q], xjj, dx) - r;  // (O_A D_X)_ij
      } else if (kBase) {
        e = (i == j) ? (bv[q] - dx) - r : (bv[q] - fma(aij[q], xjj, dx)) - r;
      } else if (i == j) {
        e = (1.0 - dx) - r;
      } else {
        e = -fma(aij[q], xjj, dx) - r;
      }
      const float ef = f32_trunc(e);
      s2 = fmaf(ef, ef, s2);
      if (Eout) Eout[(int64_t)i * lde + j] = e;
    }
    tile[ii][tx] = e;
  }
  double s2d = s2;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s2d += __shfl_xor_sync(0xffffffffu, s2d, off);
  if (tx == 0) red[ty] = s2d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int y = 0; y < 8; ++y) t += red[y];
    atomicAdd(e2sum, t);
  }
  if (!Eop) return;
  // transposed write: row j of Eop gets E[i0..i0+31][j]
  for (int jj = ty; jj < 32; jj += 8) {
    const int jg = j0 + jj;
    const int i = i0 + tx;
    if (jg < n && i < n) {
      // hi + lo keep 22 bits, within FP32's 24: the split can start from FP32
      const float v = f32_trunc(tile[tx][jj]);
      const float hi = tf32_rn(v);
      const float lo = tf32_rn(v - hi);
      Eop[(int64_t)jg * 2 * Kp + i] = hi;
      Eop[(int64_t)jg * 2 * Kp + Kp + i] = lo;
    }
  }
}

// v rounded to 11 significant bits (TF32 precision), half away from zero, as
// a double, on the integer pipe: add half a unit at bit 41 of the fraction
// and clear the 42 bits below (a carry into the exponent is the round-up).
// Zero, subnormal and non-finite v are returned as they are.
__device__ __forceinline__ double round11(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned ef = static_cast<unsigned>(b >> 52) & 0x7FFu;
  if (ef == 0 || ef == 0x7FF) return v;
  return __longlong_as_double(static_cast<long long>((b + (1ull << 41)) & ~((1ull << 42) - 1)));
}

// A double with at most 24 significant bits as FP32 bits (exact), on the
// integer pipe; below the FP32 normal range it becomes zero.
__device__ __forceinline__ float narrow_exact(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned sign = static_cast<unsigned>(b >> 32) & 0x80000000u;
  const int e = static_cast<int>((b >> 52) & 0x7FF) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return static_cast<float>(v);
  return __uint_as_float(sign | (static_cast<unsigned>(e) << 23) | static_cast<unsigned>((b >> 29) & 0x7FFFFFull));
}

// X split into TF32 hi/lo operands (rows i, columns k and Kp + k): hi = v to
// 11 significant bits, lo = the remainder (exact in FP64) to 11 bits, so
// hi + lo carries 22 bits of v; one FP64 subtraction per element.
__global__ void split_x_kernel(const double* __restrict__ X, int64_t ldx, int n, float* __restrict__ Xop, int Kp,
                               const Ctl* ctl, const int32_t* status) {
  if (halted(ctl, status)) return;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {  // row by row: no index division
    const double* x = X + (int64_t)i * ldx;
    float* o = Xop + (int64_t)i * 2 * Kp;
#pragma unroll 4
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const double v = x[k];
      const double hd = round11(v);
      o[k] = narrow_exact(hd);
      o[Kp + k] = narrow_exact(round11(v - hd));
    }
  }
}

// rho for residual `it`; decides whether refinement goes on.
// The next residual is incremental when incr_ok (its buffers exist) and
// ||E||_F <= kIncrMaxE.
//
// An update maps E to E^2 (I - A X (2I - A X) = (I - A X)^2), so with
// e = ||E||_F < 1 the iteration converges and e_k is about e_{k-1}^2 until
// the rounding floor. Refinement stops (NOT_CONVERGED) when e >= 1 (no
// guarantee), or when e fails to fall below e_{k-1} min(0.95, max(0.5,
// 2 e_{k-1})): slack over the quadratic model far from the solution (an
// ill-conditioned start at e = 0.9 drops only to 0.81), a halving near it,
// so a stall at the floor ends it after one more residual.
__global__ void decide_kernel(const double* sums, int it, double tol, int max_updates, double* hist, Ctl* ctl,
                              const int32_t* status, int incr_ok) {
  if (ctl->done || *status != 0) return;
  const double a2 = sums[0], e2 = sums[1 + 2 * it], x2 = sums[2 + 2 * it];
  const double en = sqrt(e2);
  const double rho = en / (sqrt(a2) * sqrt(x2));
  hist[it] = rho;
  ctl->last = it;
  if (ctl->inc) ctl->incs += 1;
  bool stalled = false;
  if (it > 0) {
    const double ep = sqrt(sums[1 + 2 * (it - 1)]);
    stalled = !(en < ep * fmin(0.95, fmax(0.5, 2.0 * ep)));
  }
  if (rho <= tol) {
    ctl->done = 1;
    ctl->code = BLOCKINV_OK;
  } else if (it >= max_updates || !(rho == rho) || !(en < 1.0) || stalled) {
    ctl->done = 1;
    ctl->code = BLOCKINV_ERR_NOT_CONVERGED;
  } else {
    ctl->updates = it + 1;
    ctl->inc = (incr_ok && sqrt(e2) <= kIncrMaxE) ? 1 : 0;
  }
}

__global__ void finish_kernel(const Ctl* ctl, int32_t* status) {
  if (*status == 0 && ctl->code != BLOCKINV_OK) atomicCAS(&status[0], 0, ctl->code);
}

__global__ void init_ctl_kernel(Ctl* ctl, int32_t* cexp, int n, int iters) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->done = 0;
    ctl->updates = 0;
    ctl->code = BLOCKINV_ERR_NOT_CONVERGED;
    ctl->last = -1;
    ctl->inc = 0;
    ctl->incs = 0;
    ctl->groups = 0;
  }
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * iters; t += gridDim.x * blockDim.x) cexp[t] = -2000;
}

template <int S>
cudaError_t launch_slices(const double* A0, int64_t ld0, const double* X, int64_t ldx, int n, int Kp,
                          const int32_t* rexp, int32_t* cexp, uint8_t* Asl, uint8_t* Xsl, double* x2, bool rows,
                          const Ctl* ctl, const int32_t* status, cudaStream_t s, int path) {
  if (rows) {
    const int64_t quads = (int64_t)n * (Kp / 4);
    const int grid = (int)std::min<int64_t>((quads + 255) / 256, 16 * tc::num_sms());
    slice_rows_kernel<S><<<grid, 256, 0, s>>>(A0, ld0, n, rexp, Kp, Asl, ctl, status);
    return cudaGetLastError();
  }
  dim3 g1((n + 31) / 32, (n + 255) / 256);
  col_scale_kernel<<<g1, 256, 0, s>>>(X, ldx, n, cexp, x2, ctl, status, path);
  dim3 g2((n + 31) / 32, Kp / 64);
  slice_cols_t_kernel<S><<<g2, 256, 0, s>>>(X, ldx, n, cexp, Kp, Xsl, ctl, status, path);
  return cudaGetLastError();
}

cudaError_t slices_dispatch(int S, const double* A0, int64_t ld0, const double* X, int64_t ldx, int n, int Kp,
                            const int32_t* rexp, int32_t* cexp, uint8_t* Asl, uint8_t* Xsl, double* x2, bool rows,
                            const Ctl* ctl, const int32_t* status, cudaStream_t s, int path = kAny) {
  switch (S) {
    case 7: return launch_slices<7>(A0, ld0, X, ldx, n, Kp, rexp, cexp, Asl, Xsl, x2, rows, ctl, status, s, path);
    case 8: return launch_slices<8>(A0, ld0, X, ldx, n, Kp, rexp, cexp, Asl, Xsl, x2, rows, ctl, status, s, path);
    case 9: return launch_slices<9>(A0, ld0, X, ldx, n, Kp, rexp, cexp, Asl, Xsl, x2, rows, ctl, status, s, path);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t refine_workspace_bytes(int n, int S, int max_updates) {
  const size_t Kp = (size_t)(n + 127) / 128 * 128;
  const size_t ldt = (size_t)(n + 31) / 32 * 32;
  size_t b = 0;
  b += 2 * (size_t)n * S * Kp;                  // A and X digit slices
  b += sizeof(long long) * (size_t)n * ldt;     // int64 accumulator
  b += 2 * sizeof(float) * (size_t)n * 2 * Kp;  // X and E^T TF32 hi/lo operands
  b += sizeof(int32_t) * (size_t)n * (2 * max_updates + 3);   // exponents
  b += sizeof(double) * (3 + 2 * (max_updates + 1)) + sizeof(double) * (max_updates + 1) + 64;
  if (max_updates > 0) b += 2 * sizeof(double) * (size_t)n * ldt;  // E and the change of X (incremental)
  return b + 10 * 256;
}

// Enqueue the refinement of X (n x n, FP64, in place) toward A0^-1.
// ws must hold refine_workspace_bytes(n, S, max_updates) bytes. hist (device,
// max_updates + 1 doubles) receives the rho of every residual computed; ctl
// (device, 4 int32: done, updates, code, last) the outcome. If Eout is
// non-null and max_updates == 0, the residual E = I - A0 X is written there.
// With `report`, a refinement that stops short of tol sets the status word to
// BLOCKINV_ERR_NOT_CONVERGED. With `host_steps` the host waits for each
// decision and enqueues no further iteration once the device is done (for
// blocking callers); otherwise every iteration is enqueued and the kernels of
// iterations past the decision return at once (stream-ordered, capturable).
cudaError_t enqueue_refine(const double* A0, int64_t ld0, double* X, int64_t ldx, int n, double tol,
                           int max_updates, int S, void* ws, double* hist, int32_t* ctl_words, int32_t* status,
                           double* Eout, int64_t lde, cudaStream_t s, bool report, bool host_steps) {
  if (S < kMinResidualSlices || S > kMaxResidualSlices || n < 1 || n > kMixedMaxOrder) return cudaErrorInvalidValue;
  // digit pairs per accumulator chunk: pairs * n * 2^8 <= 2^24
  const int max_pairs = (1 << 16) / n;
  Ctl* ctl = reinterpret_cast<Ctl*>(ctl_words);
  const int Kp = (n + 127) / 128 * 128;
  const int64_t ldt = (n + 31) / 32 * 32;
  auto carve = [&](size_t bytes) {
    uintptr_t p = (reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255);
    ws = reinterpret_cast<void*>(p + bytes);
    return reinterpret_cast<void*>(p);
  };
  uint8_t* Asl = static_cast<uint8_t*>(carve((size_t)n * S * Kp));
  uint8_t* Xsl = static_cast<uint8_t*>(carve((size_t)n * S * Kp));
  long long* T = static_cast<long long*>(carve(sizeof(long long) * (size_t)n * ldt));
  float* Xop = static_cast<float*>(carve(sizeof(float) * (size_t)n * 2 * Kp));
  float* Eop = static_cast<float*>(carve(sizeof(float) * (size_t)n * 2 * Kp));
  int32_t* rexp = static_cast<int32_t*>(carve(sizeof(int32_t) * n));
  // column exponent bounds: of X (or of its change) per residual, then of X
  // per incremental residual
  int32_t* cexp = static_cast<int32_t*>(carve(sizeof(int32_t) * (size_t)n * 2 * (max_updates + 1)));
  double* sums = static_cast<double*>(carve(sizeof(double) * (1 + 2 * (max_updates + 1))));
  const bool incr_ok = max_updates > 0;
  double* Ebuf = incr_ok ? static_cast<double*>(carve(sizeof(double) * (size_t)n * ldt)) : nullptr;
  double* Dbuf = incr_ok ? static_cast<double*>(carve(sizeof(double) * (size_t)n * ldt)) : nullptr;

  cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(double) * (1 + 2 * (max_updates + 1)), s);
  // K padding of the operands must be zero (only columns < n are written).
  if (e == cudaSuccess) e = cudaMemsetAsync(Asl, 0, (size_t)n * S * Kp, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(Xsl, 0, (size_t)n * S * Kp, s);
  if (e == cudaSuccess && max_updates > 0) e = cudaMemsetAsync(Xop, 0, sizeof(float) * (size_t)n * 2 * Kp, s);
  if (e == cudaSuccess && max_updates > 0) e = cudaMemsetAsync(Eop, 0, sizeof(float) * (size_t)n * 2 * Kp, s);
  if (e != cudaSuccess) return e;
  init_ctl_kernel<<<64, 256, 0, s>>>(ctl, cexp, n, 2 * (max_updates + 1));

  CUtensorMap tAs, tXs, tXo, tEo;
  if (!make_tmap_2d(&tAs, Asl, CU_TENSOR_MAP_DATA_TYPE_UINT8, (uint64_t)S * Kp, n, (uint64_t)S * Kp, 128, tc::kBM) ||
      !make_tmap_2d(&tXs, Xsl, CU_TENSOR_MAP_DATA_TYPE_UINT8, (uint64_t)S * Kp, n, (uint64_t)S * Kp, 128,
                    tc::b_rows<tc::kPairTiles>()) ||
      !make_tmap_2d(&tXo, Xop, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2ull * Kp, n, 8ull * Kp, 16, tc::kBM, true) ||
      !make_tmap_2d(&tEo, Eop, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2ull * Kp, n, 8ull * Kp, 16,
                    tc::b_rows<tc::kPairTiles>(), true))
    return cudaErrorInvalidValue;

  const double nd = n;
  {
    TraceScope t("residual_slice_a", 0, 8.0 * nd * nd + (double)S * nd * Kp, s);
    row_scale_kernel<<<(n + 7) / 8, 256, 0, s>>>(A0, ld0, n, rexp, &sums[0], ctl, status);
    e = slices_dispatch(S, A0, ld0, nullptr, 0, n, Kp, rexp, nullptr, Asl, nullptr, nullptr, true, ctl, status, s);
  }
  // The digit-group GEMMs of one residual in one launch: groups 0 .. groups - 1,
  // group g the pairs (p, g - p), each group cut into chunks of at most
  // max_pairs pairs (accumulated from zero in FP32, exact) and handed to the
  // int64 epilogue with its shift. A tile's chunks follow one another, so its
  // slice of T stays in L2 between them. With incr_groups the device word
  // ctl->groups switches off the trailing groups.
  auto group_gemms = [&](int groups, int path, bool incr_groups) -> cudaError_t {
    tc::KMap km{};
    km.kb_per_pair = Kp / 128;
    km.slice_cols = Kp;
    int np = 0, nc = 0;
    km.bounds[0] = 0;
    for (int g = 0; g < groups; ++g) {
      for (int p0 = 0; p0 <= g; p0 += max_pairs) {
        const int cnt = std::min(max_pairs, g + 1 - p0);
        if (nc >= tc::kMaxChunks || np + cnt > tc::kMaxPairs) return cudaErrorInvalidValue;
        if (p0 == 0) km.group_starts |= 1u << nc;
        for (int i = 0; i < cnt; ++i, ++np) {
          km.pa[np] = (int8_t)(p0 + i);
          km.pb[np] = (int8_t)(g - p0 - i);
        }
        km.bounds[++nc] = (int16_t)(np * km.kb_per_pair);
      }
    }
    km.nbounds = nc;
    km.kblocks = np * km.kb_per_pair;
    km.live_groups = incr_groups ? &ctl->groups : nullptr;
    EpiAccumI64 epi{T, ldt, n, groups, km.group_starts, ctl, status, path};
    TraceScope t("residual_group_gemm_e4m3", 2.0 * nd * nd * nd * np, (double)np * 2.0 * nd * Kp + 16.0 * nd * nd, s);
    return tc::launch_gemm<tc::Kind::E4M3, EpiAccumI64, false, tc::kPairTiles>(tAs, tXs, n, n, km, epi, status, s);
  };
  bool next_inc = false;  // host view of ctl->inc (host_steps)
  for (int it = 0; it <= max_updates && e == cudaSuccess; ++it) {
    int32_t* cx = cexp + (size_t)it * n;
    dim3 fg((n + 31) / 32, (n + 31) / 32);
    // Fresh residual E = I - A X from all S digits of X; or, after a residual
    // with ||E||_F <= kIncrMaxE, E_new = E - A (X - X_prev) from the leading
    // digit groups of the change of X (as many as its scale needs). Without
    // host steps both are enqueued and the device flag lets one of them run.
    const bool fresh = !host_steps || !next_inc;
    const bool incr = incr_ok && it > 0 && (!host_steps || next_inc);
    if (fresh) {
      {
        TraceScope t("residual_slice_x", 0, 16.0 * nd * nd + (double)S * nd * Kp, s);
        e = slices_dispatch(S, nullptr, 0, X, ldx, n, Kp, rexp, cx, nullptr, Xsl, &sums[2 + 2 * it], false, ctl,
                            status, s, incr ? kFresh : kAny);
      }
      if (e == cudaSuccess) e = group_gemms(S, incr ? kFresh : kAny, false);
      if (e != cudaSuccess) break;
      TraceScope t("residual_finalize", 0, 8.0 * nd * nd + (max_updates > 0 ? 16.0 * nd * nd : 0.0), s);
      finalize_kernel<false><<<fg, 256, 0, s>>>(T, ldt, n, A0, ld0, X, ldx, rexp, cx, S, &sums[1 + 2 * it],
                                         it < max_updates ? Eop : nullptr, Kp,
                                         (max_updates == 0) ? Eout : (it < max_updates ? Ebuf : nullptr),
                                         (max_updates == 0) ? lde : ldt, nullptr, 0, ctl, status,
                                         incr ? kFresh : kAny);
    }
    if (incr && e == cudaSuccess) {
      {
        TraceScope t("residual_slice_dx", 0, 24.0 * nd * nd + (double)S * nd * Kp, s);
        e = slices_dispatch(S, nullptr, 0, Dbuf, ldt, n, Kp, rexp, cx, nullptr, Xsl, nullptr, false, ctl, status, s,
                            fresh ? kIncr : kAny);
        // X's column exponent bounds and ||X||^2, then the groups needed
        int32_t* cxx = cexp + (size_t)(max_updates + 1 + it) * n;
        col_scale_kernel<<<dim3((n + 31) / 32, (n + 255) / 256), 256, 0, s>>>(X, ldx, n, cxx, &sums[2 + 2 * it], ctl,
                                                                              status, fresh ? kIncr : kAny);
        incr_groups_kernel<<<1, 1024, 0, s>>>(cxx, cx, n, S, ctl, status, fresh ? kIncr : kAny);
      }
      // all S groups enqueued; those from ctl->groups on return at once
      if (e == cudaSuccess) e = group_gemms(S, fresh ? kIncr : kAny, true);
      if (e != cudaSuccess) break;
      TraceScope t("residual_finalize", 0, 24.0 * nd * nd, s);
      finalize_kernel<true><<<fg, 256, 0, s>>>(T, ldt, n, A0, ld0, Dbuf, ldt, rexp, cx, S, &sums[1 + 2 * it],
                                         it < max_updates ? Eop : nullptr, Kp, Ebuf, ldt, Ebuf, ldt, ctl, status,
                                         fresh ? kIncr : kAny);
    }
    decide_kernel<<<1, 1, 0, s>>>(sums, it, tol, max_updates, hist, ctl, status, incr_ok ? 1 : 0);
    if (it == max_updates) break;
    if (host_steps) {
      // Blocking callers stop enqueueing as soon as the device has decided.
      int32_t h[kRefineCtlWords + 1] = {};
      e = cudaMemcpyAsync(h, ctl_words, sizeof(int32_t) * kRefineCtlWords, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&h[kRefineCtlWords], status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess || h[0] != 0 || h[kRefineCtlWords] != 0) break;
      next_inc = h[offsetof(Ctl, inc) / sizeof(int32_t)] != 0;
    }
    {
      TraceScope t("ns_split_x", 0, 16.0 * nd * nd, s);
      split_x_kernel<<<8 * tc::num_sms(), 256, 0, s>>>(X, ldx, n, Xop, Kp, ctl, status);
    }
    {
      // Split stages: each k-block is 16 columns of K of the hi and lo
      // slices of both operands, with the products hi*hi, hi*lo and lo*hi.
      tc::KMap km{};
      km.kb_per_pair = Kp / 16;
      km.slice_cols = Kp;
      km.kblocks = km.kb_per_pair;
      km.pa[0] = 0;
      km.pb[0] = 0;
      // The tensor-core FP32 accumulator drops bits on every k-step (its
      // error grows linearly with K, measured, and with the accumulator's
      // magnitude, which the hi*hi terms set), so K is cut into chunks of
      // kUpdateChunkK, each added into the FP64 X on its own.
      km.chunk_kb = kUpdateChunkK / 16;
      EpiAddF64 epi{X, ldx, n, ctl, status, Dbuf, ldt};
      const double chunks = std::ceil((double)Kp / kUpdateChunkK);
      TraceScope t("ns_update_tf32x3", 3.0 * 2.0 * nd * nd * nd, 16.0 * nd * nd * chunks + 16.0 * nd * Kp, s);
      e = tc::launch_gemm<tc::Kind::TF32, EpiAddF64, true, tc::kPairTiles>(tXo, tEo, n, n, km, epi, status, s);
    }
  }
  if (e == cudaSuccess && report) {
    finish_kernel<<<1, 1, 0, s>>>(ctl, status);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace blockinv
