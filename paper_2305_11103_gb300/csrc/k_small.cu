// Batched inversion of many small matrices (order 1..8), FP64, one thread per
// matrix. The motivating workload is the paper's repeated 5 x 5 inversions of
// systematics matrices (Sec. 2), partitioned by the paper's rule (Table 2:
// 5 -> [2, 3]). Each thread runs the in-place block Gauss-Jordan steps of
// Eq. (a) on its matrix in registers, with every index known at compile time;
// pivot blocks of order <= 4 use closed forms (the "algebraic expressions" of
// Sec. 5.1): 1/a, the 2 x 2 and 3 x 3 adjugates, and for order 4 Eq. (a)
// itself on 2 x 2 sub-blocks. Reciprocals are the 3-FMA estimate-and-correct
// of fp64_ops.cuh, and the zero / finiteness tests look at bit patterns.
//
// Memory: each warp stages 32 consecutive matrices through shared memory,
// so that the global loads and stores are coalesced. Per matrix the kernel
// moves 2 * 8 n^2 bytes and does about 2 n^3 flops; on GB300 the FP64 pipe
// (2 DFMA / clock / SM), not HBM, bounds it.
#include "fp64_ops.cuh"
#include "internal.h"

namespace blockinv {

namespace tc {
int num_sms();  // streaming multiprocessors of the current device
}  // namespace tc

namespace {

// The paper's partition for orders 1..8 (Table 2): N_k = 2^(int(log2 n) - 1)
// blocks of order 2..4, the remainder given to the last blocks; n <= 3 is one
// block.
template <int N>
struct Partition;
template <> struct Partition<1> { static constexpr int p = 1; static constexpr int s[1] = {1}; };
template <> struct Partition<2> { static constexpr int p = 1; static constexpr int s[1] = {2}; };
template <> struct Partition<3> { static constexpr int p = 1; static constexpr int s[1] = {3}; };
template <> struct Partition<4> { static constexpr int p = 2; static constexpr int s[2] = {2, 2}; };
template <> struct Partition<5> { static constexpr int p = 2; static constexpr int s[2] = {2, 3}; };
template <> struct Partition<6> { static constexpr int p = 2; static constexpr int s[2] = {3, 3}; };
template <> struct Partition<7> { static constexpr int p = 2; static constexpr int s[2] = {3, 4}; };
template <> struct Partition<8> { static constexpr int p = 4; static constexpr int s[4] = {2, 2, 2, 2}; };

// zero or non-finite, on the integer pipe
__device__ __forceinline__ bool bad(double d) { return zero_bits(d) || nonfinite_bits(d); }

// Closed-form inverses; return false if singular or non-finite.
template <int B>
struct Inv;

template <>
struct Inv<1> {
  __device__ static bool run(const double (&m)[1][1], double (&r)[1][1]) {
    if (bad(m[0][0])) return false;
    r[0][0] = recip64(m[0][0]);
    return true;
  }
};

template <>
struct Inv<2> {
  __device__ static bool run(const double (&m)[2][2], double (&r)[2][2]) {
    const double det = m[0][0] * m[1][1] - m[0][1] * m[1][0];
    if (bad(det)) return false;
    const double id = recip64(det);
    r[0][0] = m[1][1] * id;
    r[0][1] = -m[0][1] * id;
    r[1][0] = -m[1][0] * id;
    r[1][1] = m[0][0] * id;
    return true;
  }
};

template <>
struct Inv<3> {
  __device__ static bool run(const double (&m)[3][3], double (&r)[3][3]) {
    // cofactors c_ij; inverse = c^T / det
    const double c00 = m[1][1] * m[2][2] - m[1][2] * m[2][1];
    const double c01 = m[1][2] * m[2][0] - m[1][0] * m[2][2];
    const double c02 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
    const double det = m[0][0] * c00 + m[0][1] * c01 + m[0][2] * c02;
    if (bad(det)) return false;
    const double id = recip64(det);
    r[0][0] = c00 * id;
    r[1][0] = c01 * id;
    r[2][0] = c02 * id;
    r[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) * id;
    r[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) * id;
    r[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) * id;
    r[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) * id;
    r[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) * id;
    r[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) * id;
    return true;
  }
};

template <>
struct Inv<4> {
  // Eq. (a) with 2 x 2 blocks [[A, B], [C, D]].
  __device__ static bool run(const double (&m)[4][4], double (&r)[4][4]) {
    double a[2][2] = {{m[0][0], m[0][1]}, {m[1][0], m[1][1]}};
    double ai[2][2];
    if (!Inv<2>::run(a, ai)) return false;
    double p[2][2], q[2][2], s[2][2], si[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        p[i][j] = ai[i][0] * m[0][2 + j] + ai[i][1] * m[1][2 + j];        // A^-1 B
        q[i][j] = m[2 + i][0] * ai[0][j] + m[2 + i][1] * ai[1][j];        // C A^-1
      }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) s[i][j] = m[2 + i][2 + j] - (m[2 + i][0] * p[0][j] + m[2 + i][1] * p[1][j]);
    if (!Inv<2>::run(s, si)) return false;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const double tr = -(p[i][0] * si[0][j] + p[i][1] * si[1][j]);
        const double bl = -(si[i][0] * q[0][j] + si[i][1] * q[1][j]);
        r[i][2 + j] = tr;
        r[2 + i][j] = bl;
        r[2 + i][2 + j] = si[i][j];
      }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) r[i][j] = ai[i][j] - (r[i][2] * q[0][j] + r[i][3] * q[1][j]);
    return true;
  }
};

// One elimination step with the pivot block at rows/columns [O, O + B).
template <int N, int O, int B>
__device__ __forceinline__ bool gj_step(double (&x)[N][N]) {
  double pb[B][B], pi[B][B];
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) pb[r][c] = x[O + r][O + c];
  if (!Inv<B>::run(pb, pi)) return false;
  // row panel: x[O + r][j] <- sum_l pi[r][l] x[O + l][j], j outside the block
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (j >= O && j < O + B) continue;
    double v[B];
#pragma unroll
    for (int r = 0; r < B; ++r) {
      double acc = 0.0;
#pragma unroll
      for (int l = 0; l < B; ++l) acc = fma(pi[r][l], x[O + l][j], acc);
      v[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < B; ++r) x[O + r][j] = v[r];
  }
  // other rows: Schur update and column assembly
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (i >= O && i < O + B) continue;
    double u[B];
#pragma unroll
    for (int l = 0; l < B; ++l) u[l] = x[i][O + l];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if (j >= O && j < O + B) continue;
      double acc = x[i][j];
#pragma unroll
      for (int l = 0; l < B; ++l) acc = fma(-u[l], x[O + l][j], acc);
      x[i][j] = acc;
    }
#pragma unroll
    for (int c = 0; c < B; ++c) {
      double acc = 0.0;
#pragma unroll
      for (int l = 0; l < B; ++l) acc = fma(-u[l], pi[l][c], acc);
      x[i][O + c] = acc;
    }
  }
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) x[O + r][O + c] = pi[r][c];
  return true;
}

template <int N, int K, int O>
__device__ __forceinline__ int run_steps(double (&x)[N][N]) {
  using Pt = Partition<N>;
  if constexpr (K == Pt::p) {
    return -1;
  } else {
    constexpr int B = Pt::s[K];
    if (!gj_step<N, O, B>(x)) return K;
    return run_steps<N, K + 1, O + B>(x);
  }
}

// One CTA per SM, each with a contiguous share of the batch in chunks of 32
// matrices (one per lane); the CTA's warps take its chunks in turn, each
// staging its chunk through its own slice of shared memory (matrix pitch odd,
// so the per-lane accesses hit 32 banks). Even shares per SM keep the FP64
// pipes of all SMs busy to the end (a grid of 128-matrix CTAs left the second
// of 1.5 waves half empty).
// warps per CTA: as many as the registers of one SM allow for the order
template <int N>
__host__ __device__ constexpr int small_warps() { return N <= 5 ? 24 : (N <= 7 ? 16 : 8); }

template <int N>
__global__ void __launch_bounds__(32 * small_warps<N>())
small_batched_kernel(double* __restrict__ A, int64_t count, int32_t* __restrict__ status, int64_t per_cta) {
  constexpr int NN = N * N;
  constexpr int PITCH = NN | 1;
  extern __shared__ double stage_all[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* stage = stage_all + (size_t)warp * 32 * PITCH;
  const int64_t nchunks = (count + 31) / 32;
  const int64_t c0 = (int64_t)blockIdx.x * per_cta;
  const int64_t c1 = min(nchunks, c0 + per_cta);
  for (int64_t c = c0 + warp; c < c1; c += small_warps<N>()) {
    const int64_t m0 = c * 32;
    const int cnt = (int)(count - m0 < 32 ? count - m0 : 32);
    double* g = A + m0 * NN;
    for (int e = lane; e < cnt * NN; e += 32) stage[(e / NN) * PITCH + e % NN] = g[e];
    __syncwarp();
    if (lane < cnt) {
      double* mine = stage + lane * PITCH;
      double x[N][N];
      bool finite = true;
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
          x[i][j] = mine[i * N + j];
          finite = finite && !nonfinite_bits(x[i][j]);
        }
      int code = BLOCKINV_OK;
      if (!finite) {
        code = BLOCKINV_ERR_NONFINITE;
      } else if (run_steps<N, 0, 0>(x) >= 0) {
        code = BLOCKINV_ERR_SINGULAR;
      }
      if (code == BLOCKINV_OK) {  // a failed matrix keeps its input
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int j = 0; j < N; ++j) mine[i * N + j] = x[i][j];
      }
      if (status) status[m0 + lane] = code;
    }
    __syncwarp();
    for (int e = lane; e < cnt * NN; e += 32) g[e] = stage[(e / NN) * PITCH + e % NN];
    __syncwarp();
  }
}

template <int N>
cudaError_t launch_small_n(double* A, int64_t count, int32_t* status, cudaStream_t s) {
  const int grid = tc::num_sms();
  const int64_t nchunks = (count + 31) / 32;
  const int64_t per_cta = (nchunks + grid - 1) / grid;
  const size_t smem = sizeof(double) * small_warps<N>() * 32 * (size_t)((N * N) | 1);
  auto k = small_batched_kernel<N>;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, 32 * small_warps<N>(), smem, s>>>(A, count, status, per_cta);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_small_batched(int n, double* A, int64_t count, int32_t* status, cudaStream_t s) {
  switch (n) {
    case 1: return launch_small_n<1>(A, count, status, s);
    case 2: return launch_small_n<2>(A, count, status, s);
    case 3: return launch_small_n<3>(A, count, status, s);
    case 4: return launch_small_n<4>(A, count, status, s);
    case 5: return launch_small_n<5>(A, count, status, s);
    case 6: return launch_small_n<6>(A, count, status, s);
    case 7: return launch_small_n<7>(A, count, status, s);
    case 8: return launch_small_n<8>(A, count, status, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace blockinv
