// Host side of the tcgen05 GEMM (tensor maps, SM count) and the diagnostic
// entry point blockinv_diag_gemm, which runs the same kernel with a plain
// FP32 store epilogue so the tensor-core path can be checked on its own.
#include <cudaTypedefs.h>

#include <mutex>

#include "tc_gemm.cuh"

namespace blockinv {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}
}  // namespace

bool make_tmap_2d(CUtensorMap* map, const void* base, CUtensorMapDataType dt, uint64_t inner, uint64_t outer,
                  uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, bool swizzle64) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  return fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace tc {
int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}
}  // namespace tc

namespace {

// C[row, col] = accumulator (FP32), row-major with leading dimension ldc.
struct EpiStoreF32 {
  static constexpr bool kTmaC = false;  // updated through apply_cols
  float* C;
  int64_t ldc;
  int M, N;
  __device__ bool skip() const { return false; }
  __device__ void apply_cols(int row0, int col, const float (&v)[32], int chunk, int nchunks) const {
    if (col >= N) return;
#pragma unroll
    for (int r = 0; r < 32; ++r)
      if (row0 + r < M) C[(int64_t)(row0 + r) * ldc + col] = v[r];
  }
};

template <tc::Kind K, bool kPair>
int diag(int M, int N, int Kdim, const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc,
         cudaStream_t s) {
  constexpr int eb = tc::KindTraits<K>::elem_bytes;
  constexpr int BK = 128 / eb;
  const CUtensorMapDataType dt = (K == tc::Kind::BF16)   ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                 : (K == tc::Kind::TF32) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                         : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  CUtensorMap ta, tb;
  if (!make_tmap_2d(&ta, A, dt, (uint64_t)Kdim, (uint64_t)M, (uint64_t)lda * eb, BK, tc::kBM) ||
      !make_tmap_2d(&tb, B, dt, (uint64_t)Kdim, (uint64_t)N, (uint64_t)ldb * eb, BK, tc::b_rows<kPair>()))
    return BLOCKINV_ERR_INVALID;
  tc::KMap km = tc::plain_kmap((Kdim + BK - 1) / BK);
  EpiStoreF32 epi{C, ldc, M, N};
  cudaError_t e = tc::launch_gemm<K, EpiStoreF32, false, kPair>(ta, tb, M, N, km, epi, nullptr, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_status(e);
}

}  // namespace
}  // namespace blockinv

extern "C" int blockinv_diag_gemm(int kind, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                                  const void* B, int64_t ldb, float* C, int64_t ldc, void* stream) {
  using namespace blockinv;
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || lda < K || ldb < K || ldc < N || M > (1 << 30) ||
      N > (1 << 30))
    return BLOCKINV_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (kind) {
    case 0: return diag<tc::Kind::BF16, false>((int)M, (int)N, (int)K, A, lda, B, ldb, C, ldc, s);
    case 1: return diag<tc::Kind::TF32, false>((int)M, (int)N, (int)K, A, lda, B, ldb, C, ldc, s);
    case 2: return diag<tc::Kind::E4M3, false>((int)M, (int)N, (int)K, A, lda, B, ldb, C, ldc, s);
    case 3: return diag<tc::Kind::BF16, true>((int)M, (int)N, (int)K, A, lda, B, ldb, C, ldc, s);
    case 4: return diag<tc::Kind::TF32, true>((int)M, (int)N, (int)K, A, lda, B, ldb, C, ldc, s);
    case 5: return diag<tc::Kind::E4M3, true>((int)M, (int)N, (int)K, A, lda, B, ldb, C, ldc, s);
    default: return BLOCKINV_ERR_INVALID;
  }
}
