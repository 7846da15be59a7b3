// Diagnostic entry points: the library's device helpers run on caller data so
// that tests can check them directly.
//
//  - blockinv_diag_recip64: the 3-FMA FP64 reciprocal of the batched kernels
//    (fp64_ops.cuh) applied elementwise, for comparison with IEEE division.
//  - blockinv_diag_wait_timeout: one bounded mbarrier wait, of the same
//    function the tensor-core kernels use for every wait, on a barrier that
//    nothing arrives at; when its limit runs out the kernel records
//    BLOCKINV_ERR_TIMEOUT in the status word exactly as those kernels do.
//    No copy or tensor-core operation is in flight when it gives up.
#include <algorithm>

#include "fp64_ops.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace blockinv {
namespace {

__global__ void recip64_kernel(const double* __restrict__ v, double* __restrict__ out, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = recip64(v[i]);
}

__global__ void wait_timeout_kernel(uint64_t limit_ns, int32_t* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait_for(&bar, 0, limit_ns))
    atomicCAS(&status[0], 0, BLOCKINV_ERR_TIMEOUT);
}

}  // namespace
}  // namespace blockinv

using namespace blockinv;

extern "C" int blockinv_diag_recip64(const double* v, double* out, int64_t count, void* stream) {
  if (count < 0 || (count > 0 && (!v || !out))) return BLOCKINV_ERR_INVALID;
  if (count == 0) return BLOCKINV_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, 8 * 152);
  recip64_kernel<<<(int)blocks, 256, 0, s>>>(v, out, count);
  const cudaError_t e = cudaGetLastError();
  return cuda_status(e);
}

extern "C" int blockinv_diag_wait_timeout(int64_t limit_ns, void* stream) {
  if (limit_ns < 0 || limit_ns > (int64_t)tc::kWaitLimitNs) return BLOCKINV_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t* status = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&status), 2 * sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_status(e);
  int32_t host[2] = {0, 0};
  e = cudaMemsetAsync(status, 0, 2 * sizeof(int32_t), s);
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 32, 0, s>>>(static_cast<uint64_t>(limit_ns), status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, status, sizeof(host), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(status, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  return host[0];
}
