// blockinv_invert_noalloc: the FP64 in-place inversion without any device
// allocation, for callers that cannot allocate GPU memory. Examples: code
// running inside a custom allocator or memory pool callback, plugins whose
// host application owns every allocation, and contexts where allocation
// could deadlock or break a memory budget that another component enforces.
//
// The FP64 kernels need scratch memory beyond the caller's matrix: the
// inverted pivot block, a copy of the block column being eliminated, and a
// two-word status. Here that scratch is one file-scope __device__ array of
// fixed size, created when the library is loaded and kept by every GPU that
// loads it until the process exits. Limits: order n <= 2048, every diagonal
// block <= 256 (scratch: 256 x 256 + 2048 x 256 doubles + 256 bytes, about
// 4.5 MiB per device).
//
// In host code the array's name is only a host-side stand-in, not a device
// address, so the address is looked up with cudaGetSymbolAddress the first
// time the entry point runs on each device (with that device current) and
// cached. All calls share the one array and it keeps the previous call's
// contents; the status words are cleared at the start of every call. Calls
// whose GPU work overlaps (two streams, or two host threads, on the same
// device) race on the array and must be serialised by the caller.
#include <mutex>

#include "internal.h"

namespace blockinv {
namespace {

constexpr int64_t kNoAllocMaxN = 2048;
constexpr int kNoAllocMaxBlock = 256;
constexpr size_t kPinvBytes = sizeof(double) * kNoAllocMaxBlock * kNoAllocMaxBlock;
constexpr size_t kUBytes = sizeof(double) * kNoAllocMaxN * kNoAllocMaxBlock;
constexpr size_t kStatusBytes = 256;
constexpr size_t kScratchBytes = kPinvBytes + kUBytes + kStatusBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices];  // per device, filled on first use

// Device address of the scratch array on the current device.
cudaError_t scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return cudaSuccess;
}

}  // namespace
}  // namespace blockinv

extern "C" int blockinv_invert_noalloc(int64_t n, int32_t p, const int32_t* block_sizes, double* A, int64_t lda,
                                       void* stream, int64_t* failing_block) {
  using namespace blockinv;
  if (failing_block) *failing_block = -1;
  // Validate everything on the host first: no GPU work for bad arguments.
  if (n < 1 || n > kNoAllocMaxN || lda < n || !A || p < 1 || p > n || !block_sizes)
    return BLOCKINV_ERR_INVALID;
  int64_t sum = 0;
  for (int32_t k = 0; k < p; ++k) {
    if (block_sizes[k] < 1 || block_sizes[k] > kNoAllocMaxBlock) return BLOCKINV_ERR_INVALID;
    sum += block_sizes[k];
  }
  if (sum != n) return BLOCKINV_ERR_INVALID;

  unsigned char* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return BLOCKINV_ERR_CUDA;
  double* Pinv = reinterpret_cast<double*>(scratch);
  double* U = reinterpret_cast<double*>(scratch + kPinvBytes);
  int32_t* status = reinterpret_cast<int32_t*>(scratch + kPinvBytes + kUBytes);

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(status, 0, 2 * sizeof(int32_t), s);
  int o = 0;
  for (int32_t k = 0; k < p && e == cudaSuccess; ++k) {
    const int b = block_sizes[k];
    e = launch_pivot_inverse<double>(A + (int64_t)o * lda + o, lda, b, Pinv, b, status, k, s);
    if (e == cudaSuccess) e = launch_row_panel_f64(A, lda, (int)n, o, b, Pinv, U, status, s);
    if (e == cudaSuccess) e = launch_schur_update_f64(A, lda, (int)n, o, b, U, status, s);
    o += b;
  }
  int32_t host[2] = {0, -1};
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, status, sizeof(host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  if (host[0] != BLOCKINV_OK && failing_block) *failing_block = host[1];
  return host[0];
}
