// Internal declarations shared by the translation units of libblockinv.so.
// Not installed; the public ABI is include/blockinv.h.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/blockinv.h"

namespace blockinv {

// Device status word layout: status[0] = BLOCKINV_* code (0 = OK),
// status[1] = failing block index. Kernels set it with atomicCAS so that the
// first error wins, and later kernels of the same inversion return early
// once it is set.
struct DevStatus {
  int32_t code;
  int32_t block;
};

// Validated partition of an order-n matrix into diagonal blocks.
struct Plan {
  int n = 0;
  std::vector<int> sizes;
  std::vector<int> offs;
  int bmax = 0;
};

// RAII kernel tracer: when tracing is on, brackets the enclosed launch with two
// CUDA events on stream s and records its algorithmic flops and bytes.
class TraceScope {
 public:
  TraceScope(const char* name, double flops, double bytes, cudaStream_t s);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;

 private:
  const char* name_ = nullptr;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
  double flops_ = 0, bytes_ = 0;
  cudaStream_t s_ = nullptr;
};

// Host-side choice of the pivot-kernel cluster shape for a block of order b.
struct PivotPlan {
  int b;        // block order
  int rows;     // rows held by each CTA
  int ctas;     // CTAs in the cluster (1 = no cluster)
  size_t smem;  // dynamic shared memory per CTA
};

bool plan_pivot(int b, int elem_bytes, PivotPlan* plan);

// Copy an n x n FP64 matrix between row-major buffers with leading dimensions
// dld and sld (in elements): one plain copy when both are n (a pitched copy of
// contiguous rows ran at about 29 GB/s from pinned host memory, against
// 190-210 GB/s for the plain one), the pitched form otherwise.
inline cudaError_t copy_matrix(void* dst, int64_t dld, const void* src, int64_t sld, int64_t n, cudaMemcpyKind kind,
                               cudaStream_t s) {
  const size_t row = sizeof(double) * (size_t)n;
  if (dld == n && sld == n) return cudaMemcpyAsync(dst, src, row * (size_t)n, kind, s);
  return cudaMemcpy2DAsync(dst, sizeof(double) * (size_t)dld, src, sizeof(double) * (size_t)sld, row, (size_t)n,
                           kind, s);
}

// One matrix's elimination step k in a grouped (batched) launch.
struct GroupStep {
  double* X;       // matrix (device), row-major
  int64_t ldx;
  int n, o, b, k;  // order, pivot offset, pivot order, step index
  double* Pinv;    // b x b workspace
  double* U;       // n x b workspace
  int32_t* status; // this matrix's status word pair
};
// Largest pivot order of the grouped (one CTA per matrix) pivot kernel.
constexpr int kGroupedMaxB = 128;
cudaError_t launch_pivot_grouped(const GroupStep* items, int count, int bmax, cudaStream_t s);
// Grouped K2 / K3 over `count` items; col_start / tile_start are exclusive
// prefix sums (count + 1 entries) of each item's column strips / tile x tile
// tiles (tile = 64 or 32).
cudaError_t launch_row_panel_grouped(const GroupStep* items, int count, const int32_t* col_start,
                                     int total_cols, int bmax, cudaStream_t s);
cudaError_t launch_schur_update_grouped(const GroupStep* items, int count, const int32_t* tile_start,
                                        int total_tiles, int tile, cudaStream_t s);

// K1: P^-1 of the b x b pivot block at P (leading dimension ldp) into Pinv
// (leading dimension ldo). T = double (FP64 path) or float (mixed path).
template <typename T>
cudaError_t launch_pivot_inverse(const T* P, int64_t ldp, int b, T* Pinv, int64_t ldo,
                                 int32_t* status, int block_index, cudaStream_t s);

// Mixed path, after the FP32 pivot inverse Pinv of the FP32 block P (gate and
// count are device int32):
// - launch_pivot_cond estimates kappa = ||P||_inf ||Pinv||_inf on the device
//   (one CTA); if kappa > cond_limit (always when cond_limit < 0) it sets
//   *gate and counts the block in *count. With after_trigger it is launched as
//   the programmatic dependent of the kernel before it, whose completion it
//   awaits and whose own dependent it lets start at once.
// - launch_pivot_f64_gated inverts P again in FP64 arithmetic (FP32 in and
//   out) when *gate is set, and returns at once otherwise.
cudaError_t launch_pivot_cond(const float* P, int64_t ldp, int b, const float* Pinv, int64_t ldo,
                              const int32_t* status, float cond_limit, int32_t* gate, int32_t* count,
                              bool after_trigger, cudaStream_t s);
cudaError_t launch_pivot_f64_gated(const float* P, int64_t ldp, int b, float* Pinv, int64_t ldo, int32_t* status,
                                   int block_index, const int32_t* gate, cudaStream_t s);

// CTAs (hence SMs) the widest launch of one pivot inverse of order b takes:
// launch_pivot_inverse with elements of elem bytes, and with f64_check also
// launch_pivot_f64_gated.
int pivot_inverse_ctas(int b, int elem, bool f64_check);

// K2 (FP64): row panel X[o:o+b, j] <- Pinv X[o:o+b, j] for j outside the
// pivot columns, X[o:o+b, o:o+b] <- Pinv, and U <- X[:, o:o+b] for rows
// outside the pivot rows (U is n x b, leading dimension b).
cudaError_t launch_row_panel_f64(double* X, int64_t ldx, int n, int o, int b,
                                 const double* Pinv, double* U, const int32_t* status,
                                 cudaStream_t s);

// K3 (FP64): X[i, j] <- (j in pivot cols ? 0 : X[i, j]) - U[i, :] X[o:o+b, j]
// for every row i outside the pivot rows and every column j.
cudaError_t launch_schur_update_f64(double* X, int64_t ldx, int n, int o, int b,
                                    const double* U, const int32_t* status, cudaStream_t s);

// K3 split for look-ahead: next_part = the elements of block row / column
// B1 = [o1, o1 + b1) (the next step's panels); otherwise every other element.
cudaError_t launch_schur_split_f64(double* X, int64_t ldx, int n, int o, int b, const double* U,
                                   const int32_t* status, int o1, int b1, bool next_part, cudaStream_t s);

// Residual pieces (FP64): partial sums of ||A X - I||_F^2, ||A||_F^2, ||X||_F^2.
cudaError_t launch_residual_f64(int n, const double* A, int64_t lda, const double* X,
                                int64_t ldx, double* sums3, cudaStream_t s);

// Mixed-precision elimination (k_mixed.cu).
cudaError_t launch_cast_f64_to_f32(const double* A, int64_t lda, float* X, int64_t ldx, int n, cudaStream_t s);
cudaError_t launch_cast_f32_to_f64(const float* X, int64_t ldx, double* A, int64_t lda, int n, cudaStream_t s);
int mixed_kpad(int bmax);
// Runs every elimination step on X32 (n x n, leading dimension ld32). Pinv is
// bmax^2 floats; U and Vt are n x (2 * nsl * mixed_kpad(bmax)) operands of 4
// (TF32) or 2 (BF16) bytes per element (two steps' slice sets); nsl = 2
// splits each operand into hi + lo and runs the three products
// hi*hi + hi*lo + lo*hi.
// pivot_cond_limit: > 0, pivot blocks whose condition estimate exceeds it are
// inverted again in FP64 arithmetic (launch_pivot_cond, launch_pivot_f64_gated); < 0, every
// block; 0, none. piv_words: device int32[2] (gate, count of FP64 pivots).
// lookahead: with 3 or more blocks, each next pivot inverse runs beside the
// rest of the current Schur update (same stream, programmatic dependent
// launch); the result bits are the same. fuse (with lookahead, 2 or more
// blocks): the Schur updates of two consecutive steps run as one sweep over
// X32 (rank b_k + b_{k+1}), after step k has updated block row and column
// k + 1 only; the sums are associated differently from one step at a time.
cudaError_t mixed_elimination(const Plan& pl, bool bf16, int nsl, float* X32, int64_t ld32, float* Pinv, void* U,
                              void* Vt, float pivot_cond_limit, int32_t* piv_words, int32_t* status, cudaStream_t s,
                              bool lookahead, bool fuse);

// A synthetic diagonally dominant matrix of order n (U[-1,1) from a hash of
// (seed, index) plus n on the diagonal) for the autotuners (batched.cu).
cudaError_t launch_fill_diag_dominant(double* A, int n, unsigned long long seed, cudaStream_t s);

// Batched small matrices, order 1..8, one thread per matrix (k_small.cu).
cudaError_t launch_small_batched(int n, double* A, int64_t count, int32_t* status, cudaStream_t s);

// Hooks the serving loop (serve.cu) uses to run one request (api.cu).
struct ServeJob;
// The library's device memory pool for workspace on the current device.
cudaError_t workspace_pool(cudaMemPool_t* out);

// Status of a CUDA runtime result: OK, NOMEM for an allocation failure, else
// ERR_CUDA. A failure is also kept as the library's last CUDA error (any
// thread), which blockinv_last_cuda_error reports.
int cuda_status(cudaError_t e);

// The paper's partition rule (Table 2) for any order (blocks of order 2..4).
void paper_partition(int n, std::vector<int>* out);

// Batched matrices of one order n <= 32 with one partition (k_tiny.cu).
cudaError_t launch_tiny_batched(int n, const std::vector<int>& sizes, bool spd, double* A, int64_t count,
                                int32_t* status, cudaStream_t s);

// Partition plan (the checks of blockinv_invert); FP64 elimination steps
// k0 .. k1 - 1 in place, blocking, status as blockinv_invert.
int plan_for(int64_t n, int32_t p, const int32_t* block_sizes, int64_t lda, Plan* pl);
int invert_steps(const Plan& pl, double* A, int64_t lda, int k0, int k1, cudaStream_t s);
int serve_make_plan(int64_t n, int32_t p, const int32_t* block_sizes, int64_t lda, int mode, Plan* pl);
size_t serve_footprint(const Plan& pl, int mode);
int serve_enqueue(const Plan& pl, double* A, int64_t lda, int mode, int32_t* status, cudaStream_t s, double tol,
                  int max_refine, ServeJob** job);
void serve_job_info(ServeJob* job, cudaStream_t s, double* rho, int* iters);
void serve_job_release(ServeJob* job);
int serve_enqueue_fallback(ServeJob* job, const Plan& pl, double* A, int64_t lda, int32_t* status,
                           cudaStream_t s);

// Newton-Schulz refinement with the FP64-accurate tensor-core residual (k_refine.cu).
constexpr int kRefineCtlWords = 8;      // int32 control words of a refinement
constexpr int kResidualSlices = 9;      // base-32 digits per operand (44 bits)
constexpr int kMinResidualSlices = 7;
constexpr int kMaxResidualSlices = 9;    // int64 accumulator bound at n = 16384
constexpr int64_t kMixedMaxOrder = 16384;
size_t refine_workspace_bytes(int n, int S, int max_updates);
cudaError_t enqueue_refine(const double* A0, int64_t ld0, double* X, int64_t ldx, int n, double tol,
                           int max_updates, int S, void* ws, double* hist, int32_t* ctl_words, int32_t* status,
                           double* Eout, int64_t lde, cudaStream_t s, bool report, bool host_steps);

}  // namespace blockinv
