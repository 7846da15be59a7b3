// Internal declarations shared by the translation units of libblockinv.so.
// Not installed; the public ABI is include/blockinv.h.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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

// Host-side choice of the pivot-kernel cluster shape for a block of order b.
struct PivotPlan {
  int b;        // block order
  int rows;     // rows held by each CTA
  int ctas;     // CTAs in the cluster (1 = no cluster)
  size_t smem;  // dynamic shared memory per CTA
};

bool plan_pivot(int b, int elem_bytes, PivotPlan* plan);

// K1: P^-1 of the b x b pivot block at P (leading dimension ldp) into Pinv
// (leading dimension ldo). T = double (FP64 path) or float (mixed path).
template <typename T>
cudaError_t launch_pivot_inverse(const T* P, int64_t ldp, int b, T* Pinv, int64_t ldo,
                                 int32_t* status, int block_index, cudaStream_t s);

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

// Residual pieces (FP64): partial sums of ||A X - I||_F^2, ||A||_F^2, ||X||_F^2.
cudaError_t launch_residual_f64(int n, const double* A, int64_t lda, const double* X,
                                int64_t ldx, double* sums3, cudaStream_t s);

}  // namespace blockinv
