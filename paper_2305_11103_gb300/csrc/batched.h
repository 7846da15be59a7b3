// Batched (grouped) FP64 inversion of uneven matrices: plan, enqueue, run.
#pragma once
#include <vector>

#include "internal.h"

namespace blockinv {

struct BatchStep {
  int item_off = 0, count = 0;  // items of this step in the descriptor table
  int cs_off = 0, ts_off = 0;   // offsets of the strip / tile prefix sums
  int cols = 0, tiles = 0;      // total strips / tiles
  int bmax = 0;                 // largest pivot block
  std::vector<GroupStep> big;   // items whose pivot block exceeds kGroupedMaxB
};

struct BatchPlan {
  int count = 0, max_steps = 0, device = -1;
  std::vector<int> n, p, off, sizes;
  std::vector<double*> A;
  std::vector<int64_t> lda;
  std::vector<BatchStep> steps;
  void* dev = nullptr;  // descriptors, prefix sums, status words, workspace
  GroupStep* items = nullptr;
  int32_t* starts = nullptr;
  int32_t* status = nullptr;  // 2 words per matrix
  double flops = 0, bytes = 0;
  cudaGraphExec_t exec = nullptr;
};

void batch_default_partition(int n, std::vector<int>* out);
int batch_plan_create(int32_t count, const int32_t* n, const int32_t* p, const int32_t* block_sizes,
                      double* const* A, const int64_t* lda, BatchPlan** out);
cudaError_t batch_enqueue(const BatchPlan& pl, cudaStream_t s);
cudaError_t batch_run(BatchPlan& pl, cudaStream_t s, int32_t* status_out, bool use_graph);
void batch_plan_destroy(BatchPlan* pl);

}  // namespace blockinv
