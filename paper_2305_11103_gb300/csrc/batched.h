// Batched (grouped) FP64 inversion of uneven matrices: plan, enqueue, run.
#pragma once
#include <vector>

#include "internal.h"

namespace blockinv {

struct BatchStep {
  int item_off = 0, count = 0;  // items of this step in the descriptor table
  int cs_off = 0;               // offset of the strip prefix sums (all items)
  int cols = 0;                 // total strips
  int bmax = 0;                 // largest pivot block
  // Schur update in two groups by tile shape: items [item_off, item_off +
  // count64) use 64 x 64 tiles, the rest 32 x 32; each group has its own
  // tile prefix sums.
  int count64 = 0;
  int ts_off64 = 0, tiles64 = 0;
  int ts_off32 = 0, tiles32 = 0;
  std::vector<GroupStep> big;   // items whose pivot block exceeds kGroupedMaxB
};

struct BatchPlan {
  int count = 0, max_steps = 0, device = -1;
  std::vector<int> n, p, off, sizes, tile;
  std::vector<double*> A;
  std::vector<int64_t> lda;
  std::vector<BatchStep> steps;
  void* dev = nullptr;  // descriptors, prefix sums, status words, workspace
  GroupStep* items = nullptr;
  int32_t* starts = nullptr;
  int32_t* status = nullptr;  // 2 words per matrix
  double flops = 0, bytes = 0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t pool_stream = nullptr;  // pooled plans: the stream of their allocation and release
};

// Partition and Schur tile of a matrix of order n in a batch: the tuned
// choice for its size class if the tuner has one, else the default rule with
// 64 x 64 tiles.
void batch_partition(int n, std::vector<int>* out, int* tile);
void batch_default_partition(int n, std::vector<int>* out);
// force_tile: 0 = the tile of each matrix's size class (tuned, else 64);
// tiles (optional): one tile per matrix, overriding both.
// pool_stream: non-null = the device tables and workspace come from the
// library's memory pool in that stream's order (no device-wide
// synchronisation, for the serving loop) and go back to it, in the same
// order, when the plan is destroyed; the tables are copied from `staging`
// (pinned, *staging_bytes long; on return the bytes needed, and
// BLOCKINV_ERR_NOMEM if that is more), which the caller leaves untouched
// until the stream has passed the copies.
int batch_plan_create(int32_t count, const int32_t* n, const int32_t* p, const int32_t* block_sizes,
                      double* const* A, const int64_t* lda, BatchPlan** out, int force_tile = 0,
                      const int* tiles = nullptr, cudaStream_t pool_stream = nullptr, void* staging = nullptr,
                      size_t* staging_bytes = nullptr);
// Autotuner: time the candidate partitions and Schur tiles of every size
// class present in n[] and keep the fastest in the process-wide table.
int batch_tune(int32_t count, const int32_t* n, int reps, cudaStream_t s);
cudaError_t batch_enqueue(const BatchPlan& pl, cudaStream_t s);
cudaError_t batch_run(BatchPlan& pl, cudaStream_t s, int32_t* status_out, bool use_graph);
void batch_plan_destroy(BatchPlan* pl);

}  // namespace blockinv
