// Batched inversion of many independent matrices of uneven orders (FP64).
//
// Elimination step k of every matrix runs in three grouped launches over the
// whole batch: one pivot-block Gauss-Jordan CTA per matrix, one row-panel CTA
// per 32-column strip, one Schur-update CTA per 64 x 64 tile, with the
// matrix of each CTA found from prefix sums in a device descriptor table. A
// batch of 2000 matrices of 4 blocks each thus costs 12 launches, not 24000.
// A plan builds the descriptor tables and the per-matrix workspace once; its
// first run captures the launch sequence in a CUDA graph, and later runs
// replay the graph on the caller's stream.
//
// Pivot blocks of order <= 128 use the grouped one-CTA kernel; larger ones
// (rare in a batch) use the per-matrix cluster kernel, inside the same graph.
#include <algorithm>
#include <vector>

#include "batched.h"

namespace blockinv {

namespace {

__global__ void gather_status_kernel(const int32_t* __restrict__ words, int count, int32_t* __restrict__ out) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < count; m += gridDim.x * blockDim.x)
    out[m] = words[2 * m];
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

// Default partition of a matrix in a batch: the paper's Table 2 rule below
// order 8 (n <= 3: one block); otherwise four blocks of floor(n / 4) (more
// blocks when that exceeds 128), the last blocks taking the remainder.
void batch_default_partition(int n, std::vector<int>* out) {
  out->clear();
  if (n <= 3) {
    out->push_back(n);
    return;
  }
  if (n < 8) {  // N_k = 2 blocks of order 2..4
    out->assign(2, 2);
    int r = n - 4, pos = 1;
    while (r-- > 0) {
      (*out)[pos] += 1;
      pos = (pos == 0) ? 1 : 0;
    }
    return;
  }
  const int p = std::max(4, (n + kGroupedMaxB - 1) / kGroupedMaxB);
  const int q = n / p, r = n % p;
  for (int i = 0; i < p; ++i) out->push_back(q + (i >= p - r ? 1 : 0));
}

int batch_plan_create(int32_t count, const int32_t* n, const int32_t* p, const int32_t* block_sizes,
                      double* const* A, const int64_t* lda, BatchPlan** out) {
  *out = nullptr;
  if (count < 1 || !n || !A || !lda || (block_sizes && !p)) return BLOCKINV_ERR_INVALID;
  BatchPlan tmp;
  tmp.count = count;
  std::vector<int> part;
  size_t scur = 0;
  for (int m = 0; m < count; ++m) {
    if (n[m] < 1 || n[m] > (1 << 16) || lda[m] < n[m] || !A[m]) return BLOCKINV_ERR_INVALID;
    if (block_sizes) {
      if (p[m] < 1 || p[m] > n[m]) return BLOCKINV_ERR_INVALID;
      part.assign(block_sizes + scur, block_sizes + scur + p[m]);
      scur += p[m];
    } else {
      batch_default_partition(n[m], &part);
    }
    int64_t sum = 0;
    for (int b : part) {
      if (b < 1 || b > BLOCKINV_MAX_BLOCK) return BLOCKINV_ERR_INVALID;
      sum += b;
    }
    if (sum != n[m]) return BLOCKINV_ERR_INVALID;
    tmp.n.push_back(n[m]);
    tmp.p.push_back((int)part.size());
    tmp.off.push_back((int)tmp.sizes.size());
    tmp.sizes.insert(tmp.sizes.end(), part.begin(), part.end());
    tmp.A.push_back(A[m]);
    tmp.lda.push_back(lda[m]);
    tmp.max_steps = std::max(tmp.max_steps, (int)part.size());
  }
  // per-matrix workspace: Pinv (bmax^2) then U (n x bmax)
  std::vector<size_t> ws_off(count);
  std::vector<int> bm(count, 0);
  size_t ws_total = 0;
  for (int m = 0; m < count; ++m) {
    for (int k = 0; k < tmp.p[m]; ++k) bm[m] = std::max(bm[m], tmp.sizes[tmp.off[m] + k]);
    ws_off[m] = ws_total;
    ws_total = align256(ws_total + sizeof(double) * ((size_t)bm[m] * bm[m] + (size_t)tmp.n[m] * bm[m]));
  }
  // descriptor tables, step by step
  std::vector<GroupStep> items;
  std::vector<int32_t> starts;
  tmp.steps.resize(tmp.max_steps);
  std::vector<int> item_m;  // matrix of each item
  for (int k = 0; k < tmp.max_steps; ++k) {
    BatchStep& st = tmp.steps[k];
    st.item_off = (int)items.size();
    st.cs_off = (int)starts.size();
    int cols = 0, tiles = 0;
    std::vector<int32_t> ts{0};
    starts.push_back(0);
    for (int m = 0; m < count; ++m) {
      if (k >= tmp.p[m]) continue;
      const int b = tmp.sizes[tmp.off[m] + k];
      int o = 0;
      for (int q = 0; q < k; ++q) o += tmp.sizes[tmp.off[m] + q];
      GroupStep g{};
      g.X = tmp.A[m];
      g.ldx = tmp.lda[m];
      g.n = tmp.n[m];
      g.o = o;
      g.b = b;
      g.k = k;
      items.push_back(g);
      item_m.push_back(m);
      const int nn = tmp.n[m];
      cols += (nn + 31) / 32;
      tiles += ((nn + 63) / 64) * ((nn + 63) / 64);
      starts.push_back(cols);
      ts.push_back(tiles);
      st.bmax = std::max(st.bmax, b);
      ++st.count;
      const double bd = b, nd = nn, rest = nn - b;
      tmp.flops += 2.0 * bd * bd * bd + 2.0 * bd * bd * rest + 2.0 * bd * rest * nd;
      tmp.bytes += 8.0 * (2.0 * bd * bd + 2.0 * bd * nd + 2.0 * rest * nd + 2.0 * rest * bd);
    }
    st.cols = cols;
    st.tiles = tiles;
    st.ts_off = (int)starts.size();
    starts.insert(starts.end(), ts.begin(), ts.end());
  }
  const size_t o_items = 0;
  const size_t o_starts = align256(sizeof(GroupStep) * items.size());
  const size_t o_status = o_starts + align256(sizeof(int32_t) * starts.size());
  const size_t o_ws = o_status + align256(sizeof(int32_t) * 2 * count);
  const size_t total = o_ws + ws_total;
  if (cudaGetDevice(&tmp.device) != cudaSuccess) return BLOCKINV_ERR_CUDA;
  void* dev = nullptr;
  if (cudaMalloc(&dev, total) != cudaSuccess) return BLOCKINV_ERR_NOMEM;
  char* base = static_cast<char*>(dev);
  tmp.dev = dev;
  tmp.items = reinterpret_cast<GroupStep*>(base + o_items);
  tmp.starts = reinterpret_cast<int32_t*>(base + o_starts);
  tmp.status = reinterpret_cast<int32_t*>(base + o_status);
  for (size_t i = 0; i < items.size(); ++i) {
    const int m = item_m[i];
    GroupStep& g = items[i];
    g.Pinv = reinterpret_cast<double*>(base + o_ws + ws_off[m]);
    g.U = g.Pinv + (size_t)bm[m] * bm[m];
    g.status = tmp.status + 2 * m;
    if (g.b > kGroupedMaxB) tmp.steps[g.k].big.push_back(g);
  }
  cudaError_t e = cudaMemcpy(base + o_items, items.data(), sizeof(GroupStep) * items.size(),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(base + o_starts, starts.data(), sizeof(int32_t) * starts.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return BLOCKINV_ERR_CUDA;
  }
  *out = new BatchPlan(std::move(tmp));
  return BLOCKINV_OK;
}

cudaError_t batch_enqueue(const BatchPlan& pl, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(pl.status, 0, sizeof(int32_t) * 2 * pl.count, s);
  for (int k = 0; k < pl.max_steps && e == cudaSuccess; ++k) {
    const BatchStep& st = pl.steps[k];
    const GroupStep* it = pl.items + st.item_off;
    e = launch_pivot_grouped(it, st.count, std::min(st.bmax, kGroupedMaxB), s);
    for (const GroupStep& g : st.big) {
      if (e != cudaSuccess) break;
      e = launch_pivot_inverse<double>(g.X + (int64_t)g.o * g.ldx + g.o, g.ldx, g.b, g.Pinv, g.b, g.status, g.k,
                                       s);
    }
    if (e == cudaSuccess) e = launch_row_panel_grouped(it, st.count, pl.starts + st.cs_off, st.cols, st.bmax, s);
    if (e == cudaSuccess) e = launch_schur_update_grouped(it, st.count, pl.starts + st.ts_off, st.tiles, s);
  }
  return e;
}

cudaError_t batch_run(BatchPlan& pl, cudaStream_t s, int32_t* status_out, bool use_graph) {
  cudaError_t e = cudaSuccess;
  if (use_graph) {
    if (!pl.exec) {
      cudaStream_t cap;
      e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e2 = batch_enqueue(pl, cap);
        e = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&pl.exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cap);
      if (e != cudaSuccess) return e;
    }
    e = cudaGraphLaunch(pl.exec, s);
  } else {
    e = batch_enqueue(pl, s);
  }
  if (e == cudaSuccess && status_out) {
    gather_status_kernel<<<(pl.count + 255) / 256, 256, 0, s>>>(pl.status, pl.count, status_out);
    e = cudaGetLastError();
  }
  return e;
}

void batch_plan_destroy(BatchPlan* pl) {
  if (!pl) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->dev) cudaFree(pl->dev);
  delete pl;
}

}  // namespace blockinv

using namespace blockinv;

extern "C" {

int blockinv_batch_plan_create(int32_t count, const int32_t* n, const int32_t* p, const int32_t* block_sizes,
                               double* const* A, const int64_t* lda, blockinv_batch_plan** plan) {
  if (!plan) return BLOCKINV_ERR_INVALID;
  *plan = nullptr;
  BatchPlan* pl = nullptr;
  const int st = batch_plan_create(count, n, p, block_sizes, A, lda, &pl);
  if (st == BLOCKINV_OK) *plan = reinterpret_cast<blockinv_batch_plan*>(pl);
  return st;
}

int blockinv_batch_plan_run(blockinv_batch_plan* plan, void* stream, int32_t* status_dev) {
  if (!plan) return BLOCKINV_ERR_INVALID;
  BatchPlan* pl = reinterpret_cast<BatchPlan*>(plan);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  {
    TraceScope t("batched_grouped_f64", pl->flops, pl->bytes, s);
    e = batch_run(*pl, s, status_dev, true);
  }
  return e == cudaSuccess ? BLOCKINV_OK : (e == cudaErrorMemoryAllocation ? BLOCKINV_ERR_NOMEM : BLOCKINV_ERR_CUDA);
}

int blockinv_batch_plan_destroy(blockinv_batch_plan* plan) {
  batch_plan_destroy(reinterpret_cast<BatchPlan*>(plan));
  return BLOCKINV_OK;
}

int blockinv_invert_batched(int32_t count, const int32_t* n, const int32_t* p, const int32_t* block_sizes,
                            double* const* A, const int64_t* lda, int mode, void* stream, int32_t* status_dev) {
  if (mode != BLOCKINV_F64) return BLOCKINV_ERR_INVALID;
  BatchPlan* pl = nullptr;
  int st = batch_plan_create(count, n, p, block_sizes, A, lda, &pl);
  if (st != BLOCKINV_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  {
    TraceScope t("batched_grouped_f64", pl->flops, pl->bytes, s);
    e = batch_run(*pl, s, status_dev, false);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  batch_plan_destroy(pl);
  return e == cudaSuccess ? BLOCKINV_OK : BLOCKINV_ERR_CUDA;
}

}  // extern "C"
