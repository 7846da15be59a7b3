// Batched inversion of many independent matrices of uneven orders (FP64).
//
// Elimination step k of every matrix runs in grouped launches over the whole
// batch: one pivot-block Gauss-Jordan CTA per matrix, one row-panel CTA per
// 32-column strip, one Schur-update CTA per 64 x 64 (or 32 x 32) tile, with
// the matrix of each CTA found from prefix sums in a device descriptor table.
// A batch of 2000 matrices of 4 blocks each thus costs about 12 launches, not
// 24000. A plan builds the descriptor tables and the per-matrix workspace
// once; its first run captures the launch sequence in a CUDA graph, and later
// runs replay the graph on the caller's stream.
//
// Pivot blocks of order <= 128 use the grouped one-CTA kernel; larger ones
// (rare in a batch) use the per-matrix cluster kernel, inside the same graph.
//
// Autotuner. Matrices fall into size classes c = floor(log2 n) (n >= 8). The
// tuner builds a synthetic diagonally dominant batch with the caller's orders
// and, class by class (largest total work first), times every candidate
// (number of near-equal blocks p, Schur tile 64 or 32) on the whole batch
// with the other classes at their current choice, keeping the fastest (or the
// current one) in a process-wide table, which can be saved to and loaded
// from a text file. Plans built without explicit partitions use the table.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "batched.h"

namespace blockinv {

namespace {

__global__ void gather_status_kernel(const int32_t* __restrict__ words, int count, int32_t* __restrict__ out) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < count; m += gridDim.x * blockDim.x)
    out[m] = words[2 * m];
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

constexpr int kMinClass = 3;   // orders 8..15
constexpr int kMaxClass = 16;  // orders up to 2^17 - 1 (plans accept n <= 2^16)

struct Tuned {
  int p = 0;      // blocks (0 = not tuned)
  int tile = 64;  // Schur tile
};

std::mutex g_tune_mu;
Tuned g_tune[kMaxClass + 1];

int size_class(int n) {
  if (n < 8) return -1;
  int c = 0;
  while ((2 << c) <= n) ++c;
  return c;  // 2^c <= n < 2^(c+1)
}

// n split into p near-equal blocks, the last (n mod p) one larger.
void equal_partition(int n, int p, std::vector<int>* out) {
  out->clear();
  const int q = n / p, r = n % p;
  for (int i = 0; i < p; ++i) out->push_back(q + (i >= p - r ? 1 : 0));
}

// Synthetic diagonally dominant matrices for timing: a[i][j] = h(m, i, j) in
// [-1, 1) plus n on the diagonal (h: a 64-bit integer mix of the indices).
__global__ void fill_tune_kernel(double* const* __restrict__ A, const int32_t* __restrict__ n) {
  const int m = blockIdx.x;
  double* a = A[m];
  const int nn = n[m];
  for (int64_t e = threadIdx.x; e < (int64_t)nn * nn; e += blockDim.x) {
    unsigned long long z = (static_cast<unsigned long long>(m) << 40) ^ static_cast<unsigned long long>(e);
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = static_cast<double>(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    const int i = static_cast<int>(e / nn), j = static_cast<int>(e - (int64_t)i * nn);
    a[e] = u + (i == j ? static_cast<double>(nn) : 0.0);
  }
}

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
  equal_partition(n, p, out);
}

void batch_partition(int n, std::vector<int>* out, int* tile) {
  const int c = size_class(n);
  Tuned t;
  if (c >= kMinClass && c <= kMaxClass) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    t = g_tune[c];
  }
  *tile = t.tile;
  if (t.p > 0 && t.p <= n && (n + t.p - 1) / t.p <= BLOCKINV_MAX_BLOCK)
    equal_partition(n, t.p, out);
  else
    batch_default_partition(n, out);
}

namespace {

// One synthetic diagonally dominant matrix of order n for timing (row-major,
// leading dimension n): a[i][j] in [-1, 1) from a 64-bit mix of (seed, index),
// plus n on the diagonal.
__global__ void fill_dd_kernel(double* __restrict__ a, int n, unsigned long long seed) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long z = (seed << 40) ^ static_cast<unsigned long long>(e);
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = static_cast<double>(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    const int i = static_cast<int>(e / n), j = static_cast<int>(e - (int64_t)i * n);
    a[e] = u + (i == j ? static_cast<double>(n) : 0.0);
  }
}

}  // namespace

cudaError_t launch_fill_diag_dominant(double* A, int n, unsigned long long seed, cudaStream_t s) {
  const int64_t total = (int64_t)n * n;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  fill_dd_kernel<<<blocks, 256, 0, s>>>(A, n, seed);
  return cudaGetLastError();
}

int batch_plan_create(int32_t count, const int32_t* n, const int32_t* p, const int32_t* block_sizes,
                      double* const* A, const int64_t* lda, BatchPlan** out, int force_tile, const int* tiles,
                      cudaStream_t pool_stream, void* staging, size_t* staging_bytes) {
  *out = nullptr;
  if (count < 1 || !n || !A || !lda || (block_sizes && !p)) return BLOCKINV_ERR_INVALID;
  BatchPlan tmp;
  tmp.count = count;
  std::vector<int> part;
  size_t scur = 0;
  for (int m = 0; m < count; ++m) {
    if (n[m] < 1 || n[m] > (1 << 16) || lda[m] < n[m] || !A[m]) return BLOCKINV_ERR_INVALID;
    int tile = 64;
    if (block_sizes) {
      if (p[m] < 1 || p[m] > n[m]) return BLOCKINV_ERR_INVALID;
      part.assign(block_sizes + scur, block_sizes + scur + p[m]);
      scur += p[m];
      std::vector<int> unused;
      batch_partition(n[m], &unused, &tile);  // the class's tuned tile, if any
    } else {
      batch_partition(n[m], &part, &tile);
    }
    if (force_tile) tile = force_tile;
    if (tiles) tile = tiles[m];
    int64_t sum = 0;
    for (int b : part) {
      if (b < 1 || b > BLOCKINV_MAX_BLOCK) return BLOCKINV_ERR_INVALID;
      sum += b;
    }
    if (sum != n[m]) return BLOCKINV_ERR_INVALID;
    tmp.n.push_back(n[m]);
    tmp.p.push_back((int)part.size());
    tmp.off.push_back((int)tmp.sizes.size());
    tmp.tile.push_back(tile);
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
  // descriptor tables, step by step: the 64-tile items, then the 32-tile ones
  std::vector<GroupStep> items;
  std::vector<int32_t> starts;
  tmp.steps.resize(tmp.max_steps);
  std::vector<int> item_m;  // matrix of each item
  for (int k = 0; k < tmp.max_steps; ++k) {
    BatchStep& st = tmp.steps[k];
    st.item_off = (int)items.size();
    st.cs_off = (int)starts.size();
    int cols = 0;
    starts.push_back(0);
    std::vector<int32_t> ts[2] = {{0}, {0}};
    int tiles[2] = {0, 0};
    for (int grp = 0; grp < 2; ++grp) {
      const int want = grp == 0 ? 64 : 32;
      for (int m = 0; m < count; ++m) {
        if (k >= tmp.p[m] || tmp.tile[m] != want) continue;
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
        // Schur tiles over the nn - b rows outside the pivot block
        tiles[grp] += ((nn - b + want - 1) / want) * ((nn + want - 1) / want);
        starts.push_back(cols);
        ts[grp].push_back(tiles[grp]);
        st.bmax = std::max(st.bmax, b);
        ++st.count;
        if (grp == 0) ++st.count64;
        const double bd = b, nd = nn, rest = nn - b;
        tmp.flops += 2.0 * bd * bd * bd + 2.0 * bd * bd * rest + 2.0 * bd * rest * nd;
        tmp.bytes += 8.0 * (2.0 * bd * bd + 2.0 * bd * nd + 2.0 * rest * nd + 2.0 * rest * bd);
      }
    }
    st.cols = cols;
    st.tiles64 = tiles[0];
    st.tiles32 = tiles[1];
    st.ts_off64 = (int)starts.size();
    starts.insert(starts.end(), ts[0].begin(), ts[0].end());
    st.ts_off32 = (int)starts.size();
    starts.insert(starts.end(), ts[1].begin(), ts[1].end());
  }
  const size_t o_items = 0;
  const size_t o_starts = align256(sizeof(GroupStep) * items.size());
  const size_t o_status = o_starts + align256(sizeof(int32_t) * starts.size());
  const size_t o_ws = o_status + align256(sizeof(int32_t) * 2 * count);
  const size_t total = o_ws + ws_total;
  const size_t tb = sizeof(GroupStep) * items.size(), sb = sizeof(int32_t) * starts.size();
  if (pool_stream) {  // the caller's pinned staging must hold both tables
    const size_t need = tb + sb;
    const size_t cap = staging_bytes ? *staging_bytes : 0;
    if (staging_bytes) *staging_bytes = need;
    if (!staging || cap < need) return BLOCKINV_ERR_NOMEM;
  }
  const cudaError_t ed = cudaGetDevice(&tmp.device);
  if (ed != cudaSuccess) return cuda_status(ed);
  void* dev = nullptr;
  if (pool_stream) {
    // stream-ordered, from the library's pool (no device-wide synchronisation)
    cudaMemPool_t pool = nullptr;
    cudaError_t ep = workspace_pool(&pool);
    if (ep == cudaSuccess) ep = cudaMallocFromPoolAsync(&dev, total, pool, pool_stream);
    if (ep != cudaSuccess) return cuda_status(ep);
    tmp.pool_stream = pool_stream;
  } else if (cudaMalloc(&dev, total) != cudaSuccess) {
    return BLOCKINV_ERR_NOMEM;
  }
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
  cudaError_t e;
  if (pool_stream) {
    // the tables go through the caller's pinned staging, which must stay
    // untouched until the work on pool_stream has passed these copies
    memcpy(staging, items.data(), tb);
    memcpy(static_cast<char*>(staging) + tb, starts.data(), sb);
    e = cudaMemcpyAsync(base + o_items, staging, tb, cudaMemcpyHostToDevice, pool_stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(base + o_starts, static_cast<char*>(staging) + tb, sb, cudaMemcpyHostToDevice, pool_stream);
    if (e != cudaSuccess) {
      cudaFreeAsync(dev, pool_stream);
      return cuda_status(e);
    }
  } else {
    e = cudaMemcpy(base + o_items, items.data(), sizeof(GroupStep) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(base + o_starts, starts.data(), sizeof(int32_t) * starts.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(dev);
      return cuda_status(e);
    }
  }
  *out = new BatchPlan(std::move(tmp));
  return BLOCKINV_OK;
}

cudaError_t batch_enqueue(const BatchPlan& pl, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(pl.status, 0, sizeof(int32_t) * 2 * pl.count, s);
  // per-kernel tracing only when the launches run now (not into a graph)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  const bool trace = cap == cudaStreamCaptureStatusNone;
  for (int k = 0; k < pl.max_steps && e == cudaSuccess; ++k) {
    const BatchStep& st = pl.steps[k];
    const GroupStep* it = pl.items + st.item_off;
    {
      TraceScope t(trace ? "batched_step_pivot" : nullptr, 0, 0, s);
      e = launch_pivot_grouped(it, st.count, std::min(st.bmax, kGroupedMaxB), s);
      for (const GroupStep& g : st.big) {
        if (e != cudaSuccess) break;
        e = launch_pivot_inverse<double>(g.X + (int64_t)g.o * g.ldx + g.o, g.ldx, g.b, g.Pinv, g.b, g.status, g.k,
                                         s);
      }
    }
    if (e == cudaSuccess) {
      TraceScope t(trace ? "batched_step_row_panel" : nullptr, 0, 0, s);
      e = launch_row_panel_grouped(it, st.count, pl.starts + st.cs_off, st.cols, st.bmax, s);
    }
    if (e == cudaSuccess) {
      TraceScope t(trace ? "batched_step_schur" : nullptr, 0, 0, s);
      e = launch_schur_update_grouped(it, st.count64, pl.starts + st.ts_off64, st.tiles64, 64, s);
      if (e == cudaSuccess)
        e = launch_schur_update_grouped(it + st.count64, st.count - st.count64, pl.starts + st.ts_off32,
                                        st.tiles32, 32, s);
    }
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
  if (pl->dev) {
    if (pl->pool_stream)
      cudaFreeAsync(pl->dev, pl->pool_stream);  // after the plan's work on that stream
    else
      cudaFree(pl->dev);
  }
  delete pl;
}

namespace {

// Synthetic batch for the tuner: matrices of the given orders (diagonally
// dominant, refilled before every timed run, since a run overwrites them).
struct TuneBatch {
  std::vector<int32_t> n;
  std::vector<double*> hA;
  std::vector<int64_t> lda;
  void* buf = nullptr;
  double* const* dA = nullptr;
  const int32_t* dn = nullptr;
  ~TuneBatch() {
    if (buf) cudaFree(buf);
  }
  int make(const std::vector<int32_t>& orders) {
    n = orders;
    size_t total = 0;
    std::vector<size_t> off(n.size());
    for (size_t m = 0; m < n.size(); ++m) {
      off[m] = total;
      total += align256(sizeof(double) * (size_t)n[m] * n[m]);
    }
    const size_t o_ptr = total, o_n = o_ptr + align256(sizeof(double*) * n.size());
    if (cudaMalloc(&buf, o_n + sizeof(int32_t) * n.size()) != cudaSuccess) {
      buf = nullptr;
      return BLOCKINV_ERR_NOMEM;
    }
    char* base = static_cast<char*>(buf);
    hA.resize(n.size());
    lda.assign(n.begin(), n.end());
    for (size_t m = 0; m < n.size(); ++m) hA[m] = reinterpret_cast<double*>(base + off[m]);
    cudaError_t e = cudaMemcpy(base + o_ptr, hA.data(), sizeof(double*) * n.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o_n, n.data(), sizeof(int32_t) * n.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_status(e);
    dA = reinterpret_cast<double* const*>(base + o_ptr);
    dn = reinterpret_cast<const int32_t*>(base + o_n);
    return BLOCKINV_OK;
  }
};

// Partition and tile of every matrix of the batch under a candidate table.
void table_partitions(const std::vector<int32_t>& ns, const Tuned* table, std::vector<int32_t>* p,
                      std::vector<int32_t>* sizes, std::vector<int>* tiles) {
  p->clear();
  sizes->clear();
  tiles->clear();
  std::vector<int> part;
  for (int32_t nn : ns) {
    const int c = size_class(nn);
    const Tuned t = (c >= kMinClass && c <= kMaxClass) ? table[c] : Tuned();
    if (t.p > 0 && t.p <= nn && (nn + t.p - 1) / t.p <= BLOCKINV_MAX_BLOCK)
      equal_partition(nn, t.p, &part);
    else
      batch_default_partition(nn, &part);
    p->push_back((int32_t)part.size());
    sizes->insert(sizes->end(), part.begin(), part.end());
    tiles->push_back(t.tile);
  }
}

// Best of `reps` graph replays (after one warm-up) of the whole batch under
// a candidate table.
int time_table(TuneBatch& tb, const Tuned* table, int reps, cudaStream_t s, float* best_ms) {
  std::vector<int32_t> p, sizes;
  std::vector<int> tiles;
  table_partitions(tb.n, table, &p, &sizes, &tiles);
  BatchPlan* pl = nullptr;
  const int st = batch_plan_create((int32_t)tb.n.size(), tb.n.data(), p.data(), sizes.data(), tb.hA.data(),
                                   tb.lda.data(), &pl, 0, tiles.data());
  if (st != BLOCKINV_OK) return st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t e = cudaSuccess;
  *best_ms = 1e30f;
  for (int r = -1; r < reps && e == cudaSuccess; ++r) {
    fill_tune_kernel<<<(unsigned)tb.n.size(), 256, 0, s>>>(tb.dA, tb.dn);
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = batch_run(*pl, s, nullptr, true);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess && r >= 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) *best_ms = std::min(*best_ms, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  batch_plan_destroy(pl);
  return cuda_status(e);
}

}  // namespace

// Coordinate descent over the size classes of this batch, largest total
// work first: each class's candidates are timed on the whole batch (classes
// share every grouped launch, so a class is only as good as the batch it
// runs in), with the other classes at their current choice.
int batch_tune(int32_t count, const int32_t* n, int reps, cudaStream_t s) {
  if (count < 1 || !n || reps < 1 || reps > 100) return BLOCKINV_ERR_INVALID;
  std::vector<int32_t> orders;
  const int stride = std::max(1, count / 4096);  // at most about 4096 matrices are timed
  for (int m = 0; m < count; ++m) {
    if (n[m] < 1 || n[m] > (1 << 16)) return BLOCKINV_ERR_INVALID;
    if (m % stride == 0) orders.push_back(n[m]);
  }
  std::map<int, double> work;  // class -> sum of n^3
  std::map<int, std::pair<int, int>> range;
  for (int32_t nn : orders) {
    const int c = size_class(nn);
    if (c < kMinClass || c > kMaxClass) continue;
    work[c] += (double)nn * nn * nn;
    auto it = range.find(c);
    if (it == range.end()) range[c] = {nn, nn};
    else it->second = {std::min(it->second.first, (int)nn), std::max(it->second.second, (int)nn)};
  }
  std::vector<int> classes;
  for (auto& kv : work) classes.push_back(kv.first);
  std::sort(classes.begin(), classes.end(), [&](int a, int b) { return work[a] > work[b]; });
  TuneBatch tb;
  int st = tb.make(orders);
  if (st != BLOCKINV_OK) return st;
  Tuned table[kMaxClass + 1];
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (int c = 0; c <= kMaxClass; ++c) table[c] = g_tune[c];
  }
  for (int c : classes) {
    const int nmin = range[c].first, nmax = range[c].second;
    Tuned best = table[c];
    float best_ms = 1e30f;
    st = time_table(tb, table, reps, s, &best_ms);  // the current choice
    if (st != BLOCKINV_OK) return st;
    for (int p : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32}) {
      if (p > nmin || (nmax + p - 1) / p > kGroupedMaxB || (p > 1 && nmin / p < 4)) continue;
      for (int tile : {64, 32}) {
        table[c].p = p;
        table[c].tile = tile;
        float ms = 0.f;
        st = time_table(tb, table, reps, s, &ms);
        if (st != BLOCKINV_OK) return st;
        if (ms < best_ms) {
          best_ms = ms;
          best = table[c];
        }
      }
    }
    table[c] = best;
  }
  std::lock_guard<std::mutex> g(g_tune_mu);
  for (int c : classes) g_tune[c] = table[c];
  return BLOCKINV_OK;
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
  return cuda_status(e);
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
  return cuda_status(e);
}

int blockinv_batch_tune(int32_t count, const int32_t* n, int32_t reps, void* stream) {
  return batch_tune(count, n, reps, static_cast<cudaStream_t>(stream));
}

int blockinv_batch_tuning(int32_t size_class, int32_t* nblocks, int32_t* tile) {
  if (size_class < kMinClass || size_class > kMaxClass || !nblocks || !tile) return BLOCKINV_ERR_INVALID;
  std::lock_guard<std::mutex> g(g_tune_mu);
  *nblocks = g_tune[size_class].p;
  *tile = g_tune[size_class].tile;
  return BLOCKINV_OK;
}

int blockinv_batch_tuning_set(int32_t size_class, int32_t nblocks, int32_t tile) {
  if (size_class < kMinClass || size_class > kMaxClass || nblocks < 0 || nblocks > (1 << 16) ||
      (tile != 32 && tile != 64))
    return BLOCKINV_ERR_INVALID;
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune[size_class].p = nblocks;
  g_tune[size_class].tile = tile;
  return BLOCKINV_OK;
}

int blockinv_batch_tuning_clear(void) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  for (Tuned& t : g_tune) t = Tuned();
  return BLOCKINV_OK;
}

int blockinv_batch_tuning_save(const char* path) {
  if (!path) return BLOCKINV_ERR_INVALID;
  FILE* f = std::fopen(path, "w");
  if (!f) return BLOCKINV_ERR_INVALID;
  std::fprintf(f, "blockinv-batch-tuning 1\n");
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (int c = kMinClass; c <= kMaxClass; ++c)
      if (g_tune[c].p > 0) std::fprintf(f, "%d %d %d\n", c, g_tune[c].p, g_tune[c].tile);
  }
  return std::fclose(f) == 0 ? BLOCKINV_OK : BLOCKINV_ERR_INVALID;
}

int blockinv_batch_tuning_load(const char* path) {
  if (!path) return BLOCKINV_ERR_INVALID;
  FILE* f = std::fopen(path, "r");
  if (!f) return BLOCKINV_ERR_INVALID;
  int version = 0, st = BLOCKINV_OK;
  Tuned table[kMaxClass + 1];
  if (std::fscanf(f, "blockinv-batch-tuning %d", &version) != 1 || version != 1) st = BLOCKINV_ERR_INVALID;
  int c, p, tile;
  while (st == BLOCKINV_OK) {
    const int got = std::fscanf(f, "%d %d %d", &c, &p, &tile);
    if (got == EOF) break;
    if (got != 3 || c < kMinClass || c > kMaxClass || p < 0 || p > (1 << 16) || (tile != 32 && tile != 64)) {
      st = BLOCKINV_ERR_INVALID;
      break;
    }
    table[c].p = p;
    table[c].tile = tile;
  }
  std::fclose(f);
  if (st != BLOCKINV_OK) return st;
  std::lock_guard<std::mutex> g(g_tune_mu);
  for (int k = 0; k <= kMaxClass; ++k) g_tune[k] = table[k];
  return BLOCKINV_OK;
}

}  // extern "C"
