// C ABI entry points of libblockinv.so (declared in include/blockinv.h):
// argument checks, the partition plan, stream-ordered workspace, and the
// per-step kernel sequence of the blockwise inversion (Eq. (a) applied once
// per diagonal block, in place).
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace blockinv {

namespace {

thread_local int g_last_status = BLOCKINV_OK;
thread_local int64_t g_last_block = -1;

int record(int status, int64_t block) {
  g_last_status = status;
  g_last_block = block;
  return status;
}

constexpr int kDefaultBlock = 256;

// ------------------------------------------------------------- tracing ----
// When enabled, every kernel launch of the library is bracketed by two CUDA
// events on its stream and tagged with its algorithmic flops and bytes (what
// the step must compute and move at minimum, not what the kernel happens to
// touch). blockinv_trace_summary() waits for the events and reports, per
// kernel, launches, total device time, flops and bytes.
struct TraceRec {
  const char* name;
  cudaEvent_t a, b;
  double flops, bytes;
};
std::mutex g_trace_mu;
bool g_trace_on = false;
std::vector<TraceRec> g_trace;


// Block order of the single-matrix path per mode and size class
// c = floor(log2 n) chosen by the autotuner (0 = not tuned: kDefaultBlock).
constexpr int kTuneClasses = 21;
std::mutex g_block_mu;
int g_block[3][kTuneClasses] = {};

int order_class(int n) {
  int c = 0;
  while (c + 1 < kTuneClasses && (2 << c) <= n) ++c;
  return c;  // 2^c <= n < 2^(c+1) below the last class
}

int chosen_block(int n, int mode) {
  if (mode < 0 || mode > 2) return kDefaultBlock;
  std::lock_guard<std::mutex> g(g_block_mu);
  const int b = g_block[mode][order_class(n)];
  return b > 0 ? b : kDefaultBlock;
}

// Default partition when the caller passes p == 0. Small orders follow the
// paper's rule (Table 2: N_k = 2^(int(log2 n) - 1) blocks of order 2..4, the
// remainder handed to the last blocks); larger ones use blocks of the order
// the autotuner chose for the mode and size class (256 if untuned), the last
// block taking the remainder.
void default_partition(int n, std::vector<int>* out, int mode = BLOCKINV_F64) {
  if (n <= 16) {
    paper_partition(n, out);
    return;
  }
  out->clear();
  const int b = std::min(n, chosen_block(n, mode));
  const int p = (n + b - 1) / b;
  out->assign(p, b);
  out->back() = n - b * (p - 1);
}

}  // namespace

// The paper's partition rule (Table 2, Eq. (blocking)): n <= 3 is one block;
// otherwise N_k = 2^(floor(log2 n) - 1) blocks of order 2, the remainder
// handed out one by one from the last block backwards (blocks of order 2..4).
void paper_partition(int n, std::vector<int>* out) {
  out->clear();
  if (n <= 3) {
    out->push_back(n);
    return;
  }
  int e = 0;
  while ((2 << e) <= n) ++e;  // e = floor(log2 n)
  const int nk = 1 << (e - 1);
  out->assign(nk, 2);
  int r = n - 2 * nk;
  int pos = nk - 1;
  while (r-- > 0) {
    (*out)[pos] += 1;
    pos = (pos == 0) ? nk - 1 : pos - 1;
  }
}

namespace {

// Mixed modes stop at the order up to which the refinement's digit products
// are exact (FP32 group sums below 2^24, int64 accumulator below 2^63).
bool valid_mode(int mode, int64_t n) {
  if (mode == BLOCKINV_F64) return true;
  return (mode == BLOCKINV_MIXED_TF32 || mode == BLOCKINV_MIXED_BF16) && n <= kMixedMaxOrder;
}

int make_plan(int64_t n, int32_t p, const int32_t* block_sizes, int64_t lda, Plan* plan,
              int mode = BLOCKINV_F64) {
  if (n < 1 || n > (int64_t)1 << 20 || lda < n || p < 0 || p > n) return BLOCKINV_ERR_INVALID;
  plan->n = (int)n;
  if (p == 0) {
    default_partition((int)n, &plan->sizes, mode);
  } else {
    if (!block_sizes) return BLOCKINV_ERR_INVALID;
    plan->sizes.assign(block_sizes, block_sizes + p);
  }
  int64_t sum = 0;
  plan->offs.clear();
  plan->bmax = 0;
  for (int b : plan->sizes) {
    if (b < 1 || b > BLOCKINV_MAX_BLOCK) return BLOCKINV_ERR_INVALID;
    plan->offs.push_back((int)sum);
    sum += b;
    if (b > plan->bmax) plan->bmax = b;
  }
  if (sum != n) return BLOCKINV_ERR_INVALID;
  PivotPlan pp;
  if (!plan_pivot(plan->bmax, 8, &pp)) return BLOCKINV_ERR_INVALID;
  return BLOCKINV_OK;
}

// Stream-ordered device allocation that is released when the scope ends
// (the release is itself stream-ordered, so it is safe with pending work).
struct AsyncBuf {
  void* ptr = nullptr;
  cudaStream_t s = nullptr;
  cudaError_t alloc(size_t bytes, cudaStream_t stream) {
    s = stream;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = workspace_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(&ptr, bytes ? bytes : 16, pool, stream);
  }
  ~AsyncBuf() {
    if (ptr) cudaFreeAsync(ptr, s);
  }
};

}  // namespace

// Workspace comes from a memory pool of the library's own per device, which
// keeps the memory it has handed out (release threshold: unlimited) so that
// repeated solves do not map their workspace again; blockinv_release_memory
// gives it back. The caller's default pool is left as it is.
cudaError_t workspace_pool(cudaMemPool_t* out) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return e;
    }
    pools[dev] = p;
  }
  *out = pools[dev];
  return cudaSuccess;
}

std::atomic<int> g_last_cuda_error{0};

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return BLOCKINV_OK;
  g_last_cuda_error.store(static_cast<int>(e), std::memory_order_relaxed);
  if (e == cudaErrorMemoryAllocation) return BLOCKINV_ERR_NOMEM;
  return BLOCKINV_ERR_CUDA;
}

namespace {

// Side stream per device for the look-ahead (highest priority, created once).
cudaStream_t side_stream() {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!streams[dev]) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&streams[dev], cudaStreamNonBlocking, hi) != cudaSuccess) streams[dev] = nullptr;
  }
  return streams[dev];
}

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Enqueue the FP64 elimination of the whole matrix on stream s.
//
// Large problems use a one-step look-ahead: the Schur update of step k is
// split into the elements of block row / column k + 1 (the next step's
// panels) and the rest; as soon as the first part is done, the next pivot
// inverse and row panel run on a high-priority side stream while the rest of
// step k's update runs on s. The U panel is double-buffered.
//
// Steps k0 .. k1 - 1 only (0 .. p - 1 for a whole inversion): the state
// between steps is A alone, so a range picks up where the previous one
// stopped, and splitting the steps over several calls gives the same bits.
int enqueue_f64(const Plan& pl, double* A, int64_t lda, int32_t* status, cudaStream_t s, int k0 = 0,
                int k1 = -1, bool lookahead = true) {
  const int n = pl.n;
  if (k1 < 0) k1 = (int)pl.sizes.size();
  const int p = k1;
  if (k0 >= k1) return BLOCKINV_OK;
  cudaStream_t t = (lookahead && n >= 2048 && k1 - k0 >= 3) ? side_stream() : nullptr;
  const bool ahead = t != nullptr;
  AsyncBuf pinv, ubuf;
  cudaError_t e = pinv.alloc(sizeof(double) * (size_t)pl.bmax * pl.bmax, s);
  if (e == cudaSuccess) e = ubuf.alloc(sizeof(double) * (size_t)n * pl.bmax * (ahead ? 2 : 1), s);
  if (e != cudaSuccess) return cuda_status(e);
  double* Pinv = static_cast<double*>(pinv.ptr);
  double* Ub[2] = {static_cast<double*>(ubuf.ptr),
                   static_cast<double*>(ubuf.ptr) + (ahead ? (size_t)n * pl.bmax : 0)};
  EventPair ev;
  if (ahead) {
    e = cudaEventCreateWithFlags(&ev.a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev.b, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
  }
  auto panels = [&](int k, cudaStream_t st) -> cudaError_t {
    const int o = pl.offs[k], b = pl.sizes[k];
    const double bd = b, nd = n, rest = (double)(n - b);
    cudaError_t r;
    {
      TraceScope tr("pivot_inverse_f64", 2.0 * bd * bd * bd, 16.0 * bd * bd, st);
      r = launch_pivot_inverse<double>(A + (int64_t)o * lda + o, lda, b, Pinv, b, status, k, st);
    }
    if (r == cudaSuccess) {
      TraceScope tr("row_panel_f64", 2.0 * bd * bd * rest, 8.0 * (2.0 * bd * nd + bd * bd + 2.0 * rest * bd), st);
      r = launch_row_panel_f64(A, lda, n, o, b, Pinv, Ub[k & 1], status, st);
    }
    return r;
  };
  e = panels(k0, s);
  for (int k = k0; k < p && e == cudaSuccess; ++k) {
    const int o = pl.offs[k], b = pl.sizes[k];
    const double bd = b, nd = n, rest = (double)(n - b);
    double* U = Ub[k & 1];
    if (n == b) break;
    if (!ahead || k + 1 == p) {
      TraceScope tr("schur_update_f64", 2.0 * bd * rest * nd, 8.0 * (2.0 * rest * nd + rest * bd + bd * nd), s);
      e = launch_schur_update_f64(A, lda, n, o, b, U, status, s);
      if (e == cudaSuccess && !ahead && k + 1 < p) e = panels(k + 1, s);
      continue;
    }
    const int o1 = pl.offs[k + 1], b1 = pl.sizes[k + 1];
    const double b1d = b1;
    const double next_elems = b1d * nd + (rest - b1d) * b1d;
    {
      TraceScope tr("schur_update_f64", 2.0 * bd * next_elems, 8.0 * (2.0 * next_elems), s);
      e = launch_schur_split_f64(A, lda, n, o, b, U, status, o1, b1, true, s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev.a, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(t, ev.a, 0);
    if (e == cudaSuccess) e = panels(k + 1, t);
    if (e == cudaSuccess) e = cudaEventRecord(ev.b, t);
    if (e == cudaSuccess) {
      const double rest_elems = rest * nd - next_elems;
      TraceScope tr("schur_update_f64", 2.0 * bd * rest_elems, 8.0 * (2.0 * rest_elems + rest * bd + bd * nd), s);
      e = launch_schur_split_f64(A, lda, n, o, b, U, status, o1, b1, false, s);
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev.b, 0);
  }
  return cuda_status(e);
}

struct Options {
  double tol = 1e-12;
  int max_refine = 5;
  bool fallback = true;
  int split = 2;  // operand slices of the mixed Schur update (1 or 2)
  int pivot_f64 = 0;  // 0: FP64 re-inversion of ill-conditioned pivot blocks; 1: of all; -1: none
  bool reverse = false;           // pivot blocks last to first (Eq. (d))
  bool singular_fallback = false;  // FP64: retry singular pivots with another order / merged blocks
  bool lookahead = true;           // one-step look-ahead on a side stream (n >= 2048, 3 or more blocks)
  bool fuse = false;               // mixed: two elimination steps per Schur sweep (option fuse = 1)
};

// Pivot blocks whose estimate ||P||_inf ||P^-1||_inf exceeds this are inverted
// again in FP64 arithmetic by the mixed path (the FP32 Gauss-Jordan's own
// error grows with that estimate times the FP32 unit roundoff).
constexpr float kPivotCondLimit = 1e5f;

float pivot_cond_limit(const Options& o) {
  return o.pivot_f64 > 0 ? -1.f : (o.pivot_f64 < 0 ? 0.f : kPivotCondLimit);
}

Options resolve(const blockinv_options* o) {
  Options r;
  if (o) {
    if (o->tol > 0) r.tol = o->tol;
    if (o->max_refine >= 0) r.max_refine = o->max_refine;
    r.fallback = o->fallback != 0;
    if (o->split == 1) r.split = 1;
    r.pivot_f64 = o->pivot_f64 > 0 ? 1 : (o->pivot_f64 < 0 ? -1 : 0);
    r.reverse = o->pivot_order == 1;
    r.singular_fallback = o->singular_fallback != 0;
    r.lookahead = o->lookahead >= 0;
    r.fuse = r.lookahead && o->fuse > 0;
  }
  return r;
}

// The same blocks taken last to first. Block Gauss-Jordan reaches A^-1 for
// any order in which every block is the pivot once; last to first applies
// Eq. (d) (D^-1 and S_D = A - B D^-1 C) at every step.
Plan reversed(const Plan& pl) {
  Plan r = pl;
  std::reverse(r.sizes.begin(), r.sizes.end());
  std::reverse(r.offs.begin(), r.offs.end());
  return r;
}

// The spatial partition of a plan (blocks in index order).
std::vector<int> spatial_sizes(const Plan& pl) {
  std::vector<std::pair<int, int>> v;
  for (size_t i = 0; i < pl.sizes.size(); ++i) v.emplace_back(pl.offs[i], pl.sizes[i]);
  std::sort(v.begin(), v.end());
  std::vector<int> out;
  for (auto& q : v) out.push_back(q.second);
  return out;
}

// Spatial block of pivot step k.
int spatial_block(const Plan& pl, int k) {
  int j = 0;
  for (size_t i = 0; i < pl.sizes.size(); ++i)
    if (pl.offs[i] < pl.offs[k]) ++j;
  return j;
}

// Enqueue the mixed-precision elimination of A (overwritten by the FP64 copy
// of the low-precision inverse).
int enqueue_mixed_elim(const Plan& pl, double* A, int64_t lda, bool bf16, int nsl, float cond_limit,
                       int32_t* piv_words, int32_t* status, cudaStream_t s, bool lookahead, bool fuse) {
  const int n = pl.n;
  const int64_t ld32 = (n + 31) / 32 * 32;
  const int kpad = mixed_kpad(pl.bmax);
  const size_t eb = bf16 ? 2 : 4;
  AsyncBuf x32, pinv, u, vt;
  cudaError_t e = x32.alloc(sizeof(float) * (size_t)n * ld32, s);
  if (e == cudaSuccess) e = pinv.alloc(sizeof(float) * (size_t)pl.bmax * pl.bmax, s);
  // two slice sets per operand row (the panels of two steps when they are fused)
  if (e == cudaSuccess) e = u.alloc(eb * (size_t)n * kpad * nsl * 2, s);
  if (e == cudaSuccess) e = vt.alloc(eb * (size_t)n * kpad * nsl * 2, s);
  if (e != cudaSuccess) return cuda_status(e);
  float* X32 = static_cast<float*>(x32.ptr);
  {
    TraceScope t("cast_f64_to_f32", 0, 12.0 * n * (double)n, s);
    e = launch_cast_f64_to_f32(A, lda, X32, ld32, n, s);
  }
  if (e == cudaSuccess)
    e = mixed_elimination(pl, bf16, nsl, X32, ld32, static_cast<float*>(pinv.ptr), u.ptr, vt.ptr, cond_limit,
                          piv_words, status, s, lookahead && n >= 2048, fuse);
  if (e == cudaSuccess) {
    TraceScope t("cast_f32_to_f64", 0, 12.0 * n * (double)n, s);
    e = launch_cast_f32_to_f64(X32, ld32, A, lda, n, s);
  }
  return cuda_status(e);
}

// Device records of a mixed-precision solve: the untouched input (for the
// residuals and the FP64 fallback), the refinement workspace, the rho history
// and the refinement control words. Released in stream order.
struct MixedState {
  AsyncBuf a0, ws, hist, ctl, piv;
  int max_refine = 0;
  double* A0() const { return static_cast<double*>(a0.ptr); }
};

int enqueue_mixed(const Plan& pl, double* A, int64_t lda, bool bf16, int32_t* status, cudaStream_t s,
                  const Options& opt, MixedState& ms, bool host_steps) {
  const int n = pl.n;
  ms.max_refine = opt.max_refine;
  const size_t row = sizeof(double) * (size_t)n;
  cudaError_t e = ms.a0.alloc(row * n, s);
  if (e == cudaSuccess) e = ms.hist.alloc(sizeof(double) * (opt.max_refine + 1), s);
  if (e == cudaSuccess) e = ms.ctl.alloc(kRefineCtlWords * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ms.ctl.ptr, 0, kRefineCtlWords * sizeof(int32_t), s);
  if (e == cudaSuccess) e = ms.piv.alloc(2 * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ms.piv.ptr, 0, 2 * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ms.hist.ptr, 0xFF, sizeof(double) * (opt.max_refine + 1), s);
  if (e == cudaSuccess)
    e = copy_matrix(ms.a0.ptr, n, A, lda, n, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_status(e);
  int st = enqueue_mixed_elim(pl, A, lda, bf16, opt.split, pivot_cond_limit(opt), static_cast<int32_t*>(ms.piv.ptr),
                              status, s, opt.lookahead, opt.fuse);
  if (st != BLOCKINV_OK || opt.max_refine == 0) return st;
  e = ms.ws.alloc(refine_workspace_bytes(n, kResidualSlices, opt.max_refine), s);
  if (e != cudaSuccess) return cuda_status(e);
  e = enqueue_refine(ms.A0(), n, A, lda, n, opt.tol, opt.max_refine, kResidualSlices, ms.ws.ptr,
                     static_cast<double*>(ms.hist.ptr), static_cast<int32_t*>(ms.ctl.ptr), status, nullptr, 0, s,
                     true, host_steps);
  return cuda_status(e);
}

int enqueue(const Plan& pl, double* A, int64_t lda, int mode, int32_t* status, cudaStream_t s,
            const Options& opt, MixedState* ms) {
  switch (mode) {
    case BLOCKINV_F64:
      return enqueue_f64(pl, A, lda, status, s, 0, -1, opt.lookahead);
    case BLOCKINV_MIXED_TF32:
    case BLOCKINV_MIXED_BF16: {
      MixedState local;
      return enqueue_mixed(pl, A, lda, mode == BLOCKINV_MIXED_BF16, status, s, opt, ms ? *ms : local,
                           ms != nullptr);
    }
    default:
      return BLOCKINV_ERR_INVALID;
  }
}

// After a blocking mixed solve: copy the refinement record into info.
void read_mixed_info(const MixedState& ms, cudaStream_t s, blockinv_info* info) {
  if (!info || !ms.hist.ptr) return;
  std::vector<double> hist(ms.max_refine + 1, -1.0);
  int32_t ctl[kRefineCtlWords] = {0, 0, 0, -1};
  int32_t piv[2] = {0, 0};
  cudaMemcpyAsync(hist.data(), ms.hist.ptr, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(ctl, ms.ctl.ptr, sizeof(ctl), cudaMemcpyDeviceToHost, s);
  if (ms.piv.ptr) cudaMemcpyAsync(piv, ms.piv.ptr, sizeof(piv), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return;
  info->refine_iters = ctl[1];
  info->incremental_residuals = ctl[5];
  info->incremental_groups = ctl[5] > 0 ? ctl[6] : 0;
  info->fp64_pivots = piv[1];
  if (ctl[3] >= 0) {
    info->rho_initial = hist[0];
    info->rho = hist[ctl[3]];
  }
}

// Wait for the stream and turn the device status word into a return code.
int finish(const int32_t* status_dev, cudaStream_t s) {
  int32_t host[2] = {0, -1};
  cudaError_t e = cudaMemcpyAsync(host, status_dev, sizeof(host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return record(cuda_status(e), -1);
  return record(host[0], host[0] == BLOCKINV_OK ? -1 : host[1]);
}

}  // namespace

// ------------------------------------------ step ranges and checkpoints --
int plan_for(int64_t n, int32_t p, const int32_t* block_sizes, int64_t lda, Plan* pl) {
  return make_plan(n, p, block_sizes, lda, pl);
}

int invert_steps(const Plan& pl, double* A, int64_t lda, int k0, int k1, cudaStream_t s) {
  AsyncBuf sbuf;
  cudaError_t e = sbuf.alloc(2 * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sbuf.ptr, 0, 2 * sizeof(int32_t), s);
  if (e != cudaSuccess) return record(cuda_status(e), -1);
  int32_t* status = static_cast<int32_t*>(sbuf.ptr);
  const int st = enqueue_f64(pl, A, lda, status, s, k0, k1);
  if (st != BLOCKINV_OK) {
    cudaStreamSynchronize(s);
    return record(st, -1);
  }
  return finish(status, s);
}

// ---------------------------------------------- hooks for the serving loop --
struct ServeJob {
  MixedState ms;
};

int serve_make_plan(int64_t n, int32_t p, const int32_t* block_sizes, int64_t lda, int mode, Plan* pl) {
  if (!valid_mode(mode, n)) return BLOCKINV_ERR_INVALID;
  return make_plan(n, p, block_sizes, lda, pl, mode);
}

size_t serve_footprint(const Plan& pl, int mode) {
  const size_t n = pl.n, b = pl.bmax;
  size_t f = 8 * (b * b + n * b) + 256;
  if (mode != BLOCKINV_F64) {
    const size_t kp = mixed_kpad(pl.bmax);
    f = 8 * n * n + 4 * n * ((n + 31) / 32 * 32) + 4 * b * b + 2 * 2 * 2 * 4 * n * kp +
        refine_workspace_bytes(pl.n, kResidualSlices, 5) + 4096;
  }
  return f;
}

int serve_enqueue(const Plan& pl, double* A, int64_t lda, int mode, int32_t* status, cudaStream_t s, double tol,
                  int max_refine, ServeJob** job) {
  *job = nullptr;
  if (mode == BLOCKINV_F64) return enqueue_f64(pl, A, lda, status, s);
  Options opt;
  if (tol > 0) opt.tol = tol;
  if (max_refine >= 0) opt.max_refine = max_refine;
  auto j = new ServeJob();
  const int st = enqueue_mixed(pl, A, lda, mode == BLOCKINV_MIXED_BF16, status, s, opt, j->ms, false);
  *job = j;
  return st;
}

void serve_job_info(ServeJob* job, cudaStream_t s, double* rho, int* iters) {
  *rho = -1.0;
  *iters = 0;
  if (!job || !job->ms.hist.ptr) return;
  blockinv_info info{};
  info.rho = -1;
  read_mixed_info(job->ms, s, &info);
  *rho = info.rho;
  *iters = info.refine_iters;
}

void serve_job_release(ServeJob* job) { delete job; }

// After a mixed request ended NOT_CONVERGED: restore the input from the
// job's FP64 copy and enqueue the FP64 path on the same stream.
int serve_enqueue_fallback(ServeJob* job, const Plan& pl, double* A, int64_t lda, int32_t* status,
                           cudaStream_t s) {
  if (!job || !job->ms.a0.ptr) return BLOCKINV_ERR_NOT_CONVERGED;
  cudaError_t e = copy_matrix(A, lda, job->ms.a0.ptr, pl.n, pl.n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 2 * sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_status(e);
  return enqueue_f64(pl, A, lda, status, s);
}

TraceScope::TraceScope(const char* name, double flops, double bytes, cudaStream_t s) : s_(s) {
  if (!name) return;  // a scope that records nothing
  std::lock_guard<std::mutex> g(g_trace_mu);
  if (!g_trace_on) return;
  if (cudaEventCreate(&a_) != cudaSuccess) return;
  if (cudaEventCreate(&b_) != cudaSuccess) {
    cudaEventDestroy(a_);
    return;
  }
  name_ = name;
  flops_ = flops;
  bytes_ = bytes;
  cudaEventRecord(a_, s_);
}

TraceScope::~TraceScope() {
  if (!name_) return;
  cudaEventRecord(b_, s_);
  std::lock_guard<std::mutex> g(g_trace_mu);
  g_trace.push_back(TraceRec{name_, a_, b_, flops_, bytes_});
}

}  // namespace blockinv

using namespace blockinv;

extern "C" {

int blockinv_invert_async(int64_t n, int32_t p, const int32_t* block_sizes, double* A,
                          int64_t lda, int mode, void* stream, int32_t* status_dev) {
  Plan pl;
  int st = make_plan(n, p, block_sizes, lda, &pl, mode);
  if (st != BLOCKINV_OK) return record(st, -1);
  if (!A || !status_dev || !valid_mode(mode, n)) return record(BLOCKINV_ERR_INVALID, -1);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(status_dev, 0, 2 * sizeof(int32_t), s);
  if (e != cudaSuccess) return record(cuda_status(e), -1);
  return record(enqueue(pl, A, lda, mode, status_dev, s, Options(), nullptr), -1);
}

int blockinv_invert_ex(int64_t n, int32_t p, const int32_t* block_sizes, double* A, int64_t lda, int mode,
                       void* stream, const blockinv_options* options, blockinv_info* info) {
  if (info) {
    memset(info, 0, sizeof(*info));
    info->failing_block = -1;
    info->rho = -1;
    info->rho_initial = -1;
  }
  Plan pl;
  int st = make_plan(n, p, block_sizes, lda, &pl, mode);
  if (st == BLOCKINV_OK && (!A || !valid_mode(mode, n))) st = BLOCKINV_ERR_INVALID;
  if (st != BLOCKINV_OK) {
    if (info) info->status = st;
    return record(st, -1);
  }
  const Options opt = resolve(options);
  if (opt.reverse) pl = reversed(pl);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  AsyncBuf sbuf, keep;
  cudaError_t e = sbuf.alloc(2 * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sbuf.ptr, 0, 2 * sizeof(int32_t), s);
  const size_t row = sizeof(double) * (size_t)n;
  const bool may_retry = mode == BLOCKINV_F64 && opt.singular_fallback;
  if (e == cudaSuccess && may_retry) {  // the input, for retries after a singular pivot block
    e = keep.alloc(row * (size_t)n, s);
    if (e == cudaSuccess)
      e = copy_matrix(keep.ptr, n, A, lda, n, cudaMemcpyDeviceToDevice, s);
  }
  if (e != cudaSuccess) return record(cuda_status(e), -1);
  int32_t* status = static_cast<int32_t*>(sbuf.ptr);
  MixedState ms;
  st = enqueue(pl, A, lda, mode, status, s, opt, &ms);
  if (st != BLOCKINV_OK) {
    cudaStreamSynchronize(s);
    if (info) info->status = st;
    return record(st, -1);
  }
  st = finish(status, s);
  int64_t fb = g_last_block;
  read_mixed_info(ms, s, info);
  if (st == BLOCKINV_ERR_NOT_CONVERGED && opt.fallback && ms.a0.ptr) {
    // The low-precision elimination or its refinement failed: redo in FP64.
    e = copy_matrix(A, lda, ms.a0.ptr, n, n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 2 * sizeof(int32_t), s);
    if (e != cudaSuccess) return record(cuda_status(e), -1);
    st = enqueue_f64(pl, A, lda, status, s, 0, -1, opt.lookahead);
    if (st == BLOCKINV_OK) st = finish(status, s);
    fb = g_last_block;
    if (info) info->used_fallback = 1;
  }
  // A singular pivot block: the other pivot order first, then the failing
  // block merged into a neighbour, again and again (each run from the input).
  Plan cur = pl;
  int kind = 0;
  auto rerun = [&](const Plan& q) -> int {
    cudaError_t e2 = copy_matrix(A, lda, keep.ptr, n, n, cudaMemcpyDeviceToDevice, s);
    if (e2 == cudaSuccess) e2 = cudaMemsetAsync(status, 0, 2 * sizeof(int32_t), s);
    if (e2 != cudaSuccess) return cuda_status(e2);
    int r = enqueue_f64(q, A, lda, status, s, 0, -1, opt.lookahead);
    if (r == BLOCKINV_OK) r = finish(status, s);
    return r;
  };
  if (st == BLOCKINV_ERR_SINGULAR && may_retry) {
    int failed_at = spatial_block(cur, (int)fb);
    const Plan alt = reversed(cur);
    const int r = rerun(alt);
    if (r == BLOCKINV_OK) {
      cur = alt;
      kind = 1;
      st = BLOCKINV_OK;
    } else if (r != BLOCKINV_ERR_SINGULAR) {
      st = r;
    }
    std::vector<int> part = spatial_sizes(pl);
    while (st == BLOCKINV_ERR_SINGULAR && part.size() > 1) {
      const int j = failed_at;
      const int a = (j + 1 < (int)part.size()) ? j : j - 1;  // merge blocks a and a + 1
      if (a < 0 || part[a] + part[a + 1] > BLOCKINV_MAX_BLOCK) break;
      part[a] += part[a + 1];
      part.erase(part.begin() + a + 1);
      Plan q;
      if (make_plan(n, (int32_t)part.size(), part.data(), lda, &q) != BLOCKINV_OK) break;
      const int r2 = rerun(q);
      cur = q;
      kind = 2;
      if (r2 == BLOCKINV_ERR_SINGULAR) {
        failed_at = spatial_block(cur, (int)g_last_block);
        continue;
      }
      st = r2;
    }
    if (st == BLOCKINV_ERR_SINGULAR) fb = g_last_block;
  }
  const int64_t failing = (st == BLOCKINV_ERR_SINGULAR || st == BLOCKINV_ERR_NONFINITE) && fb >= 0
                              ? spatial_block(cur, (int)fb)
                              : -1;
  if (info) {
    info->status = st;
    info->failing_block = failing;
    info->partition_fallback = kind;
    info->blocks_used = (int32_t)cur.sizes.size();
  }
  return record(st, failing);
}

int blockinv_invert(int64_t n, int32_t p, const int32_t* block_sizes, double* A, int64_t lda, int mode,
                    void* stream) {
  return blockinv_invert_ex(n, p, block_sizes, A, lda, mode, stream, nullptr, nullptr);
}

int blockinv_invert_host(int64_t n, int32_t p, const int32_t* block_sizes, double* A_host,
                         int64_t lda, int mode, void* stream) {
  Plan pl;
  int st = make_plan(n, p, block_sizes, lda, &pl, mode);
  if (st != BLOCKINV_OK) return record(st, -1);
  if (!A_host || !valid_mode(mode, n)) return record(BLOCKINV_ERR_INVALID, -1);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  AsyncBuf dbuf, sbuf;
  const size_t row = sizeof(double) * (size_t)n;
  cudaError_t e = dbuf.alloc(row * (size_t)n, s);
  if (e == cudaSuccess) e = sbuf.alloc(2 * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sbuf.ptr, 0, 2 * sizeof(int32_t), s);
  if (e == cudaSuccess)
    e = copy_matrix(dbuf.ptr, n, A_host, lda, n, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return record(cuda_status(e), -1);
  int32_t* status = static_cast<int32_t*>(sbuf.ptr);
  st = enqueue(pl, static_cast<double*>(dbuf.ptr), (int64_t)n, mode, status, s, Options(), nullptr);
  if (st != BLOCKINV_OK) {
    cudaStreamSynchronize(s);
    return record(st, -1);
  }
  e = copy_matrix(A_host, lda, dbuf.ptr, n, n, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return record(cuda_status(e), -1);
  return finish(status, s);
}

// ------------------------------------ block-size autotuner (one matrix) --
// For every size class c = floor(log2 n) among the given orders above 16:
// the class's median order m, a synthetic diagonally dominant matrix of that
// order (filled on the device), and each candidate block order b <= m
// (blocks of b, the last one the remainder) timed over `reps` inversions in
// `mode` after one warm-up; the fastest goes into the table that the default
// partition (p == 0) reads.
int blockinv_tune(int32_t count, const int32_t* n, int32_t mode, int32_t reps, void* stream) {
  if (count < 1 || !n || reps < 1 || reps > 100 || mode < 0 || mode > 2) return record(BLOCKINV_ERR_INVALID, -1);
  std::map<int, std::vector<int>> classes;
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1 || n[i] > (1 << 20) || !valid_mode(mode, n[i])) return record(BLOCKINV_ERR_INVALID, -1);
    if (n[i] > 16) classes[order_class(n[i])].push_back(n[i]);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  static const int kCand[] = {64, 128, 192, 256, 320, 384, 512};
  EventPair ev;
  cudaError_t e = cudaEventCreate(&ev.a);
  if (e == cudaSuccess) e = cudaEventCreate(&ev.b);
  if (e != cudaSuccess) return record(cuda_status(e), -1);
  for (auto& kv : classes) {
    std::vector<int>& v = kv.second;
    std::sort(v.begin(), v.end());
    const int m = v[v.size() / 2];
    AsyncBuf src, work, sbuf;
    e = src.alloc(sizeof(double) * (size_t)m * m, s);
    if (e == cudaSuccess) e = work.alloc(sizeof(double) * (size_t)m * m, s);
    if (e == cudaSuccess) e = sbuf.alloc(2 * sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_fill_diag_dominant(static_cast<double*>(src.ptr), m, 0x5eedull + m, s);
    if (e != cudaSuccess) return record(cuda_status(e), -1);
    int32_t* status = static_cast<int32_t*>(sbuf.ptr);
    int best = 0;
    float best_ms = 0.f;
    for (int b : kCand) {
      if (b > m) break;
      std::vector<int> part((m + b - 1) / b, b);
      part.back() = m - b * ((int)part.size() - 1);
      Plan pl;
      if (make_plan(m, (int32_t)part.size(), part.data(), m, &pl) != BLOCKINV_OK) continue;
      float tot = 0.f;
      bool ok = true;
      for (int r = 0; r <= reps && ok; ++r) {
        e = cudaMemcpyAsync(work.ptr, src.ptr, sizeof(double) * (size_t)m * m, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 2 * sizeof(int32_t), s);
        if (e == cudaSuccess) e = cudaEventRecord(ev.a, s);
        int st = e == cudaSuccess ? enqueue(pl, static_cast<double*>(work.ptr), m, mode, status, s, Options(), nullptr)
                                  : BLOCKINV_ERR_CUDA;
        if (st == BLOCKINV_OK) e = cudaEventRecord(ev.b, s);
        int32_t h[2] = {BLOCKINV_ERR_CUDA, 0};
        if (st == BLOCKINV_OK && e == cudaSuccess)
          e = cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        float ms = 0.f;
        if (st != BLOCKINV_OK || e != cudaSuccess || h[0] != BLOCKINV_OK ||
            cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess) {
          ok = false;
          break;
        }
        if (r > 0) tot += ms;
      }
      if (e != cudaSuccess) return record(cuda_status(e), -1);
      if (ok && (best == 0 || tot < best_ms)) {
        best = b;
        best_ms = tot;
      }
    }
    if (best > 0) {
      std::lock_guard<std::mutex> g(g_block_mu);
      g_block[mode][kv.first] = best;
    }
  }
  return record(BLOCKINV_OK, -1);
}

int blockinv_tuning(int32_t mode, int32_t size_class, int32_t* block) {
  if (mode < 0 || mode > 2 || size_class < 0 || size_class >= kTuneClasses || !block) return BLOCKINV_ERR_INVALID;
  std::lock_guard<std::mutex> g(g_block_mu);
  *block = g_block[mode][size_class];
  return BLOCKINV_OK;
}

int blockinv_tuning_set(int32_t mode, int32_t size_class, int32_t block) {
  if (mode < 0 || mode > 2 || size_class < 0 || size_class >= kTuneClasses || block < 0 ||
      block > BLOCKINV_MAX_BLOCK)
    return BLOCKINV_ERR_INVALID;
  std::lock_guard<std::mutex> g(g_block_mu);
  g_block[mode][size_class] = block;
  return BLOCKINV_OK;
}

int blockinv_tuning_clear(void) {
  std::lock_guard<std::mutex> g(g_block_mu);
  for (auto& row : g_block)
    for (int& b : row) b = 0;
  return BLOCKINV_OK;
}

int blockinv_residual(int64_t n, const double* A, int64_t lda, const double* X, int64_t ldx,
                      double* rho_out, void* stream) {
  if (n < 1 || n > (int64_t)1 << 20 || lda < n || ldx < n || !A || !X || !rho_out)
    return record(BLOCKINV_ERR_INVALID, -1);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  AsyncBuf sums;
  cudaError_t e = sums.alloc(3 * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sums.ptr, 0, 3 * sizeof(double), s);
  if (e == cudaSuccess) e = launch_residual_f64((int)n, A, lda, X, ldx, static_cast<double*>(sums.ptr), s);
  double h[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, sums.ptr, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return record(cuda_status(e), -1);
  *rho_out = std::sqrt(h[0]) / (std::sqrt(h[1]) * std::sqrt(h[2]));
  return record(BLOCKINV_OK, -1);
}

int blockinv_residual_tc(int64_t n, const double* A, int64_t lda, const double* X, int64_t ldx, double* E,
                         int64_t lde, int slices, double* rho_out, void* stream) {
  if (slices == 0) slices = kResidualSlices;
  if (n < 1 || n > kMixedMaxOrder || lda < n || ldx < n || !A || !X || !rho_out || (E && lde < n) ||
      slices < kMinResidualSlices || slices > kMaxResidualSlices)
    return record(BLOCKINV_ERR_INVALID, -1);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  AsyncBuf ws, hist, ctl, sbuf;
  cudaError_t e = ws.alloc(refine_workspace_bytes((int)n, slices, 0), s);
  if (e == cudaSuccess) e = hist.alloc(sizeof(double), s);
  if (e == cudaSuccess) e = ctl.alloc(kRefineCtlWords * sizeof(int32_t), s);
  if (e == cudaSuccess) e = sbuf.alloc(2 * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sbuf.ptr, 0, 2 * sizeof(int32_t), s);
  if (e == cudaSuccess)
    e = enqueue_refine(A, lda, const_cast<double*>(X), ldx, (int)n, 0.0, 0, slices, ws.ptr,
                       static_cast<double*>(hist.ptr), static_cast<int32_t*>(ctl.ptr),
                       static_cast<int32_t*>(sbuf.ptr), E, lde, s, false, false);
  double rho = -1.0;
  int32_t st[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&rho, hist.ptr, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(st, sbuf.ptr, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return record(cuda_status(e), -1);
  *rho_out = rho;
  return record(st[0], -1);
}

int blockinv_invert_batched_small(int64_t count, int32_t n, double* A, int32_t* status_dev, void* stream) {
  if (count < 0 || n < 1 || n > 8 || (count > 0 && !A) || count > ((int64_t)1 << 31) * 64)
    return record(BLOCKINV_ERR_INVALID, -1);
  if (count == 0) return record(BLOCKINV_OK, -1);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  {
    const double nd = n;
    TraceScope t("small_batched_f64", 2.0 * nd * nd * nd * (double)count, 16.0 * nd * nd * (double)count, s);
    e = launch_small_batched(n, A, count, status_dev, s);
  }
  return record(cuda_status(e), -1);
}

int blockinv_invert_batched_fixed(int64_t count, int32_t n, int32_t p, const int32_t* block_sizes, int32_t flags,
                                  double* A, int32_t* status_dev, void* stream) {
  if (count < 0 || n < 1 || n > 32 || (count > 0 && !A) || (flags & ~BLOCKINV_BATCH_SPD) ||
      count >= (int64_t)INT32_MAX * 4)
    return record(BLOCKINV_ERR_INVALID, -1);
  std::vector<int> part;
  if (block_sizes) {
    if (p < 1 || p > n) return record(BLOCKINV_ERR_INVALID, -1);
    int sum = 0;
    for (int i = 0; i < p; ++i) {
      if (block_sizes[i] < 1) return record(BLOCKINV_ERR_INVALID, -1);
      sum += block_sizes[i];
      part.push_back(block_sizes[i]);
    }
    if (sum != n) return record(BLOCKINV_ERR_INVALID, -1);
  } else {
    paper_partition(n, &part);
  }
  if (count == 0) return record(BLOCKINV_OK, -1);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  {
    const double nd = n;
    TraceScope t("tiny_batched_f64", 2.0 * nd * nd * nd * (double)count, 16.0 * nd * nd * (double)count, s);
    e = launch_tiny_batched(n, part, (flags & BLOCKINV_BATCH_SPD) != 0, A, count, status_dev, s);
  }
  return record(cuda_status(e), -1);
}

const char* blockinv_status_str(int status) {
  switch (status) {
    case BLOCKINV_OK: return "ok";
    case BLOCKINV_PENDING: return "pending";
    case BLOCKINV_ERR_INVALID: return "invalid argument";
    case BLOCKINV_ERR_SINGULAR: return "singular pivot block";
    case BLOCKINV_ERR_NONFINITE: return "non-finite pivot block";
    case BLOCKINV_ERR_NOMEM: return "out of device memory";
    case BLOCKINV_ERR_BUDGET: return "request exceeds the memory budget";
    case BLOCKINV_ERR_NOT_CONVERGED: return "refinement did not converge";
    case BLOCKINV_ERR_TIMEOUT: return "device wait timed out";
    case BLOCKINV_ERR_CUDA: return "CUDA error";
    case BLOCKINV_ERR_CANCELLED: return "cancelled";
    default: return "unknown status";
  }
}

int blockinv_last_error_detail(int64_t* failing_block) {
  if (failing_block) *failing_block = g_last_block;
  return g_last_status;
}

int blockinv_last_cuda_error(const char** name) {
  const int e = blockinv::g_last_cuda_error.exchange(0, std::memory_order_relaxed);
  if (name) *name = e ? cudaGetErrorName(static_cast<cudaError_t>(e)) : "cudaSuccess";
  return e;
}

int blockinv_version(void) { return 100; }

int blockinv_struct_sizes(int32_t* options_bytes, int32_t* info_bytes, int32_t* result_bytes) {
  if (options_bytes) *options_bytes = (int32_t)sizeof(blockinv_options);
  if (info_bytes) *info_bytes = (int32_t)sizeof(blockinv_info);
  if (result_bytes) *result_bytes = (int32_t)sizeof(blockinv_result);
  return BLOCKINV_OK;
}

int blockinv_release_memory(void) {
  cudaMemPool_t pool = nullptr;
  cudaError_t e = workspace_pool(&pool);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
  return cuda_status(e);
}

int blockinv_trace_enable(int on) {
  std::vector<TraceRec> old;
  {
    std::lock_guard<std::mutex> g(g_trace_mu);
    g_trace_on = (on != 0);
    if (on) old.swap(g_trace);
  }
  for (auto& r : old) {
    cudaEventSynchronize(r.b);
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  return BLOCKINV_OK;
}

int64_t blockinv_trace_summary(char* buf, int64_t buflen) {
  std::vector<TraceRec> recs;
  {
    std::lock_guard<std::mutex> g(g_trace_mu);
    recs.swap(g_trace);
  }
  struct Agg {
    int64_t launches = 0;
    double ms = 0, flops = 0, bytes = 0;
  };
  std::map<std::string, Agg> agg;
  for (auto& r : recs) {
    float ms = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms, r.a, r.b);
    Agg& a = agg[r.name];
    a.launches += 1;
    a.ms += ms;
    a.flops += r.flops;
    a.bytes += r.bytes;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  std::string out = "{";
  bool first = true;
  for (auto& kv : agg) {
    char line[256];
    snprintf(line, sizeof(line), "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"flops\": %.6e, \"bytes\": %.6e}",
             first ? "" : ", ", kv.first.c_str(), (long long)kv.second.launches, kv.second.ms,
             kv.second.flops, kv.second.bytes);
    out += line;
    first = false;
  }
  out += "}";
  if (buf && buflen > 0) {
    size_t m = std::min((size_t)buflen - 1, out.size());
    memcpy(buf, out.data(), m);
    buf[m] = 0;
  }
  return (int64_t)out.size() + 1;
}

}  // extern "C"
