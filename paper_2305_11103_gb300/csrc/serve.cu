// Serving loop: a context owns a worker thread and `max_slots` CUDA streams.
// Requests (one matrix each, any order, any mode) enter a queue; the worker
// admits them first-fit whenever a slot is free and the request's device
// footprint fits in what is left of the HBM budget, and enqueues the
// inversion on that slot's stream. Requests on different slots overlap on
// the GPU, and a request that arrives while others run starts as soon as a
// slot and memory free up (continuous batching: the set of requests on the
// device changes while it works). Each request's result does not depend on
// what runs beside it: the kernels of one request read and write only that
// request's matrix and workspace.
//
// Small requests (order <= kServeBatchMax) are coalesced: at each admission
// pass every queued small request that fits in the budget (up to
// kServeBatchCap of them) goes into one batch job on one slot, inverted by
// the grouped FP64 batched engine (one launch per kernel and elimination step
// for the whole batch, partitions and Schur tiles from the batch autotuner's
// table), whatever mode was asked: at these orders the FP64 path is both
// faster than the mixed pipeline and exact to FP64 rounding. The result
// record names the mode that produced it.
//
// Per request the context records the time in the queue, the device time
// (CUDA events on its slot stream; for a batch job, the batch's) and the
// end-to-end time, plus the refinement residual for the mixed modes.
// Finished requests also enter a completion queue (blockinv_poll_done), so a
// caller with many requests in flight need not poll each one.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <memory>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batched.h"
#include "internal.h"

using Clock = std::chrono::steady_clock;

namespace blockinv {
namespace {

constexpr int kServeBatchMax = 512;  // orders inverted by the batched FP64 engine
constexpr int kServeBatchCap = 512;  // requests per batch job

// A slot's launcher thread: the worker hands it an admitted request (or
// batch job) and it enqueues the kernels, so that enqueueing, which costs
// the host about 0.2-0.4 ms per large mixed request, runs on as many
// threads as there are slots.
struct Launcher {
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool pending = false;
  bool quit = false;
  std::atomic<bool> launched{false};  // the slot's work is enqueued (its ev1 recorded)
};

struct Request {
  uint64_t id = 0;
  Plan plan;
  double* A = nullptr;
  int64_t lda = 0;
  int mode = 0;
  int mode_used = 0;      // the mode that produced the result
  bool host = false;
  bool batchable = false;
  bool explicit_sizes = false;
  size_t footprint = 0;
  Clock::time_point t_submit, t_admit, t_done;
  int status = BLOCKINV_PENDING;
  double rho = -1.0;
  int iters = 0;
  float dev_ms = 0.f;
  bool done = false;
  bool fell_back = false;
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int32_t* status_dev = nullptr;   // 2 words
  int32_t* status_host = nullptr;  // pinned, 2 words
  double* dbuf = nullptr;          // device copy of a host request
  double* X = nullptr;             // the matrix the kernels work on
  int64_t ld = 0;
  ServeJob* job = nullptr;
  Request* req = nullptr;
  int enqueue_status = BLOCKINV_OK;
  float dev_ms = 0.f;              // device time of earlier passes (fallback)
  // a batch job (req is null then)
  std::vector<Request*> batch;
  std::vector<double*> bdbuf;      // device copies of its host requests (or null)
  BatchPlan* plan = nullptr;
  int32_t* bstatus_dev = nullptr;  // kServeBatchCap words
  int32_t* bstatus_host = nullptr; // pinned, kServeBatchCap words
  void* staging = nullptr;         // pinned descriptor staging of the batch plans
  size_t staging_cap = 0;
  std::shared_ptr<Launcher> lw;
  bool busy() const { return req != nullptr || !batch.empty(); }
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace
}  // namespace blockinv

struct blockinv_ctx {
  int device = 0;
  size_t budget = 0, used = 0;
  double tol = 1e-12;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<blockinv::Request*> queue;
  std::unordered_map<uint64_t, blockinv::Request*> reqs;
  uint64_t next_id = 1;
  std::vector<blockinv::Slot> slots;
  std::thread worker;
  bool stopping = false;
  size_t busy = 0;
  std::deque<uint64_t> done_ids;  // completion queue (blockinv_poll_done)
};

namespace blockinv {
namespace {

void launch_request(blockinv_ctx* c, Slot& sl) {
  Request* r = sl.req;
  const int n = r->plan.n;
  const size_t row = sizeof(double) * (size_t)n;
  cudaStream_t s = sl.s;
  cudaEventRecord(sl.ev0, s);
  double* X = r->A;
  int64_t ld = r->lda;
  cudaError_t e = cudaSuccess;
  sl.dbuf = nullptr;
  if (r->host) {
    cudaMemPool_t pool = nullptr;
    e = workspace_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&sl.dbuf), row * n, pool, s);
    if (e == cudaSuccess)
      e = copy_matrix(sl.dbuf, n, r->A, r->lda, n, cudaMemcpyHostToDevice, s);
    X = sl.dbuf;
    ld = n;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(sl.status_dev, 0, 2 * sizeof(int32_t), s);
  int st = cuda_status(e);
  if (st == BLOCKINV_OK)
    st = serve_enqueue(r->plan, X, ld, r->mode, sl.status_dev, s, c->tol, -1, &sl.job);
  sl.X = X;
  sl.ld = ld;
  sl.dev_ms = 0.f;
  if (st == BLOCKINV_OK && r->host)
    e = copy_matrix(r->A, r->lda, sl.dbuf, n, n, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(sl.status_host, sl.status_dev, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  cudaEventRecord(sl.ev1, s);
  sl.enqueue_status = st == BLOCKINV_OK ? cuda_status(e) : st;
}

// A mixed request whose refinement failed is rerun in FP64 on its slot, from
// the FP64 copy of its input. Returns true if the rerun was enqueued.
bool fall_back(Slot& sl) {
  Request* r = sl.req;
  cudaStream_t s = sl.s;
  const int n = r->plan.n;
  cudaEventRecord(sl.ev0, s);
  int st = serve_enqueue_fallback(sl.job, r->plan, sl.X, sl.ld, sl.status_dev, s);
  if (st != BLOCKINV_OK) return false;
  if (r->host)
    copy_matrix(r->A, r->lda, sl.dbuf, n, n, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(sl.status_host, sl.status_dev, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  cudaEventRecord(sl.ev1, s);
  r->fell_back = true;
  return true;
}

// Returns false if the request continues (an FP64 rerun was enqueued).
bool finalize_request(blockinv_ctx* c, Slot& sl) {
  Request* r = sl.req;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, sl.ev0, sl.ev1);
  ms += sl.dev_ms;
  int st = sl.enqueue_status != BLOCKINV_OK ? sl.enqueue_status : sl.status_host[0];
  double rho = -1.0;
  int iters = 0;
  if (sl.job) {
    serve_job_info(sl.job, sl.s, &rho, &iters);
    if (st == BLOCKINV_ERR_NOT_CONVERGED && !r->fell_back) {
      sl.dev_ms = ms;
      r->iters = iters;
      if (fall_back(sl)) return false;
    }
    serve_job_release(sl.job);
    sl.job = nullptr;
  }
  if (r->fell_back) {
    rho = -1.0;
    iters = r->iters;
  }
  if (sl.dbuf) cudaFreeAsync(sl.dbuf, sl.s);
  sl.dbuf = nullptr;
  std::lock_guard<std::mutex> g(c->mu);
  r->dev_ms = ms;
  r->status = st;
  r->rho = rho;
  r->iters = iters;
  r->mode_used = r->fell_back ? BLOCKINV_F64 : r->mode;
  r->t_done = Clock::now();
  r->done = true;
  c->used -= r->footprint;
  c->busy -= 1;
  c->done_ids.push_back(r->id);
  sl.req = nullptr;
  c->cv_done.notify_all();
  return true;
}

// A batch job: every request's matrix (a pooled device copy for host
// requests), one pooled batch plan with each request's partition (its own,
// or the batch tuner's choice for its size class), the grouped FP64 engine,
// the per-matrix status words back to pinned memory.
void launch_batch(Slot& sl) {
  cudaStream_t s = sl.s;
  const int count = (int)sl.batch.size();
  cudaEventRecord(sl.ev0, s);
  std::vector<int32_t> nn(count), pp(count), sizes;
  std::vector<double*> X(count);
  std::vector<int64_t> ld(count);
  sl.bdbuf.assign(count, nullptr);
  cudaMemPool_t pool = nullptr;
  cudaError_t e = workspace_pool(&pool);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    Request* r = sl.batch[i];
    const int n = r->plan.n;
    nn[i] = n;
    X[i] = r->A;
    ld[i] = r->lda;
    if (r->host) {
      e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&sl.bdbuf[i]), sizeof(double) * (size_t)n * n, pool, s);
      if (e == cudaSuccess) e = copy_matrix(sl.bdbuf[i], n, r->A, r->lda, n, cudaMemcpyHostToDevice, s);
      X[i] = sl.bdbuf[i];
      ld[i] = n;
    }
    std::vector<int> part;
    int tile = 0;
    if (r->explicit_sizes)
      part = r->plan.sizes;
    else
      batch_partition(n, &part, &tile);
    pp[i] = (int32_t)part.size();
    sizes.insert(sizes.end(), part.begin(), part.end());
  }
  int st = cuda_status(e);
  sl.plan = nullptr;
  if (st == BLOCKINV_OK) {
    size_t cap = sl.staging_cap;
    st = batch_plan_create(count, nn.data(), pp.data(), sizes.data(), X.data(), ld.data(), &sl.plan, 0, nullptr, s,
                           sl.staging, &cap);
    if (st == BLOCKINV_ERR_NOMEM && cap > sl.staging_cap) {  // grow the staging (the slot is idle)
      if (sl.staging) cudaFreeHost(sl.staging);
      sl.staging = nullptr;
      sl.staging_cap = 0;
      if (cudaMallocHost(&sl.staging, 2 * cap) == cudaSuccess) sl.staging_cap = 2 * cap;
      cap = sl.staging_cap;
      st = batch_plan_create(count, nn.data(), pp.data(), sizes.data(), X.data(), ld.data(), &sl.plan, 0, nullptr,
                             s, sl.staging, &cap);
    }
  }
  if (st == BLOCKINV_OK) st = cuda_status(batch_run(*sl.plan, s, sl.bstatus_dev, false));
  if (st == BLOCKINV_OK)
    cudaMemcpyAsync(sl.bstatus_host, sl.bstatus_dev, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s);
  for (int i = 0; i < count && st == BLOCKINV_OK; ++i) {
    Request* r = sl.batch[i];
    if (r->host) copy_matrix(r->A, r->lda, sl.bdbuf[i], r->plan.n, r->plan.n, cudaMemcpyDeviceToHost, s);
  }
  cudaEventRecord(sl.ev1, s);
  sl.enqueue_status = st;
}

void finalize_batch(blockinv_ctx* c, Slot& sl) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, sl.ev0, sl.ev1);
  if (sl.plan) batch_plan_destroy(sl.plan);  // its memory goes back to the pool in stream order
  sl.plan = nullptr;
  for (double* d : sl.bdbuf)
    if (d) cudaFreeAsync(d, sl.s);
  sl.bdbuf.clear();
  const auto now = Clock::now();
  std::lock_guard<std::mutex> g(c->mu);
  for (size_t i = 0; i < sl.batch.size(); ++i) {
    Request* r = sl.batch[i];
    r->status = sl.enqueue_status != BLOCKINV_OK ? sl.enqueue_status : sl.bstatus_host[i];
    r->dev_ms = ms;
    r->rho = -1.0;
    r->iters = 0;
    r->mode_used = BLOCKINV_F64;
    r->t_done = now;
    r->done = true;
    c->used -= r->footprint;
    c->busy -= 1;
    c->done_ids.push_back(r->id);
  }
  sl.batch.clear();
  c->cv_done.notify_all();
}

void launcher_loop(blockinv_ctx* c, Slot* sl) {
  cudaSetDevice(c->device);
  Launcher& lw = *sl->lw;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(lw.mu);
      lw.cv.wait(lk, [&] { return lw.pending || lw.quit; });
      if (lw.quit && !lw.pending) return;
      lw.pending = false;
    }
    if (sl->req)
      launch_request(c, *sl);
    else
      launch_batch(*sl);
    lw.launched.store(true, std::memory_order_release);
  }
}

void worker_loop(blockinv_ctx* c) {
  cudaSetDevice(c->device);
  std::vector<Slot*> admitted;
  for (;;) {
    bool progressed = false;
    for (Slot& sl : c->slots) {
      if (sl.busy() && sl.lw->launched.load(std::memory_order_acquire) && cudaEventQuery(sl.ev1) == cudaSuccess) {
        if (sl.req)
          finalize_request(c, sl);
        else
          finalize_batch(c, sl);
        if (!sl.busy()) sl.lw->launched.store(false, std::memory_order_relaxed);
        progressed = true;
      }
    }
    admitted.clear();
    {
      std::unique_lock<std::mutex> lk(c->mu);
      if (c->stopping && c->queue.empty() && c->busy == 0) break;
      bool batched = false;  // at most one new batch job per pass
      for (Slot& sl : c->slots) {
        if (sl.busy()) continue;
        const auto now = Clock::now();
        if (!batched) {
          // every queued small request that fits, oldest first, into one batch job
          for (auto it = c->queue.begin(); it != c->queue.end() && (int)sl.batch.size() < kServeBatchCap;) {
            Request* r = *it;
            if (r->batchable && r->footprint <= c->budget - c->used) {
              it = c->queue.erase(it);
              c->used += r->footprint;
              c->busy += 1;
              r->t_admit = now;
              sl.batch.push_back(r);
            } else {
              ++it;
            }
          }
          if (!sl.batch.empty()) {
            batched = true;
            admitted.push_back(&sl);
            continue;
          }
        }
        // first fit: the oldest queued request that fits in the remaining budget
        auto it = c->queue.begin();
        for (; it != c->queue.end(); ++it)
          if (!(*it)->batchable && (*it)->footprint <= c->budget - c->used) break;
        if (it == c->queue.end()) break;
        Request* r = *it;
        c->queue.erase(it);
        c->used += r->footprint;
        c->busy += 1;
        r->t_admit = now;
        sl.req = r;
        admitted.push_back(&sl);
      }
      if (admitted.empty() && !progressed) {
        c->cv_work.wait_for(lk, std::chrono::microseconds(50));
        continue;
      }
    }
    for (Slot* sl : admitted) {  // the slot's launcher enqueues the work
      std::lock_guard<std::mutex> g(sl->lw->mu);
      sl->lw->pending = true;
      sl->lw->cv.notify_one();
    }
  }
}

}  // namespace
}  // namespace blockinv

using namespace blockinv;

extern "C" {

int blockinv_ctx_create(int device, size_t hbm_budget_bytes, int max_slots, blockinv_ctx** out) {
  if (!out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) return BLOCKINV_ERR_INVALID;
  *out = nullptr;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return BLOCKINV_ERR_INVALID;
  auto c = new blockinv_ctx();
  c->device = device;
  c->budget = hbm_budget_bytes;
  c->slots.resize(max_slots);
  cudaError_t e = cudaSuccess;
  for (Slot& sl : c->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.ev1);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sl.status_dev), 2 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&sl.status_host), 2 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sl.bstatus_dev), kServeBatchCap * sizeof(int32_t));
    if (e == cudaSuccess)
      e = cudaMallocHost(reinterpret_cast<void**>(&sl.bstatus_host), kServeBatchCap * sizeof(int32_t));
    if (e == cudaSuccess && cudaMallocHost(&sl.staging, 1 << 20) == cudaSuccess) sl.staging_cap = 1 << 20;
  }
  if (e != cudaSuccess) {
    for (Slot& sl : c->slots) {
      if (sl.s) cudaStreamDestroy(sl.s);
      if (sl.ev0) cudaEventDestroy(sl.ev0);
      if (sl.ev1) cudaEventDestroy(sl.ev1);
      if (sl.status_dev) cudaFree(sl.status_dev);
      if (sl.status_host) cudaFreeHost(sl.status_host);
      if (sl.bstatus_dev) cudaFree(sl.bstatus_dev);
      if (sl.bstatus_host) cudaFreeHost(sl.bstatus_host);
      if (sl.staging) cudaFreeHost(sl.staging);
    }
    delete c;
    cudaSetDevice(prev);
    return BLOCKINV_ERR_CUDA;
  }
  for (Slot& sl : c->slots) {
    sl.lw = std::make_shared<Launcher>();
    sl.lw->th = std::thread(launcher_loop, c, &sl);
  }
  c->worker = std::thread(worker_loop, c);
  cudaSetDevice(prev);
  *out = c;
  return BLOCKINV_OK;
}

int blockinv_submit(blockinv_ctx* c, int64_t n, int32_t p, const int32_t* block_sizes, double* A, int64_t lda,
                    int mode, int flags, uint64_t* ticket) {
  if (!c || !ticket || !A || (flags & ~BLOCKINV_SUBMIT_HOST)) return BLOCKINV_ERR_INVALID;
  auto r = new Request();
  int st = serve_make_plan(n, p, block_sizes, lda, mode, &r->plan);
  if (st != BLOCKINV_OK) {
    delete r;
    return st;
  }
  r->A = A;
  r->lda = lda;
  r->mode = mode;
  r->mode_used = mode;
  r->host = (flags & BLOCKINV_SUBMIT_HOST) != 0;
  r->batchable = n <= kServeBatchMax;
  r->explicit_sizes = p > 0;
  r->footprint = serve_footprint(r->plan, r->batchable ? BLOCKINV_F64 : mode) +
                 (r->host ? sizeof(double) * (size_t)n * n : 0);
  if (r->footprint > c->budget) {
    delete r;
    return BLOCKINV_ERR_BUDGET;
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> g(c->mu);
    if (c->stopping) {
      delete r;
      return BLOCKINV_ERR_INVALID;
    }
    r->id = c->next_id++;
    c->reqs[r->id] = r;
    c->queue.push_back(r);
  }
  c->cv_work.notify_one();
  *ticket = r->id;
  return BLOCKINV_OK;
}

static int take_result(blockinv_ctx* c, std::unordered_map<uint64_t, Request*>::iterator it, blockinv_result* out) {
  Request* r = it->second;
  const int st = r->status;
  if (out) {
    out->status = st;
    out->mode = r->mode_used;
    out->n = r->plan.n;
    out->refine_iters = r->iters;
    out->used_fallback = r->fell_back ? 1 : 0;
    out->rho = r->rho;
    out->t_queue_ms = st == BLOCKINV_ERR_CANCELLED ? ms_between(r->t_submit, r->t_done)
                                                   : ms_between(r->t_submit, r->t_admit);
    out->t_device_ms = r->dev_ms;
    out->t_total_ms = ms_between(r->t_submit, r->t_done);
  }
  c->reqs.erase(it);
  delete r;
  return st;
}

int blockinv_poll(blockinv_ctx* c, uint64_t ticket, blockinv_result* out) {
  if (!c) return BLOCKINV_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  auto it = c->reqs.find(ticket);
  if (it == c->reqs.end()) return BLOCKINV_ERR_INVALID;
  if (!it->second->done) return BLOCKINV_PENDING;
  return take_result(c, it, out);
}

int blockinv_wait(blockinv_ctx* c, uint64_t ticket, blockinv_result* out) {
  if (!c) return BLOCKINV_ERR_INVALID;
  std::unique_lock<std::mutex> lk(c->mu);
  auto it = c->reqs.find(ticket);
  if (it == c->reqs.end()) return BLOCKINV_ERR_INVALID;
  Request* r = it->second;
  c->cv_done.wait(lk, [&] { return r->done; });
  return take_result(c, c->reqs.find(ticket), out);
}

int blockinv_cancel(blockinv_ctx* c, uint64_t ticket) {
  if (!c) return BLOCKINV_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  auto it = c->reqs.find(ticket);
  if (it == c->reqs.end()) return BLOCKINV_ERR_INVALID;
  Request* r = it->second;
  if (r->done) return BLOCKINV_OK;
  for (auto q = c->queue.begin(); q != c->queue.end(); ++q) {
    if (*q == r) {
      c->queue.erase(q);
      r->status = BLOCKINV_ERR_CANCELLED;
      r->t_done = Clock::now();
      r->done = true;
      c->done_ids.push_back(r->id);
      c->cv_done.notify_all();
      return BLOCKINV_OK;
    }
  }
  return BLOCKINV_PENDING;  // already on the GPU: runs to completion
}

int blockinv_poll_done(blockinv_ctx* c, uint64_t* tickets, int32_t max_tickets, int32_t* count) {
  if (!c || !count || max_tickets < 0 || (max_tickets > 0 && !tickets)) return BLOCKINV_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  int32_t k = 0;
  while (k < max_tickets && !c->done_ids.empty()) {
    tickets[k++] = c->done_ids.front();
    c->done_ids.pop_front();
  }
  *count = k;
  return BLOCKINV_OK;
}

int blockinv_ctx_stats(blockinv_ctx* c, int64_t* queued, int64_t* running, size_t* bytes_in_use) {
  if (!c) return BLOCKINV_ERR_INVALID;
  std::lock_guard<std::mutex> g(c->mu);
  if (queued) *queued = (int64_t)c->queue.size();
  if (running) *running = (int64_t)c->busy;
  if (bytes_in_use) *bytes_in_use = c->used;
  return BLOCKINV_OK;
}

int blockinv_ctx_destroy(blockinv_ctx* c) {
  if (!c) return BLOCKINV_ERR_INVALID;
  {
    std::lock_guard<std::mutex> g(c->mu);
    c->stopping = true;
    for (Request* r : c->queue) {
      r->status = BLOCKINV_ERR_CANCELLED;
      r->done = true;
    }
    c->queue.clear();
  }
  c->cv_work.notify_all();
  c->cv_done.notify_all();
  if (c->worker.joinable()) c->worker.join();
  for (Slot& sl : c->slots) {  // the worker has seen every launched slot finish
    {
      std::lock_guard<std::mutex> g(sl.lw->mu);
      sl.lw->quit = true;
      sl.lw->cv.notify_one();
    }
    if (sl.lw->th.joinable()) sl.lw->th.join();
  }
  for (Slot& sl : c->slots) {
    cudaStreamSynchronize(sl.s);
    cudaStreamDestroy(sl.s);
    cudaEventDestroy(sl.ev0);
    cudaEventDestroy(sl.ev1);
    cudaFree(sl.status_dev);
    cudaFreeHost(sl.status_host);
    cudaFree(sl.bstatus_dev);
    cudaFreeHost(sl.bstatus_host);
    if (sl.staging) cudaFreeHost(sl.staging);
  }
  for (auto& kv : c->reqs) delete kv.second;
  delete c;
  return BLOCKINV_OK;
}

}  // extern "C"
