/*
 * blockinv.h - C ABI of libblockinv.so, GB300 (sm_103a) blockwise matrix inversion.
 *
 * The library inverts a square matrix partitioned into a p x p grid of square
 * diagonal blocks (orders m_0..m_{p-1}, sum n) by repeated Schur-complement
 * elimination: Eq. (a) of R. Thiru Senthil, "Blockwise inversion and
 * algorithms for inverting large partitioned matrices" (arXiv 2305.11103),
 * applied once per diagonal block, in place, as the paper's
 * `invertor_inplace_by_a` procedure (Sec. 4.2) generalised from 2 x 2 to
 * p x p blocks. At elimination step k, with P the current diagonal block k:
 *
 *   1. P^-1                                   (pivot-block inverse, the paper's diamond op)
 *   2. V_j = P^-1 X[k, j] for every j != k    (row panel, the paper's right-arrow op)
 *   3. X[i, j] -= X[i, k] V_j  for i, j != k  (Schur complement S_A = D - C A^-1 B)
 *   4. X[i, k] = -X[i, k] P^-1, X[k, j] = V_j, X[k, k] = P^-1   (in-place assembly)
 *
 * After the last step X holds A^-1. The method needs every pivot block (the
 * leading diagonal block and each successive Schur complement) to be
 * invertible (Sec. 3, the condition stated with Eq. (a)); there is no
 * pivoting across blocks. Inside a pivot block, Gauss-Jordan elimination
 * with partial (row) pivoting is used.
 *
 * Conventions for every entry point:
 *  - Matrices are FP64, row-major, with a leading dimension (elements) >= n.
 *    A column-major caller gets A^-1 in column-major too, since
 *    (A^T)^-1 = (A^-1)^T and the partition is symmetric.
 *  - Device pointers are CUDA device memory of the current device (for
 *    example allocated by PyTorch). The caller owns every buffer it passes;
 *    the library never frees them. Workspace comes from a memory pool of the
 *    library's own per device (cudaMallocFromPoolAsync on the caller's
 *    stream, freed in stream order before the call returns). The pool keeps
 *    the memory it has handed out, so repeated solves do not map it again;
 *    blockinv_release_memory() returns the unused part to the driver. The
 *    caller's default memory pool is not touched.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *  - Argument errors are reported synchronously and leave the matrix
 *    untouched. Numerical errors (a singular or non-finite pivot block) are
 *    reported by the blocking entry points after a stream synchronisation; the
 *    matrix contents are then unspecified (partly eliminated).
 *  - blockinv_last_error_detail() gives the failing block index of the last
 *    SINGULAR / NONFINITE status returned on the calling host thread.
 */
#ifndef BLOCKINV_H
#define BLOCKINV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Arithmetic mode.
 *  BLOCKINV_F64        every step in FP64 on the GPU.
 *  BLOCKINV_MIXED_TF32 elimination on an FP32 copy with the Schur-update
 *                      products on TF32 tensor cores (FP32 accumulation),
 *                      then Newton-Schulz refinement X <- X + X (I - A X) with
 *                      an FP64-accurate residual until rho <= tol.
 *  BLOCKINV_MIXED_BF16 the same with BF16 tensor-core products.
 * Mixed modes accept n <= 16384 (the refinement residual's digit products are
 * exact up to that order); larger n returns BLOCKINV_ERR_INVALID. */
typedef enum {
  BLOCKINV_F64 = 0,
  BLOCKINV_MIXED_TF32 = 1,
  BLOCKINV_MIXED_BF16 = 2
} blockinv_mode;

/* Status codes. */
enum {
  BLOCKINV_OK = 0,
  BLOCKINV_PENDING = 1,              /* blockinv_poll: request not finished          */
  BLOCKINV_ERR_INVALID = -1,         /* bad argument (n, lda, partition, pointer)    */
  BLOCKINV_ERR_SINGULAR = -2,        /* a pivot block has an exact zero pivot        */
  BLOCKINV_ERR_NONFINITE = -3,       /* a pivot block holds NaN or Inf               */
  BLOCKINV_ERR_NOMEM = -4,           /* device workspace allocation failed           */
  BLOCKINV_ERR_BUDGET = -5,          /* serving: request larger than the HBM budget  */
  BLOCKINV_ERR_NOT_CONVERGED = -6,   /* refinement did not reach the tolerance       */
  BLOCKINV_ERR_TIMEOUT = -7,         /* a bounded device wait gave up                */
  BLOCKINV_ERR_CUDA = -8,            /* a CUDA runtime call failed                   */
  BLOCKINV_ERR_CANCELLED = -9        /* serving: request cancelled before it ran     */
};

/* Largest diagonal block order the GPU pivot-block kernel accepts. */
#define BLOCKINV_MAX_BLOCK 512

/* Invert the n x n FP64 matrix A in place (blocking).
 *  n            order, 1 <= n.
 *  p            number of diagonal blocks, 1 <= p <= n; 0 means "choose":
 *               blocks of order 256 (the last one takes the remainder), or the
 *               paper's rule of Table 2 (orders 2..4, N_k = 2^(int(log2 n)-1)
 *               blocks) when n <= 16.
 *  block_sizes  host array of p positive orders summing to n (Eq. (blocking),
 *               Sec. 5.1: the only restriction is that the orders sum to n);
 *               ignored when p == 0. Each order <= BLOCKINV_MAX_BLOCK.
 *  A            device pointer; overwritten by A^-1.
 *  lda          leading dimension of A in elements, >= n.
 *  mode         a blockinv_mode.
 *  stream       cudaStream_t or NULL.
 * Returns BLOCKINV_OK or an error status. Synchronises `stream`. */
int blockinv_invert(int64_t n, int32_t p, const int32_t* block_sizes, double* A,
                    int64_t lda, int mode, void* stream);

/* Stream-ordered form of blockinv_invert: enqueues the work and returns
 * without synchronising. Argument errors are returned at once. The numerical
 * status (a BLOCKINV_* code) and the failing block index are written to
 * status_dev[0] and status_dev[1] (device memory, two int32) when the work
 * completes. */
int blockinv_invert_async(int64_t n, int32_t p, const int32_t* block_sizes, double* A,
                          int64_t lda, int mode, void* stream, int32_t* status_dev);

/* Host-buffer form: A_host (host memory, pinned or pageable) is copied to the
 * device, inverted, and copied back into A_host. Blocking. */
int blockinv_invert_host(int64_t n, int32_t p, const int32_t* block_sizes, double* A_host,
                         int64_t lda, int mode, void* stream);

/* FP64 in-place inversion that allocates no device memory (the paper has no
 * counterpart: this is a deployment variant of blockinv_invert, mode
 * BLOCKINV_F64). For callers that cannot call cudaMalloc or any other
 * allocator - for example code that runs inside a memory-pool callback, or a
 * plugin whose host application owns every allocation. The scratch the
 * kernels need lives in a fixed file-scope device array (about 4.5 MiB on
 * every GPU that loads the library, kept until the process exits).
 *  n, p, block_sizes, A, lda as for blockinv_invert, with n <= 2048, every
 *               block order <= 256, and an explicit partition (p >= 1);
 *               larger sizes return BLOCKINV_ERR_INVALID with A untouched.
 *  stream       cudaStream_t or NULL; the call synchronises it.
 *  failing_block (host, may be NULL) receives the failing block index for
 *               SINGULAR / NONFINITE, else -1.
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the one scratch array: calls whose GPU work overlaps on
 * the same device (other streams or host threads) race and must be
 * serialised by the caller. */
int blockinv_invert_noalloc(int64_t n, int32_t p, const int32_t* block_sizes, double* A, int64_t lda,
                            void* stream, int64_t* failing_block);

/* Batched inversion of `count` small FP64 matrices of one order n (1..8), in
 * place: the paper's repeated small inversions (Sec. 2, systematics matrices
 * of order 5), each matrix partitioned by the paper's rule (Sec. 5.1, Table 2:
 * 5 -> [2, 3], 8 -> [2, 2, 2, 2]) and inverted by Eq. (a) block by block with
 * closed-form pivot-block inverses (the "algebraic expressions" for orders
 * 2..4). A: device, count matrices of n * n doubles each, row-major,
 * contiguous (matrix m starts at A + m * n * n). status_dev: device int32
 * per matrix (may be NULL): 0, BLOCKINV_ERR_SINGULAR (a pivot block with a
 * zero determinant) or BLOCKINV_ERR_NONFINITE; a failed matrix is left
 * unchanged. Stream-ordered: returns after enqueueing; argument errors are
 * returned at once. */
int blockinv_invert_batched_small(int64_t count, int32_t n, double* A, int32_t* status_dev, void* stream);

/* Batched inversion of `count` matrices of one order n <= 32 with one
 * partition: the paper's tau-neutrino workload (Sec. 2: 11 x 11 matrices
 * split into blocks of 5 and 6) and its relatives. block_sizes (host, p
 * entries summing to n) or NULL for the paper's Table 2 rule. Eq. (a) block
 * by block: each pivot block's Gauss-Jordan with partial pivoting inside the
 * block, its row operations applied to whole rows (forming the row panel,
 * the Schur complement and the column panel). A: device, count contiguous
 * row-major n x n matrices. flags: BLOCKINV_BATCH_SPD for symmetric positive
 * definite inputs (diagonal pivots without a search; the result is made
 * exactly symmetric from its upper triangle). status_dev: device int32 per
 * matrix (may be NULL): 0, SINGULAR or NONFINITE; a failed matrix is left
 * unchanged. One matrix per 16 lanes (n <= 16) or per warp. Stream-ordered;
 * argument errors are returned at once. */
#define BLOCKINV_BATCH_SPD 1
int blockinv_invert_batched_fixed(int64_t count, int32_t n, int32_t p, const int32_t* block_sizes, int32_t flags,
                                  double* A, int32_t* status_dev, void* stream);

/* Batched inversion of `count` independent FP64 matrices of uneven orders,
 * each in place (the paper's method applied to every matrix; matrices do not
 * interact). For each elimination step k, the pivot inverses, row panels and
 * Schur updates of all matrices run as one grouped launch each.
 *  n            host int32[count]: orders.
 *  p            host int32[count]: blocks per matrix (ignored if block_sizes
 *               is NULL).
 *  block_sizes  host int32, the partitions concatenated, or NULL for the
 *               default: the paper's Table 2 rule below order 8, else four
 *               blocks of floor(n/4) (more when that exceeds 128), the last
 *               blocks taking the remainder. Every block order <= 512.
 *  A            host array of `count` device pointers; lda host int64[count].
 *  mode         BLOCKINV_F64 (other modes return BLOCKINV_ERR_INVALID).
 *  status_dev   device int32[count] (may be NULL): per-matrix BLOCKINV_OK,
 *               SINGULAR or NONFINITE.
 * Blocking (synchronises stream). Argument errors return at once. */
int blockinv_invert_batched(int32_t count, const int32_t* n, const int32_t* p, const int32_t* block_sizes,
                            double* const* A, const int64_t* lda, int mode, void* stream, int32_t* status_dev);

/* Reusable batch plan: validates the partitions and allocates the descriptor
 * tables and workspace once (the plan owns that device memory until
 * destroyed); the matrices' pointers are fixed in the plan. The first run
 * captures the launch sequence in a CUDA graph; every run replays it on
 * `stream` (stream-ordered, no synchronisation) and, if status_dev is not
 * NULL, writes the per-matrix status there. A plan must not be run on two
 * streams at the same time. */
typedef struct blockinv_batch_plan blockinv_batch_plan;
int blockinv_batch_plan_create(int32_t count, const int32_t* n, const int32_t* p, const int32_t* block_sizes,
                               double* const* A, const int64_t* lda, blockinv_batch_plan** plan);
int blockinv_batch_plan_run(blockinv_batch_plan* plan, void* stream, int32_t* status_dev);
int blockinv_batch_plan_destroy(blockinv_batch_plan* plan);

/* Batch autotuner. Matrices of order n >= 8 fall into size classes
 * c = floor(log2 n) (3 <= c <= 16). blockinv_batch_tune builds a synthetic
 * diagonally dominant batch with the orders n[count] (about 4096 of them at
 * most; device memory allocated and freed inside) and, class by class in
 * order of total work, times each candidate partition (p near-equal blocks,
 * every block of order 4..128) and Schur-update tile (64 x 64 or 32 x 32) on
 * the whole batch with the other classes at their current choice (best of
 * `reps` graph replays after one warm-up, 1 <= reps <= 100); the fastest,
 * or the class's current choice if none beats it, goes into a process-wide
 * table. Plans and blockinv_invert_batched calls made without
 * explicit partitions then use the table (explicit partitions keep their
 * blocks and take the class's tile). Blocking. Not part of the paper's
 * method: it chooses among partitions the method allows.
 * blockinv_batch_tuning reads a class's entry (nblocks 0 = not tuned);
 * blockinv_batch_tuning_set writes one (nblocks 0 clears it); _clear forgets
 * all; _save / _load write / read the table as text ("blockinv-batch-tuning 1"
 * then one "class nblocks tile" line per tuned class; load replaces the whole
 * table and leaves it unchanged on a malformed file). These five touch no
 * GPU state. */
int blockinv_batch_tune(int32_t count, const int32_t* n, int32_t reps, void* stream);
int blockinv_batch_tuning(int32_t size_class, int32_t* nblocks, int32_t* tile);
int blockinv_batch_tuning_set(int32_t size_class, int32_t nblocks, int32_t tile);
int blockinv_batch_tuning_clear(void);
int blockinv_batch_tuning_save(const char* path);
int blockinv_batch_tuning_load(const char* path);

/* ------------------------------------------------------------- serving ---
 * A serving context inverts independent requests (one matrix each, any
 * order and mode) as they arrive. A worker thread admits queued requests
 * first-fit whenever one of `max_slots` slots (CUDA streams) is free and the
 * request's device footprint fits in what is left of `hbm_budget_bytes`;
 * admitted requests run concurrently on their slots, and new arrivals join
 * as slots and memory free up (continuous batching). A request's result does
 * not depend on the other requests in flight. Not part of the paper's method:
 * a serving front end for it. */
typedef struct blockinv_ctx blockinv_ctx;

/* Submit flag: A is host memory (pinned for overlap); the context copies it
 * in and the inverse back out, counting the device copy in the budget. */
#define BLOCKINV_SUBMIT_HOST 1

typedef struct {
  int32_t status;        /* final status of the request                     */
  int32_t mode;          /* the mode that produced the result (see below)   */
  int64_t n;
  int32_t refine_iters;  /* mixed modes: Newton-Schulz updates              */
  int32_t used_fallback; /* 1: refinement failed, the FP64 path was rerun   */
  double rho;            /* mixed modes: final residual; else -1            */
  double t_queue_ms;     /* submit -> admitted                              */
  double t_device_ms;    /* GPU time of the request on its slot stream      */
  double t_total_ms;     /* submit -> result available                      */
} blockinv_result;

/* Create a context on `device` (1 <= max_slots <= 64). */
int blockinv_ctx_create(int device, size_t hbm_budget_bytes, int max_slots, blockinv_ctx** ctx);
/* Queue one inversion (arguments as blockinv_invert; A device memory unless
 * flags has BLOCKINV_SUBMIT_HOST). A must hold the input when this is called
 * (the context's streams do not wait for the caller's: finish any copy into
 * A first) and stay valid until the request is finished. Returns
 * BLOCKINV_ERR_BUDGET if the request alone exceeds the budget. *ticket
 * identifies the request.
 * Requests of order <= 512 are coalesced: at each admission pass every
 * queued one that fits in the budget (up to 512) is inverted in one batch
 * job by the grouped FP64 batched engine (partitions and Schur tiles from the
 * batch autotuner's table unless block_sizes is given), whatever the mode:
 * at these orders FP64 is faster than the mixed pipeline and exact to FP64
 * rounding. blockinv_result.mode then reads BLOCKINV_F64. */
int blockinv_submit(blockinv_ctx* ctx, int64_t n, int32_t p, const int32_t* block_sizes, double* A, int64_t lda,
                    int mode, int flags, uint64_t* ticket);
/* A mixed-mode request whose refinement does not converge (for example an
 * ill-conditioned input) is rerun on its slot with the FP64 path. */
/* BLOCKINV_PENDING while the request is queued or running; otherwise its
 * final status, with the record in *out; the ticket is then released. */
int blockinv_poll(blockinv_ctx* ctx, uint64_t ticket, blockinv_result* out);
/* As blockinv_poll, but blocks until the request is finished. */
int blockinv_wait(blockinv_ctx* ctx, uint64_t ticket, blockinv_result* out);
/* Cancel a queued request (its status becomes BLOCKINV_ERR_CANCELLED);
 * returns BLOCKINV_PENDING if it is already running. */
int blockinv_cancel(blockinv_ctx* ctx, uint64_t ticket);
/* Queued and running request counts and the device bytes admitted. */
int blockinv_ctx_stats(blockinv_ctx* ctx, int64_t* queued, int64_t* running, size_t* bytes_in_use);
/* Completion queue: up to max_tickets tickets of requests that finished (or
 * were cancelled) since they were last reported here, oldest first, into
 * tickets[]; *count receives how many. Their records are still taken with
 * blockinv_poll. */
int blockinv_poll_done(blockinv_ctx* ctx, uint64_t* tickets, int32_t max_tickets, int32_t* count);
/* Finish running requests, cancel queued ones, release everything. */
int blockinv_ctx_destroy(blockinv_ctx* ctx);

/* ------------------------------------------- step ranges and checkpoints ---
 * The paper's stop-and-resume by step (Sec. 5): the FP64 in-place
 * elimination after k steps leaves the whole state in A, so it can stop
 * between steps and continue later, in this or another process.
 *
 * blockinv_invert_steps applies elimination steps k0 .. k1 - 1
 * (0 <= k0 <= k1 <= number of blocks) of the FP64 path to A in place
 * (arguments as blockinv_invert; block_sizes NULL = the default partition).
 * Steps 0 .. p - 1 in one call or in consecutive ranges give the same bits as
 * blockinv_invert(..., BLOCKINV_F64, ...). Blocking; status as
 * blockinv_invert (SINGULAR / NONFINITE name the global block index).
 *
 * blockinv_checkpoint_write saves A (device, n x n, lda) with k_done and the
 * partition to `path`: "BLKINVC1", int64 n, int32 p, int32 k_done,
 * int32 sizes[p], uint64 FNV-1a hash of the matrix bytes, n * n doubles row by
 * row (little-endian). blockinv_checkpoint_read checks the file against n and
 * the partition and the hash on the host, then copies the matrix into A and
 * sets *k_done; any mismatch or damage returns BLOCKINV_ERR_INVALID with A
 * untouched. Both blocking (they synchronise `stream`). */
int blockinv_invert_steps(int64_t n, int32_t p, const int32_t* block_sizes, double* A, int64_t lda, int32_t k0,
                          int32_t k1, void* stream);
int blockinv_checkpoint_write(const char* path, int64_t n, int32_t p, const int32_t* block_sizes, const double* A,
                              int64_t lda, int32_t k_done, void* stream);
int blockinv_checkpoint_read(const char* path, int64_t n, int32_t p, const int32_t* block_sizes, double* A,
                             int64_t lda, int32_t* k_done, void* stream);

/* Block-size autotuner of the single-matrix path (and of the serving
 * context's requests above order 512). For every size class
 * c = floor(log2 n) among the orders n[count] above 16, it takes the
 * class's median order m, a synthetic diagonally dominant matrix of that
 * order (device memory allocated and freed inside), and times blocks of
 * order 64, 128, 192, 256, 320, 384 and 512 (those <= m; the last block the
 * remainder) over `reps` inversions in `mode` after one warm-up (1 <= reps
 * <= 100); the fastest goes into a process-wide table per mode and class.
 * Calls with p == 0 for n > 16 then use blocks of the tuned order (256 where
 * the class is untuned). Blocking. Not part of the paper's method: it
 * chooses among the partitions Eq. (blocking) allows.
 * blockinv_tuning reads an entry (0 = not tuned), blockinv_tuning_set writes
 * one (0 clears it), blockinv_tuning_clear forgets all; these three touch no
 * GPU state. Size classes run from 0 to 20. */
int blockinv_tune(int32_t count, const int32_t* n, int32_t mode, int32_t reps, void* stream);
int blockinv_tuning(int32_t mode, int32_t size_class, int32_t* block);
int blockinv_tuning_set(int32_t mode, int32_t size_class, int32_t block);
int blockinv_tuning_clear(void);

/* Options and per-call report for blockinv_invert_ex. */
typedef struct {
  double tol;          /* refinement target for rho (mixed modes); <= 0 means 1e-12     */
  int32_t max_refine;  /* Newton-Schulz iteration cap (mixed modes); < 0 means 5;      */
                       /* 0 returns the low-precision elimination unrefined           */
  int32_t fallback;    /* mixed modes: 1 = rerun in FP64 if refinement fails (default) */
  int32_t split;       /* mixed modes: 0 or 2 (default) = split each Schur-update operand */
                       /* into hi + lo and run hi*hi + hi*lo + lo*hi on the tensor cores; */
                       /* 1 = a single product                                           */
  int32_t pivot_f64;   /* mixed modes: 0 (default) = invert again in FP64 arithmetic the */
                       /* pivot blocks whose estimate ||P||_inf ||P^-1||_inf from the    */
                       /* FP32 inverse exceeds 1e5; 1 = every pivot block; -1 = none     */
  int32_t pivot_order; /* 0 (default) = pivot blocks first to last (Eq. (a) at every    */
                       /* step); 1 = last to first (Eq. (d): D and S_D = A - B D^-1 C)  */
  int32_t singular_fallback; /* FP64 mode: 1 = when a pivot block is singular, retry  */
                       /* from a saved copy of A with the other pivot order, then with  */
                       /* the failing block merged into a neighbour (up to order 512),  */
                       /* repeatedly; 0 (default) = return BLOCKINV_ERR_SINGULAR        */
  int32_t lookahead;   /* 0 (default) = for n >= 2048 and 3 or more blocks, start the next */
                       /* pivot inverse (FP64: and row panel) on a high-priority stream  */
                       /* of the library's while the rest of the current Schur update    */
                       /* runs; -1 = one step at a time. The result bits are the same.   */
  int32_t fuse;        /* mixed modes: 1 = unless lookahead is -1, apply the Schur       */
                       /* updates of two consecutive elimination steps in one sweep over  */
                       /* X (a rank b_k + b_{k+1} tensor-core update, after step k has    */
                       /* updated block row and column k + 1 alone), so that X is loaded  */
                       /* once for two steps' updates, as the paper's combined up/down    */
                       /* calculation (Sec. 5.6) avoids reloading blocks; the products   */
                       /* are summed in another order, so the bits differ. 0 (default) = */
                       /* one step per sweep (on this GPU the update is bound by the      */
                       /* tensor-core operand feed, not by moving X, and the second      */
                       /* step's pivot inverse can no longer overlap an update).         */
} blockinv_options;

typedef struct {
  int32_t status;         /* the returned status                                       */
  int32_t refine_iters;   /* Newton-Schulz updates applied                             */
  int64_t failing_block;  /* block index for SINGULAR / NONFINITE, else -1             */
  double rho;             /* final rho measured on the GPU (mixed modes), else -1      */
  double rho_initial;     /* rho of the unrefined low-precision inverse, else -1       */
  int32_t used_fallback;  /* 1 if the FP64 path produced the result after a failed     */
                          /* refinement                                                */
  int32_t fp64_pivots;    /* mixed modes: pivot blocks inverted again in FP64          */
  int32_t partition_fallback; /* 0: the requested partition and order; 1: the other  */
                          /* pivot order; 2: merged blocks (singular_fallback)          */
  int32_t blocks_used;    /* pivot blocks of the partition that produced the result    */
  int32_t incremental_residuals; /* mixed modes: residuals formed as E - A (X - X_prev) */
  int32_t incremental_groups; /* base-32 digit groups of the last one (1..9: 9 minus a  */
                          /* fifth of the exponent gap between X and its change)      */
  int32_t reserved[2];
} blockinv_info;

/* blockinv_invert with options and a report (either pointer may be NULL). */
int blockinv_invert_ex(int64_t n, int32_t p, const int32_t* block_sizes, double* A, int64_t lda,
                       int mode, void* stream, const blockinv_options* opt, blockinv_info* info);

/* Diagnostic: C[M x N] (FP32, row-major, ldc) = A[M x K] B[N x K]^T on the
 * tcgen05 tensor-core GEMM used by the mixed path, with A and B row-major
 * (K contiguous, leading dimensions lda / ldb in elements, rows 16-byte
 * aligned). kind 0: BF16 operands; 1: FP32 storage read as TF32; 2: FP8 E4M3;
 * each on single-CTA 128 x 256 output tiles. kind 3, 4, 5: the same three on
 * CTA pairs (256 x 256 tiles, the form the library's GEMMs run in).
 * Device pointers; blocking. Not part of the paper's method: it exists to
 * check the tensor-core path in isolation. */
int blockinv_diag_gemm(int kind, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                       const void* B, int64_t ldb, float* C, int64_t ldc, void* stream);

/* Diagnostic: out[i] = 1 / v[i] by the reciprocal the batched FP64 kernels
 * use (the hardware estimate and one third-order correction of the series
 * 1 / v = r / (1 - e), 3 FMAs; within one ulp of the IEEE quotient where v
 * and 1 / v are normal, the IEEE division elsewhere). count elements, device
 * pointers, stream-ordered (not blocking). Not part of the paper's method. */
int blockinv_diag_recip64(const double* v, double* out, int64_t count, void* stream);

/* Diagnostic: one bounded wait on an mbarrier that nothing arrives at, with
 * the wait function every tensor-core kernel of the library uses, limited to
 * limit_ns nanoseconds (0 .. 2e9; the kernels themselves use 2e9). When the
 * limit runs out the kernel records BLOCKINV_ERR_TIMEOUT in a status word
 * the way those kernels do, and this call returns that status (blocking).
 * No copy or tensor-core operation is pending when the wait gives up.
 * Not part of the paper's method: it exercises the timeout path. */
int blockinv_diag_wait_timeout(int64_t limit_ns, void* stream);

/* rho = ||A X - I||_F / (||A||_F ||X||_F), computed on the GPU with FP64
 * products and sums (device pointers, row-major). The normwise residual used
 * as the acceptance gate for every result. Blocking; the result goes to
 * *rho_out (host). */
int blockinv_residual(int64_t n, const double* A, int64_t lda, const double* X,
                      int64_t ldx, double* rho_out, void* stream);

/* FP64-accurate residual on the tensor cores: E = I - A X and
 * rho = ||E||_F / (||A||_F ||X||_F). The diagonal terms are exact FP64
 * products; the off-diagonal product comes from `slices` (7..9, 0 = 9)
 * base-32 FP8 digits of A (by rows) and X (by columns), 5 slices - 1 bits
 * of each entry relative to its row or column maximum, whose products
 * accumulate exactly. This is the residual the mixed modes' Newton-Schulz
 * refinement uses; blockinv_residual is the plain FP64 reference. Device
 * pointers; E (leading dimension lde) may be NULL. n <= 16384. Blocking. */
int blockinv_residual_tc(int64_t n, const double* A, int64_t lda, const double* X, int64_t ldx, double* E,
                         int64_t lde, int slices, double* rho_out, void* stream);

/* Workspace of the calls above comes from a device memory pool of the
 * library's own (one per device), which keeps what it has handed out so that
 * repeated calls do not map their workspace again. blockinv_release_memory
 * synchronises the current device and returns the pool's unused memory. */
int blockinv_release_memory(void);

/* Human-readable name of a status code (static string). */
const char* blockinv_status_str(int status);

/* Failing block index of the last SINGULAR / NONFINITE status returned on this
 * host thread (-1 if none); also returns that status. */
int blockinv_last_error_detail(int64_t* failing_block);

/* The cudaError_t value of the most recent CUDA runtime failure that a
 * library call (on any thread, serving workers included) reported as
 * BLOCKINV_ERR_CUDA or BLOCKINV_ERR_NOMEM, or 0 if there was none since the
 * library was loaded or this function was last called (it clears the value).
 * *name, if name is not NULL, gets the error's name (static string). */
int blockinv_last_cuda_error(const char** name);

/* ABI version: major * 10000 + minor * 100 + patch. */
int blockinv_version(void);

/* Sizes in bytes of blockinv_options, blockinv_info and blockinv_result as
 * this library was compiled (any pointer may be NULL), so that a binding can
 * check its own copies of the structures. Returns BLOCKINV_OK. */
int blockinv_struct_sizes(int32_t* options_bytes, int32_t* info_bytes, int32_t* result_bytes);

/* Kernel tracing (the library's own profiling hook; not part of the paper's
 * method). blockinv_trace_enable(1) clears and starts recording: every kernel
 * launch of the library is then bracketed by two CUDA events on its stream
 * and tagged with its algorithmic flops and bytes. blockinv_trace_enable(0)
 * stops recording. blockinv_trace_summary() waits for the recorded events,
 * writes a JSON object {"kernel": {"launches", "ms", "flops", "bytes"}, ...}
 * into buf (truncated to buflen - 1 characters, NUL-terminated), clears the
 * record and returns the length needed including the NUL. */
int blockinv_trace_enable(int on);
int64_t blockinv_trace_summary(char* buf, int64_t buflen);

#ifdef __cplusplus
}
#endif

#endif /* BLOCKINV_H */
