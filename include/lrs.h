/*
 * lrs.h - C ABI of the GB300 AltGDmin-LR+S solver (liblrs.so).
 *
 * Problem (arXiv 2311.03824, Section I-A): recover the n x q matrix
 * X* = L* + S*, L* = U* B* of rank r, S* with rho nonzeros per column, from
 * per-column measurements y_k = A_k x*_k (k = 0..q-1), A_k m x n.  A_k is a
 * dense Gaussian matrix or a row subset of the unitary 2D DFT (Section I-A,
 * "random Fourier matrix"; Section I-A notes the 2D-DFT case of dynamic MRI).
 * The solver runs Algorithm 1 (AltGDmin-L+S, Section II) with Algorithm 2
 * (IHT, Section II-D) entirely in CUDA kernels on one GPU.
 *
 * Conventions shared by every call:
 *  - Every call returns an lrs_status; nothing throws or aborts across the ABI.
 *    lrs_last_error() returns a thread-local message for the last failure.
 *  - Handle states: CREATED -> MEASURED (lrs_set_measurements) ->
 *    INITIALISED (lrs_init) -> ITERATING (lrs_iterate).  A call made in the
 *    wrong state returns LRS_ERR_STATE and changes nothing.
 *  - The handle owns all device memory it allocates; lrs_destroy frees it.
 *    Inputs are copied into the handle's own layout during the call that
 *    receives them (host or device pointers); the caller may free them after
 *    that call returns.  Outputs go to caller-owned buffers.
 *  - All kernels run on the stream given in lrs_options.stream (a
 *    cudaStream_t; NULL = the legacy default stream).  Calls that return host
 *    data synchronise that stream.
 *  - Matrices are column-major unless stated: "m x q column-major" means
 *    element (i, k) at offset i + k*m, i.e. each column is contiguous.
 */
#ifndef LRS_H_
#define LRS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lrs_ctx* lrs_t;

typedef enum {
  LRS_OK = 0,
  LRS_ERR_ARG = 1,          /* invalid argument (sizes, pointers, options)     */
  LRS_ERR_STATE = 2,        /* call made in the wrong handle state             */
  LRS_ERR_OOM = 3,          /* device or host allocation failed                */
  LRS_ERR_CUDA = 4,         /* a CUDA runtime call failed                      */
  LRS_ERR_NUMERICAL = 5,    /* non-SPD r x r Gram (LS step / QR) or NaN/Inf    */
  LRS_ERR_TIMEOUT = 6,      /* a bounded device wait or a request timed out    */
  LRS_ERR_UNSUPPORTED = 7   /* valid input this build does not handle          */
} lrs_status;

typedef enum {
  LRS_OP_GAUSSIAN = 0,      /* dense A_k, i.i.d. N(0,1) in the paper           */
  LRS_OP_DFT2D_MASK = 1     /* A_k x = (F2 x)[Omega_k], F2 unitary 2D DFT      */
} lrs_op_kind;

typedef enum {
  LRS_A_FP32 = 0,           /* A_k kept in float32 (the exact operator)        */
  LRS_A_BF16 = 1,           /* A_k kept in bfloat16                            */
  LRS_A_FP8_HI = 2,         /* e4m3 hi with one float32 scale per row          */
  LRS_A_FP8_HILO = 3        /* e4m3 hi + e4m3 lo of the remainder, row scale   */
} lrs_a_dtype;

/* Column-sharded solves (Section II-E: the columns are split across nodes
 * and only n x r sums travel): a handle holds a contiguous range of the
 * columns of a larger problem, and at every column reduction (each
 * subspace-iteration step of lrs_init, each gradient of lrs_iterate) the
 * library calls this function with its partial sums: nb_mine blocks of
 * n x w float32 (row-major, one block per grad_block columns, in column
 * order; host memory).  It must write into `all` (room for cap blocks) the
 * partial blocks of every shard in global column order and return how many
 * it wrote, or a negative value on failure (the call then returns
 * LRS_ERR_ARG).  The library adds the blocks in that order, so a solve whose
 * shards start at multiples of grad_block gives bit for bit the result of
 * one handle over all columns with the same grad_block.  Every shard makes
 * the same sequence of calls. */
typedef int32_t (*lrs_reducer)(void* ctx, const float* mine, int32_t nb_mine, int64_t n,
                               int32_t w, float* all, int32_t cap);

/* Options.  A zero-initialised struct selects the paper's defaults
 * (Algorithm 1 and Section II-F): tau0 = 10, tau = 3, T = 200, c_eta = 0.14,
 * rho_max = rho, float32 A_k. */
typedef struct {
  int32_t tau0;             /* IHT sweeps in the initialisation (0 -> 10)      */
  int32_t tau;              /* IHT sweeps per GDmin iteration (0 -> 3)         */
  int32_t T;                /* iterations run by lrs_solve (0 -> 200)          */
  double c_eta;             /* eta = c_eta / ||grad_U f(U0,B1,S1)||_2 (0 -> 0.14) */
  int32_t rho_max;          /* entries HardThreshold keeps (0 -> rho)          */
  int32_t nx, ny;           /* DFT frame: n = nx*ny (powers of two, or n <= 4096) */
  lrs_a_dtype a_dtype;      /* storage of A_k for the sweeps                   */
  int32_t refine_every;     /* low-precision A_k: defect correction of y_k with
                               the exact FP32 operator every this many
                               iterations (0 -> 8); see lrs_iterate          */
  int32_t cluster;          /* Gaussian sweep: CTAs per column (0 -> autotune) */
  int32_t power_iters;      /* cap on subspace iterations in lrs_init (0 -> 1000) */
  double power_tol;         /* stop when ||(I - U_old U_old^T) U||_F < tol (0 -> 1e-6;
                               float32 products resolve about 1e-7)      */
  int32_t use_graph;        /* 1: replay steady-state iterations as a CUDA graph */
  void* stream;             /* cudaStream_t for every launch (NULL = default)  */
  uint64_t seed;            /* seed of the subspace-iteration start            */
  int32_t profile;          /* 1: time each phase of lrs_iterate with CUDA events;
                               2: also count SM cycles per sweep phase       */
  int32_t slab_mode;        /* Gaussian sweep: 0 auto, 1 slab resident in shared
                               memory, 2 slab streamed through a tile ring   */
  int32_t stages;           /* tile stages of the streamed ring (0 -> auto)    */
  int32_t engine;           /* Gaussian sweep engine: 0 auto, 1 one thread-block
                               cluster per column, 2 persistent task engine
                               (passes over A_k split into tasks, columns
                               in flight share the GPU), 3 register-resident
                               cluster engine (each CTA keeps its 128
                               columns of A_k in registers through the whole
                               column sweep; float32 A_k, r <= 8, m <= 192,
                               n <= 1024, rho_max <= 32)                     */
  int32_t inflight;         /* task engine: columns in flight (0 -> all q)    */
  int32_t task_kib;         /* task engine: A_k bytes per task in KiB (0 -> 256) */
  int32_t ctas_per_sm;      /* task engine: resident CTAs per SM (0 -> 2, or 1
                               when two do not fit; 3 allowed for r <= 6)    */
  int32_t autotune;         /* task engine: 1 = run lrs_autotune (2 trial
                               iterations per shape) before the first
                               iteration unless this shape is cached         */
  int32_t grid;             /* task engine: CTAs of the persistent launch (0 ->
                               all that fit; fewer let concurrent handles on
                               other streams share the GPU); resident engine:
                               at most grid / cluster clusters             */
  int32_t wait_ms;          /* bound of every device-side wait of the task and
                               resident engines (0 -> 10000 ms); a wait that
                               expires makes the call return LRS_ERR_TIMEOUT */
  int32_t grad_block;       /* columns per partial sum of the column reductions
                               (0 -> chosen for the grid; fixed when a
                               reducer is set or results must match a
                               column-sharded solve)                         */
  lrs_reducer reduce;       /* column-sharded solve (see lrs_reducer); NULL for
                               a handle that holds the whole problem; needs
                               grad_block > 0 and use_graph = 0             */
  void* reduce_ctx;         /* first argument of reduce                        */
  int32_t reduce_cap;       /* partial blocks of all shards together (the `cap`
                               of reduce)                                    */
  int32_t test_withhold;    /* test aid for the failure path (0 in use): the
                               task engine's queue holds one ticket that is
                               never published, so the wait for it runs out
                               after wait_ms and the call returns
                               LRS_ERR_TIMEOUT with the device still usable  */
} lrs_options;

/* Create a solver for one problem (Section I-A sizes).
 * n, m, q >= 1; 1 <= r <= 16 and r <= min(m, n); 0 <= rho <= n; for
 * LRS_OP_DFT2D_MASK, opt->nx * opt->ny == n with both powers of two, or
 * n <= 4096 for other sides (a direct DFT along those) (m may
 * exceed n only for the Gaussian operator's special cases; for the DFT
 * m <= n).  opt may be NULL (paper defaults).  On success *out holds a new
 * handle in state CREATED.  Errors: LRS_ERR_ARG, LRS_ERR_OOM, LRS_ERR_CUDA. */
lrs_status lrs_create(int64_t n, int64_t m, int64_t q, int32_t r, int32_t rho,
                      lrs_op_kind kind, const lrs_options* opt, lrs_t* out);

/* Give the measurements y_k and the operator (Section I-A: y_k = A_k x*_k).
 *  y:         m x q column-major; float for GAUSSIAN, interleaved complex64
 *             (re, im float pairs) for DFT2D_MASK.
 *  A_or_mask: GAUSSIAN: q consecutive m x n row-major float blocks (A_k
 *             element (i, j) at offset k*m*n + i*n + j).
 *             DFT2D_MASK: q x m int32 row indices, column k (m consecutive
 *             values) lists the kept DFT rows kx*ny + ky of frame k, each in
 *             [0, n) and strictly ascending.
 *  mem_kind:  0 = host pointers, 1 = device pointers.  Either way the data is
 *             copied (and re-laid-out) before the call returns.
 * With a_dtype BF16 / FP8_HI / FP8_HILO the handle keeps the FP32 blocks as
 * given (the exact operator, used by the defect correction) plus the sweep's
 * encoded copy: BF16 by round-to-nearest; FP8_HI as e4m3(A(i,j)/s1_i) with
 * s1_i = max_j |A(i,j)| / 448; FP8_HILO adds a second e4m3 plane of the
 * remainder A - s1_i hi with its own row scale s2_i.
 * State: CREATED or later (re-measuring resets the handle to MEASURED).
 * Errors: LRS_ERR_ARG (NULL pointer, bad mem_kind, mask out of range or not
 * ascending), LRS_ERR_STATE, LRS_ERR_OOM, LRS_ERR_CUDA. */
lrs_status lrs_set_measurements(lrs_t h, const void* y, const void* A_or_mask,
                                int32_t mem_kind);

/* Initialisation of Algorithm 1: s_k = IHT(y_k, A_k, rho, tau0, 0),
 * L0 = [A_k^T (y_k - A_k s_k)], U0 = top-r left singular subspace of L0
 * (subspace iteration: float32 products L0^T U and L0 P, Cholesky-QR2 with
 * FP64 r x r factors, to power_tol), b_k = (A_k U0)^+ (y_k - A_k s_k).  State: MEASURED or later -> INITIALISED.
 * Errors: LRS_ERR_STATE, LRS_ERR_NUMERICAL (non-SPD Gram, NaN), LRS_ERR_CUDA. */
lrs_status lrs_init(lrs_t h);

/* Automatic rank (Section II-F, parameter setting): the b% energy threshold
 * on the leading singular values of L0.  Runs the IHT of the initialisation
 * (s_k = IHT(y_k, A_k, rho, tau0, 0), L0 = [A_k^T (y_k - A_k s_k)], which does
 * not depend on r), estimates the first N = max(1, floor(min(n, q, m) / 10))
 * singular values of L0 by subspace iteration in blocks of 16 columns (the
 * widest the r x r kernels hold; one block of min(16, n, q) when N <= 16),
 * each block deflated by the ones before it (float32 products, FP64
 * Cholesky-QR2 factors and Rayleigh-Ritz values), and returns in *r_out the
 * smallest r <= N with sigma_1^2 + ... + sigma_r^2 >= energy * (sigma_1^2 +
 * ... + sigma_N^2).  N is capped at 64 (four blocks).
 * sv: NULL or a host array of sv_len doubles that receives the first
 * min(N, sv_len) singular values (descending); *n_sv (if not NULL) = N.
 * The handle's rank is the one it was created with: to solve at the
 * estimated rank, create a handle with r = *r_out.  The call leaves the
 * handle in state MEASURED (call it before lrs_init).  Gaussian operators.
 * Errors: LRS_ERR_ARG (energy outside (0, 1], r_out NULL), LRS_ERR_STATE (not
 * MEASURED), LRS_ERR_UNSUPPORTED (DFT operator), LRS_ERR_NUMERICAL,
 * LRS_ERR_CUDA. */
lrs_status lrs_estimate_rank(lrs_t h, double energy, int32_t* r_out, double* sv,
                             int32_t sv_len, int32_t* n_sv);

/* Run `iters` GDmin iterations of Algorithm 1 (t continues from the last
 * call): P_perp-projected IHT for s_k (tau sweeps), LS for b_k,
 * grad = sum_k A_k^T (A_k(U b_k + s_k) - y_k) b_k^T, eta from the t = 1
 * gradient (spectral norm), U <- Q(U - eta grad) by Cholesky-QR2.
 * err_log: NULL, or a host array of `iters` doubles that receives
 * ||X_t - X_ref||_F / ||X_ref||_F after each iteration (needs
 * lrs_set_reference).
 * Low-precision A_k (a_dtype != FP32): the sweep runs on the encoded copy
 * Ã_k against corrected measurements ỹ_k = y_k - (A_k - Ã_k)(U b_k + s_k),
 * refreshed with the exact operator before the first iteration after
 * lrs_init / lrs_set_state and then every refine_every iterations, so that
 * an exact solution of y_k = A_k x_k is a fixed point of the iteration
 * (defect correction; the paper computes in one precision throughout).
 * State: INITIALISED or ITERATING -> ITERATING.
 * Errors: LRS_ERR_ARG (iters < 0, err_log without reference), LRS_ERR_STATE,
 * LRS_ERR_NUMERICAL (column id in lrs_last_error), LRS_ERR_CUDA. */
lrs_status lrs_iterate(lrs_t h, int32_t iters, double* err_log);

/* `iters` GDmin iterations of several problems at once: every sweep is one
 * persistent launch of the task engine whose work table holds the columns of
 * all nh handles (Section II-E: the per-column work is independent, so
 * uneven problems share the GPU's SMs in one launch); each handle then runs
 * its own gradient, step size and QR on its own stream.  Every handle ends
 * exactly as lrs_iterate(h, iters, NULL) would leave it alone, bit for bit.
 * hs: nh distinct handles (1 <= nh <= 64), INITIALISED or later, Gaussian,
 * task engine (engine 2), one rank width class and one A_k form, no reducer.
 * The call returns when every handle's work is done.  State -> ITERATING.
 * Errors: LRS_ERR_ARG, LRS_ERR_STATE, LRS_ERR_UNSUPPORTED (handles that
 * cannot share a launch), LRS_ERR_NUMERICAL, LRS_ERR_TIMEOUT, LRS_ERR_CUDA. */
lrs_status lrs_iterate_batch(lrs_t* hs, int32_t nh, int32_t iters);

/* lrs_init followed by lrs_iterate(h, T, NULL).  State: MEASURED or later. */
lrs_status lrs_solve(lrs_t h);

/* Copy out the current factors (Algorithm 1, Output: x_k = U b_k + s_k).
 *  U:     n x r column-major (float, or complex64 for DFT2D_MASK), or NULL
 *  B:     r x q column-major (same type), or NULL
 *  S_idx: rho_max x q column-major int32, each column ascending, or NULL
 *  S_val: rho_max x q column-major values matching S_idx, or NULL
 * mem_kind: 0 = host buffers (the call synchronises the stream), 1 = device.
 * State: INITIALISED or ITERATING.  Errors: LRS_ERR_STATE, LRS_ERR_ARG,
 * LRS_ERR_CUDA. */
lrs_status lrs_get(lrs_t h, void* U, void* B, int32_t* S_idx, void* S_val,
                   int32_t mem_kind);

/* The current iterate itself, X = U B + S (Algorithm 1, Output:
 * x_k = U b_k + s_k), assembled on the device in float32 (complex64 for
 * DFT2D_MASK).  X: n x q column-major; mem_kind 0 = host buffer (the call
 * synchronises the stream), 1 = device.  State: INITIALISED or ITERATING.
 * Errors: LRS_ERR_ARG, LRS_ERR_STATE, LRS_ERR_OOM, LRS_ERR_CUDA. */
lrs_status lrs_get_x(lrs_t h, void* X, int32_t mem_kind);

/* Restore a state written by lrs_get (same layouts, host or device), so that
 * a run can be resumed: t is the number of iterations already done and eta
 * the frozen step size (ignored when t == 0).  State: MEASURED or later ->
 * INITIALISED (t == 0) or ITERATING.  Errors: LRS_ERR_ARG, LRS_ERR_STATE,
 * LRS_ERR_CUDA. */
lrs_status lrs_set_state(lrs_t h, const void* U, const void* B,
                         const int32_t* S_idx, const void* S_val, int32_t t,
                         double eta, int32_t mem_kind);

/* Frozen step size eta and the number of iterations done so far. */
lrs_status lrs_get_progress(lrs_t h, double* eta, int32_t* t);

/* Reference X* (n x q column-major, float or complex64, host or device) for
 * the error log of lrs_iterate (Section III error metric
 * ||X* - X||_F / ||X*||_F).  The data is copied.  Errors: LRS_ERR_ARG,
 * LRS_ERR_STATE, LRS_ERR_OOM, LRS_ERR_CUDA. */
lrs_status lrs_set_reference(lrs_t h, const void* Xref, int32_t mem_kind);

/* Device time accumulated by lrs_iterate since the previous call, measured
 * with CUDA events on the handle's stream when lrs_options.profile = 1
 * (tracing aid; Algorithm 1 phases):
 *   out[0] ms in the per-column sweep kernel (IHT, LS, gradient terms)
 *   out[1] ms in the column reduction of the gradient
 *   out[2] ms in the step size and Cholesky-QR2 of U
 *   out[3] number of iterations timed
 * The counters restart at zero after the call.  Errors: LRS_ERR_ARG,
 * LRS_ERR_CUDA. */
lrs_status lrs_phase_times(lrs_t h, double* out4);

/* Autotuner of the task engine (the paper has no counterpart): from the
 * current iterate, run trial_iters GDmin iterations
 * with each candidate task shape (128 / 256 / 512 KiB of A_k per task x
 * q, q/2 or 2 x grid columns in flight), restoring the iterate (U, B, S,
 * eta, t and the corrected measurements) after each, keep the fastest and
 * cache it for the process, keyed by (n, m, q, r, rho_max, a_dtype, grid):
 * later handles of the same shape start with it.  report: NULL or a buffer
 * of len bytes receiving a JSON summary of the trials.  State: INITIALISED
 * or later (unchanged on return).  Errors: LRS_ERR_ARG, LRS_ERR_STATE,
 * LRS_ERR_UNSUPPORTED (cluster engine or DFT operator), LRS_ERR_OOM,
 * LRS_ERR_CUDA, LRS_ERR_NUMERICAL. */
lrs_status lrs_autotune(lrs_t h, int32_t trial_iters, char* report, int32_t len);

/* Orthonormalise the columns of Z by Cholesky-QR2 (the QR step of
 * Algorithm 1, U+ = QR(U - eta grad)): Q = Z R^{-1} with R the upper
 * triangular factor with positive diagonal, i.e. the Q factor of the QR
 * decomposition with diag(R) > 0.  Gram matrices and Cholesky factors are
 * FP64 (r x r), products FP32, two passes.
 *  Z, Q:   device pointers, n x r row-major float (row i at offset i*r);
 *          Q may equal Z.  1 <= r <= 16, n >= r.
 *  stream: cudaStream_t (NULL = legacy default stream); the call allocates
 *          its scratch with cudaMalloc, runs on the stream and synchronises it.
 * Errors: LRS_ERR_ARG, LRS_ERR_OOM, LRS_ERR_NUMERICAL (Z rank deficient),
 * LRS_ERR_CUDA. */
lrs_status lrs_orthonormalize(const float* Z, float* Q, int64_t n, int32_t r, void* stream);

/* lrs_orthonormalize without any device allocation.  The paper has no
 * counterpart: this call exists for callers that cannot allocate device
 * memory at the moment they need the step - an application that has handed
 * all of its device memory to its own pool, or a serving loop that must not
 * stall the other streams on the device-wide synchronisation that
 * cudaMalloc/cudaFree imply.  It computes exactly what lrs_orthonormalize
 * computes, with the same arguments and layouts, but uses a fixed scratch
 * array of about 4.6 MB that lives in the library's device image: every GPU
 * that loads the library holds it until the process exits.
 *  Limits: 1 <= r <= 16, r <= n <= 65536; larger sizes return LRS_ERR_ARG.
 *  The first call on a device (with that device current) looks up the
 *  scratch's device address with cudaGetSymbolAddress and keeps it for the
 *  process; make that first call before any stream capture, and do not use
 *  the call on a device after its context has been reset (cudaDeviceReset)
 *  in the same process.  All calls share the one array and the error word in
 *  it (cleared at the start of every call): calls whose work can overlap on
 *  the GPU (different streams, or different host threads on one device)
 *  race on it and must be serialised by the caller.  Each call runs on
 *  `stream`, copies the error word back to the host and synchronises the
 *  stream before it returns.  Its own error message is returned by
 *  lrs_noalloc_last_error().
 * Errors: LRS_ERR_ARG, LRS_ERR_NUMERICAL (Z rank deficient), LRS_ERR_CUDA. */
lrs_status lrs_orthonormalize_noalloc(const float* Z, float* Q, int64_t n, int32_t r,
                                      void* stream);
const char* lrs_noalloc_last_error(void);

/* ---- serving (the paper has no counterpart: a request loop for many
 * problems of Section I-A on one GPU) ------------------------------------ */

/* One reconstruction problem for the server: the arguments of lrs_create and
 * lrs_set_measurements, the iterations to run (opt.T, 0 -> 200) and where
 * to put the result (as lrs_get; NULL pointers are skipped).  opt.stream is
 * ignored (each worker has its own stream); opt.grid 0 lets the server
 * share the SMs among the Gaussian requests running.  The input and output
 * buffers belong to the caller and must stay valid until lrs_server_wait has
 * returned the request's result.  Device inputs must be ready (their
 * producing work complete) when the request is submitted. */
typedef struct {
  int64_t n, m, q;
  int32_t r, rho;
  lrs_op_kind kind;
  lrs_options opt;
  const void* y;
  const void* A_or_mask;
  int32_t mem_kind;         /* of y and A_or_mask: 0 host, 1 device           */
  void* U;
  void* B;
  int32_t* S_idx;
  void* S_val;
  int32_t out_mem_kind;     /* of U, B, S_idx, S_val: 0 host, 1 device        */
  void* user;               /* opaque, handed to a custom runner               */
} lrs_request;

/* Outcome of one request.  Times are seconds since lrs_server_create. */
typedef struct {
  lrs_status status;        /* of the request's own calls                     */
  char message[256];        /* lrs_last_error() of the failing call, or ""    */
  double submit_s, start_s, end_s;
  size_t footprint;         /* device bytes reserved while it ran             */
  int32_t worker;           /* slot that ran it                               */
  int32_t grid;             /* SM share (CTAs) offered to its sweep           */
  int64_t admitted;         /* its place in the order of admission (0, 1, ..) */
  int64_t group;            /* `admitted` of the first request of the batch it
                               ran in (its own when it ran alone)            */
  int32_t group_size;       /* requests of that batch                         */
} lrs_result;

/* A replacement for the solver of one request (used to test the admission
 * logic without a GPU): returns an lrs_status. */
typedef int32_t (*lrs_runner)(void* ctx, const lrs_request* req, int32_t grid, int32_t worker);

typedef struct {
  size_t hbm_budget;        /* device bytes the requests in flight may hold
                               (0 -> 85 % of the free memory at creation)    */
  int32_t slots;            /* requests (or batches) in flight at most (0 -> 8) */
  int32_t sms;              /* SMs shared by the sweeps (0 -> the device's)   */
  lrs_runner runner;        /* NULL: the library's solver                     */
  void* runner_ctx;
  int32_t batch;            /* up to this many Gaussian requests admitted
                               together run their iterations in one
                               persistent launch per sweep (lrs_iterate_batch;
                               0 or 1: every request alone)                 */
} lrs_server_options;

typedef struct lrs_server_s* lrs_server_t;

/* Create a server: `slots` worker threads, each with its own CUDA stream,
 * and a dispatcher.  Requests are admitted in submission order as soon as a
 * slot is free and lrs_request_footprint(req) fits what the requests in
 * flight leave of hbm_budget; each runs lrs_create, lrs_set_measurements,
 * lrs_init, lrs_iterate(T) and lrs_get on its worker's stream, so the work
 * of concurrent requests overlaps on the GPU, and a Gaussian request's
 * persistent sweep gets max(16, 2 x SMs / requests running) CTAs, and its
 * steady iterations replay as a CUDA graph.  With
 * batch > 1, when the admitted request is Gaussian the queued requests right
 * behind it of the same rank, A_k form and iteration count that also fit
 * (budget) are admitted with it, up to `batch` of them, into the same slot,
 * and its worker runs their iterations together (lrs_iterate_batch).  The kernels'
 * results depend neither on the other requests, nor on that share, nor on
 * the batch: every result equals the request solved alone.
 * Errors: LRS_ERR_ARG, LRS_ERR_CUDA (no device). */
lrs_status lrs_server_create(const lrs_server_options* opt, lrs_server_t* out);

/* Queue a request; *ticket identifies it for lrs_server_wait.  The request
 * is copied (not its buffers).  Errors: LRS_ERR_ARG, LRS_ERR_OOM (larger
 * than the whole budget), LRS_ERR_STATE (server being destroyed). */
lrs_status lrs_server_submit(lrs_server_t s, const lrs_request* req, uint64_t* ticket);

/* Wait until the request of `ticket` has finished (timeout_ms < 0: no
 * limit) and copy its outcome to *res; the ticket is then released.
 * Errors: LRS_ERR_ARG (unknown ticket), LRS_ERR_TIMEOUT (not finished in
 * timeout_ms; the ticket stays valid). */
lrs_status lrs_server_wait(lrs_server_t s, uint64_t ticket, int32_t timeout_ms, lrs_result* res);

/* Stop accepting requests, run those already queued, join the workers and
 * free the server.  Outcomes not yet waited for are discarded. */
lrs_status lrs_server_destroy(lrs_server_t s);

/* Device bytes the server reserves for a request while it runs (its stored
 * operator, the exact copy of a low-precision form, the staging of host
 * inputs, per-column scratch and the iterate, with 10 % and 64 MiB of
 * headroom). */
size_t lrs_request_footprint(const lrs_request* req);

/* Thread-local message of the last failed server call ("" if none). */
const char* lrs_server_last_error(void);

/* Per-column SM cycle counts of the sweep phases accumulated by
 * lrs_iterate since the previous call (handle created with profile = 2;
 * tracing aid).  out receives q x 12 counters, column-major by column k:
 * setup, W = A U, A s exchange, projection of u, column product (IHT),
 * A g_G exchange, projection and norm of M g_G, HardThreshold, final A s,
 * LS and residual, final column product, output writes.  With the task
 * engine (engine = 2) out receives 15 launch-wide counters instead (cycles
 * summed over CTAs): waiting for a task, in W tasks, in A^T tasks, waiting
 * for pieces inside tasks, in the small steps after W / IHT / final passes,
 * producer waiting for a ticket, the numbers of tasks and small steps, then
 * the IHT step's parts: loads, mu, HardThreshold, next residual, publish.
 * A DFT2D_MASK handle gives 8 counters (thread-0 cycles summed over the
 * frames' CTAs): set-up and Gram, sparse DFTs, norms and updates, FFTs,
 * HardThreshold, final stage, LS solves, projection applies.
 * len is the capacity of out in elements.  Counters restart at zero.
 * Errors: LRS_ERR_ARG, LRS_ERR_STATE (no trace buffer), LRS_ERR_CUDA. */
lrs_status lrs_sweep_trace(lrs_t h, uint64_t* out, int64_t len);

/* Write a one-line JSON description of the handle's launch shape (operator,
 * CTAs per column or frame, slab width, shared memory per CTA, resident
 * clusters, and "launches_per_iteration": the kernels one steady iteration
 * launches; DFT handles also give "fused_qr", 1 when the step and its
 * Cholesky-QR2 run as one cooperative launch) into buf (NUL-terminated,
 * truncated to len bytes).  Errors: LRS_ERR_ARG. */
lrs_status lrs_describe(lrs_t h, char* buf, int32_t len);

/* Release every resource of the handle (NULL is accepted). */
lrs_status lrs_destroy(lrs_t h);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* lrs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LRS_H_ */
