// Internal interfaces between the C ABI driver (lrs_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace lrs {

// Error codes written to the device error word {code, column} (first writer wins).
enum : int { kErrNone = 0, kErrNotSPD = 1, kErrNaN = 2, kErrTimeout = 3 };

// Sweep modes of the per-column kernel (Algorithm 1).
enum SweepMode : int {
  kModeInit = 0,  // IHT(y_k, A_k, rho, tau0, 0) then L0 column A_k^T(y_k - A_k s_k)
  kModeLS = 1,    // b_k = (A_k U)^+ (y_k - A_k s_k) with the current s_k
  kModeIter = 2   // one GDmin iteration's per-column work (lines z_k .. gradient term)
};

// Layout of the Gaussian operator inside the handle ("slab" layout): column k's
// A_k is split by columns j into `cs` slabs of `ns` columns (ns a multiple of
// 32); slab c holds columns [c*ns, min(n, (c+1)*ns)), zero-padded, as ns/32
// consecutive tiles of m rows x 32 elements; inside a tile, row i is 32
// consecutive elements whose 4-element chunks are XOR-permuted by (i mod 8):
//   A_k(i, c*ns + 32*b + 4*q + e) is element
//   ((k*cs + c)*ns*m) + b*32*m + i*32 + 4*(q ^ (i & 7)) + e
// counted in elements of the stored type.  The FP8 hi/lo form stores each
// tile as its hi plane (m x 32 bytes) followed by its lo plane, so a tile is
// 64*m bytes and element offsets inside a plane are as above.
struct GaussLayout {
  int n, m, q, r, rho;
  int cs;      // CTAs per column (thread-block cluster size)
  int ns;      // slab width (multiple of 32)
  int stages;  // tile stages of the streamed ring (ignored when resident)
  int et;      // element type of the stored A_k: 0 fp32, 1 bf16, 2 fp8 e4m3 (row scale),
               // 3 fp8 e4m3 hi + lo planes (two row scales)
};

// bytes per element of a tile (both planes for the hi/lo form)
__host__ __device__ inline int elem_bytes(int et) { return et == 0 ? 4 : (et == 1 || et == 3) ? 2 : 1; }

struct SweepArgs {
  GaussLayout L;
  int mode;
  int tau;
  const void* A;    // slab layout, element type L.et
  const float* y;   // q x m (y_k contiguous)
  const float* U;   // n x r row-major
  const float* Upad;  // (cs*ns) x sweep_rpad(r) row-major, zero padded
  const float* rscale;  // FP8 forms: q x m x (1 or 2) per-row scales (hi, lo)
  int* S_idx;       // q x rho (ascending per column), in/out
  float* S_val;     // q x rho
  float* B;         // q x r (b_k contiguous)
  float* H;         // q x n: ITER: h_k = A_k^T(W b + A s - y); INIT: L0 column
  int* err;         // device error word pair {code, column}
  int resident;     // 1: slab staged once in shared memory; 0: streamed per product
  unsigned long long* trace;  // optional: per-column cycle counts of the sweep phases
};

// Phases of the per-column sweep recorded by the trace (cycles, summed over
// the IHT steps): setup, W pass, A s exchange, projection of u, column pass
// (IHT), A g_G exchange, projection + norm of M g_G, HardThreshold, final
// A s, LS + residual, final column pass, output writes.
constexpr int kTracePhases = 12;

// Largest dynamic shared memory a CTA may request on the current device.
// Kernels shared by every handle get this as their limit once and for all:
// a per-handle value would race with handles of other sizes launching
// concurrently on other streams.
inline int smem_optin_limit() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v > 0 ? v : 232448;
}

// Sweep kernel (sweep_gauss.cu).
size_t sweep_smem_bytes(const GaussLayout& L, int resident, int nthreads);
cudaError_t sweep_launch(const SweepArgs& a, int nthreads, cudaStream_t s);
cudaError_t sweep_prepare(const GaussLayout& L, int nthreads);  // set attributes
int sweep_max_active_clusters(const GaussLayout& L, int resident, int nthreads);
cudaError_t repack_gauss(const GaussLayout& L, const float* A_rowmajor, int k0, int kc,
                         void* A_int, float* rscale, cudaStream_t s);
// ycorr_k = y_k - (A_k - Atilde_k)(U b_k + s_k) for every column (exact FP32
// operator A row-major q x m x n, Atilde in the slab layout of element type
// L.et != 0); xbuf: q x n scratch that receives x_k = U b_k + s_k.
cudaError_t refine_residual(const GaussLayout& L, const float* A_exact, const void* A_int,
                            const float* rscale, const float* U, const float* Bk,
                            const int* S_idx, const float* S_val, const float* y, float* ycorr,
                            float* xbuf, cudaStream_t s);

// ---- persistent task engine (task_sweep.cu) ---------------------------------
// The per-column sweep split into tasks: every product over A_k is cut into
// blocks (W = A_k U: row block x column chunk; A_k^T v: column chunk, all
// rows), each streamed by TMA in pieces of one 32-column tile x a row range.
// A persistent grid pops tasks from a global ticket queue; the CTA that
// completes the last task of a column's pass runs that column's small step
// (Gram + Cholesky, mu, HardThreshold, LS, projections) and pushes the next
// pass.  Up to F columns are in flight (all q by default).
enum TaskType : int { kTaskW = 0, kTaskG = 1, kTaskF = 2, kTaskNop = 3, kTaskExit = 4 };

struct TaskProblem {
  GaussLayout L;        // cs == 1 layout (one slab per column, ns = n rounded up to 32)
  int mode, tau_eff;    // sweep mode; IHT sweeps actually run (0 when rho == 0)
  const void* A;        // slab layout, element type L.et
  const float* rscale;  // FP8 forms: q x m x (1 or 2) row scales
  const float* y;       // q x m measurements seen by the sweep
  const float* Upad;    // ns x R zero-padded U
  int* S_idx;           // q x rho in/out (ascending)
  float* S_val;
  float* B;             // q x r
  float* H;             // q x n
  int* err;
  // per-column scratch
  float* Wk;            // q x wstride (m x R)
  float* Wp;            // q x ncw x wstride: partial W per column chunk
  double* Gi;           // q x kMaxR x kMaxR  G^{-1} (FP64)
  float* uvec;          // q x m  vector of the next A^T pass
  float* g;             // q x ns result of the IHT pass
  int* supj;            // q x rho current support (global indices, key order)
  float* As;            // q x astride: A_k s_k for the current support values (unprojected)
  float* supv;
  int* nsup;            // q
  int* cnt;             // q tasks completed in the current pass (zero between launches)
  int* stop;            // q IHT stopped (||M g_G|| = 0)
  // task shapes
  int rp, nrc;          // rows per piece of an A^T pass, row chunks per tile
  int rpw, nrb;         // rows per W block (<= 128), W row blocks
  int TB, ngb;          // tiles per A^T task, A^T tasks per pass
  int TBW, ncw;         // tiles per W task, W column chunks
  int col0;             // index of this problem's first column in the launch
  int tasks_per_col;
  int wstride;          // floats per column of Wk and per column chunk of Wp (m R rounded
                        // up to 4: every block starts on a 16-byte boundary)
  int astride;          // floats per column of As (m rounded up to 4)
};

struct TaskQueue {
  unsigned long long* tasks;  // [total] descriptors
  int* seq;                   // [total] 1 once tasks[t] is published
  int* ctr;                   // [0] head, [1] tail, [2] next column to admit, [3] abort
  int total;                  // tasks of the launch
  int ncols;                  // columns of all problems
  int F;                      // columns in flight
  int nprob;
  const TaskProblem* probs;   // device copy
  unsigned long long* prof;   // optional kTaskProf counters (cycles summed over CTAs)
  unsigned long long wait_ns = 10ull * 1000 * 1000 * 1000;  // bound of every device wait
};
// Task-engine profile counters: consumer cycles waiting for a task, in W
// tasks, in A^T tasks, waiting for pieces (inside tasks), in the small steps
// after W / IHT / final passes, producer cycles waiting for a ticket,
// tasks run, small steps run; then the IHT step's parts: loads, mu, the
// HardThreshold, the next residual (or final LS), publishing.
constexpr int kTaskProf = 15;

// ---- task descriptors: k (32) | prob (6) | type (3) | phase (7) | block (16)
__host__ __device__ inline unsigned long long tdesc(int k, int prob, int type, int ph, int blk) {
  return (static_cast<unsigned long long>(static_cast<unsigned>(k)) << 32) |
         (static_cast<unsigned long long>(prob & 63) << 26) |
         (static_cast<unsigned long long>(type & 7) << 23) |
         (static_cast<unsigned long long>(ph & 127) << 16) |
         static_cast<unsigned long long>(blk & 0xFFFF);
}
__host__ __device__ inline int td_k(unsigned long long d) { return static_cast<int>(d >> 32); }
__host__ __device__ inline int td_prob(unsigned long long d) { return static_cast<int>((d >> 26) & 63); }
__host__ __device__ inline int td_type(unsigned long long d) { return static_cast<int>((d >> 23) & 7); }
__host__ __device__ inline int td_ph(unsigned long long d) { return static_cast<int>((d >> 16) & 127); }
__host__ __device__ inline int td_blk(unsigned long long d) { return static_cast<int>(d & 0xFFFF); }

// Pass `ph` of a column: its task type and number of tasks.
__host__ __device__ inline int phase_type(const TaskProblem& P, int ph) {
  const int te = P.tau_eff;
  if (P.mode == kModeLS) return kTaskW;
  if (P.mode == kModeInit) return ph < te ? kTaskG : kTaskF;
  return ph == 0 ? kTaskW : (ph <= te ? kTaskG : kTaskF);
}
__host__ __device__ inline int phase_tasks(const TaskProblem& P, int ph) {
  return phase_type(P, ph) == kTaskW ? P.nrb * P.ncw : P.ngb;
}
__host__ __device__ inline int last_phase(const TaskProblem& P) {
  if (P.mode == kModeLS) return 0;
  return P.mode == kModeInit ? P.tau_eff : P.tau_eff + 1;
}

struct TaskShape {  // launch configuration chosen on the host
  int stages, piece_bytes, grid, ctas_per_sm;
  size_t smem;
};
// The ring has exactly kTaskStages stages: A^T pieces go to the consumer
// warps round-robin, and with one stage per warp the previous use of a
// piece's stage is that same warp's previous piece (or a finished task's),
// so no warp ever waits on a barrier phase more than one ahead.
constexpr int kTaskStages = 8;
constexpr int kTileCols = 32;       // columns per tile of the slab layout
constexpr int kMaxTaskPieces = 128;  // pieces of one A^T task (tiles x row chunks)
// Fill the task fields of P (nrc, rpw, TB, ...) for target task bytes and
// rp rows per A^T piece.
void task_plan(TaskProblem& P, int R, size_t task_bytes, int rp);
// Rows per A^T piece that fit piece_cap bytes (0: not even 8 rows fit).
int task_rows_per_piece(int et, int m, int piece_cap);
size_t task_smem_bytes(int R, int et, int m_max, int ns_max, int rho_max, int stages,
                       int piece_bytes);
cudaError_t task_prepare(int R, int et, size_t smem);
int task_ctas_per_sm(int R, int et, size_t smem);
// Run one sweep (mode in each problem) of every problem of the table on
// stream s: reset the queue (publish the n_seed tasks of `seed`, the first
// passes of the first F columns; zero the ncols pass counters cnt_all that
// the problems' cnt point into), then the persistent launch.
cudaError_t task_launch_seeded(const TaskQueue& Q, const unsigned long long* seed, int n_seed,
                               int* cnt_all, int R, int et, const TaskShape& S, int m_max,
                               int ns_max, int rho_max, cudaStream_t s);

// ---- register-resident cluster engine (resident.cu) ---------------------------
// One thread-block cluster of CS CTAs per column at a time (persistent: the
// clusters take columns k = cluster, cluster + clusters, ...).  CTA c keeps
// the columns [128c, 128c + 128) of A_k in registers for the whole sweep of
// that column (W = A_k U, the IHT products and the final A^T pass read the
// registers, never memory); slabs of later columns are prefetched into L2 by
// bulk copies while the current column computes.  Partial products are
// combined through distributed shared memory.
//
// Layout of A_k ("register order"): column k is CS consecutive slabs; slab c
// holds the 4-column chunks ch = 0 .. nchc-1 of columns 4 (32c + ch) + e
// (e < 4), nchc = min(32, nch4 - 32c), nch4 = ceil(n/4); inside a slab, rows
// are taken in blocks of 32 (row i = 32p + l, l < 32; the last block has
// m_last = m - 32 (MR - 1) rows) and element (i, ch, e) is the float at
//   p * 128 nchc + ch * 4 Lp + 4 l + e,   Lp = 32 (p < MR - 1) or m_last,
// so that lane l of warp w loads its rows of chunk ch = 8 cc + w with one
// coalesced 16-byte load per row block.  Column k starts at float
// k * m * 4 nch4 and slab c at float 128 m c inside it (columns beyond n are
// zero).
constexpr int kResNT = 256;            // threads per CTA (8 warps)
constexpr int kResChunks = 32;         // 4-column chunks per CTA (4 per warp)
constexpr int kResCols = 4 * kResChunks;  // columns per CTA

struct ResArgs {
  int n, m, q, r, rho, mode, tau, CS, nch4;
  const float* A;       // register-order layout
  const float* y;       // q x m measurements seen by the sweep
  const float* U;       // n x r row-major
  int* S_idx;           // q x rho in/out (ascending)
  float* S_val;
  float* B;             // q x r
  float* H;             // q x n (ITER: h_k; INIT: L0 column)
  int* err;
  unsigned long long wait_ns;   // bound of every inter-CTA wait
  unsigned long long* prof;     // optional kResProf counters (SM cycles summed over CTAs)
};
// Resident-engine profile counters: cycles in the column set-up, the W
// pass, waiting in exchanges, the Gram/Cholesky, the IHT projection and A^T
// pass, the A g_G product, mu, the local HardThreshold, the candidate merge,
// the A s update, the LS and final pass; then the numbers of columns,
// exchanges, support changes and IHT sweeps.
constexpr int kResProf = 15;
// Rank widths and rows-per-lane the engine is compiled for.
__host__ __device__ inline int res_rpad(int r) { return r <= 2 ? 2 : r <= 6 ? r : 8; }
inline bool res_supported(int n, int m, int r, int rho, int et) {
  return et == 0 && r <= 8 && m >= 1 && m <= 192 && n <= 8 * kResCols && rho <= 32;
}
inline int res_cluster(int n) { return (((n + 3) / 4) + kResChunks - 1) / kResChunks; }
size_t res_smem_bytes(int R, int MR, int m, int rho, int CS);
cudaError_t res_prepare(int R, int MR);
// clusters of CS CTAs that can be resident at once (0: the shape cannot run)
int res_max_clusters(int R, int MR, int CS, size_t smem);
cudaError_t res_launch(const ResArgs& a, int nclusters, cudaStream_t s);
// row-major A (kc columns starting at k0, q x m x n) -> register-order layout
cudaError_t res_repack(const float* A_rowmajor, int n, int m, int k0, int kc, float* A_res,
                       cudaStream_t s);

// Global (column-reduced) steps (global_ops.cu).
// Row stride of the padded copy of U the sweep stages by TMA: r rounded up
// to one of the compiled widths.
__host__ __device__ inline int sweep_rpad(int r) {
  return r <= 2 ? 2 : r <= 6 ? r : r <= 8 ? 8 : r <= 10 ? 10 : r <= 12 ? 12 : 16;
}

struct GlobalWork {
  int n, q, r;
  float* Upad;       // (padded n) x rpad copy of U for the sweep (optional)
  int rpad;
  float* grad;       // n x r row-major
  double* part;      // partial r x r FP64 Grams: nblk x (r*r)
  double* small;     // scratch: [0,r*r) Rinv1, [r*r,2r*r) Rinv2, [2r*r] eta, ...
  float* Z;          // n x r scratch (U - eta grad, Q1)
  int nblk;          // blocks of the row-parallel kernels
  int ks = 1;        // k-splits of the column reductions (grad, subspace step)
  float* gsplit = nullptr;   // ks x n x r FP32 partial sums (ks > 1, or qc > 0)
  int qc = 0;        // columns per k-split (0: ceil(q / ks)); > 0 always splits
};
cudaError_t grad_reduce(const GlobalWork& g, const float* H, const float* Bk, cudaStream_t s);
// The k-split partial sums of grad_reduce alone (g.ks blocks of g.qc columns
// into g.gsplit), and the fixed-order sum of nb such n x r blocks into out.
cudaError_t grad_partials(const GlobalWork& g, const float* H, const float* Bk, cudaStream_t s);
cudaError_t sum_blocks(int n, int r, int nb, const float* parts, float* out, cudaStream_t s);
cudaError_t eta_from_grad(const GlobalWork& g, double c_eta, double* eta_dev, cudaStream_t s);
cudaError_t qr_step(const GlobalWork& g, float* U, const double* eta_dev, int* err,
                    cudaStream_t s);
cudaError_t cholqr2(const GlobalWork& g, const float* Zin, float* Uout, int* err,
                    cudaStream_t s);
cudaError_t project_cols(const GlobalWork& g, const float* H, const float* U, float* P,
                         cudaStream_t s);  // P(q x r) = H U  (H: q x n)
// ||(I - Uold Uold^T) Unew||_F^2 (FP64) into *out, D = Uold^T Unew into D_rr.
cudaError_t subspace_change(const GlobalWork& g, const float* Uold, const float* Unew,
                            double* D_rr, double* out, cudaStream_t s);
// Cholesky-QR2 of an n x r row-major FP32 matrix Z into Q with caller-given
// scratch: tmp (n*r floats), part (nblk*r*r doubles), rfac (2*r*r doubles),
// err (2 ints, zero on entry).  Blocks: qr_blocks(n).
int qr_blocks(int64_t n);
// Eigenvalues (descending) of the FP64 Gram P^T P of a rows x r FP32 matrix P
// into out[0..r): nblk row blocks, part holds nblk r x r partials.
cudaError_t ritz_values(int rows, int r, const float* P, double* part, int nblk, double* out,
                        cudaStream_t s);
// Z <- Z - Ua (Ua^T Z) for an n x r block Ua with orthonormal columns (g.n, g.r,
// g.part, g.nblk); D receives Ua^T Z (r x r FP64).
cudaError_t deflate(const GlobalWork& g, const float* Ua, float* Z, double* D, cudaStream_t s);
cudaError_t cholqr2_into(int n, int r, const float* Z, float* Q, float* tmp, double* part,
                         double* rfac, int* err, int nblk, cudaStream_t s);

cudaError_t subspace_overlap(const GlobalWork& g, const float* Ua, const float* Ub,
                             double* out_rr, cudaStream_t s);

}  // namespace lrs
