// C ABI of the solver (include/lrs.h): argument checks, the handle state
// machine, device memory of one problem, and the launch sequence of
// Algorithm 1 (initialisation, then GDmin iterations) on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <initializer_list>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lrs.h"
#include "lrs_internal.h"

using namespace lrs;

namespace lrs {
struct FourierSolver;
FourierSolver* fourier_create(int nx, int ny, int m, int q, int r, int rho, int tau0, int tau,
                              double c_eta, int power_iters, double power_tol, uint64_t seed,
                              cudaStream_t s, std::string* msg);
void fourier_destroy(FourierSolver* F);
int fourier_set_measurements(FourierSolver* F, const void* y, const void* mask, int mem_kind,
                             std::string* msg);
int fourier_init(FourierSolver* F, std::string* msg);
int fourier_iterate(FourierSolver* F, int iters, std::string* msg, cudaEvent_t* evs);
int fourier_get(FourierSolver* F, void* U, void* B, int* S_idx, void* S_val, int mem_kind);
int fourier_set_state(FourierSolver* F, const void* U, const void* B, const int* S_idx,
                      const void* S_val, int t, double eta, int mem_kind);
double fourier_eta(FourierSolver* F);
int fourier_t(FourierSolver* F);
int fourier_launches_per_iteration(FourierSolver* F);
int fourier_fused_qr(FourierSolver* F);
int fourier_prof_enable(FourierSolver* F);
int fourier_prof_read(FourierSolver* F, unsigned long long* out, int len);
}  // namespace lrs

namespace {

thread_local std::string g_last_error;

lrs_status fail(lrs_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

#define CUDA_TRY(expr)                                                              \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      return fail(e_ == cudaErrorMemoryAllocation ? LRS_ERR_OOM : LRS_ERR_CUDA,     \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));              \
    }                                                                               \
  } while (0)

enum State { kCreated = 0, kMeasured = 1, kInitialised = 2, kIterating = 3 };

constexpr int kThreads = 256;

}  // namespace

struct lrs_ctx {
  int64_t n = 0, m = 0, q = 0;
  int r = 0, rho_true = 0, rho = 0;
  lrs_op_kind kind = LRS_OP_GAUSSIAN;
  lrs_options opt{};
  cudaStream_t stream = nullptr;
  State state = kCreated;
  int t = 0;
  GaussLayout L{};
  int resident = 1;
  // device buffers
  void* A = nullptr;       // slab layout, element type L.et
  float* y = nullptr;      // q x m
  float* Aex = nullptr;    // low-precision forms: exact FP32 A_k, row-major q x m x n
  float* rscale = nullptr; // FP8 forms: q x m x (1 or 2) row scales
  float* ycorr = nullptr;  // low-precision forms: defect-corrected y (q x m)
  int last_refine = -1;    // iteration count t at the last refinement (-1: none since set-up)
  float* U = nullptr;      // n x r row-major
  float* Upad = nullptr;   // (cs*ns) x rpad row-major, zero padded (sweep input)
  float* Bk = nullptr;     // q x r
  int* S_idx = nullptr;    // q x rho
  float* S_val = nullptr;  // q x rho
  float* H = nullptr;      // q x n
  float* grad = nullptr;   // n x r
  float* Z = nullptr;      // n x r
  float* U2 = nullptr;     // n x r (subspace iteration)
  float* P = nullptr;      // q x r
  double* part = nullptr;  // nblk x r x r
  double* small = nullptr;
  double* eta = nullptr;   // device scalar
  int* err = nullptr;      // {code, column}
  float* Xref = nullptr;   // q x n (error log)
  double* errpart = nullptr;
  int ks = 1;                // k-splits of the column reductions
  int qc = 0;                // columns per k-split when fixed (grad_block)
  float* gsplit = nullptr;   // ks x n x r
  // column-sharded solves: this shard's partial sums and every shard's
  // (pinned host), and every shard's on the device
  float *rd_mine = nullptr, *rd_all = nullptr, *rd_dev = nullptr;
  unsigned long long* trace = nullptr;  // q x kTracePhases (profile = 2)
  int nblk = 0;
  int power_iters_done = 0;
  FourierSolver* F = nullptr;  // DFT2D_MASK operator
  // register-resident cluster engine (engine == 3)
  int res_CS = 0, res_ncl = 0;
  // persistent task engine (engine == 2)
  int engine = 1;
  TaskShape tshape{};
  TaskProblem tp[3]{};               // per sweep mode (INIT, LS, ITER)
  TaskProblem* dtp = nullptr;        // device copies [3]
  unsigned long long* dseed = nullptr;  // [3][F * first-pass tasks]
  int n_seed[3] = {0, 0, 0};
  size_t seed_stride = 0;
  int total[3] = {0, 0, 0};
  int tF = 0;                        // columns in flight
  int t_kib = 256;                   // KiB of A_k per task
  int t_ncw_max = 1;                 // W chunks the scratch holds
  int64_t t_total_max = 0;           // tasks the queue holds
  int tuned = 0;                     // autotuner ran (or its cache was used)
  int trp = 0;                       // rows per A^T piece
  float *tWk = nullptr, *tWp = nullptr, *tu = nullptr, *tg = nullptr, *tsupv = nullptr;
  float* tAs = nullptr;  // q x astride: A_k s_k (task engine)
  double* tGi = nullptr;
  int *tsupj = nullptr, *tnsup = nullptr, *tcnt = nullptr, *tstop = nullptr, *tseq = nullptr,
      *tctr = nullptr;
  unsigned long long* ttasks = nullptr;
  unsigned long long* tprof = nullptr;  // kTaskProf counters (profile = 2)
  // graphs of one steady-state iteration: [0] plain, [1] with the refinement
  // of the measurements (low-precision forms)
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  // phase timing (profile = 1): 4 events per iteration
  std::vector<cudaEvent_t> ev;
  double phase_ms[3] = {0, 0, 0};
  int64_t phase_iters = 0;
};

namespace {

GlobalWork gw(lrs_ctx* h) {
  GlobalWork g;
  g.n = static_cast<int>(h->n);
  g.q = static_cast<int>(h->q);
  g.r = h->r;
  g.grad = h->grad;
  g.part = h->part;
  g.small = h->small;
  g.Z = h->Z;
  g.nblk = h->nblk;
  g.Upad = h->Upad;
  g.rpad = sweep_rpad(h->r);
  g.ks = h->ks;
  g.gsplit = h->gsplit;
  g.qc = h->qc;
  return g;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

GaussLayout gauss_shape(const lrs_ctx* h, int cs, int stages) {
  GaussLayout L{};
  L.n = static_cast<int>(h->n);
  L.m = static_cast<int>(h->m);
  L.q = static_cast<int>(h->q);
  L.r = h->r;
  L.rho = h->rho;
  L.cs = cs;
  const int64_t w = (h->n + cs - 1) / cs;
  L.ns = static_cast<int>((w + 31) / 32 * 32);
  L.stages = stages;
  L.et = static_cast<int>(h->opt.a_dtype);
  return L;
}

bool shape_valid(const lrs_ctx* h, const GaussLayout& L) {
  return static_cast<int64_t>(L.cs - 1) * L.ns < h->n;
}

int max_smem_optin() {
  int max_optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return max_optin > 0 ? max_optin : 232448;
}

// Pick the cluster size (CTAs per column), the slab mode and the ring depth.
// Preference: a slab resident in shared memory with two CTAs per SM, then a
// streamed slab with the deepest ring that keeps two CTAs per SM, then any
// shape that fits one CTA per SM.  Options can force each choice.
void choose_layout(lrs_ctx* h) {
  const size_t two_per_sm = 113 * 1024, one_per_sm = static_cast<size_t>(max_smem_optin());
  const int cands[5] = {1, 2, 4, 8, 16};
  const int want_cs = h->opt.cluster, want_mode = h->opt.slab_mode, want_st = h->opt.stages;
  for (size_t lim : {two_per_sm, one_per_sm}) {
    for (int cs : cands) {
      if (want_cs && cs != want_cs) continue;
      if (want_mode != 2) {  // resident
        GaussLayout L = gauss_shape(h, cs, 1);
        if (shape_valid(h, L) && sweep_smem_bytes(L, 1, 0) <= lim) {
          h->L = L;
          h->resident = 1;
          return;
        }
      }
      if (want_mode != 1) {  // streamed
        for (int st : {4, 3, 2}) {
          if (want_st && st != want_st) continue;
          GaussLayout L = gauss_shape(h, cs, st);
          if (shape_valid(h, L) && sweep_smem_bytes(L, 0, 0) <= lim) {
            h->L = L;
            h->resident = 0;
            return;
          }
        }
      }
    }
  }
  h->L = gauss_shape(h, want_cs ? want_cs : 16, 2);
  h->resident = 0;
}

// Row-major float A_k of columns k0 .. k0 + kc - 1 (device) into the
// engine's layout.
cudaError_t repack_a(lrs_ctx* h, const float* src, int64_t k0, int64_t kc) {
  if (h->engine == 3)
    return res_repack(src, static_cast<int>(h->n), static_cast<int>(h->m), static_cast<int>(k0),
                      static_cast<int>(kc), static_cast<float*>(h->A), h->stream);
  return repack_gauss(h->L, src, static_cast<int>(k0), static_cast<int>(kc), h->A, nullptr,
                      h->stream);
}

lrs_status check_device_error(lrs_ctx* h, const char* where) {
  int e[2] = {0, 0};
  CUDA_TRY(cudaMemcpyAsync(e, h->err, sizeof(e), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (e[0] == 0) return LRS_OK;
  CUDA_TRY(cudaMemsetAsync(h->err, 0, 2 * sizeof(int), h->stream));
  const char* what = e[0] == kErrNotSPD  ? "r x r Gram matrix not positive definite"
                     : e[0] == kErrNaN   ? "NaN/Inf in the iteration"
                     : e[0] == kErrTimeout ? "bounded device wait expired"
                                           : "device error";
  std::string msg = std::string(where) + ": " + what;
  if (e[1] >= 0) msg += " (column " + std::to_string(e[1]) + ")";
  return fail(e[0] == kErrTimeout ? LRS_ERR_TIMEOUT : LRS_ERR_NUMERICAL, msg);
}

// Bound of every device-side wait of the task and resident engines.
unsigned long long wait_bound_ns(const lrs_ctx* h) {
  return static_cast<unsigned long long>(h->opt.wait_ms > 0 ? h->opt.wait_ms : 10000) * 1000000ull;
}

lrs_status launch_sweep(lrs_ctx* h, int mode, int tau) {
  if (h->engine == 3) {
    ResArgs a{};
    a.n = static_cast<int>(h->n);
    a.m = static_cast<int>(h->m);
    a.q = static_cast<int>(h->q);
    a.r = h->r;
    a.rho = h->rho;
    a.mode = mode;
    a.tau = tau;
    a.CS = h->res_CS;
    a.nch4 = static_cast<int>((h->n + 3) / 4);
    a.A = static_cast<const float*>(h->A);
    a.y = h->y;
    a.U = h->U;
    a.S_idx = h->S_idx;
    a.S_val = h->S_val;
    a.B = h->Bk;
    a.H = h->H;
    a.err = h->err;
    a.wait_ns = wait_bound_ns(h);
    a.prof = (h->opt.profile == 2 && mode == kModeIter) ? h->tprof : nullptr;
    CUDA_TRY(res_launch(a, h->res_ncl, h->stream));
    return LRS_OK;
  }
  if (h->engine == 2) {
    TaskQueue Q{};
    Q.tasks = h->ttasks;
    Q.seq = h->tseq;
    Q.ctr = h->tctr;
    // test_withhold: one ticket more than the launch's tasks, never published
    // (room for it is allocated), so the wait for it runs out
    Q.total = h->total[mode] + (h->opt.test_withhold ? 1 : 0);
    Q.ncols = static_cast<int>(h->q);
    Q.wait_ns = wait_bound_ns(h);
    Q.F = h->tF;
    Q.nprob = 1;
    Q.probs = h->dtp + mode;
    Q.prof = (h->opt.profile == 2 && mode == kModeIter) ? h->tprof : nullptr;
    CUDA_TRY(task_launch_seeded(Q, h->dseed + static_cast<size_t>(mode) * h->seed_stride,
                                h->n_seed[mode], h->tcnt, sweep_rpad(h->r), h->L.et, h->tshape,
                                h->L.m, h->L.ns, h->rho, h->stream));
    (void)tau;
    return LRS_OK;
  }
  SweepArgs a{};
  a.L = h->L;
  a.mode = mode;
  a.tau = tau;
  a.A = h->A;
  a.y = (mode == kModeIter && h->L.et != 0) ? h->ycorr : h->y;
  a.rscale = h->rscale;
  a.U = h->U;
  a.Upad = h->Upad;
  a.S_idx = h->S_idx;
  a.S_val = h->S_val;
  a.B = h->Bk;
  a.H = h->H;
  a.err = h->err;
  a.resident = h->resident;
  a.trace = (h->opt.profile == 2 && mode == kModeIter) ? h->trace : nullptr;
  CUDA_TRY(sweep_launch(a, kThreads, h->stream));
  return LRS_OK;
}

lrs_status column_reduce(lrs_ctx* h, const GlobalWork& g, const float* H, const float* Bk);

// One GDmin iteration (Algorithm 1): sweep, gradient, eta at t = 1, QR.
// With `evs` (4 events) the phase boundaries are recorded on the stream.
// Low-precision forms of A_k first refresh the defect-corrected measurements
// when `refine` is set (counted in the sweep phase).
lrs_status enqueue_iteration(lrs_ctx* h, bool first, cudaEvent_t* evs = nullptr,
                             bool refine = false) {
  if (evs) CUDA_TRY(cudaEventRecord(evs[0], h->stream));
  if (refine)
    CUDA_TRY(refine_residual(h->L, h->Aex, h->A, h->rscale, h->U, h->Bk, h->S_idx, h->S_val,
                             h->y, h->ycorr, h->H, h->stream));
  lrs_status st = launch_sweep(h, kModeIter, h->opt.tau);
  if (st != LRS_OK) return st;
  if (evs) CUDA_TRY(cudaEventRecord(evs[1], h->stream));
  GlobalWork g = gw(h);
  st = column_reduce(h, g, h->H, h->Bk);
  if (st != LRS_OK) return st;
  if (evs) CUDA_TRY(cudaEventRecord(evs[2], h->stream));
  if (first) CUDA_TRY(eta_from_grad(g, h->opt.c_eta, h->eta, h->stream));
  CUDA_TRY(qr_step(g, h->U, h->eta, h->err, h->stream));
  if (evs) CUDA_TRY(cudaEventRecord(evs[3], h->stream));
  return LRS_OK;
}

__global__ void err_kernel(int n, int q, int r, int rho, const float* U, const float* Bk,
                           const int* S_idx, const float* S_val, const float* Xref,
                           double* out) {
  __shared__ double sd[8], sr[8];
  const int k = blockIdx.x;
  double d2 = 0.0, r2 = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    float x = 0.f;
    for (int l = 0; l < r; ++l) x = fmaf(U[static_cast<size_t>(j) * r + l], Bk[static_cast<size_t>(k) * r + l], x);
    for (int e = 0; e < rho; ++e)
      if (S_idx[static_cast<size_t>(k) * rho + e] == j) x += S_val[static_cast<size_t>(k) * rho + e];
    const double xr = Xref[static_cast<size_t>(k) * n + j];
    d2 += (x - xr) * (x - xr);
    r2 += xr * xr;
  }
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sd[threadIdx.x >> 5] = d2;
    sr[threadIdx.x >> 5] = r2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sd[w]; b += sr[w]; }
    out[2 * k] = a;
    out[2 * k + 1] = b;
  }
}

lrs_status error_now(lrs_ctx* h, double* out) {
  err_kernel<<<static_cast<unsigned>(h->q), 256, 0, h->stream>>>(
      static_cast<int>(h->n), static_cast<int>(h->q), h->r, h->rho, h->U, h->Bk, h->S_idx,
      h->S_val, h->Xref, h->errpart);
  CUDA_TRY(cudaGetLastError());
  std::vector<double> p(2 * h->q);
  CUDA_TRY(cudaMemcpyAsync(p.data(), h->errpart, p.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  double a = 0, b = 0;
  for (int64_t k = 0; k < h->q; ++k) { a += p[2 * k]; b += p[2 * k + 1]; }
  *out = b > 0 ? std::sqrt(a / b) : 0.0;
  return LRS_OK;
}

__global__ void pad_rows_kernel(const float* in, float* out, int rows, int cols, int ldo) {
  // out[r*ldo + c] = in[r*cols + c]
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < rows * cols) {
    const int rr = t / cols, cc = t - rr * cols;
    out[static_cast<size_t>(rr) * ldo + cc] = in[t];
  }
}

__global__ void transpose_kernel(const float* in, float* out, int rows, int cols) {
  // out[c*rows + r] = in[r*cols + c]
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < rows * cols) {
    const int rr = t / cols, cc = t - rr * cols;
    out[static_cast<size_t>(cc) * rows + rr] = in[t];
  }
}

// X = U B + S (Algorithm 1, Output: x_k = U b_k + s_k), one block per column
// k.  U n x r column-major, B r x q column-major, S rho x q (indices, values);
// X n x q column-major.  CT = 1 real float, 2 interleaved complex64.
template <int CT>
__global__ void assemble_x_kernel(int n, int q, int r, int rho, const float* U, const float* B,
                                  const int* S_idx, const float* S_val, float* X) {
  const int k = blockIdx.x;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    float re = 0.f, im = 0.f;
    for (int l = 0; l < r; ++l) {
      const size_t iu = static_cast<size_t>(l) * n + j, ib = static_cast<size_t>(k) * r + l;
      if (CT == 1) {
        re = fmaf(U[iu], B[ib], re);
      } else {
        const float ur = U[2 * iu], ui = U[2 * iu + 1], br = B[2 * ib], bi = B[2 * ib + 1];
        re = fmaf(ur, br, fmaf(-ui, bi, re));
        im = fmaf(ur, bi, fmaf(ui, br, im));
      }
    }
    const size_t ix = static_cast<size_t>(k) * n + j;
    if (CT == 1) {
      X[ix] = re;
    } else {
      X[2 * ix] = re;
      X[2 * ix + 1] = im;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rho; e += blockDim.x) {   // indices of a column are distinct
    const int j = S_idx[static_cast<size_t>(k) * rho + e];
    const size_t ix = static_cast<size_t>(k) * n + j, is = static_cast<size_t>(k) * rho + e;
    if (CT == 1) {
      X[ix] += S_val[is];
    } else {
      X[2 * ix] += S_val[2 * is];
      X[2 * ix + 1] += S_val[2 * is + 1];
    }
  }
}

// Deterministic start of the subspace iteration: splitmix64 + Box-Muller.
std::vector<float> start_block(int64_t n, int r, uint64_t seed) {
  std::vector<float> v(static_cast<size_t>(n) * r);
  uint64_t s = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  auto next = [&]() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (size_t i = 0; i < v.size(); i += 2) {
    const double u1 = ((next() >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = (next() >> 11) * 0x1.0p-53;
    const double rad = std::sqrt(-2.0 * std::log(u1));
    v[i] = static_cast<float>(rad * std::cos(6.283185307179586 * u2));
    if (i + 1 < v.size()) v[i + 1] = static_cast<float>(rad * std::sin(6.283185307179586 * u2));
  }
  return v;
}

// Device memory of a handle: stream-ordered (cudaMallocAsync / cudaFreeAsync on
// the handle's stream), so that creating or destroying one handle never waits
// for work that other handles run on other streams.
template <typename T>
lrs_status dalloc(T** p, size_t count, cudaStream_t s) {
  if (count == 0) count = 1;
  CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(p), count * sizeof(T), s));
  return LRS_OK;
}

void free_all(lrs_ctx* h) {
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  h->ev.clear();
  for (int g = 0; g < 2; ++g) {
    if (h->gexec[g]) cudaGraphExecDestroy(h->gexec[g]);
    if (h->graph[g]) cudaGraphDestroy(h->graph[g]);
    h->gexec[g] = nullptr;
    h->graph[g] = nullptr;
  }
  void* ps2[] = {h->dtp, h->dseed, h->tWk, h->tWp, h->tu, h->tg, h->tsupv, h->tGi, h->tsupj, h->tAs,
                 h->tnsup, h->tcnt, h->tstop, h->tseq, h->tctr, h->ttasks, h->tprof};
  for (void* p : ps2)
    if (p) cudaFreeAsync(p, h->stream);
  void* ps[] = {h->gsplit, h->A, h->y, h->Aex, h->rscale, h->ycorr, h->U, h->Upad, h->Bk, h->S_idx, h->S_val, h->H, h->grad, h->Z,
                h->U2, h->P, h->part, h->small, h->eta, h->err, h->Xref, h->errpart, h->trace,
                h->rd_dev};
  for (void* p : ps)
    if (p) cudaFreeAsync(p, h->stream);
  if (h->rd_mine) cudaFreeHost(h->rd_mine);
  if (h->rd_all) cudaFreeHost(h->rd_all);
  h->rd_mine = h->rd_all = nullptr;
}

// ---- autotuner: shapes per problem, cached for the process -----------------------
struct TuneKey {
  int64_t n, m, q;
  int r, rho, et, grid;
  bool operator<(const TuneKey& o) const {
    return std::tie(n, m, q, r, rho, et, grid) < std::tie(o.n, o.m, o.q, o.r, o.rho, o.et, o.grid);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;  // -> (KiB per task, columns in flight)

TuneKey tune_key(const lrs_ctx* h) {
  return TuneKey{h->n, h->m, h->q, h->r, h->rho, h->L.et, h->tshape.grid};
}

// Task engine shapes: task sizes, ring stages (two CTAs per SM when they
// fit), columns in flight.  False when no shape fits shared memory.
bool plan_task_engine(lrs_ctx* h, int nsm) {
  const int R = sweep_rpad(h->r), et = h->L.et;
  const size_t task_bytes = static_cast<size_t>(h->opt.task_kib > 0 ? h->opt.task_kib : 256) * 1024;
  // piece height from the shared-memory budget: two CTAs per SM if 8 rows fit
  const size_t fixed = task_smem_bytes(R, et, h->L.m, h->L.ns, h->rho, 0, 0);
  // two CTAs per SM by default (three, which the registers allow for r <= 6,
  // only on request: their pieces get too short), else one
  const size_t optin = static_cast<size_t>(max_smem_optin());
  const int cps_max = (R <= 6 && h->opt.ctas_per_sm == 3) ? 3 : 2;
  int rp = 0, cps = 0;
  for (int c = cps_max; c >= 1 && !rp; --c) {
    if (h->opt.ctas_per_sm > 0 && c != h->opt.ctas_per_sm) continue;
    const size_t budget = c == 1 ? optin : (228 * 1024) / c - 1024;
    if (budget <= fixed + 64) continue;
    const size_t per_stage = (budget - fixed) / kTaskStages;
    const long cap = static_cast<long>(per_stage) - static_cast<long>(kTileCols) * R * 4 - 16;
    if (cap <= 0) continue;
    rp = task_rows_per_piece(et, h->L.m, static_cast<int>(cap));
    cps = c;
  }
  if (!rp) return false;
  TaskProblem P{};
  P.L = h->L;
  P.mode = kModeIter;
  P.tau_eff = h->rho > 0 ? h->opt.tau : 0;
  task_plan(P, R, task_bytes, rp);
  if (P.nrc > kMaxTaskPieces) return false;  // rows too tall for one A^T task
  const int pbytes = rp * kTileCols * elem_bytes(et);
  h->tshape.stages = kTaskStages;
  h->tshape.piece_bytes = pbytes;
  h->tshape.smem = task_smem_bytes(R, et, h->L.m, h->L.ns, h->rho, kTaskStages, pbytes);
  h->trp = rp;
  const int grid = cps * nsm;
  // columns in flight: all of them unless asked otherwise (the small steps
  // of a column are latency-bound, so the more columns advance at once the
  // better the grid stays busy; measured on the n=1000, q=1000, m=150 case)
  h->tshape.grid = grid;
  const int F = h->opt.inflight > 0 ? h->opt.inflight : static_cast<int>(h->q);
  h->tF = static_cast<int>(std::min<int64_t>(F, h->q));
  h->t_kib = h->opt.task_kib > 0 ? h->opt.task_kib : 256;
  if (h->opt.task_kib <= 0 && h->opt.inflight <= 0) {  // a shape the autotuner chose before
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(tune_key(h));
    if (it != g_tune_cache.end()) {
      h->t_kib = it->second.first;
      h->tF = it->second.second;
      h->tuned = 1;
    }
  }
  return true;
}

// Column reductions (gradient, subspace step) split over k so that about
// four blocks per SM work on them; FP32 and FP64 partial buffers.
lrs_status alloc_split(lrs_ctx* h, int nsm) {
  const int64_t jb = (h->n + 31) / 32;
  int ks = static_cast<int>(std::max<int64_t>(1, (4 * nsm + jb - 1) / jb));
  ks = std::min<int>(ks, 32);
  ks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ks, h->q / 8)));
  if (h->opt.grad_block > 0) {  // fixed blocks of grad_block columns
    h->qc = h->opt.grad_block;
    ks = static_cast<int>((h->q + h->qc - 1) / h->qc);
  }
  h->ks = ks;
  if (ks <= 1 && h->qc == 0) return LRS_OK;
  lrs_status st = LRS_OK;
  const size_t blk = static_cast<size_t>(h->n) * h->r;
  if ((st = dalloc(&h->gsplit, ks * blk, h->stream))) return st;
  if (h->opt.reduce) {
    const size_t cap = static_cast<size_t>(h->opt.reduce_cap) * blk;
    CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&h->rd_mine), ks * blk * sizeof(float)));
    CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&h->rd_all), cap * sizeof(float)));
    if ((st = dalloc(&h->rd_dev, cap, h->stream))) return st;
  }
  return LRS_OK;
}

// A column reduction (Section II-A gradient, or the subspace step of the
// initialisation): sum_k H[k]^T Bk[k] into g.grad (n x g.r).  With a reducer
// (column-sharded solve) this shard's k-split partials go to the host, the
// reducer returns every shard's in column order, and their fixed-order sum
// is formed on the device.
lrs_status column_reduce(lrs_ctx* h, const GlobalWork& g, const float* H, const float* Bk) {
  if (!h->opt.reduce) {
    CUDA_TRY(grad_reduce(g, H, Bk, h->stream));
    return LRS_OK;
  }
  const size_t blk = static_cast<size_t>(h->n) * g.r;
  CUDA_TRY(grad_partials(g, H, Bk, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->rd_mine, g.gsplit, g.ks * blk * sizeof(float),
                           cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  const int nb = h->opt.reduce(h->opt.reduce_ctx, h->rd_mine, g.ks, h->n, g.r, h->rd_all,
                               h->opt.reduce_cap);
  if (nb < 1 || nb > h->opt.reduce_cap)
    return fail(LRS_ERR_ARG, "column reduction: the reducer returned " + std::to_string(nb) +
                                 " blocks (capacity " + std::to_string(h->opt.reduce_cap) + ")");
  CUDA_TRY(cudaMemcpyAsync(h->rd_dev, h->rd_all, nb * blk * sizeof(float), cudaMemcpyHostToDevice,
                           h->stream));
  CUDA_TRY(sum_blocks(static_cast<int>(h->n), g.r, nb, h->rd_dev, g.grad, h->stream));
  return LRS_OK;
}

// Task sizes the autotuner tries (KiB of A_k per task).
constexpr int kTuneKib[4] = {128, 256, 512, 1024};

// Problem tables (one per sweep mode) and seeds for `task_kib` KiB per task
// and F columns in flight, uploaded to the device.
lrs_status plan_tables(lrs_ctx* h, int task_kib, int F) {
  const int R = sweep_rpad(h->r);
  const size_t task_bytes = static_cast<size_t>(task_kib) * 1024;
  F = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(F, h->q)));
  for (int mode = 0; mode < 3; ++mode) {
    TaskProblem& P = h->tp[mode];
    P = TaskProblem{};
    P.L = h->L;
    P.mode = mode;
    P.tau_eff = h->rho == 0 ? 0 : (mode == kModeInit ? h->opt.tau0 : mode == kModeIter ? h->opt.tau : 0);
    task_plan(P, R, task_bytes, h->trp);
    if (P.ncw > h->t_ncw_max) return fail(LRS_ERR_STATE, "task engine: W chunks exceed the scratch");
    P.A = h->A;
    P.rscale = h->rscale;
    P.y = (mode == kModeIter && h->L.et != 0) ? h->ycorr : h->y;
    P.Upad = h->Upad;
    P.S_idx = h->S_idx;
    P.S_val = h->S_val;
    P.B = h->Bk;
    P.H = h->H;
    P.err = h->err;
    P.Wk = h->tWk;
    P.Wp = h->tWp;
    P.Gi = h->tGi;
    P.uvec = h->tu;
    P.As = h->tAs;
    P.g = h->tg;
    P.supj = h->tsupj;
    P.supv = h->tsupv;
    P.nsup = h->tnsup;
    P.cnt = h->tcnt;
    P.stop = h->tstop;
    P.col0 = 0;
    const int64_t tot = static_cast<int64_t>(P.tasks_per_col) * h->q;
    if (tot > h->t_total_max) return fail(LRS_ERR_STATE, "task engine: tasks exceed the queue");
    h->total[mode] = static_cast<int>(tot);
    h->n_seed[mode] = F * phase_tasks(P, 0);
    if (static_cast<size_t>(h->n_seed[mode]) > h->seed_stride)
      return fail(LRS_ERR_STATE, "task engine: seed exceeds its buffer");
  }
  std::vector<unsigned long long> seed(3 * h->seed_stride, 0ull);
  for (int mode = 0; mode < 3; ++mode) {
    const TaskProblem& P = h->tp[mode];
    const int n0 = phase_tasks(P, 0);
    for (int c = 0; c < F; ++c)
      for (int i = 0; i < n0; ++i)
        seed[mode * h->seed_stride + static_cast<size_t>(c) * n0 + i] =
            tdesc(c, 0, phase_type(P, 0), 0, i);
  }
  CUDA_TRY(cudaMemcpyAsync(h->dseed, seed.data(), seed.size() * 8, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->dtp, h->tp, sizeof(h->tp), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));  // the host tables may go once this returns
  h->tF = F;
  h->t_kib = task_kib;
  return LRS_OK;
}

// Scratch, queue and seeds sized for every shape the autotuner may pick
// (the smallest tasks and all q columns in flight), then the tables.
lrs_status alloc_task_engine(lrs_ctx* h) {
  const int R = sweep_rpad(h->r), m = static_cast<int>(h->m);
  const size_t q = static_cast<size_t>(h->q), ns = h->L.ns, rho1 = std::max(1, h->rho);
  const int kib = h->t_kib;
  const int kib_min = std::min(kib, kTuneKib[0]);
  int ncw_max = 1, n0_max = 1;
  int64_t total_max = 0;
  const size_t wstride = static_cast<size_t>((m * R + 3) & ~3);  // as task_plan sets it
  for (int mode = 0; mode < 3; ++mode) {
    TaskProblem P{};
    P.L = h->L;
    P.mode = mode;
    P.tau_eff = h->rho == 0 ? 0 : (mode == kModeInit ? h->opt.tau0 : mode == kModeIter ? h->opt.tau : 0);
    task_plan(P, R, static_cast<size_t>(kib_min) * 1024, h->trp);
    ncw_max = std::max(ncw_max, P.ncw);
    n0_max = std::max(n0_max, phase_tasks(P, 0));
    total_max = std::max<int64_t>(total_max, static_cast<int64_t>(P.tasks_per_col) * h->q);
  }
  if (total_max >= (int64_t(1) << 31)) return fail(LRS_ERR_UNSUPPORTED, "task engine: too many tasks");
  h->t_ncw_max = ncw_max;
  h->t_total_max = total_max;
  h->seed_stride = q * static_cast<size_t>(n0_max);
  lrs_status st = LRS_OK;
  if ((st = dalloc(&h->tWk, q * wstride, h->stream)) || (st = dalloc(&h->tWp, q * ncw_max * wstride, h->stream)) ||
      (st = dalloc(&h->tGi, q * 16 * 16, h->stream)) || (st = dalloc(&h->tu, q * m, h->stream)) ||
      (st = dalloc(&h->tAs, q * static_cast<size_t>((m + 3) & ~3), h->stream)) ||
      (st = dalloc(&h->tg, q * ns, h->stream)) || (st = dalloc(&h->tsupj, q * rho1, h->stream)) ||
      (st = dalloc(&h->tsupv, q * rho1, h->stream)) || (st = dalloc(&h->tnsup, q, h->stream)) ||
      (st = dalloc(&h->tcnt, q, h->stream)) || (st = dalloc(&h->tstop, q, h->stream)) || (st = dalloc(&h->tctr, 4, h->stream)) ||
      (st = dalloc(&h->dtp, 3, h->stream)) || (st = dalloc(&h->tprof, 16, h->stream)) ||
      (st = dalloc(&h->ttasks, static_cast<size_t>(total_max) + 1, h->stream)) ||
      (st = dalloc(&h->tseq, static_cast<size_t>(total_max) + 1, h->stream)) ||
      (st = dalloc(&h->dseed, 3 * h->seed_stride, h->stream)))
    return st;
  CUDA_TRY(cudaMemsetAsync(h->tprof, 0, 16 * sizeof(unsigned long long), h->stream));
  CUDA_TRY(cudaMemsetAsync(h->tcnt, 0, q * sizeof(int), h->stream));
  CUDA_TRY(cudaMemsetAsync(h->tAs, 0, q * static_cast<size_t>((m + 3) & ~3) * sizeof(float), h->stream));
  CUDA_TRY(cudaMemsetAsync(h->tnsup, 0, q * sizeof(int), h->stream));
  CUDA_TRY(cudaMemsetAsync(h->tstop, 0, q * sizeof(int), h->stream));
  return plan_tables(h, kib, h->tF);
}

}  // namespace

extern "C" {

const char* lrs_last_error(void) { return g_last_error.c_str(); }

lrs_status lrs_create(int64_t n, int64_t m, int64_t q, int32_t r, int32_t rho, lrs_op_kind kind,
                      const lrs_options* opt, lrs_t* out) {
  if (!out) return fail(LRS_ERR_ARG, "lrs_create: out is NULL");
  *out = nullptr;
  if (n < 1 || m < 1 || q < 1) return fail(LRS_ERR_ARG, "lrs_create: n, m, q must be >= 1");
  if (r < 1 || r > 16 || r > std::min(m, n))
    return fail(LRS_ERR_ARG, "lrs_create: need 1 <= r <= min(16, m, n)");
  if (rho < 0 || rho > n) return fail(LRS_ERR_ARG, "lrs_create: need 0 <= rho <= n");
  if (n >= (int64_t(1) << 30) || m >= (int64_t(1) << 30) || q >= (int64_t(1) << 30))
    return fail(LRS_ERR_ARG, "lrs_create: sizes must be < 2^30");
  if (kind != LRS_OP_GAUSSIAN && kind != LRS_OP_DFT2D_MASK)
    return fail(LRS_ERR_ARG, "lrs_create: unknown operator kind");
  lrs_options o{};
  if (opt) o = *opt;
  if (kind == LRS_OP_DFT2D_MASK) {
    if (o.nx <= 0 || o.ny <= 0 || int64_t(o.nx) * o.ny != n)
      return fail(LRS_ERR_ARG, "lrs_create: DFT frames need nx, ny > 0 with nx*ny = n");
    if ((!is_pow2(o.nx) || !is_pow2(o.ny)) && n > 4096)
      return fail(LRS_ERR_ARG,
                  "lrs_create: DFT frames need nx, ny powers of two, or nx*ny <= 4096");
    if (m > n) return fail(LRS_ERR_ARG, "lrs_create: DFT needs m <= n");
  }
  if (o.tau0 < 0 || o.tau < 0 || o.T < 0 || o.rho_max < 0 || o.c_eta < 0 || o.cluster < 0 ||
      o.power_iters < 0 || o.refine_every < 0 || o.grid < 0 || o.wait_ms < 0 || o.engine < 0 ||
      o.engine > 3 || o.grad_block < 0 || o.reduce_cap < 0)
    return fail(LRS_ERR_ARG, "lrs_create: negative option");
  if (o.reduce) {
    if (kind != LRS_OP_GAUSSIAN)
      return fail(LRS_ERR_UNSUPPORTED, "lrs_create: column-sharded solves take Gaussian operators");
    if (o.grad_block <= 0 || o.use_graph || o.autotune)
      return fail(LRS_ERR_ARG, "lrs_create: a reducer needs grad_block > 0, use_graph = 0, autotune = 0");
    if (int64_t(o.reduce_cap) < (q + o.grad_block - 1) / o.grad_block)
      return fail(LRS_ERR_ARG, "lrs_create: reduce_cap below this shard's own partial blocks");
  }
  if (o.cluster != 0 && o.cluster != 1 && o.cluster != 2 && o.cluster != 4 && o.cluster != 8 &&
      o.cluster != 16)
    return fail(LRS_ERR_ARG, "lrs_create: cluster must be 0, 1, 2, 4, 8 or 16");
  if (o.slab_mode < 0 || o.slab_mode > 2 || o.stages < 0 || o.stages > 16)
    return fail(LRS_ERR_ARG, "lrs_create: slab_mode in 0..2, stages in 0..16");
  if (o.a_dtype < LRS_A_FP32 || o.a_dtype > LRS_A_FP8_HILO)
    return fail(LRS_ERR_ARG, "lrs_create: unknown a_dtype");
  if (kind == LRS_OP_DFT2D_MASK && o.a_dtype != LRS_A_FP32)
    return fail(LRS_ERR_ARG, "lrs_create: a_dtype applies to the Gaussian operator only");
  if (o.tau0 == 0) o.tau0 = 10;
  if (o.tau == 0) o.tau = 3;
  if (o.T == 0) o.T = 200;
  if (o.c_eta == 0) o.c_eta = 0.14;
  if (o.rho_max == 0) o.rho_max = rho;
  if (o.rho_max > n) return fail(LRS_ERR_ARG, "lrs_create: rho_max > n");
  if (o.power_iters == 0) o.power_iters = 1000;
  if (o.power_tol == 0) o.power_tol = 1e-6;
  if (o.refine_every == 0) o.refine_every = 8;

  if (kind == LRS_OP_DFT2D_MASK) {
    lrs_ctx* h = new lrs_ctx();
    h->n = n;
    h->m = m;
    h->q = q;
    h->r = r;
    h->rho_true = rho;
    h->rho = o.rho_max;
    h->kind = kind;
    h->opt = o;
    h->stream = static_cast<cudaStream_t>(o.stream);
    std::string msg;
    h->F = fourier_create(o.nx, o.ny, static_cast<int>(m), static_cast<int>(q), r, o.rho_max, o.tau0,
                          o.tau, o.c_eta, o.power_iters, o.power_tol, o.seed, h->stream, &msg);
    if (!h->F || !msg.empty()) {
      const lrs_status st = h->F ? LRS_ERR_OOM : LRS_ERR_UNSUPPORTED;
      if (h->F) fourier_destroy(h->F);
      delete h;
      return fail(st, "lrs_create: " + msg);
    }
    if (o.profile == 2) {
      const int pst = fourier_prof_enable(h->F);
      if (pst) {
        fourier_destroy(h->F);
        delete h;
        return fail(static_cast<lrs_status>(pst), "lrs_create: profile counters");
      }
    }
    *out = h;
    return LRS_OK;
  }
  lrs_ctx* h = new lrs_ctx();
  h->n = n;
  h->m = m;
  h->q = q;
  h->r = r;
  h->rho_true = rho;
  h->rho = o.rho_max;
  h->kind = kind;
  h->opt = o;
  h->stream = static_cast<cudaStream_t>(o.stream);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (nsm <= 0) nsm = 148;
  // engine: the task engine unless the cluster sweep is asked for (or the
  // task engine has no shape and the cluster sweep has one)
  h->engine = o.engine == 1 ? 1 : (o.engine == 3 ? 3 : 2);
  if (h->engine == 3 && !res_supported(static_cast<int>(n), static_cast<int>(m), r, o.rho_max,
                                       static_cast<int>(o.a_dtype))) {
    delete h;
    return fail(LRS_ERR_UNSUPPORTED,
                "lrs_create: the resident engine needs float32 A_k, r <= 8, m <= 192, n <= 1024, "
                "rho_max <= 32");
  }
  if (h->engine == 3) {
    h->L = gauss_shape(h, 1, 0);   // descriptive only: the engine keeps its own layout
    h->res_CS = res_cluster(static_cast<int>(n));
  }
  if (h->engine == 2) {
    h->L = gauss_shape(h, 1, 0);
    if (!plan_task_engine(h, nsm)) {
      if (o.engine == 2 || m > 512) {
        delete h;
        return fail(LRS_ERR_UNSUPPORTED, "lrs_create: no task-engine shape fits shared memory");
      }
      h->engine = 1;
    }
  }
  if (h->engine == 1) {
    if (m > 512) {
      delete h;
      return fail(LRS_ERR_UNSUPPORTED, "lrs_create: the cluster sweep handles m <= 512");
    }
    choose_layout(h);
    if (!shape_valid(h, h->L) ||
        sweep_smem_bytes(h->L, h->resident, 0) > static_cast<size_t>(max_smem_optin())) {
      delete h;
      return fail(LRS_ERR_ARG, "lrs_create: no sweep shape fits (cluster/slab options)");
    }
  }
  h->nblk = std::max(1, std::min<int>(nsm, static_cast<int>((n + 63) / 64)));
  const size_t per_col = h->engine == 3
                             ? static_cast<size_t>(m) * 16 * static_cast<size_t>((n + 3) / 4)
                             : static_cast<size_t>(h->L.cs) * h->L.m * h->L.ns * elem_bytes(h->L.et);
  lrs_status st = LRS_OK;
  const size_t upad_n = static_cast<size_t>(h->L.cs) * h->L.ns * sweep_rpad(r);
  const int lowp = h->L.et != 0, per_row = h->L.et == 3 ? 2 : 1;
  if ((st = dalloc(reinterpret_cast<unsigned char**>(&h->A), per_col * q, h->stream)) ||
      (st = dalloc(&h->y, size_t(m) * q, h->stream)) ||
      (lowp && (st = dalloc(&h->Aex, size_t(m) * n * q, h->stream))) ||
      (lowp && (st = dalloc(&h->ycorr, size_t(m) * q, h->stream))) ||
      (h->L.et >= 2 && (st = dalloc(&h->rscale, size_t(m) * q * per_row, h->stream))) ||
      (st = dalloc(&h->Upad, upad_n, h->stream)) ||
      (st = dalloc(&h->U, size_t(n) * r, h->stream)) || (st = dalloc(&h->Bk, size_t(q) * r, h->stream)) ||
      (st = dalloc(&h->S_idx, size_t(q) * std::max(1, h->rho), h->stream)) || (st = dalloc(&h->S_val, size_t(q) * std::max(1, h->rho), h->stream)) ||
      (st = dalloc(&h->H, size_t(q) * n, h->stream)) || (st = dalloc(&h->grad, size_t(n) * r, h->stream)) ||
      (st = dalloc(&h->Z, size_t(n) * r, h->stream)) || (st = dalloc(&h->U2, size_t(n) * r, h->stream)) ||
      (st = dalloc(&h->P, size_t(q) * r, h->stream)) || (st = dalloc(&h->part, size_t(h->nblk) * r * r, h->stream)) ||
      (st = dalloc(&h->small, 4 * 16 * 16 + 64, h->stream)) || (st = dalloc(&h->eta, 1, h->stream)) ||
      (st = dalloc(&h->err, 2, h->stream)) || (st = dalloc(&h->errpart, 2 * size_t(q), h->stream)) ||
      (h->engine == 2 && (st = alloc_task_engine(h))) || (st = alloc_split(h, nsm))) {
    std::string msg = g_last_error;
    free_all(h);
    delete h;
    return fail(st, "lrs_create: " + msg);
  }
  if (o.profile == 2) {
    if ((st = dalloc(&h->trace, size_t(q) * kTracePhases, h->stream)) ||
        (h->engine == 3 && (st = dalloc(&h->tprof, 16, h->stream)))) {
      free_all(h);
      delete h;
      return st;
    }
    cudaMemsetAsync(h->trace, 0, sizeof(unsigned long long) * size_t(q) * kTracePhases, h->stream);
    if (h->engine == 3) cudaMemsetAsync(h->tprof, 0, sizeof(unsigned long long) * 16, h->stream);
  }
  cudaError_t e = h->engine == 1   ? sweep_prepare(h->L, kThreads)
                  : h->engine == 3 ? res_prepare(res_rpad(r), static_cast<int>((m + 31) / 32))
                                   : task_prepare(sweep_rpad(r), h->L.et, h->tshape.smem);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, 2 * sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Upad, 0, sizeof(float) * upad_n, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->S_idx, 0, sizeof(int) * size_t(q) * std::max(1, h->rho), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->S_val, 0, sizeof(float) * size_t(q) * std::max(1, h->rho), h->stream);
  // the handle's memory is ready for any stream once its own stream gets here
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    free_all(h);
    delete h;
    return fail(LRS_ERR_CUDA, std::string("lrs_create: ") + cudaGetErrorString(e));
  }
  if (h->engine == 1 && sweep_max_active_clusters(h->L, h->resident, kThreads) <= 0) {
    free_all(h);
    delete h;
    return fail(LRS_ERR_UNSUPPORTED, "lrs_create: sweep kernel shape cannot be scheduled");
  }
  if (h->engine == 3) {
    const int R = res_rpad(r), MR = static_cast<int>((m + 31) / 32);
    const size_t smem = res_smem_bytes(R, MR, static_cast<int>(m), h->rho, h->res_CS);
    const int ncl = smem <= static_cast<size_t>(max_smem_optin())
                        ? res_max_clusters(R, MR, h->res_CS, smem) : 0;
    if (ncl <= 0) {
      free_all(h);
      delete h;
      return fail(LRS_ERR_UNSUPPORTED, "lrs_create: resident engine shape cannot be scheduled");
    }
    h->res_ncl = static_cast<int>(std::min<int64_t>(ncl, q));
    if (o.grid > 0) h->res_ncl = std::max(1, std::min(h->res_ncl, o.grid / h->res_CS));
  }
  if (h->engine == 2) {
    const int cps = task_ctas_per_sm(sweep_rpad(r), h->L.et, h->tshape.smem);
    if (cps <= 0) {
      free_all(h);
      delete h;
      return fail(LRS_ERR_UNSUPPORTED, "lrs_create: task engine cannot be scheduled");
    }
    h->tshape.ctas_per_sm = cps;
    h->tshape.grid = cps * nsm;
    if (o.grid > 0) h->tshape.grid = std::min(o.grid, h->tshape.grid);
  }
  *out = h;
  return LRS_OK;
}

lrs_status lrs_set_measurements(lrs_t h, const void* y, const void* A_or_mask, int32_t mem_kind) {
  if (!h || !y || !A_or_mask) return fail(LRS_ERR_ARG, "lrs_set_measurements: NULL argument");
  if (mem_kind != 0 && mem_kind != 1)
    return fail(LRS_ERR_ARG, "lrs_set_measurements: mem_kind must be 0 or 1");
  if (h->F) {
    std::string msg;
    const int st = fourier_set_measurements(h->F, y, A_or_mask, mem_kind, &msg);
    if (st) return fail(static_cast<lrs_status>(st), "lrs_set_measurements: " + msg);
    h->state = kMeasured;
    h->t = 0;
    return LRS_OK;
  }
  const cudaMemcpyKind kin = mem_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUDA_TRY(cudaMemcpyAsync(h->y, y, sizeof(float) * h->m * h->q, kin, h->stream));
  const size_t col_elems = static_cast<size_t>(h->m) * h->n;
  h->last_refine = -1;
  if (h->L.et != 0) {
    // low-precision forms: keep the exact FP32 operator, encode the sweep's copy from it
    CUDA_TRY(cudaMemcpyAsync(h->Aex, A_or_mask, sizeof(float) * col_elems * h->q, kin, h->stream));
    const int64_t chunk = std::max<int64_t>(1, (int64_t(1) << 30) / (int64_t)(col_elems * 4));
    for (int64_t k0 = 0; k0 < h->q; k0 += chunk) {
      const int64_t kc = std::min(chunk, h->q - k0);
      CUDA_TRY(repack_gauss(h->L, h->Aex + k0 * col_elems, static_cast<int>(k0),
                            static_cast<int>(kc), h->A, h->rscale, h->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->state = kMeasured;
    h->t = 0;
    return LRS_OK;
  }
  // A: row-major blocks -> slab layout, in chunks of columns
  int64_t chunk = std::max<int64_t>(1, (int64_t(256) << 20) / (int64_t)(col_elems * 4));
  chunk = std::min<int64_t>(chunk, h->q);
  float* tmp = nullptr;
  if (mem_kind == 0) CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&tmp), sizeof(float) * col_elems * chunk, h->stream));
  for (int64_t k0 = 0; k0 < h->q; k0 += chunk) {
    const int64_t kc = std::min(chunk, h->q - k0);
    const float* src = static_cast<const float*>(A_or_mask) + k0 * col_elems;
    if (mem_kind == 0) {
      cudaError_t e = cudaMemcpyAsync(tmp, src, sizeof(float) * col_elems * kc,
                                      cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = repack_a(h, tmp, k0, kc);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) {
        cudaFreeAsync(tmp, h->stream);
        return fail(LRS_ERR_CUDA, std::string("lrs_set_measurements: ") + cudaGetErrorString(e));
      }
    } else {
      CUDA_TRY(repack_a(h, src, k0, kc));
    }
  }
  if (tmp) cudaFreeAsync(tmp, h->stream);
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->state = kMeasured;
  h->t = 0;
  return LRS_OK;
}

lrs_status lrs_init(lrs_t h) {
  if (!h) return fail(LRS_ERR_ARG, "lrs_init: NULL handle");
  if (h->state < kMeasured) return fail(LRS_ERR_STATE, "lrs_init: no measurements");
  if (h->F) {
    std::string msg;
    const int st = fourier_init(h->F, &msg);
    if (st) return fail(static_cast<lrs_status>(st), "lrs_init: " + msg);
    h->state = kInitialised;
    h->t = 0;
    return LRS_OK;
  }
  GlobalWork g = gw(h);
  // s_k = IHT(y_k, A_k, rho, tau0, 0); L0 column k = A_k^T (y_k - A_k s_k) -> H
  lrs_status st = launch_sweep(h, kModeInit, h->opt.tau0);
  if (st) return st;
  // U0: top-r left singular subspace of L0 (= H^T) by subspace iteration:
  // FP32 products P = L0^T U and Z = L0 P, then Cholesky-QR2 of Z (FP64
  // r x r Gram and factors), until the subspace moves by less than power_tol.
  const size_t nr = static_cast<size_t>(h->n) * h->r;
  std::vector<float> U0f = start_block(h->n, h->r, h->opt.seed + 1);
  cudaError_t e = cudaMemcpyAsync(h->U2, U0f.data(), nr * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cholqr2(g, h->U2, h->U, h->err, h->stream);
  double* D = h->small + 2 * 16 * 16;
  int it = 0;
  for (; it < h->opt.power_iters && e == cudaSuccess; ++it) {
    e = cudaMemcpyAsync(h->U2, h->U, nr * 4, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = project_cols(g, h->H, h->U2, h->P, h->stream);
    if (e == cudaSuccess) {
      st = column_reduce(h, g, h->H, h->P);
      if (st) return st;
    }
    if (e == cudaSuccess) e = cholqr2(g, h->grad, h->U, h->err, h->stream);
    if (e == cudaSuccess && ((it % 5) == 4 || it + 1 == h->opt.power_iters)) {
      e = subspace_change(g, h->U2, h->U, D, D + 16 * 16, h->stream);
      double chg2 = 0.0;
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&chg2, D + 16 * 16, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e == cudaSuccess && std::sqrt(std::max(0.0, chg2)) < h->opt.power_tol) break;
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(LRS_ERR_CUDA, std::string("lrs_init: ") + cudaGetErrorString(e));
  h->power_iters_done = it;
  // b_k = (A_k U0)^+ (y_k - A_k s_k)
  st = launch_sweep(h, kModeLS, 0);
  if (st) return st;
  st = check_device_error(h, "lrs_init");
  if (st) return st;
  h->state = kInitialised;
  h->t = 0;
  h->last_refine = -1;
  return LRS_OK;
}

// problems of one batched launch (6 bits of a task descriptor)
constexpr int kMaxBatch = 64;

// automatic rank: subspace blocks of 16 columns, at most four
constexpr int kRankBlock = 16;
constexpr int kRankBlocks = 4;

lrs_status lrs_estimate_rank(lrs_t h, double energy, int32_t* r_out, double* sv,
                             int32_t sv_len, int32_t* n_sv) {
  if (!h) return fail(LRS_ERR_ARG, "lrs_estimate_rank: NULL handle");
  if (!r_out) return fail(LRS_ERR_ARG, "lrs_estimate_rank: r_out is NULL");
  if (!(energy > 0.0 && energy <= 1.0))
    return fail(LRS_ERR_ARG, "lrs_estimate_rank: energy must lie in (0, 1]");
  if (h->state != kMeasured)
    return fail(LRS_ERR_STATE, "lrs_estimate_rank: needs state MEASURED (before lrs_init)");
  if (h->F) return fail(LRS_ERR_UNSUPPORTED, "lrs_estimate_rank: Gaussian operators only");
  if (h->opt.reduce)
    return fail(LRS_ERR_UNSUPPORTED, "lrs_estimate_rank: not on a column-sharded handle");
  // L0 (= H^T) from the initialisation's IHT
  lrs_status st = launch_sweep(h, kModeInit, h->opt.tau0);
  if (st) return st;
  st = check_device_error(h, "lrs_estimate_rank");
  if (st) return st;
  const int n = static_cast<int>(h->n), q = static_cast<int>(h->q);
  const int64_t mnq = std::min<int64_t>(h->n, h->q);
  const int64_t want = std::max<int64_t>(1, std::min<int64_t>(mnq, h->m) / 10);
  // blocks of 16 (the widest the r x r kernels hold), at most four; a single
  // block narrower than 16 when n or q is
  const int B0 = static_cast<int>(std::min<int64_t>(kRankBlock, mnq));
  const int N = static_cast<int>(std::min<int64_t>(want, kRankBlock * kRankBlocks));
  const int nblocks = N <= B0 ? 1 : (N + kRankBlock - 1) / kRankBlock;
  if (nblocks > 1 && mnq < static_cast<int64_t>(nblocks) * kRankBlock)
    return fail(LRS_ERR_ARG, "lrs_estimate_rank: problem too small for the requested count");
  const int nb_n = qr_blocks(n), nb_q = qr_blocks(q);
  const size_t nw = static_cast<size_t>(n) * kRankBlock;
  float *U2 = nullptr, *Ub = nullptr, *P = nullptr, *Zg = nullptr, *Zt = nullptr;
  double *part = nullptr, *small = nullptr;
  cudaStream_t s = h->stream;
  auto release = [&]() {
    for (void* p : {static_cast<void*>(U2), static_cast<void*>(Ub), static_cast<void*>(P),
                    static_cast<void*>(Zg), static_cast<void*>(Zt), static_cast<void*>(part),
                    static_cast<void*>(small)})
      if (p) cudaFreeAsync(p, s);
  };
  st = dalloc(&U2, nw, s);
  if (!st) st = dalloc(&Ub, nw * nblocks, s);  // the converged blocks, one after another
  if (!st) st = dalloc(&P, static_cast<size_t>(q) * kRankBlock, s);
  if (!st) st = dalloc(&Zg, nw, s);
  if (!st) st = dalloc(&Zt, nw, s);
  if (!st) st = dalloc(&part, static_cast<size_t>(std::max(nb_n, nb_q)) * kRankBlock * kRankBlock, s);
  if (!st) st = dalloc(&small, static_cast<size_t>(4) * kRankBlock * kRankBlock + 8 + kRankBlock * kRankBlocks, s);
  if (st) {
    release();
    return st;
  }
  constexpr int WW = kRankBlock * kRankBlock;
  double* D = small + 2 * WW;          // small[0, 2 WW): the Cholesky-QR2 factors
  double* chg = small + 3 * WW;        // subspace change
  double* ritz = small + 3 * WW + 1;   // Ritz values, block after block
  GlobalWork g{};
  g.n = n;
  g.q = q;
  g.grad = Zg;
  g.part = part;
  g.small = small;
  g.Z = Zt;
  g.nblk = nb_n;
  g.ks = 1;
  cudaError_t e = cudaSuccess;
  // Block b: subspace iteration on L0 L0^T deflated by the blocks before it
  // (classical Gram-Schmidt, twice, after every product), as in lrs_init,
  // then its Rayleigh-Ritz values.
  for (int b = 0; b < nblocks && e == cudaSuccess; ++b) {
    const int W = b == 0 ? B0 : kRankBlock;
    g.r = W;
    float* U = Ub + static_cast<size_t>(b) * nw;
    auto deflate_all = [&](float* Z) {
      cudaError_t x = cudaSuccess;
      for (int pass = 0; pass < 2 && x == cudaSuccess; ++pass)
        for (int j = 0; j < b && x == cudaSuccess; ++j)
          x = deflate(g, Ub + static_cast<size_t>(j) * nw, Z, D, s);
      return x;
    };
    std::vector<float> U0f = start_block(h->n, W, h->opt.seed + 2 + b);
    e = cudaMemcpyAsync(U2, U0f.data(), static_cast<size_t>(n) * W * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = deflate_all(U2);
    if (e == cudaSuccess) e = cholqr2(g, U2, U, h->err, s);
    for (int it = 0; it < h->opt.power_iters && e == cudaSuccess; ++it) {
      e = cudaMemcpyAsync(U2, U, static_cast<size_t>(n) * W * 4, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = project_cols(g, h->H, U2, P, s);
      if (e == cudaSuccess) e = grad_reduce(g, h->H, P, s);
      if (e == cudaSuccess) e = deflate_all(Zg);
      if (e == cudaSuccess) e = cholqr2(g, Zg, U, h->err, s);
      if (e == cudaSuccess && ((it % 5) == 4 || it + 1 == h->opt.power_iters)) {
        e = subspace_change(g, U2, U, D, chg, s);
        double chg2 = 0.0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&chg2, chg, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && std::sqrt(std::max(0.0, chg2)) < h->opt.power_tol) break;
      }
    }
    // Rayleigh-Ritz: P = L0^T U, eigenvalues of P^T P = sigma^2
    if (e == cudaSuccess) e = project_cols(g, h->H, U, P, s);
    if (e == cudaSuccess) e = ritz_values(q, W, P, part, nb_q, ritz + b * kRankBlock, s);
  }
  const int nval = nblocks == 1 ? B0 : nblocks * kRankBlock;
  std::vector<double> lam(nval, 0.0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(lam.data(), ritz, nval * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess)
    return fail(LRS_ERR_CUDA, std::string("lrs_estimate_rank: ") + cudaGetErrorString(e));
  st = check_device_error(h, "lrs_estimate_rank");
  if (st) return st;
  std::sort(lam.begin(), lam.end(), [](double x, double y) { return x > y; });
  // energy threshold on the first N values
  double total = 0.0;
  for (int j = 0; j < N; ++j) total += std::max(0.0, lam[j]);
  int r = 1;
  if (total > 0.0) {
    double acc = 0.0;
    r = N;
    for (int j = 0; j < N; ++j) {
      acc += std::max(0.0, lam[j]);
      if (acc >= energy * total) {
        r = j + 1;
        break;
      }
    }
  }
  *r_out = r;
  if (sv)
    for (int j = 0; j < std::min(N, static_cast<int>(sv_len)); ++j)
      sv[j] = std::sqrt(std::max(0.0, lam[j]));
  if (n_sv) *n_sv = N;
  return LRS_OK;
}

lrs_status lrs_iterate(lrs_t h, int32_t iters, double* err_log) {
  if (!h) return fail(LRS_ERR_ARG, "lrs_iterate: NULL handle");
  if (iters < 0) return fail(LRS_ERR_ARG, "lrs_iterate: iters < 0");
  if (h->state < kInitialised) return fail(LRS_ERR_STATE, "lrs_iterate: call lrs_init first");
  if (err_log && !h->Xref) return fail(LRS_ERR_ARG, "lrs_iterate: err_log needs lrs_set_reference");
  if (h->F) {
    if (err_log) return fail(LRS_ERR_UNSUPPORTED, "lrs_iterate: no error log for the DFT operator");
    const bool fprof = h->opt.profile != 0;
    if (fprof) {
      while (h->ev.size() < 4 * static_cast<size_t>(iters)) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        h->ev.push_back(e);
      }
    }
    std::string msg;
    const int st = fourier_iterate(h->F, iters, &msg, fprof ? h->ev.data() : nullptr);
    h->t = fourier_t(h->F);
    h->state = kIterating;
    if (st) return fail(static_cast<lrs_status>(st), "lrs_iterate: " + msg);
    if (fprof && iters > 0) {  // the stream is synchronised by the error check above
      for (int i = 0; i < iters; ++i) {
        float a = 0, b = 0, c = 0;
        cudaEvent_t* evs = &h->ev[4 * static_cast<size_t>(i)];
        CUDA_TRY(cudaEventElapsedTime(&a, evs[0], evs[1]));
        CUDA_TRY(cudaEventElapsedTime(&b, evs[1], evs[2]));
        CUDA_TRY(cudaEventElapsedTime(&c, evs[2], evs[3]));
        h->phase_ms[0] += a;
        h->phase_ms[1] += b;
        h->phase_ms[2] += c;
      }
      h->phase_iters += iters;
    }
    return LRS_OK;
  }
  if (h->opt.autotune && h->engine == 2 && !h->tuned && iters > 0) {
    lrs_status st = lrs_autotune(h, 2, nullptr, 0);
    if (st) return st;
  }
  const bool prof = h->opt.profile != 0;
  if (prof) {
    while (h->ev.size() < 4 * static_cast<size_t>(iters)) {
      cudaEvent_t e;
      CUDA_TRY(cudaEventCreate(&e));
      h->ev.push_back(e);
    }
  }
  for (int i = 0; i < iters; ++i) {
    const bool first = (h->t == 0);
    cudaEvent_t* evs = prof ? &h->ev[4 * static_cast<size_t>(i)] : nullptr;
    const bool refine = h->L.et != 0 &&
                        (h->last_refine < 0 || h->t - h->last_refine >= h->opt.refine_every);
    if (refine) h->last_refine = h->t;
    if (!first && h->opt.use_graph && h->stream && !prof) {
      // replay the captured iteration (captured on first use; every launch of
      // it reads only device state, so one capture serves all later iterations)
      const int gi = refine ? 1 : 0;
      if (!h->gexec[gi]) {
        CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        lrs_status st = enqueue_iteration(h, false, nullptr, refine);
        cudaGraph_t gph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->stream, &gph);
        if (st) return st;
        CUDA_TRY(e);
        h->graph[gi] = gph;
        CUDA_TRY(cudaGraphInstantiate(&h->gexec[gi], h->graph[gi], 0));
      }
      CUDA_TRY(cudaGraphLaunch(h->gexec[gi], h->stream));
    } else {
      lrs_status st = enqueue_iteration(h, first, evs, refine);
      if (st) return st;
    }
    h->t += 1;
    if (err_log) {
      lrs_status st = error_now(h, &err_log[i]);
      if (st) return st;
    }
  }
  h->state = kIterating;
  if (prof && iters > 0) {
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < iters; ++i) {
      float a = 0, b = 0, c = 0;
      cudaEvent_t* evs = &h->ev[4 * static_cast<size_t>(i)];
      CUDA_TRY(cudaEventElapsedTime(&a, evs[0], evs[1]));
      CUDA_TRY(cudaEventElapsedTime(&b, evs[1], evs[2]));
      CUDA_TRY(cudaEventElapsedTime(&c, evs[2], evs[3]));
      h->phase_ms[0] += a;
      h->phase_ms[1] += b;
      h->phase_ms[2] += c;
    }
    h->phase_iters += iters;
  }
  return check_device_error(h, "lrs_iterate");
}

lrs_status lrs_iterate_batch(lrs_t* hs, int32_t nh, int32_t iters) {
  if (!hs || nh < 1 || nh > kMaxBatch)
    return fail(LRS_ERR_ARG, "lrs_iterate_batch: need 1 <= nh <= 64 handles");
  if (iters < 0) return fail(LRS_ERR_ARG, "lrs_iterate_batch: iters < 0");
  for (int i = 0; i < nh; ++i) {
    if (!hs[i]) return fail(LRS_ERR_ARG, "lrs_iterate_batch: NULL handle");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(LRS_ERR_ARG, "lrs_iterate_batch: a handle appears twice");
    if (hs[i]->state < kInitialised)
      return fail(LRS_ERR_STATE, "lrs_iterate_batch: call lrs_init on every handle first");
  }
  lrs_ctx* h0 = hs[0];
  const int R = sweep_rpad(h0->r), et = h0->L.et;
  for (int i = 0; i < nh; ++i) {
    const lrs_ctx* h = hs[i];
    if (h->F || h->engine != 2 || h->opt.reduce || sweep_rpad(h->r) != R || h->L.et != et)
      return fail(LRS_ERR_UNSUPPORTED,
                  "lrs_iterate_batch: Gaussian task-engine handles of one rank width and A_k form");
  }
  if (nh == 1) return lrs_iterate(h0, iters, nullptr);
  // the launch's work table: every handle's ITER-mode problem, columns
  // numbered across the handles in order; all columns in flight
  std::vector<TaskProblem> P(nh);
  int64_t cols = 0, total = 0, nseed = 0;
  int m_max = 0, ns_max = 0, rho_max = 0, pb_max = 0;
  for (int i = 0; i < nh; ++i) {
    const lrs_ctx* h = hs[i];
    P[i] = h->tp[kModeIter];
    P[i].col0 = static_cast<int>(cols);
    cols += h->q;
    total += static_cast<int64_t>(P[i].tasks_per_col) * h->q;
    nseed += static_cast<int64_t>(phase_tasks(P[i], 0)) * h->q;
    m_max = std::max<int>(m_max, static_cast<int>(h->m));
    ns_max = std::max(ns_max, h->L.ns);
    rho_max = std::max(rho_max, h->rho);
    pb_max = std::max(pb_max, h->tshape.piece_bytes);
  }
  if (total >= (int64_t(1) << 31) || cols >= (int64_t(1) << 30))
    return fail(LRS_ERR_UNSUPPORTED, "lrs_iterate_batch: too many tasks for one launch");
  int dev = 0, nsm = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  TaskShape shape = h0->tshape;
  shape.stages = kTaskStages;
  shape.piece_bytes = pb_max;
  shape.smem = task_smem_bytes(R, et, m_max, ns_max, rho_max, kTaskStages, pb_max);
  if (shape.smem > static_cast<size_t>(max_smem_optin()))
    return fail(LRS_ERR_UNSUPPORTED, "lrs_iterate_batch: the problems' shared memory does not fit one CTA");
  const int cps = std::min(2, task_ctas_per_sm(R, et, shape.smem));
  if (cps < 1) return fail(LRS_ERR_UNSUPPORTED, "lrs_iterate_batch: no CTA fits an SM");
  int grid = cps * nsm;
  if (h0->opt.grid > 0) grid = std::min(grid, h0->opt.grid);
  shape.grid = grid;
  // device tables (freed at the end of the call, stream-ordered)
  cudaStream_t s = h0->stream;
  TaskProblem* dP = nullptr;
  unsigned long long *dtasks = nullptr, *dseed = nullptr;
  int *dseq = nullptr, *dctr = nullptr, *dcnt = nullptr;
  lrs_status st = dalloc(&dP, nh, s);
  if (!st) st = dalloc(&dtasks, total, s);
  if (!st) st = dalloc(&dseq, total, s);
  if (!st) st = dalloc(&dctr, 4, s);
  if (!st) st = dalloc(&dcnt, cols, s);
  if (!st) st = dalloc(&dseed, nseed, s);
  auto release = [&]() {
    for (void* p : {static_cast<void*>(dP), static_cast<void*>(dtasks), static_cast<void*>(dseed),
                    static_cast<void*>(dseq), static_cast<void*>(dctr), static_cast<void*>(dcnt)})
      if (p) cudaFreeAsync(p, s);
  };
  if (st) {
    release();
    return st;
  }
  std::vector<unsigned long long> seed;
  seed.reserve(nseed);
  for (int i = 0; i < nh; ++i) {
    P[i].cnt = dcnt + P[i].col0;
    const int n0 = phase_tasks(P[i], 0);
    for (int64_t k = 0; k < hs[i]->q; ++k)
      for (int t = 0; t < n0; ++t)
        seed.push_back(tdesc(static_cast<int>(k), i, phase_type(P[i], 0), 0, t));
  }
  // every handle's stream waits for what was queued on it before; the
  // shared sweep runs on the first handle's stream, each handle's gradient,
  // step size and QR on its own stream after it
  std::vector<cudaEvent_t> evs(nh + 1, nullptr);
  cudaError_t e = cudaSuccess;
  for (auto& ev : evs)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dP, P.data(), nh * sizeof(TaskProblem), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dseed, seed.data(), nseed * 8, cudaMemcpyHostToDevice, s);
  lrs_status rs = LRS_OK;
  for (int it = 0; it < iters && e == cudaSuccess && rs == LRS_OK; ++it) {
    for (int i = 1; i < nh && e == cudaSuccess; ++i) {
      e = cudaEventRecord(evs[i], hs[i]->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, evs[i], 0);
    }
    for (int i = 0; i < nh && e == cudaSuccess; ++i) {
      lrs_ctx* h = hs[i];
      const bool refine = h->L.et != 0 &&
                          (h->last_refine < 0 || h->t - h->last_refine >= h->opt.refine_every);
      if (refine) {
        h->last_refine = h->t;
        e = refine_residual(h->L, h->Aex, h->A, h->rscale, h->U, h->Bk, h->S_idx, h->S_val, h->y,
                            h->ycorr, h->H, s);
      }
    }
    if (e != cudaSuccess) break;
    TaskQueue Q{};
    Q.tasks = dtasks;
    Q.seq = dseq;
    Q.ctr = dctr;
    Q.total = static_cast<int>(total);
    Q.ncols = static_cast<int>(cols);
    Q.F = static_cast<int>(cols);
    Q.nprob = nh;
    Q.probs = dP;
    Q.prof = nullptr;
    Q.wait_ns = wait_bound_ns(h0);
    e = task_launch_seeded(Q, dseed, static_cast<int>(nseed), dcnt, R, et, shape, m_max, ns_max,
                           rho_max, s);
    if (e == cudaSuccess) e = cudaEventRecord(evs[0], s);
    for (int i = 0; i < nh && e == cudaSuccess && rs == LRS_OK; ++i) {
      lrs_ctx* h = hs[i];
      if (i > 0) e = cudaStreamWaitEvent(h->stream, evs[0], 0);
      if (e != cudaSuccess) break;
      GlobalWork g = gw(h);
      rs = column_reduce(h, g, h->H, h->Bk);
      if (rs == LRS_OK && h->t == 0) e = eta_from_grad(g, h->opt.c_eta, h->eta, h->stream);
      if (rs == LRS_OK && e == cudaSuccess) e = qr_step(g, h->U, h->eta, h->err, h->stream);
      h->t += 1;
      h->state = kIterating;
    }
    // the next sweep reads every handle's new U
    for (int i = 1; i < nh && e == cudaSuccess; ++i) {
      e = cudaEventRecord(evs[i], hs[i]->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, evs[i], 0);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  for (int i = 0; i < nh; ++i) cudaStreamSynchronize(hs[i]->stream);
  for (auto ev : evs)
    if (ev) cudaEventDestroy(ev);
  if (rs != LRS_OK) return rs;
  if (e != cudaSuccess)
    return fail(LRS_ERR_CUDA, std::string("lrs_iterate_batch: ") + cudaGetErrorString(e));
  for (int i = 0; i < nh; ++i) {
    st = check_device_error(hs[i], "lrs_iterate_batch");
    if (st) return st;
  }
  return LRS_OK;
}

lrs_status lrs_solve(lrs_t h) {
  lrs_status st = lrs_init(h);
  if (st) return st;
  return lrs_iterate(h, h->opt.T, nullptr);
}

lrs_status lrs_get(lrs_t h, void* U, void* B, int32_t* S_idx, void* S_val, int32_t mem_kind) {
  if (!h) return fail(LRS_ERR_ARG, "lrs_get: NULL handle");
  if (mem_kind != 0 && mem_kind != 1) return fail(LRS_ERR_ARG, "lrs_get: mem_kind must be 0 or 1");
  if (h->state < kInitialised) return fail(LRS_ERR_STATE, "lrs_get: no iterate yet");
  if (h->F) {
    if (fourier_get(h->F, U, B, S_idx, S_val, mem_kind)) return fail(LRS_ERR_CUDA, "lrs_get: copy failed");
    return LRS_OK;
  }
  const cudaMemcpyKind kout = mem_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (U) {
    const int tot = static_cast<int>(h->n) * h->r;
    transpose_kernel<<<(tot + 255) / 256, 256, 0, h->stream>>>(h->U, h->Z, static_cast<int>(h->n), h->r);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(U, h->Z, sizeof(float) * tot, kout, h->stream));
  }
  if (B) CUDA_TRY(cudaMemcpyAsync(B, h->Bk, sizeof(float) * h->q * h->r, kout, h->stream));
  if (S_idx && h->rho)
    CUDA_TRY(cudaMemcpyAsync(S_idx, h->S_idx, sizeof(int) * h->q * h->rho, kout, h->stream));
  if (S_val && h->rho)
    CUDA_TRY(cudaMemcpyAsync(S_val, h->S_val, sizeof(float) * h->q * h->rho, kout, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return LRS_OK;
}

lrs_status lrs_get_x(lrs_t h, void* X, int32_t mem_kind) {
  if (!h || !X) return fail(LRS_ERR_ARG, "lrs_get_x: NULL argument");
  if (mem_kind != 0 && mem_kind != 1) return fail(LRS_ERR_ARG, "lrs_get_x: mem_kind must be 0 or 1");
  if (h->state < kInitialised) return fail(LRS_ERR_STATE, "lrs_get_x: no iterate yet");
  const int ct = h->F ? 2 : 1;
  const size_t nU = static_cast<size_t>(h->n) * h->r * ct, nB = static_cast<size_t>(h->q) * h->r * ct;
  const size_t nS = static_cast<size_t>(h->q) * h->rho, nX = static_cast<size_t>(h->n) * h->q * ct;
  float *U = nullptr, *B = nullptr, *Sv = nullptr, *Xd = nullptr;
  int* Si = nullptr;
  const size_t bytes = sizeof(float) * (nU + nB + nS * ct + (mem_kind ? 0 : nX)) + sizeof(int) * nS + 256;
  char* buf = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&buf), bytes, h->stream) != cudaSuccess)
    return fail(LRS_ERR_OOM, "lrs_get_x: scratch");
  U = reinterpret_cast<float*>(buf);     // [U | B | S values | X (host case) | S indices]
  B = U + nU;
  Sv = B + nB;
  float* after = Sv + nS * ct;
  if (mem_kind) {
    Xd = static_cast<float*>(X);
  } else {
    Xd = after;
    after += nX;
  }
  Si = reinterpret_cast<int*>(after);
  lrs_status st = lrs_get(h, U, B, h->rho ? Si : nullptr, h->rho ? Sv : nullptr, 1);
  if (st == LRS_OK) {
    if (ct == 1)
      assemble_x_kernel<1><<<static_cast<unsigned>(h->q), 256, 0, h->stream>>>(
          static_cast<int>(h->n), static_cast<int>(h->q), h->r, h->rho, U, B, Si, Sv, Xd);
    else
      assemble_x_kernel<2><<<static_cast<unsigned>(h->q), 256, 0, h->stream>>>(
          static_cast<int>(h->n), static_cast<int>(h->q), h->r, h->rho, U, B, Si, Sv, Xd);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !mem_kind)
      e = cudaMemcpyAsync(X, Xd, sizeof(float) * nX, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) st = fail(LRS_ERR_CUDA, std::string("lrs_get_x: ") + cudaGetErrorString(e));
  }
  cudaFreeAsync(buf, h->stream);
  return st;
}

lrs_status lrs_set_state(lrs_t h, const void* U, const void* B, const int32_t* S_idx,
                         const void* S_val, int32_t t, double eta, int32_t mem_kind) {
  if (!h || !U || !B || (h->rho && (!S_idx || !S_val)))
    return fail(LRS_ERR_ARG, "lrs_set_state: NULL argument");
  if (mem_kind != 0 && mem_kind != 1) return fail(LRS_ERR_ARG, "lrs_set_state: bad mem_kind");
  if (t < 0) return fail(LRS_ERR_ARG, "lrs_set_state: t < 0");
  if (h->state < kMeasured) return fail(LRS_ERR_STATE, "lrs_set_state: no measurements");
  if (h->F) {
    if (fourier_set_state(h->F, U, B, S_idx, S_val, t, eta, mem_kind))
      return fail(LRS_ERR_CUDA, "lrs_set_state: copy failed");
    h->t = t;
    h->state = t == 0 ? kInitialised : kIterating;
    return LRS_OK;
  }
  const cudaMemcpyKind kin = mem_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const int tot = static_cast<int>(h->n) * h->r;
  CUDA_TRY(cudaMemcpyAsync(h->Z, U, sizeof(float) * tot, kin, h->stream));
  transpose_kernel<<<(tot + 255) / 256, 256, 0, h->stream>>>(h->Z, h->U, h->r, static_cast<int>(h->n));
  CUDA_TRY(cudaGetLastError());
  pad_rows_kernel<<<(tot + 255) / 256, 256, 0, h->stream>>>(h->U, h->Upad, static_cast<int>(h->n),
                                                            h->r, sweep_rpad(h->r));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(h->Bk, B, sizeof(float) * h->q * h->r, kin, h->stream));
  if (h->rho) {
    CUDA_TRY(cudaMemcpyAsync(h->S_idx, S_idx, sizeof(int) * h->q * h->rho, kin, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->S_val, S_val, sizeof(float) * h->q * h->rho, kin, h->stream));
  }
  CUDA_TRY(cudaMemcpyAsync(h->eta, &eta, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->t = t;
  h->last_refine = -1;
  h->state = t == 0 ? kInitialised : kIterating;
  return LRS_OK;
}

lrs_status lrs_get_progress(lrs_t h, double* eta, int32_t* t) {
  if (!h) return fail(LRS_ERR_ARG, "lrs_get_progress: NULL handle");
  if (h->F) {
    if (eta) *eta = fourier_eta(h->F);
    if (t) *t = fourier_t(h->F);
    return LRS_OK;
  }
  if (eta) {
    CUDA_TRY(cudaMemcpyAsync(eta, h->eta, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (h->t == 0) *eta = 0.0;
  }
  if (t) *t = h->t;
  return LRS_OK;
}

lrs_status lrs_set_reference(lrs_t h, const void* Xref, int32_t mem_kind) {
  if (!h || !Xref) return fail(LRS_ERR_ARG, "lrs_set_reference: NULL argument");
  if (mem_kind != 0 && mem_kind != 1) return fail(LRS_ERR_ARG, "lrs_set_reference: bad mem_kind");
  if (!h->Xref) CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&h->Xref), sizeof(float) * h->n * h->q, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->Xref, Xref, sizeof(float) * h->n * h->q,
                           mem_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return LRS_OK;
}

lrs_status lrs_phase_times(lrs_t h, double* out4) {
  if (!h || !out4) return fail(LRS_ERR_ARG, "lrs_phase_times: NULL argument");
  for (int i = 0; i < 3; ++i) out4[i] = h->phase_ms[i];
  out4[3] = static_cast<double>(h->phase_iters);
  h->phase_ms[0] = h->phase_ms[1] = h->phase_ms[2] = 0;
  h->phase_iters = 0;
  return LRS_OK;
}

lrs_status lrs_sweep_trace(lrs_t h, uint64_t* out, int64_t len) {
  if (!h || !out || len < 0) return fail(LRS_ERR_ARG, "lrs_sweep_trace: bad argument");
  if (h->F) {
    if (h->opt.profile != 2) return fail(LRS_ERR_STATE, "lrs_sweep_trace: create the handle with profile = 2");
    const int st = fourier_prof_read(h->F, reinterpret_cast<unsigned long long*>(out),
                                     static_cast<int>(std::min<int64_t>(len, 1 << 20)));
    if (st) return fail(static_cast<lrs_status>(st), "lrs_sweep_trace: reading the counters failed");
    return LRS_OK;
  }
  if ((h->engine == 2 || h->engine == 3) && h->opt.profile == 2) {
    const int64_t n = std::min<int64_t>(len, h->engine == 3 ? kResProf : kTaskProf);
    CUDA_TRY(cudaMemcpyAsync(out, h->tprof, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemsetAsync(h->tprof, 0, sizeof(uint64_t) * 16, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return LRS_OK;
  }
  if (!h->trace) return fail(LRS_ERR_STATE, "lrs_sweep_trace: create the handle with profile = 2");
  const int64_t n = std::min<int64_t>(len, h->q * kTracePhases);
  CUDA_TRY(cudaMemcpyAsync(out, h->trace, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaMemsetAsync(h->trace, 0, sizeof(uint64_t) * h->q * kTracePhases, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return LRS_OK;
}

// Kernels one steady GDmin iteration launches (no refinement of the
// measurements, step size already frozen): the sweep (task engine: queue
// reset + persistent kernel), the gradient (k-split partials + their sum, or
// one kernel), Cholesky-QR2 (Gram partials, two factorisations, two
// applications).
static int launches_per_iteration(const lrs_ctx* h) {
  const int sweep = h->engine == 2 ? 2 : 1;
  const int grad = (h->ks > 1 || h->qc > 0) ? 2 : 1;
  return sweep + grad + 5;
}

lrs_status lrs_describe(lrs_t h, char* buf, int32_t len) {
  if (!h || !buf || len <= 0) return fail(LRS_ERR_ARG, "lrs_describe: bad argument");
  if (h->F) {
    snprintf(buf, static_cast<size_t>(len),
             "{\"op\": \"dft2d\", \"nx\": %d, \"ny\": %d, \"cta_per_frame\": 1, "
             "\"fused_qr\": %d, \"launches_per_iteration\": %d}",
             h->opt.nx, h->opt.ny, fourier_fused_qr(h->F), fourier_launches_per_iteration(h->F));
    return LRS_OK;
  }
  if (h->engine == 3) {
    const int R = res_rpad(h->r), MR = static_cast<int>((h->m + 31) / 32);
    snprintf(buf, static_cast<size_t>(len),
             "{\"op\": \"gaussian\", \"engine\": \"resident\", \"cluster\": %d, "
             "\"clusters\": %d, \"rows_per_lane\": %d, \"rank_width\": %d, "
             "\"smem_per_cta\": %zu, \"launches_per_iteration\": %d}",
             h->res_CS, h->res_ncl, MR, R,
             res_smem_bytes(R, MR, static_cast<int>(h->m), h->rho, h->res_CS),
             launches_per_iteration(h));
    return LRS_OK;
  }
  if (h->engine == 2) {
    const TaskProblem& P = h->tp[kModeIter];
    snprintf(buf, static_cast<size_t>(len),
             "{\"op\": \"gaussian\", \"engine\": \"task\", \"grid\": %d, \"ctas_per_sm\": %d, "
             "\"stages\": %d, \"piece_bytes\": %d, \"smem_per_cta\": %zu, \"inflight\": %d, "
             "\"w_tasks\": %d, \"g_tasks\": %d, \"rows_per_piece\": %d, \"tiles_per_task\": %d, "
             "\"a_dtype\": %d, \"refine_every\": %d, \"launches_per_iteration\": %d}",
             h->tshape.grid, h->tshape.ctas_per_sm, h->tshape.stages, h->tshape.piece_bytes,
             h->tshape.smem, h->tF, P.nrb * P.ncw, P.ngb, P.rp, P.TB, h->L.et, h->opt.refine_every,
             launches_per_iteration(h));
    return LRS_OK;
  }
  const size_t sm = sweep_smem_bytes(h->L, h->resident, kThreads);
  const int nc = sweep_max_active_clusters(h->L, h->resident, kThreads);
  snprintf(buf, static_cast<size_t>(len),
           "{\"op\": \"%s\", \"engine\": \"cluster\", \"cluster\": %d, \"ns\": %d, \"stages\": %d, \"resident\": %d, "
           "\"smem_per_cta\": %zu, \"max_active_clusters\": %d, \"a_dtype\": %d, "
           "\"refine_every\": %d, \"launches_per_iteration\": %d}",
           h->kind == LRS_OP_GAUSSIAN ? "gaussian" : "dft2d", h->L.cs, h->L.ns, h->L.stages,
           h->resident, sm, nc, h->L.et, h->opt.refine_every, launches_per_iteration(h));
  return LRS_OK;
}

lrs_status lrs_autotune(lrs_t h, int32_t trial_iters, char* report, int32_t len) {
  if (!h) return fail(LRS_ERR_ARG, "lrs_autotune: NULL handle");
  if (trial_iters < 1) return fail(LRS_ERR_ARG, "lrs_autotune: trial_iters < 1");
  if (h->F || h->engine != 2) return fail(LRS_ERR_UNSUPPORTED, "lrs_autotune: task engine only");
  if (h->opt.reduce)
    return fail(LRS_ERR_UNSUPPORTED, "lrs_autotune: not on a column-sharded handle");
  if (h->state < kInitialised) return fail(LRS_ERR_STATE, "lrs_autotune: call lrs_init first");
  const size_t nr = static_cast<size_t>(h->n) * h->r, qr = static_cast<size_t>(h->q) * h->r;
  const size_t qs = static_cast<size_t>(h->q) * std::max(1, h->rho);
  const size_t upad_n = static_cast<size_t>(h->L.ns) * sweep_rpad(h->r);
  const size_t qm = h->L.et != 0 ? static_cast<size_t>(h->q) * h->m : 0;
  // the state the trials start from, restored after each of them
  float *U = nullptr, *Up = nullptr, *B = nullptr, *Sv = nullptr, *Yc = nullptr;
  int* Si = nullptr;
  double* eta = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    for (void* p : {static_cast<void*>(U), static_cast<void*>(Up), static_cast<void*>(B),
                    static_cast<void*>(Sv), static_cast<void*>(Yc), static_cast<void*>(Si),
                    static_cast<void*>(eta)})
      if (p) cudaFreeAsync(p, h->stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  auto am = [&](auto** p, size_t bytes) {
    return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, h->stream) == cudaSuccess;
  };
  if (!am(&U, nr * 4) || !am(&Up, upad_n * 4) || !am(&B, qr * 4) || !am(&Sv, qs * 4) ||
      !am(&Si, qs * 4) || !am(&eta, 8) || (qm && !am(&Yc, qm * 4)) ||
      cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cleanup();
    return fail(LRS_ERR_OOM, "lrs_autotune: no memory for the saved state");
  }
  const int t_saved = h->t, lr_saved = h->last_refine;
  auto copy_state = [&](bool save) -> cudaError_t {
    auto cp = [&](void* keep, void* live, size_t bytes) {
      return save ? cudaMemcpyAsync(keep, live, bytes, cudaMemcpyDeviceToDevice, h->stream)
                  : cudaMemcpyAsync(live, keep, bytes, cudaMemcpyDeviceToDevice, h->stream);
    };
    cudaError_t e = cp(U, h->U, nr * 4);
    if (e == cudaSuccess) e = cp(Up, h->Upad, upad_n * 4);
    if (e == cudaSuccess) e = cp(B, h->Bk, qr * 4);
    if (e == cudaSuccess) e = cp(Si, h->S_idx, qs * 4);
    if (e == cudaSuccess) e = cp(Sv, h->S_val, qs * 4);
    if (e == cudaSuccess) e = cp(eta, h->eta, 8);
    if (e == cudaSuccess && qm) e = cp(Yc, h->ycorr, qm * 4);
    if (!save) {
      h->t = t_saved;
      h->last_refine = lr_saved;
    }
    return e;
  };
  cudaError_t e = copy_state(true);
  const int q = static_cast<int>(h->q);
  std::vector<std::pair<int, int>> cands;
  for (int kib : kTuneKib)
    for (int F : {q, std::max(1, q / 2), std::min(q, 2 * h->tshape.grid)}) {
      std::pair<int, int> c{kib, F};
      if (std::find(cands.begin(), cands.end(), c) == cands.end()) cands.push_back(c);
    }
  const int kib0 = h->t_kib, F0 = h->tF;
  std::pair<int, int> best{kib0, F0};
  float best_ms = 1e30f;
  std::string rep = "{\"trials\": [";
  for (size_t ci = 0; ci < cands.size() && e == cudaSuccess; ++ci) {
    lrs_status st = plan_tables(h, cands[ci].first, cands[ci].second);
    if (st) {
      cleanup();
      return st;
    }
    e = copy_state(false);
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int i = 0; i < trial_iters && e == cudaSuccess; ++i) {
      const bool refine = h->L.et != 0 &&
                          (h->last_refine < 0 || h->t - h->last_refine >= h->opt.refine_every);
      if (refine) h->last_refine = h->t;
      st = enqueue_iteration(h, h->t == 0, nullptr, refine);
      if (st) {
        cleanup();
        return st;
      }
      h->t += 1;
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    ms /= static_cast<float>(trial_iters);
    if (ms < best_ms) {
      best_ms = ms;
      best = cands[ci];
    }
    char buf[96];
    snprintf(buf, sizeof(buf), "%s{\"task_kib\": %d, \"inflight\": %d, \"ms\": %.4f}",
             ci ? ", " : "", cands[ci].first, cands[ci].second, ms);
    rep += buf;
  }
  lrs_status st = LRS_OK;
  if (e == cudaSuccess) st = plan_tables(h, best.first, best.second);
  if (e == cudaSuccess && st == LRS_OK) e = copy_state(false);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cleanup();
  if (e != cudaSuccess) return fail(LRS_ERR_CUDA, std::string("lrs_autotune: ") + cudaGetErrorString(e));
  if (st) return st;
  for (int g = 0; g < 2; ++g) {  // captured iterations carry the old task shapes
    if (h->gexec[g]) cudaGraphExecDestroy(h->gexec[g]);
    if (h->graph[g]) cudaGraphDestroy(h->graph[g]);
    h->gexec[g] = nullptr;
    h->graph[g] = nullptr;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[tune_key(h)] = best;
  }
  h->tuned = 1;
  lrs_status stc = check_device_error(h, "lrs_autotune");
  if (report && len > 0) {
    char buf[128];
    snprintf(buf, sizeof(buf), "], \"chosen\": {\"task_kib\": %d, \"inflight\": %d, \"ms\": %.4f}}",
             best.first, best.second, best_ms);
    rep += buf;
    snprintf(report, static_cast<size_t>(len), "%s", rep.c_str());
  }
  return stc;
}

lrs_status lrs_orthonormalize(const float* Z, float* Q, int64_t n, int32_t r, void* stream) {
  if (!Z || !Q) return fail(LRS_ERR_ARG, "lrs_orthonormalize: NULL pointer");
  if (r < 1 || r > 16 || n < r || n >= (int64_t(1) << 30))
    return fail(LRS_ERR_ARG, "lrs_orthonormalize: need 1 <= r <= 16 and r <= n < 2^30");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nblk = qr_blocks(n);
  float* tmp = nullptr;
  double* part = nullptr;
  int* err = nullptr;
  auto cleanup = [&]() {
    if (tmp) cudaFreeAsync(tmp, s);
    if (part) cudaFreeAsync(part, s);
    if (err) cudaFreeAsync(err, s);
  };
  if (cudaMallocAsync(reinterpret_cast<void**>(&tmp), sizeof(float) * n * r, s) != cudaSuccess ||
      cudaMallocAsync(reinterpret_cast<void**>(&part),
                      sizeof(double) * (static_cast<size_t>(nblk) * r * r + 2 * r * r), s) != cudaSuccess ||
      cudaMallocAsync(reinterpret_cast<void**>(&err), 2 * sizeof(int), s) != cudaSuccess) {
    cleanup();
    return fail(LRS_ERR_OOM, "lrs_orthonormalize: scratch allocation failed");
  }
  int eh[2] = {0, 0};
  cudaError_t e = cudaMemsetAsync(err, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess)
    e = cholqr2_into(static_cast<int>(n), r, Z, Q, tmp, part, part + static_cast<size_t>(nblk) * r * r,
                     err, nblk, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(eh, err, sizeof(eh), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return fail(LRS_ERR_CUDA, std::string("lrs_orthonormalize: ") + cudaGetErrorString(e));
  if (eh[0]) return fail(LRS_ERR_NUMERICAL, "lrs_orthonormalize: Z^T Z not positive definite");
  return LRS_OK;
}

lrs_status lrs_destroy(lrs_t h) {
  if (!h) return LRS_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->F) {
    fourier_destroy(h->F);
    delete h;
    return LRS_OK;
  }
  free_all(h);
  if (h->stream) cudaStreamSynchronize(h->stream);
  delete h;
  return LRS_OK;
}

}  // extern "C"
