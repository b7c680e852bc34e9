// Launch side of the persistent task engine (kernel body in
// task_sweep_impl.cuh; one translation unit per compiled rank width): task
// shapes, shared-memory sizing, queue reset and the persistent launch.
#include <algorithm>

#include "task_sweep_impl.cuh"

namespace lrs {
void* task_kernel_r2(int et);
void* task_kernel_r3(int et);
void* task_kernel_r4(int et);
void* task_kernel_r5(int et);
void* task_kernel_r6(int et);
void* task_kernel_r8(int et);
void* task_kernel_r10(int et);
void* task_kernel_r12(int et);
void* task_kernel_r16(int et);

namespace {
using namespace task;

void* pick(int R, int et) {
  switch (R) {
    case 2: return task_kernel_r2(et);
    case 3: return task_kernel_r3(et);
    case 4: return task_kernel_r4(et);
    case 5: return task_kernel_r5(et);
    case 6: return task_kernel_r6(et);
    case 8: return task_kernel_r8(et);
    case 10: return task_kernel_r10(et);
    case 12: return task_kernel_r12(et);
    default: return task_kernel_r16(et);
  }
}

int round8(int x) { return (x + 7) / 8 * 8; }

// Queue reset of one launch: the first F columns' first-pass tasks published,
// every other ticket unpublished, pass counters zero.
__global__ void reset_kernel(TaskQueue Q, const unsigned long long* seed, int n_seed, int* cnt_all) {
  const int stride = gridDim.x * blockDim.x;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Q.total; t += stride) {
    if (t < n_seed) Q.tasks[t] = seed[t];
    Q.seq[t] = t < n_seed ? 1 : 0;
  }
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < Q.ncols; c += stride) cnt_all[c] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Q.ctr[0] = 0;
    Q.ctr[1] = n_seed;
    Q.ctr[2] = Q.F;
    Q.ctr[3] = 0;  // abort flag
  }
}

}  // namespace

// Rows of one A^T piece: as many as fit `piece_cap` bytes (a multiple of 8),
// spread evenly over the row chunks of a tile.
int task_rows_per_piece(int et, int m, int piece_cap) {
  const int eb = elem_bytes(et);
  const int max_rows = std::min(round8(m), (piece_cap / (kTW * eb)) / 8 * 8);
  if (max_rows < 8) return 0;
  const int nrc = (m + max_rows - 1) / max_rows;
  return round8((m + nrc - 1) / nrc);
}

void task_plan(TaskProblem& P, int R, size_t task_bytes, int rp) {
  const GaussLayout& L = P.L;
  const int m = L.m, eb = elem_bytes(L.et), ntile = L.ns / kTW;
  P.rp = rp;
  P.nrc = (m + rp - 1) / rp;
  P.nrb = (m + std::min(128, rp) - 1) / std::min(128, rp);
  P.rpw = round8((m + P.nrb - 1) / P.nrb);
  const size_t tile = static_cast<size_t>(m) * kTW * eb;
  P.TB = static_cast<int>(std::max<size_t>(1, std::min<size_t>(ntile, task_bytes / tile)));
  P.TB = std::max(1, std::min(P.TB, kMaxTaskPieces / P.nrc));
  P.ngb = (ntile + P.TB - 1) / P.TB;
  const size_t wpiece = static_cast<size_t>(P.rpw) * kTW * eb;
  P.TBW = static_cast<int>(std::max<size_t>(1, std::min<size_t>(ntile, task_bytes / wpiece)));
  P.ncw = (ntile + P.TBW - 1) / P.TBW;
  int tot = 0;
  for (int ph = 0; ph <= last_phase(P); ++ph) tot += phase_tasks(P, ph);
  P.tasks_per_col = tot;
  P.wstride = (m * R + 3) & ~3;
  P.astride = (m + 3) & ~3;
}

size_t task_smem_bytes(int R, int /*et*/, int m_max, int ns_max, int rho_max, int stages,
                       int piece_bytes) {
  return tcarve(R, m_max, ns_max, rho_max, stages, piece_bytes).total;
}

cudaError_t task_prepare(int R, int et, size_t smem) {
  (void)smem;
  return cudaFuncSetAttribute(pick(R, et), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_optin_limit());
}

int task_ctas_per_sm(int R, int et, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick(R, et), kThreadsAll, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// seed: device array of the first tasks (n_seed), cnt_all: ncols counters
// (the problems' cnt pointers point into it).
cudaError_t task_launch_seeded(const TaskQueue& Q, const unsigned long long* seed, int n_seed,
                               int* cnt_all, int R, int et, const TaskShape& S, int m_max,
                               int ns_max, int rho_max, cudaStream_t s) {
  reset_kernel<<<64, 256, 0, s>>>(Q, seed, n_seed, cnt_all);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  void* f = pick(R, et);
  int stages = S.stages, pbytes = S.piece_bytes;
  void* args[] = {const_cast<TaskQueue*>(&Q), &stages, &pbytes, &m_max, &ns_max, &rho_max};
  return cudaLaunchKernel(f, dim3(S.grid), dim3(kThreadsAll), args, S.smem, s);
}

}  // namespace lrs
