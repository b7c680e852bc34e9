// Device-side helpers shared by the solver's kernels: thread-block-cluster
// barriers and distributed-shared-memory addressing, TMA bulk copies with a
// bounded mbarrier wait, deterministic block reductions and the small FP64
// r x r Cholesky routines used by the LS step and by Cholesky-QR2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lrs_internal.h"

namespace lrs {

constexpr int kWarp = 32;

__device__ __forceinline__ void report_error(int* err, int code, int column) {
  if (err && atomicCAS(err, 0, code) == 0) err[1] = column;
}

// ---------------------------------------------------------------- cluster --
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_id_x() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
// Full cluster barrier: every thread of every CTA of the cluster arrives
// (release: its prior shared-memory writes become visible cluster-wide) and
// waits (acquire).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Generic address of the same shared-memory location in CTA `rank` of this
// cluster (distributed shared memory).
template <typename T>
__device__ __forceinline__ const T* peer_ptr(const T* p, unsigned rank) {
  uint64_t in = reinterpret_cast<uint64_t>(p), out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(in), "r"(rank));
  return reinterpret_cast<const T*>(out);
}

// ------------------------------------------------------------ TMA / mbarrier --
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// One TMA bulk (non-tensor) copy global -> this CTA's shared memory.  Both
// addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// arrive with weight n (counts as n of the barrier's expected arrivals)
__device__ __forceinline__ void mbar_arrive_local_n(uint64_t* bar, unsigned n) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(n)
               : "memory");
}
// Bounded wait: gives up after `limit` polls and returns false (the caller
// records a timeout and carries on with whatever the buffer holds, so that
// no CTA ever blocks its cluster).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  unsigned limit = (1u << 20)) {
  for (unsigned it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ------------------------------------------------------------- reductions --
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of one value per thread, returned to every thread.  Fixed order
// (butterfly inside warps, then warps in index order), so identical inputs
// give identical bits.  `scratch` holds >= blockDim.x/32 elements.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  T s = 0;
  for (int i = 0; i < nw; ++i) s += scratch[i];
  return s;
}

// Sum over threads of R per-thread values acc[0..nv); results to out[0..nv)
// (shared memory), visible to all threads on return.  Fixed order.
template <int R>
__device__ __forceinline__ void block_sum_vec(const float (&acc)[R], int nv, float* scratch,
                                              float* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float v[R];
#pragma unroll
  for (int l = 0; l < R; ++l) v[l] = warp_sum(acc[l]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int l = 0; l < R; ++l)
      if (l < nv) scratch[w * R + l] = v[l];
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    float s = 0.f;
    for (int i = 0; i < nw; ++i) s += scratch[i * R + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// ------------------------------------------------------- r x r FP64 algebra --
// 1/sqrt(s) in FP64 without a division: float estimate refined by two
// Newton-Raphson steps y <- y (3 - s y^2) / 2 (each doubles the correct bits).
__device__ __forceinline__ double rsqrt_newton(double s) {
  if (!(s > 1e-36 && s < 1e36)) return 1.0 / sqrt(s);
  double y = static_cast<double>(rsqrtf(static_cast<float>(s)));
  y = y * (1.5 - 0.5 * s * y * y);
  y = y * (1.5 - 0.5 * s * y * y);
  return y;
}

// One warp: lower Cholesky factor of the SPD r x r matrix G (row-major, ld),
// then L^{-1} (lower, into Li) with one column per lane.  Column j of L: every
// lane i >= j forms t_i = G_ij - sum_{p<j} L_ip L_jp at once (t_j is the
// pivot), so a column costs one chain of j multiply-adds, the pivot's
// reciprocal square root and one multiply (dependent FP64 operations are
// slow).  Returns false (all lanes) when a pivot is not positive relative to
// its diagonal; L and Li are then the identity.
__device__ inline bool chol_inverse_warp(const double* G, double* L, double* Li, double* iL,
                                         int r, int ld) {
  const int lane = threadIdx.x & 31;
  int ok = 1;
  for (int j = 0; j < r; ++j) {
    double t = 0.0;
    if (lane >= j && lane < r) {
      t = G[lane * ld + j];
      for (int p = 0; p < j; ++p) t = __fma_rn(-L[lane * ld + p], L[j * ld + p], t);
    }
    const double s = __shfl_sync(0xffffffffu, t, j);
    if (!(s > 1e-13 * G[j * ld + j]) || !(s < 1e300)) { ok = 0; break; }
    const double ij = rsqrt_newton(s);
    if (lane == j) {
      L[j * ld + j] = s * ij;
      iL[j] = ij;
    } else if (lane > j && lane < r) {
      L[lane * ld + j] = t * ij;
    }
    __syncwarp();
  }
  if (!ok && lane == 0)
    for (int i = 0; i < r; ++i) {
      for (int p = 0; p < r; ++p) L[i * ld + p] = (i == p) ? 1.0 : 0.0;
      iL[i] = 1.0;
    }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  if (lane < r) {
    const int cc = lane;
    for (int i = 0; i < r; ++i) {
      double t = (i == cc) ? 1.0 : 0.0;
      for (int p = cc; p < i; ++p) t -= L[i * ld + p] * Li[p * ld + cc];
      Li[i * ld + cc] = (i < cc) ? 0.0 : t * iL[i];
    }
  }
  __syncwarp();
  return ok != 0;
}

// In-place lower Cholesky of the symmetric positive definite r x r matrix
// G (row-major, lower triangle read).  Returns false when a pivot is not
// positive relative to its diagonal (the matrix is treated as not SPD).
__device__ inline bool chol_lower(const double* G, double* L, int r, int ld) {
  for (int j = 0; j < r; ++j) {
    double s = G[j * ld + j];
    for (int p = 0; p < j; ++p) s -= L[j * ld + p] * L[j * ld + p];
    if (!(s > 1e-13 * G[j * ld + j]) || !(s < 1e300)) return false;
    const double d = sqrt(s);
    L[j * ld + j] = d;
    for (int i = j + 1; i < r; ++i) {
      double t = G[i * ld + j];
      for (int p = 0; p < j; ++p) t -= L[i * ld + p] * L[j * ld + p];
      L[i * ld + j] = t / d;
    }
    for (int i = 0; i < j; ++i) L[i * ld + j] = 0.0;
  }
  return true;
}
// Solve (L L^T) x = b in place (x holds b on entry).
__device__ inline void chol_solve(const double* L, double* x, int r, int ld) {
  for (int i = 0; i < r; ++i) {
    double t = x[i];
    for (int p = 0; p < i; ++p) t -= L[i * ld + p] * x[p];
    x[i] = t / L[i * ld + i];
  }
  for (int i = r - 1; i >= 0; --i) {
    double t = x[i];
    for (int p = i + 1; p < r; ++p) t -= L[p * ld + i] * x[p];
    x[i] = t / L[i * ld + i];
  }
}

}  // namespace lrs
