// Launch side of the per-column Gaussian sweep (kernel body in
// sweep_gauss_impl.cuh, one translation unit per compiled rank width so the
// build runs in parallel): shared-memory sizing, cluster launch, and the
// repacking of row-major A_k into the tiled slab layout.
#include "sweep_gauss_impl.cuh"

namespace lrs {
void* sweep_kernel_r2(int resident, int et);
void* sweep_kernel_r3(int resident, int et);
void* sweep_kernel_r4(int resident, int et);
void* sweep_kernel_r5(int resident, int et);
void* sweep_kernel_r6(int resident, int et);
void* sweep_kernel_r8(int resident, int et);
void* sweep_kernel_r10(int resident, int et);
void* sweep_kernel_r12(int resident, int et);
void* sweep_kernel_r16(int resident, int et);

namespace {
using namespace sweep;

void* pick_kernel(int r, int resident, int et) {
  switch (sweep_rpad(r)) {
    case 2: return sweep_kernel_r2(resident, et);
    case 3: return sweep_kernel_r3(resident, et);
    case 4: return sweep_kernel_r4(resident, et);
    case 5: return sweep_kernel_r5(resident, et);
    case 6: return sweep_kernel_r6(resident, et);
    case 8: return sweep_kernel_r8(resident, et);
    case 10: return sweep_kernel_r10(resident, et);
    case 12: return sweep_kernel_r12(resident, et);
    default: return sweep_kernel_r16(resident, et);
  }
}

__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// e4m3 code of v (round to nearest even, saturated to +-448) and its value
__device__ __forceinline__ unsigned char to_e4m3(float v) {
  return static_cast<unsigned char>(__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3));
}
__device__ __forceinline__ float e4m3_value(unsigned char c) {
  __nv_fp8_e4m3 f;
  f.__x = c;
  return static_cast<float>(f);
}

// Per-row scales of the FP8 forms for columns [k0, k0 + kc): one warp per row
// (k, i).  hi = e4m3(A / s1) with s1 = max_j |A(i, j)| / 448 (the largest
// finite e4m3 value); for the hi/lo form, lo = e4m3((A - s1 hi) / s2) with
// s2 = max_j |A(i, j) - s1 hi(i, j)| / 448, the residual A - s1 hi rounded once
// (fused multiply-add).  An all-zero row takes scale 1.
__global__ void rowscale_kernel(GaussLayout L, const float* __restrict__ Ain, int k0, int kc,
                                float* __restrict__ rscale) {
  const int lane = threadIdx.x & 31;
  const long nw = (static_cast<long>(gridDim.x) * blockDim.x) >> 5;
  const int per = L.et == 3 ? 2 : 1;
  for (long row = (static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
       row < static_cast<long>(kc) * L.m; row += nw) {
    const float* a = Ain + row * L.n;
    float mx = 0.f;
    for (int j = lane; j < L.n; j += 32) mx = fmaxf(mx, fabsf(a[j]));
    mx = warp_max(mx);
    const float s1 = mx > 0.f ? mx / 448.f : 1.f;
    float s2 = 1.f;
    if (per == 2) {
      float mr = 0.f;
      for (int j = lane; j < L.n; j += 32)
        mr = fmaxf(mr, fabsf(fmaf(-e4m3_value(to_e4m3(a[j] / s1)), s1, a[j])));
      mr = warp_max(mr);
      s2 = mr > 0.f ? mr / 448.f : 1.f;
    }
    if (lane == 0) {
      const size_t o = (static_cast<size_t>(k0) * L.m + row) * per;
      rscale[o] = s1;
      if (per == 2) rscale[o + 1] = s2;
    }
  }
}

// repack columns [k0, k0 + kc) of row-major FP32 A_k into the tiled slab
// layout of element type ET (FP8 forms use the row scales already written)
template <int ET>
__global__ void repack_kernel(GaussLayout L, const float* __restrict__ Ain, int k0, int kc,
                              unsigned char* __restrict__ Aout, const float* __restrict__ rscale) {
  const size_t tb = static_cast<size_t>(L.m) * kTW * elem_bytes(ET);  // bytes per tile
  const size_t slab = static_cast<size_t>(L.ns / kTW) * tb;          // bytes per slab
  const size_t per_col = static_cast<size_t>(L.cs) * L.ns * L.m;     // elements per column
  const size_t total = per_col * kc;
  constexpr int pb = ET == 0 ? 4 : ET == 1 ? 2 : 1;                  // bytes per element of a plane
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<size_t>(gridDim.x) * blockDim.x) {
    // t enumerates source order: column kk, row i, column j (padded to cs*ns)
    const size_t kk = t / per_col;
    const size_t rem = t - kk * per_col;
    const int i = static_cast<int>(rem / (static_cast<size_t>(L.cs) * L.ns));
    const int j = static_cast<int>(rem - static_cast<size_t>(i) * L.cs * L.ns);
    const int c = j / L.ns, jl = j - c * L.ns;
    const float v = (j < L.n) ? Ain[(kk * L.m + i) * L.n + j] : 0.f;
    unsigned char* dst = Aout + ((static_cast<size_t>(k0) + kk) * L.cs + c) * slab +
                         static_cast<size_t>(jl >> 5) * tb +
                         static_cast<size_t>(i * kTW + ((((jl & 31) >> 2) ^ (i & 7)) << 2) + (jl & 3)) * pb;
    if constexpr (ET == 0) {
      *reinterpret_cast<float*>(dst) = v;
    } else if constexpr (ET == 1) {
      *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
    } else {
      const size_t ro = ((static_cast<size_t>(k0) + kk) * L.m + i) * (ET == 3 ? 2 : 1);
      const float s1 = rscale[ro];
      const unsigned char hi = to_e4m3(v / s1);
      dst[0] = hi;
      if constexpr (ET == 3) {
        const float s2 = rscale[ro + 1];
        dst[static_cast<size_t>(L.m) * kTW] = to_e4m3(fmaf(-e4m3_value(hi), s1, v) / s2);
      }
    }
  }
}

// Defect correction of the low-precision forms: for column k (one block),
// x_k = U b_k + s_k (kept in xbuf row k), then
// ycorr_k(i) = y_k(i) - sum_j (A_k(i, j) - Atilde_k(i, j)) x_k(j)
// with A the exact FP32 operator (row-major) and Atilde the stored form.
template <int ET>
__global__ void refine_kernel(GaussLayout L, const float* __restrict__ Aex,
                              const unsigned char* __restrict__ Aq, const float* __restrict__ rscale,
                              const float* __restrict__ U, const float* __restrict__ Bk,
                              const int* __restrict__ S_idx, const float* __restrict__ S_val,
                              const float* __restrict__ y, float* __restrict__ ycorr,
                              float* __restrict__ xbuf) {
  const int k = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
  const int n = L.n, m = L.m, r = L.r;
  float* x = xbuf + static_cast<size_t>(k) * n;
  for (int j = tid; j < n; j += blockDim.x) {
    float v = 0.f;
    for (int l = 0; l < r; ++l)
      v = fmaf(U[static_cast<size_t>(j) * r + l], Bk[static_cast<size_t>(k) * r + l], v);
    x[j] = v;
  }
  __syncthreads();
  for (int e = tid; e < L.rho; e += blockDim.x) {
    const int j = S_idx[static_cast<size_t>(k) * L.rho + e];
    if (j >= 0 && j < n) atomicAdd(&x[j], S_val[static_cast<size_t>(k) * L.rho + e]);
  }
  __syncthreads();
  const size_t slab = static_cast<size_t>(L.ns / kTW) * m * kTW * elem_bytes(ET);
  const int per = ET == 3 ? 2 : 1;
  for (int i = tid >> 5; i < m; i += blockDim.x >> 5) {
    const float* arow = Aex + (static_cast<size_t>(k) * m + i) * n;
    const size_t ro = (static_cast<size_t>(k) * m + i) * per;
    const float s1 = ET >= 2 ? rscale[ro] : 0.f, s2 = ET == 3 ? rscale[ro + 1] : 0.f;
    float d = 0.f;
    for (int j = lane; j < n; j += 32) {
      const int c = j / L.ns, jl = j - c * L.ns;
      const float at = elem1s<ET>(Aq + (static_cast<size_t>(k) * L.cs + c) * slab, m, i, jl, s1, s2);
      d = fmaf(arow[j] - at, x[j], d);
    }
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) ycorr[static_cast<size_t>(k) * m + i] = y[static_cast<size_t>(k) * m + i] - d;
  }
}

}  // namespace

size_t sweep_smem_bytes(const GaussLayout& L, int resident, int /*nthreads*/) {
  return carve(L, resident).total;
}

cudaError_t sweep_prepare(const GaussLayout& L, int /*nthreads*/) {
  for (int res = 0; res < 2; ++res) {
    void* f = pick_kernel(L.r, res, L.et);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_optin_limit());
    if (e != cudaSuccess) cudaGetLastError();
    e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) cudaGetLastError();
  }
  return cudaSuccess;
}

static void fill_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, const GaussLayout& L,
                        int resident, int ncols, cudaStream_t s) {
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3(static_cast<unsigned>(ncols) * L.cs, 1, 1);
  cfg.blockDim = dim3(kThreadsAll, 1, 1);
  cfg.dynamicSmemBytes = sweep_smem_bytes(L, resident, kThreadsAll);
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = L.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

int sweep_max_active_clusters(const GaussLayout& L, int resident, int /*nthreads*/) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, L, resident, L.q, nullptr);
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, pick_kernel(L.r, resident, L.et), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

cudaError_t sweep_launch(const SweepArgs& a, int /*nthreads*/, cudaStream_t s) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, a.L, a.resident, a.L.q, s);
  void* f = pick_kernel(a.L.r, a.resident, a.L.et);
  void* args[] = {const_cast<SweepArgs*>(&a)};
  return cudaLaunchKernelExC(&cfg, f, args);
}

cudaError_t repack_gauss(const GaussLayout& L, const float* A_rowmajor, int k0, int kc,
                         void* A_int, float* rscale, cudaStream_t s) {
  unsigned char* out = static_cast<unsigned char*>(A_int);
  switch (L.et) {
    case 0: repack_kernel<0><<<1024, 256, 0, s>>>(L, A_rowmajor, k0, kc, out, rscale); break;
    case 1: repack_kernel<1><<<1024, 256, 0, s>>>(L, A_rowmajor, k0, kc, out, rscale); break;
    case 2:
      rowscale_kernel<<<1024, 256, 0, s>>>(L, A_rowmajor, k0, kc, rscale);
      repack_kernel<2><<<1024, 256, 0, s>>>(L, A_rowmajor, k0, kc, out, rscale);
      break;
    case 3:
      rowscale_kernel<<<1024, 256, 0, s>>>(L, A_rowmajor, k0, kc, rscale);
      repack_kernel<3><<<1024, 256, 0, s>>>(L, A_rowmajor, k0, kc, out, rscale);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t refine_residual(const GaussLayout& L, const float* A_exact, const void* A_int,
                            const float* rscale, const float* U, const float* Bk,
                            const int* S_idx, const float* S_val, const float* y, float* ycorr,
                            float* xbuf, cudaStream_t s) {
  const unsigned char* aq = static_cast<const unsigned char*>(A_int);
  const dim3 grid(static_cast<unsigned>(L.q)), block(256);
  switch (L.et) {
    case 1: refine_kernel<1><<<grid, block, 0, s>>>(L, A_exact, aq, rscale, U, Bk, S_idx, S_val, y, ycorr, xbuf); break;
    case 2: refine_kernel<2><<<grid, block, 0, s>>>(L, A_exact, aq, rscale, U, Bk, S_idx, S_val, y, ycorr, xbuf); break;
    case 3: refine_kernel<3><<<grid, block, 0, s>>>(L, A_exact, aq, rscale, U, Bk, S_idx, S_val, y, ycorr, xbuf); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lrs
