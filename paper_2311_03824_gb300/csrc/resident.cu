// Launch side of the register-resident cluster engine (kernel body in
// resident_impl.cuh; one translation unit per compiled rank width): shared
// memory sizing, occupancy, the cluster launch, and the repack of A_k into
// the engine's register-order layout.
#include <algorithm>

#include "resident_impl.cuh"

namespace lrs {
void* res_kernel_r2(int MR);
void* res_kernel_r3(int MR);
void* res_kernel_r4(int MR);
void* res_kernel_r5(int MR);
void* res_kernel_r6(int MR);
void* res_kernel_r8(int MR);

namespace {

void* pick(int R, int MR) {
  switch (R) {
    case 2: return res_kernel_r2(MR);
    case 3: return res_kernel_r3(MR);
    case 4: return res_kernel_r4(MR);
    case 5: return res_kernel_r5(MR);
    case 6: return res_kernel_r6(MR);
    case 8: return res_kernel_r8(MR);
    default: return nullptr;
  }
}

// One thread per 4-column chunk of one row of one column: A (row-major,
// columns k0 .. k0 + kc - 1) into the register-order layout.
__global__ void res_repack_kernel(const float* A, int n, int m, int k0, int kc, int nch4, int MR,
                                  float* out) {
  const int64_t per_col = static_cast<int64_t>(m) * nch4;
  const int64_t tot = per_col * kc;
  const int m_last = m - 32 * (MR - 1);
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < tot;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int kl = static_cast<int>(t / per_col);
    const int64_t rem = t - kl * per_col;
    const int i = static_cast<int>(rem / nch4);
    const int J = static_cast<int>(rem - static_cast<int64_t>(i) * nch4);
    const float* src = A + (static_cast<int64_t>(kl) * m + i) * n;
    float4 v;
    v.x = 4 * J + 0 < n ? src[4 * J + 0] : 0.f;
    v.y = 4 * J + 1 < n ? src[4 * J + 1] : 0.f;
    v.z = 4 * J + 2 < n ? src[4 * J + 2] : 0.f;
    v.w = 4 * J + 3 < n ? src[4 * J + 3] : 0.f;
    const int c = J / kResChunks, ch = J - c * kResChunks;
    const int nchc = min(kResChunks, nch4 - kResChunks * c);
    const int p = i >> 5, l = i & 31;
    const int Lp = p < MR - 1 ? 32 : m_last;
    const int64_t off = static_cast<int64_t>(k0 + kl) * m * 4 * nch4 + static_cast<int64_t>(128) * m * c +
                        static_cast<int64_t>(p) * 128 * nchc + static_cast<int64_t>(ch) * 4 * Lp + 4 * l;
    *reinterpret_cast<float4*>(out + off) = v;
  }
}

}  // namespace

namespace {
template <int R>
size_t smem_r(int MR, int rho, int CS) {
  switch (MR) {
    case 1: return res::smem_total<R, 1>(rho, CS);
    case 2: return res::smem_total<R, 2>(rho, CS);
    case 3: return res::smem_total<R, 3>(rho, CS);
    case 4: return res::smem_total<R, 4>(rho, CS);
    case 5: return res::smem_total<R, 5>(rho, CS);
    default: return res::smem_total<R, 6>(rho, CS);
  }
}
}  // namespace

size_t res_smem_bytes(int R, int MR, int m, int rho, int CS) {
  (void)m;
  switch (R) {
    case 2: return smem_r<2>(MR, rho, CS);
    case 3: return smem_r<3>(MR, rho, CS);
    case 4: return smem_r<4>(MR, rho, CS);
    case 5: return smem_r<5>(MR, rho, CS);
    case 6: return smem_r<6>(MR, rho, CS);
    default: return smem_r<8>(MR, rho, CS);
  }
}

cudaError_t res_prepare(int R, int MR) {
  void* f = pick(R, MR);
  if (!f) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_limit());
}

int res_max_clusters(int R, int MR, int CS, size_t smem) {
  void* f = pick(R, MR);
  if (!f) return 0;
  if (CS == 1) {
    int nb = 0, dev = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kResNT, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nb * nsm;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS);
  cfg.blockDim = dim3(kResNT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, f, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return ncl;
}

cudaError_t res_launch(const ResArgs& a, int nclusters, cudaStream_t s) {
  const int R = res_rpad(a.r), MR = (a.m + 31) / 32;
  void* f = pick(R, MR);
  if (!f || nclusters < 1) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(nclusters * a.CS));
  cfg.blockDim = dim3(kResNT);
  cfg.dynamicSmemBytes = res_smem_bytes(R, MR, a.m, a.rho, a.CS);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = a.CS > 1 ? 1 : 0;
  ResArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchKernelExC(&cfg, f, args);
}

cudaError_t res_repack(const float* A_rowmajor, int n, int m, int k0, int kc, float* A_res,
                       cudaStream_t s) {
  const int nch4 = (n + 3) / 4, MR = (m + 31) / 32;
  const int64_t tot = static_cast<int64_t>(m) * nch4 * kc;
  const int blocks = static_cast<int>(std::min<int64_t>((tot + 255) / 256, 4096));
  res_repack_kernel<<<blocks, 256, 0, s>>>(A_rowmajor, n, m, k0, kc, nch4, MR, A_res);
  return cudaGetLastError();
}

}  // namespace lrs
