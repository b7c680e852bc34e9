// Launch side of the per-column Gaussian sweep (kernel body in
// sweep_gauss_impl.cuh, one translation unit per compiled rank width so the
// build runs in parallel): shared-memory sizing, cluster launch, and the
// repacking of row-major A_k into the tiled slab layout.
#include "sweep_gauss_impl.cuh"

namespace lrs {
void* sweep_kernel_r2(int resident);
void* sweep_kernel_r3(int resident);
void* sweep_kernel_r4(int resident);
void* sweep_kernel_r5(int resident);
void* sweep_kernel_r6(int resident);
void* sweep_kernel_r8(int resident);
void* sweep_kernel_r10(int resident);
void* sweep_kernel_r12(int resident);
void* sweep_kernel_r16(int resident);

namespace {
using namespace sweep;

void* pick_kernel(int r, int resident) {
  switch (sweep_rpad(r)) {
    case 2: return sweep_kernel_r2(resident);
    case 3: return sweep_kernel_r3(resident);
    case 4: return sweep_kernel_r4(resident);
    case 5: return sweep_kernel_r5(resident);
    case 6: return sweep_kernel_r6(resident);
    case 8: return sweep_kernel_r8(resident);
    case 10: return sweep_kernel_r10(resident);
    case 12: return sweep_kernel_r12(resident);
    default: return sweep_kernel_r16(resident);
  }
}

// repack columns [k0, k0 + kc) of row-major A_k into the tiled slab layout
__global__ void repack_kernel(GaussLayout L, const float* __restrict__ Ain, int k0, int kc,
                              float* __restrict__ Aout) {
  const size_t slab = static_cast<size_t>(L.ns) * L.m;   // elements per slab
  const size_t per_col = slab * L.cs;
  const size_t total = per_col * kc;
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<size_t>(gridDim.x) * blockDim.x) {
    // t enumerates source order: column kk, row i, column j (padded to cs*ns)
    const size_t kk = t / per_col;
    const size_t rem = t - kk * per_col;
    const int i = static_cast<int>(rem / (static_cast<size_t>(L.cs) * L.ns));
    const int j = static_cast<int>(rem - static_cast<size_t>(i) * L.cs * L.ns);
    const int c = j / L.ns, jl = j - c * L.ns;
    const float v = (j < L.n) ? Ain[(kk * L.m + i) * L.n + j] : 0.f;
    const size_t dst = (static_cast<size_t>(k0) + kk) * per_col + static_cast<size_t>(c) * slab +
                       static_cast<size_t>(jl >> 5) * L.m * kTW + static_cast<size_t>(i) * kTW +
                       ((((jl & 31) >> 2) ^ (i & 7)) << 2) + (jl & 3);
    Aout[dst] = v;
  }
}

}  // namespace

size_t sweep_smem_bytes(const GaussLayout& L, int resident, int /*nthreads*/) {
  return carve(L, resident).total;
}

cudaError_t sweep_prepare(const GaussLayout& L, int nthreads) {
  for (int res = 0; res < 2; ++res) {
    void* f = pick_kernel(L.r, res);
    const size_t sm = sweep_smem_bytes(L, res, nthreads);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
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
  if (cudaOccupancyMaxActiveClusters(&nc, pick_kernel(L.r, resident), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

cudaError_t sweep_launch(const SweepArgs& a, int /*nthreads*/, cudaStream_t s) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, a.L, a.resident, a.L.q, s);
  void* f = pick_kernel(a.L.r, a.resident);
  void* args[] = {const_cast<SweepArgs*>(&a)};
  return cudaLaunchKernelExC(&cfg, f, args);
}

cudaError_t repack_gauss(const GaussLayout& L, const float* A_rowmajor, int k0, int kc,
                         float* A_int, cudaStream_t s) {
  repack_kernel<<<1024, 256, 0, s>>>(L, A_rowmajor, k0, kc, A_int);
  return cudaGetLastError();
}

}  // namespace lrs
