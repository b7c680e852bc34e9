// lrs_orthonormalize_noalloc: the Cholesky-QR2 orthonormalisation of
// lrs_orthonormalize with its scratch in a file-scope device array instead of
// memory allocated per call.
//
// Some callers cannot allocate device memory at the point where they need
// this step: an application that has already handed all device memory to its
// own pool, or a serving loop that must not stall other streams on the
// implicit synchronisation of cudaMalloc/cudaFree.  This entry point serves
// them: it calls no cudaMalloc, cudaFree or other allocating routine.  The
// price is a fixed scratch array of kNoAllocScratchBytes (about 4.6 MB) that
// every GPU which loads the library keeps until the process exits, and fixed
// size limits (n <= 65536, r <= 16).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lrs.h"
#include "lrs_internal.h"

namespace {

constexpr int64_t kNoAllocMaxN = 65536;
constexpr int kNoAllocMaxR = 16;
constexpr int kNoAllocMaxBlocks = 256;
constexpr size_t kTmpBytes = sizeof(float) * kNoAllocMaxN * kNoAllocMaxR;
constexpr size_t kPartBytes = sizeof(double) * kNoAllocMaxBlocks * kNoAllocMaxR * kNoAllocMaxR;
constexpr size_t kRfacBytes = sizeof(double) * 2 * kNoAllocMaxR * kNoAllocMaxR;
constexpr size_t kNoAllocScratchBytes = kTmpBytes + kPartBytes + kRfacBytes + 256;

// The scratch.  Host code must not use this name as a device address: its
// device address comes from cudaGetSymbolAddress, once per device, and is
// kept for the process (a context reset on that device invalidates it).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

thread_local std::string g_msg;

lrs_status fail_na(lrs_status st, const std::string& m) {
  g_msg = m;
  return st;
}

}  // namespace

extern "C" const char* lrs_noalloc_last_error(void) { return g_msg.c_str(); }

extern "C" lrs_status lrs_orthonormalize_noalloc(const float* Z, float* Q, int64_t n, int32_t r,
                                                 void* stream) {
  if (!Z || !Q) return fail_na(LRS_ERR_ARG, "lrs_orthonormalize_noalloc: NULL pointer");
  if (r < 1 || r > kNoAllocMaxR || n < r || n > kNoAllocMaxN)
    return fail_na(LRS_ERR_ARG,
                   "lrs_orthonormalize_noalloc: need 1 <= r <= 16 and r <= n <= 65536 "
                   "(the size of its fixed scratch)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail_na(LRS_ERR_CUDA, "lrs_orthonormalize_noalloc: no usable current device");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      // first call on this device (with this device current): look up the
      // device address of the scratch array
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return fail_na(LRS_ERR_CUDA, std::string("lrs_orthonormalize_noalloc: cudaGetSymbolAddress: ") +
                                         cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  float* tmp = reinterpret_cast<float*>(b);
  double* part = reinterpret_cast<double*>(b + kTmpBytes);
  double* rfac = reinterpret_cast<double*>(b + kTmpBytes + kPartBytes);
  int* err = reinterpret_cast<int*>(b + kTmpBytes + kPartBytes + kRfacBytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nblk = lrs::qr_blocks(n);
  if (nblk > kNoAllocMaxBlocks) return fail_na(LRS_ERR_UNSUPPORTED, "lrs_orthonormalize_noalloc: too many SMs");
  int eh[2] = {0, 0};
  // the array keeps the previous call's contents: the error word starts at zero
  cudaError_t e = cudaMemsetAsync(err, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess)
    e = lrs::cholqr2_into(static_cast<int>(n), r, Z, Q, tmp, part, rfac, err, nblk, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(eh, err, sizeof(eh), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess)
    return fail_na(LRS_ERR_CUDA, std::string("lrs_orthonormalize_noalloc: ") + cudaGetErrorString(e));
  if (eh[0]) return fail_na(LRS_ERR_NUMERICAL, "lrs_orthonormalize_noalloc: Z^T Z not positive definite");
  return LRS_OK;
}
