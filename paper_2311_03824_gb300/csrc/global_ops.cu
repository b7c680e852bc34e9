// Column-reduced steps of Algorithm 1 (the only places where the q columns
// interact) and the r-column orthonormalisation:
//   grad = sum_k h_k b_k^T                         (Section II-A, U-gradient)
//   eta  = c_eta / ||grad||_2  at t = 1            (Algorithm 1, step size)
//   U+   = Q(U - eta grad)                         (Algorithm 1, projected GD)
// The Q factor comes from Cholesky-QR2: Gram matrices and Cholesky factors
// in FP64 (r x r), the n x r products in FP32, two passes so that the
// result is orthonormal to float32 precision.  R = R2 R1 has a positive
// diagonal, so Q is the unique QR factor with positive diag(R).
// Every reduction runs in a fixed order: results are bit-reproducible.
#include "lrs_dev.cuh"
#include "lrs_internal.h"

namespace lrs {
namespace {

constexpr int kMaxR = 16;

// grad[j][l] = sum_k H[k][j] * Bk[k][l]; lane <-> j, warp w <-> k = w (mod 8).
__global__ void __launch_bounds__(256) grad_kernel(int n, int q, int r,
                                                   const float* __restrict__ H,
                                                   const float* __restrict__ Bk,
                                                   float* __restrict__ grad) {
  __shared__ float part[8][kMaxR][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  float acc[kMaxR];
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) acc[l] = 0.f;
  if (j < n) {
    for (int k = w; k < q; k += 8) {
      const float h = H[static_cast<size_t>(k) * n + j];
      const float* b = Bk + static_cast<size_t>(k) * r;
#pragma unroll
      for (int l = 0; l < kMaxR; ++l)
        if (l < r) acc[l] = fmaf(h, b[l], acc[l]);
    }
  }
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) part[w][l][lane] = acc[l];
  __syncthreads();
  for (int t = threadIdx.x; t < 32 * r; t += blockDim.x) {
    const int l = t / 32, jj = t - l * 32;
    float s = 0.f;
    for (int ww = 0; ww < 8; ++ww) s += part[ww][l][jj];
    const int jg = blockIdx.x * 32 + jj;
    if (jg < n) grad[static_cast<size_t>(jg) * r + l] = s;
  }
}

// Split form of the two column reductions above for many SMs: block (jb, ks)
// sums rows k of its k-range (warps k = w mod 8) into out[ks][j][l]; the
// finishing kernel adds the ks partials in index order (fixed order).
template <typename T>
__global__ void __launch_bounds__(256) kred_part_kernel(int n, int q, int r, int qc,
                                                        const float* __restrict__ H,
                                                        const T* __restrict__ Bk,
                                                        T* __restrict__ out) {
  __shared__ T part[8][kMaxR][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  const int k0 = blockIdx.y * qc, k1 = min(q, k0 + qc);
  T acc[kMaxR];
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) acc[l] = T(0);
  if (j < n) {
    for (int k = k0 + w; k < k1; k += 8) {
      const T h = static_cast<T>(H[static_cast<size_t>(k) * n + j]);
      const T* b = Bk + static_cast<size_t>(k) * r;
#pragma unroll
      for (int l = 0; l < kMaxR; ++l)
        if (l < r) acc[l] = fma(h, b[l], acc[l]);
    }
  }
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) part[w][l][lane] = acc[l];
  __syncthreads();
  for (int t = threadIdx.x; t < 32 * r; t += blockDim.x) {
    const int l = t / 32, jj = t - l * 32;
    T sum = T(0);
    for (int ww = 0; ww < 8; ++ww) sum += part[ww][l][jj];
    const int jg = blockIdx.x * 32 + jj;
    if (jg < n) out[(static_cast<size_t>(blockIdx.y) * n + jg) * r + l] = sum;
  }
}
template <typename T>
__global__ void kred_fin_kernel(int nr, int ks, const T* __restrict__ part, T* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nr) {
    T sum = T(0);
    for (int s = 0; s < ks; ++s) sum += part[static_cast<size_t>(s) * nr + t];
    out[t] = sum;
  }
}

// Partial FP64 Gram X^T X of the row range handled by this block (X n x r
// row-major); optionally X is first formed as U - eta*G and stored.
// part[blk][a*r+b] (a >= b filled).
__global__ void __launch_bounds__(256) gram_part_kernel(int n, int r, const float* __restrict__ X,
                                                        const float* __restrict__ Gr,
                                                        const double* __restrict__ eta,
                                                        float* __restrict__ Xout,
                                                        double* __restrict__ part) {
  __shared__ float tile[256 * kMaxR];
  const int rows = (n + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * rows, hi = min(n, lo + rows);
  double acc = 0.0;
  const int t = threadIdx.x;
  const int a = t / kMaxR, b = t - (t / kMaxR) * kMaxR;  // 16 x 16 threads
  const float e = eta ? static_cast<float>(*eta) : 0.f;
  for (int base = lo; base < hi; base += 256) {
    const int cnt = min(256, hi - base);
    __syncthreads();
    for (int u = threadIdx.x; u < cnt * r; u += blockDim.x) {
      const size_t gi = static_cast<size_t>(base) * r + u;
      float v = X[gi];
      if (Gr) v = fmaf(-e, Gr[gi], v);
      if (Xout) Xout[gi] = v;
      tile[u] = v;
    }
    __syncthreads();
    if (a < r && b <= a)
      for (int i = 0; i < cnt; ++i)
        acc += static_cast<double>(tile[i * r + a]) * static_cast<double>(tile[i * r + b]);
  }
  if (a < r && b <= a) part[static_cast<size_t>(blockIdx.x) * r * r + a * r + b] = acc;
}

// Sum the partial Grams (fixed order: lanes over blocks, then a butterfly),
// Cholesky G = L L^T, and write Rinv = L^{-T} (upper triangular, r x r
// row-major, FP64).  One block of 256 threads; warp 0 factors.
__global__ void chol_fin_kernel(int r, int nblk, const double* __restrict__ part,
                                double* __restrict__ Rinv, int* err) {
  __shared__ double G[kMaxR * kMaxR], L[kMaxR * kMaxR], Li[kMaxR * kMaxR], iL[kMaxR];
  // the partials of each entry: one warp per entry, lanes over the blocks,
  // butterfly sum (fixed order); then warp 0 factors
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = threadIdx.x >> 5; t < r * r; t += nw) {
    const int a = t / r, b = t - a * r;
    if (b > a) continue;
    double s = 0.0;
    for (int k = lane; k < nblk; k += 32) s += part[static_cast<size_t>(k) * r * r + a * r + b];
    s = warp_sum(s);
    if (lane == 0) {
      G[a * kMaxR + b] = s;
      G[b * kMaxR + a] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  if (!chol_inverse_warp(G, L, Li, iL, r, kMaxR) && threadIdx.x == 0) report_error(err, kErrNotSPD, -1);
  for (int t = lane; t < r * r; t += 32) {
    const int a = t / r, b = t - a * r;
    Rinv[a * r + b] = Li[b * kMaxR + a];
  }
}

// Y = X Rinv (row-wise, FP32 multiply of the rounded FP64 factor); optional
// partial Gram of Y as in gram_part_kernel.
__global__ void __launch_bounds__(256) apply_rinv_kernel(int n, int r, const float* __restrict__ X,
                                                         const double* __restrict__ Rinv,
                                                         float* __restrict__ Y,
                                                         double* __restrict__ part,
                                                         float* __restrict__ Ypad = nullptr,
                                                         int rpad = 0) {
  __shared__ float Rf[kMaxR * kMaxR];
  __shared__ float tile[256 * kMaxR];
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) Rf[t] = static_cast<float>(Rinv[t]);
  const int rows = (n + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * rows, hi = min(n, lo + rows);
  const int t = threadIdx.x;
  const int a = t / kMaxR, b = t - (t / kMaxR) * kMaxR;
  double acc = 0.0;
  for (int base = lo; base < hi; base += 256) {
    const int cnt = min(256, hi - base);
    __syncthreads();
    for (int u = threadIdx.x; u < cnt * r; u += blockDim.x) {
      const int i = u / r, l = u - i * r;
      const float* x = X + static_cast<size_t>(base + i) * r;
      float s = 0.f;
      for (int p = 0; p <= l; ++p) s = fmaf(x[p], Rf[p * r + l], s);
      Y[static_cast<size_t>(base + i) * r + l] = s;
      if (Ypad) Ypad[static_cast<size_t>(base + i) * rpad + l] = s;
      tile[u] = s;
    }
    __syncthreads();
    if (part && a < r && b <= a)
      for (int i = 0; i < cnt; ++i)
        acc += static_cast<double>(tile[i * r + a]) * static_cast<double>(tile[i * r + b]);
  }
  if (part && a < r && b <= a) part[static_cast<size_t>(blockIdx.x) * r * r + a * r + b] = acc;
}

// Cyclic Jacobi rotations on the symmetric r x r FP64 matrix A, in place,
// until the off-diagonal part is negligible: the diagonal then holds the
// eigenvalues.
__device__ void jacobi_sweeps(double (&A)[kMaxR][kMaxR], int r) {
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b) (a == b ? diag : off) += A[a][b] * A[a][b];
    if (off <= 1e-30 * diag) break;
    for (int p = 0; p < r - 1; ++p)
      for (int q2 = p + 1; q2 < r; ++q2) {
        if (A[p][q2] == 0.0) continue;
        const double th = (A[q2][q2] - A[p][p]) / (2.0 * A[p][q2]);
        const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int kk = 0; kk < r; ++kk) {  // A <- J^T A J
          const double akp = A[kk][p], akq = A[kk][q2];
          A[kk][p] = cs * akp - sn * akq;
          A[kk][q2] = sn * akp + cs * akq;
        }
        for (int kk = 0; kk < r; ++kk) {
          const double apk = A[p][kk], aqk = A[q2][kk];
          A[p][kk] = cs * apk - sn * aqk;
          A[q2][kk] = sn * apk + cs * aqk;
        }
      }
  }
}

// the symmetric r x r matrix summed from nblk partials (partial k at part + k r r)
__device__ void sum_partials(double (&A)[kMaxR][kMaxR], int r, int nblk,
                             const double* __restrict__ part) {
  for (int a = 0; a < r; ++a)
    for (int b = 0; b <= a; ++b) {
      double s = 0.0;
      for (int k = 0; k < nblk; ++k) s += part[static_cast<size_t>(k) * r * r + a * r + b];
      A[a][b] = s;
      A[b][a] = s;
    }
}

// eta = c_eta / sqrt(lambda_max(G)), G = grad^T grad (sum of partials), by
// cyclic Jacobi rotations on the r x r FP64 matrix.
__global__ void eta_kernel(int r, int nblk, const double* __restrict__ part, double c_eta,
                           double* __restrict__ eta, int* err) {
  if (threadIdx.x != 0) return;
  double A[kMaxR][kMaxR];
  sum_partials(A, r, nblk, part);
  jacobi_sweeps(A, r);
  double lmax = 0.0;
  for (int a = 0; a < r; ++a) lmax = fmax(lmax, A[a][a]);
  const double nrm = sqrt(lmax);
  if (!(nrm < 1e300)) report_error(err, kErrNaN, -1);
  *eta = (nrm > 0.0) ? c_eta / nrm : 0.0;
}

// Rayleigh-Ritz values: the eigenvalues of the r x r FP64 Gram P^T P (sum of
// partials) in descending order; for P = L0^T U with U an orthonormal basis of
// a converged dominant subspace they are the squared singular values of L0.
__global__ void ritz_kernel(int r, int nblk, const double* __restrict__ part,
                            double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double A[kMaxR][kMaxR];
  sum_partials(A, r, nblk, part);
  jacobi_sweeps(A, r);
  double ev[kMaxR];
  for (int a = 0; a < r; ++a) ev[a] = A[a][a];
  for (int a = 1; a < r; ++a)  // insertion sort, descending
    for (int b = a; b > 0 && ev[b] > ev[b - 1]; --b) {
      const double t = ev[b];
      ev[b] = ev[b - 1];
      ev[b - 1] = t;
    }
  for (int a = 0; a < r; ++a) out[a] = ev[a];
}

// P[k][l] = sum_j H[k][j] U[j][l]: one warp per column k.
__global__ void __launch_bounds__(256) project_kernel(int n, int q, int r,
                                                      const float* __restrict__ H,
                                                      const float* __restrict__ U,
                                                      float* __restrict__ P) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (k >= q) return;
  float acc[kMaxR];
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) acc[l] = 0.f;
  const float* h = H + static_cast<size_t>(k) * n;
  for (int j = lane; j < n; j += 32) {
    const float hv = h[j];
    const float* u = U + static_cast<size_t>(j) * r;
#pragma unroll
    for (int l = 0; l < kMaxR; ++l)
      if (l < r) acc[l] = fmaf(hv, u[l], acc[l]);
  }
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) {
    const float s = warp_sum(acc[l]);
    if (lane == 0 && l < r) P[static_cast<size_t>(k) * r + l] = s;
  }
}

// D = Ua^T Ub (r x r FP64), partials per block then a fixed-order sum.
__global__ void __launch_bounds__(256) overlap_part_kernel(int n, int r, const float* __restrict__ Ua,
                                                           const float* __restrict__ Ub,
                                                           double* __restrict__ part) {
  const int rows = (n + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * rows, hi = min(n, lo + rows);
  const int t = threadIdx.x, a = t / kMaxR, b = t - (t / kMaxR) * kMaxR;
  if (a >= r || b >= r) return;
  double s = 0.0;
  for (int i = lo; i < hi; ++i)
    s += static_cast<double>(Ua[static_cast<size_t>(i) * r + a]) *
         static_cast<double>(Ub[static_cast<size_t>(i) * r + b]);
  part[static_cast<size_t>(blockIdx.x) * r * r + a * r + b] = s;
}
__global__ void overlap_fin_kernel(int r, int nblk, const double* __restrict__ part,
                                   double* __restrict__ out) {
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[static_cast<size_t>(k) * r * r + t];
    out[t] = s;
  }
}

// sum over rows of ||Ub[j] - Ua[j] D||^2 (FP64), partial per block
__global__ void __launch_bounds__(256) resid_part_kernel(int n, int r, const float* __restrict__ Ua,
                                                         const float* __restrict__ Ub,
                                                         const double* __restrict__ D,
                                                         double* __restrict__ part) {
  __shared__ double sD[kMaxR * kMaxR];
  __shared__ double red[8];
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) sD[t] = D[t];
  __syncthreads();
  const int rows = (n + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * rows, hi = min(n, lo + rows);
  double acc = 0.0;
  for (int u = lo * r + threadIdx.x; u < hi * r; u += blockDim.x) {
    const int i = u / r, l = u - i * r;
    double s = Ub[u];
    for (int p = 0; p < r; ++p) s -= static_cast<double>(Ua[static_cast<size_t>(i) * r + p]) * sD[p * r + l];
    acc += s * s;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}
__global__ void sum_fin_kernel(int nblk, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[k];
    *out = s;
  }
}

}  // namespace

cudaError_t subspace_change(const GlobalWork& g, const float* Uold, const float* Unew,
                            double* D_rr, double* out, cudaStream_t s) {
  overlap_part_kernel<<<g.nblk, 256, 0, s>>>(g.n, g.r, Uold, Unew, g.part);
  overlap_fin_kernel<<<1, 256, 0, s>>>(g.r, g.nblk, g.part, D_rr);
  resid_part_kernel<<<g.nblk, 256, 0, s>>>(g.n, g.r, Uold, Unew, D_rr, g.part);
  sum_fin_kernel<<<1, 32, 0, s>>>(g.nblk, g.part, out);
  return cudaGetLastError();
}

cudaError_t grad_partials(const GlobalWork& g, const float* H, const float* Bk, cudaStream_t s) {
  const int qc = g.qc > 0 ? g.qc : (g.q + g.ks - 1) / g.ks;
  kred_part_kernel<float><<<dim3((g.n + 31) / 32, g.ks), 256, 0, s>>>(g.n, g.q, g.r, qc, H, Bk,
                                                                      g.gsplit);
  return cudaGetLastError();
}

cudaError_t sum_blocks(int n, int r, int nb, const float* parts, float* out, cudaStream_t s) {
  const int nr = n * r;
  kred_fin_kernel<float><<<(nr + 255) / 256, 256, 0, s>>>(nr, nb, parts, out);
  return cudaGetLastError();
}

cudaError_t grad_reduce(const GlobalWork& g, const float* H, const float* Bk, cudaStream_t s) {
  if ((g.ks > 1 || g.qc > 0) && g.gsplit) {
    const int qc = g.qc > 0 ? g.qc : (g.q + g.ks - 1) / g.ks;
    kred_part_kernel<float><<<dim3((g.n + 31) / 32, g.ks), 256, 0, s>>>(g.n, g.q, g.r, qc, H, Bk,
                                                                        g.gsplit);
    const int nr = g.n * g.r;
    kred_fin_kernel<float><<<(nr + 255) / 256, 256, 0, s>>>(nr, g.ks, g.gsplit, g.grad);
  } else {
    grad_kernel<<<(g.n + 31) / 32, 256, 0, s>>>(g.n, g.q, g.r, H, Bk, g.grad);
  }
  return cudaGetLastError();
}

cudaError_t eta_from_grad(const GlobalWork& g, double c_eta, double* eta_dev, cudaStream_t s) {
  gram_part_kernel<<<g.nblk, 256, 0, s>>>(g.n, g.r, g.grad, nullptr, nullptr, nullptr, g.part);
  eta_kernel<<<1, 32, 0, s>>>(g.r, g.nblk, g.part, c_eta, eta_dev, nullptr);
  return cudaGetLastError();
}

cudaError_t cholqr2(const GlobalWork& g, const float* Zin, float* Uout, int* err, cudaStream_t s) {
  const int rr = g.r * g.r;
  double* R1 = g.small;
  double* R2 = g.small + rr;
  gram_part_kernel<<<g.nblk, 256, 0, s>>>(g.n, g.r, Zin, nullptr, nullptr, nullptr, g.part);
  chol_fin_kernel<<<1, 256, 0, s>>>(g.r, g.nblk, g.part, R1, err);
  apply_rinv_kernel<<<g.nblk, 256, 0, s>>>(g.n, g.r, Zin, R1, g.Z, g.part);
  chol_fin_kernel<<<1, 256, 0, s>>>(g.r, g.nblk, g.part, R2, err);
  apply_rinv_kernel<<<g.nblk, 256, 0, s>>>(g.n, g.r, g.Z, R2, Uout, nullptr, g.Upad, g.rpad);
  return cudaGetLastError();
}

int qr_blocks(int64_t n) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + 63) / 64;
  const int64_t nb = want < (nsm > 0 ? nsm : 148) ? want : (nsm > 0 ? nsm : 148);
  return static_cast<int>(nb > 0 ? nb : 1);
}

cudaError_t cholqr2_into(int n, int r, const float* Z, float* Q, float* tmp, double* part,
                         double* rfac, int* err, int nblk, cudaStream_t s) {
  double* R1 = rfac;
  double* R2 = rfac + r * r;
  gram_part_kernel<<<nblk, 256, 0, s>>>(n, r, Z, nullptr, nullptr, nullptr, part);
  chol_fin_kernel<<<1, 256, 0, s>>>(r, nblk, part, R1, err);
  apply_rinv_kernel<<<nblk, 256, 0, s>>>(n, r, Z, R1, tmp, part);
  chol_fin_kernel<<<1, 256, 0, s>>>(r, nblk, part, R2, err);
  apply_rinv_kernel<<<nblk, 256, 0, s>>>(n, r, tmp, R2, Q, nullptr);
  return cudaGetLastError();
}

cudaError_t qr_step(const GlobalWork& g, float* U, const double* eta_dev, int* err,
                    cudaStream_t s) {
  const int rr = g.r * g.r;
  double* R1 = g.small;
  double* R2 = g.small + rr;
  // Z = U - eta grad, Gram(Z)
  gram_part_kernel<<<g.nblk, 256, 0, s>>>(g.n, g.r, U, g.grad, eta_dev, g.Z, g.part);
  chol_fin_kernel<<<1, 256, 0, s>>>(g.r, g.nblk, g.part, R1, err);
  // Q1 = Z R1^{-1} (into grad's buffer: grad is no longer needed), Gram(Q1)
  apply_rinv_kernel<<<g.nblk, 256, 0, s>>>(g.n, g.r, g.Z, R1, g.grad, g.part);
  chol_fin_kernel<<<1, 256, 0, s>>>(g.r, g.nblk, g.part, R2, err);
  apply_rinv_kernel<<<g.nblk, 256, 0, s>>>(g.n, g.r, g.grad, R2, U, nullptr, g.Upad, g.rpad);
  return cudaGetLastError();
}

cudaError_t project_cols(const GlobalWork& g, const float* H, const float* U, float* P,
                         cudaStream_t s) {
  project_kernel<<<(g.q + 7) / 8, 256, 0, s>>>(g.n, g.q, g.r, H, U, P);
  return cudaGetLastError();
}

// Z <- Z - Ua D with D = Ua^T Z (n x r row-major FP32, D r x r FP64): the
// components of Z along the orthonormal columns of Ua removed.
__global__ void __launch_bounds__(256) deflate_kernel(int n, int r, float* __restrict__ Z,
                                                      const float* __restrict__ Ua,
                                                      const double* __restrict__ D) {
  __shared__ double sD[kMaxR * kMaxR];
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) sD[t] = D[t];
  __syncthreads();
  const size_t total = static_cast<size_t>(n) * r;
  for (size_t u = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; u < total;
       u += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t i = u / r;
    const int b = static_cast<int>(u - i * r);
    double acc = Z[u];
    for (int a = 0; a < r; ++a) acc -= static_cast<double>(Ua[i * r + a]) * sD[a * r + b];
    Z[u] = static_cast<float>(acc);
  }
}

cudaError_t deflate(const GlobalWork& g, const float* Ua, float* Z, double* D, cudaStream_t s) {
  overlap_part_kernel<<<g.nblk, 256, 0, s>>>(g.n, g.r, Ua, Z, g.part);
  overlap_fin_kernel<<<1, 256, 0, s>>>(g.r, g.nblk, g.part, D);
  deflate_kernel<<<g.nblk, 256, 0, s>>>(g.n, g.r, Z, Ua, D);
  return cudaGetLastError();
}

cudaError_t ritz_values(int rows, int r, const float* P, double* part, int nblk, double* out,
                        cudaStream_t s) {
  gram_part_kernel<<<nblk, 256, 0, s>>>(rows, r, P, nullptr, nullptr, nullptr, part);
  ritz_kernel<<<1, 32, 0, s>>>(r, nblk, part, out);
  return cudaGetLastError();
}

cudaError_t subspace_overlap(const GlobalWork& g, const float* Ua, const float* Ub,
                             double* out_rr, cudaStream_t s) {
  overlap_part_kernel<<<g.nblk, 256, 0, s>>>(g.n, g.r, Ua, Ub, g.part);
  overlap_fin_kernel<<<1, 256, 0, s>>>(g.r, g.nblk, g.part, out_rr);
  return cudaGetLastError();
}

}  // namespace lrs
