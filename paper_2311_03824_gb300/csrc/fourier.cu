// AltGDmin-LR+S for the row-masked 2D DFT operator (the Fourier / dynamic-MRI
// case of Section I-A): A_k x = (F2 x)[Omega_k], A_k^H v = F2^H(zero-fill_k v),
// F2 the unitary 2D DFT of an nx x ny frame, rows indexed kx*ny + ky in natural
// order.  Complex throughout: transposes become conjugate transposes and
// HardThreshold ranks by the modulus.
//
// Per GDmin iteration (Algorithm 1):
//   FU = F2 U                      r forward 2D FFTs (shared by all frames),
//                                  so W_k = A_k U = FU[Omega_k, :]
//   sweep (one CTA per frame k)    G_k = W_k^H W_k and its inverse (FP64),
//                                  IHT: A s and A g_G as sparse DFTs, g = A^H u
//                                  as one inverse 2D FFT of the frame held in
//                                  shared memory, HardThreshold by radix select,
//                                  then b_k and res_k = W_k b_k + A_k s_k - y_k
//   K = sum_k zero-fill_k(res_k) b_k^H   k-space accumulation through the
//                                  inverse index of the masks (fixed order)
//   grad = F2^H K                  r inverse 2D FFTs (linearity of F2)
//   eta at t = 1, U <- Q(U - eta grad) by complex Cholesky-QR2 (FP64 r x r).
// The initialisation forms L0 = [A_k^H (y_k - A_k s_k)] and its top-r left
// singular subspace by FP64 complex subspace iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lrs_dev.cuh"
#include "lrs_internal.h"

namespace lrs {
namespace fourier {

constexpr int kFT = 512;   // threads of the frame kernels
constexpr int kFW = kFT / 32;
// sweep profile slots: set-up and Gram, sparse DFTs, norms and vector
// updates, 2D FFTs with the frame's fills and scalings, HardThreshold, final
// stage, projections' W^H v and G^-1 solve, projections' v - W x
constexpr int kFProf = 8;
// static shared memory of the sweep (its profile counters), an upper bound
constexpr size_t kFStaticSmem = 256;
constexpr int kMaxR = 16;

// ------------------------------------------------------------ complex --
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// acc += a * b
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
  return acc;
}
// acc += conj(a) * b
__device__ __forceinline__ float2 ccfma(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
  return acc;
}
__device__ __forceinline__ double2 dcmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 dccmul(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// Double-float accumulation (a value carried as hi + lo, two float32 words:
// about 48 bits of significand on the FP32 units, whose dependent operations
// are far cheaper than FP64's on this part).  df_fma: (hi, lo) += a * b with
// the product's rounding error from an fma and the sum's from Knuth's
// two-sum.  df_add: (hi, lo) += (bh, bl).
__device__ __forceinline__ void df_fma(float& hi, float& lo, float a, float b) {
  const float p = a * b;
  const float pe = fmaf(a, b, -p);
  const float s = hi + p;
  const float bb = s - hi;
  const float se = (hi - (s - bb)) + (p - bb);
  hi = s;
  lo += se + pe;
}
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float bb = s - hi;
  const float se = (hi - (s - bb)) + (bh - bb);
  hi = s;
  lo += se + bl;
}
// warp sum of double-float values (xor butterfly: every lane ends with the
// same value, the pairs added in a fixed order)
__device__ __forceinline__ double warp_sum_df(float hi, float lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
    df_add(hi, lo, oh, ol);
  }
  return static_cast<double>(hi) + static_cast<double>(lo);
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------ 2D FFT --
// Sides that are not powers of two take a direct DFT (frames of at most
// kDirectPer * blockDim.x pixels): each thread keeps its outputs in
// registers until every thread has read the frame.
constexpr int kDirectPer = 8;

__device__ void dft_direct_smem(float2* X, int nx, int ny, bool rows, const float2* tw,
                                bool inverse) {
  const int ld = ny + 1, n = nx * ny, len = rows ? ny : nx;
  float2 acc[kDirectPer];
#pragma unroll
  for (int u = 0; u < kDirectPer; ++u) {
    const int e = threadIdx.x + u * blockDim.x;
    float2 s = make_float2(0.f, 0.f);
    if (e < n) {
      const int row = e / ny, col = e - row * ny;
      const int j = rows ? col : row;  // output frequency along the transformed side
      int idx = 0;                     // j * k mod len
      for (int k = 0; k < len; ++k) {
        float2 w = tw[idx];
        if (inverse) w.y = -w.y;
        s = cfma(rows ? X[row * ld + k] : X[k * ld + col], w, s);
        idx += j;
        if (idx >= len) idx -= len;
      }
    }
    acc[u] = s;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kDirectPer; ++u) {
    const int e = threadIdx.x + u * blockDim.x;
    if (e < n) {
      const int row = e / ny, col = e - row * ny;
      X[row * ld + col] = acc[u];
    }
  }
  __syncthreads();
}

// Two radix-2 decimation-in-time stages s and s + 1 on the quad x0, x1, x2,
// x3 at offsets 0, h, 2h, 3h (h = 2^s) of a block of 4h: stage s pairs
// (x0, x1) and (x2, x3) with twiddle w1, stage s + 1 pairs (x0, x2) with w2a
// and (x1, x3) with w2b.  Every element gets the operations of the two
// stages run one after the other, in the same order, so the result is that
// of two single-stage passes, with one shared-memory round trip instead of two.
__device__ __forceinline__ void stage_pair(float2& x0, float2& x1, float2& x2, float2& x3,
                                           float2 w1, float2 w2a, float2 w2b, bool inverse) {
  if (inverse) {
    w1.y = -w1.y;
    w2a.y = -w2a.y;
    w2b.y = -w2b.y;
  }
  const float2 a0 = x0, a2 = x2;
  const float2 c1 = cmul(x1, w1), c3 = cmul(x3, w1);
  const float2 b0 = cadd(a0, c1), b1 = csub(a0, c1), b2 = cadd(a2, c3), b3 = csub(a2, c3);
  const float2 d2 = cmul(b2, w2a), d3 = cmul(b3, w2b);
  x0 = cadd(b0, d2);
  x2 = csub(b0, d2);
  x1 = cadd(b1, d3);
  x3 = csub(b1, d3);
}

// In-place unitary 2D FFT of the frame X (nx rows x ny columns, row stride
// ny + 1 complex) in shared memory: along the rows, then along the columns,
// each by radix-2 decimation in time (a power-of-two side, lny / lnx its
// log2) or a direct DFT (lny / lnx = -1).  tx[k] = exp(-2 pi i k / nx),
// k < nx (same for ty); inverse uses the conjugate twiddles.  All threads of
// the CTA call it.
__device__ void fft2_smem(float2* X, int nx, int ny, int lnx, int lny, const float2* tx,
                          const float2* ty, bool inverse) {
  const int ld = ny + 1, n = nx * ny;
  if (lny < 0) {
    dft_direct_smem(X, nx, ny, true, ty, inverse);
  } else {
    // rows: bit reversal, then lny stages.  Consecutive threads take the
    // same position in consecutive rows: the row stride ny + 1 puts them in
    // distinct banks, and they share the twiddle (a broadcast)
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int j = lnx >= 0 ? e >> lnx : e / nx, row = e - j * nx;
      const int p = static_cast<int>(__brev(static_cast<unsigned>(j)) >> (32 - lny));
      if (lny > 0 && p > j) {
        const float2 t = X[row * ld + j];
        X[row * ld + j] = X[row * ld + p];
        X[row * ld + p] = t;
      }
    }
    __syncthreads();
    int s = 0;
    for (; s + 1 < lny; s += 2) {  // stages s and s + 1 in one pass
      const int h = 1 << s;
      for (int b = threadIdx.x; b < n / 4; b += blockDim.x) {
        const int t = lnx >= 0 ? b >> lnx : b / nx, row = b - t * nx;
        const int j = t & (h - 1), i0 = ((t >> s) << (s + 2)) + j;
        float2* x = X + row * ld;
        stage_pair(x[i0], x[i0 + h], x[i0 + 2 * h], x[i0 + 3 * h], ty[j * (ny >> (s + 1))],
                   ty[j * (ny >> (s + 2))], ty[(j + h) * (ny >> (s + 2))], inverse);
      }
      __syncthreads();
    }
    if (s < lny) {  // a last single stage
      const int half = 1 << s, step = ny >> (s + 1);
      for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
        const int t = lnx >= 0 ? b >> lnx : b / nx, row = b - t * nx;
        const int j = t & (half - 1), i1 = ((t >> s) << (s + 1)) + j, i2 = i1 + half;
        float2 w = ty[j * step];
        if (inverse) w.y = -w.y;
        const float2 a = X[row * ld + i1], c = cmul(X[row * ld + i2], w);
        X[row * ld + i1] = cadd(a, c);
        X[row * ld + i2] = csub(a, c);
      }
      __syncthreads();
    }
  }
  // the unitary scale 1/sqrt(n) is applied by the last column pass as it
  // stores (the same multiply as a separate pass), else by a pass of its own
  const float sc = rsqrtf(static_cast<float>(n));
  bool scaled = false;
  if (lnx < 0) {
    dft_direct_smem(X, nx, ny, false, tx, inverse);
  } else {
    // columns: bit reversal, then lnx stages
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int i = lny >= 0 ? e >> lny : e / ny, col = e - i * ny;
      const int p = static_cast<int>(__brev(static_cast<unsigned>(i)) >> (32 - lnx));
      if (lnx > 0 && p > i) {
        const float2 t = X[i * ld + col];
        X[i * ld + col] = X[p * ld + col];
        X[p * ld + col] = t;
      }
    }
    __syncthreads();
    int s = 0;
    for (; s + 1 < lnx; s += 2) {  // stages s and s + 1 in one pass
      const int h = 1 << s;
      const float f = (s + 2 == lnx) ? sc : 1.f;  // the last pass scales
      for (int b = threadIdx.x; b < n / 4; b += blockDim.x) {
        const int t = lny >= 0 ? b >> lny : b / ny, col = b - t * ny;
        const int j = t & (h - 1), i0 = ((t >> s) << (s + 2)) + j;
        float2* p0 = X + i0 * ld + col;
        float2 x0 = p0[0], x1 = p0[h * ld], x2 = p0[2 * h * ld], x3 = p0[3 * h * ld];
        stage_pair(x0, x1, x2, x3, tx[j * (nx >> (s + 1))], tx[j * (nx >> (s + 2))],
                   tx[(j + h) * (nx >> (s + 2))], inverse);
        if (s + 2 == lnx) {
          x0 = make_float2(x0.x * f, x0.y * f);
          x1 = make_float2(x1.x * f, x1.y * f);
          x2 = make_float2(x2.x * f, x2.y * f);
          x3 = make_float2(x3.x * f, x3.y * f);
        }
        p0[0] = x0;
        p0[h * ld] = x1;
        p0[2 * h * ld] = x2;
        p0[3 * h * ld] = x3;
      }
      __syncthreads();
    }
    if (s < lnx) {  // a last single stage
      const int half = 1 << s, step = nx >> (s + 1);
      for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
        const int t = lny >= 0 ? b >> lny : b / ny, col = b - t * ny;
        const int j = t & (half - 1), i1 = ((t >> s) << (s + 1)) + j, i2 = i1 + half;
        float2 w = tx[j * step];
        if (inverse) w.y = -w.y;
        const float2 a = X[i1 * ld + col], c = cmul(X[i2 * ld + col], w);
        const float2 o1 = cadd(a, c), o2 = csub(a, c);
        X[i1 * ld + col] = make_float2(o1.x * sc, o1.y * sc);
        X[i2 * ld + col] = make_float2(o2.x * sc, o2.y * sc);
      }
      __syncthreads();
    }
    scaled = lnx > 0;
  }
  if (!scaled) {
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int row = e / ny, j = e - row * ny;
      X[row * ld + j].x *= sc;
      X[row * ld + j].y *= sc;
    }
    __syncthreads();
  }
}

// g = log2 G consecutive radix-2 decimation-in-time stages s .. s + g - 1 on
// the G elements x[t] at positions i0 + t h (h = 2^s, i0 = j mod h) of a block
// of G h along a side of length N.  Stage s + u pairs x[t] with x[t + d]
// (d = 2^u, bit u of t clear) with twiddle tw[(j + (t mod d) h) N / 2^(s+u+1)]:
// the butterflies of g single-stage passes, in the same order, on registers.
template <int G>
__device__ __forceinline__ void dit_group(float2 (&x)[G], int j, int h, int s, int N,
                                          const float2* tw, bool inverse) {
#pragma unroll
  for (int d = 1; d < G; d <<= 1) {
    const int sig = s + __ffs(d) - 1;  // the global stage
    const int step = N >> (sig + 1);
#pragma unroll
    for (int t = 0; t < G; ++t) {
      if (t & d) continue;
      float2 w = tw[(j + (t & (d - 1)) * h) * step];
      if (inverse) w.y = -w.y;
      const float2 a = x[t], c = cmul(x[t + d], w);
      x[t] = cadd(a, c);
      x[t + d] = csub(a, c);
    }
  }
}

// One pass of g stages over every line of one side: nl lines of N elements,
// element p of line l at X[l * ls + p * es].  Consecutive threads take the
// same group of consecutive lines (distinct banks for the row stride ny + 1,
// contiguous for columns; the twiddles are broadcasts).  With brev (the first
// pass, when a round of the CTA's threads holds whole lines) the inputs come
// from the bit-reversed positions: a round's reads all end before its writes.
// f scales the outputs.
template <int G>
__device__ void dit_pass(float2* X, int nl, int ls, int es, int N, int lN, int s,
                         const float2* tw, bool inverse, float f, bool brev) {
  const int h = 1 << s, gpl = N / G, g = __ffs(G) - 1, bd = blockDim.x;
  if (!brev) {
    for (int b = threadIdx.x; b < nl * gpl; b += bd) {
      const int line = b % nl, t = b / nl, j = t & (h - 1);
      const int i0 = ((t >> s) << (s + g)) + j;
      float2* L = X + line * ls;
      float2 x[G];
#pragma unroll
      for (int u = 0; u < G; ++u) x[u] = L[(i0 + u * h) * es];
      dit_group<G>(x, j, h, s, N, tw, inverse);
#pragma unroll
      for (int u = 0; u < G; ++u) L[(i0 + u * h) * es] = make_float2(x[u].x * f, x[u].y * f);
    }
    __syncthreads();
    return;
  }
  const int lpr = min(nl, bd / gpl);  // lines per round (>= 1: checked by the caller)
  for (int l0 = 0; l0 < nl; l0 += lpr) {
    const int b = threadIdx.x;
    const bool on = b < lpr * gpl && l0 + b % lpr < nl;
    float2 x[G];
    int line = 0, i0 = 0;
    if (on) {
      line = l0 + b % lpr;
      i0 = (b / lpr) << g;  // s = 0: h = 1, j = 0
      float2* L = X + line * ls;
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int src = static_cast<int>(__brev(static_cast<unsigned>(i0 + u)) >> (32 - lN));
        x[u] = L[src * es];
      }
      dit_group<G>(x, 0, 1, 0, N, tw, inverse);
    }
    __syncthreads();
    if (on) {
      float2* L = X + line * ls;
#pragma unroll
      for (int u = 0; u < G; ++u) L[(i0 + u) * es] = make_float2(x[u].x * f, x[u].y * f);
    }
    __syncthreads();
  }
}

// Radix-2 DIT transform of every line of one power-of-two side (lN = log2 N),
// in passes of up to kDitMax stages (a register budget: 3 in the FFT kernel,
// 2 inside the sweep); the last pass scales by f.  The bit reversal is read
// by the first pass, or (lines longer than the CTA's threads hold) swapped in
// a pass of its own.
template <int kDitMax>
__device__ __forceinline__ void dit_side(float2* X, int nl, int ls, int es, int N, int lN, const float2* tw,
                         bool inverse, float f) {
  if (lN <= 0) return;
  const bool fused = (N >> min(kDitMax, lN)) <= static_cast<int>(blockDim.x);
  if (!fused) {
    for (int e = threadIdx.x; e < nl * N; e += blockDim.x) {
      const int line = e % nl, p = e / nl;
      const int q = static_cast<int>(__brev(static_cast<unsigned>(p)) >> (32 - lN));
      if (q > p) {
        float2* L = X + line * ls;
        const float2 t = L[p * es];
        L[p * es] = L[q * es];
        L[q * es] = t;
      }
    }
    __syncthreads();
  }
  for (int s = 0; s < lN;) {
    const int g = min(kDitMax, lN - s);
    const float fs = (s + g == lN) ? f : 1.f;
    const bool br = fused && s == 0;
    switch (g) {
      case 1: dit_pass<2>(X, nl, ls, es, N, lN, s, tw, inverse, fs, br); break;
      case 2: dit_pass<4>(X, nl, ls, es, N, lN, s, tw, inverse, fs, br); break;
      default: dit_pass<(kDitMax >= 3 ? 8 : 4)>(X, nl, ls, es, N, lN, s, tw, inverse, fs, br); break;
    }
    s += g;
  }
}

// The unitary 2D FFT of the frame kernel: as fft2_smem, with every side in
// register passes of up to three stages (the bit reversal read by the first).
__device__ void fft2_dit(float2* X, int nx, int ny, int lnx, int lny, const float2* tx,
                         const float2* ty, bool inverse) {
  const int ld = ny + 1, n = nx * ny;
  const float sc = rsqrtf(static_cast<float>(n));
  if (lny < 0)
    dft_direct_smem(X, nx, ny, true, ty, inverse);
  else
    dit_side<3>(X, nx, ld, 1, ny, lny, ty, inverse, 1.f);  // rows
  bool scaled = false;
  if (lnx < 0) {
    dft_direct_smem(X, nx, ny, false, tx, inverse);
  } else {
    dit_side<3>(X, ny, 1, ld, nx, lnx, tx, inverse, sc);  // columns
    scaled = lnx > 0;
  }
  if (!scaled) {
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int row = e / ny, j = e - row * ny;
      X[row * ld + j].x *= sc;
      X[row * ld + j].y *= sc;
    }
    __syncthreads();
  }
}

struct Geo {
  int nx, ny, lnx, lny, n;  // lnx / lny: log2 of a power-of-two side, else -1
  int L, sxL, syL, lL;      // L = lcm(nx, ny), L / nx, L / ny, log2 L (or -1)
};

// row, column of pixel e = row * ny + column, and an index modulo nx (ny)
__device__ __forceinline__ int frow(const Geo& g, int e) { return g.lny >= 0 ? e >> g.lny : e / g.ny; }
__device__ __forceinline__ int fcol(const Geo& g, int e) {
  return g.lny >= 0 ? e & (g.ny - 1) : e - (e / g.ny) * g.ny;
}
__device__ __forceinline__ int fwrapx(const Geo& g, int v) { return g.lnx >= 0 ? v & (g.nx - 1) : v % g.nx; }
__device__ __forceinline__ int fwrapy(const Geo& g, int v) { return g.lny >= 0 ? v & (g.ny - 1) : v % g.ny; }
__device__ __forceinline__ int fwrapL(const Geo& g, int v) { return g.lL >= 0 ? v & (g.L - 1) : v % g.L; }

// out[f] = F2(in[f]) (or F2^H) for frames f; frames are n-vectors in natural
// row-major order (pixel kx*ny + ky), frame f at in + f*n.
__global__ void __launch_bounds__(kFT) fft_frames_kernel(Geo g, const float2* __restrict__ in,
                                                         float2* __restrict__ out, int inverse,
                                                         const float2* __restrict__ twx,
                                                         const float2* __restrict__ twy) {
  extern __shared__ __align__(16) unsigned char sm[];
  float2* X = reinterpret_cast<float2*>(sm);
  float2* tx = X + static_cast<size_t>(g.nx) * (g.ny + 1);
  float2* ty = tx + g.nx;
  const size_t f = blockIdx.x;
  for (int k = threadIdx.x; k < g.nx; k += blockDim.x) tx[k] = twx[k];
  for (int k = threadIdx.x; k < g.ny; k += blockDim.x) ty[k] = twy[k];
  for (int e = threadIdx.x; e < g.n; e += blockDim.x) {
    const int row = e / g.ny, j = e - row * g.ny;
    X[row * (g.ny + 1) + j] = in[f * g.n + e];
  }
  __syncthreads();
  fft2_dit(X, g.nx, g.ny, g.lnx, g.lny, tx, ty, inverse != 0);
  for (int e = threadIdx.x; e < g.n; e += blockDim.x) {
    const int row = e / g.ny, j = e - row * g.ny;
    out[f * g.n + e] = X[row * (g.ny + 1) + j];
  }
}

// ----------------------------------------------------------- the sweep --
struct FArgs {
  Geo g;
  int m, q, r, rho, tau, mode;
  const float2* y;      // q x m
  const int* mask;      // q x m
  const float2* FU;     // r x n (column l = F2 u_l)
  int* S_idx;           // q x rho
  float2* S_val;        // q x rho
  float2* B;            // q x r
  float2* RES;          // q x m: W b + A s - y (iteration)
  float2* H;            // q x n: L0 columns A^H (y - A s) (initialisation)
  const float2* twx;
  const float2* twy;
  const float2* twl;    // exp(-2 pi i j / L), j < L = lcm(nx, ny)
  int* err;
  float2* vecs;         // q x 3m: y, and the two m-vectors of the sweep, when
                        // they do not fit shared memory beside the frame
  float2* Wk;           // q x r x m: W_k = (F2 U)[Omega_k], gathered once per
                        // frame and sweep (row l of frame k contiguous)
  float2* AS;           // q x m: A_k s_k of the last sweep's final stage
  int* asv;             // q: 1 while AS[k] is A_k s_k of the current s_k
  unsigned long long* prof;  // optional kFProf cycle counters (thread 0 of each CTA)
};

struct FCarve {
  size_t X, tx, ty, tl, yv, dv, ev, msk, sp, pq, spo, sv, gv, G, Gi, vec, red, hist, cand, cl, ck, total;
};

// HardThreshold candidates of the threshold filter (indices and keys; the
// sort needs one thread per candidate)
constexpr int kCandCap = 512;
static_assert(kCandCap <= kFT, "one thread per threshold-filter candidate");

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared-memory carve of the sweep; with vglob the three m-vectors (y, and
// the sweep's two) live in global memory (FArgs::vecs) and take no space.
__host__ __device__ inline FCarve fcarve(const Geo& g, int m, int rho, bool vglob = false) {
  FCarve c;
  size_t o = 0;
  const int rh = rho > 0 ? rho : 1;
  const size_t mv = vglob ? 0 : al16(static_cast<size_t>(m) * 8);
  c.X = o;    o += al16(static_cast<size_t>(g.nx) * (g.ny + 1) * 8);
  c.tx = o;   o += al16(static_cast<size_t>(g.nx) * 8);
  c.ty = o;   o += al16(static_cast<size_t>(g.ny) * 8);
  c.tl = o;   o += al16(static_cast<size_t>(g.L) * 8);
  c.yv = o;   o += mv;
  c.dv = o;   o += mv;
  c.ev = o;   o += mv;
  c.msk = o;  o += al16(static_cast<size_t>(m) * 4);
  c.sp = o;   o += al16(static_cast<size_t>(rh) * 4 + 16);
  c.pq = o;   o += al16(static_cast<size_t>(rh) * 8);
  c.spo = o;  o += al16(static_cast<size_t>(rh) * 4);
  c.sv = o;   o += al16(static_cast<size_t>(rh) * 8);
  c.gv = o;   o += al16(static_cast<size_t>(rh) * 8);
  c.G = o;    o += al16(4 * kMaxR * kMaxR * 16);     // G, L, Linv, Ginv (complex FP64)
  c.vec = o;  o += al16((64 + kMaxR * kMaxR) * 16);   // c, x, scalars, iL; r x r products
  c.red = o;  o += al16(static_cast<size_t>(kFW) * 2 * kMaxR * 4 + 64);
  c.hist = o; o += al16(256 * 4 + 64);
  c.cand = o; o += al16(static_cast<size_t>(2 * rh + 64) * 4);
  c.cl = o;   o += al16(static_cast<size_t>(kCandCap) * 4);
  c.ck = o;   o += al16(static_cast<size_t>(kCandCap) * 4);
  c.total = o;
  return c;
}

struct FCtx {
  Geo g;
  int m, r, rho, k;
  float2* X;
  float2* tx;      // full-period twiddles exp(-2 pi i k / nx), k < nx
  float2* ty;
  float2* tl;      // exp(-2 pi i j / L), j < L = lcm(nx, ny)
  int2* pq;        // sparse DFT: a support pixel's row and column scaled to L
  int* spo;        // the support before the last HardThreshold
  float2* yv;
  float2* dv;
  float2* ev;
  int* msk;
  int* sp;         // support pixels
  float2* sv;      // support values
  float2* gv;      // g on the support
  double2* G;      // r x r (ld kMaxR): G, then scratch
  double2* Lc;
  double2* Li;
  double2* Gi;
  double2* vec;    // [0,16) c, [16,32) x
  float* red;
  int* hist;
  int* cand;
  int* cl;         // threshold-filter candidates: pixels
  unsigned* ck;    // and their keys
  const float2* FU;
  float2* Wk;      // this frame's W_k (r x m, row l contiguous)
  int* err;
};

__device__ __forceinline__ float2 W_at(const FCtx& C, int i, int l) {
  return C.Wk[static_cast<size_t>(l) * C.m + i];
}

// out[i] = (A x)[i] for the sparse frame x with pixels p[e], values v[e]
// (direct DFT of the nonzeros at the sampled frequencies).  With L =
// lcm(nx, ny), exp(-2 pi i (kx px / nx + ky py / ny)) is the one table entry
// j = (kx px L/nx + ky py L/ny) mod L: one look-up (or, along a run of
// pixels in a row, one complex multiply) and one complex multiply-add per
// term.
constexpr int kSdPer = 4;
__device__ void sparse_dft(const FCtx& C, const int* p, const float2* v, int nnz, float2* out) {
  const float sc = rsqrtf(static_cast<float>(C.g.n));
  for (int e = threadIdx.x; e < nnz; e += blockDim.x) {
    const int pe = p[e];
    C.pq[e] = make_int2(frow(C.g, pe) * C.g.sxL, fcol(C.g, pe) * C.g.syL);
  }
  __syncthreads();
  // each thread takes kSdPer frequencies at once, so that a term's index and
  // value (shared-memory broadcasts) serve all of them
  const int bd = blockDim.x;
  for (int i0 = threadIdx.x; i0 < C.m; i0 += kSdPer * bd) {
    int kx[kSdPer], ky[kSdPer];
    float2 wy[kSdPer], acc[kSdPer];
#pragma unroll
    for (int u = 0; u < kSdPer; ++u) {
      const int i = i0 + u * bd;
      const int om = i < C.m ? C.msk[i] : 0;
      kx[u] = frow(C.g, om);
      ky[u] = fcol(C.g, om);
      wy[u] = C.tl[fwrapL(C.g, ky[u] * C.g.syL)];  // exp(-2 pi i ky / ny)
      acc[u] = make_float2(0.f, 0.f);
    }
    // a pixel right after the previous one in its row (blob supports; the
    // pixels are ascending) takes the previous twiddle times exp(-2 pi i ky / ny)
    float2 w[kSdPer];
    int2 qp = make_int2(-1, -1);
    for (int e = 0; e < nnz; ++e) {
      const int2 q = C.pq[e];
      const float2 ve = v[e];
      if (q.x == qp.x && q.y == qp.y + C.g.syL) {  // the same for every lane
#pragma unroll
        for (int u = 0; u < kSdPer; ++u) w[u] = cmul(w[u], wy[u]);
      } else {
#pragma unroll
        for (int u = 0; u < kSdPer; ++u) w[u] = C.tl[fwrapL(C.g, kx[u] * q.x + ky[u] * q.y)];
      }
      qp = q;
#pragma unroll
      for (int u = 0; u < kSdPer; ++u) acc[u] = cfma(w[u], ve, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < kSdPer; ++u) {
      const int i = i0 + u * bd;
      if (i < C.m) out[i] = make_float2(acc[u].x * sc, acc[u].y * sc);
    }
  }
}

// rows of W a thread takes at once in the solves and projections
constexpr int kApPer = 4;

// x = G^{-1} W^H v (W^H v in FP32, block-summed in fixed order; solve FP64);
// x in C.vec[16 + l] (double2)
__device__ void fls_solve(const FCtx& C, const float2* v) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, r = C.r;
  float2 acc[kMaxR];
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) acc[l] = make_float2(0.f, 0.f);
  // kApPer rows per thread at once (their W loads independent), each sum
  // still over the thread's rows in increasing order
  const int bd = blockDim.x;
  for (int i0 = threadIdx.x; i0 < C.m; i0 += kApPer * bd) {
    float2 vi[kApPer];
#pragma unroll
    for (int u = 0; u < kApPer; ++u) {
      const int i = i0 + u * bd;
      vi[u] = i < C.m ? v[i] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int l = 0; l < kMaxR; ++l) {
      if (l < r) {
        float2 wv[kApPer];
#pragma unroll
        for (int u = 0; u < kApPer; ++u) {
          const int i = i0 + u * bd;
          wv[u] = i < C.m ? W_at(C, i, l) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kApPer; ++u)
          if (i0 + u * bd < C.m) acc[l] = ccfma(wv[u], vi[u], acc[l]);
      }
    }
  }
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) {
    if (l >= r) break;
    const float sx = warp_sumf(acc[l].x), sy = warp_sumf(acc[l].y);
    if (lane == 0) {
      C.red[(w * kMaxR + l) * 2] = sx;
      C.red[(w * kMaxR + l) * 2 + 1] = sy;
    }
  }
  __syncthreads();
  if (threadIdx.x < r) {  // the warps' partials in warp order (float32, like the sums)
    float sx = 0.f, sy = 0.f;
    for (int ww = 0; ww < kFW; ++ww) {
      sx += C.red[(ww * kMaxR + threadIdx.x) * 2];
      sy += C.red[(ww * kMaxR + threadIdx.x) * 2 + 1];
    }
    C.vec[threadIdx.x] = make_double2(sx, sy);
  }
  __syncthreads();
  // x = G^{-1} c (FP64): the r x r products in parallel, then each row's sum
  double2* prod = C.vec + 64;
  if (threadIdx.x < r * r) {
    const int a = threadIdx.x / r, b = threadIdx.x - a * r;
    prod[threadIdx.x] = dcmul(C.Gi[a * kMaxR + b], C.vec[b]);
  }
  __syncthreads();
  if (threadIdx.x < r) {
    double2 x = make_double2(0, 0);
    for (int b = 0; b < r; ++b) {
      x.x += prod[threadIdx.x * r + b].x;
      x.y += prod[threadIdx.x * r + b].y;
    }
    C.vec[16 + threadIdx.x] = x;
  }
  __syncthreads();
}

// v <- v - W x with x from fls_solve (float arithmetic).  A thread takes
// kApPer rows at once, so that the loads of W for one l are independent.
__device__ void fapply_Wx(const FCtx& C, float2* v, float sign) {
  const int bd = blockDim.x;
  for (int i0 = threadIdx.x; i0 < C.m; i0 += kApPer * bd) {
    float2 s[kApPer];
#pragma unroll
    for (int u = 0; u < kApPer; ++u) {
      const int i = i0 + u * bd;
      s[u] = i < C.m ? v[i] : make_float2(0.f, 0.f);
    }
    for (int l = 0; l < C.r; ++l) {
      const double2 xd = C.vec[16 + l];
      const float2 x = make_float2(sign * static_cast<float>(xd.x), sign * static_cast<float>(xd.y));
      float2 wv[kApPer];
#pragma unroll
      for (int u = 0; u < kApPer; ++u) {
        const int i = i0 + u * bd;
        wv[u] = i < C.m ? W_at(C, i, l) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kApPer; ++u) s[u] = cfma(wv[u], x, s[u]);
    }
#pragma unroll
    for (int u = 0; u < kApPer; ++u) {
      const int i = i0 + u * bd;
      if (i < C.m) v[i] = s[u];
    }
  }
  __syncthreads();
}

__device__ double fnorm2(const FCtx& C, const float2* v) {
  float acc = 0.f;
  for (int i = threadIdx.x; i < C.m; i += blockDim.x) acc += cabs2(v[i]);
  acc = warp_sumf(acc);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) C.red[threadIdx.x >> 5] = acc;
  __syncthreads();
  float s = 0.f;  // the warps' partials in warp order
  for (int i = 0; i < kFW; ++i) s += C.red[i];
  __syncthreads();
  return s;
}

// Hermitian Gram G = W^H W (products exact, sums in double-float, stored as
// FP64), complex Cholesky G = L L^H in FP64 (lane 0, inverse pivots by
// Newton rsqrt), L^{-1} per lane, G^{-1} = L^{-H} L^{-1}.
__device__ void fgram_factor(const FCtx& C) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, r = C.r;
  // entry t of the lower triangle: (a, b), b <= a; a lane's rows i are
  // spread over four independent double-float chains
  for (int t = w; t < r * (r + 1) / 2; t += kFW) {
    int a = 0, b = t;
    while (b > a) b -= ++a;
    // conj(W_ib) W_ia summed in double-float: exact products, ~48-bit sums
    constexpr int kCh = 4;
    float xh[kCh], xl[kCh], yh[kCh], yl[kCh];
#pragma unroll
    for (int hh = 0; hh < kCh; ++hh) xh[hh] = xl[hh] = yh[hh] = yl[hh] = 0.f;
    for (int i0 = lane; i0 < C.m; i0 += 32 * kCh) {
      float2 wa[kCh], wb[kCh];
#pragma unroll
      for (int hh = 0; hh < kCh; ++hh) {
        const int i = i0 + 32 * hh;
        wa[hh] = i < C.m ? W_at(C, i, a) : make_float2(0.f, 0.f);
        wb[hh] = i < C.m ? W_at(C, i, b) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int hh = 0; hh < kCh; ++hh) {
        df_fma(xh[hh], xl[hh], wb[hh].x, wa[hh].x);
        df_fma(xh[hh], xl[hh], wb[hh].y, wa[hh].y);
        df_fma(yh[hh], yl[hh], wb[hh].x, wa[hh].y);
        df_fma(yh[hh], yl[hh], -wb[hh].y, wa[hh].x);
      }
    }
#pragma unroll
    for (int hh = 1; hh < kCh; ++hh) {
      df_add(xh[0], xl[0], xh[hh], xl[hh]);
      df_add(yh[0], yl[0], yh[hh], yl[hh]);
    }
    const double sx = warp_sum_df(xh[0], xl[0]);
    const double sy = warp_sum_df(yh[0], yl[0]);
    if (lane == 0) {
      C.G[a * kMaxR + b] = make_double2(sx, sy);             // G[a][b] = sum conj(W_b) W_a ... (lower)
      C.G[b * kMaxR + a] = make_double2(sx, -sy);
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double* iL = reinterpret_cast<double*>(C.vec + 32);
    // G here holds G[a][b] = sum_i conj(W_ib) W_ia = (W^H W)[b][a]; factor the
    // Hermitian matrix M = W^H W with M[a][b] = conj(G[a][b]), column j by the
    // lanes i >= j at once (lane j's entry is the pivot)
    bool ok = true;
    for (int j = 0; j < r; ++j) {
      double2 t = make_double2(0.0, 0.0);
      if (lane >= j && lane < r) {
        t = make_double2(C.G[lane * kMaxR + j].x, -C.G[lane * kMaxR + j].y);
        for (int p = 0; p < j; ++p) {
          const double2 x = C.Lc[lane * kMaxR + p], y = C.Lc[j * kMaxR + p];
          // t -= L[i][p] * conj(L[j][p])
          t.x -= x.x * y.x + x.y * y.y;
          t.y -= x.y * y.x - x.x * y.y;
        }
      }
      const double sj = __shfl_sync(0xffffffffu, t.x, j);
      if (!(sj > 1e-13 * C.G[j * kMaxR + j].x) || !(sj < 1e300)) {
        ok = false;
        break;
      }
      const double ij = rsqrt_newton(sj);
      if (lane == j) {
        C.Lc[j * kMaxR + j] = make_double2(sj * ij, 0.0);
        iL[j] = ij;
      } else if (lane > j && lane < r) {
        C.Lc[lane * kMaxR + j] = make_double2(t.x * ij, t.y * ij);
      }
      __syncwarp();
    }
    if (!ok && lane == 0) {
      report_error(C.err, kErrNotSPD, C.k);
      for (int i = 0; i < r; ++i) {
        for (int p = 0; p < r; ++p) C.Lc[i * kMaxR + p] = make_double2(i == p ? 1.0 : 0.0, 0.0);
        iL[i] = 1.0;
      }
    }
    __syncwarp();
    if (lane < r) {  // column lane of L^{-1}
      const int cc = lane;
      for (int i = 0; i < r; ++i) {
        double2 t = make_double2(i == cc ? 1.0 : 0.0, 0.0);
        for (int p = cc; p < i; ++p) {
          const double2 q = dcmul(C.Lc[i * kMaxR + p], C.Li[p * kMaxR + cc]);
          t.x -= q.x;
          t.y -= q.y;
        }
        C.Li[i * kMaxR + cc] = (i < cc) ? make_double2(0, 0) : make_double2(t.x * iL[i], t.y * iL[i]);
      }
    }
    __syncwarp();
    // G^{-1} = L^{-H} L^{-1}: Gi[a][b] = sum_p conj(Li[p][a]) Li[p][b]
    for (int t = lane; t < r * r; t += 32) {
      const int a = t / r, b = t - a * r;
      double2 s = make_double2(0, 0);
      for (int p = (a > b ? a : b); p < r; ++p) {
        const double2 q = dccmul(C.Li[p * kMaxR + a], C.Li[p * kMaxR + b]);
        s.x += q.x;
        s.y += q.y;
      }
      C.Gi[a * kMaxR + b] = s;
    }
  }
  __syncthreads();
}

// HardThreshold of the frame values X (modulus; ties to the lower pixel
// index) -> the rho kept pixels and values (support order: by key).
__device__ void fhard_threshold(const FCtx& C, bool keep_values) {
  const int n = C.g.n, ld = C.g.ny + 1, rho = C.rho, lane = threadIdx.x & 31;
  int* info = C.hist + 256;
  int* sel = C.cand;            // rho entries
  auto key_of = [&](int e) {
    return __float_as_uint(cabs2(C.X[frow(C.g, e) * ld + fcol(C.g, e)]));
  };
  // Threshold filter (with a current support, after v = s - mu g): the rho
  // entries of the support have keys >= T0, their smallest key, so the rho
  // largest keys are all >= T0.  The entries at or above T0 are ranked by
  // (key descending, pixel ascending), the order of the radix path below,
  // unless there are more than kCandCap of them.
  if (keep_values) {
    if (threadIdx.x < 32) {
      unsigned mn = 0xffffffffu;
      for (int e = lane; e < rho; e += 32) mn = min(mn, key_of(C.sp[e]));
      mn = __reduce_min_sync(0xffffffffu, mn);
      if (lane == 0) {
        info[4] = static_cast<int>(mn);
        info[5] = 0;
      }
    }
    __syncthreads();
    const unsigned T0 = static_cast<unsigned>(info[4]);
    for (int e0 = threadIdx.x - lane; e0 < n; e0 += blockDim.x) {
      const int e = e0 + lane;
      unsigned key = 0u;
      bool c = false;
      if (e < n) {
        key = key_of(e);
        c = key >= T0;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, c);
      int base = 0;
      if (lane == 0 && bal) base = atomicAdd(&info[5], __popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (c) {
        const int pos = base + __popc(bal & ((1u << lane) - 1u));
        if (pos < kCandCap) {
          C.cl[pos] = e;
          C.ck[pos] = key;
        }
      }
    }
    __syncthreads();
    const int cnt = info[5];
    if (cnt >= rho && cnt <= kCandCap) {
      // bitonic sort of the candidates, descending by (key, ~pixel): the
      // order (key descending, pixel ascending); the 64-bit sort keys take
      // the place of cl and ck (adjacent, 2 kCandCap words)
      int P = 1;
      while (P < cnt) P <<= 1;
      const int t = threadIdx.x;  // blockDim.x >= kCandCap >= P
      unsigned long long mine = 0ull;
      if (t < cnt)
        mine = (static_cast<unsigned long long>(C.ck[t]) << 32) |
               static_cast<unsigned long long>(0xffffffffu - static_cast<unsigned>(C.cl[t]));
      __syncthreads();
      unsigned long long* K = reinterpret_cast<unsigned long long*>(C.cl);
      if (t < P) K[t] = mine;
      __syncthreads();
      for (int kk = 2; kk <= P; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
          const int o = t ^ j;
          if (t < P && o > t) {
            const unsigned long long x = K[t], y = K[o];
            if (((t & kk) == 0) ? (x < y) : (x > y)) {
              K[t] = y;
              K[o] = x;
            }
          }
          __syncthreads();
        }
      }
      if (t < rho) sel[t] = static_cast<int>(0xffffffffu - static_cast<unsigned>(K[t] & 0xffffffffull));
      __syncthreads();
      for (int t = threadIdx.x; t < rho; t += blockDim.x) {  // ascending by pixel
        const int e = sel[t];
        int pos = 0;
        for (int u = 0; u < rho; ++u) pos += sel[u] < e;
        C.sp[pos] = e;
        C.sv[pos] = C.X[frow(C.g, e) * ld + fcol(C.g, e)];
      }
      __syncthreads();
      return;
    }
    __syncthreads();
  }
  unsigned prefix = 0, mask = 0;
  if (threadIdx.x == 0) info[1] = rho;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int t = threadIdx.x; t < 256; t += blockDim.x) C.hist[t] = 0;
    __syncthreads();
    for (int e0 = threadIdx.x - lane; e0 < n; e0 += blockDim.x) {
      const int e = e0 + lane;
      unsigned key = 0u;
      if (e < n) {
        const int row = frow(C.g, e), col = fcol(C.g, e);
        key = __float_as_uint(cabs2(C.X[row * ld + col]));
      }
      const bool in = e < n && (key & mask) == prefix;
      const unsigned digit = in ? ((key >> shift) & 255u) : 256u;
      const unsigned peers = __match_any_sync(0xffffffffu, digit);
      if (in && (__ffs(peers) - 1) == lane) atomicAdd(&C.hist[digit], __popc(peers));
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int need = info[1];
      int own[8], tot = 0;
#pragma unroll
      for (int z = 0; z < 8; ++z) { own[z] = C.hist[255 - 8 * lane - z]; tot += own[z]; }
      int incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int excl = incl - tot;
      if (excl < need && incl >= need) {
        int acc = excl;
        for (int z = 0; z < 8; ++z) {
          if (acc + own[z] >= need) {
            info[0] = 255 - 8 * lane - z;
            info[1] = need - acc;
            break;
          }
          acc += own[z];
        }
      }
    }
    __syncthreads();
    prefix |= static_cast<unsigned>(info[0]) << shift;
    mask |= 255u << shift;
  }
  const unsigned T = prefix;
  const int need = info[1];
  int* ties = C.cand + rho + 8; // tie candidates (bounded below)
  const int tie_cap = 56;
  if (threadIdx.x == 0) { info[2] = 0; info[3] = 0; }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int row = frow(C.g, e), col = fcol(C.g, e);
    const unsigned key = __float_as_uint(cabs2(C.X[row * ld + col]));
    if (key > T) sel[atomicAdd(&info[3], 1)] = e;
    else if (key == T) {
      const int s = atomicAdd(&info[2], 1);
      if (s < tie_cap) ties[s] = e;
    }
  }
  __syncthreads();
  const int nt = min(info[2], tie_cap), ngt = info[3];
  if (info[2] > tie_cap && threadIdx.x == 0) report_error(C.err, kErrNaN, C.k);
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const int e = ties[t];
    int rank = 0;
    for (int u = 0; u < nt; ++u) rank += ties[u] < e;
    if (rank < need) sel[ngt + rank] = e;
  }
  __syncthreads();
  // store ascending by pixel (fixed order for every later sum over the support)
  for (int t = threadIdx.x; t < rho; t += blockDim.x) {
    const int e = sel[t];
    int pos = 0;
    for (int u = 0; u < rho; ++u) pos += sel[u] < e;
    const int row = frow(C.g, e), col = fcol(C.g, e);
    C.sp[pos] = e;
    C.sv[pos] = keep_values ? C.X[row * ld + col] : make_float2(0.f, 0.f);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kFT, 1) fsweep_kernel(const FArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const FCarve cv = fcarve(a.g, a.m, a.rho, a.vecs != nullptr);
  FCtx C;
  C.g = a.g;
  C.m = a.m;
  C.r = a.r;
  C.rho = a.rho;
  C.k = blockIdx.x;
  C.X = reinterpret_cast<float2*>(sm + cv.X);
  C.tx = reinterpret_cast<float2*>(sm + cv.tx);
  C.ty = reinterpret_cast<float2*>(sm + cv.ty);
  C.tl = reinterpret_cast<float2*>(sm + cv.tl);
  C.pq = reinterpret_cast<int2*>(sm + cv.pq);
  C.spo = reinterpret_cast<int*>(sm + cv.spo);
  if (a.vecs) {
    float2* v = a.vecs + static_cast<size_t>(blockIdx.x) * 3 * a.m;
    C.yv = v;
    C.dv = v + a.m;
    C.ev = v + 2 * static_cast<size_t>(a.m);
  } else {
    C.yv = reinterpret_cast<float2*>(sm + cv.yv);
    C.dv = reinterpret_cast<float2*>(sm + cv.dv);
    C.ev = reinterpret_cast<float2*>(sm + cv.ev);
  }
  C.msk = reinterpret_cast<int*>(sm + cv.msk);
  C.sp = reinterpret_cast<int*>(sm + cv.sp);
  C.sv = reinterpret_cast<float2*>(sm + cv.sv);
  C.gv = reinterpret_cast<float2*>(sm + cv.gv);
  C.G = reinterpret_cast<double2*>(sm + cv.G);
  C.Lc = C.G + kMaxR * kMaxR;
  C.Li = C.G + 2 * kMaxR * kMaxR;
  C.Gi = C.G + 3 * kMaxR * kMaxR;
  C.vec = reinterpret_cast<double2*>(sm + cv.vec);
  C.red = reinterpret_cast<float*>(sm + cv.red);
  C.hist = reinterpret_cast<int*>(sm + cv.hist);
  C.cand = reinterpret_cast<int*>(sm + cv.cand);
  C.cl = reinterpret_cast<int*>(sm + cv.cl);
  C.ck = reinterpret_cast<unsigned*>(sm + cv.ck);
  C.FU = a.FU;
  C.Wk = a.Wk + static_cast<size_t>(blockIdx.x) * a.r * a.m;
  C.err = a.err;
  const int k = C.k, m = C.m, r = C.r, rho = C.rho, n = C.g.n, ld = C.g.ny + 1;
  for (int t = threadIdx.x; t < C.g.nx; t += blockDim.x) C.tx[t] = a.twx[t];
  for (int t = threadIdx.x; t < C.g.ny; t += blockDim.x) C.ty[t] = a.twy[t];
  for (int t = threadIdx.x; t < C.g.L; t += blockDim.x) C.tl[t] = a.twl[t];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    C.yv[i] = a.y[static_cast<size_t>(k) * m + i];
    C.msk[i] = a.mask[static_cast<size_t>(k) * m + i];
  }
  for (int e = threadIdx.x; e < rho; e += blockDim.x) {
    if (a.mode != kModeInit) {
      C.sp[e] = a.S_idx[static_cast<size_t>(k) * rho + e];
      C.sv[e] = a.S_val[static_cast<size_t>(k) * rho + e];
    } else {
      C.sp[e] = 0;
      C.sv[e] = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  // phase cycle counters (profile): thread 0's clock between the CTA's phases
  // (kept in shared memory: registers are scarce in this kernel)
  __shared__ unsigned long long pc[kFProf];
  __shared__ long long tl;
  if (a.prof && threadIdx.x == 0) {
    for (int slot = 0; slot < kFProf; ++slot) pc[slot] = 0ull;
    tl = clock64();
  }
  auto mark = [&](int slot) {
    if (a.prof && threadIdx.x == 0) {
      const long long t = clock64();
      pc[slot] += static_cast<unsigned long long>(t - tl);
      tl = t;
    }
  };
  // A_k s_k of this s_k from the previous sweep's final stage (the same
  // sparse DFT of the same support, pixels and values in the same order)
  const bool as_ok = a.asv[k] != 0;
  const bool project = (a.mode != kModeInit);
  if (project) {
    // W_k = (F2 U)[Omega_k] into the frame's contiguous copy (read
    // coalesced by the Gram, the solves and the projections)
    constexpr int kG = 8;  // gathers issued together per thread
    for (int t0 = threadIdx.x; t0 < r * m; t0 += kG * blockDim.x) {
      float2 g[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < r * m) {
          const int l = t / m, i = t - l * m;
          g[u] = __ldg(C.FU + static_cast<size_t>(l) * n + C.msk[i]);
        }
      }
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < r * m) C.Wk[t] = g[u];
      }
    }
    __syncthreads();
    fgram_factor(C);
  }
  mark(0);
  const int tau = (a.mode == kModeLS || rho == 0) ? 0 : a.tau;
  // After a sweep whose HardThreshold kept the support, s_new = s - mu g_G on
  // it, so the next u = P_perp(A s_new - y) is u - mu P_perp A g_G, both of
  // which the sweep still holds (dv, ev): no sparse DFT or projection then.
  bool kept = false;
  float mu_prev = 0.f;
  for (int it = 0; it < tau; ++it) {
    const bool zero_start = (a.mode == kModeInit && it == 0);
    // u = P_perp (A s - y)
    if (zero_start) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) C.dv[i] = make_float2(-C.yv[i].x, -C.yv[i].y);
      __syncthreads();
    } else if (kept) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const float2 d = C.dv[i], e = C.ev[i];
        C.dv[i] = make_float2(fmaf(-mu_prev, e.x, d.x), fmaf(-mu_prev, e.y, d.y));
      }
      __syncthreads();
      mark(2);
    } else {
      if (it == 0 && as_ok) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) C.dv[i] = a.AS[static_cast<size_t>(k) * m + i];
      } else {
        sparse_dft(C, C.sp, C.sv, rho, C.dv);
      }
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += blockDim.x) C.dv[i] = csub(C.dv[i], C.yv[i]);
      __syncthreads();
      mark(1);
      if (project) {
        fls_solve(C, C.dv);
        mark(6);
        fapply_Wx(C, C.dv, -1.f);
        mark(7);
      }
    }
    // g = A^H u: zero-filled frame, inverse 2D FFT
    for (int e = threadIdx.x; e < C.g.nx * ld; e += blockDim.x) C.X[e] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const int om = C.msk[i];
      C.X[(frow(C.g, om)) * ld + (fcol(C.g, om))] = C.dv[i];
    }
    __syncthreads();
    fft2_smem(C.X, C.g.nx, C.g.ny, C.g.lnx, C.g.lny, C.tx, C.ty, true);
    mark(3);
    if (zero_start) {
      fhard_threshold(C, false);  // support of the zero start: the rho largest |g|
    }
    // g on the support, ||g_G||^2, A g_G
    __syncthreads();
    mark(4);
    for (int e = threadIdx.x; e < rho; e += blockDim.x) {
      const int p = C.sp[e];
      C.gv[e] = C.X[(frow(C.g, p)) * ld + (fcol(C.g, p))];
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // ||g_G||^2: lanes over the support, a fixed butterfly
      float s = 0.f;
      for (int e = threadIdx.x; e < rho; e += 32) s += cabs2(C.gv[e]);
      s = warp_sumf(s);
      if (threadIdx.x == 0) C.vec[48] = make_double2(s, 0.0);
    }
    __syncthreads();
    mark(2);
    sparse_dft(C, C.sp, C.gv, rho, C.ev);
    __syncthreads();
    mark(1);
    if (project) {
      fls_solve(C, C.ev);
      mark(6);
      fapply_Wx(C, C.ev, -1.f);
      mark(7);
    }
    const double num = C.vec[48].x;
    const double den = fnorm2(C, C.ev);
    mark(2);
    if (!(den > 0.0)) break;
    double mu = num / den;
    if (!isfinite(mu)) {
      if (threadIdx.x == 0) report_error(a.err, kErrNaN, k);
      mu = 0.0;
    }
    const float muf = static_cast<float>(mu);
    // v = s - mu g in the frame
    for (int e = threadIdx.x; e < C.g.nx * ld; e += blockDim.x) {
      C.X[e].x *= -muf;
      C.X[e].y *= -muf;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rho; e += blockDim.x) {
      const int p = C.sp[e];
      float2& x = C.X[(frow(C.g, p)) * ld + (fcol(C.g, p))];
      x = cadd(x, C.sv[e]);
    }
    __syncthreads();
    mark(3);
    for (int e = threadIdx.x; e < rho; e += blockDim.x) C.spo[e] = C.sp[e];
    __syncthreads();
    fhard_threshold(C, true);
    int same = 1;
    for (int e = threadIdx.x; e < rho; e += blockDim.x) same &= C.spo[e] == C.sp[e];
    kept = __syncthreads_and(same) != 0;
    mu_prev = muf;
    mark(4);
  }
  // ---- final stage ----
  const bool as_kept = (tau == 0 && as_ok);  // s unchanged by this sweep
  if (as_kept) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) C.dv[i] = a.AS[static_cast<size_t>(k) * m + i];
  } else {
    sparse_dft(C, C.sp, C.sv, rho, C.dv);  // A s
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {  // y - A s; A s kept for the next sweep
    const float2 as = C.dv[i];
    if (!as_kept) a.AS[static_cast<size_t>(k) * m + i] = as;
    C.dv[i] = csub(C.yv[i], as);
  }
  if (threadIdx.x == 0) a.asv[k] = 1;
  __syncthreads();
  if (a.mode == kModeInit) {
    for (int e = threadIdx.x; e < C.g.nx * ld; e += blockDim.x) C.X[e] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const int om = C.msk[i];
      C.X[(frow(C.g, om)) * ld + (fcol(C.g, om))] = C.dv[i];
    }
    __syncthreads();
    fft2_smem(C.X, C.g.nx, C.g.ny, C.g.lnx, C.g.lny, C.tx, C.ty, true);
    float2* Hk = a.H + static_cast<size_t>(k) * n;
    for (int e = threadIdx.x; e < n; e += blockDim.x) Hk[e] = C.X[(frow(C.g, e)) * ld + (fcol(C.g, e))];
  } else {
    fls_solve(C, C.dv);  // b = G^{-1} W^H (y - A s)
    if (threadIdx.x < r) {
      const double2 b = C.vec[16 + threadIdx.x];
      a.B[static_cast<size_t>(k) * r + threadIdx.x] = make_float2(static_cast<float>(b.x), static_cast<float>(b.y));
    }
    if (a.mode == kModeIter) {
      // res = W b - (y - A s)
      for (int i = threadIdx.x; i < m; i += blockDim.x) C.ev[i] = make_float2(-C.dv[i].x, -C.dv[i].y);
      __syncthreads();
      fapply_Wx(C, C.ev, 1.f);
      for (int i = threadIdx.x; i < m; i += blockDim.x) a.RES[static_cast<size_t>(k) * m + i] = C.ev[i];
    }
  }
  if (a.mode != kModeLS) {
    // S_k ascending by pixel
    for (int e = threadIdx.x; e < rho; e += blockDim.x) {
      const int p = C.sp[e];
      int pos = 0;
      for (int f = 0; f < rho; ++f) pos += C.sp[f] < p;
      a.S_idx[static_cast<size_t>(k) * rho + pos] = p;
      a.S_val[static_cast<size_t>(k) * rho + pos] = C.sv[e];
    }
  }
  mark(5);
  if (a.prof && threadIdx.x == 0)
    for (int slot = 0; slot < kFProf; ++slot) atomicAdd(a.prof + slot, pc[slot]);
}

// K[l][w] = sum over the (k, i) with mask_k[i] = w of res_k[i] conj(b_k[l]).
// One warp per frequency w (a frequency every frame samples has q entries,
// most have a few): lanes take entries lane, lane + 32, ... of its list, then
// a butterfly per component (fixed order).
__global__ void kspace_kernel(int n, int m, int r, const int* __restrict__ ptr,
                              const int* __restrict__ list, const float2* __restrict__ RES,
                              const float2* __restrict__ B, float2* __restrict__ K) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= n) return;  // uniform over the warp
  float2 acc[kMaxR];
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) acc[l] = make_float2(0.f, 0.f);
  for (int t = ptr[w] + lane; t < ptr[w + 1]; t += 32) {
    const int ki = list[t];
    const int k = ki / m;
    const float2 rv = RES[ki];
#pragma unroll
    for (int l = 0; l < kMaxR; ++l)
      if (l < r) acc[l] = cfma(rv, cconj(B[static_cast<size_t>(k) * r + l]), acc[l]);
  }
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) {
    if (l < r) {
      const float x = warp_sum(acc[l].x), y = warp_sum(acc[l].y);
      if (lane == 0) K[static_cast<size_t>(l) * n + w] = make_float2(x, y);
    }
  }
}

// ---- complex column-reduced ops on r x n column-major matrices (l-major) ----
// partial Hermitian Grams: part[blk][a][b] = sum_j conj(X_ja) X_jb (a >= b)
// Gram partials of the rows [lo, hi) of the block Y (r x n column-major):
// out[a * r + b] = sum_j conj(y_a[j]) y_b[j] (a >= b) in FP64.  Entry p of the
// lower triangle (row-major) and row group g: the rows g, g + ng, ... of the
// range; the groups are added in order afterwards.  All threads of the block.
__device__ void cgram_rows(int n, int r, const float2* __restrict__ Y, int lo, int hi,
                           double2* __restrict__ out) {
  __shared__ double2 red[256];
  const int npair = r * (r + 1) / 2, ng = max(1, static_cast<int>(blockDim.x) / npair);
  const int t = threadIdx.x, p = t % npair, g = t / npair;
  int a = 0, b = p;
  while (b > a) b -= ++a;
  double sx = 0, sy = 0;
  if (g < ng && t < 256) {
    for (int j = lo + g; j < hi; j += ng) {
      const float2 xa = Y[static_cast<size_t>(a) * n + j], xb = Y[static_cast<size_t>(b) * n + j];
      sx += static_cast<double>(xa.x) * xb.x + static_cast<double>(xa.y) * xb.y;  // conj(x_a) x_b
      sy += static_cast<double>(xa.x) * xb.y - static_cast<double>(xa.y) * xb.x;
    }
    red[t] = make_double2(sx, sy);
  }
  __syncthreads();
  if (t < npair) {
    double2 s = red[t];
    for (int gg = 1; gg < ng; ++gg) {
      s.x += red[gg * npair + t].x;
      s.y += red[gg * npair + t].y;
    }
    out[a * r + b] = s;
  }
  __syncthreads();
}
// Z = X - eta G2 on the rows [lo, hi) (float32, as the sweep's update)
__device__ void cstep_rows(int n, int r, const float2* __restrict__ X, const float2* __restrict__ G2,
                           float e, float2* __restrict__ Xout, int lo, int hi) {
  for (int j = lo + threadIdx.x; j < hi; j += blockDim.x)
    for (int l = 0; l < r; ++l) {
      float2 v = X[static_cast<size_t>(l) * n + j];
      if (G2) {
        const float2 g = G2[static_cast<size_t>(l) * n + j];
        v = make_float2(fmaf(-e, g.x, v.x), fmaf(-e, g.y, v.y));
      }
      Xout[static_cast<size_t>(l) * n + j] = v;
    }
  __syncthreads();
}
__global__ void cgram_part_kernel(int n, int r, const float2* __restrict__ X,
                                  const float2* __restrict__ G2, const double* __restrict__ eta,
                                  float2* __restrict__ Xout, double2* __restrict__ part) {
  const int rows = (n + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * rows, hi = min(n, lo + rows);
  if (Xout) cstep_rows(n, r, X, G2, eta ? static_cast<float>(*eta) : 0.f, Xout, lo, hi);
  cgram_rows(n, r, Xout ? Xout : X, lo, hi, part + static_cast<size_t>(blockIdx.x) * r * r);
}
// M = sum of partials (M[a][b] for a >= b = sum conj(x_a) x_b), Hermitian;
// M = R^H R with R = L^H (L lower from the Cholesky of M^T... we factor the
// matrix N[i][j] = sum conj(x_i) x_j directly: N = L L^H), Rinv = L^{-H}.
// (All threads of the block; the partials read through L2.)
__device__ void cchol_block(int r, int nblk, const double2* __restrict__ part,
                            double2* __restrict__ Rinv, int* err) {
  __shared__ double2 N[kMaxR * kMaxR], Lw[kMaxR * kMaxR], Li[kMaxR * kMaxR];
  __shared__ double iL[kMaxR];
  // the partials of each entry: one warp per entry, lanes over the blocks,
  // butterfly sum (fixed order); then warp 0 factors
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = threadIdx.x >> 5; t < r * r; t += nw) {
    const int a = t / r, b = t - a * r;
    if (b > a) continue;
    double sx = 0, sy = 0;
    for (int k = lane; k < nblk; k += 32) {
      const double2 v = __ldcg(part + static_cast<size_t>(k) * r * r + a * r + b);
      sx += v.x;
      sy += v.y;
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (lane == 0) {
      // N[a][b] = sum conj(x_a) x_b ; N[b][a] = conj(N[a][b])
      N[a * kMaxR + b] = make_double2(sx, sy);
      N[b * kMaxR + a] = make_double2(sx, -sy);
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // (X^H X)[i][j] = sum conj(x_i) x_j = N[i][j]: factor N = L L^H, column j
    // by the lanes i >= j at once (lane j's entry is the pivot)
    bool ok = true;
    for (int j = 0; j < r; ++j) {
      double2 t = make_double2(0.0, 0.0);
      if (lane >= j && lane < r) {
        t = N[lane * kMaxR + j];
        for (int p = 0; p < j; ++p) {
          const double2 a = Lw[lane * kMaxR + p], b = Lw[j * kMaxR + p];
          t.x -= a.x * b.x + a.y * b.y;
          t.y -= a.y * b.x - a.x * b.y;
        }
      }
      const double s = __shfl_sync(0xffffffffu, t.x, j);
      if (!(s > 1e-13 * N[j * kMaxR + j].x) || !(s < 1e300)) {
        ok = false;
        break;
      }
      const double ij = rsqrt_newton(s);
      if (lane == j) {
        Lw[j * kMaxR + j] = make_double2(s * ij, 0);
        iL[j] = ij;
      } else if (lane > j && lane < r) {
        Lw[lane * kMaxR + j] = make_double2(t.x * ij, t.y * ij);
      }
      __syncwarp();
    }
    if (!ok) {
      if (lane == 0) {
        report_error(err, kErrNotSPD, -1);
        for (int i = 0; i < r; ++i) {
          for (int p = 0; p < r; ++p) Lw[i * kMaxR + p] = make_double2(i == p ? 1.0 : 0.0, 0);
          iL[i] = 1.0;
        }
      }
    }
    __syncwarp();
    if (lane < r) {
      const int cc = lane;
      for (int i = 0; i < r; ++i) {
        double2 t = make_double2(i == cc ? 1.0 : 0.0, 0.0);
        for (int p = cc; p < i; ++p) {
          const double2 q = dcmul(Lw[i * kMaxR + p], Li[p * kMaxR + cc]);
          t.x -= q.x;
          t.y -= q.y;
        }
        Li[i * kMaxR + cc] = (i < cc) ? make_double2(0, 0) : make_double2(t.x * iL[i], t.y * iL[i]);
      }
    }
    __syncwarp();
    // X^H X = L L^H  ->  with R = L^H (upper), Q = X R^{-1} = X L^{-H}:
    // Rinv[a][b] = (L^{-H})[a][b] = conj(Li[b][a])
    for (int t = lane; t < r * r; t += 32) {
      const int a = t / r, b = t - a * r;
      const double2 v = Li[b * kMaxR + a];
      Rinv[a * r + b] = make_double2(v.x, -v.y);
    }
  }
  __syncthreads();
}
__global__ void cchol_fin_kernel(int r, int nblk, const double2* __restrict__ part,
                                 double2* __restrict__ Rinv, int* err) {
  cchol_block(r, nblk, part, Rinv, err);
}
// Y = X Rinv (column-major complex, FP64 accumulation) for the entries
// (l, j), j in [lo, hi), of the block's range; Rinv r x r (row-major).
__device__ __forceinline__ float2 capply_one(int n, int r, const float2* __restrict__ X,
                                             const double2* __restrict__ Rinv, int l, int j) {
  double sx = 0, sy = 0;
  for (int p = 0; p <= l; ++p) {
    const float2 x = X[static_cast<size_t>(p) * n + j];
    const double2 q = Rinv[p * r + l];
    sx += x.x * q.x - x.y * q.y;
    sy += x.x * q.y + x.y * q.x;
  }
  return make_float2(static_cast<float>(sx), static_cast<float>(sy));
}
__global__ void capply_kernel(int n, int r, const float2* __restrict__ X,
                              const double2* __restrict__ Rinv, float2* __restrict__ Y) {
  const size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (t >= static_cast<size_t>(n) * r) return;
  const int l = static_cast<int>(t / n), j = static_cast<int>(t - static_cast<size_t>(l) * n);
  Y[t] = capply_one(n, r, X, Rinv, l, j);
}

// Grid barrier of a cooperative launch (every block resident): thread 0
// counts in and waits, bounded by wait_ns on the global timer, for
// `target` arrivals; on expiry the launch's error flag records a timeout and
// the block goes on (its results are then void, the host reports the error).
__device__ void grid_barrier(unsigned* ctr, unsigned target, int* err, unsigned long long wait_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
      if (v >= target) break;
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > wait_ns) {
        report_error(err, kErrTimeout, -1);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
}

// The whole complex Cholesky-QR2 of Z = X - eta G2 (G2 null: Z = X) in one
// cooperative launch of nblk blocks, block b on the same rows in every
// phase: Z and its Gram partials; barrier; every block factors the Gram
// (the same sums in the same order, so the same R^{-1}) and forms its rows of
// Z2 = Z R^{-1} and their Gram partials; barrier; R2^{-1} and U = Z2 R2^{-1}.
// The arithmetic is that of the separate kernels (gram, chol, apply twice).
__global__ void __launch_bounds__(256) cqr2_fused_kernel(int n, int r, const float2* X,
                                                         const float2* __restrict__ G2,
                                                         const double* __restrict__ eta,
                                                         float2* __restrict__ Z, float2* __restrict__ Z2,
                                                         float2* Uout, double2* __restrict__ part,
                                                         double2* __restrict__ part2, unsigned* bar,
                                                         int* err, unsigned long long wait_ns) {
  __shared__ double2 Rs[kMaxR * kMaxR];
  const int nb = gridDim.x, rows = (n + nb - 1) / nb;
  const int lo = blockIdx.x * rows, hi = min(n, lo + rows);
  const float2* Y = X;
  if (G2) {
    cstep_rows(n, r, X, G2, static_cast<float>(*eta), Z, lo, hi);
    Y = Z;
  }
  cgram_rows(n, r, Y, lo, hi, part + static_cast<size_t>(blockIdx.x) * r * r);
  grid_barrier(bar, static_cast<unsigned>(nb), err, wait_ns);
  cchol_block(r, nb, part, Rs, err);
  for (int t = threadIdx.x; t < (hi - lo) * r; t += blockDim.x) {
    const int l = t / (hi - lo), j = lo + (t - l * (hi - lo));
    Z2[static_cast<size_t>(l) * n + j] = capply_one(n, r, Y, Rs, l, j);
  }
  __syncthreads();
  cgram_rows(n, r, Z2, lo, hi, part2 + static_cast<size_t>(blockIdx.x) * r * r);
  grid_barrier(bar, 2u * static_cast<unsigned>(nb), err, wait_ns);
  cchol_block(r, nb, part2, Rs, err);
  for (int t = threadIdx.x; t < (hi - lo) * r; t += blockDim.x) {
    const int l = t / (hi - lo), j = lo + (t - l * (hi - lo));
    Uout[static_cast<size_t>(l) * n + j] = capply_one(n, r, Z2, Rs, l, j);
  }
}

// eta = c / sqrt(lambda_max(grad^H grad)), from the real 2r x 2r symmetric
// embedding [[Re, -Im], [Im, Re]] of the Hermitian Gram (every eigenvalue of
// the Gram appears twice).  The embedding is summed in FP64; a cyclic Jacobi
// in FP32 (normalised by the largest diagonal entry) gives an eigenvector v of
// the largest eigenvalue, and lambda_max is the FP64 Rayleigh quotient
// v^T A v / v^T v, whose error is second order in v's error.
__global__ void ceta_kernel(int r, int nblk, const double2* __restrict__ part, double c_eta,
                            double* __restrict__ eta) {
  __shared__ double A[2 * kMaxR][2 * kMaxR];
  __shared__ float Af[2 * kMaxR][2 * kMaxR + 1], V[2 * kMaxR][2 * kMaxR + 1];
  __shared__ int best;
  const int R2 = 2 * r, lane = threadIdx.x;
  if (lane >= 32) return;
  // entries of the lower triangle, each summed over the blocks in order
  for (int t = lane; t < r * r; t += 32) {
    const int a = t / r, b = t - a * r;
    if (b > a) continue;
    double sx = 0, sy = 0;
    for (int k = 0; k < nblk; ++k) {
      const double2 v = part[static_cast<size_t>(k) * r * r + a * r + b];
      sx += v.x;
      sy += v.y;
    }
    // N[a][b] = sx + i sy, N[b][a] = sx - i sy
    A[a][b] = sx; A[b][a] = sx; A[a + r][b + r] = sx; A[b + r][a + r] = sx;
    A[a + r][b] = sy; A[b][a + r] = sy; A[a][b + r] = -sy; A[b + r][a] = -sy;
  }
  __syncwarp();
  if (lane == 0) {
    double dmax = 0.0;
    for (int a = 0; a < R2; ++a) dmax = fmax(dmax, A[a][a]);
    const double sc = dmax > 0.0 ? 1.0 / dmax : 0.0;
    for (int a = 0; a < R2; ++a)
      for (int b = 0; b < R2; ++b) {
        Af[a][b] = static_cast<float>(A[a][b] * sc);
        V[a][b] = a == b ? 1.f : 0.f;
      }
    for (int sweep = 0; sweep < 30; ++sweep) {
      float off = 0.f, diag = 0.f;
      for (int a = 0; a < R2; ++a)
        for (int b = 0; b < R2; ++b) (a == b ? diag : off) += Af[a][b] * Af[a][b];
      if (off <= 1e-13f * diag) break;
      for (int p = 0; p < R2 - 1; ++p)
        for (int q2 = p + 1; q2 < R2; ++q2) {
          const float apq = Af[p][q2];
          if (apq == 0.f) continue;
          const float th = (Af[q2][q2] - Af[p][p]) / (2.f * apq);
          const float t = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(th * th + 1.f));
          const float cs = 1.f / sqrtf(t * t + 1.f), sn = t * cs;
          for (int kk = 0; kk < R2; ++kk) {
            const float akp = Af[kk][p], akq = Af[kk][q2];
            Af[kk][p] = cs * akp - sn * akq;
            Af[kk][q2] = sn * akp + cs * akq;
            const float vkp = V[kk][p], vkq = V[kk][q2];
            V[kk][p] = cs * vkp - sn * vkq;
            V[kk][q2] = sn * vkp + cs * vkq;
          }
          for (int kk = 0; kk < R2; ++kk) {
            const float apk = Af[p][kk], aqk = Af[q2][kk];
            Af[p][kk] = cs * apk - sn * aqk;
            Af[q2][kk] = sn * apk + cs * aqk;
          }
        }
    }
    int bi = 0;
    for (int a = 1; a < R2; ++a)
      if (Af[a][a] > Af[bi][bi]) bi = a;
    best = bi;
  }
  __syncwarp();
  // Rayleigh quotient in FP64: lane a holds (A v)_a v_a and v_a^2
  double num = 0.0, den = 0.0;
  if (lane < R2) {
    double y = 0.0;
    for (int b = 0; b < R2; ++b) y += A[lane][b] * static_cast<double>(V[b][best]);
    const double va = V[lane][best];
    num = y * va;
    den = va * va;
  }
  num = warp_sum(num);
  den = warp_sum(den);
  if (lane == 0) {
    const double lmax = den > 0.0 ? fmax(0.0, num / den) : 0.0;
    const double nrm = sqrt(lmax);
    *eta = (nrm > 0.0) ? c_eta / nrm : 0.0;
  }
}

// ---- subspace iteration of the initialisation: float32 products -----------
// P[k][l] = sum_j conj(H[k][j]) U[l][j] (U column-major: column l contiguous),
// in two steps.  Partials: block (kb, c) takes the 8 columns k = 8 kb + w (one
// per warp) over the chunk c of cs rows j; the chunk's U is staged in shared
// memory 256 rows at a time and serves all 8 warps (H read once, U once per 8
// columns); lanes over j, then a warp butterfly.  Then the chunks' partials
// are added in chunk order.
constexpr int kProjRows = 256;
__global__ void __launch_bounds__(256) cproject_part_kernel(int n, int q, int r, int cs,
                                                            const float2* __restrict__ H,
                                                            const float2* __restrict__ U,
                                                            float2* __restrict__ part) {
  __shared__ float2 Us[kMaxR][kProjRows];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k = blockIdx.x * 8 + w, c = blockIdx.y;
  const int j0 = c * cs, j1 = min(n, j0 + cs);
  float2 acc[kMaxR];
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) acc[l] = make_float2(0.f, 0.f);
  for (int jb = j0; jb < j1; jb += kProjRows) {
    const int nj = min(kProjRows, j1 - jb);
    __syncthreads();
    for (int t = threadIdx.x; t < r * kProjRows; t += blockDim.x) {
      const int l = t / kProjRows, jj = t - l * kProjRows;
      Us[l][jj] = jj < nj ? U[static_cast<size_t>(l) * n + jb + jj] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (k < q)
      for (int jj = lane; jj < nj; jj += 32) {
        const float2 h = H[static_cast<size_t>(k) * n + jb + jj];
#pragma unroll
        for (int l = 0; l < kMaxR; ++l)
          if (l < r) acc[l] = ccfma(h, Us[l][jj], acc[l]);
      }
  }
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) {
    if (l >= r) break;
    const float sx = warp_sumf(acc[l].x), sy = warp_sumf(acc[l].y);
    if (lane == 0 && k < q) part[(static_cast<size_t>(c) * q + k) * r + l] = make_float2(sx, sy);
  }
}
__global__ void cproject_sum_kernel(int q, int r, int nc, const float2* __restrict__ part,
                                    float2* __restrict__ P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= q * r) return;
  float2 s = make_float2(0.f, 0.f);
  for (int c = 0; c < nc; ++c) s = cadd(s, part[static_cast<size_t>(c) * q * r + t]);
  P[t] = s;
}
// Z[l][j] = sum_k H[k][j] P[k][l]: a block holds 32 columns j; its 8 warps
// take contiguous runs of k, and their sums are added in warp (k) order
__global__ void __launch_bounds__(256) cgrad_kernel(int n, int q, int r,
                                                    const float2* __restrict__ H,
                                                    const float2* __restrict__ P,
                                                    float2* __restrict__ Z) {
  __shared__ float2 red[8][kMaxR][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  const int per = (q + 7) / 8, k0 = w * per, k1 = min(q, k0 + per);
  float2 acc[kMaxR];
#pragma unroll
  for (int l = 0; l < kMaxR; ++l) acc[l] = make_float2(0.f, 0.f);
  if (j < n)
    for (int k = k0; k < k1; ++k) {
      const float2 h = H[static_cast<size_t>(k) * n + j];
#pragma unroll
      for (int l = 0; l < kMaxR; ++l)
        if (l < r) acc[l] = cfma(h, P[static_cast<size_t>(k) * r + l], acc[l]);
    }
#pragma unroll
  for (int l = 0; l < kMaxR; ++l)
    if (l < r) red[w][l][lane] = acc[l];
  __syncthreads();
  // thread (l, lane) of the first r warps adds the 8 runs in order
  if (w < 8 && j < n)
    for (int l = w; l < r; l += 8) {
      float2 s = red[0][l][lane];
      for (int ww = 1; ww < 8; ++ww) s = cadd(s, red[ww][l][lane]);
      Z[static_cast<size_t>(l) * n + j] = s;
    }
}
// subspace change ||Un - Uo (Uo^H Un)||_F^2 of float32 blocks, in FP64:
// partials of D = Uo^H Un per row block, then per row block the residual
// (every block adds the partials of D in block order), then their sum
__global__ void coverlap_part_kernel(int n, int r, const float2* __restrict__ Uo,
                                     const float2* __restrict__ Un, double2* __restrict__ part) {
  const int rows = (n + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * rows, hi = min(n, lo + rows);
  const int t = threadIdx.x, a = t / kMaxR, b = t - (t / kMaxR) * kMaxR;
  if (a >= r || b >= r) return;
  double sx = 0, sy = 0;
  for (int j = lo; j < hi; ++j) {
    const float2 x = Uo[static_cast<size_t>(a) * n + j], y = Un[static_cast<size_t>(b) * n + j];
    sx += static_cast<double>(x.x) * y.x + static_cast<double>(x.y) * y.y;
    sy += static_cast<double>(x.x) * y.y - static_cast<double>(x.y) * y.x;
  }
  part[static_cast<size_t>(blockIdx.x) * r * r + a * r + b] = make_double2(sx, sy);
}
__global__ void cresid_part_kernel(int n, int r, int nblk, const double2* __restrict__ part,
                                   const float2* __restrict__ Uo, const float2* __restrict__ Un,
                                   double* __restrict__ rpart) {
  __shared__ double2 D[kMaxR * kMaxR];
  __shared__ double red[32];
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
    double2 s = make_double2(0, 0);
    for (int k = 0; k < nblk; ++k) {
      s.x += part[static_cast<size_t>(k) * r * r + t].x;
      s.y += part[static_cast<size_t>(k) * r * r + t].y;
    }
    D[t] = s;
  }
  __syncthreads();
  const int rows = (n + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * rows, hi = min(n, lo + rows);
  double acc = 0.0;
  for (int e = threadIdx.x; e < (hi - lo) * r; e += blockDim.x) {
    const int l = e / (hi - lo), j = lo + (e - l * (hi - lo));
    const float2 un = Un[static_cast<size_t>(l) * n + j];
    double sx = un.x, sy = un.y;
    for (int p = 0; p < r; ++p) {
      const float2 u = Uo[static_cast<size_t>(p) * n + j];
      const double2 d = D[p * r + l];
      sx -= u.x * d.x - u.y * d.y;
      sy -= u.x * d.y + u.y * d.x;
    }
    acc += sx * sx + sy * sy;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s2 = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s2 += red[w];
    rpart[blockIdx.x] = s2;
  }
}
__global__ void csum_fin_kernel(int nblk, const double* __restrict__ rpart, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s2 = 0;
  for (int k = 0; k < nblk; ++k) s2 += rpart[k];
  *out = s2;
}

}  // namespace fourier

using namespace fourier;

// --------------------------------------------------------------- driver --
struct FourierSolver {
  Geo g{};
  int m = 0, q = 0, r = 0, rho = 0;
  int tau0 = 10, tau = 3;
  double c_eta = 0.14;
  int power_iters = 1000;
  double power_tol = 1e-11;
  uint64_t seed = 0;
  cudaStream_t s = nullptr;
  int nblk = 1;
  int t = 0;
  bool have_eta = false;
  // device
  float2 *y = nullptr, *U = nullptr, *FU = nullptr, *B = nullptr, *S_val = nullptr, *RES = nullptr,
         *H = nullptr, *K = nullptr, *grad = nullptr, *Z = nullptr, *Z2 = nullptr, *twx = nullptr,
         *twl = nullptr,
         *twy = nullptr;
  int *mask = nullptr, *S_idx = nullptr, *iptr = nullptr, *ilist = nullptr, *err = nullptr;
  double2* part = nullptr;
  double2* part2 = nullptr;  // second Gram partials of the fused Cholesky-QR2
  unsigned* qbar = nullptr;  // its grid-barrier counter
  bool coop = false;         // the fused Cholesky-QR2 fits one cooperative launch
  double2* rfac = nullptr;
  double* eta = nullptr;
  double* scal = nullptr;
  float2* vecs = nullptr;  // the sweep's m-vectors in global memory (large m)
  float2* Wk = nullptr;    // q x r x m gathered W_k of the sweep
  float2* AS = nullptr;    // q x m: A_k s_k from the last sweep's final stage
  int* asv = nullptr;      // q flags: AS[k] matches the current s_k
  unsigned long long* prof = nullptr;  // kFProf sweep cycle counters (profiling)
  size_t smem = 0;
};

static size_t fft_smem(const Geo& g) {
  return al16(static_cast<size_t>(g.nx) * (g.ny + 1) * 8) + static_cast<size_t>(g.nx + g.ny) * 8;
}

static cudaError_t fft_frames(FourierSolver* F, const float2* in, float2* out, int nframes,
                              bool inverse) {
  fft_frames_kernel<<<nframes, kFT, fft_smem(F->g), F->s>>>(F->g, in, out, inverse ? 1 : 0, F->twx,
                                                             F->twy);
  return cudaGetLastError();
}

// log2 of a power of two, -1 for any other side (direct DFT)
static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return (1 << l) == v ? l : -1;
}

FourierSolver* fourier_create(int nx, int ny, int m, int q, int r, int rho, int tau0, int tau,
                              double c_eta, int power_iters, double power_tol, uint64_t seed,
                              cudaStream_t s, std::string* msg) {
  FourierSolver* F = new FourierSolver();
  F->g.nx = nx;
  F->g.ny = ny;
  F->g.lnx = ilog2(nx);
  F->g.lny = ilog2(ny);
  F->g.n = nx * ny;
  {
    int a = nx, b = ny;  // L = lcm(nx, ny) by Euclid's gcd
    while (b) {
      const int t = a % b;
      a = b;
      b = t;
    }
    F->g.L = nx / a * ny;
    F->g.sxL = F->g.L / nx;
    F->g.syL = F->g.L / ny;
    F->g.lL = ilog2(F->g.L);
  }
  F->m = m;
  F->q = q;
  F->r = r;
  F->rho = rho;
  F->tau0 = tau0;
  F->tau = tau;
  F->c_eta = c_eta;
  F->power_iters = power_iters;
  F->power_tol = power_tol;
  F->seed = seed;
  F->s = s;
  const int n = F->g.n;
  F->nblk = std::max(1, std::min(152, (n + 63) / 64));
  F->smem = fcarve(F->g, m, rho).total;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  {  // the fused Cholesky-QR2 needs all its blocks resident at once
    int coop = 0, nsm = 0, per_sm = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cqr2_fused_kernel, 256, 0) != cudaSuccess)
      cudaGetLastError();
    F->coop = coop != 0 && per_sm * nsm >= F->nblk;
  }
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // the m-vectors go to global memory when they do not fit beside the frame
  // (the sweep also holds kFStaticSmem bytes of static shared memory)
  const size_t room = static_cast<size_t>(optin) - kFStaticSmem;
  const bool vglob = F->smem > room;
  if (vglob) F->smem = fcarve(F->g, m, rho, true).total;
  if (F->smem > room || fft_smem(F->g) > static_cast<size_t>(optin)) {
    *msg = "frame too large for one CTA's shared memory (n <= 16384 fits)";
    delete F;
    return nullptr;
  }
  cudaFuncSetAttribute(fsweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       smem_optin_limit() - static_cast<int>(kFStaticSmem));
  cudaFuncSetAttribute(fft_frames_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       smem_optin_limit());
  const size_t rr = static_cast<size_t>(r) * r;
  bool ok = cudaMallocAsync(reinterpret_cast<void**>(&F->y), sizeof(float2) * m * q, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->mask), sizeof(int) * m * q, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->U), sizeof(float2) * n * r, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->FU), sizeof(float2) * n * r, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->B), sizeof(float2) * q * r, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->S_idx), sizeof(int) * q * std::max(1, rho), F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->S_val), sizeof(float2) * q * std::max(1, rho), F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->RES), sizeof(float2) * m * q, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->H), sizeof(float2) * static_cast<size_t>(n) * q, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->K), sizeof(float2) * n * r, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->grad), sizeof(float2) * n * r, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->Z), sizeof(float2) * n * r, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->Z2), sizeof(float2) * n * r, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->twx), sizeof(float2) * nx, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->twl), sizeof(float2) * F->g.L, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->twy), sizeof(float2) * ny, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->iptr), sizeof(int) * (n + 1), F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->ilist), sizeof(int) * m * q, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->err), sizeof(int) * 2, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->part), sizeof(double2) * F->nblk * rr, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->part2), sizeof(double2) * F->nblk * rr, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->qbar), sizeof(unsigned), F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->rfac), sizeof(double2) * 2 * rr, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->eta), sizeof(double), F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->scal), sizeof(double) * 4, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->Wk),
                            sizeof(float2) * static_cast<size_t>(r) * m * q, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->AS),
                            sizeof(float2) * static_cast<size_t>(m) * q, F->s) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&F->asv), sizeof(int) * q, F->s) == cudaSuccess &&
            (!vglob || cudaMallocAsync(reinterpret_cast<void**>(&F->vecs),
                                       sizeof(float2) * 3 * static_cast<size_t>(m) * q, F->s) == cudaSuccess);
  if (!ok) {
    *msg = "device allocation failed";
    return F;  // caller frees
  }
  std::vector<float2> tw(std::max(nx, ny));
  for (int k = 0; k < nx; ++k) {
    const double a = -2.0 * M_PI * k / nx;
    tw[k] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
  }
  cudaMemcpyAsync(F->twx, tw.data(), sizeof(float2) * nx, cudaMemcpyHostToDevice, F->s);
  for (int k = 0; k < ny; ++k) {
    const double a = -2.0 * M_PI * k / ny;
    tw[k] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
  }
  cudaMemcpyAsync(F->twy, tw.data(), sizeof(float2) * ny, cudaMemcpyHostToDevice, F->s);
  std::vector<float2> twl(F->g.L);
  for (int k = 0; k < F->g.L; ++k) {
    const double a = -2.0 * M_PI * k / F->g.L;
    twl[k] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
  }
  cudaMemcpyAsync(F->twl, twl.data(), sizeof(float2) * F->g.L, cudaMemcpyHostToDevice, F->s);
  cudaMemsetAsync(F->err, 0, 8, F->s);
  cudaMemsetAsync(F->asv, 0, sizeof(int) * q, F->s);
  cudaMemsetAsync(F->S_idx, 0, sizeof(int) * q * std::max(1, rho), F->s);
  cudaMemsetAsync(F->S_val, 0, sizeof(float2) * q * std::max(1, rho), F->s);
  cudaStreamSynchronize(F->s);  // the twiddle tables' host staging ends here
  return F;
}

void fourier_destroy(FourierSolver* F) {
  if (!F) return;
  void* ps[] = {F->y, F->mask, F->U, F->FU, F->B, F->S_idx, F->S_val, F->RES, F->H, F->K, F->grad,
                F->Z, F->Z2, F->twx, F->twy, F->twl, F->iptr, F->ilist, F->err, F->part, F->rfac, F->eta,
                F->scal,
                F->vecs, F->Wk, F->AS, F->asv, F->part2, F->qbar, F->prof};
  for (void* p : ps)
    if (p) cudaFreeAsync(p, F->s);
  cudaStreamSynchronize(F->s);
  delete F;
}

// masks: host int32 q x m (each column ascending, in [0, n)); y host or device
int fourier_set_measurements(FourierSolver* F, const void* y, const void* mask, int mem_kind,
                             std::string* msg) {
  const int n = F->g.n, m = F->m, q = F->q;
  std::vector<int> hm(static_cast<size_t>(m) * q);
  if (mem_kind) {
    if (cudaMemcpyAsync(hm.data(), mask, sizeof(int) * hm.size(), cudaMemcpyDeviceToHost, F->s) !=
            cudaSuccess ||
        cudaStreamSynchronize(F->s) != cudaSuccess) {
      *msg = "mask copy failed";
      return 4;
    }
  } else {
    std::memcpy(hm.data(), mask, sizeof(int) * hm.size());
  }
  for (int k = 0; k < q; ++k)
    for (int i = 0; i < m; ++i) {
      const int v = hm[static_cast<size_t>(k) * m + i];
      if (v < 0 || v >= n || (i > 0 && v <= hm[static_cast<size_t>(k) * m + i - 1])) {
        *msg = "mask row indices must be strictly ascending in [0, n)";
        return 1;
      }
    }
  // inverse index: for each frequency the (k, i) that sample it, k ascending
  std::vector<int> ptr(n + 1, 0), list(static_cast<size_t>(m) * q);
  for (int v : hm) ptr[v + 1]++;
  for (int w = 0; w < n; ++w) ptr[w + 1] += ptr[w];
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (int k = 0; k < q; ++k)
    for (int i = 0; i < m; ++i) list[fill[hm[static_cast<size_t>(k) * m + i]]++] = k * m + i;
  cudaError_t e = cudaMemcpyAsync(F->mask, hm.data(), sizeof(int) * hm.size(), cudaMemcpyHostToDevice, F->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(F->iptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice, F->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(F->ilist, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, F->s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(F->y, y, sizeof(float2) * m * q,
                        mem_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, F->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(F->asv, 0, sizeof(int) * q, F->s);  // new A_k
  if (e == cudaSuccess) e = cudaStreamSynchronize(F->s);
  if (e != cudaSuccess) {
    *msg = cudaGetErrorString(e);
    return 4;
  }
  F->t = 0;
  F->have_eta = false;
  return 0;
}

static cudaError_t launch_fsweep(FourierSolver* F, int mode, int tau) {
  FArgs a{};
  a.g = F->g;
  a.m = F->m;
  a.q = F->q;
  a.r = F->r;
  a.rho = F->rho;
  a.tau = tau;
  a.mode = mode;
  a.y = F->y;
  a.mask = F->mask;
  a.FU = F->FU;
  a.S_idx = F->S_idx;
  a.S_val = F->S_val;
  a.B = F->B;
  a.RES = F->RES;
  a.H = F->H;
  a.twx = F->twx;
  a.twy = F->twy;
  a.twl = F->twl;
  a.err = F->err;
  a.vecs = F->vecs;
  a.Wk = F->Wk;
  a.AS = F->AS;
  a.asv = F->asv;
  a.prof = F->prof;
  fsweep_kernel<<<F->q, kFT, F->smem, F->s>>>(a);
  return cudaGetLastError();
}

// complex Cholesky-QR2 of Zin (r x n column-major) into Uout
static cudaError_t ccholqr2(FourierSolver* F, const float2* Zin, float2* Uout) {
  const int n = F->g.n, r = F->r;
  const unsigned nb = static_cast<unsigned>((static_cast<size_t>(n) * r + 255) / 256);
  cgram_part_kernel<<<F->nblk, 256, 0, F->s>>>(n, r, Zin, nullptr, nullptr, nullptr, F->part);
  cchol_fin_kernel<<<1, 256, 0, F->s>>>(r, F->nblk, F->part, F->rfac, F->err);
  capply_kernel<<<nb, 256, 0, F->s>>>(n, r, Zin, F->rfac, F->Z2);
  cgram_part_kernel<<<F->nblk, 256, 0, F->s>>>(n, r, F->Z2, nullptr, nullptr, nullptr, F->part);
  cchol_fin_kernel<<<1, 256, 0, F->s>>>(r, F->nblk, F->part, F->rfac + r * r, F->err);
  capply_kernel<<<nb, 256, 0, F->s>>>(n, r, F->Z2, F->rfac + r * r, Uout);
  return cudaGetLastError();
}

// Z = X - eta G2 (G2 null: Z = X), then Uout = its Cholesky-QR2: one
// cooperative launch when every block fits on the device at once, else the
// separate kernels.  Uout may be X.
static cudaError_t cqr2(FourierSolver* F, const float2* X, const float2* G2, const double* eta,
                        float2* Uout) {
  const int n = F->g.n, r = F->r;
  if (F->coop) {
    cudaError_t e = cudaMemsetAsync(F->qbar, 0, sizeof(unsigned), F->s);
    if (e != cudaSuccess) return e;
    float2* Z = F->Z;
    float2* Z2 = F->Z2;
    unsigned long long wait_ns = 10ull * 1000 * 1000 * 1000;
    int nn = n, rr = r;
    void* args[] = {&nn, &rr, const_cast<float2**>(&X), const_cast<float2**>(&G2),
                    const_cast<double**>(&eta), &Z, &Z2, &Uout, &F->part, &F->part2, &F->qbar,
                    &F->err, &wait_ns};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(cqr2_fused_kernel),
                                       dim3(F->nblk), dim3(256), args, 0, F->s);
  }
  if (G2) {
    cgram_part_kernel<<<F->nblk, 256, 0, F->s>>>(n, r, X, G2, eta, F->Z, F->part);
    return ccholqr2(F, F->Z, Uout);
  }
  return ccholqr2(F, X, Uout);
}

int fourier_check_error(FourierSolver* F, std::string* msg) {
  int e[2] = {0, 0};
  cudaMemcpyAsync(e, F->err, sizeof(e), cudaMemcpyDeviceToHost, F->s);
  if (cudaStreamSynchronize(F->s) != cudaSuccess) {
    *msg = "CUDA error";
    return 4;
  }
  if (e[0]) {
    cudaMemsetAsync(F->err, 0, 8, F->s);
    *msg = e[0] == kErrNotSPD ? "r x r Gram matrix not positive definite" : "NaN/Inf in the iteration";
    if (e[1] >= 0) *msg += " (frame " + std::to_string(e[1]) + ")";
    return 5;
  }
  return 0;
}

int fourier_init(FourierSolver* F, std::string* msg) {
  const int n = F->g.n, q = F->q, r = F->r;
  cudaError_t e = launch_fsweep(F, kModeInit, F->tau0);  // s_k and the L0 columns in H
  // Complex subspace iteration for the top-r left singular vectors of L0:
  // float32 products P = L0^H U and Z = L0 P, complex Cholesky-QR2 of Z with
  // FP64 r x r factors, until the subspace moves by less than power_tol or by
  // less than the float32 resolution of U (4 eps sqrt(n r): a converged
  // float32 iteration moves U by its rounding).
  const size_t nr = static_cast<size_t>(n) * r;
  float2 *Uo = nullptr, *Zf = nullptr, *Pf = nullptr;
  double* rpart = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&Uo), nr * 8, F->s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&Zf), nr * 8, F->s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&Pf), static_cast<size_t>(q) * r * 8, F->s);
  // the projection's row chunks: about two blocks per SM in all
  const int kb = (q + 7) / 8;
  int cs = (n + std::max(1, 304 / kb) - 1) / std::max(1, 304 / kb);
  cs = (cs + kProjRows - 1) / kProjRows * kProjRows;
  const int nc = (n + cs - 1) / cs;
  float2* Pp = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&Pp), static_cast<size_t>(nc) * q * r * 8, F->s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&rpart), F->nblk * sizeof(double), F->s);
  // start: deterministic complex Gaussian block
  std::vector<float2> st(nr);
  uint64_t sd = F->seed * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull;
  auto nxt = [&]() {
    uint64_t z = (sd += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (auto& v : st) {
    const double u1 = ((nxt() >> 11) + 1.0) * 0x1.0p-53, u2 = (nxt() >> 11) * 0x1.0p-53;
    const double rad = std::sqrt(-2.0 * std::log(u1));
    v = make_float2(static_cast<float>(rad * std::cos(6.283185307179586 * u2)),
                    static_cast<float>(rad * std::sin(6.283185307179586 * u2)));
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(Zf, st.data(), nr * 8, cudaMemcpyHostToDevice, F->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(F->s);  // the host block may go
  if (e == cudaSuccess) e = cqr2(F, Zf, nullptr, nullptr, F->U);
  const double floor_tol = 4.0 * 0x1.0p-24 * std::sqrt(static_cast<double>(nr));
  const double tol = std::max(F->power_tol, floor_tol);
  for (int it = 0; it < F->power_iters && e == cudaSuccess; ++it) {
    e = cudaMemcpyAsync(Uo, F->U, nr * 8, cudaMemcpyDeviceToDevice, F->s);
    cproject_part_kernel<<<dim3(kb, nc), 256, 0, F->s>>>(n, q, r, cs, F->H, Uo, Pp);
    cproject_sum_kernel<<<(q * r + 255) / 256, 256, 0, F->s>>>(q, r, nc, Pp, Pf);
    cgrad_kernel<<<(n + 31) / 32, 256, 0, F->s>>>(n, q, r, F->H, Pf, Zf);
    if (e == cudaSuccess) e = cqr2(F, Zf, nullptr, nullptr, F->U);
    if (e == cudaSuccess && ((it % 5) == 4 || it + 1 == F->power_iters)) {
      coverlap_part_kernel<<<F->nblk, 256, 0, F->s>>>(n, r, Uo, F->U, F->part);
      cresid_part_kernel<<<F->nblk, 256, 0, F->s>>>(n, r, F->nblk, F->part, Uo, F->U, rpart);
      csum_fin_kernel<<<1, 32, 0, F->s>>>(F->nblk, rpart, F->scal);
      double chg2 = 0;
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaMemcpyAsync(&chg2, F->scal, sizeof(double), cudaMemcpyDeviceToHost, F->s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(F->s);
      if (e == cudaSuccess && std::sqrt(std::max(0.0, chg2)) < tol) break;
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(F->s);
  for (void* p : {static_cast<void*>(Uo), static_cast<void*>(Zf), static_cast<void*>(Pf),
                  static_cast<void*>(Pp), static_cast<void*>(rpart)})
    if (p) cudaFreeAsync(p, F->s);
  // b_k = (A_k U0)^+ (y_k - A_k s_k)
  if (e == cudaSuccess) e = fft_frames(F, F->U, F->FU, r, false);
  if (e == cudaSuccess) e = launch_fsweep(F, kModeLS, 0);
  if (e != cudaSuccess) {
    *msg = cudaGetErrorString(e);
    return 4;
  }
  F->t = 0;
  F->have_eta = false;
  return fourier_check_error(F, msg);
}

// evs (optional): 4 events per iteration, recorded before FU = F2 U, after
// the per-frame sweep, after the gradient and after the QR.
int fourier_iterate(FourierSolver* F, int iters, std::string* msg, cudaEvent_t* evs) {
  const int n = F->g.n, r = F->r;
  for (int i = 0; i < iters; ++i) {
    cudaEvent_t* ev = evs ? evs + 4 * static_cast<size_t>(i) : nullptr;
    if (ev) cudaEventRecord(ev[0], F->s);
    cudaError_t e = fft_frames(F, F->U, F->FU, r, false);            // FU = F2 U
    if (e == cudaSuccess) e = launch_fsweep(F, kModeIter, F->tau);   // per-frame work
    if (ev) cudaEventRecord(ev[1], F->s);
    kspace_kernel<<<(n + 7) / 8, 256, 0, F->s>>>(n, F->m, r, F->iptr, F->ilist, F->RES, F->B, F->K);
    if (e == cudaSuccess) e = fft_frames(F, F->K, F->grad, r, true);  // grad = F2^H K
    if (e == cudaSuccess && F->t == 0) {
      cgram_part_kernel<<<F->nblk, 256, 0, F->s>>>(n, r, F->grad, nullptr, nullptr, nullptr, F->part);
      ceta_kernel<<<1, 32, 0, F->s>>>(r, F->nblk, F->part, F->c_eta, F->eta);
    }
    if (ev) cudaEventRecord(ev[2], F->s);
    // Z = U - eta grad, then complex Cholesky-QR2
    if (e == cudaSuccess) e = cqr2(F, F->U, F->grad, F->eta, F->U);
    if (ev) cudaEventRecord(ev[3], F->s);
    if (e != cudaSuccess) {
      *msg = cudaGetErrorString(e);
      return 4;
    }
    F->t += 1;
  }
  return fourier_check_error(F, msg);
}

// host/device copies of U (n x r column-major = our layout), B, S
int fourier_get(FourierSolver* F, void* U, void* B, int* S_idx, void* S_val, int mem_kind) {
  const cudaMemcpyKind k = mem_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t n = F->g.n;
  if (U) cudaMemcpyAsync(U, F->U, sizeof(float2) * n * F->r, k, F->s);
  if (B) cudaMemcpyAsync(B, F->B, sizeof(float2) * F->q * F->r, k, F->s);
  if (S_idx && F->rho) cudaMemcpyAsync(S_idx, F->S_idx, sizeof(int) * F->q * F->rho, k, F->s);
  if (S_val && F->rho) cudaMemcpyAsync(S_val, F->S_val, sizeof(float2) * F->q * F->rho, k, F->s);
  return cudaStreamSynchronize(F->s) == cudaSuccess ? 0 : 4;
}

int fourier_set_state(FourierSolver* F, const void* U, const void* B, const int* S_idx,
                      const void* S_val, int t, double eta, int mem_kind) {
  const cudaMemcpyKind k = mem_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t n = F->g.n;
  cudaMemcpyAsync(F->U, U, sizeof(float2) * n * F->r, k, F->s);
  cudaMemcpyAsync(F->B, B, sizeof(float2) * F->q * F->r, k, F->s);
  if (F->rho) {
    cudaMemcpyAsync(F->S_idx, S_idx, sizeof(int) * F->q * F->rho, k, F->s);
    cudaMemcpyAsync(F->S_val, S_val, sizeof(float2) * F->q * F->rho, k, F->s);
  }
  cudaMemsetAsync(F->asv, 0, sizeof(int) * F->q, F->s);  // a new s_k
  cudaMemcpyAsync(F->eta, &eta, sizeof(double), cudaMemcpyHostToDevice, F->s);
  F->t = t;
  return cudaStreamSynchronize(F->s) == cudaSuccess ? 0 : 4;
}

double fourier_eta(FourierSolver* F) {
  double v = 0;
  cudaMemcpyAsync(&v, F->eta, sizeof(double), cudaMemcpyDeviceToHost, F->s);
  cudaStreamSynchronize(F->s);
  return F->t ? v : 0.0;
}
int fourier_t(FourierSolver* F) { return F->t; }

// Kernels one steady iteration launches: F2 U, the sweep, the k-space
// reduction, F2^H K, and the step with its Cholesky-QR2 (one cooperative
// launch, else the Gram partials and two factorisations and applications).
int fourier_launches_per_iteration(FourierSolver* F) { return 4 + (F->coop ? 1 : 6); }
int fourier_fused_qr(FourierSolver* F) { return F->coop ? 1 : 0; }

// Sweep cycle counters: enable (allocate, zero) and read-and-zero.
int fourier_prof_enable(FourierSolver* F) {
  if (F->prof) return 0;
  if (cudaMallocAsync(reinterpret_cast<void**>(&F->prof), sizeof(unsigned long long) * kFProf, F->s) !=
      cudaSuccess)
    return 3;  // LRS_ERR_OOM
  return cudaMemsetAsync(F->prof, 0, sizeof(unsigned long long) * kFProf, F->s) == cudaSuccess
             ? 0
             : 4;  // LRS_ERR_CUDA
}
int fourier_prof_read(FourierSolver* F, unsigned long long* out, int len) {
  if (!F->prof) return 2;  // LRS_ERR_STATE
  const int n = len < kFProf ? len : kFProf;
  if (cudaMemcpyAsync(out, F->prof, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, F->s) !=
          cudaSuccess ||
      cudaMemsetAsync(F->prof, 0, sizeof(unsigned long long) * kFProf, F->s) != cudaSuccess ||
      cudaStreamSynchronize(F->s) != cudaSuccess)
    return 4;  // LRS_ERR_CUDA
  return 0;
}

}  // namespace lrs
