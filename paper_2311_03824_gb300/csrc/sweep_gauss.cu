// Per-column sweep of AltGDmin-LR+S for the Gaussian operator (Algorithm 1
// with Algorithm 2), one thread-block cluster of CS CTAs per column k.
//
// The cluster's CTAs split A_k by columns j into slabs (GaussLayout).  A slab
// either stays in shared memory for the whole column (staged once by TMA bulk
// copies) or, when it does not fit, is streamed from global memory (L2) for
// each product.  The products of one column-iteration are
//   W_k = A_k U                                 (row pass, r wide)
//   u   = P_perp(A_k s - y_k)                   (sparse gather + r x r solve)
//   g   = A_k^T u                               (column pass)
//   mu  = ||g_G||^2 / ||P_perp A_k g_G||^2      (gather on the support G)
//   s   = HardThreshold(s - mu g, rho)          (cluster-wide top-rho)
//   b_k = G_k^{-1} W_k^T (y_k - A_k s)          (FP64 inverse Gram)
//   h_k = A_k^T (W_k b_k + A_k s - y_k)         (column pass; gradient term)
// with P_perp v = v - W_k G_k^{-1} W_k^T v and G_k = W_k^T W_k.  The r x r
// Gram, its Cholesky factor and inverse are FP64; the m-space dot products of
// the projections accumulate in FP64; the passes over A_k run in FP32.
//
// Partial results of the slabs are combined through distributed shared
// memory: each CTA writes its partial into one of two exchange slots of its
// own shared memory, a cluster barrier publishes it, and every CTA sums all
// partials in rank order, so every CTA holds bit-identical reduced values and
// takes identical control-flow decisions.
#include "lrs_dev.cuh"
#include "lrs_internal.h"

namespace lrs {
namespace {

constexpr int kSelBlk = 128;  // block size of the local all-pairs ranking
constexpr int kMaxR = 16;
constexpr int kNT = 256;      // threads per CTA
constexpr int kNW = kNT / 32;

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

struct Carve {
  size_t mbar, slab, Us, W, yv, dv, ev, gs, sl, vv, gpart, keys, bc, ck, cv, cn, Ginv, fsm,
      flags, redd, sup, xch, xs, total;
};

__host__ __device__ inline Carve carve(const GaussLayout& L, int resident) {
  Carve c;
  size_t o = 0;
  const int RP = (L.r + 3) & ~3;
  const int rho = L.rho > 0 ? L.rho : 1;
  const int nb = (L.ns + kSelBlk - 1) / kSelBlk;
  c.mbar = o;  o += 16;
  c.slab = o;  if (resident) o += a16((size_t)L.m * L.ns_pad * 4);
  c.Us = o;    o += a16((size_t)L.ns_pad * RP * 4);
  c.W = o;     o += a16((size_t)L.m * RP * 4);
  c.yv = o;    o += a16((size_t)L.m * 4);
  c.dv = o;    o += a16((size_t)L.m * 4);
  c.ev = o;    o += a16((size_t)L.m * 4);
  c.gs = o;    o += a16((size_t)L.ns_pad * 4);
  c.sl = o;    o += a16((size_t)L.ns_pad * 4);
  c.vv = o;    o += a16((size_t)L.ns_pad * 4);
  c.gpart = o; o += a16((size_t)kNW * L.ns_pad * 4);
  c.keys = o;  o += a16((size_t)L.ns_pad * 8);
  c.bc = o;    o += a16((size_t)nb * rho * 4);
  c.ck = o;    o += a16((size_t)L.cs * rho * 8);
  c.cv = o;    o += a16((size_t)L.cs * rho * 4);
  c.cn = o;    o += a16((size_t)L.cs * 4);
  c.Ginv = o;  o += a16(3 * kMaxR * kMaxR * 8);       // G, L, Ginv (FP64)
  c.fsm = o;   o += a16(4 * kMaxR * 8);               // FP64 r-vectors (c, x)
  c.flags = o; o += a16((size_t)(rho + 4) * 4);
  c.redd = o;  o += a16((size_t)kNT * 8 + 64);
  c.sup = o;   o += a16((size_t)rho * 8 + 16);
  const size_t xw = (size_t)L.m * RP * 4;                           // W partial
  const size_t xa = a16((size_t)L.m * 4) + kMaxR * kMaxR * 8 + 16;  // A s partial + Gram + count
  const size_t xg = a16((size_t)L.m * 4) + 16;                      // A g_G partial + ||g_G||^2
  const size_t xc = 16 + (size_t)rho * 16;                          // candidates
  size_t mx = xw > xa ? xw : xa;
  mx = mx > xg ? mx : xg;
  mx = mx > xc ? mx : xc;
  c.xs = a16(mx);
  c.xch = o;   o += 2 * c.xs;
  c.total = o;
  return c;
}

__device__ __forceinline__ uint64_t ht_key(float v, int jglob) {
  return (static_cast<uint64_t>(__float_as_uint(fabsf(v))) << 32) |
         static_cast<uint64_t>(0xFFFFFFFFu - static_cast<unsigned>(jglob));
}
__device__ __forceinline__ int key_index(uint64_t key) {
  return static_cast<int>(0xFFFFFFFFu - static_cast<unsigned>(key & 0xFFFFFFFFull));
}
// number of entries of the descending list l[0..len) that are > x
__device__ __forceinline__ int count_greater(const uint64_t* l, int len, uint64_t x) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (l[mid] > x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double dfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// 1/sqrt(s) in FP64: float estimate refined by two Newton-Raphson steps
// y <- y (3 - s y^2) / 2 (each step doubles the number of correct bits).
__device__ __forceinline__ double rsqrt_fp64(double s) {
  if (!(s > 1e-36 && s < 1e36)) return 1.0 / sqrt(s);
  double y = static_cast<double>(rsqrtf(static_cast<float>(s)));
  y = y * (1.5 - 0.5 * s * y * y);
  y = y * (1.5 - 0.5 * s * y * y);
  return y;
}

// Everything one CTA needs about its column and its shared memory.
struct Ctx {
  const float* Asl;  // slab: shared (resident) or global (streamed), m x ld row-major
  int m, n, r, rho, ld, nsc, nq, j0, c, CS, k;
  float* Us;         // ld x R (row j: U[j0 + j][0..R), zero padded)
  float* W;          // m x R
  float* yv;
  float* dv;
  float* ev;
  float* gs;
  float* sl;
  float* vv;
  float* gpart;
  uint64_t* keys;
  int* bc;
  uint64_t* ck;
  float* cvv;
  int* cn;
  double* G;         // r x r (ld kMaxR)
  double* Lc;
  double* Gi;        // G^{-1}
  double* fv;        // FP64 vectors: [0,16) c, [16,32) x
  int* flags;
  double* redd;
  int* sup_j;
  float* sup_v;
  int* nloc;
  unsigned char* xch;
  size_t xs;
  int* err;
};

__device__ __forceinline__ unsigned char* xslot(const Ctx& C, int e) {
  return C.xch + (e & 1) * C.xs;
}

// ---------------------------------------------------------------- passes --
// g[0..nsc) = A_slab^T v: warps split rows, lanes take float4 column quads;
// per-warp partials summed over warps in a fixed order.
__device__ __forceinline__ void col_pass(const Ctx& C, const float* v, bool streamed) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int RB = (C.m + kNW - 1) / kNW;
  const int rlo = wid * RB, rhi = min(C.m, rlo + RB);
  for (int qd = lane; qd < C.nq; qd += 32) {
    float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0;
    int i = rlo;
    for (; i + 1 < rhi; i += 2) {
      const float4* p0 = reinterpret_cast<const float4*>(C.Asl + static_cast<size_t>(i) * C.ld) + qd;
      const float4* p1 = reinterpret_cast<const float4*>(C.Asl + static_cast<size_t>(i + 1) * C.ld) + qd;
      const float4 a0 = streamed ? __ldg(p0) : *p0;
      const float4 a1 = streamed ? __ldg(p1) : *p1;
      const float u0 = v[i], u1 = v[i + 1];
      acc0.x = fmaf(a0.x, u0, acc0.x); acc0.y = fmaf(a0.y, u0, acc0.y);
      acc0.z = fmaf(a0.z, u0, acc0.z); acc0.w = fmaf(a0.w, u0, acc0.w);
      acc1.x = fmaf(a1.x, u1, acc1.x); acc1.y = fmaf(a1.y, u1, acc1.y);
      acc1.z = fmaf(a1.z, u1, acc1.z); acc1.w = fmaf(a1.w, u1, acc1.w);
    }
    if (i < rhi) {
      const float4* p0 = reinterpret_cast<const float4*>(C.Asl + static_cast<size_t>(i) * C.ld) + qd;
      const float4 a0 = streamed ? __ldg(p0) : *p0;
      const float u0 = v[i];
      acc0.x = fmaf(a0.x, u0, acc0.x); acc0.y = fmaf(a0.y, u0, acc0.y);
      acc0.z = fmaf(a0.z, u0, acc0.z); acc0.w = fmaf(a0.w, u0, acc0.w);
    }
    float4 s;
    s.x = acc0.x + acc1.x; s.y = acc0.y + acc1.y; s.z = acc0.z + acc1.z; s.w = acc0.w + acc1.w;
    reinterpret_cast<float4*>(C.gpart + static_cast<size_t>(wid) * C.ld)[qd] = s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < C.nsc; j += kNT) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kNW; ++w) s += C.gpart[w * C.ld + j];
    C.gs[j] = s;
  }
  __syncthreads();
}

// out[i] = sum_e coef[e] A(i, sup_j[e]) over the local support (partial of
// the cluster sum).
__device__ __forceinline__ void gather(const Ctx& C, const float* coef, float* out,
                                       bool streamed) {
  const int nl = *C.nloc;
  for (int i = threadIdx.x; i < C.m; i += kNT) {
    float s = 0.f;
    const float* row = C.Asl + static_cast<size_t>(i) * C.ld;
    for (int e = 0; e < nl; ++e) {
      const float a = streamed ? __ldg(row + C.sup_j[e]) : row[C.sup_j[e]];
      s = fmaf(a, coef[e], s);
    }
    out[i] = s;
  }
}

// cluster-sum of an m-vector partial held in slot x -> out (rank order)
__device__ __forceinline__ void reduce_m(const Ctx& C, const float* x, float* out) {
  for (int i = threadIdx.x; i < C.m; i += kNT) {
    float s = 0.f;
    for (int p = 0; p < C.CS; ++p) s += peer_ptr(x, p)[i];
    out[i] = s;
  }
}

// FP64 sum over the CTA of nv per-thread values acc[0..nv) -> C.fv[0..nv)
template <int R>
__device__ __forceinline__ void block_sum_d(const Ctx& C, double (&acc)[R], int nv) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int l = 0; l < R; ++l) acc[l] = warp_sum(acc[l]);
  if (lane == 0) {
#pragma unroll
    for (int l = 0; l < R; ++l)
      if (l < nv) C.redd[w * kMaxR + l] = acc[l];
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kNW; ++i) s += C.redd[i * kMaxR + threadIdx.x];
    C.fv[threadIdx.x] = s;
  }
  __syncthreads();
}

// x = G^{-1} W^T v  (FP64 dot products), x (FP64) in C.fv[16 + l]
template <int R>
__device__ __forceinline__ void ls_solve(const Ctx& C, const float* v) {
  double acc[R];
#pragma unroll
  for (int l = 0; l < R; ++l) acc[l] = 0.0;
  for (int i = threadIdx.x; i < C.m; i += kNT) {
    const double vi = v[i];
#pragma unroll
    for (int l = 0; l < R; ++l) acc[l] = dfma(static_cast<double>(C.W[i * R + l]), vi, acc[l]);
  }
  block_sum_d<R>(C, acc, C.r);
  if (threadIdx.x < R) {
    double s = 0.0;
    if (threadIdx.x < C.r)
      for (int b = 0; b < C.r; ++b) s = dfma(C.Gi[threadIdx.x * kMaxR + b], C.fv[b], s);
    C.fv[16 + threadIdx.x] = s;
  }
  __syncthreads();
}

// v <- P_perp v = v - W G^{-1} W^T v   (in place; FP64 for the m-space sums)
template <int R>
__device__ __forceinline__ void proj(const Ctx& C, float* v) {
  ls_solve<R>(C, v);
  for (int i = threadIdx.x; i < C.m; i += kNT) {
    double s = v[i];
#pragma unroll
    for (int l = 0; l < R; ++l) s = dfma(-static_cast<double>(C.W[i * R + l]), C.fv[16 + l], s);
    v[i] = static_cast<float>(s);
  }
  __syncthreads();
}

// sum of squares of an m-vector in FP64 (returned to all threads)
__device__ __forceinline__ double norm2_m(const Ctx& C, const float* v) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < C.m; i += kNT) acc = dfma(static_cast<double>(v[i]), v[i], acc);
  acc = warp_sum(acc);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) C.redd[threadIdx.x >> 5] = acc;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kNW; ++i) s += C.redd[i];
  return s;
}

// Cholesky of G (lane 0, FP64, no division: inverse pivots by rsqrt_fp64),
// then G^{-1} = L^{-T} L^{-1} by warp 0.  A pivot that is not positive
// marks the column as numerically failed (identity used to keep going).
__device__ __forceinline__ void factor_gram(const Ctx& C) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x, r = C.r;
  double* L = C.Lc;
  double* iL = C.fv + 32;  // inverse pivots
  if (lane == 0) {
    bool ok = true;
    for (int j = 0; j < r && ok; ++j) {
      double s = C.G[j * kMaxR + j];
      for (int p = 0; p < j; ++p) s -= L[j * kMaxR + p] * L[j * kMaxR + p];
      if (!(s > 1e-13 * C.G[j * kMaxR + j]) || !(s < 1e300)) { ok = false; break; }
      const double ij = rsqrt_fp64(s);
      L[j * kMaxR + j] = s * ij;
      iL[j] = ij;
      for (int i = j + 1; i < r; ++i) {
        double t = C.G[i * kMaxR + j];
        for (int p = 0; p < j; ++p) t -= L[i * kMaxR + p] * L[j * kMaxR + p];
        L[i * kMaxR + j] = t * ij;
      }
    }
    if (!ok) {
      C.flags[0] = 1;
      report_error(C.err, kErrNotSPD, C.k);
      for (int i = 0; i < r; ++i) {
        for (int p = 0; p < r; ++p) L[i * kMaxR + p] = (i == p) ? 1.0 : 0.0;
        iL[i] = 1.0;
      }
    }
  }
  __syncwarp();
  // column `lane` of L^{-1} (lower triangular), stored in G's buffer
  double* Li = C.G;
  if (lane < r) {
    const int cc = lane;
    for (int i = 0; i < r; ++i) {
      double t = (i == cc) ? 1.0 : 0.0;
      for (int p = cc; p < i; ++p) t -= L[i * kMaxR + p] * Li[p * kMaxR + cc];
      Li[i * kMaxR + cc] = (i < cc) ? 0.0 : t * iL[i];
    }
  }
  __syncwarp();
  for (int t = lane; t < r * r; t += 32) {
    const int a = t / r, b = t - a * r;
    double s = 0.0;
    for (int p = (a > b ? a : b); p < r; ++p) s = dfma(Li[p * kMaxR + a], Li[p * kMaxR + b], s);
    C.Gi[a * kMaxR + b] = s;
  }
}

// ------------------------------------------------------------- exchanges --
// A s over the cluster with the local support values; with_gram also carries
// the FP64 partial Gram of this CTA's row range and factors it.  Result A s
// in dv; the local support counts of every CTA in cn[].
template <int R>
__device__ __forceinline__ void exchange_As(const Ctx& C, int& ex, bool with_gram, bool streamed) {
  unsigned char* x = xslot(C, ex);
  float* xa = reinterpret_cast<float*>(x);
  double* xgram = reinterpret_cast<double*>(x + a16(static_cast<size_t>(C.m) * 4));
  int* xcnt = reinterpret_cast<int*>(x + a16(static_cast<size_t>(C.m) * 4) + kMaxR * kMaxR * 8);
  gather(C, C.sup_v, xa, streamed);
  if (with_gram) {
    const int mc = (C.m + C.CS - 1) / C.CS;
    const int ilo = C.c * mc, ihi = min(C.m, ilo + mc);
    const int r = C.r, E = r * r;
    // thread t < E*P: entry t % E over rows ilo + t / E (step P); phases
    // summed in order
    const int P = max(1, kNT / E);
    if (threadIdx.x < E * P) {
      const int e = threadIdx.x % E, ph = threadIdx.x / E;
      const int p = e / r, q2 = e - p * r;
      double s = 0.0;
      if (q2 <= p)
        for (int i = ilo + ph; i < ihi; i += P)
          s = dfma(static_cast<double>(C.W[i * R + p]), static_cast<double>(C.W[i * R + q2]), s);
      C.redd[threadIdx.x] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < E; e += kNT) {
      double s = 0.0;
      for (int ph = 0; ph < P; ++ph) s += C.redd[ph * E + e];
      xgram[e] = s;
    }
  }
  if (threadIdx.x == 0) *xcnt = *C.nloc;
  cluster_sync_all();
  reduce_m(C, xa, C.dv);
  if (threadIdx.x < C.CS) C.cn[threadIdx.x] = *peer_ptr(xcnt, threadIdx.x);
  if (with_gram) {
    const int r = C.r;
    for (int t = threadIdx.x; t < r * r; t += kNT) {
      const int p = t / r, q2 = t - p * r;
      if (q2 <= p) {
        double s = 0.0;
        for (int pp = 0; pp < C.CS; ++pp) s += peer_ptr(xgram, pp)[t];
        C.G[p * kMaxR + q2] = s;
        C.G[q2 * kMaxR + p] = s;
      }
    }
  }
  ++ex;
  __syncthreads();
  if (with_gram) {
    factor_gram(C);
    __syncthreads();
  }
}

// HardThreshold over the cluster: values vv[0..nsc) -> new local support
// (exactly rho entries cluster-wide, largest |v| first, ties to the lower
// index).  keep_values = false keeps zero values (support of g at s = 0).
__device__ __forceinline__ void hard_threshold(const Ctx& C, int& ex, bool keep_values) {
  const int rho = C.rho, nsc = C.nsc;
  for (int j = threadIdx.x; j < nsc; j += kNT) C.keys[j] = ht_key(C.vv[j], C.j0 + j);
  __syncthreads();
  // rank inside blocks of kSelBlk; the first rho of each block are candidates
  for (int j = threadIdx.x; j < nsc; j += kNT) {
    const int blk = j / kSelBlk, lo = blk * kSelBlk, hi = min(nsc, lo + kSelBlk);
    const uint64_t kj = C.keys[j];
    int cnt = 0;
    for (int l = lo; l < hi; ++l) cnt += C.keys[l] > kj;
    if (cnt < rho) C.bc[blk * rho + cnt] = j;
  }
  __syncthreads();
  unsigned char* x = xslot(C, ex);
  int* xcnt = reinterpret_cast<int*>(x);
  uint64_t* xkey = reinterpret_cast<uint64_t*>(x + 16);
  float* xval = reinterpret_cast<float*>(x + 16 + static_cast<size_t>(rho) * 8);
  const int nb = (nsc + kSelBlk - 1) / kSelBlk;
  if (nb <= 1) {
    for (int s = threadIdx.x; s < min(rho, nsc); s += kNT) {
      const int j = C.bc[s];
      xkey[s] = C.keys[j];
      xval[s] = keep_values ? C.vv[j] : 0.f;
    }
  } else {
    int ncb = 0;
    for (int b = 0; b < nb; ++b) ncb += min(rho, min(nsc, (b + 1) * kSelBlk) - b * kSelBlk);
    for (int t = threadIdx.x; t < ncb; t += kNT) {
      int b = 0, s = t;
      while (s >= min(rho, min(nsc, (b + 1) * kSelBlk) - b * kSelBlk)) {
        s -= min(rho, min(nsc, (b + 1) * kSelBlk) - b * kSelBlk);
        ++b;
      }
      const int j = C.bc[b * rho + s];
      const uint64_t kj = C.keys[j];
      int cnt = 0;
      for (int b2 = 0; b2 < nb; ++b2) {
        const int nb2 = min(rho, min(nsc, (b2 + 1) * kSelBlk) - b2 * kSelBlk);
        for (int s2 = 0; s2 < nb2; ++s2) cnt += C.keys[C.bc[b2 * rho + s2]] > kj;
      }
      if (cnt < rho) {
        xkey[cnt] = kj;
        xval[cnt] = keep_values ? C.vv[j] : 0.f;
      }
    }
  }
  if (threadIdx.x == 0) *xcnt = min(rho, nsc);
  if (C.CS > 1) cluster_sync_all(); else __syncthreads();
  for (int t = threadIdx.x; t < C.CS * rho; t += kNT) {
    const int p = t / rho, s = t - p * rho;
    const unsigned char* px = peer_ptr(x, p);
    const int cp = *reinterpret_cast<const int*>(px);
    if (s < cp) {
      C.ck[t] = reinterpret_cast<const uint64_t*>(px + 16)[s];
      C.cvv[t] = reinterpret_cast<const float*>(px + 16 + static_cast<size_t>(rho) * 8)[s];
    } else {
      C.ck[t] = 0ull;
    }
    if (s == 0) C.cn[p] = cp;
  }
  ++ex;
  __syncthreads();
  // own candidates: selected iff their cluster-wide rank is < rho; the
  // selected ones are a prefix of the (descending) own list
  const int own = C.cn[C.c];
  for (int s = threadIdx.x; s < own; s += kNT) {
    const uint64_t kj = C.ck[C.c * rho + s];
    int g = 0;
    for (int p = 0; p < C.CS; ++p) g += count_greater(C.ck + p * rho, C.cn[p], kj);
    C.flags[1 + s] = (g < rho) ? 1 : 0;
  }
  // clear the old support in the dense local s
  const int nl_old = *C.nloc;
  for (int e = threadIdx.x; e < nl_old; e += kNT) C.sl[C.sup_j[e]] = 0.f;
  __syncthreads();
  if (threadIdx.x == 0) {
    int cnt = 0;
    while (cnt < own && C.flags[1 + cnt]) ++cnt;
    *C.nloc = cnt;
  }
  __syncthreads();
  const int cnt = *C.nloc;
  for (int s = threadIdx.x; s < cnt; s += kNT) {
    const int j = key_index(C.ck[C.c * rho + s]) - C.j0;
    const float val = C.cvv[C.c * rho + s];
    C.sup_j[s] = j;
    C.sup_v[s] = val;
    C.sl[j] = val;
  }
  __syncthreads();
}

template <int R, bool RES>
__global__ void __launch_bounds__(kNT, 2) sweep_kernel(const SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const GaussLayout& L = a.L;
  const int tid = threadIdx.x;
  Ctx C;
  C.c = static_cast<int>(cluster_rank());
  C.CS = static_cast<int>(cluster_size());
  C.k = static_cast<int>(cluster_id_x());
  C.m = L.m;
  C.n = L.n;
  C.r = L.r;
  C.rho = L.rho;
  C.ld = L.ns_pad;
  C.j0 = C.c * L.ns;
  C.nsc = max(0, min(L.ns, L.n - C.j0));
  C.nq = (C.nsc + 3) >> 2;
  C.err = a.err;
  const Carve cv = carve(L, RES ? 1 : 0);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + cv.mbar);
  const float* gslab = a.A + (static_cast<size_t>(C.k) * C.CS + C.c) * static_cast<size_t>(C.m) * C.ld;
  C.Asl = RES ? reinterpret_cast<const float*>(smem + cv.slab) : gslab;
  C.Us = reinterpret_cast<float*>(smem + cv.Us);
  C.W = reinterpret_cast<float*>(smem + cv.W);
  C.yv = reinterpret_cast<float*>(smem + cv.yv);
  C.dv = reinterpret_cast<float*>(smem + cv.dv);
  C.ev = reinterpret_cast<float*>(smem + cv.ev);
  C.gs = reinterpret_cast<float*>(smem + cv.gs);
  C.sl = reinterpret_cast<float*>(smem + cv.sl);
  C.vv = reinterpret_cast<float*>(smem + cv.vv);
  C.gpart = reinterpret_cast<float*>(smem + cv.gpart);
  C.keys = reinterpret_cast<uint64_t*>(smem + cv.keys);
  C.bc = reinterpret_cast<int*>(smem + cv.bc);
  C.ck = reinterpret_cast<uint64_t*>(smem + cv.ck);
  C.cvv = reinterpret_cast<float*>(smem + cv.cv);
  C.cn = reinterpret_cast<int*>(smem + cv.cn);
  C.G = reinterpret_cast<double*>(smem + cv.Ginv);
  C.Lc = C.G + kMaxR * kMaxR;
  C.Gi = C.G + 2 * kMaxR * kMaxR;
  C.fv = reinterpret_cast<double*>(smem + cv.fsm);
  C.flags = reinterpret_cast<int*>(smem + cv.flags);
  C.redd = reinterpret_cast<double*>(smem + cv.redd);
  const int rho1 = max(C.rho, 1);
  C.sup_j = reinterpret_cast<int*>(smem + cv.sup);
  C.sup_v = reinterpret_cast<float*>(smem + cv.sup + static_cast<size_t>(rho1) * 4);
  C.nloc = reinterpret_cast<int*>(smem + cv.sup + static_cast<size_t>(rho1) * 8);
  C.xch = smem + cv.xch;
  C.xs = cv.xs;
  int ex = 0;
  const int m = C.m, r = C.r, rho = C.rho, k = C.k;
  const bool streamed = !RES;

  // ---- stage the slab (TMA bulk copies on one mbarrier) -------------------
  if (RES && tid == 0) {
    mbar_init(mbar, 1);
    const size_t bytes = static_cast<size_t>(m) * C.ld * 4;
    mbar_arrive_expect_tx(mbar, static_cast<unsigned>(bytes));
    const char* src = reinterpret_cast<const char*>(gslab);
    char* dst = reinterpret_cast<char*>(smem + cv.slab);
    for (size_t off = 0; off < bytes; off += 32768) {
      const size_t rem = bytes - off;
      bulk_copy_g2s(dst + off, src + off, static_cast<unsigned>(rem < 32768 ? rem : 32768), mbar);
    }
  }
  // ---- small operands --------------------------------------------------
  for (int t = tid; t < C.ld * R; t += kNT) {
    const int j = t / R, l = t - j * R;
    C.Us[t] = (j < C.nsc && l < r) ? a.U[static_cast<size_t>(C.j0 + j) * r + l] : 0.f;
  }
  for (int i = tid; i < m; i += kNT) C.yv[i] = a.y[static_cast<size_t>(k) * m + i];
  for (int j = tid; j < C.ld; j += kNT) C.sl[j] = 0.f;
  if (tid == 0) {
    C.flags[0] = 0;
    int cnt = 0;
    if (a.mode != kModeInit) {
      for (int e = 0; e < rho; ++e) {
        const int jg = a.S_idx[static_cast<size_t>(k) * rho + e];
        if (jg >= C.j0 && jg < C.j0 + C.nsc) {
          C.sup_j[cnt] = jg - C.j0;
          C.sup_v[cnt] = a.S_val[static_cast<size_t>(k) * rho + e];
          ++cnt;
        }
      }
    }
    *C.nloc = cnt;
  }
  __syncthreads();
  for (int e = tid; e < *C.nloc; e += kNT) C.sl[C.sup_j[e]] = C.sup_v[e];
  if (RES) {
    if (!mbar_wait_bounded(mbar, 0) && (tid & 31) == 0) report_error(a.err, kErrTimeout, k);
  }
  if (C.CS > 1) cluster_sync_all(); else __syncthreads();

  const bool project = (a.mode != kModeInit);

  // ---------------------------------------------------------- W pass -----
  bool need_gram = false;
  if (project) {
    float* xw = reinterpret_cast<float*>(xslot(C, ex));
    for (int i = tid; i < m; i += kNT) {
      float acc[R];
#pragma unroll
      for (int l = 0; l < R; ++l) acc[l] = 0.f;
      const float4* arow = reinterpret_cast<const float4*>(C.Asl + static_cast<size_t>(i) * C.ld);
      for (int jq = 0; jq < C.nq; ++jq) {
        const float4 av = streamed ? __ldg(arow + jq) : arow[jq];
        const float* u0 = C.Us + (4 * jq) * R;
#pragma unroll
        for (int l = 0; l < R; ++l) {
          float t = acc[l];
          t = fmaf(av.x, u0[l], t);
          t = fmaf(av.y, u0[R + l], t);
          t = fmaf(av.z, u0[2 * R + l], t);
          t = fmaf(av.w, u0[3 * R + l], t);
          acc[l] = t;
        }
      }
      float* dst = (C.CS > 1) ? xw : C.W;
#pragma unroll
      for (int l = 0; l < R; ++l) dst[i * R + l] = acc[l];
    }
    if (C.CS > 1) {
      cluster_sync_all();
      for (int t = tid; t < m * R; t += kNT) {
        float s = 0.f;
        for (int p = 0; p < C.CS; ++p) s += peer_ptr(xw, p)[t];
        C.W[t] = s;
      }
      ++ex;
    }
    __syncthreads();
    need_gram = true;
  }

  // ----------------------------------------------------- IHT (Alg. 2) ----
  const int tau = (a.mode == kModeLS || rho == 0) ? 0 : a.tau;
  for (int it = 0; it < tau; ++it) {
    const bool zero_start = (a.mode == kModeInit && it == 0);
    // u = P_perp (A s - y)   (A s = 0 for the zero start)
    if (zero_start) {
      for (int i = tid; i < m; i += kNT) C.dv[i] = -C.yv[i];
      __syncthreads();
    } else {
      exchange_As<R>(C, ex, need_gram, streamed);
      need_gram = false;
      for (int i = tid; i < m; i += kNT) C.dv[i] -= C.yv[i];
      __syncthreads();
      if (project) proj<R>(C, C.dv);
    }
    col_pass(C, C.dv, streamed);  // g = A^T u  (= M^T (M s - z): P_perp is a projector)
    if (zero_start) {
      // support G of the zero start: the rho largest |g_i|
      for (int j = tid; j < C.nsc; j += kNT) C.vv[j] = C.gs[j];
      __syncthreads();
      hard_threshold(C, ex, false);
    }
    // ||g_G||^2 and A g_G on the support, then mu
    {
      unsigned char* x = xslot(C, ex);
      float* xg = reinterpret_cast<float*>(x);
      double* xnum = reinterpret_cast<double*>(x + a16(static_cast<size_t>(m) * 4));
      const int nl = *C.nloc;
      for (int e = tid; e < nl; e += kNT) C.vv[e] = C.gs[C.sup_j[e]];
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int e = 0; e < nl; ++e) s = dfma(static_cast<double>(C.vv[e]), C.vv[e], s);
        *xnum = s;
      }
      gather(C, C.vv, xg, streamed);
      double num = 0.0;
      if (C.CS > 1) {
        cluster_sync_all();
        reduce_m(C, xg, C.ev);
        for (int p = 0; p < C.CS; ++p) num += *peer_ptr(xnum, p);
        ++ex;
      } else {
        __syncthreads();
        for (int i = tid; i < m; i += kNT) C.ev[i] = xg[i];
        num = *xnum;
      }
      __syncthreads();
      if (project) proj<R>(C, C.ev);
      const double den = norm2_m(C, C.ev);
      if (!(den > 0.0)) break;  // ||M g_G|| = 0: the column's IHT stops
      double mu = num / den;
      if (!isfinite(mu)) {
        if (tid == 0) report_error(a.err, kErrNaN, k);
        mu = 0.0;
      }
      const float muf = static_cast<float>(mu);
      for (int j = tid; j < C.nsc; j += kNT) C.vv[j] = fmaf(-muf, C.gs[j], C.sl[j]);
      __syncthreads();
    }
    hard_threshold(C, ex, true);
  }

  // ------------------------------------------------------ final stage -----
  exchange_As<R>(C, ex, need_gram, streamed);  // A s with the final support
  for (int i = tid; i < m; i += kNT) C.dv[i] = C.yv[i] - C.dv[i];  // y - A s
  __syncthreads();
  if (a.mode != kModeInit) {
    ls_solve<R>(C, C.dv);  // b = G^{-1} W^T (y - A s)   (FP64)
    if (C.c == 0 && tid < r) a.B[static_cast<size_t>(k) * r + tid] = static_cast<float>(C.fv[16 + tid]);
    if (a.mode == kModeIter) {
      for (int i = tid; i < m; i += kNT) {  // W b + A s - y
        double s = -static_cast<double>(C.dv[i]);
#pragma unroll
        for (int l = 0; l < R; ++l) s = dfma(static_cast<double>(C.W[i * R + l]), C.fv[16 + l], s);
        C.ev[i] = static_cast<float>(s);
      }
      __syncthreads();
    }
  }
  if (a.mode != kModeLS) {
    col_pass(C, a.mode == kModeInit ? C.dv : C.ev, streamed);
    float* Hk = a.H + static_cast<size_t>(k) * C.n + C.j0;
    for (int j = tid; j < C.nsc; j += kNT) Hk[j] = C.gs[j];
    // S_k: this CTA's entries ascending by index, after those of lower ranks
    const int nl = *C.nloc;
    int off = 0;
    for (int p = 0; p < C.c; ++p) off += C.cn[p];
    for (int e = tid; e < nl; e += kNT) {
      const int je = C.sup_j[e];
      int pos = 0;
      for (int f = 0; f < nl; ++f) pos += C.sup_j[f] < je;
      if (off + pos < rho) {
        a.S_idx[static_cast<size_t>(k) * rho + off + pos] = C.j0 + je;
        a.S_val[static_cast<size_t>(k) * rho + off + pos] = C.sup_v[e];
      }
    }
  }
  if (C.CS > 1) cluster_sync_all();  // no CTA leaves while a peer may still read its slots
}

template <int R, bool RES>
void* kernel_ptr() {
  return reinterpret_cast<void*>(&sweep_kernel<R, RES>);
}

void* pick_kernel(int r, int resident) {
  const int RP = (r + 3) & ~3;
  switch (RP) {
    case 4: return resident ? kernel_ptr<4, true>() : kernel_ptr<4, false>();
    case 8: return resident ? kernel_ptr<8, true>() : kernel_ptr<8, false>();
    case 12: return resident ? kernel_ptr<12, true>() : kernel_ptr<12, false>();
    default: return resident ? kernel_ptr<16, true>() : kernel_ptr<16, false>();
  }
}

// repack columns [k0, k0 + kc) of row-major A_k into the slab layout
__global__ void repack_kernel(GaussLayout L, const float* __restrict__ Ain, int k0, int kc,
                              float* __restrict__ Aout) {
  const size_t per_col = static_cast<size_t>(L.cs) * L.m * L.ns_pad;
  const size_t total = per_col * kc;
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t kk = t / per_col;
    const size_t rem = t - kk * per_col;
    const int c = static_cast<int>(rem / (static_cast<size_t>(L.m) * L.ns_pad));
    const size_t rem2 = rem - static_cast<size_t>(c) * L.m * L.ns_pad;
    const int i = static_cast<int>(rem2 / L.ns_pad);
    const int jj = static_cast<int>(rem2 - static_cast<size_t>(i) * L.ns_pad);
    const int j = c * L.ns + jj;
    float v = 0.f;
    if (jj < L.ns && j < L.n) v = Ain[(kk * L.m + i) * L.n + j];
    Aout[(static_cast<size_t>(k0) + kk) * per_col + rem] = v;
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
    if (e != cudaSuccess && res == 0) return e;
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
  cfg.blockDim = dim3(kNT, 1, 1);
  cfg.dynamicSmemBytes = sweep_smem_bytes(L, resident, kNT);
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
