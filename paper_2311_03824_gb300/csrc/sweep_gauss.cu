// Per-column sweep of AltGDmin-LR+S for the Gaussian operator (Algorithm 1
// with Algorithm 2), one thread-block cluster per column k.
//
// The cluster's CS CTAs split A_k by columns j into slabs (GaussLayout); each
// CTA stages its slab in shared memory with TMA bulk copies (or streams it
// from global memory when it does not fit) and keeps it there for every
// product of the column's iteration:
//   W_k = A_k U                                 (W pass, r-wide row products)
//   u   = P_perp(A_k s - y_k)                   (sparse gather + r x r solve)
//   g   = A_k^T u                               (column pass)
//   mu  = ||g_G||^2 / ||P_perp A_k g_G||^2      (gather on the support G)
//   s   = HardThreshold(s - mu g, rho)          (cluster-wide top-rho)
//   b_k = G_k^{-1} W_k^T (y_k - A_k s)          (FP64 Cholesky of W_k^T W_k)
//   h_k = A_k^T (W_k b_k + A_k s - y_k)         (column pass; gradient term)
// Partial results of the slabs are combined through distributed shared
// memory: every CTA writes its partial into one of two exchange slots of its
// own shared memory, the cluster barrier publishes it, and every CTA sums all
// partials in cluster-rank order, so all CTAs hold bit-identical reduced
// values and take identical control-flow decisions.
#include "lrs_dev.cuh"
#include "lrs_internal.h"

namespace lrs {
namespace {

constexpr int kSelBlk = 128;  // block size of the local all-pairs ranking
constexpr int kMaxR = 16;

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

struct Carve {
  size_t mbar, slab, Us, W, yv, dv, ev, gs, sl, vv, gpart, keys, bc, ck, cv, cn, Gm, Lc, xsol,
      flags, redf, redd, sup, xch, xs, total;
};

__host__ __device__ inline Carve carve(const GaussLayout& L, int resident, int nt) {
  Carve c;
  size_t o = 0;
  const int RP = (L.r + 3) & ~3;
  const int nw = nt / 32;
  const int rho = L.rho > 0 ? L.rho : 1;
  const int nb = (L.ns + kSelBlk - 1) / kSelBlk;
  c.mbar = o; o += 16;
  c.slab = o; if (resident) o += a16((size_t)L.m * L.ns_pad * 4);
  c.Us = o;    o += a16((size_t)L.ns_pad * RP * 4);
  c.W = o;     o += a16((size_t)L.m * RP * 4);
  c.yv = o;    o += a16((size_t)L.m * 4);
  c.dv = o;    o += a16((size_t)L.m * 4);
  c.ev = o;    o += a16((size_t)L.m * 4);
  c.gs = o;    o += a16((size_t)L.ns_pad * 4);
  c.sl = o;    o += a16((size_t)L.ns_pad * 4);
  c.vv = o;    o += a16((size_t)L.ns_pad * 4);
  c.gpart = o; o += a16((size_t)nw * L.ns_pad * 4);
  c.keys = o;  o += a16((size_t)L.ns_pad * 8);
  c.bc = o;    o += a16((size_t)nb * rho * 4);
  c.ck = o;    o += a16((size_t)L.cs * rho * 8);
  c.cv = o;    o += a16((size_t)L.cs * rho * 4);
  c.cn = o;    o += a16((size_t)L.cs * 4);
  c.Gm = o;    o += a16(kMaxR * kMaxR * 8);
  c.Lc = o;    o += a16(kMaxR * kMaxR * 8);
  c.xsol = o;  o += a16(kMaxR * 8 + kMaxR * 4);
  c.flags = o; o += a16((size_t)(rho + 4) * 4);
  c.redf = o;  o += a16((size_t)nw * kMaxR * 4);
  c.redd = o;  o += a16((size_t)nw * 8);
  c.sup = o;   o += a16((size_t)rho * 8 + 16);
  const size_t xw = (size_t)L.m * RP * 4;                       // W partial
  const size_t xa = a16((size_t)L.m * 4) + kMaxR * kMaxR * 8 + 16;  // A s partial + Gram + count
  const size_t xg = a16((size_t)L.m * 4) + 16;                  // A g_G partial + ||g_G||^2
  const size_t xc = 16 + (size_t)rho * 16;                      // candidates
  size_t mx = xw > xa ? xw : xa;
  mx = mx > xg ? mx : xg;
  mx = mx > xc ? mx : xc;
  c.xs = a16(mx);
  c.xch = o; o += 2 * c.xs;
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
// number of entries of the descending list `l[0..len)` that are > x
__device__ __forceinline__ int count_greater(const uint64_t* l, int len, uint64_t x) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (l[mid] > x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <int R, bool RES>
__global__ void __launch_bounds__(256) sweep_kernel(const SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const GaussLayout& L = a.L;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int c = static_cast<int>(cluster_rank());
  const int CS = static_cast<int>(cluster_size());
  const int k = static_cast<int>(cluster_id_x());
  const int m = L.m, n = L.n, r = L.r, rho = L.rho, ld = L.ns_pad;
  const int j0 = c * L.ns;
  const int nsc = max(0, min(L.ns, n - j0));
  const int nq = (nsc + 3) >> 2;
  const Carve cv = carve(L, RES ? 1 : 0, nt);

  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + cv.mbar);
  const float* gslab = a.A + (static_cast<size_t>(k) * CS + c) * static_cast<size_t>(m) * ld;
  const float* Asl = RES ? reinterpret_cast<const float*>(smem + cv.slab) : gslab;
  float* Us = reinterpret_cast<float*>(smem + cv.Us);
  float* W = reinterpret_cast<float*>(smem + cv.W);
  float* yv = reinterpret_cast<float*>(smem + cv.yv);
  float* dv = reinterpret_cast<float*>(smem + cv.dv);
  float* ev = reinterpret_cast<float*>(smem + cv.ev);
  float* gs = reinterpret_cast<float*>(smem + cv.gs);
  float* sl = reinterpret_cast<float*>(smem + cv.sl);
  float* vv = reinterpret_cast<float*>(smem + cv.vv);
  float* gpart = reinterpret_cast<float*>(smem + cv.gpart);
  uint64_t* keys = reinterpret_cast<uint64_t*>(smem + cv.keys);
  int* bc = reinterpret_cast<int*>(smem + cv.bc);
  uint64_t* ck = reinterpret_cast<uint64_t*>(smem + cv.ck);
  float* cvv = reinterpret_cast<float*>(smem + cv.cv);
  int* cn = reinterpret_cast<int*>(smem + cv.cn);
  double* Gm = reinterpret_cast<double*>(smem + cv.Gm);
  double* Lc = reinterpret_cast<double*>(smem + cv.Lc);
  double* xsol = reinterpret_cast<double*>(smem + cv.xsol);
  float* cvec = reinterpret_cast<float*>(smem + cv.xsol + kMaxR * 8);
  int* flags = reinterpret_cast<int*>(smem + cv.flags);
  float* redf = reinterpret_cast<float*>(smem + cv.redf);
  float* redd_f = reinterpret_cast<float*>(smem + cv.redd);
  int* sup_j = reinterpret_cast<int*>(smem + cv.sup);
  float* sup_v = reinterpret_cast<float*>(smem + cv.sup + static_cast<size_t>(max(rho, 1)) * 4);
  int* nloc_p = reinterpret_cast<int*>(smem + cv.sup + static_cast<size_t>(max(rho, 1)) * 8);
  auto xslot = [&](int e) -> unsigned char* { return smem + cv.xch + (e & 1) * cv.xs; };
  int ex = 0;  // exchange counter (slot parity)

  // ---- stage the slab (TMA bulk copies on one mbarrier) -------------------
  if (RES && tid == 0) {
    mbar_init(mbar, 1);
    const size_t bytes = static_cast<size_t>(m) * ld * 4;
    mbar_arrive_expect_tx(mbar, static_cast<unsigned>(bytes));
    const char* src = reinterpret_cast<const char*>(gslab);
    char* dst = reinterpret_cast<char*>(smem + cv.slab);
    for (size_t off = 0; off < bytes; off += 32768) {
      const size_t rem = bytes - off;
      bulk_copy_g2s(dst + off, src + off, static_cast<unsigned>(rem < 32768 ? rem : 32768), mbar);
    }
  }
  // ---- small operands --------------------------------------------------
  for (int t = tid; t < ld * R; t += nt) {
    const int j = t / R, l = t - j * R;
    Us[t] = (j < nsc && l < r) ? a.U[static_cast<size_t>(j0 + j) * r + l] : 0.f;
  }
  for (int i = tid; i < m; i += nt) yv[i] = a.y[static_cast<size_t>(k) * m + i];
  for (int j = tid; j < ld; j += nt) sl[j] = 0.f;
  if (tid == 0) {
    flags[0] = 0;  // 1: Cholesky failed in this column
    int cnt = 0;
    if (a.mode != kModeInit) {
      for (int e = 0; e < rho; ++e) {
        const int jg = a.S_idx[static_cast<size_t>(k) * rho + e];
        if (jg >= j0 && jg < j0 + nsc) {
          sup_j[cnt] = jg - j0;
          sup_v[cnt] = a.S_val[static_cast<size_t>(k) * rho + e];
          ++cnt;
        }
      }
    }
    *nloc_p = cnt;
  }
  __syncthreads();
  if (tid == 0)
    for (int e = 0; e < *nloc_p; ++e) sl[sup_j[e]] = sup_v[e];
  if (RES) {
    if (!mbar_wait_bounded(mbar, 0) && lane == 0) report_error(a.err, kErrTimeout, k);
  }
  cluster_sync_all();  // every CTA of the cluster is running and staged

  const bool project = (a.mode != kModeInit);

  // ---------------------------------------------------------- helpers ----
  // A_slab^T v  ->  gs[0..nsc)
  auto col_pass = [&](const float* v) {
    const int RB = (m + nw - 1) / nw;
    const int rlo = wid * RB, rhi = min(m, rlo + RB);
    for (int qd = lane; qd < nq; qd += 32) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int i = rlo; i < rhi; ++i) {
        const float4 av = reinterpret_cast<const float4*>(Asl + static_cast<size_t>(i) * ld)[qd];
        const float ui = v[i];
        acc.x = fmaf(av.x, ui, acc.x);
        acc.y = fmaf(av.y, ui, acc.y);
        acc.z = fmaf(av.z, ui, acc.z);
        acc.w = fmaf(av.w, ui, acc.w);
      }
      reinterpret_cast<float4*>(gpart + static_cast<size_t>(wid) * ld)[qd] = acc;
    }
    __syncthreads();
    for (int j = tid; j < nsc; j += nt) {
      float s = 0.f;
      for (int w = 0; w < nw; ++w) s += gpart[w * ld + j];
      gs[j] = s;
    }
    __syncthreads();
  };
  // sum over the local support of coef[e] * A(:, sup_j[e])  ->  out[0..m)
  auto gather = [&](const float* coef, float* out) {
    const int nl = *nloc_p;
    for (int i = tid; i < m; i += nt) {
      float s = 0.f;
      const float* row = Asl + static_cast<size_t>(i) * ld;
      for (int e = 0; e < nl; ++e) s = fmaf(row[sup_j[e]], coef[e], s);
      out[i] = s;
    }
  };
  // cluster-sum of an m-vector partial in slot `x` -> out
  auto reduce_m = [&](const float* x, float* out) {
    for (int i = tid; i < m; i += nt) {
      float s = 0.f;
      for (int p = 0; p < CS; ++p) s += peer_ptr(x, p)[i];
      out[i] = s;
    }
  };
  // v <- P_perp v = v - W G^{-1} W^T v   (in place, all threads)
  auto proj = [&](float* v) {
    float acc[R];
#pragma unroll
    for (int l = 0; l < R; ++l) acc[l] = 0.f;
    for (int i = tid; i < m; i += nt) {
      const float vi = v[i];
#pragma unroll
      for (int l = 0; l < R; ++l) acc[l] = fmaf(W[i * R + l], vi, acc[l]);
    }
    block_sum_vec<R>(acc, r, redf, cvec);
    if (tid == 0) {
      for (int l = 0; l < R; ++l) xsol[l] = l < r ? static_cast<double>(cvec[l]) : 0.0;
      chol_solve(Lc, xsol, r, kMaxR);
      for (int l = 0; l < R; ++l) cvec[l] = l < r ? static_cast<float>(xsol[l]) : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < m; i += nt) {
      float s = v[i];
#pragma unroll
      for (int l = 0; l < R; ++l) s = fmaf(-W[i * R + l], cvec[l], s);
      v[i] = s;
    }
    __syncthreads();
  };
  // W^T v solved by G: coefficients (float) in cvec[0..r)
  auto ls_coef = [&](const float* v) {
    float acc[R];
#pragma unroll
    for (int l = 0; l < R; ++l) acc[l] = 0.f;
    for (int i = tid; i < m; i += nt) {
      const float vi = v[i];
#pragma unroll
      for (int l = 0; l < R; ++l) acc[l] = fmaf(W[i * R + l], vi, acc[l]);
    }
    block_sum_vec<R>(acc, r, redf, cvec);
    if (tid == 0) {
      for (int l = 0; l < R; ++l) xsol[l] = l < r ? static_cast<double>(cvec[l]) : 0.0;
      chol_solve(Lc, xsol, r, kMaxR);
      for (int l = 0; l < R; ++l) cvec[l] = l < r ? static_cast<float>(xsol[l]) : 0.f;
    }
    __syncthreads();
  };
  // A s exchange (local support values sup_v); optionally carries the Gram
  // partial and the local support count.  Result (A s) in dv; Gram -> Lc.
  auto exchange_As = [&](bool with_gram) {
    unsigned char* x = xslot(ex);
    float* xa = reinterpret_cast<float*>(x);
    double* xgram = reinterpret_cast<double*>(x + a16(static_cast<size_t>(m) * 4));
    int* xcnt = reinterpret_cast<int*>(x + a16(static_cast<size_t>(m) * 4) + kMaxR * kMaxR * 8);
    gather(sup_v, xa);
    if (with_gram) {
      const int mc = (m + CS - 1) / CS;
      const int ilo = c * mc, ihi = min(m, ilo + mc);
      for (int t = tid; t < r * r; t += nt) {
        const int p = t / r, q2 = t - p * r;
        double s = 0.0;
        if (q2 <= p)
          for (int i = ilo; i < ihi; ++i)
            s += static_cast<double>(W[i * R + p]) * static_cast<double>(W[i * R + q2]);
        xgram[p * kMaxR + q2] = s;
      }
    }
    if (tid == 0) *xcnt = *nloc_p;
    cluster_sync_all();
    reduce_m(xa, dv);
    if (tid < CS) cn[tid] = *peer_ptr(xcnt, tid);
    if (with_gram) {
      for (int t = tid; t < r * r; t += nt) {
        const int p = t / r, q2 = t - p * r;
        if (q2 <= p) {
          double s = 0.0;
          for (int pp = 0; pp < CS; ++pp) s += peer_ptr(xgram, pp)[p * kMaxR + q2];
          Gm[p * kMaxR + q2] = s;
          Gm[q2 * kMaxR + p] = s;
        }
      }
    }
    ++ex;
    __syncthreads();
    if (with_gram && tid == 0) {
      if (!chol_lower(Gm, Lc, r, kMaxR)) {
        flags[0] = 1;
        report_error(a.err, kErrNotSPD, k);
        for (int p = 0; p < r; ++p)
          for (int q2 = 0; q2 < r; ++q2) Lc[p * kMaxR + q2] = (p == q2) ? 1.0 : 0.0;
      }
    }
    __syncthreads();
  };

  // HardThreshold over the cluster: values vv[0..nsc) -> new local support.
  // When keep_values is false the new support keeps zero values (used for
  // the support of g when s = 0).
  auto hard_threshold = [&](bool keep_values) {
    for (int j = tid; j < nsc; j += nt) keys[j] = ht_key(vv[j], j0 + j);
    __syncthreads();
    for (int j = tid; j < nsc; j += nt) {
      const int blk = j / kSelBlk, lo = blk * kSelBlk, hi = min(nsc, lo + kSelBlk);
      const uint64_t kj = keys[j];
      int cnt = 0;
      for (int l = lo; l < hi; ++l) cnt += keys[l] > kj;
      if (cnt < rho) bc[blk * rho + cnt] = j;
    }
    __syncthreads();
    unsigned char* x = xslot(ex);
    int* xcnt = reinterpret_cast<int*>(x);
    uint64_t* xkey = reinterpret_cast<uint64_t*>(x + 16);
    float* xval = reinterpret_cast<float*>(x + 16 + static_cast<size_t>(rho) * 8);
    const int nb = (nsc + kSelBlk - 1) / kSelBlk;
    // candidates of all local blocks (block b contributes min(rho, size_b))
    int ncb = 0;
    for (int b = 0; b < nb; ++b) ncb += min(rho, min(nsc, (b + 1) * kSelBlk) - b * kSelBlk);
    for (int t = tid; t < ncb; t += nt) {
      int b = 0, s = t;
      while (s >= min(rho, min(nsc, (b + 1) * kSelBlk) - b * kSelBlk)) {
        s -= min(rho, min(nsc, (b + 1) * kSelBlk) - b * kSelBlk);
        ++b;
      }
      const int j = bc[b * rho + s];
      const uint64_t kj = keys[j];
      int cnt = 0;
      for (int b2 = 0; b2 < nb; ++b2) {
        const int nb2 = min(rho, min(nsc, (b2 + 1) * kSelBlk) - b2 * kSelBlk);
        for (int s2 = 0; s2 < nb2; ++s2) cnt += keys[bc[b2 * rho + s2]] > kj;
      }
      if (cnt < rho) {
        xkey[cnt] = kj;
        xval[cnt] = keep_values ? vv[j] : 0.f;
      }
    }
    if (tid == 0) *xcnt = min(rho, nsc);
    cluster_sync_all();
    for (int t = tid; t < CS * rho; t += nt) {
      const int p = t / rho, s = t - p * rho;
      const unsigned char* px = peer_ptr(x, p);
      const int cp = *reinterpret_cast<const int*>(px);
      if (s < cp) {
        ck[t] = reinterpret_cast<const uint64_t*>(px + 16)[s];
        cvv[t] = reinterpret_cast<const float*>(px + 16 + static_cast<size_t>(rho) * 8)[s];
      } else {
        ck[t] = 0ull;
      }
      if (s == 0) cn[p] = cp;
    }
    ++ex;
    __syncthreads();
    // clear the old support in the dense local s
    if (tid == 0) {
      const int nl = *nloc_p;
      for (int e = 0; e < nl; ++e) sl[sup_j[e]] = 0.f;
    }
    __syncthreads();
    // own candidates: selected iff their cluster-wide rank is < rho; the
    // selected ones form a prefix of the (descending) own list.
    const int own = cn[c];
    for (int s = tid; s < own; s += nt) {
      const uint64_t kj = ck[c * rho + s];
      int g = 0;
      for (int p = 0; p < CS; ++p) g += count_greater(ck + p * rho, cn[p], kj);
      flags[1 + s] = (g < rho) ? 1 : 0;
    }
    __syncthreads();
    if (tid == 0) {
      int cnt = 0;
      for (int s = 0; s < own; ++s) {
        if (!flags[1 + s]) break;
        const int j = key_index(ck[c * rho + s]) - j0;
        sup_j[cnt] = j;
        sup_v[cnt] = cvv[c * rho + s];
        sl[j] = cvv[c * rho + s];
        ++cnt;
      }
      *nloc_p = cnt;
    }
    __syncthreads();
  };

  // ---------------------------------------------------------- W pass -----
  bool need_gram = false;
  if (project) {
    float* xw = reinterpret_cast<float*>(xslot(ex));
    for (int i = tid; i < m; i += nt) {
      float acc[R];
#pragma unroll
      for (int l = 0; l < R; ++l) acc[l] = 0.f;
      const float4* arow = reinterpret_cast<const float4*>(Asl + static_cast<size_t>(i) * ld);
      for (int jq = 0; jq < nq; ++jq) {
        const float4 av = arow[jq];
        const float* u0 = Us + (4 * jq) * R;
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
#pragma unroll
      for (int l = 0; l < R; ++l) xw[i * R + l] = acc[l];
    }
    cluster_sync_all();
    for (int t = tid; t < m * R; t += nt) {
      float s = 0.f;
      for (int p = 0; p < CS; ++p) s += peer_ptr(xw, p)[t];
      W[t] = s;
    }
    ++ex;
    __syncthreads();
    need_gram = true;
  }

  // ----------------------------------------------------- IHT (Alg. 2) ----
  const int tau = (a.mode == kModeLS || rho == 0) ? 0 : a.tau;
  for (int it = 0; it < tau; ++it) {
    const bool zero_start = (a.mode == kModeInit && it == 0);
    // u = P_perp (A s - y)   (A s = 0 for the zero start)
    if (zero_start) {
      for (int i = tid; i < m; i += nt) dv[i] = -yv[i];
      __syncthreads();
    } else {
      exchange_As(need_gram);
      need_gram = false;
      for (int i = tid; i < m; i += nt) dv[i] -= yv[i];
      __syncthreads();
      if (project) proj(dv);
    }
    col_pass(dv);  // g = A^T u  (= M^T (M s - z) because P_perp is a projector)
    if (zero_start) {
      // support G of the zero start: the rho largest |g_i|
      for (int j = tid; j < nsc; j += nt) vv[j] = gs[j];
      __syncthreads();
      hard_threshold(false);
    }
    // ||g_G||^2 and A g_G on the support, then mu
    {
      unsigned char* x = xslot(ex);
      float* xg = reinterpret_cast<float*>(x);
      float* xnum = reinterpret_cast<float*>(x + a16(static_cast<size_t>(m) * 4));
      if (tid == 0) {
        const int nl = *nloc_p;
        float s = 0.f;
        for (int e = 0; e < nl; ++e) {
          const float gv = gs[sup_j[e]];
          s = fmaf(gv, gv, s);
        }
        *xnum = s;
      }
      // coefficients g on the support
      if (tid < *nloc_p) vv[tid] = gs[sup_j[tid]];
      __syncthreads();
      gather(vv, xg);
      cluster_sync_all();
      reduce_m(xg, ev);
      float num = 0.f;
      for (int p = 0; p < CS; ++p) num += *peer_ptr(xnum, p);
      ++ex;
      __syncthreads();
      if (project) proj(ev);
      float part = 0.f;
      for (int i = tid; i < m; i += nt) part = fmaf(ev[i], ev[i], part);
      const float den = block_sum(part, redd_f);
      if (!(den > 0.f)) break;  // ||M g_G|| = 0: the column's IHT stops
      float mu = num / den;
      if (!isfinite(mu)) {
        if (tid == 0) report_error(a.err, kErrNaN, k);
        mu = 0.f;
      }
      for (int j = tid; j < nsc; j += nt) vv[j] = fmaf(-mu, gs[j], sl[j]);
      __syncthreads();
    }
    hard_threshold(true);
  }

  // ------------------------------------------------------ final stage -----
  exchange_As(need_gram);  // A s with the final support (+ counts of every CTA)
  if (a.mode == kModeInit) {
    for (int i = tid; i < m; i += nt) dv[i] = yv[i] - dv[i];  // y - A s
    __syncthreads();
  } else {
    for (int i = tid; i < m; i += nt) dv[i] = yv[i] - dv[i];  // y - A s
    __syncthreads();
    ls_coef(dv);                                                // b = G^{-1} W^T (y - A s)
    if (c == 0 && tid < r) a.B[static_cast<size_t>(k) * r + tid] = cvec[tid];
    if (a.mode == kModeIter) {
      for (int i = tid; i < m; i += nt) {  // W b + A s - y
        float s = -dv[i];
#pragma unroll
        for (int l = 0; l < R; ++l) s = fmaf(W[i * R + l], cvec[l], s);
        dv[i] = s;
      }
      __syncthreads();
    }
  }
  if (a.mode != kModeLS) {
    col_pass(dv);
    float* Hk = a.H + static_cast<size_t>(k) * n + j0;
    for (int j = tid; j < nsc; j += nt) Hk[j] = gs[j];
    // S_k: this CTA's entries, ascending by index, after those of lower ranks
    if (tid == 0) {
      int off = 0;
      for (int p = 0; p < c; ++p) off += cn[p];
      const int nl = *nloc_p;
      for (int e = 1; e < nl; ++e) {  // insertion sort by local index
        const int jj = sup_j[e];
        const float vvv = sup_v[e];
        int f = e - 1;
        while (f >= 0 && sup_j[f] > jj) {
          sup_j[f + 1] = sup_j[f];
          sup_v[f + 1] = sup_v[f];
          --f;
        }
        sup_j[f + 1] = jj;
        sup_v[f + 1] = vvv;
      }
      for (int e = 0; e < nl && off + e < rho; ++e) {
        a.S_idx[static_cast<size_t>(k) * rho + off + e] = j0 + sup_j[e];
        a.S_val[static_cast<size_t>(k) * rho + off + e] = sup_v[e];
      }
    }
  }
  cluster_sync_all();  // no CTA leaves while a peer may still read its slots
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

// repack q_chunk columns of row-major A_k into the slab layout
__global__ void repack_kernel(GaussLayout L, const float* __restrict__ Ain, int k0, int kc,
                              float* __restrict__ Aout) {
  const size_t per_col = static_cast<size_t>(L.cs) * L.m * L.ns_pad;
  const size_t total = per_col * kc;
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t kk = t / per_col;
    size_t rem = t - kk * per_col;
    const int c = static_cast<int>(rem / (static_cast<size_t>(L.m) * L.ns_pad));
    rem -= static_cast<size_t>(c) * L.m * L.ns_pad;
    const int i = static_cast<int>(rem / L.ns_pad);
    const int jj = static_cast<int>(rem - static_cast<size_t>(i) * L.ns_pad);
    const int j = c * L.ns + jj;
    float v = 0.f;
    if (jj < L.ns && j < L.n) v = Ain[(kk * L.m + i) * L.n + j];
    Aout[(static_cast<size_t>(k0) + kk) * per_col + rem + static_cast<size_t>(c) * L.m * L.ns_pad] = v;
  }
}

}  // namespace

size_t sweep_smem_bytes(const GaussLayout& L, int resident, int nthreads) {
  return carve(L, resident, nthreads).total;
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
                        int resident, int nthreads, int ncols, cudaStream_t s) {
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3(static_cast<unsigned>(ncols) * L.cs, 1, 1);
  cfg.blockDim = dim3(nthreads, 1, 1);
  cfg.dynamicSmemBytes = sweep_smem_bytes(L, resident, nthreads);
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = L.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

int sweep_max_active_clusters(const GaussLayout& L, int resident, int nthreads) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, L, resident, nthreads, L.q, nullptr);
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, pick_kernel(L.r, resident), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

cudaError_t sweep_launch(const SweepArgs& a, int nthreads, cudaStream_t s) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, a.L, a.resident, nthreads, a.L.q, s);
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
