// Per-column sweep of AltGDmin-LR+S for the Gaussian operator (Algorithm 1
// with Algorithm 2), one thread-block cluster of CS CTAs per column k.
//
// Storage.  The cluster's CTAs split A_k by columns j into slabs of `ns`
// columns; a slab is a run of 32-column tiles, each tile m rows x 128 bytes
// with the 16-byte chunks of row i XOR-permuted by (i mod 8), so that 128-bit
// reads by a thread per row (row products) and by lanes spread over
// (4 rows x 8 chunks) (column products) hit distinct shared-memory banks.  A
// slab either stays in shared memory for the whole column (one TMA bulk
// copy) or streams through a ring of S tile stages that a producer warp fills
// with TMA bulk copies, once per product, while the consumer warps work on
// earlier tiles (the slab stays hot in L2 after the first product).  The
// columns of A_k on the current support are kept in a small shared-memory
// cache so that the sparse products A s and A g_G need no global loads.
//
// Products of one column-iteration:
//   W_k = A_k U                                 (row pass, r wide)
//   u   = P_perp(A_k s - y_k)                   (sparse product + r x r solve)
//   g   = A_k^T u                               (column pass)
//   mu  = ||g_G||^2 / ||P_perp A_k g_G||^2      (sparse product on the support G)
//   s   = HardThreshold(s - mu g, rho)          (radix select, cluster merge)
//   b_k = G_k^{-1} W_k^T (y_k - A_k s)          (FP64 inverse Gram)
//   h_k = A_k^T (W_k b_k + A_k s - y_k)         (column pass; gradient term)
// with P_perp v = v - W_k G_k^{-1} W_k^T v and G_k = W_k^T W_k.  G_k, its
// Cholesky factor, its inverse and the r x r solves are FP64; everything
// else is FP32.
//
// Cluster exchanges.  Partial results of the slabs are combined through
// distributed shared memory: each CTA writes its partial into one of two
// exchange slots in its own shared memory and signals every peer's mbarrier
// for that slot (release at cluster scope); each CTA waits on its own
// mbarrier and sums the partials of all CTAs in rank order, so every CTA
// holds bit-identical reduced values and takes identical control-flow
// decisions.  A slot is rewritten two exchanges later, after every peer has
// signalled the exchange in between, i.e. after it finished reading.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "lrs_dev.cuh"
#include "lrs_internal.h"

namespace lrs {
namespace sweep {

constexpr int kMaxR = 16;
constexpr int kNT = 256;      // consumer threads per CTA
constexpr int kNW = kNT / 32;
constexpr int kThreadsAll = kNT + 32;  // + one producer warp
constexpr int kTW = 32;       // tile width (columns)
constexpr int kCacheBytes = 24 * 1024;  // support-column cache (streamed slabs)

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline int cache_slots(const GaussLayout& L, int resident) {
  if (resident || L.rho == 0) return 0;
  int c = static_cast<int>(kCacheBytes / (static_cast<size_t>(L.m) * 4));
  return c < L.rho ? c : L.rho;
}

struct Carve {
  size_t bars, slab, Us, W, yv, dv, ev, gs, sl, vv, gpart, hist, tie, ck, cv, cn, Gm, fsm, flags,
      redf, sup, cache, rsc, xch, xs, total;
};

__host__ __device__ inline size_t tile_bytes(const GaussLayout& L) {
  return (size_t)L.m * kTW * elem_bytes(L.et);
}

__host__ __device__ inline Carve carve(const GaussLayout& L, int resident) {
  Carve c;
  size_t o = 0;
  const int R = sweep_rpad(L.r);
  const int rho = L.rho > 0 ? L.rho : 1;
  const int ntile = L.ns / kTW;
  const int nc = cache_slots(L, resident);
  c.bars = o;  o += a16(8 * (2 * 16 + 4));                   // ring full/empty, slab, exchange
  c.slab = o;  o += a16(tile_bytes(L) * (resident ? ntile : L.stages));
  c.Us = o;    o += a16((size_t)L.ns * R * 4);
  c.W = o;     o += a16((size_t)L.m * R * 4);
  c.yv = o;    o += a16((size_t)L.m * 4);
  c.dv = o;    o += a16((size_t)L.m * 4);
  c.ev = o;    o += a16((size_t)L.m * 4);
  c.gs = o;    o += a16((size_t)L.ns * 4);
  c.sl = o;    o += a16((size_t)L.ns * 4);
  c.vv = o;    o += a16((size_t)L.ns * 4);
  c.gpart = o; o += a16((size_t)kNW * L.ns * 4);
  c.hist = o;  o += a16(256 * 4 + 64);
  c.tie = o;   o += a16((size_t)(L.ns + 2 * rho + 8) * 4);   // tie list + selection list
  c.ck = o;    o += a16((size_t)L.cs * rho * 8);
  c.cv = o;    o += a16((size_t)L.cs * rho * 4);
  c.cn = o;    o += a16((size_t)L.cs * 4);
  c.Gm = o;    o += a16(3 * kMaxR * kMaxR * 8);       // G (then L^-1), L, G^-1 (FP64)
  c.fsm = o;   o += a16(4 * kMaxR * 8);               // FP64 r-vectors
  c.flags = o; o += a16((size_t)(rho + 8) * 4);
  c.redf = o;  o += a16((size_t)kNW * kMaxR * 4 + 256);
  c.sup = o;   o += a16((size_t)rho * 12 + 16);        // sup_j, sup_v, slot
  c.cache = o; o += a16((size_t)nc * L.m * 4 + (size_t)(nc + 1) * 4);
  c.rsc = o;   o += a16((size_t)2 * L.m * 4);                  // row scales (FP8 forms)
  const size_t xw = (size_t)L.m * R * 4;                            // W partial
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

// offset of element (i, j) inside a slab (tiles of m x 32, swizzled chunks)
__device__ __forceinline__ int elem_off(int m, int i, int j) {
  return (j >> 5) * (m * kTW) + i * kTW + ((((j & 31) >> 2) ^ (i & 7)) << 2) + (j & 3);
}

// ---- element access for the stored forms of A_k -----------------------------
// 4 consecutive columns 4q..4q+3 of row i of a tile (chunk q), dequantised
// (sc1/sc2: per-row scales of the FP8 forms, in shared memory).
template <int ET>
__device__ __forceinline__ float4 load4(const unsigned char* tile, int m, int i, int q,
                                        const float* sc1, const float* sc2) {
  const int off = i * kTW + ((q ^ (i & 7)) << 2);  // element offset of the chunk
  if constexpr (ET == 0) {
    return *reinterpret_cast<const float4*>(tile + static_cast<size_t>(off) * 4);
  } else if constexpr (ET == 1) {
    const uint2 raw = *reinterpret_cast<const uint2*>(tile + static_cast<size_t>(off) * 2);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
  } else {
    const __nv_fp8x4_e4m3 h = *reinterpret_cast<const __nv_fp8x4_e4m3*>(tile + off);
    const float4 fh = static_cast<float4>(h);
    const float s1 = sc1[i];
    float4 v = make_float4(fh.x * s1, fh.y * s1, fh.z * s1, fh.w * s1);
    if constexpr (ET == 3) {
      const __nv_fp8x4_e4m3 lo = *reinterpret_cast<const __nv_fp8x4_e4m3*>(tile + static_cast<size_t>(m) * kTW + off);
      const float4 fl = static_cast<float4>(lo);
      const float s2 = sc2[i];
      v.x = fmaf(fl.x, s2, v.x);
      v.y = fmaf(fl.y, s2, v.y);
      v.z = fmaf(fl.z, s2, v.z);
      v.w = fmaf(fl.w, s2, v.w);
    }
    return v;
  }
}
// element (i, j) of a slab (any tile), dequantised with the row's scales s1, s2
template <int ET>
__device__ __forceinline__ float elem1s(const unsigned char* slab, int m, int i, int j, float s1,
                                        float s2) {
  const size_t tb = static_cast<size_t>(m) * kTW * elem_bytes(ET);
  const unsigned char* tile = slab + static_cast<size_t>(j >> 5) * tb;
  const int off = i * kTW + ((((j & 31) >> 2) ^ (i & 7)) << 2) + (j & 3);
  if constexpr (ET == 0) {
    return *reinterpret_cast<const float*>(tile + static_cast<size_t>(off) * 4);
  } else if constexpr (ET == 1) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(tile + static_cast<size_t>(off) * 2));
  } else {
    float v = static_cast<float>(*reinterpret_cast<const __nv_fp8_e4m3*>(tile + off)) * s1;
    if constexpr (ET == 3)
      v = fmaf(static_cast<float>(*reinterpret_cast<const __nv_fp8_e4m3*>(tile + static_cast<size_t>(m) * kTW + off)),
               s2, v);
    return v;
  }
}
template <int ET>
__device__ __forceinline__ float elem1(const unsigned char* slab, int m, int i, int j,
                                       const float* sc1, const float* sc2) {
  if constexpr (ET >= 2)
    return elem1s<ET>(slab, m, i, j, sc1[i], ET == 3 ? sc2[i] : 0.f);
  else
    return elem1s<ET>(slab, m, i, j, 0.f, 0.f);
}

// HardThreshold order: larger |v| first, then the lower index.
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

// barrier among the consumer warps only (the producer warp runs ahead)
__device__ __forceinline__ void csync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kNT) : "memory");
}

// remote mbarrier arrive (release at cluster scope) on CTA `rank`'s copy
__device__ __forceinline__ void mbar_arrive_remote(uint64_t* bar, unsigned rank) {
  unsigned local = smem_u32(bar), remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive_local(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Per-phase cycle accounting (consumer thread 0 of cluster rank 0 only).
struct Tracer {
  unsigned long long* out;
  long long t0;
  __device__ __forceinline__ void mark(int phase) {
    if (out) {
      const long long t = clock64();
      out[phase] += static_cast<unsigned long long>(t - t0);
      t0 = t;
    }
  }
};

// Everything one CTA needs about its column and its shared memory.
struct Ctx {
  const unsigned char* Asl;   // resident slab (shared) or nullptr
  const unsigned char* Ag;    // this CTA's slab in global memory
  const unsigned char* ring;  // ring stages (streamed)
  size_t tbytes;              // bytes of one tile
  const float* sc1;           // per-row scales of the FP8 forms (shared)
  const float* sc2;
  uint64_t* full;    // ring barriers
  uint64_t* empty;
  uint64_t* xbar;    // exchange barriers [2]
  int stages, ntile;
  int m, n, r, rho, nsc, j0, c, CS, k;
  unsigned tile_seq; // consumer tile counter (uniform across consumer threads)
  float* Us;
  float* W;
  float* yv;
  float* dv;
  float* ev;
  float* gs;
  float* sl;
  float* vv;
  float* gpart;
  int* hist;
  int* tie;
  uint64_t* ck;
  float* cvv;
  int* cn;
  double* G;
  double* Lc;
  double* Gi;
  double* fv;
  int* flags;
  float* redf;
  int* sup_j;
  float* sup_v;
  int* sup_slot;     // cache slot of each local support entry (-1: not cached)
  int* nloc;
  float* cache;      // nc x m support columns
  int* cache_col;    // local column held by each slot (-1: free)
  int nc;
  unsigned char* xch;
  size_t xs;
  int* err;
};

__device__ __forceinline__ unsigned char* xslot(const Ctx& C, int e) {
  return C.xch + (e & 1) * C.xs;
}

// Publish this CTA's slot of exchange e to the cluster and wait for all
// peers' slots (consumer threads only).
__device__ __forceinline__ void xchg_publish_wait(const Ctx& C, int e) {
  csync();
  if (C.CS > 1) {
    if (threadIdx.x == 0) {
      asm volatile("fence.acq_rel.cluster;" ::: "memory");
      for (int p = 0; p < C.CS; ++p) mbar_arrive_remote(&C.xbar[e & 1], p);
    }
    const unsigned parity = (static_cast<unsigned>(e) >> 1) & 1u;
    unsigned it = 0;
    while (!mbar_try_wait_cluster(&C.xbar[e & 1], parity)) {
      if (++it > (1u << 22)) {
        if (threadIdx.x == 0) report_error(C.err, kErrTimeout, C.k);
        break;
      }
    }
  }
}

// ---- tile access --------------------------------------------------------
// Returns tile b of the current product (waiting for it when streamed).
__device__ __forceinline__ const unsigned char* acquire_tile(Ctx& C, int b) {
  if (C.Asl) return C.Asl + static_cast<size_t>(b) * C.tbytes;
  const unsigned s = C.tile_seq % C.stages, use = C.tile_seq / C.stages;
  unsigned it = 0;
  while (!mbar_try_wait(&C.full[s], use & 1u)) {
    if (++it > (1u << 22)) {
      if (threadIdx.x == 0) report_error(C.err, kErrTimeout, C.k);
      break;
    }
  }
  return C.ring + static_cast<size_t>(s) * C.tbytes;
}
__device__ __forceinline__ void release_tile(Ctx& C) {
  if (C.Asl) return;
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive_local(&C.empty[C.tile_seq % C.stages]);
  ++C.tile_seq;
}
// consume (without computing) the tiles of a product that is skipped
__device__ __forceinline__ void drain_pass(Ctx& C) {
  if (C.Asl) return;
  for (int b = 0; b < C.ntile; ++b) {
    acquire_tile(C, b);
    release_tile(C);
  }
}
// While the slots are pending (flag in cache_col[nc]), warp 0 copies the
// cached support columns that lie in tile b out of the tile.
template <int ET>
__device__ __forceinline__ void cache_fill_from_tile(const Ctx& C, const unsigned char* t, int b) {
  if ((threadIdx.x >> 5) != 0 || C.nc == 0 || !C.cache_col[C.nc]) return;
  for (int s = 0; s < C.nc; ++s) {
    const int j = C.cache_col[s];
    if (j >= b * kTW && j < (b + 1) * kTW)
      for (int i = threadIdx.x & 31; i < C.m; i += 32)
        C.cache[s * C.m + i] = elem1<ET>(t, C.m, i, j & 31, C.sc1, C.sc2);
  }
}

// ---------------------------------------------------------------- passes --
// g[0..nsc) = A_slab^T v.  Warps split the rows; in a tile each lane takes 4
// consecutive columns (chunk q = lane % 8) of rows i = 4t + lane / 8, summed
// over the lanes of a chunk by shuffles; per-warp partials then summed over
// warps in a fixed order.
template <int ET>
__device__ __forceinline__ void col_pass(Ctx& C, const float* v, bool fill_cache) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int RB = ((C.m + kNW - 1) / kNW + 3) & ~3;
  const int rlo = wid * RB, rhi = min(C.m, rlo + RB);
  const int q = lane & 7, ro = lane >> 3;
  for (int b = 0; b < C.ntile; ++b) {
    const unsigned char* t = acquire_tile(C, b);
    if (fill_cache) cache_fill_from_tile<ET>(C, t, b);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int i = rlo + ro; i < rhi; i += 4) {
      const float4 a = load4<ET>(t, C.m, i, q, C.sc1, C.sc2);
      const float u = v[i];
      acc.x = fmaf(a.x, u, acc.x);
      acc.y = fmaf(a.y, u, acc.y);
      acc.z = fmaf(a.z, u, acc.z);
      acc.w = fmaf(a.w, u, acc.w);
    }
#pragma unroll
    for (int o = 8; o <= 16; o <<= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
      acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
    }
    if (ro == 0)
      *reinterpret_cast<float4*>(C.gpart + wid * C.ntile * kTW + b * kTW + 4 * q) = acc;
    release_tile(C);
  }
  csync();
  for (int j = threadIdx.x; j < C.nsc; j += kNT) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kNW; ++w) s += C.gpart[w * C.ntile * kTW + j];
    C.gs[j] = s;
  }
  csync();
}

// Row iterations per lane of the W pass and the number of sub-passes over
// the slab it needs (each sub-pass covers up to 8 row iterations per lane).
__host__ __device__ inline int w_row_iters(int m) { return (((m + 7) / 8 + 3) / 4); }
__host__ __device__ inline int w_chunks(int m) { return (w_row_iters(m) + 7) / 8; }

// W partial = A_slab U_slab into dst (m x R).  Warps split the rows (RB per
// warp); in a tile, lane (ro = lane / 8, q = lane % 8) holds U for the tile's
// columns 4q..4q+3 in registers and accumulates rows w*RB + 4t + ro over all
// tiles; the 8 lanes of a row are summed by shuffles at the end.
template <int R, int ET>
__device__ __forceinline__ void w_pass(Ctx& C, float* dst) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int q = lane & 7, ro = lane >> 3;
  const int nri = w_row_iters(C.m), RB = 4 * nri;
  const int nch = (nri + 7) / 8;
  for (int ch = 0; ch < nch; ++ch) {
    float acc[8][R];
#pragma unroll
    for (int t = 0; t < 8; ++t)
#pragma unroll
      for (int l = 0; l < R; ++l) acc[t][l] = 0.f;
    for (int b = 0; b < C.ntile; ++b) {
      const unsigned char* tl = acquire_tile(C, b);
      if (ch == 0) cache_fill_from_tile<ET>(C, tl, b);
      float u[4 * R];
      const float4* u4 = reinterpret_cast<const float4*>(C.Us + (b * kTW + 4 * q) * R);
#pragma unroll
      for (int z = 0; z < R; ++z) {
        const float4 w = u4[z];
        u[4 * z] = w.x; u[4 * z + 1] = w.y; u[4 * z + 2] = w.z; u[4 * z + 3] = w.w;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = wid * RB + 4 * (ch * 8 + t) + ro;
        if (ch * 8 + t < nri && i < C.m) {
          const float4 a = load4<ET>(tl, C.m, i, q, C.sc1, C.sc2);
#pragma unroll
          for (int l = 0; l < R; ++l) {
            float s = acc[t][l];
            s = fmaf(a.x, u[l], s);
            s = fmaf(a.y, u[R + l], s);
            s = fmaf(a.z, u[2 * R + l], s);
            s = fmaf(a.w, u[3 * R + l], s);
            acc[t][l] = s;
          }
        }
      }
      release_tile(C);
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int i = wid * RB + 4 * (ch * 8 + t) + ro;
#pragma unroll
      for (int l = 0; l < R; ++l) {
        float v = acc[t][l];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        if ((l & 7) == q && ch * 8 + t < nri && i < C.m) dst[i * R + l] = v;
      }
    }
  }
}

// column e of the local support: A(i, sup_j[e])
template <int ET>
__device__ __forceinline__ float support_elem(const Ctx& C, int e, int i) {
  if (C.Asl) return elem1<ET>(C.Asl, C.m, i, C.sup_j[e], C.sc1, C.sc2);
  const int s = C.sup_slot[e];
  if (s >= 0) return C.cache[s * C.m + i];
  return elem1<ET>(C.Ag, C.m, i, C.sup_j[e], C.sc1, C.sc2);
}

// out[i] = sum_e coef[e] A(i, sup_j[e]) over the local support (partial of
// the cluster sum), in entry order.
template <int ET>
__device__ __forceinline__ void gather(const Ctx& C, const float* coef, float* out) {
  const int nl = *C.nloc;
  for (int i = threadIdx.x; i < C.m; i += kNT) {
    float s = 0.f;
    for (int e = 0; e < nl; ++e) s = fmaf(support_elem<ET>(C, e, i), coef[e], s);
    out[i] = s;
  }
}

// Give every local support entry a cache slot: entries whose column is
// already cached keep it; the others take free slots and are loaded from the
// slab in global memory (slots run out -> entry read from global when used).
template <int ET>
__device__ __forceinline__ void cache_assign_load(const Ctx& C) {
  if (C.Asl || C.nc == 0) return;
  const int nl = *C.nloc;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C.nc; ++s) C.flags[4 + s] = 0;  // slot in use by the new support
    for (int e = 0; e < nl; ++e) {
      C.sup_slot[e] = -1;
      for (int s = 0; s < C.nc; ++s)
        if (C.cache_col[s] == C.sup_j[e]) { C.sup_slot[e] = s; C.flags[4 + s] = 1; break; }
    }
    int fs = 0;
    for (int e = 0; e < nl; ++e) {
      if (C.sup_slot[e] >= 0) continue;
      while (fs < C.nc && C.flags[4 + fs]) ++fs;
      if (fs < C.nc) {
        C.sup_slot[e] = fs;
        C.flags[4 + fs] = 1;
        C.cache_col[fs] = -2 - C.sup_j[e];  // marks "load from global"
      }
    }
  }
  csync();
  // load the newly assigned slots from the slab in global memory
  for (int t = threadIdx.x; t < C.nc * C.m; t += kNT) {
    const int s = t / C.m, i = t - s * C.m;
    const int cc = C.cache_col[s];
    if (cc <= -2) C.cache[s * C.m + i] = elem1<ET>(C.Ag, C.m, i, -2 - cc, C.sc1, C.sc2);
  }
  csync();
  if (threadIdx.x == 0)
    for (int s = 0; s < C.nc; ++s)
      if (C.cache_col[s] <= -2) C.cache_col[s] = -2 - C.cache_col[s];
  csync();
}

// cluster-sum of an m-vector partial held in slot x -> out (rank order)
__device__ __forceinline__ void reduce_m(const Ctx& C, const float* x, float* out) {
  for (int i = threadIdx.x; i < C.m; i += kNT) {
    float s = 0.f;
    for (int p = 0; p < C.CS; ++p) s += peer_ptr(x, p)[i];
    out[i] = s;
  }
}

// x = G^{-1} W^T v: W^T v in FP32 (fixed-order block sum), the r x r solve in
// FP64; x (FP64) in C.fv[16 + l], as float in C.redf[kNW*kMaxR + l]
template <int R>
__device__ __forceinline__ void ls_solve(const Ctx& C, const float* v) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float acc[R];
#pragma unroll
  for (int l = 0; l < R; ++l) acc[l] = 0.f;
  for (int i = threadIdx.x; i < C.m; i += kNT) {
    const float vi = v[i];
#pragma unroll
    for (int l = 0; l < R; ++l) acc[l] = fmaf(C.W[i * R + l], vi, acc[l]);
  }
#pragma unroll
  for (int l = 0; l < R; ++l) acc[l] = warp_sum(acc[l]);
  if (lane == 0) {
#pragma unroll
    for (int l = 0; l < R; ++l) C.redf[w * kMaxR + l] = acc[l];
  }
  csync();
  if (threadIdx.x < 32) {
    double cvec = 0.0;
    if (lane < C.r) {
      float s = 0.f;
#pragma unroll
      for (int ww = 0; ww < kNW; ++ww) s += C.redf[ww * kMaxR + lane];
      cvec = s;
    }
    double x = 0.0;
    for (int b = 0; b < C.r; ++b) {
      const double cb = __shfl_sync(0xffffffffu, cvec, b);
      if (lane < C.r) x = dfma(C.Gi[lane * kMaxR + b], cb, x);
    }
    if (lane < R) {
      C.fv[16 + lane] = lane < C.r ? x : 0.0;
      C.redf[kNW * kMaxR + lane] = lane < C.r ? static_cast<float>(x) : 0.f;
    }
  }
  csync();
}

// v <- P_perp v = v - W G^{-1} W^T v (in place)
template <int R>
__device__ __forceinline__ void proj(const Ctx& C, float* v) {
  ls_solve<R>(C, v);
  const float* xf = C.redf + kNW * kMaxR;
  for (int i = threadIdx.x; i < C.m; i += kNT) {
    float s = v[i];
#pragma unroll
    for (int l = 0; l < R; ++l) s = fmaf(-C.W[i * R + l], xf[l], s);
    v[i] = s;
  }
  csync();
}

// sum of squares of an m-vector (returned to every consumer thread, FP64 of
// an FP32 fixed-order sum)
__device__ __forceinline__ double norm2_m(const Ctx& C, const float* v) {
  float acc = 0.f;
  for (int i = threadIdx.x; i < C.m; i += kNT) acc = fmaf(v[i], v[i], acc);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) C.redf[kNW * kMaxR + 16 + (threadIdx.x >> 5)] = acc;
  csync();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kNW; ++i) s += C.redf[kNW * kMaxR + 16 + i];
  csync();
  return s;
}

// Cholesky of G (lane 0, FP64, no division: inverse pivots by rsqrt_fp64),
// then G^{-1} = L^{-T} L^{-1} by warp 0.  A pivot that is not positive
// marks the column as numerically failed (identity used to keep going).
__device__ __forceinline__ void factor_gram(const Ctx& C) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x, r = C.r;
  double* L = C.Lc;
  double* iL = C.fv + 32;
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
  double* Li = C.G;  // L^{-1}, lower triangular (G no longer needed)
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
// the FP64 partial Gram of this CTA's row range and factors it.  A s -> dv;
// every CTA's local support count -> cn[].
template <int R, int ET>
__device__ __forceinline__ void exchange_As(Ctx& C, int& ex, bool with_gram) {
  unsigned char* x = xslot(C, ex);
  float* xa = reinterpret_cast<float*>(x);
  double* xgram = reinterpret_cast<double*>(x + a16(static_cast<size_t>(C.m) * 4));
  int* xcnt = reinterpret_cast<int*>(x + a16(static_cast<size_t>(C.m) * 4) + kMaxR * kMaxR * 8);
  gather<ET>(C, C.sup_v, xa);
  if (with_gram) {
    // FP64 Gram of this CTA's row range: warp w takes entries t = w, w+8, ...
    // of the lower triangle; lanes stride the rows; fixed-order warp sum.
    const int mc = (C.m + C.CS - 1) / C.CS;
    const int ilo = C.c * mc, ihi = min(C.m, ilo + mc);
    const int r = C.r, lane = threadIdx.x & 31;
    for (int t = threadIdx.x >> 5; t < r * r; t += kNW) {
      const int p = t / r, q2 = t - p * r;
      if (q2 > p) continue;
      double s = 0.0;
      for (int i = ilo + lane; i < ihi; i += 32)
        s = dfma(static_cast<double>(C.W[i * R + p]), static_cast<double>(C.W[i * R + q2]), s);
      s = warp_sum(s);
      if (lane == 0) xgram[t] = s;
    }
  }
  if (threadIdx.x == 0) *xcnt = *C.nloc;
  xchg_publish_wait(C, ex);
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
  csync();
  if (with_gram) {
    factor_gram(C);
    csync();
  }
}

// Local top-K (K = min(rho, nsc)) of the keys (|vv[j]|, then lower index) by
// an 8-bit radix select on the float bits; the selected local indices are
// written in key order (descending) to C.tie[ns + 8 ...] and their count
// returned.
__device__ __forceinline__ int local_topk(Ctx& C) {
  const int nsc = C.nsc, K = min(C.rho, nsc);
  const int lane = threadIdx.x & 31;
  int* hist = C.hist;
  int* info = C.hist + 256;   // [0] digit, [1] remaining, [2] tie count, [3] sel count
  int* ties = C.tie;
  int* sel = C.tie + C.ntile * kTW;
  unsigned prefix = 0, mask = 0;
  if (threadIdx.x == 0) info[1] = K;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int t = threadIdx.x; t < 256; t += kNT) hist[t] = 0;
    csync();
    for (int j0 = threadIdx.x - lane; j0 < nsc; j0 += kNT) {
      const int j = j0 + lane;
      const unsigned key = j < nsc ? __float_as_uint(fabsf(C.vv[j])) : 0u;
      const bool in = j < nsc && (key & mask) == prefix;
      const unsigned digit = in ? ((key >> shift) & 255u) : 256u;
      const unsigned peers = __match_any_sync(0xffffffffu, digit);
      if (in && (__ffs(peers) - 1) == lane) atomicAdd(&hist[digit], __popc(peers));
    }
    csync();
    if (threadIdx.x < 32) {
      // lane owns bins 255-8*lane .. 248-8*lane (descending)
      const int need = info[1];
      int own[8], tot = 0;
#pragma unroll
      for (int z = 0; z < 8; ++z) { own[z] = hist[255 - 8 * lane - z]; tot += own[z]; }
      int incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int excl = incl - tot;
      if (excl < need && incl >= need) {
        int acc = excl;
#pragma unroll
        for (int z = 0; z < 8; ++z) {
          if (acc + own[z] >= need) {
            info[0] = 255 - 8 * lane - z;
            info[1] = need - acc;  // still to take among the chosen digit
            break;
          }
          acc += own[z];
        }
      }
    }
    csync();
    prefix |= static_cast<unsigned>(info[0]) << shift;
    mask |= 255u << shift;
  }
  // keys above T are in; among keys equal to T take the `need` lowest indices
  const unsigned T = prefix;
  const int need = info[1];
  if (threadIdx.x == 0) { info[2] = 0; info[3] = 0; }
  csync();
  for (int j = threadIdx.x; j < nsc; j += kNT) {
    const unsigned key = __float_as_uint(fabsf(C.vv[j]));
    if (key > T) sel[atomicAdd(&info[3], 1)] = j;
    else if (key == T) ties[atomicAdd(&info[2], 1)] = j;
  }
  csync();
  const int nt = info[2];
  for (int t = threadIdx.x; t < nt; t += kNT) {
    const int j = ties[t];
    int rank = 0;
    for (int u = 0; u < nt; ++u) rank += ties[u] < j;
    if (rank < need) sel[info[3] + rank] = j;  // placed after the > T ones
  }
  csync();
  // order the K selected by key (descending) into ties[] (reused)
  for (int t = threadIdx.x; t < K; t += kNT) {
    const int j = sel[t];
    const uint64_t kj = ht_key(C.vv[j], C.j0 + j);
    int rank = 0;
    for (int u = 0; u < K; ++u) rank += ht_key(C.vv[sel[u]], C.j0 + sel[u]) > kj;
    ties[rank] = j;
  }
  csync();
  return K;
}

// HardThreshold over the cluster: values vv[0..nsc) -> new local support
// (exactly rho entries cluster-wide, largest |v| first, ties to the lower
// index).  keep_values = false keeps zero values (support of g at s = 0).
// Single-CTA fast path of the local top-K: when this CTA holds the whole
// current support (rho entries), every element of the new top-rho has |v| at
// least the smallest |v| on the current support, so the candidates are the
// elements at or above it; they are ranked exactly by the full key.  Returns
// the number of candidates in key order in C.tie[0..K), or -1 when the
// candidate set is too large (the caller then uses the radix select).
__device__ __forceinline__ int local_topk_support(Ctx& C) {
  const int nl = *C.nloc, K = min(C.rho, C.nsc);
  if (C.CS != 1 || nl != C.rho || K == 0) return -1;
  int* info = C.hist + 256;
  int* cand = C.tie + C.ntile * kTW;   // up to 2*rho + 8 entries
  const int cap = 2 * C.rho + 8;
  float* tmin = reinterpret_cast<float*>(C.hist);
  if (threadIdx.x < 32) {
    float t = INFINITY;
    for (int e = threadIdx.x; e < nl; e += 32) t = fminf(t, fabsf(C.vv[C.sup_j[e]]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fminf(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (threadIdx.x == 0) { tmin[0] = t; info[3] = 0; }
  }
  csync();
  const float t0 = tmin[0];
  for (int j = threadIdx.x; j < C.nsc; j += kNT) {
    if (fabsf(C.vv[j]) >= t0) {
      const int slot = atomicAdd(&info[3], 1);
      if (slot < cap) cand[slot] = j;
    }
  }
  csync();
  const int c = info[3];
  if (c > cap) return -1;
  for (int t = threadIdx.x; t < c; t += kNT) {
    const int j = cand[t];
    const uint64_t kj = ht_key(C.vv[j], C.j0 + j);
    int rank = 0;
    for (int u = 0; u < c; ++u) rank += ht_key(C.vv[cand[u]], C.j0 + cand[u]) > kj;
    if (rank < K) C.tie[rank] = j;
  }
  csync();
  return K;
}

template <int ET>
__device__ __forceinline__ void hard_threshold(Ctx& C, int& ex, bool keep_values) {
  const int rho = C.rho;
  int K = local_topk_support(C);
  if (K < 0) K = local_topk(C);  // local candidates in key order in C.tie[0..K)
  unsigned char* x = xslot(C, ex);
  int* xcnt = reinterpret_cast<int*>(x);
  uint64_t* xkey = reinterpret_cast<uint64_t*>(x + 16);
  float* xval = reinterpret_cast<float*>(x + 16 + static_cast<size_t>(rho) * 8);
  for (int s = threadIdx.x; s < K; s += kNT) {
    const int j = C.tie[s];
    xkey[s] = ht_key(C.vv[j], C.j0 + j);
    xval[s] = keep_values ? C.vv[j] : 0.f;
  }
  if (threadIdx.x == 0) *xcnt = K;
  xchg_publish_wait(C, ex);
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
  csync();
  const int own = C.cn[C.c];
  for (int s = threadIdx.x; s < own; s += kNT) {
    const uint64_t kj = C.ck[C.c * rho + s];
    int g = 0;
    for (int p = 0; p < C.CS; ++p) g += count_greater(C.ck + p * rho, C.cn[p], kj);
    C.flags[1 + s] = (g < rho) ? 1 : 0;
  }
  const int nl_old = *C.nloc;
  for (int e = threadIdx.x; e < nl_old; e += kNT) C.sl[C.sup_j[e]] = 0.f;
  csync();
  if (threadIdx.x == 0) {
    int cnt = 0;
    while (cnt < own && C.flags[1 + cnt]) ++cnt;
    *C.nloc = cnt;
  }
  csync();
  const int cnt = *C.nloc;
  for (int s = threadIdx.x; s < cnt; s += kNT) {
    const int j = key_index(C.ck[C.c * rho + s]) - C.j0;
    const float val = C.cvv[C.c * rho + s];
    C.sup_j[s] = j;
    C.sup_v[s] = val;
    C.sl[j] = val;
  }
  csync();
  cache_assign_load<ET>(C);
}

// number of products over A_k of one column in each mode (the producer
// streams the slab once per product)
__device__ __forceinline__ int passes_of(int mode, int tau, int rho, int m) {
  const int wp = w_chunks(m);
  if (mode == kModeLS) return wp;
  const int t = (rho == 0) ? 0 : tau;
  return mode == kModeInit ? t + 1 : t + 1 + wp;
}

template <int R, bool RES, int ET>
__global__ void __launch_bounds__(kThreadsAll, 2) sweep_kernel(const SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const GaussLayout& L = a.L;
  const int tid = threadIdx.x;
  const bool producer = tid >= kNT;
  Ctx C;
  C.c = static_cast<int>(cluster_rank());
  C.CS = static_cast<int>(cluster_size());
  C.k = static_cast<int>(cluster_id_x());
  C.m = L.m;
  C.n = L.n;
  C.r = L.r;
  C.rho = L.rho;
  C.j0 = C.c * L.ns;
  C.nsc = max(0, min(L.ns, L.n - C.j0));
  C.ntile = L.ns / kTW;
  C.stages = L.stages;
  C.err = a.err;
  C.tile_seq = 0;
  const Carve cv = carve(L, RES ? 1 : 0);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + cv.bars);
  C.full = bars;
  C.empty = bars + 16;
  uint64_t* slab_bar = bars + 32;
  C.xbar = bars + 33;
  uint64_t* u_bar = bars + 35;
  C.tbytes = tile_bytes(L);
  const size_t slab_bytes = static_cast<size_t>(C.ntile) * C.tbytes;
  C.Ag = reinterpret_cast<const unsigned char*>(a.A) + (static_cast<size_t>(C.k) * C.CS + C.c) * slab_bytes;
  C.Asl = RES ? reinterpret_cast<const unsigned char*>(smem + cv.slab) : nullptr;
  C.ring = reinterpret_cast<const unsigned char*>(smem + cv.slab);
  C.sc1 = reinterpret_cast<const float*>(smem + cv.rsc);
  C.sc2 = C.sc1 + L.m;
  C.Us = reinterpret_cast<float*>(smem + cv.Us);
  C.W = reinterpret_cast<float*>(smem + cv.W);
  C.yv = reinterpret_cast<float*>(smem + cv.yv);
  C.dv = reinterpret_cast<float*>(smem + cv.dv);
  C.ev = reinterpret_cast<float*>(smem + cv.ev);
  C.gs = reinterpret_cast<float*>(smem + cv.gs);
  C.sl = reinterpret_cast<float*>(smem + cv.sl);
  C.vv = reinterpret_cast<float*>(smem + cv.vv);
  C.gpart = reinterpret_cast<float*>(smem + cv.gpart);
  C.hist = reinterpret_cast<int*>(smem + cv.hist);
  C.tie = reinterpret_cast<int*>(smem + cv.tie);
  C.ck = reinterpret_cast<uint64_t*>(smem + cv.ck);
  C.cvv = reinterpret_cast<float*>(smem + cv.cv);
  C.cn = reinterpret_cast<int*>(smem + cv.cn);
  C.G = reinterpret_cast<double*>(smem + cv.Gm);
  C.Lc = C.G + kMaxR * kMaxR;
  C.Gi = C.G + 2 * kMaxR * kMaxR;
  C.fv = reinterpret_cast<double*>(smem + cv.fsm);
  C.flags = reinterpret_cast<int*>(smem + cv.flags);
  C.redf = reinterpret_cast<float*>(smem + cv.redf);
  const int rho1 = max(C.rho, 1);
  C.sup_j = reinterpret_cast<int*>(smem + cv.sup);
  C.sup_v = reinterpret_cast<float*>(smem + cv.sup + static_cast<size_t>(rho1) * 4);
  C.sup_slot = reinterpret_cast<int*>(smem + cv.sup + static_cast<size_t>(rho1) * 8);
  C.nloc = reinterpret_cast<int*>(smem + cv.sup + static_cast<size_t>(rho1) * 12);
  C.nc = cache_slots(L, RES ? 1 : 0);
  C.cache = reinterpret_cast<float*>(smem + cv.cache);
  C.cache_col = reinterpret_cast<int*>(smem + cv.cache + static_cast<size_t>(C.nc) * C.m * 4);
  C.xch = smem + cv.xch;
  C.xs = cv.xs;
  int ex = 0;
  const int m = C.m, r = C.r, rho = C.rho, k = C.k;
  const size_t tbytes = tile_bytes(L);
  Tracer tr;
  tr.out = (a.trace && tid == 0 && C.c == 0) ? a.trace + static_cast<size_t>(k) * kTracePhases : nullptr;
  tr.t0 = clock64();

  // ---- barriers -----------------------------------------------------------
  if (tid == kNT) {
    if (RES) {
      mbar_init(slab_bar, 1);
    } else {
      for (int s = 0; s < C.stages; ++s) {
        mbar_init(&C.full[s], 1);
        mbar_init(&C.empty[s], kNW);
      }
    }
    mbar_init(&C.xbar[0], C.CS);
    mbar_init(&C.xbar[1], C.CS);
    mbar_init(u_bar, 1);
  }
  __syncthreads();
  if (C.CS > 1) cluster_sync_all();  // peers' barriers initialised before any remote arrive

  if (producer) {
    // ---- producer warp: U slab, then the A slab's tiles for every product --
    if (tid == kNT) {
      const unsigned ubytes = static_cast<unsigned>(static_cast<size_t>(L.ns) * R * 4);
      mbar_arrive_expect_tx(u_bar, ubytes);
      bulk_copy_g2s(C.Us, a.Upad + static_cast<size_t>(C.j0) * R, ubytes, u_bar);
      const char* src = reinterpret_cast<const char*>(C.Ag);
      char* dst = reinterpret_cast<char*>(smem + cv.slab);
      if (RES) {
        const size_t bytes = slab_bytes;
        mbar_arrive_expect_tx(slab_bar, static_cast<unsigned>(bytes));
        for (size_t off = 0; off < bytes; off += 32768) {
          const size_t rem = bytes - off;
          bulk_copy_g2s(dst + off, src + off, static_cast<unsigned>(rem < 32768 ? rem : 32768),
                        slab_bar);
        }
      } else {
        const unsigned total = static_cast<unsigned>(passes_of(a.mode, a.tau, rho, m) * C.ntile);
        for (unsigned t = 0; t < total; ++t) {
          const unsigned s = t % C.stages, use = t / C.stages;
          if (use > 0) {
            unsigned it = 0;
            while (!mbar_try_wait(&C.empty[s], (use - 1) & 1u))
              if (++it > (1u << 22)) { report_error(a.err, kErrTimeout, k); break; }
          }
          mbar_arrive_expect_tx(&C.full[s], static_cast<unsigned>(tbytes));
          bulk_copy_g2s(dst + s * tbytes, src + static_cast<size_t>(t % C.ntile) * tbytes,
                        static_cast<unsigned>(tbytes), &C.full[s]);
        }
      }
    }
    __syncwarp();
    if (C.CS > 1) cluster_sync_all();  // final cluster barrier (matches the consumers')
    return;
  }

  // ---- consumers: small operands -------------------------------------------
  for (int i = tid; i < m; i += kNT) C.yv[i] = a.y[static_cast<size_t>(k) * m + i];
  if (ET >= 2) {
    float* scw = reinterpret_cast<float*>(smem + cv.rsc);
    const int per = (ET == 3) ? 2 : 1;
    for (int i = tid; i < m; i += kNT) {
      scw[i] = a.rscale[(static_cast<size_t>(k) * m + i) * per];
      scw[m + i] = (ET == 3) ? a.rscale[(static_cast<size_t>(k) * m + i) * per + 1] : 0.f;
    }
  }
  for (int j = tid; j < L.ns; j += kNT) C.sl[j] = 0.f;
  for (int s = tid; s <= C.nc; s += kNT) C.cache_col[s] = -1;
  if (tid == 0) {
    C.flags[0] = 0;
    int cnt = 0;
    if (a.mode != kModeInit) {
      for (int e = 0; e < rho; ++e) {
        const int jg = a.S_idx[static_cast<size_t>(k) * rho + e];
        if (jg >= C.j0 && jg < C.j0 + C.nsc) {
          C.sup_j[cnt] = jg - C.j0;
          C.sup_v[cnt] = a.S_val[static_cast<size_t>(k) * rho + e];
          C.sup_slot[cnt] = cnt < C.nc ? cnt : -1;
          ++cnt;
        }
      }
    }
    *C.nloc = cnt;
    for (int s = 0; s < C.nc && s < cnt; ++s) C.cache_col[s] = C.sup_j[s];
    C.cache_col[C.nc] = 1;  // slots pending a fill from the streamed tiles
  }
  csync();
  for (int e = tid; e < *C.nloc; e += kNT) C.sl[C.sup_j[e]] = C.sup_v[e];
  if (!mbar_wait_bounded(u_bar, 0) && (tid & 31) == 0) report_error(a.err, kErrTimeout, k);
  if (RES) {
    if (!mbar_wait_bounded(slab_bar, 0) && (tid & 31) == 0) report_error(a.err, kErrTimeout, k);
  }
  csync();
  tr.mark(0);

  const bool project = (a.mode != kModeInit);

  // ---------------------------------------------------------- W pass -----
  bool need_gram = false;
  if (project) {
    float* xw = reinterpret_cast<float*>(xslot(C, ex));
    w_pass<R, ET>(C, C.CS > 1 ? xw : C.W);
    if (C.CS > 1) {
      xchg_publish_wait(C, ex);
      for (int t = tid; t < m * R; t += kNT) {
        float s = 0.f;
        for (int p = 0; p < C.CS; ++p) s += peer_ptr(xw, p)[t];
        C.W[t] = s;
      }
      ++ex;
    }
    need_gram = true;
  }
  if (tid == 0) C.cache_col[C.nc] = 0;  // W pass filled the slots (no-op if no W pass)
  csync();
  if (!project) cache_assign_load<ET>(C);  // no W pass streamed: load the slots directly
  tr.mark(1);

  // ----------------------------------------------------- IHT (Alg. 2) ----
  const int tau = (a.mode == kModeLS || rho == 0) ? 0 : a.tau;
  int it = 0;
  for (; it < tau; ++it) {
    const bool zero_start = (a.mode == kModeInit && it == 0);
    // u = P_perp (A s - y)   (A s = 0 for the zero start)
    if (zero_start) {
      for (int i = tid; i < m; i += kNT) C.dv[i] = -C.yv[i];
      csync();
    } else {
      exchange_As<R, ET>(C, ex, need_gram);
      need_gram = false;
      for (int i = tid; i < m; i += kNT) C.dv[i] -= C.yv[i];
      csync();
      tr.mark(2);
      if (project) proj<R>(C, C.dv);
      tr.mark(3);
    }
    col_pass<ET>(C, C.dv, false);  // g = A^T u  (= M^T (M s - z): P_perp is a projector)
    tr.mark(4);
    if (zero_start) {
      for (int j = tid; j < C.nsc; j += kNT) C.vv[j] = C.gs[j];
      csync();
      hard_threshold<ET>(C, ex, false);  // support G of the zero start
    }
    // ||g_G||^2 and A g_G on the support, then mu
    unsigned char* x = xslot(C, ex);
    float* xg = reinterpret_cast<float*>(x);
    double* xnum = reinterpret_cast<double*>(x + a16(static_cast<size_t>(m) * 4));
    const int nl = *C.nloc;
    for (int e = tid; e < nl; e += kNT) C.vv[e] = C.gs[C.sup_j[e]];
    csync();
    if (tid == 0) {
      double s = 0.0;
      for (int e = 0; e < nl; ++e) s = dfma(static_cast<double>(C.vv[e]), C.vv[e], s);
      *xnum = s;
    }
    gather<ET>(C, C.vv, xg);
    xchg_publish_wait(C, ex);
    reduce_m(C, xg, C.ev);
    double num = 0.0;
    for (int p = 0; p < C.CS; ++p) num += *peer_ptr(xnum, p);
    ++ex;
    csync();
    tr.mark(5);
    if (project) proj<R>(C, C.ev);
    const double den = norm2_m(C, C.ev);
    tr.mark(6);
    if (!(den > 0.0)) {  // ||M g_G|| = 0: the column's IHT stops
      ++it;
      break;
    }
    double mu = num / den;
    if (!isfinite(mu)) {
      if (tid == 0) report_error(a.err, kErrNaN, k);
      mu = 0.0;
    }
    const float muf = static_cast<float>(mu);
    for (int j = tid; j < C.nsc; j += kNT) C.vv[j] = fmaf(-muf, C.gs[j], C.sl[j]);
    csync();
    hard_threshold<ET>(C, ex, true);
    tr.mark(7);
  }
  for (; it < tau; ++it) drain_pass(C);  // products the stopped IHT no longer needs

  // ------------------------------------------------------ final stage -----
  exchange_As<R, ET>(C, ex, need_gram);  // A s with the final support
  for (int i = tid; i < m; i += kNT) C.dv[i] = C.yv[i] - C.dv[i];  // y - A s
  csync();
  tr.mark(8);
  if (a.mode != kModeInit) {
    ls_solve<R>(C, C.dv);  // b = G^{-1} W^T (y - A s)   (FP64 solve)
    if (C.c == 0 && tid < r) a.B[static_cast<size_t>(k) * r + tid] = static_cast<float>(C.fv[16 + tid]);
    if (a.mode == kModeIter) {
      const float* xf = C.redf + kNW * kMaxR;
      for (int i = tid; i < m; i += kNT) {  // W b + A s - y
        float s = -C.dv[i];
#pragma unroll
        for (int l = 0; l < R; ++l) s = fmaf(C.W[i * R + l], xf[l], s);
        C.ev[i] = s;
      }
      csync();
    }
  }
  tr.mark(9);
  if (a.mode != kModeLS) {
    col_pass<ET>(C, a.mode == kModeInit ? C.dv : C.ev, false);
    tr.mark(10);
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
  csync();
  tr.mark(11);
  if (C.CS > 1) cluster_sync_all();  // no CTA leaves while a peer may still read its slots
}

}  // namespace sweep
}  // namespace lrs
