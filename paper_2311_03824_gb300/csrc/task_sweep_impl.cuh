// Persistent task engine of the Gaussian sweep (kernel body; instantiated
// per rank width and element type in task_sweep.cu).
//
// One launch runs one sweep (mode INIT, LS or ITER of Algorithm 1's
// per-column work) over every column of every problem in a table.  Each
// column's work is a chain of passes over A_k:
//   ITER: W (W_k = A_k U), tau IHT passes (g = A_k^T u), final pass
//         (h_k = A_k^T e);   LS: W only;   INIT: tau0 IHT passes, final pass.
// A pass is split into tasks (W: row block x column chunk of tiles; A^T:
// column chunk of tiles over all rows).  A persistent grid of CTAs (8
// consumer warps + 1 producer warp) pops tasks from a global ticket queue:
// the producer warp pops the next ticket, waits until it is published and
// streams the task's pieces (one 32-column tile x a row range, plus the U
// rows of that tile for W tasks) by TMA bulk copies into a ring of shared
// stages; the consumer warps compute.  The CTA whose task completes a pass
// of column k (per-column counter) runs column k's small step on its
// consumer warps - Gram and Cholesky after W; mu and HardThreshold after an
// IHT pass (Algorithm 2); the LS for b_k and the residual before the final
// pass - and publishes the next pass's tasks.  A finished column admits the
// next one, so at most F columns are in flight (with few enough of them a
// column's A_k can stay in L2 between its passes; with all of them in flight,
// the default, each pass streams from HBM).
//
// Every wait is bounded (global timer); on expiry the CTA records
// kErrTimeout and leaves, so a launch always ends.
#pragma once

#include "sweep_gauss_impl.cuh"

namespace lrs {
namespace task {

using namespace sweep;

constexpr int kMaxStages = kTaskStages;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---- shared-memory carve -----------------------------------------------------
struct TCarve {
  size_t bars, task, ring, stage, W, yv, dv, ev, uv, gs, sl, vv, gpart, hist, tie, Gm, fv,
      flags, redf, sup, rsc, asv, osup, bcast, prof, total;
};
__host__ __device__ inline TCarve tcarve(int R, int m, int ns, int rho, int stages,
                                         int piece_bytes) {
  TCarve c;
  size_t o = 0;
  rho = rho > 0 ? rho : 1;
  c.bars = o;  o += a16(8 * (2 * kMaxStages + 6));  // ring, task slots, step copies
  c.task = o;  o += a16(2 * 8);
  c.stage = a16(static_cast<size_t>(piece_bytes) + static_cast<size_t>(kTW) * R * 4);
  c.ring = o;  o += c.stage * stages;
  c.W = o;     o += a16(static_cast<size_t>(m) * R * 4);
  c.yv = o;    o += a16(static_cast<size_t>(m) * 4);
  c.dv = o;    o += a16(static_cast<size_t>(m) * 4);
  c.ev = o;    o += a16(static_cast<size_t>(m) * 4);
  c.uv = o;    o += a16(static_cast<size_t>(m) * 4);
  c.gs = o;    o += a16(static_cast<size_t>(ns) * 4);
  c.sl = o;    o += a16(static_cast<size_t>(ns) * 4);
  c.vv = o;    o += a16(static_cast<size_t>(ns) * 4);
  // per-piece sums of one A^T task: at most kMaxTaskPieces, and at most the
  // column's tiles x row chunks (rows per piece >= 8)
  // ... and the W tasks' cross-warp sums (kNW x 32 rows x R)
  const int max_pieces = min(kMaxTaskPieces, (ns / kTW) * ((m + 7) / 8));
  const size_t gfl = max(static_cast<size_t>(max_pieces) * kTW, static_cast<size_t>(kNW) * 32 * R);
  c.gpart = o; o += a16(gfl * 4);
  c.hist = o;  o += a16(256 * 4 + 64);
  c.tie = o;   o += a16(static_cast<size_t>(ns + 2 * rho + 8) * 4);
  c.Gm = o;    o += a16(3 * kMaxR * kMaxR * 8);
  c.fv = o;    o += a16(4 * kMaxR * 8);
  c.flags = o; o += a16(static_cast<size_t>(rho + 8) * 4);
  c.redf = o;  o += a16(static_cast<size_t>(kNW) * kMaxR * 4 + 256);
  c.sup = o;   o += a16(static_cast<size_t>(rho) * 12 + 16);
  c.rsc = o;   o += a16(static_cast<size_t>(2) * m * 4);
  c.asv = o;   o += a16(static_cast<size_t>(m) * 4);              // A s of the column (step)
  c.osup = o;  o += a16(static_cast<size_t>(rho + 4) * 4);        // support before HardThreshold
  c.bcast = o; o += 16;  // [0] last task of a pass, [1] descriptor arrived
  c.prof = o;  o += 16 * 8;
  c.total = o;
  return c;
}

// ---- per-CTA state -------------------------------------------------------------
struct TCtx {
  uint64_t* full;
  uint64_t* empty;
  uint64_t* tfull;   // task slots [2]
  uint64_t* tempty;
  unsigned long long* tslot;
  unsigned char* ring;
  size_t stage;
  int stages;
  unsigned seq;      // consumer piece counter
  float* uv;
  float* gpart;
  float* rsc;
  int* bcast;
  int* err;
  int* abort;        // launch-wide: set once any wait of any CTA expired
  unsigned long long wait_ns;  // bound of every wait of the launch
  long long pw;      // thread 0: cycles waiting for pieces (profile)
};

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void set_abort(int* abort, int* err) {
  report_error(err, kErrTimeout, -1);
  atomicExch(abort, 1);
}

// Bounded wait on a shared-memory barrier: false after wait_ns or as soon as
// the launch is aborted (the caller then runs on without the data; every
// later wait returns at once, so all CTAs leave quickly).
__device__ __forceinline__ bool wait_bar(uint64_t* bar, unsigned parity, int* err, int* abort,
                                         unsigned long long wait_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try_wait(bar, parity)) {
    if (ld_relaxed(abort)) return false;
    if (gtimer() - t0 > wait_ns) {
      set_abort(abort, err);
      return false;
    }
  }
  return true;
}

// piece acquire / release on the consumer side (all 256 consumer threads)
__device__ __forceinline__ const unsigned char* acquire_piece(TCtx& T, bool& ok) {
  const unsigned s = T.seq % T.stages, use = T.seq / T.stages;
  const long long c0 = clock64();
  ok = wait_bar(&T.full[s], use & 1u, T.err, T.abort, T.wait_ns);
  T.pw += clock64() - c0;
  return T.ring + static_cast<size_t>(s) * T.stage;
}
__device__ __forceinline__ void release_piece(TCtx& T) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive_local(&T.empty[T.seq % T.stages]);
  ++T.seq;
}

__device__ __forceinline__ int ld_acquire_(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- queue -----------------------------------------------------------------------
// Publish n tasks (thread 0 of the consumers).  More tasks than the launch
// counts would be a bookkeeping error: the launch is aborted instead.
__device__ __forceinline__ void push_tasks(const TaskQueue& Q, int k, int prob, int type, int ph,
                                           int n) {
  const int t0 = atomicAdd(&Q.ctr[1], n);
  if (t0 + n > Q.total) {
    set_abort(&Q.ctr[3], Q.probs[prob].err);
    return;
  }
  for (int i = 0; i < n; ++i) Q.tasks[t0 + i] = tdesc(k, prob, type, ph, i);
  __threadfence();
  for (int i = 0; i < n; ++i) st_release(&Q.seq[t0 + i], 1);
}

// Publish n tasks at tickets [t0, t0 + n) reserved earlier (thread 0 of the
// consumers, after the barrier that ends the step): the descriptors, one
// fence that also covers the CTA's writes ordered by that barrier, then the
// flags.
__device__ __forceinline__ void publish_reserved(const TaskQueue& Q, int t0, int k, int prob,
                                                 int type, int ph, int n) {
  if (t0 < 0 || t0 + n > Q.total) {
    set_abort(&Q.ctr[3], Q.probs[prob].err);
    return;
  }
  for (int i = 0; i < n; ++i) Q.tasks[t0 + i] = tdesc(k, prob, type, ph, i);
  __threadfence();
  for (int i = 0; i < n; ++i) st_relaxed(&Q.seq[t0 + i], 1);
}

// problem owning global column c (the table is ordered by col0)
__device__ __forceinline__ int prob_of(const TaskQueue& Q, int c) {
  int p = 0;
  while (p + 1 < Q.nprob && Q.probs[p + 1].col0 <= c) ++p;
  return p;
}

// column finished: admit the next column of the launch (thread 0)
__device__ __forceinline__ void admit_next(const TaskQueue& Q) {
  const int c = atomicAdd(&Q.ctr[2], 1);
  if (c >= Q.ncols) return;
  const int p = prob_of(Q, c);
  const TaskProblem& P = Q.probs[p];
  push_tasks(Q, c - P.col0, p, phase_type(P, 0), 0, phase_tasks(P, 0));
}

// ---- producer: stream the pieces of one task ---------------------------------------
template <int R, int ET>
__device__ __forceinline__ void produce_task(TCtx& T, const TaskProblem& P, int k, int type,
                                             int blk, unsigned& pseq) {
  const GaussLayout& L = P.L;
  const int m = L.m, ntile = L.ns / kTW;
  constexpr int pb = ET == 0 ? 4 : ET == 1 ? 2 : 1;  // bytes per element of a plane
  const size_t tb = static_cast<size_t>(m) * kTW * elem_bytes(ET);
  const unsigned char* col = static_cast<const unsigned char*>(P.A) + static_cast<size_t>(k) * ntile * tb;
  auto piece = [&](int b, int i0, int i1, bool with_u) {
    const unsigned s = pseq % T.stages, use = pseq / T.stages;
    if (use > 0 && !wait_bar(&T.empty[s], (use - 1) & 1u, T.err, T.abort, T.wait_ns)) return false;
    unsigned char* dst = T.ring + static_cast<size_t>(s) * T.stage;
    const unsigned hb = static_cast<unsigned>((i1 - i0) * kTW * pb);
    const unsigned ub = with_u ? static_cast<unsigned>(kTW * R * 4) : 0u;
    mbar_arrive_expect_tx(&T.full[s], hb * (ET == 3 ? 2u : 1u) + ub);
    const unsigned char* src = col + static_cast<size_t>(b) * tb + static_cast<size_t>(i0) * kTW * pb;
    bulk_copy_g2s(dst, src, hb, &T.full[s]);
    if (ET == 3) bulk_copy_g2s(dst + hb, src + static_cast<size_t>(m) * kTW, hb, &T.full[s]);
    if (with_u)
      bulk_copy_g2s(dst + (T.stage - static_cast<size_t>(kTW) * R * 4),
                    P.Upad + static_cast<size_t>(b) * kTW * R, ub, &T.full[s]);
    ++pseq;
    return true;
  };
  if (type == kTaskW) {
    const int rb = blk / P.ncw, cc = blk - rb * P.ncw;
    const int i0 = rb * P.rpw, i1 = min(m, i0 + P.rpw);
    const int b0 = cc * P.TBW, b1 = min(ntile, b0 + P.TBW);
    for (int b = b0; b < b1; ++b)
      if (!piece(b, i0, i1, true)) return;
  } else if (type == kTaskG || type == kTaskF) {
    const int b0 = blk * P.TB, b1 = min(ntile, b0 + P.TB);
    for (int b = b0; b < b1; ++b)
      for (int c = 0; c < P.nrc; ++c)
        if (!piece(b, c * P.rp, min(m, c * P.rp + P.rp), false)) return;
  }
}

// ---- consumer: W task (partial W rows of one row block over a column chunk) -------
template <int R, int ET>
__device__ __forceinline__ void consume_w(TCtx& T, const TaskProblem& P, int k, int blk) {
  const GaussLayout& L = P.L;
  const int m = L.m, ntile = L.ns / kTW;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int q = lane & 7, ro = lane >> 3;
  const int rb = blk / P.ncw, cc = blk - rb * P.ncw;
  const int i0 = rb * P.rpw, nr = min(m, i0 + P.rpw) - i0;
  const int b0 = cc * P.TBW, b1 = min(ntile, b0 + P.TBW);
  const int RBw = ((nr + kNW - 1) / kNW + 3) & ~3;  // rows per warp (<= 16)
  const float* sc1 = T.rsc + i0;
  const float* sc2 = T.rsc + m + i0;
  float acc[4][R];
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int l = 0; l < R; ++l) acc[t][l] = 0.f;
  for (int b = b0; b < b1; ++b) {
    bool ok;
    const unsigned char* st = acquire_piece(T, ok);
    const float* Us = reinterpret_cast<const float*>(st + T.stage - static_cast<size_t>(kTW) * R * 4);
    float u[4 * R];
    const float4* u4 = reinterpret_cast<const float4*>(Us + 4 * q * R);
#pragma unroll
    for (int z = 0; z < R; ++z) {
      const float4 w = u4[z];
      u[4 * z] = w.x; u[4 * z + 1] = w.y; u[4 * z + 2] = w.z; u[4 * z + 3] = w.w;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int i = wid * RBw + 4 * t + ro;
      if (4 * t < RBw && i < nr) {
        const float4 a = load4<ET>(st, nr, i, q, sc1, sc2);
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
    release_piece(T);
  }
  float* out = P.Wp + (static_cast<size_t>(k) * P.ncw + cc) * P.wstride;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int i = wid * RBw + 4 * t + ro;
#pragma unroll
    for (int l = 0; l < R; ++l) {
      float v = acc[t][l];
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      if ((l & 7) == q && 4 * t < RBw && i < nr) out[static_cast<size_t>(i0 + i) * R + l] = v;
    }
  }
}

// ---- consumer: W task, pieces to warps round-robin (8 <= R <= 12) ----------------------
// Piece p of the task (tile b0 + p, rows i0..i0+nr) goes to warp p mod 8, as in
// the A^T tasks; a lane owns rows lane, lane + 32, ... (at most 4) of the row
// block over all 32 columns of its pieces (U of the tile read from the stage,
// the same address for every lane).  The warps' partial rows are then added
// in warp order through shared memory, 32 rows at a time.
template <int R, int ET>
__device__ __forceinline__ void consume_w_rr(TCtx& T, const TaskProblem& P, int k, int blk) {
  const GaussLayout& L = P.L;
  const int m = L.m, ntile = L.ns / kTW;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rb = blk / P.ncw, cc = blk - rb * P.ncw;
  const int i0 = rb * P.rpw, nr = min(m, i0 + P.rpw) - i0;
  const int b0 = cc * P.TBW, b1 = min(ntile, b0 + P.TBW);
  const int npieces = b1 - b0;
  const float* sc1 = T.rsc + i0;
  const float* sc2 = T.rsc + m + i0;
  float acc[4][R];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int l = 0; l < R; ++l) acc[u][l] = 0.f;
  const unsigned s0 = T.seq;
  for (int p = wid; p < npieces; p += kNW) {
    const unsigned sq = s0 + p, s = sq % T.stages, use = sq / T.stages;
    const long long c0 = clock64();
    wait_bar(&T.full[s], use & 1u, T.err, T.abort, T.wait_ns);
    if (lane == 0) T.pw += clock64() - c0;
    const unsigned char* st = T.ring + static_cast<size_t>(s) * T.stage;
    const float* Us = reinterpret_cast<const float*>(st + T.stage - static_cast<size_t>(kTW) * R * 4);
#pragma unroll 1
    for (int q = 0; q < kTW / 4; ++q) {  // 16-byte chunk of 4 columns
      float4 a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = lane + 32 * u;
        if constexpr (ET == 2) {  // FP8 hi: raw values, the row scale applied once below
          a[u] = i < nr ? static_cast<float4>(*reinterpret_cast<const __nv_fp8x4_e4m3*>(
                              st + i * kTW + ((q ^ (i & 7)) << 2)))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
          a[u] = i < nr ? load4<ET>(st, nr, i, q, sc1, sc2) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int l = 0; l < R; ++l) {
          const float uv = Us[(4 * q + c) * R + l];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float av = c == 0 ? a[u].x : c == 1 ? a[u].y : c == 2 ? a[u].z : a[u].w;
            acc[u][l] = fmaf(av, uv, acc[u][l]);
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive_local_n(&T.empty[s], kNW);  // the piece is free
  }
  T.seq = s0 + npieces;
  if constexpr (ET == 2) {  // a lane's rows are the same in all its pieces
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = lane + 32 * u;
      const float s1 = i < nr ? sc1[i] : 0.f;
#pragma unroll
      for (int l = 0; l < R; ++l) acc[u][l] *= s1;
    }
  }
  float* red = T.gpart;  // kNW x 32 x R
  float* out = P.Wp + (static_cast<size_t>(k) * P.ncw + cc) * P.wstride;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (32 * u >= nr) break;
    csync();
#pragma unroll
    for (int l = 0; l < R; ++l) red[(wid * 32 + lane) * R + l] = acc[u][l];
    csync();
    for (int t = threadIdx.x; t < 32 * R; t += kNT) {
      const int row = t / R, l = t - row * R, i = 32 * u + row;
      float sum = 0.f;
#pragma unroll
      for (int w = 0; w < kNW; ++w) sum += red[(w * 32 + row) * R + l];
      if (i < nr) out[static_cast<size_t>(i0 + i) * R + l] = sum;
    }
  }
}

// ---- consumer: A^T v task (one column chunk of tiles, all rows) ----------------------
// Pieces go to warps round-robin (piece p of the task -> warp p mod 8), each
// warp reduces its piece (rows of one tile) by shuffles alone and releases
// it with the weight of all warps; the per-piece sums of a tile are added in
// row-chunk order once the task's pieces are done (one barrier per task).
template <int ET>
__device__ __forceinline__ void consume_g(TCtx& T, const TaskProblem& P, int k, int blk,
                                          float* out) {
  const GaussLayout& L = P.L;
  const int m = L.m, ntile = L.ns / kTW;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int q = lane & 7, ro = lane >> 3;
  const int b0 = blk * P.TB, b1 = min(ntile, b0 + P.TB);
  const int npieces = (b1 - b0) * P.nrc;
  const unsigned s0 = T.seq;
  for (int p = wid; p < npieces; p += kNW) {
    const int bt = p / P.nrc, c = p - bt * P.nrc;
    const int i0 = c * P.rp, nr = min(m, i0 + P.rp) - i0;
    const unsigned sq = s0 + p, s = sq % T.stages, use = sq / T.stages;
    const long long c0 = clock64();
    wait_bar(&T.full[s], use & 1u, T.err, T.abort, T.wait_ns);
    if (lane == 0) T.pw += clock64() - c0;
    const unsigned char* st = T.ring + static_cast<size_t>(s) * T.stage;
    const float* uu = T.uv + i0;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (ET >= 2) {
      // FP8 forms: T.rsc holds the row scales times the pass vector, so an
      // element costs one multiply-add per plane
      const float* w1 = T.rsc + i0;
      const float* w2 = T.rsc + m + i0;
#pragma unroll 4
      for (int i = ro; i < nr; i += 4) {
        const int off = i * kTW + ((q ^ (i & 7)) << 2);
        const float4 fh = static_cast<float4>(*reinterpret_cast<const __nv_fp8x4_e4m3*>(st + off));
        const float a1 = w1[i];
        acc.x = fmaf(fh.x, a1, acc.x);
        acc.y = fmaf(fh.y, a1, acc.y);
        acc.z = fmaf(fh.z, a1, acc.z);
        acc.w = fmaf(fh.w, a1, acc.w);
        if constexpr (ET == 3) {
          const float4 fl = static_cast<float4>(
              *reinterpret_cast<const __nv_fp8x4_e4m3*>(st + static_cast<size_t>(nr) * kTW + off));
          const float a2 = w2[i];
          acc.x = fmaf(fl.x, a2, acc.x);
          acc.y = fmaf(fl.y, a2, acc.y);
          acc.z = fmaf(fl.z, a2, acc.z);
          acc.w = fmaf(fl.w, a2, acc.w);
        }
      }
    } else {
#pragma unroll 4
      for (int i = ro; i < nr; i += 4) {
        const float4 a = load4<ET>(st, nr, i, q, T.rsc + i0, T.rsc + m + i0);
        const float w = uu[i];
        acc.x = fmaf(a.x, w, acc.x);
        acc.y = fmaf(a.y, w, acc.y);
        acc.z = fmaf(a.z, w, acc.z);
        acc.w = fmaf(a.w, w, acc.w);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive_local_n(&T.empty[s], kNW);  // the piece is free
#pragma unroll
    for (int o = 8; o <= 16; o <<= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
      acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
    }
    if (ro == 0) *reinterpret_cast<float4*>(T.gpart + p * kTW + 4 * q) = acc;
  }
  T.seq = s0 + npieces;
  csync();
  for (int j = threadIdx.x; j < (b1 - b0) * kTW; j += kNT) {
    const int bt = j / kTW, jj = j - bt * kTW;
    float sum = 0.f;
    for (int c = 0; c < P.nrc; ++c) sum += T.gpart[(bt * P.nrc + c) * kTW + jj];
    const int jg = b0 * kTW + j;
    if (jg < L.n) out[jg] = sum;
  }
}

// ---- the column's small steps (consumer warps of the finishing CTA) ------------------
// Ctx of column k over this CTA's shared memory (single CTA: CS = 1).
__device__ __forceinline__ void small_ctx(Ctx& C, const TaskProblem& P, int k, unsigned char* smem,
                                          const TCarve& cv) {
  const GaussLayout& L = P.L;
  C.Asl = nullptr;
  C.tbytes = static_cast<size_t>(L.m) * kTW * elem_bytes(L.et);
  C.Ag = static_cast<const unsigned char*>(P.A) + static_cast<size_t>(k) * (L.ns / kTW) * C.tbytes;
  C.ring = nullptr;
  C.sc1 = reinterpret_cast<const float*>(smem + cv.rsc);
  C.sc2 = C.sc1 + L.m;
  C.stages = 0;
  C.ntile = L.ns / kTW;
  C.m = L.m;
  C.n = L.n;
  C.r = L.r;
  C.rho = L.rho;
  C.nsc = L.n;
  C.j0 = 0;
  C.c = 0;
  C.CS = 1;
  C.k = k;
  C.W = reinterpret_cast<float*>(smem + cv.W);
  C.yv = reinterpret_cast<float*>(smem + cv.yv);
  C.dv = reinterpret_cast<float*>(smem + cv.dv);
  C.ev = reinterpret_cast<float*>(smem + cv.ev);
  C.gs = reinterpret_cast<float*>(smem + cv.gs);
  C.sl = reinterpret_cast<float*>(smem + cv.sl);
  C.vv = reinterpret_cast<float*>(smem + cv.vv);
  C.hist = reinterpret_cast<int*>(smem + cv.hist);
  C.tie = reinterpret_cast<int*>(smem + cv.tie);
  C.G = reinterpret_cast<double*>(smem + cv.Gm);
  C.Lc = C.G + kMaxR * kMaxR;
  C.Gi = C.G + 2 * kMaxR * kMaxR;
  C.fv = reinterpret_cast<double*>(smem + cv.fv);
  C.flags = reinterpret_cast<int*>(smem + cv.flags);
  C.redf = reinterpret_cast<float*>(smem + cv.redf);
  const int rho1 = max(L.rho, 1);
  C.sup_j = reinterpret_cast<int*>(smem + cv.sup);
  C.sup_v = reinterpret_cast<float*>(smem + cv.sup + static_cast<size_t>(rho1) * 4);
  C.sup_slot = reinterpret_cast<int*>(smem + cv.sup + static_cast<size_t>(rho1) * 8);
  C.nloc = reinterpret_cast<int*>(smem + cv.sup + static_cast<size_t>(rho1) * 12);
  C.nc = 0;
  C.cache = nullptr;
  C.cache_col = nullptr;
  C.err = P.err;
}

// load y_k, W_k, G^{-1} (optional) and the support into shared memory
enum SupportSource : int { kSupNone = 0, kSupInput = 1, kSupState = 2 };
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async;" ::: "memory");
}

// y_k, W_k, G^{-1} (optional), the support and (optional) the IHT pass result
// g into shared memory.  W_k, G^{-1} and g (16-byte aligned blocks) come by
// TMA bulk copies that thread 0 issues while the threads load the rest; the
// proxy fence orders this CTA's earlier generic accesses to those buffers
// (and the other CTAs' writes it has acquired) before the copies.
template <int R>
__device__ __forceinline__ void load_column(Ctx& C, const TaskProblem& P, int k, bool with_w,
                                            bool with_gi, int source, bool with_g,
                                            uint64_t* sbar, unsigned& sphase, int* abort,
                                            unsigned long long wait_ns, float* asv = nullptr) {
  const int m = C.m, tid = threadIdx.x, rho = C.rho, ns = P.L.ns, n = P.L.n;
  const bool bulk = with_w || with_gi || with_g || asv;
  if (bulk) {
    fence_proxy_async();
    csync();
    if (tid == 0) {
      const unsigned bw = with_w ? static_cast<unsigned>(P.wstride) * 4u : 0u;
      const unsigned bgi = with_gi ? static_cast<unsigned>(kMaxR * kMaxR * 8) : 0u;
      const unsigned bg = with_g ? static_cast<unsigned>(ns) * 4u : 0u;
      const unsigned ba = asv ? static_cast<unsigned>(P.astride) * 4u : 0u;
      mbar_arrive_expect_tx(sbar, bw + bgi + bg + ba);
      if (ba) bulk_copy_g2s(asv, P.As + static_cast<size_t>(k) * P.astride, ba, sbar);
      if (bw) bulk_copy_g2s(C.W, P.Wk + static_cast<size_t>(k) * P.wstride, bw, sbar);
      if (bgi) bulk_copy_g2s(C.Gi, P.Gi + static_cast<size_t>(k) * kMaxR * kMaxR, bgi, sbar);
      if (bg) bulk_copy_g2s(C.gs, P.g + static_cast<size_t>(k) * ns, bg, sbar);
    }
  }
  for (int i = tid; i < m; i += kNT) C.yv[i] = __ldcg(P.y + static_cast<size_t>(k) * m + i);
  for (int j = tid; j < ns; j += kNT) C.sl[j] = 0.f;
  if (source == kSupState) {
    for (int e = tid; e < rho; e += kNT) {
      C.sup_j[e] = __ldcg(P.supj + static_cast<size_t>(k) * rho + e);
      C.sup_v[e] = __ldcg(P.supv + static_cast<size_t>(k) * rho + e);
      C.sup_slot[e] = -1;
    }
    if (tid == 0) *C.nloc = min(max(__ldcg(P.nsup + k), 0), rho);
  } else if (source == kSupInput) {
    // input support: loaded in parallel, then compacted (entries outside
    // the column are dropped)
    for (int e = tid; e < rho; e += kNT) {
      C.sup_slot[e] = P.S_idx[static_cast<size_t>(k) * rho + e];
      C.vv[e] = P.S_val[static_cast<size_t>(k) * rho + e];
    }
    csync();
    if (tid == 0) {
      int cnt = 0;
      for (int e = 0; e < rho; ++e) {
        const int j = C.sup_slot[e];
        if (j < 0 || j >= n) continue;
        C.sup_j[cnt] = j;
        C.sup_v[cnt] = C.vv[e];
        ++cnt;
      }
      for (int e = 0; e < rho; ++e) C.sup_slot[e] = -1;
      *C.nloc = cnt;
    }
  } else if (tid == 0) {
    *C.nloc = 0;
  }
  if (bulk && tid == 0) wait_bar(sbar, sphase, C.err, abort, wait_ns);  // on expiry the launch aborts
  if (bulk) sphase ^= 1u;
  csync();
  if (with_g)
    for (int j = n + tid; j < ns; j += kNT) C.gs[j] = 0.f;
  for (int e = tid; e < *C.nloc; e += kNT) C.sl[C.sup_j[e]] = C.sup_v[e];
  csync();
}

__device__ __forceinline__ void store_support(const Ctx& C, const TaskProblem& P, int k) {
  const int nl = *C.nloc;
  for (int e = threadIdx.x; e < nl; e += kNT) {
    P.supj[static_cast<size_t>(k) * C.rho + e] = C.sup_j[e];
    P.supv[static_cast<size_t>(k) * C.rho + e] = C.sup_v[e];
  }
  if (threadIdx.x == 0) P.nsup[k] = nl;
}

// HardThreshold of vv[0..n) on one CTA: the top-rho keys become the support
// (values vv, or 0 when keep_values is false); sl follows.
__device__ __forceinline__ void ht_single(Ctx& C, bool keep_values) {
  int K = local_topk_support(C);
  if (K < 0) K = local_topk(C);
  const int nl_old = *C.nloc;
  for (int e = threadIdx.x; e < nl_old; e += kNT) C.sl[C.sup_j[e]] = 0.f;
  csync();
  for (int s = threadIdx.x; s < K; s += kNT) {
    const int j = C.tie[s];
    const float v = keep_values ? C.vv[j] : 0.f;
    C.sup_j[s] = j;
    C.sup_v[s] = v;
    C.sup_slot[s] = -1;
  }
  if (threadIdx.x == 0) *C.nloc = K;
  csync();
  for (int s = threadIdx.x; s < K; s += kNT) C.sl[C.sup_j[s]] = C.sup_v[s];
  csync();
}

// G = W^T W and G^{-1} into C.Gi.  The Gram is summed in FP64 (exact FP64
// products of the FP32 entries; lane partials in row order, then a
// butterfly: a fixed order).  Dependent FP64 operations cost hundreds of
// cycles on this part, so the inverse starts from a Cholesky in FP32 and is
// refined by one Newton-Schulz step X <- X (2I - G X) in FP64 against the
// FP64 Gram: the FP32 inverse has a relative error of about cond(G) 1e-7 and
// the step squares it.  A pivot FP32 cannot take (G close to singular) falls
// back to the FP64 Cholesky of factor_gram.
template <int R>
__device__ __forceinline__ void gram_factor(Ctx& C) {
  const int r = C.r, lane = threadIdx.x & 31;
  for (int t = threadIdx.x >> 5; t < r * r; t += kNW) {
    const int p = t / r, q2 = t - p * r;
    if (q2 > p) continue;
    // FP64 sums of the exact FP64 products of the FP32 entries of W
    double s = 0.0;
    for (int i = lane; i < C.m; i += 32)
      s = dfma(static_cast<double>(C.W[i * R + p]), static_cast<double>(C.W[i * R + q2]), s);
    s = warp_sum(s);
    if (lane == 0) {
      C.G[p * kMaxR + q2] = s;
      C.G[q2 * kMaxR + p] = s;
    }
  }
  if (threadIdx.x == 0) C.flags[0] = 0;
  csync();
  if (threadIdx.x < 32) {
    float* Lf = reinterpret_cast<float*>(C.Lc);  // L (FP32), then L^{-1} after it
    float* Lif = Lf + kMaxR * kMaxR;
    float* iLf = reinterpret_cast<float*>(C.fv + 32);
    int ok = 1;
    if (lane == 0) {
      for (int j = 0; j < r && ok; ++j) {
        const float gjj = static_cast<float>(C.G[j * kMaxR + j]);
        float sj = gjj;
        for (int p = 0; p < j; ++p) sj = fmaf(-Lf[j * kMaxR + p], Lf[j * kMaxR + p], sj);
        if (!(sj > 1e-5f * gjj) || !(sj < 1e30f)) { ok = 0; break; }
        const float ij = rsqrtf(sj);
        Lf[j * kMaxR + j] = sj * ij;
        iLf[j] = ij;
        for (int i = j + 1; i < r; ++i) {
          float t = static_cast<float>(C.G[i * kMaxR + j]);
          for (int p = 0; p < j; ++p) t = fmaf(-Lf[i * kMaxR + p], Lf[j * kMaxR + p], t);
          Lf[i * kMaxR + j] = t * ij;
        }
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    if (!ok) {
      factor_gram(C);  // FP64 path (also reports a pivot that is not positive)
    } else {
      if (lane < r) {  // L^{-1}, one column per lane
        const int cc = lane;
        for (int i = 0; i < r; ++i) {
          float t = (i == cc) ? 1.f : 0.f;
          for (int p = cc; p < i; ++p) t = fmaf(-Lf[i * kMaxR + p], Lif[p * kMaxR + cc], t);
          Lif[i * kMaxR + cc] = (i < cc) ? 0.f : t * iLf[i];
        }
      }
      __syncwarp();
      for (int t = lane; t < r * r; t += 32) {  // X0 = L^{-T} L^{-1} into Gi
        const int a = t / r, b = t - a * r;
        float x = 0.f;
        for (int p = (a > b ? a : b); p < r; ++p) x = fmaf(Lif[p * kMaxR + a], Lif[p * kMaxR + b], x);
        C.Gi[a * kMaxR + b] = x;
      }
      __syncwarp();
      double* T = C.Lc;  // T = G X0 (FP64); the FP32 factors are no longer needed
      for (int t = lane; t < r * r; t += 32) {
        const int a = t / r, b = t - a * r;
        double x = 0.0;
        for (int p = 0; p < r; ++p) x = dfma(C.G[a * kMaxR + p], C.Gi[p * kMaxR + b], x);
        T[a * kMaxR + b] = x;
      }
      __syncwarp();
      for (int t = lane; t < r * r; t += 32) {  // X1 = 2 X0 - X0 T into G
        const int a = t / r, b = t - a * r;
        double x = 2.0 * C.Gi[a * kMaxR + b];
        for (int p = 0; p < r; ++p) x = dfma(-C.Gi[a * kMaxR + p], T[p * kMaxR + b], x);
        C.G[a * kMaxR + b] = x;
      }
      __syncwarp();
      for (int t = lane; t < r * r; t += 32) {
        const int a = t / r, b = t - a * r;
        C.Gi[a * kMaxR + b] = C.G[a * kMaxR + b];
      }
    }
  }
  csync();
}

// sum of squares of an m-vector in FP32 (warp butterflies, then the warps in
// index order), returned to every consumer thread
__device__ __forceinline__ float norm2_mf(const Ctx& C, const float* v) {
  float acc = 0.f;
  for (int i = threadIdx.x; i < C.m; i += kNT) acc = fmaf(v[i], v[i], acc);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) C.redf[kNW * kMaxR + 16 + (threadIdx.x >> 5)] = acc;
  csync();
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kNW; ++i) s += C.redf[kNW * kMaxR + 16 + i];
  csync();
  return s;
}

// u = P_perp(A s - y) (project) into dv and out.  A s is gathered, or already
// in dv (as_ready); it is kept in As for the column's next step.
template <int R, int ET>
__device__ __forceinline__ void residual_u(Ctx& C, const TaskProblem& P, int k, bool project,
                                           float* out, bool as_ready = false) {
  if (!as_ready) gather<ET>(C, C.sup_v, C.dv);
  csync();
  float* As = P.As + static_cast<size_t>(k) * P.astride;
  for (int i = threadIdx.x; i < C.m; i += kNT) {
    As[i] = C.dv[i];
    C.dv[i] -= C.yv[i];
  }
  csync();
  if (project) proj<R>(C, C.dv);
  for (int i = threadIdx.x; i < C.m; i += kNT) out[i] = C.dv[i];
}

// final stage before the last pass: A s, b = G^{-1} W^T (y - A s), e
template <int R, int ET>
__device__ __forceinline__ void final_prep(Ctx& C, const TaskProblem& P, int k, float* out,
                                           bool as_ready = false) {
  const int m = C.m, tid = threadIdx.x;
  if (!as_ready) gather<ET>(C, C.sup_v, C.dv);
  csync();
  for (int i = tid; i < m; i += kNT) C.dv[i] = C.yv[i] - C.dv[i];  // y - A s
  csync();
  if (P.mode == kModeInit) {
    for (int i = tid; i < m; i += kNT) out[i] = C.dv[i];
    return;
  }
  ls_solve<R>(C, C.dv);
  if (tid < C.r) P.B[static_cast<size_t>(k) * C.r + tid] = static_cast<float>(C.fv[16 + tid]);
  if (P.mode == kModeIter) {
    const float* xf = C.redf + kNW * kMaxR;
    for (int i = tid; i < m; i += kNT) {  // W b + A s - y
      float s = -C.dv[i];
#pragma unroll
      for (int l = 0; l < R; ++l) s = fmaf(C.W[i * R + l], xf[l], s);
      out[i] = s;
    }
  }
}

// S_k ascending by index
__device__ __forceinline__ void store_output_support(const Ctx& C, const TaskProblem& P, int k) {
  const int nl = *C.nloc, rho = C.rho;
  for (int e = threadIdx.x; e < nl; e += kNT) {
    const int je = C.sup_j[e];
    int pos = 0;
    for (int f = 0; f < nl; ++f) pos += C.sup_j[f] < je;
    P.S_idx[static_cast<size_t>(k) * rho + pos] = je;
    P.S_val[static_cast<size_t>(k) * rho + pos] = C.sup_v[e];
  }
}

// The small step after pass `ph` of column k completed (all consumer threads).
// Thread 0 publishes what follows.
template <int R, int ET>
__device__ void column_step(const TaskQueue& Q, int prob, int k, int ph, int type,
                            unsigned char* smem, const TCarve& cv, uint64_t* sbar,
                            unsigned& sphase) {
  const TaskProblem& P = Q.probs[prob];
  long long* sprof = reinterpret_cast<long long*>(smem + cv.prof);
  long long tlast = clock64();
  auto mark = [&](int slot) {  // IHT step sub-phases (profile)
    if (Q.prof && threadIdx.x == 0) {
      const long long t = clock64();
      sprof[slot] += t - tlast;
      tlast = t;
    }
  };
  const int tid = threadIdx.x, m = P.L.m;
  const bool project = P.mode != kModeInit;
  const int te = P.tau_eff, lastph = last_phase(P);
  // what follows is known now: admit the next column (the column is done) or
  // the next pass's tasks, whose tickets thread 0 reserves at once so that the
  // atomic's round trip overlaps the step
  const bool admit = type == kTaskF || (type == kTaskW && P.mode == kModeLS) || ph >= lastph;
  const int n_next = admit ? 0 : phase_tasks(P, ph + 1);
  int t_res = -1;
  if (tid == 0 && n_next > 0) t_res = atomicAdd(&Q.ctr[1], n_next);
  Ctx C;
  small_ctx(C, P, k, smem, cv);
  if (ET >= 2) {
    float* scw = reinterpret_cast<float*>(smem + cv.rsc);
    const int per = ET == 3 ? 2 : 1;
    for (int i = tid; i < m; i += kNT) {
      scw[i] = P.rscale[(static_cast<size_t>(k) * m + i) * per];
      scw[m + i] = ET == 3 ? P.rscale[(static_cast<size_t>(k) * m + i) * per + 1] : 0.f;
    }
  }
  float* uout = P.uvec + static_cast<size_t>(k) * m;
  int next_type = -1;  // what to publish after this step

  if (type == kTaskW) {
    // W_k = sum of the column-chunk partials (fixed order), Gram, Cholesky
    load_column<R>(C, P, k, false, false, kSupInput, false, sbar, sphase, Q.ctr + 3, Q.wait_ns);
    for (int t = tid; t < m * R; t += kNT) {
      float s = 0.f;
      for (int cc = 0; cc < P.ncw; ++cc)
        s += __ldcg(P.Wp + (static_cast<size_t>(k) * P.ncw + cc) * P.wstride + t);
      C.W[t] = s;
      P.Wk[static_cast<size_t>(k) * P.wstride + t] = s;
    }
    csync();
    gram_factor<R>(C);
    for (int t = tid; t < kMaxR * kMaxR; t += kNT)
      P.Gi[static_cast<size_t>(k) * kMaxR * kMaxR + t] = C.Gi[t];
    if (tid == 0) P.stop[k] = 0;
    if (P.mode == kModeLS) {
      final_prep<R, ET>(C, P, k, uout);
      next_type = -2;  // column done
    } else if (te > 0) {
      residual_u<R, ET>(C, P, k, true, uout);
      store_support(C, P, k);
      next_type = kTaskG;
    } else {
      final_prep<R, ET>(C, P, k, uout);
      store_support(C, P, k);
      next_type = kTaskF;
    }
  } else if (type == kTaskG || type == kTaskNop) {
    const bool zero_start = (P.mode == kModeInit && ph == 0);
    const int stop_in = zero_start ? 0 : __ldcg(P.stop + k);
    // A s of the current support, kept by the column's previous step: when
    // HardThreshold keeps the support, the new values are s - mu g on it and
    // A s_new = A s - mu A g_G, so the residual needs no gather
    const bool may_update = !zero_start && type == kTaskG;
    float* asv = reinterpret_cast<float*>(smem + cv.asv);
    int* osup = reinterpret_cast<int*>(smem + cv.osup);
    load_column<R>(C, P, k, project, project, zero_start ? kSupNone : kSupState,
                   type != kTaskNop, sbar, sphase, Q.ctr + 3, Q.wait_ns, may_update ? asv : nullptr);
    if (zero_start && tid == 0) P.stop[k] = 0;
    const int sweep = P.mode == kModeInit ? ph : ph - 1;  // 0-based IHT sweep just run
    bool stopped = stop_in != 0 || type == kTaskNop;
    bool as_ready = false;  // A s of the new support values in dv
    mark(10);
    if (!stopped) {
      if (zero_start) {
        for (int j = tid; j < P.L.n; j += kNT) C.vv[j] = C.gs[j];
        csync();
        ht_single(C, false);  // support G of the zero start
      }
      // mu = ||g_G||^2 / ||P_perp A g_G||^2 on the current support G
      const int nl = *C.nloc;
      for (int e = tid; e < nl; e += kNT) {
        C.vv[e] = C.gs[C.sup_j[e]];
        osup[e] = C.sup_j[e];
      }
      if (tid == 0) osup[C.rho + 1] = 1;  // "support kept", cleared below if not
      csync();
      // ||g_G||^2 by warp 0 (FP32, fixed order), shared through redf
      float* numf = C.redf + kNW * kMaxR + 32;
      if (tid < 32) {
        float t = 0.f;
        for (int e = tid; e < nl; e += 32) t = fmaf(C.vv[e], C.vv[e], t);
        t = warp_sum(t);
        if (tid == 0) *numf = t;
      }
      gather<ET>(C, C.vv, C.ev);
      csync();
      const float num = *numf;
      if (may_update)  // A g_G before the projection
        for (int i = tid; i < C.m; i += kNT) C.dv[i] = C.ev[i];
      if (project) proj<R>(C, C.ev);
      const float den = norm2_mf(C, C.ev);
      mark(11);
      if (!(den > 0.f)) {
        stopped = true;
        if (tid == 0) P.stop[k] = 1;
      } else {
        float muf = num / den;
        if (!isfinite(muf)) {
          if (tid == 0) report_error(P.err, kErrNaN, k);
          muf = 0.f;
        }
        for (int j = tid; j < P.L.n; j += kNT) C.vv[j] = fmaf(-muf, C.gs[j], C.sl[j]);
        csync();
        ht_single(C, true);
        store_support(C, P, k);
        if (may_update) {
          const int K = *C.nloc;
          for (int e = tid; e < K; e += kNT) {
            const int j = C.sup_j[e];
            bool found = false;
            for (int f = 0; f < nl; ++f) found |= osup[f] == j;
            if (!found) osup[C.rho + 1] = 0;
          }
          csync();
          if (K == nl && osup[C.rho + 1]) {
            for (int i = tid; i < C.m; i += kNT) C.dv[i] = fmaf(-muf, C.dv[i], asv[i]);
            as_ready = true;
          }
        }
      }
    }
    mark(12);
    if (sweep + 1 < te) {
      if (!stopped) residual_u<R, ET>(C, P, k, project, uout, as_ready);
      next_type = stopped ? kTaskNop : kTaskG;
    } else {
      final_prep<R, ET>(C, P, k, uout, as_ready);
      next_type = kTaskF;
    }
    mark(13);
  } else {  // kTaskF: H row written by the tasks; outputs
    load_column<R>(C, P, k, false, false, kSupState, false, sbar, sphase, Q.ctr + 3, Q.wait_ns);
    store_output_support(C, P, k);
    next_type = -2;
  }
  // publish: the barrier orders every write of this step before thread 0's
  // fence (cumulative), which comes before the flags of the next tasks
  csync();
  if (tid == 0) {
    P.cnt[k] = 0;
    if (admit) {
      __threadfence();
      admit_next(Q);
    } else {
      const int nph = ph + 1;
      const int nt = next_type == kTaskNop ? kTaskNop : phase_type(P, nph);
      publish_reserved(Q, t_res, k, prob, nt, nph, n_next);
    }
  }
  csync();
  if (type == kTaskG) mark(14);
}

// ---- the kernel --------------------------------------------------------------------
template <int R, int ET>
__global__ void __launch_bounds__(kThreadsAll, R <= 6 ? 3 : 2) task_kernel(const TaskQueue Q, int stages,
                                                             int piece_bytes, int m_max,
                                                             int ns_max, int rho_max) {
  extern __shared__ __align__(16) unsigned char smem[];
  stages = kTaskStages;  // the ring protocol relies on one stage per consumer warp
  const TCarve cv = tcarve(R, m_max, ns_max, rho_max, stages, piece_bytes);
  const int tid = threadIdx.x;
  TCtx T;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + cv.bars);
  T.full = bars;
  T.empty = bars + kMaxStages;
  T.tfull = bars + 2 * kMaxStages;
  T.tempty = bars + 2 * kMaxStages + 2;
  T.tslot = reinterpret_cast<unsigned long long*>(smem + cv.task);
  T.ring = smem + cv.ring;
  T.stage = cv.stage;
  T.stages = stages;
  T.seq = 0;
  T.uv = reinterpret_cast<float*>(smem + cv.uv);
  T.gpart = reinterpret_cast<float*>(smem + cv.gpart);
  T.rsc = reinterpret_cast<float*>(smem + cv.rsc);
  T.bcast = reinterpret_cast<int*>(smem + cv.bcast);
  T.err = Q.probs[0].err;
  T.abort = &Q.ctr[3];
  T.wait_ns = Q.wait_ns;
  T.pw = 0;
  long long* prof = reinterpret_cast<long long*>(smem + cv.prof);  // thread 0 / producer
  if (tid < kTaskProf) prof[tid] = 0;
  auto flush_prof = [&]() {
    if (!Q.prof) return;
    if (tid == 0) {
      prof[3] = T.pw;
      for (int i = 0; i < kTaskProf; ++i)
        if (i != 7 && prof[i]) atomicAdd(&Q.prof[i], static_cast<unsigned long long>(prof[i]));
    } else if (tid == kNT && prof[7]) {
      atomicAdd(&Q.prof[7], static_cast<unsigned long long>(prof[7]));
    }
  };
  if (tid == kNT) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&T.full[s], 1);
      mbar_init(&T.empty[s], kNW);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&T.tfull[s], 1);
      mbar_init(&T.tempty[s], kNW);
    }
    mbar_init(bars + 2 * kMaxStages + 4, 1);  // the steps' bulk copies
  }
  __syncthreads();

  if (tid >= kNT) {
    // ---------------- producer warp ----------------
    if (tid != kNT) return;
    unsigned pseq = 0;
    for (unsigned it = 0;; ++it) {
      const unsigned ts = it & 1u, use = it >> 1;
      const int h = atomicAdd(&Q.ctr[0], 1);
      unsigned long long d = tdesc(0, 0, kTaskExit, 0, 0);
      bool ok = true;
      const long long c0 = clock64();
      if (h < Q.total) {
        if (ld_acquire_(&Q.seq[h]) == 0) {
          const unsigned long long t0 = gtimer();
          while (ld_acquire_(&Q.seq[h]) == 0) {
            __nanosleep(200);
            if (ld_relaxed(T.abort)) { ok = false; break; }
            if (gtimer() - t0 > T.wait_ns) {
              set_abort(T.abort, T.err);
              ok = false;
              break;
            }
          }
        }
        if (ok) d = __ldcg(&Q.tasks[h]);
      }
      if (Q.prof) prof[7] += clock64() - c0;
      if (use > 0 && !wait_bar(&T.tempty[ts], (use - 1) & 1u, T.err, T.abort, T.wait_ns))
        d = tdesc(0, 0, kTaskExit, 0, 0);
      T.tslot[ts] = d;
      mbar_arrive_local(&T.tfull[ts]);
      const int type = td_type(d);
      if (type == kTaskExit || ld_relaxed(T.abort)) break;
      if (type != kTaskNop)
        produce_task<R, ET>(T, Q.probs[td_prob(d)], td_k(d), type, td_blk(d), pseq);
    }
    // no copy may still be landing in this CTA's shared memory when it leaves:
    // wait (bounded) for the last use of every stage
    for (int s = 0; s < stages; ++s) {
      if (pseq <= static_cast<unsigned>(s)) break;
      const unsigned last = (pseq - 1 - s) / stages * stages + s;  // last piece on stage s
      const unsigned long long t0 = gtimer();
      while (!mbar_try_wait(&T.full[s], (last / stages) & 1u))
        if (gtimer() - t0 > T.wait_ns) break;
    }
    flush_prof();
    return;
  }

  // ---------------- consumer warps ----------------
  uint64_t* sbar = bars + 2 * kMaxStages + 4;
  unsigned sphase = 0;
  for (unsigned it = 0;; ++it) {
    const unsigned ts = it & 1u, use = it >> 1;
    // one thread waits for the descriptor, so that leaving is uniform
    long long c0 = clock64();
    if (tid == 0) T.bcast[1] = wait_bar(&T.tfull[ts], use & 1u, T.err, T.abort, T.wait_ns) ? 1 : 0;
    csync();
    if (!T.bcast[1]) {
      flush_prof();
      return;
    }
    const unsigned long long d = T.tslot[ts];
    csync();
    if ((tid & 31) == 0) mbar_arrive_local(&T.tempty[ts]);
    const int type = td_type(d);
    if (type == kTaskExit) {
      flush_prof();
      return;
    }
    long long c1 = clock64();
    if (Q.prof && tid == 0) prof[0] += c1 - c0;
    const int prob = td_prob(d), k = td_k(d), ph = td_ph(d), blk = td_blk(d);
    const TaskProblem& P = Q.probs[prob];
    const int m = P.L.m;
    if (type != kTaskNop) {
      if (ET >= 2) {
        const int per = ET == 3 ? 2 : 1;
        for (int i = tid; i < m; i += kNT) {
          T.rsc[i] = P.rscale[(static_cast<size_t>(k) * m + i) * per];
          T.rsc[m + i] = ET == 3 ? P.rscale[(static_cast<size_t>(k) * m + i) * per + 1] : 0.f;
        }
      }
      if (type == kTaskW) {
        csync();
        if constexpr (R >= 8 && R <= 12)  // measured: faster for these widths only
          consume_w_rr<R, ET>(T, P, k, blk);
        else
          consume_w<R, ET>(T, P, k, blk);
      } else {
        // the vector of this pass: -y (zero start of INIT), y (INIT with no IHT), or
        // the one the previous step published
        const bool first_init = P.mode == kModeInit && ph == 0;
        for (int i = tid; i < m; i += kNT) {
          float v;
          if (first_init) {
            const float yi = P.y[static_cast<size_t>(k) * m + i];
            v = type == kTaskG ? -yi : yi;
          } else {
            v = __ldcg(P.uvec + static_cast<size_t>(k) * m + i);
          }
          T.uv[i] = v;
          if (ET >= 2) {  // this thread loaded the scales of row i above
            T.rsc[i] *= v;
            T.rsc[m + i] *= v;
          }
        }
        csync();
        float* out = type == kTaskF ? P.H + static_cast<size_t>(k) * P.L.n
                                    : P.g + static_cast<size_t>(k) * P.L.ns;
        consume_g<ET>(T, P, k, blk, out);
      }
    }
    c0 = clock64();
    if (Q.prof && tid == 0) {
      prof[type == kTaskW ? 1 : 2] += c0 - c1;
      prof[8] += 1;
    }
    // completion of the task; the last task of the pass runs the column step.
    // The barrier orders the CTA's writes of this task before thread 0's
    // fence (cumulative) and count; the last one's second fence orders the
    // other tasks' writes before the step reads them.
    csync();
    if (tid == 0) {
      __threadfence();
      const int done = atomicAdd(&P.cnt[k], 1) + 1;
      const int last = done == phase_tasks(P, ph) ? 1 : 0;
      if (last) __threadfence();
      *T.bcast = last;
    }
    csync();
    if (*T.bcast) {
      column_step<R, ET>(Q, prob, k, ph, type, smem, cv, sbar, sphase);
      c1 = clock64();
      if (Q.prof && tid == 0) {
        prof[type == kTaskW ? 4 : type == kTaskF ? 6 : 5] += c1 - c0;
        prof[9] += 1;
      }
    }
    csync();
  }
}

}  // namespace task
}  // namespace lrs
