// Register-resident cluster engine of the Gaussian sweep (Algorithm 1, the
// per-column lines "Compute z_k, M_k" .. the gradient term, with the IHT of
// Algorithm 2), one thread-block cluster of CS CTAs per column at a time.
//
// CTA c holds the columns [128c, 128c + 128) of A_k in registers: lane l of
// warp w keeps rows 32p + l (p < MR) of the 4-column chunks 8cc + w
// (cc < 4), 16 MR floats.  Every pass over A_k reads these registers:
//   W = A_k U            per-thread partial rows, summed over the warps in
//                        shared memory and over the CTAs through
//                        distributed shared memory (the one reduction over
//                        the cluster that every column needs);
//   g = A_k^T u          per-lane partial sums over the lane's rows, reduced
//                        over the 32 lanes of the warp (its columns are
//                        complete inside the warp: no exchange).
// Every CTA also keeps a copy of the rho columns of A_k on the current
// support G (gathered from their owners when the support changes, which
// after the first iterations is rare), so that g_G, A g_G, mu and A s need
// no exchange: they are computed from the copies, identically in every CTA.
// HardThreshold then needs one exchange per IHT sweep: a column can enter
// the support only if |v_j| reaches the smallest |v| on the current support
// (the current support already offers rho entries at least that large), so
// each CTA sends just those of its columns (usually none) and every CTA
// merges them with the current support by (|v| descending, index
// ascending).  The small steps (the Gram G_k = W^T W and its factor, the
// P_perp projections, mu, the LS step) run in every CTA on identical
// values, so every CTA takes identical decisions.
//
// Exchanges: each CTA writes its contribution into every CTA's buffer
// (st.shared::cluster), then thread 0 signals every CTA's mbarrier of that
// exchange's parity (release at cluster scope) and waits for its own
// (acquire), bounded by a time limit.  The candidate slots alternate by the
// exchange's parity: slot e & 1 is rewritten by exchange e + 2 only after
// every CTA has signalled exchange e + 1, which each does after it finished
// reading exchange e.  The W buffer and the gathered-column buffer are read
// right after their exchange, before the CTA signals the next one; an
// exchange that would refill one of them right after the exchange that
// filled it is preceded by an empty exchange.
//
// Memory traffic: A_k is read from memory once per sweep (a bulk L2
// prefetch of the next columns' slabs overlaps the current column's work);
// y_k, S_k and b_k are read and written once; h_k is written once.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lrs_dev.cuh"
#include "lrs_internal.h"

namespace lrs {
namespace res {

constexpr int NT = kResNT;
constexpr int NW = NT / 32;
constexpr int NCH = kResChunks / NW;   // chunks per thread (4)
constexpr int NS = kResCols;           // columns per CTA (128)
constexpr unsigned FULL = 0xffffffffu;
// thread coordinates, read from the special registers where used
#define TID (static_cast<int>(threadIdx.x))
#define LANE (static_cast<int>(threadIdx.x & 31))
#define WARP (static_cast<int>(threadIdx.x >> 5))

__host__ __device__ inline int up4(int x) { return (x + 3) & ~3; }
__host__ __device__ inline size_t up16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline int imax(int a, int b) { return a > b ? a : b; }

// Shared-memory layout (byte offsets), identical on host and device: the
// buffers whose sizes depend only on the compiled rank width R and rows per
// lane MR at fixed offsets, then those that depend on rho (padded to rp) and
// the cluster size CS.
__host__ __device__ constexpr unsigned a16u(unsigned x) { return (x + 15u) & ~15u; }

template <int R, int MR>
struct Lay {
  static constexpr unsigned mp = 32 * MR;          // rows padded to 32 MR
  static constexpr unsigned RU = (R + 3) & ~3;     // floats per staged U row
  static constexpr unsigned bars = 0;
  static constexpr unsigned Us = 16;
  static constexpr unsigned sd = Us + 4u * NS * RU;
  static constexpr unsigned gd = sd + 4u * NS;
  static constexpr unsigned vv = gd + 4u * NS;
  static constexpr unsigned spos = vv + 4u * NS;
  static constexpr unsigned cidx = spos + 4u * NS;
  static constexpr unsigned cval = cidx + 4u * NS;
  static constexpr unsigned Wm = cval + 4u * NS;
  static constexpr unsigned Gi32 = Wm + 4u * R * mp;
  static constexpr unsigned yv = Gi32 + a16u(4u * R * R);
  static constexpr unsigned As = yv + 4u * mp;
  static constexpr unsigned AgG = As + 4u * mp;
  static constexpr unsigned u = AgG + 4u * mp;
  static constexpr unsigned t1 = u + 4u * mp;
  static constexpr unsigned red = t1 + 4u * mp;
  static constexpr unsigned scal = red + 4u * NW * R * mp;
  static constexpr unsigned Lf = scal + 256u;
  static constexpr unsigned dG = Lf + a16u(4u * (10 * R * R + 4 * R));
  static constexpr unsigned pacc = dG + a16u(8u * (4 * R * R + 2 * R + 2));
  static constexpr unsigned dyn = pacc + 256u;    // start of the rp / CS dependent part
};
__host__ __device__ inline int rho_pad(int rho) { return up4(rho > 0 ? rho : 1); }
__host__ __device__ inline int xslot_floats(int rp) { return up4(4 + 3 * rp); }
// rp / CS dependent part, in order: AG[2] (rp x mp each), AGin (rp x mp),
// wx (CS x R x mp), xs (2 x CS x XS), wgG (NW x rp), 9 arrays of rp
// (sup_i, sup_v, gG, vG, nsup_i, nsup_v, opos, rk_i, rk_v), midx, mval
// ((CS + 1) rp each), mkey ((CS + 1) rp u64), keys (max(NS, CS rp) u64).
template <int R, int MR>
__host__ __device__ inline unsigned dyn_bytes(int rp, int CS) {
  using L = Lay<R, MR>;
  const unsigned rpmp = 4u * rp * L::mp;
  const unsigned nm = static_cast<unsigned>((CS + 1) * rp);
  const unsigned nk = static_cast<unsigned>(imax(NS, CS * rp));
  return 3 * rpmp + a16u(4u * CS * R * L::mp) + a16u(8u * CS * xslot_floats(rp)) +
         a16u(4u * NW * rp) + 9 * a16u(4u * rp) + 2 * a16u(4u * nm) + a16u(8u * nm) + a16u(8u * nk);
}
template <int R, int MR>
__host__ __device__ inline size_t smem_total(int rho, int CS) {
  return Lay<R, MR>::dyn + dyn_bytes<R, MR>(rho_pad(rho), CS);
}

// scalar slots in scal[]
enum : int { kSFlag = 2, kSSame = 3, kSB = 8, kSWcnt = 16 };
// profile phases (the counters of kResProf) and the timestamp slot
enum : int {
  kPLoad = 0, kPW, kPWait, kPGram, kPProj, kPAgG, kPMu, kPHT, kPMerge, kPAs, kPFinal,
  kPCols, kPEx, kPChg, kPSweeps, kPStamp = 31
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned mapa_u32(unsigned local, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_f32(unsigned addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote_u32(unsigned local_bar, unsigned rank) {
  const unsigned remote = mapa_u32(local_bar, rank);
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_acq_cluster(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ float comp(const float4& v, int e) {
  return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}
// key of a HardThreshold candidate: larger |v| first, then the lower index
__device__ __forceinline__ unsigned long long ht_key(float absv, int j) {
  return (static_cast<unsigned long long>(__float_as_uint(absv)) << 32) |
         static_cast<unsigned long long>(~static_cast<unsigned>(j));
}
// double-float arithmetic (a sum carried as an unevaluated pair hi + lo of
// floats; Knuth's error-free sum): the Gram's sums in about twice float
// precision with single-precision units
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
  float s, e;
  two_sum(hi, bh, s, e);
  e += lo + bl;
  hi = s + e;
  lo = e - (hi - s);
}

template <int R, int MR>
struct Ctx {
  using L = Lay<R, MR>;
  int n, m, r, rho, CS, c, nchc, j0, m_last, nv, k;
  int ex;          // exchanges done by this CTA
  int ex_agin;     // last exchange that carried gathered columns (AGin)
  int ex_wx;       // last exchange that carried W partials (wx)
  int broken;      // a wait expired: the CTA stops
  int profon;
  int agsel;       // which of the two AG buffers holds the current support's columns
  int rp, XS;
  unsigned smem0;  // shared address of the carve base
  unsigned long long wait_ns;
  unsigned char* base;
  int* err;
  static constexpr int mp = L::mp;
  __device__ float* F(unsigned off) const { return reinterpret_cast<float*>(base + off); }
  __device__ int* I(unsigned off) const { return reinterpret_cast<int*>(base + off); }
  __device__ unsigned long long* U64(unsigned off) const {
    return reinterpret_cast<unsigned long long*>(base + off);
  }
  // fixed buffers
  __device__ float* Us() const { return F(L::Us); }
  __device__ float* sd() const { return F(L::sd); }
  __device__ float* gd() const { return F(L::gd); }
  __device__ float* vv() const { return F(L::vv); }
  __device__ int* spos() const { return I(L::spos); }
  __device__ int* cidx() const { return I(L::cidx); }
  __device__ float* cval() const { return F(L::cval); }
  __device__ float* Wm() const { return F(L::Wm); }
  __device__ float* Gi32() const { return F(L::Gi32); }
  __device__ float* yv() const { return F(L::yv); }
  __device__ float* As() const { return F(L::As); }
  __device__ float* AgG() const { return F(L::AgG); }
  __device__ float* u() const { return F(L::u); }
  __device__ float* t1() const { return F(L::t1); }
  __device__ float* red() const { return F(L::red); }
  __device__ float* scal() const { return F(L::scal); }
  __device__ float* Lf() const { return F(L::Lf); }
  __device__ double* dG() const { return reinterpret_cast<double*>(base + L::dG); }
  __device__ unsigned long long* pacc() const { return U64(L::pacc); }
  // rp / CS dependent buffers
  __device__ unsigned rpmp() const { return 4u * rp * L::mp; }
  __device__ float* AG() const { return F(L::dyn + agsel * rpmp()); }
  __device__ float* AGn() const { return F(L::dyn + (1 - agsel) * rpmp()); }
  __device__ float* AGin() const { return F(L::dyn + 2 * rpmp()); }
  __device__ unsigned o_wx() const { return L::dyn + 3 * rpmp(); }
  __device__ float* wx() const { return F(o_wx()); }
  __device__ unsigned o_xs() const { return o_wx() + a16u(4u * CS * R * L::mp); }
  __device__ float* xs() const { return F(o_xs()); }
  __device__ unsigned o_wgG() const { return o_xs() + a16u(8u * CS * XS); }
  __device__ float* wgG() const { return F(o_wgG()); }
  __device__ unsigned o_arr(int q) const { return o_wgG() + a16u(4u * NW * rp) + q * a16u(4u * rp); }
  __device__ int* sup_i() const { return I(o_arr(0)); }
  __device__ float* sup_v() const { return F(o_arr(1)); }
  __device__ float* gG() const { return F(o_arr(2)); }
  __device__ float* vG() const { return F(o_arr(3)); }
  __device__ int* nsup_i() const { return I(o_arr(4)); }
  __device__ float* nsup_v() const { return F(o_arr(5)); }
  __device__ int* opos() const { return I(o_arr(6)); }
  __device__ int* rk_i() const { return I(o_arr(7)); }
  __device__ float* rk_v() const { return F(o_arr(8)); }
  __device__ unsigned nm() const { return static_cast<unsigned>((CS + 1) * rp); }
  __device__ int* midx() const { return I(o_arr(9)); }
  __device__ float* mval() const { return F(o_arr(9) + a16u(4u * nm())); }
  __device__ unsigned long long* mkey() const { return U64(o_arr(9) + 2 * a16u(4u * nm())); }
  __device__ unsigned long long* keys() const {
    return U64(o_arr(9) + 2 * a16u(4u * nm()) + a16u(8u * nm()));
  }
};

// Close profile phase ph (thread 0): the cycles since the previous mark.
template <int R, int MR>
__device__ __forceinline__ void pmark(const Ctx<R, MR>& C, int ph) {
  if (C.profon && TID == 0) {
    const unsigned long long t = clock64();
    C.pacc()[ph] += t - C.pacc()[kPStamp];
    C.pacc()[kPStamp] = t;
  }
}
template <int R, int MR>
__device__ __forceinline__ void pcount(const Ctx<R, MR>& C, int ph) {
  if (C.profon && TID == 0) C.pacc()[ph] += 1;
}

template <int R, int MR>
__device__ __forceinline__ unsigned saddr(const Ctx<R, MR>& C, const void* p) {
  return C.smem0 + static_cast<unsigned>(static_cast<const unsigned char*>(p) - C.base);
}

// Push v to float slot `p_local` (an address in this CTA's buffer) of every
// CTA of the cluster.
template <int R, int MR>
__device__ __forceinline__ void push_all(const Ctx<R, MR>& C, const float* p_local, float v) {
  const unsigned a = saddr(C, p_local);
  if (C.CS == 1) {
    *const_cast<float*>(p_local) = v;
    return;
  }
  for (int p = 0; p < C.CS; ++p) st_cluster_f32(mapa_u32(a, p), v);
}

// Finish an exchange: every thread's pushes are done; signal every CTA, wait
// for all of them.  On expiry of the wait the CTA records a timeout and stops.
// ph: the profile phase of the work before the exchange.
template <int R, int MR>
__device__ __forceinline__ void xchg(Ctx<R, MR>& C, int ph) {
  __syncthreads();
  pmark(C, ph);
  pcount(C, kPEx);
  if (C.CS > 1) {
    const int slot = C.ex & 1;
    const unsigned par = static_cast<unsigned>(C.ex >> 1) & 1u;
    const unsigned bar = C.smem0 + Lay<R, MR>::bars + 8u * slot;
    if (TID < C.CS) mbar_arrive_remote_u32(bar, TID);  // one signalling thread per CTA
    if (TID == 0) {
      const unsigned long long t0 = gtimer();
      int expired = 0;
      while (!mbar_try_wait_acq_cluster(bar, par)) {
        if (gtimer() - t0 > C.wait_ns) {
          expired = 1;
          break;
        }
      }
      if (expired) {
        report_error(C.err, kErrTimeout, C.k);
        C.scal()[kSFlag] = 1.f;
      }
    }
    __syncthreads();
    C.broken = C.scal()[kSFlag] != 0.f;
  }
  pmark(C, kPWait);
  ++C.ex;
}

// Before pushing into a buffer last filled by exchange `last`: the next
// exchange must come at least two after it (every CTA has then read it), so
// an empty exchange is inserted when it would be the very next one.
template <int R, int MR>
__device__ __forceinline__ void reuse_guard(Ctx<R, MR>& C, int last, int ph) {
  if (C.ex == last + 1) xchg(C, ph);
}

template <int R, int MR>
__device__ __forceinline__ float* xslot(const Ctx<R, MR>& C, int ex, int c) {
  return C.xs() + (static_cast<size_t>(ex & 1) * C.CS + c) * C.XS;
}

// ---- passes over the register-resident slab -------------------------------------
template <int R, int MR>
__device__ __forceinline__ void load_slab(const Ctx<R, MR>& C, const float* slab, float4 (&a)[MR][NCH]) {
#pragma unroll
  for (int cc = 0; cc < NCH; ++cc) {
    const int ch = cc * NW + WARP;
#pragma unroll
    for (int p = 0; p < MR; ++p) {
      const bool last = p == MR - 1;
      const int Lp = last ? C.m_last : 32;
      if (ch < C.nchc && LANE < Lp) {
        const size_t off = static_cast<size_t>(p) * 128 * C.nchc + static_cast<size_t>(ch) * 4 * Lp +
                           4 * LANE;
        a[p][cc] = __ldcs(reinterpret_cast<const float4*>(slab + off));
      } else {
        a[p][cc] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
}

// g = A^T u for the warp's 16 columns; returns the value of column index
// (lane >> 1) of the warp (both lanes of a pair hold it).
template <int R, int MR>
__device__ __forceinline__ float at_pass(const Ctx<R, MR>& C, const float4 (&a)[MR][NCH], const float* u) {
  float up[MR];
#pragma unroll
  for (int p = 0; p < MR; ++p) up[p] = u[LANE + 32 * p];
  float v[16];
#pragma unroll
  for (int cc = 0; cc < NCH; ++cc) {
    float x = 0.f, y = 0.f, z = 0.f, t = 0.f;
#pragma unroll
    for (int p = 0; p < MR; ++p) {
      x = fmaf(a[p][cc].x, up[p], x);
      y = fmaf(a[p][cc].y, up[p], y);
      z = fmaf(a[p][cc].z, up[p], z);
      t = fmaf(a[p][cc].w, up[p], t);
    }
    v[4 * cc] = x;
    v[4 * cc + 1] = y;
    v[4 * cc + 2] = z;
    v[4 * cc + 3] = t;
  }
  // reduce-scatter over the 32 lanes: after the steps over lane bits 4..1 a
  // lane holds the sum of index 8 b4 + 4 b3 + 2 b2 + b1 over 16 lanes; the
  // last step adds the pair
#pragma unroll
  for (int half = 8, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
    const bool hi = (LANE & bit) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = hi ? v[i] : v[i + half];
      const float keep = hi ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(FULL, send, bit);
    }
  }
  return v[0] + __shfl_xor_sync(FULL, v[0], 1);
}
// local column (0..127) of the value at_pass returns to this lane
template <int R, int MR>
__device__ __forceinline__ int at_col(const Ctx<R, MR>& C) {
  const int c16 = (LANE >> 1) & 15;
  return 4 * ((c16 >> 2) * NW + WARP) + (c16 & 3);
}

// at_pass with the pass vector u held per warp in registers (lane l holds
// rows l + 32p), as the register-resident steps below keep it.
template <int R, int MR>
__device__ __forceinline__ float at_pass_reg(const Ctx<R, MR>& C, const float4 (&a)[MR][NCH],
                                             const float (&up)[MR]) {
  float v[16];
#pragma unroll
  for (int cc = 0; cc < NCH; ++cc) {
    float x = 0.f, y = 0.f, z = 0.f, t = 0.f;
#pragma unroll
    for (int p = 0; p < MR; ++p) {
      x = fmaf(a[p][cc].x, up[p], x);
      y = fmaf(a[p][cc].y, up[p], y);
      z = fmaf(a[p][cc].z, up[p], z);
      t = fmaf(a[p][cc].w, up[p], t);
    }
    v[4 * cc] = x;
    v[4 * cc + 1] = y;
    v[4 * cc + 2] = z;
    v[4 * cc + 3] = t;
  }
#pragma unroll
  for (int half = 8, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
    const bool hi = (LANE & bit) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = hi ? v[i] : v[i + half];
      const float keep = hi ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(FULL, send, bit);
    }
  }
  return v[0] + __shfl_xor_sync(FULL, v[0], 1);
}

// Row vectors held per warp in registers (lane l: rows l + 32p).  Every warp
// forms the same m-space quantities itself, in the same order, so that the
// steps between two passes need no block barrier.
// c = W^T x (every lane receives all r sums; rows >= m of W and x are zero)
template <int R, int MR>
__device__ __forceinline__ void wt_rows(const Ctx<R, MR>& C, const float (&x)[MR], float (&c)[R]) {
#pragma unroll
  for (int l = 0; l < R; ++l) c[l] = 0.f;
#pragma unroll
  for (int p = 0; p < MR; ++p) {
    const int i = LANE + 32 * p;
#pragma unroll
    for (int l = 0; l < R; ++l) c[l] = fmaf(C.Wm()[l * C.mp + i], x[p], c[l]);
  }
#pragma unroll
  for (int l = 0; l < R; ++l) c[l] = warp_sum(c[l]);
}
// x <- x - W G^{-1} c  (with c = W^T x: x <- P_perp x)
template <int R, int MR>
__device__ __forceinline__ void sub_w(const Ctx<R, MR>& C, float (&x)[MR], const float (&c)[R]) {
  float z[R];
#pragma unroll
  for (int l = 0; l < R; ++l) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < R; ++j) s = fmaf(C.Gi32()[l * R + j], c[j], s);
    z[l] = s;
  }
#pragma unroll
  for (int p = 0; p < MR; ++p) {
    const int i = LANE + 32 * p;
#pragma unroll
    for (int l = 0; l < R; ++l) x[p] = fmaf(-C.Wm()[l * C.mp + i], z[l], x[p]);
  }
}
template <int MR>
__device__ __forceinline__ float norm2_reg(const float (&x)[MR]) {
  float s = 0.f;
#pragma unroll
  for (int p = 0; p < MR; ++p) s = fmaf(x[p], x[p], s);
  return warp_sum(s);
}

// Push local column jl of the register slab (rows of this warp's lanes) to
// row block `dst` (m floats, an address in this CTA's buffer) of every CTA.
// Called by the owning warp only: warp (jl / 4) mod 8.
template <int R, int MR>
__device__ __forceinline__ void push_column(const Ctx<R, MR>& C, const float4 (&a)[MR][NCH], int jl,
                                            const float* dst) {
  const int ch = jl >> 2, cc = ch / NW, e = jl & 3;
#pragma unroll
  for (int p = 0; p < MR; ++p) {
    const int i = LANE + 32 * p;
    float4 v = a[p][0];
#pragma unroll
    for (int q = 1; q < NCH; ++q)
      if (cc == q) v = a[p][q];
    if (i < C.m) push_all(C, dst + i, comp(v, e));
  }
}
// Every CTA pushes the columns it owns among the support positions e (only
// those with keep[e] < 0 when keep is given: the entering ones) into AGin[e]
// of every CTA.
template <int R, int MR>
__device__ __forceinline__ void push_support_columns(const Ctx<R, MR>& C, const float4 (&a)[MR][NCH],
                                                     const int* idx, const int* keep) {
  for (int e = 0; e < C.rho; ++e) {
    if (keep && keep[e] >= 0) continue;
    const int jl = idx[e] - C.j0;
    if (jl < 0 || jl >= NS) continue;
    if (((jl >> 2) % NW) != WARP) continue;
    push_column(C, a, jl, C.AGin() + static_cast<size_t>(e) * C.mp);
  }
}

// W = A U (U staged in Us: row j = U(j0 + j, :)): per-thread partial rows,
// summed over the warps, pushed to slot c of every CTA's W buffer; the
// support columns this CTA owns go to every CTA's AGin in the same exchange.
// After it: W (Wm), the support columns (AG) and A s formed from them.
template <int R, int MR>
__device__ __forceinline__ void w_pass(Ctx<R, MR>& C, const float4 (&a)[MR][NCH]) {
  constexpr int RU = (R + 3) & ~3;
  reuse_guard(C, C.ex_wx, kPW);
  reuse_guard(C, C.ex_agin, kPW);
  // rows in two groups (p < PH, then p >= PH): fewer accumulators live at once
  constexpr int PH = (MR + 1) / 2;
#pragma unroll
  for (int g0 = 0; g0 < MR; g0 += PH) {
    float acc[PH][R];
#pragma unroll
    for (int p = 0; p < PH; ++p)
#pragma unroll
      for (int l = 0; l < R; ++l) acc[p][l] = 0.f;
#pragma unroll
    for (int cc = 0; cc < NCH; ++cc) {
      const int jb = 4 * (cc * NW + WARP);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float* ur = C.Us() + (jb + e) * RU;
        float uv[RU];
#pragma unroll
        for (int q4 = 0; q4 < RU; q4 += 4) {
          const float4 t = *reinterpret_cast<const float4*>(ur + q4);
          uv[q4] = t.x;
          uv[q4 + 1] = t.y;
          uv[q4 + 2] = t.z;
          uv[q4 + 3] = t.w;
        }
#pragma unroll
        for (int p = 0; p < PH; ++p) {
          if (g0 + p >= MR) continue;
          const float av = comp(a[g0 + p][cc], e);
#pragma unroll
          for (int l = 0; l < R; ++l) acc[p][l] = fmaf(av, uv[l], acc[p][l]);
        }
      }
    }
#pragma unroll
    for (int p = 0; p < PH; ++p) {
      if (g0 + p >= MR) continue;
#pragma unroll
      for (int l = 0; l < R; ++l)
        C.red()[(WARP * R + l) * C.mp + LANE + 32 * (g0 + p)] = acc[p][l];
    }
  }
  push_support_columns(C, a, C.sup_i(), nullptr);
  __syncthreads();
  for (int l = 0; l < R; ++l) {
    float* dst = C.wx() + (static_cast<size_t>(C.c) * R + l) * C.mp;
    for (int i = TID; i < C.m; i += NT) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < NW; ++w) s += C.red()[(w * R + l) * C.mp + i];
      push_all(C, dst + i, s);
    }
  }
  C.ex_wx = C.ex;
  C.ex_agin = C.ex;
  xchg(C, kPW);
  for (int l = 0; l < R; ++l) {
    for (int i = TID; i < C.mp; i += NT) {
      float s = 0.f;
      if (i < C.m)
        for (int c = 0; c < C.CS; ++c) s += C.wx()[(static_cast<size_t>(c) * R + l) * C.mp + i];
      C.Wm()[l * C.mp + i] = s;
    }
  }
  // the support columns, and A s = sum_e A_{j_e} s_e from them (support order)
  for (int i = TID; i < C.mp; i += NT) {
    float s = 0.f;
    for (int e = 0; e < C.rho; ++e) {
      const float v = i < C.m ? C.AGin()[e * C.mp + i] : 0.f;
      C.AG()[e * C.mp + i] = v;
      s = fmaf(v, C.sup_v()[e], s);
    }
    C.As()[i] = s;
  }
  __syncthreads();
}

// Entry e of an r x r matrix held one per lane in two slots (entries e and
// e + 32): the value of entry `src` (fetched by every lane of the warp).
__device__ __forceinline__ float fetch2(float s0, float s1, int src) {
  const float a = __shfl_sync(FULL, s0, src & 31);
  const float b = __shfl_sync(FULL, s1, src & 31);
  return src < 32 ? a : b;
}

// G = W^T W and G^{-1}.  G's entries are summed in double-float arithmetic
// (error-free products and sums of the FP32 entries of W: about 2^-48
// relative, the accuracy of an FP64 sum).  Warp 0 then holds G one entry per
// lane (entries e and e + 32 of the row-major r x r matrix) and inverts it
// in registers: Gauss-Jordan elimination in FP32 (G is symmetric positive
// definite, so the diagonal pivots need no exchanges; a pivot FP32 cannot
// take sends the column to an FP64 Cholesky instead), then one Newton-Schulz
// step X1 = X0 (2I - G X0) in double-float arithmetic against the
// double-float G, which squares X0's relative error (about cond(G) 1e-7).
// Dependent FP64 operations take several hundred cycles on this part, and
// this chain sits between two passes of every column; double-float gives the
// accuracy with single-precision units.  A pivot FP64 cannot take is
// reported as a Gram that is not positive definite.  The inverse is kept as
// a double-float pair (Xh, Xl) for the LS solve and as its FP32 rounding Gi32
// for the projections.
template <int R, int MR>
__device__ __forceinline__ void gram_factor(Ctx<R, MR>& C) {
  const int r = C.r;
  float* Gh = C.Lf();
  float* Gl = C.Lf() + R * R;
  float* Xh = C.Lf() + 7 * R * R;
  float* Xl = C.Lf() + 8 * R * R;
  const int npairs = r * (r + 1) / 2;
  for (int pr = WARP; pr < npairs; pr += NW) {
    int a = 0, rem = pr;
    while (rem >= r - a) {
      rem -= r - a;
      ++a;
    }
    const int b = a + rem;
    float hi = 0.f, lo = 0.f;
    for (int i = LANE; i < C.m; i += 32) {
      const float x = C.Wm()[a * C.mp + i], y = C.Wm()[b * C.mp + i];
      const float p = x * y;
      const float pe = fmaf(x, y, -p);
      df_add(hi, lo, p, pe);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(FULL, hi, o), ol = __shfl_xor_sync(FULL, lo, o);
      df_add(hi, lo, oh, ol);
    }
    if (LANE == 0) {
      Gh[a * r + b] = hi;
      Gh[b * r + a] = hi;
      Gl[a * r + b] = lo;
      Gl[b * r + a] = lo;
    }
  }
  __syncthreads();
  if (WARP == 0) {
    const int rr = r * r;
    const int e0 = LANE, e1 = LANE + 32;
    const int a0 = e0 / r, b0 = e0 - a0 * r, a1 = e1 / r, b1 = e1 - a1 * r;
    const float gh0 = e0 < rr ? Gh[e0] : 0.f, gl0 = e0 < rr ? Gl[e0] : 0.f;
    const float gh1 = e1 < rr ? Gh[e1] : 0.f, gl1 = e1 < rr ? Gl[e1] : 0.f;
    // Gauss-Jordan inverse in place (FP32)
    float x0 = gh0, x1 = gh1;
    int ok = 1;
    for (int k = 0; k < r; ++k) {
      const float pkk = fetch2(x0, x1, k * r + k);
      const float dkk = fetch2(gh0, gh1, k * r + k);
      if (!(pkk > 1e-6f * dkk) || !(pkk < 1e30f)) {
        ok = 0;
        break;
      }
      const float ip = 1.f / pkk;
      const float aik0 = fetch2(x0, x1, a0 * r + k), akj0 = fetch2(x0, x1, k * r + b0);
      const float aik1 = fetch2(x0, x1, (a1 < r ? a1 : 0) * r + k);
      const float akj1 = fetch2(x0, x1, k * r + b1);
      float n0, n1;
      if (a0 == k && b0 == k) n0 = ip;
      else if (a0 == k) n0 = x0 * ip;
      else if (b0 == k) n0 = -x0 * ip;
      else n0 = fmaf(-aik0 * ip, akj0, x0);
      if (a1 == k && b1 == k) n1 = ip;
      else if (a1 == k) n1 = x1 * ip;
      else if (b1 == k) n1 = -x1 * ip;
      else n1 = fmaf(-aik1 * ip, akj1, x1);
      x0 = e0 < rr ? n0 : 0.f;
      x1 = e1 < rr ? n1 : 0.f;
    }
    float xh0, xl0, xh1, xl1;
    if (ok) {
      // T = G X0 (double-float), one entry per lane
      float th0 = 0.f, tl0 = 0.f, th1 = 0.f, tl1 = 0.f;
      for (int p = 0; p < r; ++p) {
        const float ga0 = fetch2(gh0, gh1, a0 * r + p), gb0 = fetch2(gl0, gl1, a0 * r + p);
        const float xp0 = fetch2(x0, x1, p * r + b0);
        const float ga1 = fetch2(gh0, gh1, (a1 < r ? a1 : 0) * r + p);
        const float gb1 = fetch2(gl0, gl1, (a1 < r ? a1 : 0) * r + p);
        const float xp1 = fetch2(x0, x1, p * r + b1);
        float ph = ga0 * xp0, pe = fmaf(ga0, xp0, -ph) + gb0 * xp0;
        df_add(th0, tl0, ph, pe);
        ph = ga1 * xp1;
        pe = fmaf(ga1, xp1, -ph) + gb1 * xp1;
        df_add(th1, tl1, ph, pe);
      }
      // X1 = 2 X0 - X0 T (double-float)
      xh0 = 2.f * x0;
      xl0 = 0.f;
      xh1 = 2.f * x1;
      xl1 = 0.f;
      for (int p = 0; p < r; ++p) {
        const float xa0 = fetch2(x0, x1, a0 * r + p), xa1 = fetch2(x0, x1, (a1 < r ? a1 : 0) * r + p);
        const float tph0 = fetch2(th0, th1, p * r + b0), tpl0 = fetch2(tl0, tl1, p * r + b0);
        const float tph1 = fetch2(th0, th1, p * r + b1), tpl1 = fetch2(tl0, tl1, p * r + b1);
        float ph = xa0 * tph0, pe = fmaf(xa0, tph0, -ph) + xa0 * tpl0;
        df_add(xh0, xl0, -ph, -pe);
        ph = xa1 * tph1;
        pe = fmaf(xa1, tph1, -ph) + xa1 * tpl1;
        df_add(xh1, xl1, -ph, -pe);
      }
    } else {
      // FP64 Cholesky of the double-float G (slow, rare: near-singular Grams)
      double* G = C.dG();
      double* Ld = C.dG() + R * R;
      double* Lid = C.dG() + 2 * R * R;
      double* iLd = C.dG() + 3 * R * R;
      if (e0 < rr) G[a0 * R + b0] = static_cast<double>(gh0) + static_cast<double>(gl0);
      if (e1 < rr) G[a1 * R + b1] = static_cast<double>(gh1) + static_cast<double>(gl1);
      __syncwarp();
      const bool ok64 = chol_inverse_warp(G, Ld, Lid, iLd, r, R);
      double v0 = 0.0, v1 = 0.0;
      if (e0 < rr)
        for (int p = (a0 > b0 ? a0 : b0); p < r; ++p) v0 = __fma_rn(Lid[p * R + a0], Lid[p * R + b0], v0);
      if (e1 < rr)
        for (int p = (a1 > b1 ? a1 : b1); p < r; ++p) v1 = __fma_rn(Lid[p * R + a1], Lid[p * R + b1], v1);
      xh0 = static_cast<float>(v0);
      xl0 = static_cast<float>(v0 - static_cast<double>(xh0));
      xh1 = static_cast<float>(v1);
      xl1 = static_cast<float>(v1 - static_cast<double>(xh1));
      if (!ok64 && LANE == 0) report_error(C.err, kErrNotSPD, C.k);
    }
    if (e0 < rr) {
      Xh[a0 * R + b0] = xh0;
      Xl[a0 * R + b0] = xl0;
    }
    if (e1 < rr) {
      Xh[a1 * R + b1] = xh1;
      Xl[a1 * R + b1] = xl1;
    }
#pragma unroll
    for (int q = 0; q < (R * R + 31) / 32; ++q) {  // FP32 copy, zero beyond r
      const int e = LANE + 32 * q;
      const int a = e / R, b = e - a * R;
      const bool in = e < R * R && a < r && b < r;
      const int src = in ? a * r + b : 0;
      const float v = fetch2(xh0, xh1, src);   // every lane takes part in the shuffles
      if (e < R * R) C.Gi32()[e] = in ? v : 0.f;
    }
  }
  __syncthreads();
}

// b = G^{-1} c with the double-float inverse (every lane receives all r
// values; the products and sums in double-float, the result rounded).
template <int R, int MR>
__device__ __forceinline__ void ls_solve(const Ctx<R, MR>& C, const float (&c)[R], float (&b)[R]) {
  const float* Xh = C.Lf() + 7 * R * R;
  const float* Xl = C.Lf() + 8 * R * R;
#pragma unroll
  for (int l = 0; l < R; ++l) {
    float bh = 0.f, bl = 0.f;
    if (l < C.r) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        if (j >= C.r) continue;
        const float ph = Xh[l * R + j] * c[j];
        const float pe = fmaf(Xh[l * R + j], c[j], -ph) + Xl[l * R + j] * c[j];
        df_add(bh, bl, ph, pe);
      }
    }
    b[l] = bh + bl;
  }
}

// out = P_perp v = v - W G^{-1} W^T v (every warp forms W^T v itself, in the
// same order, then writes its share of the rows).  v and out distinct; the
// caller synchronises before (v complete) and after (out complete).
template <int R, int MR>
__device__ __forceinline__ void project(const Ctx<R, MR>& C, const float* v, float* out) {
  float cl[R];
#pragma unroll
  for (int l = 0; l < R; ++l) cl[l] = 0.f;
  for (int i = LANE; i < C.m; i += 32) {
    const float vi = v[i];
#pragma unroll
    for (int l = 0; l < R; ++l) cl[l] = fmaf(C.Wm()[l * C.mp + i], vi, cl[l]);
  }
#pragma unroll
  for (int l = 0; l < R; ++l) cl[l] = warp_sum(cl[l]);
  float x[R];
#pragma unroll
  for (int l = 0; l < R; ++l) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < R; ++j) s = fmaf(C.Gi32()[l * R + j], cl[j], s);
    x[l] = s;
  }
  for (int i = WARP * 32 + LANE; i < C.mp; i += NT) {
    float t = v[i];
#pragma unroll
    for (int l = 0; l < R; ++l) t = fmaf(-C.Wm()[l * C.mp + i], x[l], t);
    out[i] = i < C.m ? t : 0.f;
  }
}

// ||v||^2 over the m rows, formed by every warp in the same order.
template <int R, int MR>
__device__ __forceinline__ float norm2_rows(const Ctx<R, MR>& C, const float* v) {
  float s = 0.f;
  for (int i = LANE; i < C.m; i += 32) s = fmaf(v[i], v[i], s);
  return warp_sum(s);
}

// The rho largest |vals_j| over the whole column (the first IHT sweep of the
// initialisation, from s = 0, where the step's support is the rho largest
// |g_i|): each CTA's rho best go to slot c of the exchange; every CTA merges
// the CS x rho candidates and writes the kept indices, ascending, to nsup_i
// (values zero).
template <int R, int MR>
__device__ __forceinline__ void top_rho_full(Ctx<R, MR>& C, const float* vals) {
  const int rho = C.rho;
  if (TID < NS) {
    const int j = TID;
    C.keys()[j] = j < C.nv ? ht_key(fabsf(vals[j]), C.j0 + j) : 0ull;
  }
  __syncthreads();
  float* my = xslot(C, C.ex, C.c);
  if (TID < NS) {
    const int j = TID;
    const unsigned long long kj = C.keys()[j];
    if (kj != 0ull) {
      int rank = 0;
      for (int u = 0; u < NS; u += 2) {
        const ulonglong2 k2 = *reinterpret_cast<const ulonglong2*>(C.keys() + u);
        rank += (k2.x > kj) + (k2.y > kj);
      }
      if (rank < rho) {
        push_all(C, my + 4 + 3 * rank, fabsf(vals[j]));
        push_all(C, my + 4 + 3 * rank + 1, __int_as_float(C.j0 + j));
        push_all(C, my + 4 + 3 * rank + 2, vals[j]);
      }
    }
  }
  // slots of a slab with fewer than rho valid columns: marked empty
  for (int t = C.nv + TID; t < rho; t += NT) push_all(C, my + 4 + 3 * t + 1, __int_as_float(-1));
  const int e = C.ex;
  xchg(C, kPHT);
  const int ncand = C.CS * rho;
  for (int t = TID; t < ncand; t += NT) {
    const float* s = xslot(C, e, t / rho) + 4 + 3 * (t % rho);
    const int j = __float_as_int(s[1]);
    C.keys()[t] = j >= 0 ? ht_key(s[0], j) : 0ull;
  }
  __syncthreads();
  for (int t = TID; t < ncand; t += NT) {
    const unsigned long long kt = C.keys()[t];
    if (kt == 0ull) continue;
    int rank = 0;
    for (int u = 0; u < ncand; ++u) rank += C.keys()[u] > kt;
    if (rank < rho) C.rk_i()[rank] = static_cast<int>(~static_cast<unsigned>(kt & 0xffffffffull));
  }
  __syncthreads();
  if (TID < rho) {
    const int j = C.rk_i()[TID];
    int pos = 0;
    for (int u = 0; u < rho; ++u) pos += C.rk_i()[u] < j;
    C.nsup_i()[pos] = j;
    C.nsup_v()[pos] = 0.f;
  }
  __syncthreads();
}

// HardThreshold(v, rho) of an IHT sweep with a current support G whose
// values vG are known to every CTA.  Any index outside G that enters the new
// support has |v_j| >= min_G |vG| (G itself offers rho entries at least that
// large); the caller has listed this CTA's such columns per warp (cidx/cval
// at 16 w + q, counts in scal[kSWcnt + w]).  Each CTA sends them (all when
// at most rho, else its rho best); every CTA merges them with G.  Writes the
// new support, ascending, to nsup_i / nsup_v and scal[kSSame].
template <int R, int MR>
__device__ __forceinline__ void hard_threshold_sweep(Ctx<R, MR>& C) {
  const int rho = C.rho;
  const int* wcnt = reinterpret_cast<const int*>(C.scal()) + kSWcnt;
  int tot = 0;
  for (int w = 0; w < NW; ++w) tot += wcnt[w];
  // compact the per-warp lists in warp order (gd and vv, NS entries each, are
  // free during the merge: the indices go to gd as int bits, the values to vv)
  int* cj = reinterpret_cast<int*>(C.gd());
  float* cvl = C.vv();
  if (tot > 0) {
    for (int t = TID; t < NW * 16; t += NT) {
      const int w = t >> 4, q = t & 15;
      if (q < wcnt[w]) {
        int off = 0;
        for (int w2 = 0; w2 < w; ++w2) off += wcnt[w2];
        cj[off + q] = C.cidx()[t];
        cvl[off + q] = C.cval()[t];
      }
    }
    __syncthreads();
  }
  float* my = xslot(C, C.ex, C.c);
  const int nsend = tot < rho ? tot : rho;
  for (int q = TID; q < tot; q += NT) {
    int slot = q;
    if (tot > rho) {  // keep this CTA's rho best
      const unsigned long long kq = ht_key(fabsf(cvl[q]), cj[q]);
      int rank = 0;
      for (int u = 0; u < tot; ++u) rank += ht_key(fabsf(cvl[u]), cj[u]) > kq;
      slot = rank < rho ? rank : -1;
    }
    if (slot >= 0) {
      push_all(C, my + 4 + 3 * slot, fabsf(cvl[q]));
      push_all(C, my + 4 + 3 * slot + 1, __int_as_float(cj[q]));
      push_all(C, my + 4 + 3 * slot + 2, cvl[q]);
    }
  }
  if (TID == 0) push_all(C, my, __int_as_float(nsend));
  const int ex = C.ex;
  xchg(C, kPHT);
  // merge: the current support and every CTA's candidates
  int ntot = 0;
  for (int c = 0; c < C.CS; ++c) ntot += __float_as_int(xslot(C, ex, c)[0]);
  if (ntot == 0) {  // nothing reaches the support: it is kept with the new values
    if (TID < rho) {
      C.nsup_i()[TID] = C.sup_i()[TID];
      C.nsup_v()[TID] = C.vG()[TID];
    }
    if (TID == 0) C.scal()[kSSame] = 1.f;
    __syncthreads();
    return;
  }
  const int L = rho + ntot;
  for (int t = TID; t < L; t += NT) {
    int j;
    float v;
    if (t < rho) {
      j = C.sup_i()[t];
      v = C.vG()[t];
    } else {
      int q = t - rho, c = 0;
      while (q >= __float_as_int(xslot(C, ex, c)[0])) {
        q -= __float_as_int(xslot(C, ex, c)[0]);
        ++c;
      }
      const float* s = xslot(C, ex, c) + 4 + 3 * q;
      j = __float_as_int(s[1]);
      v = s[2];
    }
    C.midx()[t] = j;
    C.mval()[t] = v;
    C.mkey()[t] = ht_key(fabsf(v), j);
  }
  __syncthreads();
  for (int t = TID; t < L; t += NT) {
    const unsigned long long kt = C.mkey()[t];
    int rank = 0;
    for (int u = 0; u < L; ++u) rank += C.mkey()[u] > kt;
    if (rank < rho) {
      C.rk_i()[rank] = C.midx()[t];
      C.rk_v()[rank] = C.mval()[t];
    }
  }
  __syncthreads();
  if (TID < rho) {
    const int j = C.rk_i()[TID];
    int pos = 0;
    for (int u = 0; u < rho; ++u) pos += C.rk_i()[u] < j;
    C.nsup_i()[pos] = j;
    C.nsup_v()[pos] = C.rk_v()[TID];
  }
  __syncthreads();
  if (TID == 0) {
    int same = 1;
    for (int e = 0; e < rho; ++e) same &= C.nsup_i()[e] == C.sup_i()[e];
    C.scal()[kSSame] = same ? 1.f : 0.f;
  }
  __syncthreads();
}

// Make (nsup_i, nsup_v) the current support: the columns entering it are
// gathered from their owners (one exchange), the copies are re-ordered to
// the new support, the slab vectors follow, and A s is formed from the
// copies.
template <int R, int MR>
__device__ __forceinline__ void adopt_support(Ctx<R, MR>& C, const float4 (&a)[MR][NCH]) {
  const int rho = C.rho;
  if (TID < rho) {  // old positions of the new indices (-1: entering)
    const int j = C.nsup_i()[TID];
    int op = -1;
    for (int e = 0; e < rho; ++e)
      if (C.sup_i()[e] == j) op = e;
    C.opos()[TID] = op;
    const int jl = C.sup_i()[TID] - C.j0;  // the old entries leave the slab vectors
    if (jl >= 0 && jl < NS) {
      C.sd()[jl] = 0.f;
      C.spos()[jl] = -1;
    }
  }
  __syncthreads();
  reuse_guard(C, C.ex_agin, kPAs);
  push_support_columns(C, a, C.nsup_i(), C.opos());
  C.ex_agin = C.ex;
  xchg(C, kPAs);
  for (int t = TID; t < rho * C.mp; t += NT) {
    const int e = t / C.mp, i = t - e * C.mp;
    const int op = C.opos()[e];
    C.AGn()[t] = op >= 0 ? C.AG()[op * C.mp + i] : (i < C.m ? C.AGin()[t] : 0.f);
  }
  __syncthreads();
  C.agsel ^= 1;
  if (TID < rho) {
    const int jg = C.nsup_i()[TID];
    const float v = C.nsup_v()[TID];
    C.sup_i()[TID] = jg;
    C.sup_v()[TID] = v;
    const int jl = jg - C.j0;
    if (jl >= 0 && jl < NS) {
      C.sd()[jl] = v;
      C.spos()[jl] = TID;
    }
  }
  __syncthreads();
  for (int i = TID; i < C.mp; i += NT) {
    float s = 0.f;
    for (int e = 0; e < rho; ++e) s = fmaf(C.AG()[e * C.mp + i], C.sup_v()[e], s);
    C.As()[i] = s;
  }
  __syncthreads();
}

// ---- the kernel ----------------------------------------------------------------
// Two CTAs per SM while the slab and the W accumulators fit 128 registers
// a thread (rows per lane <= 5); one otherwise.
template <int MR>
struct MinBlocks {
  static constexpr int value = MR <= 5 ? 2 : 1;
};

template <int R, int MR>
__global__ void __launch_bounds__(NT, MinBlocks<MR>::value) resident_kernel(ResArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  Ctx<R, MR> C;
  C.n = a.n;
  C.m = a.m;
  C.r = a.r;
  C.rho = a.rho;
  C.CS = a.CS;
  C.c = C.CS > 1 ? static_cast<int>(cluster_rank()) : 0;
  C.ex = 0;
  C.ex_agin = -2;
  C.ex_wx = -2;
  C.broken = 0;
  C.k = -1;
  C.err = a.err;
  C.wait_ns = a.wait_ns;
  C.base = smem;
  C.smem0 = smem_u32(smem);
  C.rp = rho_pad(a.rho);
  C.XS = xslot_floats(C.rp);
  C.agsel = 0;
  C.profon = a.prof != nullptr;
  if (TID < 32) C.pacc()[TID] = 0ull;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lay<R, MR>::bars);

  const int CS = C.CS;
  const int cl = blockIdx.x / CS, ncl = gridDim.x / CS;
  C.j0 = kResCols * C.c;
  C.nchc = min(kResChunks, a.nch4 - kResChunks * C.c);
  C.m_last = C.m - 32 * (MR - 1);
  C.nv = max(0, min(NS, C.n - C.j0));
  const int mode = a.mode;
  const int sweeps = (mode == kModeLS || C.rho == 0) ? 0 : a.tau;
  const size_t col_floats = static_cast<size_t>(C.m) * 4 * a.nch4;
  const size_t slab_off = static_cast<size_t>(128) * C.m * C.c;
  const unsigned slab_bytes = static_cast<unsigned>(16u * C.m * (C.nchc > 0 ? C.nchc : 0));

  if (TID == 0) {
    mbar_init(&bars[0], CS);
    mbar_init(&bars[1], CS);
  }
  if (TID < 64) C.scal()[TID] = 0.f;
  if (mode != kModeInit) {  // U rows of this slab (zero beyond n and beyond r)
    for (int e = TID; e < NS * Ctx<R, MR>::L::RU; e += NT) {
      const int j = e / Ctx<R, MR>::L::RU, l = e - j * Ctx<R, MR>::L::RU;
      const int jg = C.j0 + j;
      C.Us()[e] = (l < C.r && jg < C.n) ? a.U[static_cast<size_t>(jg) * C.r + l] : 0.f;
    }
  }
  for (int j = TID; j < NS; j += NT) {
    C.sd()[j] = 0.f;
    C.spos()[j] = -1;
  }
  if (CS > 1) cluster_sync_all();  // barriers initialised before any remote arrive
  else __syncthreads();
  if (C.profon && TID == 0) C.pacc()[kPStamp] = clock64();
  if (TID == 0 && cl < a.q && slab_bytes)  // first column's slab
    prefetch_l2(a.A + static_cast<size_t>(cl) * col_floats + slab_off, slab_bytes);

  float4 A4[MR][NCH];
  for (int k = cl; k < a.q && !C.broken; k += ncl) {
    C.k = k;
    load_slab(C, a.A + static_cast<size_t>(k) * col_floats + slab_off, A4);
    if (TID == 0 && slab_bytes) {
      if (k + ncl < a.q)
        prefetch_l2(a.A + static_cast<size_t>(k + ncl) * col_floats + slab_off, slab_bytes);
      if (k + 2 * ncl < a.q)
        prefetch_l2(a.A + static_cast<size_t>(k + 2 * ncl) * col_floats + slab_off, slab_bytes);
    }
    // measurements and current support (ascending)
    const float* yk = a.y + static_cast<size_t>(k) * C.m;
    for (int i = TID; i < C.mp; i += NT) {
      C.yv()[i] = i < C.m ? yk[i] : 0.f;
      if (mode == kModeInit) C.As()[i] = 0.f;
    }
    if (TID < C.rho) {
      int jg = -1;
      float v = 0.f;
      if (mode != kModeInit) {
        jg = a.S_idx[static_cast<size_t>(k) * C.rho + TID];
        v = a.S_val[static_cast<size_t>(k) * C.rho + TID];
        if (jg < 0 || jg >= C.n) jg = 0;  // guard against a corrupt state
      }
      C.sup_i()[TID] = jg;
      C.sup_v()[TID] = v;
      const int jl = jg - C.j0;
      if (jg >= 0 && jl >= 0 && jl < NS) {
        C.sd()[jl] = v;
        C.spos()[jl] = TID;
      }
    }
    __syncthreads();
    pcount(C, kPCols);
    pmark(C, kPLoad);

    bool have_support = mode != kModeInit;
    if (mode != kModeInit) {
      w_pass(C, A4);  // W, the support columns and A s
      pmark(C, kPW);
      if (C.broken) break;
      gram_factor(C);
      pmark(C, kPGram);
    }

    // ---- IHT (Algorithm 2) ----
    for (int it = 0; it < sweeps && !C.broken; ++it) {
      // u = P_perp (A s - y), every warp in registers (P_perp = I in the
      // initialisation)
      float uu[MR];
#pragma unroll
      for (int p = 0; p < MR; ++p) uu[p] = C.As()[LANE + 32 * p] - C.yv()[LANE + 32 * p];
      if (mode == kModeIter) {
        float cw[R];
        wt_rows(C, uu, cw);
        sub_w(C, uu, cw);
      }
      const float g = at_pass_reg(C, A4, uu);
      const int jl = at_col(C);
      pcount(C, kPSweeps);
      pmark(C, kPProj);
      if (!have_support) {
        // s = 0: the step's support is the rho largest |g_i|; gather its columns
        if ((LANE & 1) == 0) C.gd()[jl] = g;
        __syncthreads();
        top_rho_full(C, C.gd());
        if (C.broken) break;
        adopt_support(C, A4);  // no old entries (sup_i = -1): every column gathered
        if (C.broken) break;
        have_support = true;
        pmark(C, kPMerge);
      }
      // g on the support from the copies (every warp forms all rho values, in
      // the same order in every CTA), then A g_G, ||g_G||^2, ||M g_G||^2, mu
      float* wg = C.gG();
      for (int e = WARP; e < C.rho; e += NW) {
        float d = 0.f;
#pragma unroll
        for (int p = 0; p < MR; ++p) d = fmaf(C.AG()[e * C.mp + LANE + 32 * p], uu[p], d);
        d = warp_sum(d);
        if (LANE == 0) wg[e] = d;
      }
      __syncthreads();
      float ag[MR];
#pragma unroll
      for (int p = 0; p < MR; ++p) ag[p] = 0.f;
      float num = 0.f;
      for (int e = 0; e < C.rho; ++e) {
        const float ge = wg[e];
        num = fmaf(ge, ge, num);
#pragma unroll
        for (int p = 0; p < MR; ++p) ag[p] = fmaf(C.AG()[e * C.mp + LANE + 32 * p], ge, ag[p]);
      }
      if (WARP == 0) {  // A g_G for the update of A s
#pragma unroll
        for (int p = 0; p < MR; ++p) C.AgG()[LANE + 32 * p] = ag[p];
      }
      if (mode == kModeIter) {  // ag <- P_perp A g_G
        float cw[R];
        wt_rows(C, ag, cw);
        sub_w(C, ag, cw);
      }
      const float den = norm2_reg<MR>(ag);
      pmark(C, kPAgG);
      if (!(den > 0.f)) {  // ||M g_G|| = 0: the column's IHT stops (every CTA alike)
        if (mode == kModeInit && it == 0) {
          // no step from s = 0: the support reported is 0 .. rho-1 with zero values
          __syncthreads();
          if (TID < C.rho) {
            const int j2 = C.sup_i()[TID] - C.j0;
            if (j2 >= 0 && j2 < NS) C.spos()[j2] = -1;
          }
          __syncthreads();
          if (TID < C.rho) {
            C.sup_i()[TID] = TID;
            C.sup_v()[TID] = 0.f;
          }
        }
        __syncthreads();
        break;
      }
      const float mu = num / den;
      // v on this warp's columns (support entries from the copies); an index
      // off the support can enter only if |v_j| >= tau = min_G |v|
      float tau = 3.0e38f;
      for (int e = 0; e < C.rho; ++e) tau = fminf(tau, fabsf(C.sup_v()[e] - mu * wg[e]));
      const int e_own = C.spos()[jl];
      const float v = e_own >= 0 ? C.sup_v()[e_own] - mu * wg[e_own] : C.sd()[jl] - mu * g;
      const bool cand = ((LANE & 1) == 0) && jl < C.nv && e_own < 0 && fabsf(v) >= tau;
      const unsigned bal = __ballot_sync(FULL, cand);
      if (cand) {
        const int q = __popc(bal & ((1u << LANE) - 1u));
        C.cidx()[WARP * 16 + q] = C.j0 + jl;
        C.cval()[WARP * 16 + q] = v;
      }
      if (LANE == 0) reinterpret_cast<int*>(C.scal())[kSWcnt + WARP] = __popc(bal);
      if (WARP == 0 && LANE < C.rho) C.vG()[LANE] = C.sup_v()[LANE] - mu * wg[LANE];
      __syncthreads();
      pmark(C, kPMu);
      hard_threshold_sweep(C);
      if (C.broken) break;
      pmark(C, kPMerge);
      if (C.scal()[kSSame] != 0.f) {
        // kept support: s_new = v on it, A s_new = A s - mu A g_G
        if (TID < C.rho) {
          const float vn = C.nsup_v()[TID];
          C.sup_v()[TID] = vn;
          const int j2 = C.sup_i()[TID] - C.j0;
          if (j2 >= 0 && j2 < NS) C.sd()[j2] = vn;
        }
        for (int i = TID; i < C.mp; i += NT) C.As()[i] = fmaf(-mu, C.AgG()[i], C.As()[i]);
        __syncthreads();
      } else {
        pcount(C, kPChg);
        adopt_support(C, A4);
        if (C.broken) break;
      }
      pmark(C, kPAs);
    }
    if (C.broken) break;

    if (mode == kModeInit) {
      // L0 column: A^T (y - A s)
      float uu[MR];
#pragma unroll
      for (int p = 0; p < MR; ++p) uu[p] = C.yv()[LANE + 32 * p] - C.As()[LANE + 32 * p];
      const float h = at_pass_reg(C, A4, uu);
      const int j = at_col(C);
      if ((LANE & 1) == 0 && j < C.nv) a.H[static_cast<size_t>(k) * C.n + C.j0 + j] = h;
    } else {
      // LS: b = G^{-1} W^T (y - A s), every warp alike
      float t[MR];
#pragma unroll
      for (int p = 0; p < MR; ++p) t[p] = C.yv()[LANE + 32 * p] - C.As()[LANE + 32 * p];
      float cw[R], b[R];
      wt_rows(C, t, cw);
      ls_solve(C, cw, b);
      if (TID == 0) {
        bool bad = false;
#pragma unroll
        for (int l = 0; l < R; ++l) bad |= l < C.r && !(fabsf(b[l]) < 3.0e38f);
        if (bad) report_error(C.err, kErrNaN, k);
      }
      if (mode == kModeIter) {
        // h_k = A^T (W b + A s - y)
#pragma unroll
        for (int p = 0; p < MR; ++p) {
          const int i = LANE + 32 * p;
          float x = -t[p];
#pragma unroll
          for (int l = 0; l < R; ++l) x = fmaf(C.Wm()[l * C.mp + i], b[l], x);
          t[p] = x;
        }
        const float h = at_pass_reg(C, A4, t);
        const int j = at_col(C);
        if ((LANE & 1) == 0 && j < C.nv) a.H[static_cast<size_t>(k) * C.n + C.j0 + j] = h;
      }
      if (C.c == 0 && WARP == 0) {
#pragma unroll
        for (int l = 0; l < R; ++l)
          if (LANE == l && l < C.r) a.B[static_cast<size_t>(k) * C.r + l] = b[l];
      }
    }
    if (mode != kModeLS && C.c == 0 && TID < C.rho) {
      a.S_idx[static_cast<size_t>(k) * C.rho + TID] = C.sup_i()[TID];
      a.S_val[static_cast<size_t>(k) * C.rho + TID] = C.sup_v()[TID];
    }
    // clear this column's support from the slab vectors
    __syncthreads();
    if (TID < C.rho) {
      const int jl = C.sup_i()[TID] - C.j0;
      if (jl >= 0 && jl < NS) {
        C.sd()[jl] = 0.f;
        C.spos()[jl] = -1;
      }
    }
    __syncthreads();
    pmark(C, kPFinal);
  }
  if (C.profon && TID == 0)
    for (int i = 0; i < kResProf; ++i) atomicAdd(a.prof + i, C.pacc()[i]);
  // no CTA leaves while a peer may still write into its shared memory
  if (CS > 1) cluster_sync_all();
}

#undef TID
#undef LANE
#undef WARP
}  // namespace res
}  // namespace lrs
