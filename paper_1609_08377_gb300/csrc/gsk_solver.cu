// Batched shifted B-Lanczos solver of libgsk (device kernels + orchestration).
//
// Method (Sec. III-A/III-B of the paper: generalized shifted equations
// (z B - A) x = e_j solved with one Krylov subspace for all shifts). With
// H = B^{-1} A, self-adjoint in <x, y>_B = x^T B y, the equations become
// (z I - H) x = B^{-1} e_j. A Lanczos process on H started from B^{-1} e_j
// keeps q_n and B q_n:
//   seed:   u = e_j, v = B^{-1} u, beta_0 = sqrt(u.v), q_1 = v/beta_0, Bq_1 = u/beta_0
//   step n: w = A q_n, alpha_n = q_n.w, u = w - alpha_n Bq_n - beta_{n-1} Bq_{n-1},
//           v = B^{-1} u (inner CG), beta_n = sqrt(u.v), q_{n+1} = v/beta_n,
//           Bq_{n+1} = u/beta_n.
// For every shift sigma_k the solution x_n = Q_n (sigma_k - T_n)^{-1} beta_0 e_1
// is updated by the LDL^T ("direct Lanczos") recurrence of sigma_k I - T_n:
//   d_1 = sigma - alpha_1, g_1 = beta_0;  l_{n-1} = -beta_{n-1}/d_{n-1},
//   d_n = sigma - alpha_n + l_{n-1} beta_{n-1}, g_n = -l_{n-1} g_{n-1},
//   zeta_n = g_n/d_n, p_n = q_n - l_{n-1} p_{n-1}, x_n = x_{n-1} + zeta_n p_n,
// restricted to the rows of A's pattern in column j (Sec. II-B). The
// residual of shift k after step n is |zeta_n| * ||u_n||_2 because
// e_j - (sigma B - A) x_n = zeta_n u_n. Im sigma != 0 keeps every d_n away
// from zero (Im d_n >= Im sigma), so the recurrence cannot break down.
//
// Columns are independent (Eq. TRACE-X-DECOMP); W of them run as lanes of one
// batch in lock step, and a lane whose column finishes takes the next job
// from a device work queue at the end of the step.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <string>
#include <type_traits>
#include <vector>

#include "gsk_common.cuh"
#include "gsk_ctx.h"
#include "gsk_df64.cuh"

namespace gsk {

// ===========================================================================
// Bounds-checked build (-DGSK_DEBUG)
// ===========================================================================
// The solve's kernels test the block-layout, tile and work-queue indices
// before they use them. A failed test records the first offence -- a code
// naming the check (include/gsk.h lists them) and the offending index -- in
// g_dbg, and the access is skipped or sent to a valid row, so the kernel ends
// normally and gsk_solve / gsk_spmm return GSK_EBOUNDS. No check traps. In the
// normal build every check is the constant true and compiles away.
#ifdef GSK_DEBUG
__device__ int g_dbg[4];       // first code, index (low, high word), failed checks
__device__ __noinline__ void dbg_fail(int code, long long idx) {
  if (atomicCAS(&g_dbg[0], 0, code) == 0) {
    g_dbg[1] = (int)(idx & 0xffffffffLL);
    g_dbg[2] = (int)(idx >> 32);
  }
  atomicAdd(&g_dbg[3], 1);
}
#define GSK_IDX_OK(cond, code, idx) ((cond) ? true : (::gsk::dbg_fail((code), (long long)(idx)), false))
#else
#define GSK_IDX_OK(cond, code, idx) true
#endif

// ===========================================================================
// Finalisation of per-lane sums (runs in the last CTA of a reducing kernel)
// ===========================================================================
__device__ void finalize_lane(const RedArgs& r, int l, double s) {
  const LaneCtl& c = r.c;
  switch (r.fin) {
    case FIN_ALPHA:
      c.alpha[l] = s;
      break;
    case FIN_UNORM: {
      const int st = c.state[l];
      c.unorm[l] = sqrt(s);
      c.rr[l] = s;
      c.rr_target[l] = r.inner_tol2 * s;
      c.cg_a[l] = 0.0;
      c.cg_b[l] = 0.0;
      c.cg_on[l] = (st != LS_IDLE && !c.brk[l] && s > 0.0 && isfinite(s)) ? 1 : 0;
      break;
    }
    case FIN_CG_A:
      if (c.cg_on[l]) {
        if (s > 0.0 && isfinite(s)) {
          c.cg_a[l] = c.rr[l] / s;
        } else {            // p.Bp <= 0: B is not positive definite for this lane
          c.cg_a[l] = 0.0;
          c.cg_on[l] = 0;
          c.brk[l] = 1;
        }
      } else {
        c.cg_a[l] = 0.0;
      }
      break;
    case FIN_CG_RR:
      if (c.cg_on[l]) {
        if (!isfinite(s)) {
          c.cg_b[l] = 0.0;
          c.cg_on[l] = 0;
          c.brk[l] = 1;
        } else {
          c.cg_b[l] = s / c.rr[l];
          c.rr[l] = s;
          if (s <= c.rr_target[l]) c.cg_on[l] = 0;
        }
      } else {
        c.cg_b[l] = 0.0;
      }
      break;
    case FIN_RESID: {
      const int st = c.state[l];
      c.rr[l] = s;
      c.rr_target[l] = r.inner_tol2 * s;
      c.cg_a[l] = 0.0;
      c.cg_b[l] = 0.0;
      c.cg_on[l] = (st != LS_IDLE && !c.done[l] && !c.brk[l] && s > 0.0 && isfinite(s)) ? 1 : 0;
      break;
    }
    case FIN_BETA: {
      const int st = c.state[l];
      if (st == LS_ACTIVE) {
        if (c.done[l]) {
          c.inv_beta[l] = 0.0;
        } else if (!c.brk[l] && s > 0.0 && isfinite(s)) {
          const double b = sqrt(s);
          c.beta_prev[l] = b;
          c.inv_beta[l] = 1.0 / b;
          c.n[l] += 1;
        } else {
          c.brk[l] = 1;
          c.inv_beta[l] = 0.0;
          c.n[l] += 1;
        }
      } else if (st == LS_SEED) {
        c.state[l] = LS_ACTIVE;
        c.n[l] = 0;
        c.beta_prev[l] = 0.0;
        if (!c.brk[l] && s > 0.0 && isfinite(s)) {
          const double b0 = sqrt(s);
          c.beta0[l] = b0;
          c.inv_beta[l] = 1.0 / b0;
        } else {
          c.brk[l] = 1;
          c.inv_beta[l] = 0.0;
        }
      } else {
        c.inv_beta[l] = 0.0;
      }
      break;
    }
    case FIN_SUM:
    default:
      c.red_out[l] = s;
      break;
  }
}

__device__ __forceinline__ void set_cond(const GraphCtl& gc, cudaGraphConditionalHandle h, int v) {
  if (gc.use_graph) cudaGraphSetConditional(h, v ? 1u : 0u);
}

// Solve-wide bookkeeping after the per-lane finalisation (thread 0 of the last
// CTA). The CG kernels of the refinement pass carry max_iter == -1 in their
// RedArgs, which selects the conditional handle of the second inner loop.
__device__ void finalize_all(const RedArgs& r) {
  const LaneCtl& c = r.c;
  const int W = r.W;
  switch (r.fin) {
    case FIN_UNORM: {
      *c.cg_iter = 0;
      int any = 0;
      for (int l = 0; l < W; ++l) any += c.cg_on[l];
      *c.unfinished = any;
      set_cond(r.gc, r.gc.h_inner1, any > 0);
      break;
    }
    case FIN_RESID: {
      *c.cg_iter = 0;
      int any = 0;
      for (int l = 0; l < W; ++l) any += c.cg_on[l];
      *c.unfinished = any;
      set_cond(r.gc, r.gc.h_inner2, any > 0);
      break;
    }
    case FIN_CG_RR: {
      const int it = ++(*c.cg_iter);
      ++(*c.cg_total);
      int any = 0;
      for (int l = 0; l < W; ++l) any += c.cg_on[l];
      if (any > 0 && it >= r.gc.max_inner) {       // inner solve failed to converge
        for (int l = 0; l < W; ++l)
          if (c.cg_on[l]) {
            c.cg_on[l] = 0;
            c.brk[l] = 1;
          }
        any = 0;
      }
      *c.unfinished = any;
      set_cond(r.gc, r.max_iter == -1 ? r.gc.h_inner2 : r.gc.h_inner1, any > 0);
      break;
    }
    case FIN_BETA: {
      const int step = ++(*c.step);
      int qh = *c.queue_head;
      int busy = 0;
      for (int l = 0; l < W; ++l) {
        const int st = c.state[l];
        if ((st == LS_ACTIVE && c.done[l]) || st == LS_IDLE) {
          if (qh < r.jobs.n_jobs) {
            c.job[l] = r.jobs.queue[qh++];
            c.state[l] = LS_SEED;
#ifdef GSK_DEBUG
            if (!GSK_IDX_OK(c.job[l] >= 0 && c.job[l] < r.jobs.n_jobs, 20, qh - 1)) {
              c.job[l] = -1;
              c.state[l] = LS_IDLE;
            }
#endif
          } else {
            c.job[l] = -1;
            c.state[l] = LS_IDLE;
          }
          c.done[l] = 0;
          c.brk[l] = 0;
          c.n[l] = 0;
          c.inv_beta[l] = 0.0;
        }
        busy += (c.state[l] != LS_IDLE);
      }
      *c.queue_head = qh;
      const int unfinished = busy + (r.jobs.n_jobs - qh);
      *c.unfinished = unfinished;
      set_cond(r.gc, r.gc.h_outer, unfinished > 0 && step < r.gc.step_cap);
      break;
    }
    default:
      break;
  }
}

// ===========================================================================
// K1: block SpMM  Y[:, lanes] = S X[:, lanes]  (S = A or B, W lanes)
// ===========================================================================
// SP_DOT: Y = S X and the per-lane dot X.Y (own rows).
// SP_RESID: Y = P = u - S X (refinement residual), Z = 0, dot Y.Y.
// SP_CG: one CG step with the direction update folded in: X = r (gathered);
//   for own rows p <- r + b p and Y = B p <- B r + b (B p) with the lane's
//   direction coefficient b (0 starts a new direction), dot p.(B p).
enum SpmmMode : int { SP_DOT = 0, SP_RESID = 1, SP_CG = 2 };

template <typename TV, typename TX, typename TY>
struct SpmmArgs {
  Layout g;
  const TV* val;
  const TX* X;
  TY* Y;
  const double* U;   // SP_RESID: right-hand side u (FP64)
  TY* P;             // SP_RESID: CG direction, set to the residual
  TY* Z;             // SP_RESID: CG solution, set to zero
  RedArgs red;
};

template <typename T>
__device__ __forceinline__ T fmadd(T a, T b, T c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fmadd<float>(float a, float b, float c) { return fmaf(a, b, c); }

// Prefetch of a contiguous range into L2 (a hint: it never faults on the
// range given, which must be 16-byte aligned with a size multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Block kernels of the SpMM: one neighbour block times L lanes of X.
// 4-orbital row atom, 4-orbital neighbour: 4 X rows, 4 value columns.
template <typename TV, typename TX, typename TA, int L>
__device__ __forceinline__ void blk_4x4(const TV* __restrict__ v, const TX* __restrict__ xp, int W,
                                        TA (&acc)[4][L]) {
  TX x0[L], x1[L], x2[L], x3[L];
  ld_lanes<TX, L>(xp, x0);
  ld_lanes<TX, L>(xp + W, x1);
  ld_lanes<TX, L>(xp + 2 * W, x2);
  ld_lanes<TX, L>(xp + 3 * W, x3);
  const Quad<TV> c0 = ld_quad(v), c1 = ld_quad(v + 4), c2 = ld_quad(v + 8), c3 = ld_quad(v + 12);
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const TA y0 = TA(x0[i]), y1 = TA(x1[i]), y2 = TA(x2[i]), y3 = TA(x3[i]);
    acc[0][i] = fmadd<TA>(TA(c0.x), y0, fmadd<TA>(TA(c1.x), y1, fmadd<TA>(TA(c2.x), y2, fmadd<TA>(TA(c3.x), y3, acc[0][i]))));
    acc[1][i] = fmadd<TA>(TA(c0.y), y0, fmadd<TA>(TA(c1.y), y1, fmadd<TA>(TA(c2.y), y2, fmadd<TA>(TA(c3.y), y3, acc[1][i]))));
    acc[2][i] = fmadd<TA>(TA(c0.z), y0, fmadd<TA>(TA(c1.z), y1, fmadd<TA>(TA(c2.z), y2, fmadd<TA>(TA(c3.z), y3, acc[2][i]))));
    acc[3][i] = fmadd<TA>(TA(c0.w), y0, fmadd<TA>(TA(c1.w), y1, fmadd<TA>(TA(c2.w), y2, fmadd<TA>(TA(c3.w), y3, acc[3][i]))));
  }
}
// 4-orbital row atom, 1-orbital neighbour: 1 X row, one value per row.
template <typename TV, typename TX, typename TA, int L>
__device__ __forceinline__ void blk_4x1(const TV* __restrict__ v, const TX* __restrict__ xp, TA (&acc)[4][L]) {
  TX x0[L];
  ld_lanes<TX, L>(xp, x0);
  const Quad<TV> c0 = ld_quad(v);
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const TA y0 = TA(x0[i]);
    acc[0][i] = fmadd<TA>(TA(c0.x), y0, acc[0][i]);
    acc[1][i] = fmadd<TA>(TA(c0.y), y0, acc[1][i]);
    acc[2][i] = fmadd<TA>(TA(c0.z), y0, acc[2][i]);
    acc[3][i] = fmadd<TA>(TA(c0.w), y0, acc[3][i]);
  }
}
// 1-orbital row atom: four X rows (one 4-orbital neighbour, or four 1-orbital
// neighbours) against four values.
template <typename TV, typename TX, typename TA, int L>
__device__ __forceinline__ void blk_1x4(const TV* __restrict__ v, const TX* __restrict__ xa,
                                        const TX* __restrict__ xb, const TX* __restrict__ xc,
                                        const TX* __restrict__ xd, TA (&acc)[4][L]) {
  TX x0[L], x1[L], x2[L], x3[L];
  ld_lanes<TX, L>(xa, x0);
  ld_lanes<TX, L>(xb, x1);
  ld_lanes<TX, L>(xc, x2);
  ld_lanes<TX, L>(xd, x3);
  const Quad<TV> c0 = ld_quad(v);
#pragma unroll
  for (int i = 0; i < L; ++i)
    acc[0][i] = fmadd<TA>(TA(c0.x), TA(x0[i]), fmadd<TA>(TA(c0.y), TA(x1[i]),
                fmadd<TA>(TA(c0.z), TA(x2[i]), fmadd<TA>(TA(c0.w), TA(x3[i]), acc[0][i]))));
}

// Block arithmetic policies of the SpMM traversal.
template <typename TV, typename TX, typename TA, int L>
struct PlainOps {
  using V = TV;
  using X = TX;
  using Acc = TA;
  static __device__ __forceinline__ void zero(Acc (&acc)[4][L]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < L; ++i) acc[a][i] = TA(0);
  }
  static __device__ __forceinline__ void b44(const V* v, const X* xp, int W, Acc (&acc)[4][L]) {
    blk_4x4<TV, TX, TA, L>(v, xp, W, acc);
  }
  static __device__ __forceinline__ void b41(const V* v, const X* xp, Acc (&acc)[4][L]) {
    blk_4x1<TV, TX, TA, L>(v, xp, acc);
  }
  static __device__ __forceinline__ void b14(const V* v, const X* xa, const X* xb, const X* xc, const X* xd,
                                             Acc (&acc)[4][L]) {
    blk_1x4<TV, TX, TA, L>(v, xa, xb, xc, xd, acc);
  }
};

// Double-float policy: values are (hi, lo) FP32 pairs, X is double-float
// (float2) or single (float); every product enters an error-free accumulator.
__device__ __forceinline__ void ld_quad_df(const float2* __restrict__ p, float2 (&c)[4]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  c[0] = make_float2(a.x, a.y);
  c[1] = make_float2(a.z, a.w);
  c[2] = make_float2(b.x, b.y);
  c[3] = make_float2(b.z, b.w);
}
template <typename TX, int L>
__device__ __forceinline__ void ld_x(const TX* __restrict__ p, TX (&o)[L]) {
  if constexpr (sizeof(TX) == 8) {   // float2 lanes
    const float* f = reinterpret_cast<const float*>(p);
    if constexpr (L == 1) {
      const float2 v = *reinterpret_cast<const float2*>(f);
      o[0] = v;
    } else {
#pragma unroll
      for (int h = 0; h < L / 2; ++h) {
        const float4 v = reinterpret_cast<const float4*>(f)[h];
        o[2 * h] = make_float2(v.x, v.y);
        o[2 * h + 1] = make_float2(v.z, v.w);
      }
    }
  } else {
    ld_lanes<float, L>(reinterpret_cast<const float*>(p), reinterpret_cast<float(&)[L]>(o));
  }
}
template <typename TX, int L>
struct DfOps {
  using V = float2;
  using X = TX;
  using Acc = dfacc;
  static __device__ __forceinline__ void zero(Acc (&acc)[4][L]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < L; ++i) acc_zero(acc[a][i]);
  }
  static __device__ __forceinline__ void b44(const V* v, const X* xp, int W, Acc (&acc)[4][L]) {
    X x[4][L];
#pragma unroll
    for (int b = 0; b < 4; ++b) ld_x<X, L>(xp + b * W, x[b]);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      float2 c[4];
      ld_quad_df(v + 4 * b, c);
#pragma unroll
      for (int i = 0; i < L; ++i)
#pragma unroll
        for (int a = 0; a < 4; ++a) acc_fma(acc[a][i], c[a], x[b][i]);
    }
  }
  static __device__ __forceinline__ void b41(const V* v, const X* xp, Acc (&acc)[4][L]) {
    X x[L];
    ld_x<X, L>(xp, x);
    float2 c[4];
    ld_quad_df(v, c);
#pragma unroll
    for (int i = 0; i < L; ++i)
#pragma unroll
      for (int a = 0; a < 4; ++a) acc_fma(acc[a][i], c[a], x[i]);
  }
  static __device__ __forceinline__ void b14(const V* v, const X* xa, const X* xb, const X* xc, const X* xd,
                                             Acc (&acc)[4][L]) {
    X x[4][L];
    ld_x<X, L>(xa, x[0]);
    ld_x<X, L>(xb, x[1]);
    ld_x<X, L>(xc, x[2]);
    ld_x<X, L>(xd, x[3]);
    float2 c[4];
    ld_quad_df(v, c);
#pragma unroll
    for (int i = 0; i < L; ++i)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc_fma(acc[0][i], c[b], x[b][i]);
  }
};

// Split traversal: each thread owns 4 consecutive lanes (16- or 32-byte X
// loads); the warp's 32 / (W / 4) = G thread groups each take every G-th
// neighbour block of the same atom, so a warp runs G independent load chains
// without divergence; the groups' partial sums are combined by shuffles.
template <typename T>
__device__ __forceinline__ void combine_groups(T& v, int G) {
  for (int m = 32 / G; m < 32; m <<= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
}
__device__ __forceinline__ void combine_groups(dfacc& v, int G) {
  for (int m = 32 / G; m < 32; m <<= 1) {
    const float ohi = __shfl_xor_sync(0xffffffffu, v.hi, m);
    const float olo = __shfl_xor_sync(0xffffffffu, v.lo, m);
    const df s = two_sum(v.hi, ohi);
    v.hi = s.hi;
    v.lo = s.lo + (v.lo + olo);
  }
}

template <class Ops, int L, int G>
__device__ __forceinline__ void atom_row_product_split(const Layout& g, const typename Ops::V* __restrict__ val,
                                                       const typename Ops::X* __restrict__ X, int W, int I,
                                                       typename Ops::Acc (&acc)[4][L], int& oI, int& r0) {
  using TV = typename Ops::V;
  using TX = typename Ops::X;
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int grp = lane / (32 / G);
  const int lane0 = (lane % (32 / G)) * L;
  Ops::zero(acc);
#ifdef GSK_DEBUG
  // the atom, its own rows, its neighbour range and its value range (warp-uniform)
  oI = 0;
  r0 = 0;
  if (!GSK_IDX_OK(I >= 0 && I < g.n_atoms, 1, I)) return;
  {
    const int o = g.atom_orb[I], rr = g.atom_roff[I];
    if (!GSK_IDX_OK((o == 1 || o == 4) && rr >= 0 && rr + o <= g.M, 1, I)) return;
    const int b0 = g.nbr_ptr[I], bm = g.nbr_mid[I], b1 = g.nbr_ptr[I + 1];
    const int64_t vb0 = g.val_ptr[I];
    const int64_t nv = o == 4 ? 16 * (int64_t)(bm - b0) + 4 * (int64_t)(b1 - bm) : 4 * (int64_t)(bm - b0) + (b1 - bm);
    if (!GSK_IDX_OK(b0 >= 0 && b0 <= bm && bm <= b1 && b1 <= g.n_nbr && vb0 >= 0 && vb0 + nv <= g.n_vals, 2, I))
      return;
  }
#endif
  oI = g.atom_orb[I];
  r0 = g.atom_roff[I];
  const TV* v = val + g.val_ptr[I];
  const int e0 = g.nbr_ptr[I];
  const int em = g.nbr_mid[I];
  const int e1 = g.nbr_ptr[I + 1];
  auto xrow = [&](int r) { return X + (size_t)r * W + lane0; };
  if (oI == 4) {
    for (int base = e0; base < em; base += 32) {
      const int cnt = min(32, em - base);
      int myr = lane < cnt ? __ldg(&g.nbr_roff[base + lane]) : 0;
#ifdef GSK_DEBUG
      if (lane < cnt && !GSK_IDX_OK(myr >= 0 && myr + 4 <= g.M, 3, base + lane)) myr = 0;
#endif
      const TV* vb = v + (size_t)(base - e0) * 16;
      for (int t0 = 0; t0 < cnt; t0 += 2 * G) {
        const int ta = t0 + grp, tb = t0 + G + grp;
        const int ra = __shfl_sync(kFull, myr, ta & 31);
        const int rb = __shfl_sync(kFull, myr, tb & 31);
        if (ta < cnt) Ops::b44(vb + ta * 16, xrow(ra), W, acc);
        if (tb < cnt) Ops::b44(vb + tb * 16, xrow(rb), W, acc);
      }
    }
    const TV* vh = v + (size_t)(em - e0) * 16;
    for (int base = em; base < e1; base += 32) {
      const int cnt = min(32, e1 - base);
      int myr = lane < cnt ? __ldg(&g.nbr_roff[base + lane]) : 0;
#ifdef GSK_DEBUG
      if (lane < cnt && !GSK_IDX_OK(myr >= 0 && myr + 1 <= g.M, 3, base + lane)) myr = 0;
#endif
      const TV* vb = vh + (size_t)(base - em) * 4;
      for (int t0 = 0; t0 < cnt; t0 += 4 * G) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int t = t0 + k * G + grp;
          const int rr = __shfl_sync(kFull, myr, t & 31);
          if (t < cnt) Ops::b41(vb + t * 4, xrow(rr), acc);
        }
      }
    }
  } else {
    for (int base = e0; base < em; base += 32) {
      const int cnt = min(32, em - base);
      int myr = lane < cnt ? __ldg(&g.nbr_roff[base + lane]) : 0;
#ifdef GSK_DEBUG
      if (lane < cnt && !GSK_IDX_OK(myr >= 0 && myr + 4 <= g.M, 3, base + lane)) myr = 0;
#endif
      const TV* vb = v + (size_t)(base - e0) * 4;
      for (int t0 = 0; t0 < cnt; t0 += 2 * G) {
        const int ta = t0 + grp, tb = t0 + G + grp;
        const int ra = __shfl_sync(kFull, myr, ta & 31);
        const int rb = __shfl_sync(kFull, myr, tb & 31);
        if (ta < cnt) {
          const TX* xa = xrow(ra);
          Ops::b14(vb + ta * 4, xa, xa + W, xa + 2 * W, xa + 3 * W, acc);
        }
        if (tb < cnt) {
          const TX* xb = xrow(rb);
          Ops::b14(vb + tb * 4, xb, xb + W, xb + 2 * W, xb + 3 * W, acc);
        }
      }
    }
    // 1-orbital neighbours come padded to a multiple of 4: one value quad per 4 neighbours
    const TV* vh = v + (size_t)(em - e0) * 4;
    for (int base = em; base < e1; base += 32) {
      const int cnt = min(32, e1 - base);
      int myr = lane < cnt ? __ldg(&g.nbr_roff[base + lane]) : 0;
#ifdef GSK_DEBUG
      if (lane < cnt && !GSK_IDX_OK(myr >= 0 && myr + 1 <= g.M, 3, base + lane)) myr = 0;
#endif
      const TV* vb = vh + (base - em);
      const int nq = cnt / 4;
      for (int q0 = 0; q0 < nq; q0 += G) {
        const int q = q0 + grp;
        const int r0q = __shfl_sync(kFull, myr, (4 * q) & 31);
        const int r1q = __shfl_sync(kFull, myr, (4 * q + 1) & 31);
        const int r2q = __shfl_sync(kFull, myr, (4 * q + 2) & 31);
        const int r3q = __shfl_sync(kFull, myr, (4 * q + 3) & 31);
        if (q < nq) Ops::b14(vb + 4 * q, xrow(r0q), xrow(r1q), xrow(r2q), xrow(r3q), acc);
      }
    }
  }
  if constexpr (G > 1) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < L; ++i) combine_groups(acc[a][i], G);
  }
}

// Lanes per thread of the SpMM traversal: 4 for FP32 data (16-byte loads),
// 2 for 8-byte values or lanes (4 when the batch is 128 wide).
template <typename TV, typename TX, int LW>
constexpr int spmm_lanes() {
  return (sizeof(TV) == 4 && sizeof(TX) == 4) ? 4 : (LW > 2 ? LW : 2);
}

template <typename TV, typename TX, typename TY, typename TA, int LW, int MODE>
__global__ void __launch_bounds__(kThreads) k_spmm(const SpmmArgs<TV, TX, TY> a) {
  // W = 32 * LW lanes; each thread owns L lanes, L / LW thread groups per warp
  constexpr int L = spmm_lanes<TV, TX, LW>();
  constexpr int G = L / LW;
  const int W = a.red.W;
  const int lane = threadIdx.x & 31;
  const bool writer = lane < 32 / G;
  const int lane0 = (lane % (32 / G)) * L;
  const int warp = threadIdx.x >> 5;
  TA dot[L];
  TY cb[L];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    dot[i] = TA(0);
    cb[i] = (MODE == SP_CG) ? TY(a.red.c.cg_b[lane0 + i]) : TY(0);
  }
  const int gw = blockIdx.x * kWarps + warp;
  const int a1 = a.g.warp_atoms[gw + 1];
  for (int I = a.g.warp_atoms[gw]; I < a1; ++I) {
    TA acc[4][L];
    int oI, r0;
    atom_row_product_split<PlainOps<TV, TX, TA, L>, L, G>(a.g, a.val, a.X, W, I, acc, oI, r0);
    if (!writer) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (r >= oI) break;
      const size_t base = (size_t)(r0 + r) * W + lane0;
      TY y[L];
      if constexpr (MODE == SP_DOT) {
#pragma unroll
        for (int i = 0; i < L; ++i) y[i] = TY(acc[r][i]);
        st_lanes<TY, L>(a.Y + base, y);
        TX xo[L];
        ld_lanes<TX, L>(a.X + base, xo);
#pragma unroll
        for (int i = 0; i < L; ++i) dot[i] = fmadd<TA>(TA(xo[i]), TA(y[i]), dot[i]);
      } else if constexpr (MODE == SP_CG) {
        TX ro[L];
        TY po[L], so[L];
        ld_lanes<TX, L>(a.X + base, ro);
        ld_lanes<TY, L>(a.P + base, po);
        ld_lanes<TY, L>(a.Y + base, so);
#pragma unroll
        for (int i = 0; i < L; ++i) {
          const bool fresh = (cb[i] == TY(0));
          po[i] = fresh ? TY(ro[i]) : fmadd<TY>(cb[i], po[i], TY(ro[i]));
          y[i] = fresh ? TY(acc[r][i]) : fmadd<TY>(cb[i], so[i], TY(acc[r][i]));
          dot[i] = fmadd<TA>(TA(po[i]), TA(y[i]), dot[i]);
        }
        st_lanes<TY, L>(a.P + base, po);
        st_lanes<TY, L>(a.Y + base, y);
      } else {
        double uu[L];
        ld_lanes<double, L>(a.U + base, uu);
        TY z[L];
#pragma unroll
        for (int i = 0; i < L; ++i) {
          y[i] = TY(uu[i] - double(acc[r][i]));
          z[i] = TY(0);
          dot[i] = fmadd<TA>(TA(y[i]), TA(y[i]), dot[i]);
        }
        st_lanes<TY, L>(a.Y + base, y);
        st_lanes<TY, L>(a.P + base, y);
        st_lanes<TY, L>(a.Z + base, z);
      }
    }
  }
  double d[L];
#pragma unroll
  for (int i = 0; i < L; ++i) d[i] = double(dot[i]);
  lane_reduce_commit_at<L>(d, a.red, lane0, writer);
}

// ===========================================================================
// K1t: staged block SpMM for the FP32 inner CG (SP_CG form of k_spmm).
// ===========================================================================
// One CTA per SM works through a static list of items (tile, lane quarter):
// a W-lane batch runs W/32 lane quarters per tile, and gridDim.x is a
// multiple of W/32, so a CTA keeps one quarter q = blockIdx.x % (W/32).
// kProducers producer warps fill two shared-memory stages in turn: the row
// union of X = r and the tile's own rows of P and Y -- with 32 lanes (a row
// run is then contiguous in memory) by one 1-D TMA bulk copy per row-run
// piece and per own-row range, with 64 or 128 lanes by 16-byte asynchronous
// copies (cp.async, 4 rows x 128 bytes per warp instruction) -- and the
// tile's matrix values, local neighbour indices and atom descriptors by 1-D
// TMA bulk copies, all completing on the stage's "full" mbarrier. kTileWarps consumer
// warps run each item's fixed atom lists out of the stage -- four groups of 8
// threads take every fourth neighbour block of an atom, the groups are
// combined by shuffles, and group g writes own row g: p <- r + b p,
// B p <- B r + b B p, with the dot p.(B p) kept per lane -- and arrive on the
// stage's "empty" mbarrier, after which the producers refill it with the item
// two ahead. So one item's copies run while the previous one is computed, and
// a warp may start an item while slower warps finish the one before. Every
// wait is bounded; a wait that gives up sets *err and the waiting warp stops.
struct SpmmStagedArgs {
  Layout g;
  TileArgs t;
  const float* val;      // FP32 values of B in the block layout
  const float* X;        // r (gathered)
  float* P;              // CG direction
  float* Y;              // B p
  int W;                 // lanes of the batch
  int nq;                // W / 32
  int* err;
  RedArgs red;
};

constexpr int kProducers = 4;                                        // producer warps of the staged kernel
constexpr int kStagedThreads = 32 * (kTileWarps + kProducers);      // consumer warps + producer warps

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_add_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Test of a phase; a thread whose phase is still open is suspended for up to
// about 0.5 us (woken early when the phase completes) instead of spinning.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(500)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity; gives up after about 2 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > 4000000000LL) return false;
  return true;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// Shared row of a neighbour entry of a staged tile (checked in the bounds-checked build).
__device__ __forceinline__ int srow_of(const int16_t* lc, int t, int rows, int x_cap) {
  const int li = lc[t];
#ifdef GSK_DEBUG
  return GSK_IDX_OK(li >= 0 && li + rows <= x_cap, 14, t) ? li : 0;
#else
  (void)rows;
  (void)x_cap;
  return li;
#endif
}

// 16-byte asynchronous global -> shared copy (L2 only), and the arrival on an
// mbarrier once all of this thread's earlier copies have landed (the arrival
// is counted in the barrier's expected count).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fma_col(float (&acc)[4][4], const float4 c, const float4 x) {
  const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    acc[0][i] = fmaf(c.x, xs[i], acc[0][i]);
    acc[1][i] = fmaf(c.y, xs[i], acc[1][i]);
    acc[2][i] = fmaf(c.z, xs[i], acc[2][i]);
    acc[3][i] = fmaf(c.w, xs[i], acc[3][i]);
  }
}

// Shared-memory layout of one stage (offsets in bytes from the stage base).
struct StageLayout {
  uint32_t x, p, y, v, l, d, hdr, bytes;
  __host__ __device__ StageLayout(const TileArgs& t) {
    x = 0;
    p = x + (uint32_t)t.x_cap * kTileLanes * sizeof(float);
    y = p + (uint32_t)t.own_cap * kTileLanes * sizeof(float);
    v = y + (uint32_t)t.own_cap * kTileLanes * sizeof(float);
    l = v + (uint32_t)t.v_cap * sizeof(float);
    d = l + (uint32_t)t.l_cap * sizeof(int16_t);
    hdr = d + (uint32_t)t.d_cap * sizeof(int4);
    bytes = (hdr + sizeof(TileHead) + 127u) / 128u * 128u;
  }
};

#ifdef GSK_DEBUG
// A tile header whose copies stay inside the tile arrays, the value copy, the
// stage's buffers and the rows of X, with 16-byte aligned bulk copies.
__device__ __forceinline__ bool tile_head_ok(const TileHead& hd, const TileArgs& t, int M) {
  return hd.n_atoms >= 1 && hd.n_atoms <= t.d_cap && hd.d0 >= 0 && hd.d0 + hd.n_atoms <= t.n_desc &&
         hd.nval >= 0 && hd.nval <= t.v_cap && hd.v0 >= 0 && hd.v0 + hd.nval <= t.n_vals && (hd.v0 & 3) == 0 &&
         (hd.nval & 3) == 0 && hd.nloc >= 0 && hd.nloc <= t.l_cap && hd.l0 >= 0 && hd.l0 + hd.nloc <= t.n_loc &&
         (hd.l0 & 7) == 0 && (hd.nloc & 7) == 0 && hd.nbox >= 0 && hd.b0 >= 0 && hd.b0 + hd.nbox <= t.n_box &&
         hd.n_own >= 0 && hd.n_own <= t.own_cap && hd.r0 >= 0 && hd.r0 + hd.n_own <= M &&
         hd.wptr[kTileWarps] == hd.n_atoms;
}
// A row piece inside X and inside the stage's row buffer.
__device__ __forceinline__ bool piece_ok(int g0, int rows, int s0, const TileArgs& t, int M) {
  return rows >= 1 && rows <= kPieceRows && g0 >= 0 && g0 + rows <= M && s0 >= 0 && s0 + rows <= t.x_cap;
}
#endif

__global__ void __launch_bounds__(kStagedThreads, 1) k_spmm_staged(const SpmmStagedArgs a) {
  extern __shared__ __align__(128) unsigned char sm_raw[];
  __shared__ double sred[kTileWarps][kMaxW];
  __shared__ __align__(8) uint64_t full_bar[2], empty_bar[2];
  const StageLayout SL(a.t);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x % a.nq;      // lane quarter of this CTA
  const int qlane = q * kTileLanes;
  const int n_items = a.t.n_tiles * a.nq;
  const int n_mine = blockIdx.x < n_items ? (n_items - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&full_bar[s], 32 * kProducers + 1);   // every producer thread's copies + the bulk copies
      mbar_init(&empty_bar[s], kTileWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  float dot[4] = {0.f, 0.f, 0.f, 0.f};
  const int grp = (lane >> 3);          // consumers: 4 groups of 8 threads share one atom
  const int lane0 = (lane & 7) * 4;     // 4 lanes per thread
  bool ok = true;
  if (warp >= kTileWarps) {
    // ---------------- producers ----------------
    const int pw = warp - kTileWarps;         // producer warp pw copies boxes pw, pw + kProducers, ...
    int issued = 0;
    const int sub = lane >> 3, ch = (lane & 7) * 4;
    // the next item's header and this warp's first 32 boxes are loaded one
    // item ahead, so their latency overlaps the wait for a free stage
    TileHead hd_next;
    int2 box_next = make_int2(0, 0);
    auto fetch = [&](int j) {
      hd_next = a.t.head[(blockIdx.x + j * gridDim.x) / a.nq];
#ifdef GSK_DEBUG
      const int nm = (tile_head_ok(hd_next, a.t, a.g.M) && hd_next.nbox > pw)
                         ? (hd_next.nbox - pw + kProducers - 1) / kProducers : 0;
#else
      const int nm = hd_next.nbox > pw ? (hd_next.nbox - pw + kProducers - 1) / kProducers : 0;
#endif
      box_next = lane < nm ? a.t.box[hd_next.b0 + pw + kProducers * lane] : make_int2(0, 0);
    };
    if (n_mine > 0) fetch(0);
    for (int j = 0; j < n_mine && ok; ++j) {
      const int s = j & 1;
      unsigned char* st = sm_raw + (size_t)s * SL.bytes;
      const TileHead hd = hd_next;
      const int2 box0 = box_next;
#ifdef GSK_DEBUG
      const bool hok = (pw == 0 && lane == 0)
                           ? GSK_IDX_OK(tile_head_ok(hd, a.t, a.g.M), 10, (blockIdx.x + j * gridDim.x) / a.nq)
                           : tile_head_ok(hd, a.t, a.g.M);
#else
      constexpr bool hok = true;
#endif
      if (j + 1 < n_mine) fetch(j + 1);
      if (j >= 2) ok = __all_sync(0xffffffffu, mbar_wait_bounded(&empty_bar[s], ((j >> 1) - 1) & 1));  // item j-2 consumed
      if (!ok) break;
      // the consumers' generic reads of this stage are ordered before the async writes
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (pw == 0 && lane == 0) {
        *reinterpret_cast<TileHead*>(st + SL.hdr) = hd;
        const uint32_t bytes = hok ? (uint32_t)hd.nval * sizeof(float) + (uint32_t)hd.nloc * sizeof(int16_t) +
                                         (uint32_t)hd.n_atoms * sizeof(int4)
                                   : 0u;
        mbar_expect_tx(&full_bar[s], bytes);     // releases the header store with the arrival
        if (hok) {
          bulk_copy(st + SL.v, a.val + hd.v0, (uint32_t)hd.nval * sizeof(float), &full_bar[s]);
          bulk_copy(st + SL.l, a.t.loc + hd.l0, (uint32_t)hd.nloc * sizeof(int16_t), &full_bar[s]);
          bulk_copy(st + SL.d, a.t.desc + hd.d0, (uint32_t)hd.n_atoms * sizeof(int4), &full_bar[s]);
        }
      }
      // row union of X: 4 rows x 8 chunks of 16 bytes per warp instruction; this
      // warp copies boxes pw, pw + kProducers, ... (32 of them per register load)
      float* sX = reinterpret_cast<float*>(st + SL.x);
      float* sP = reinterpret_cast<float*>(st + SL.p);
      float* sYs = reinterpret_cast<float*>(st + SL.y);
      const int nmine = (hok && hd.nbox > pw) ? (hd.nbox - pw + kProducers - 1) / kProducers : 0;
      if (a.nq == 1) {
        // 32 lanes: a piece of a row run is contiguous in X, one bulk copy per piece
        for (int k0 = 0; k0 < nmine; k0 += 32) {
          int2 mybox = box0;
          if (k0 > 0) mybox = (k0 + lane < nmine) ? a.t.box[hd.b0 + pw + kProducers * (k0 + lane)] : make_int2(0, 0);
#ifdef GSK_DEBUG
          if (k0 + lane < nmine &&
              GSK_IDX_OK(piece_ok(mybox.x, mybox.y >> 16, mybox.y & 0xffff, a.t, a.g.M), 11,
                         hd.b0 + pw + kProducers * (k0 + lane))) {
#else
          if (k0 + lane < nmine) {
#endif
            const uint32_t bytes = (uint32_t)(kTileLanes * sizeof(float)) * (uint32_t)(mybox.y >> 16);
            mbar_add_tx(&full_bar[s], bytes);
            bulk_copy(sX + (mybox.y & 0xffff) * kTileLanes, a.X + (size_t)mybox.x * kTileLanes, bytes, &full_bar[s]);
          }
        }
        if (hok && pw == 1 && lane < 2) {
          const uint32_t bytes = (uint32_t)hd.n_own * kTileLanes * sizeof(float);
          mbar_add_tx(&full_bar[s], bytes);
          bulk_copy(lane == 0 ? sP : sYs, (lane == 0 ? a.P : a.Y) + (size_t)hd.r0 * kTileLanes, bytes, &full_bar[s]);
        }
      } else {
        for (int k0 = 0; k0 < nmine; k0 += 32) {
          int2 mybox = box0;
          if (k0 > 0) mybox = (k0 + lane < nmine) ? a.t.box[hd.b0 + pw + kProducers * (k0 + lane)] : make_int2(0, 0);
          const int kn = min(32, nmine - k0);
          for (int k = 0; k < kn; ++k) {
            const int g0 = __shfl_sync(0xffffffffu, mybox.x, k);
            const int code = __shfl_sync(0xffffffffu, mybox.y, k);
            const int hgt = code >> 16, s0 = code & 0xffff;
#ifdef GSK_DEBUG
            if (!GSK_IDX_OK(piece_ok(g0, hgt, s0, a.t, a.g.M), 11, hd.b0 + pw + kProducers * (k0 + k))) continue;
#endif
            for (int r = sub; r < hgt; r += 4)
              cp_async16(sX + (s0 + r) * kTileLanes + ch, a.X + (size_t)(g0 + r) * a.W + qlane + ch);
          }
        }
        // own rows of P and Y
        for (int r = pw * 4 + sub; hok && r < hd.n_own; r += 4 * kProducers) {
          const size_t g = (size_t)(hd.r0 + r) * a.W + qlane + ch;
          cp_async16(sP + r * kTileLanes + ch, a.P + g);
          cp_async16(sYs + r * kTileLanes + ch, a.Y + g);
        }
      }
      cp_async_arrive(&full_bar[s]);
      issued = j + 1;
    }
    // before exiting, every copy issued into this CTA's shared memory has landed
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (lane == 0)
      for (int j = max(0, issued - 2); j < issued; ++j)
        if (!mbar_wait_bounded(&full_bar[j & 1], (j >> 1) & 1)) ok = false;
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    if (!ok && lane == 0) atomicExch(a.err, 1);
  } else {
    // ---------------- consumers ----------------
    float cb[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) cb[i] = (float)a.red.c.cg_b[qlane + lane0 + i];
    for (int j = 0; j < n_mine; ++j) {
      const int s = j & 1;
      const unsigned char* st = sm_raw + (size_t)s * SL.bytes;
      if (!mbar_wait_bounded(&full_bar[s], (j >> 1) & 1)) {
        ok = false;
        break;
      }
      const TileHead* shd = reinterpret_cast<const TileHead*>(st + SL.hdr);
      const float* sX = reinterpret_cast<const float*>(st + SL.x);
      const float* sP = reinterpret_cast<const float*>(st + SL.p);
      const float* sY = reinterpret_cast<const float*>(st + SL.y);
      const float* sV = reinterpret_cast<const float*>(st + SL.v);
      const int16_t* sL = reinterpret_cast<const int16_t*>(st + SL.l);
      const int4* sD = reinterpret_cast<const int4*>(st + SL.d);
      const int r0 = shd->r0;
      const int k1 = shd->wptr[warp + 1];
#ifdef GSK_DEBUG
      // the warp's list inside the tile's descriptors (else the list is skipped)
      const int kb = GSK_IDX_OK(shd->wptr[warp] <= k1 && k1 <= shd->n_atoms && k1 <= a.t.d_cap, 12, warp)
                         ? (int)shd->wptr[warp] : k1;
#else
      const int kb = shd->wptr[warp];
#endif
      for (int k = kb; k < k1; ++k) {
        const int4 d = sD[k];
        const int oI = d.x & 0xff;
        const int prow = (d.x >> 8) & 0xff;
        const int xown = d.x >> 16;
        const int n4 = d.y & 0xffff, n1 = d.y >> 16;
#ifdef GSK_DEBUG
        {
          // the atom's own rows, values and neighbour indices inside the stage (warp-uniform)
          const int nv = oI == 4 ? 16 * n4 + 4 * n1 : 4 * n4 + n1;
          const bool ok = (oI == 4 || (oI == 1 && (n1 & 3) == 0)) && prow + oI <= shd->n_own &&
                          shd->n_own <= a.t.own_cap && r0 >= 0 && r0 + prow + oI <= a.g.M && xown >= 0 &&
                          xown + oI <= a.t.x_cap && d.z >= 0 && d.z + nv <= shd->nval && shd->nval <= a.t.v_cap &&
                          d.w >= 0 && d.w + n4 + n1 <= shd->nloc && shd->nloc <= a.t.l_cap;
          if (!GSK_IDX_OK(ok, 13, k)) continue;
        }
#endif
        const float* v = sV + d.z;
        const int16_t* lc = sL + d.w;
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[r][i] = 0.f;
        if (oI == 4) {
#pragma unroll 2
          for (int t = grp; t < n4; t += 4) {
            const float* xp = sX + srow_of(lc, t, 4, a.t.x_cap) * kTileLanes + lane0;
            const float4 x0 = lds4(xp), x1 = lds4(xp + kTileLanes), x2 = lds4(xp + 2 * kTileLanes),
                         x3 = lds4(xp + 3 * kTileLanes);
            const float* vb = v + t * 16;
            fma_col(acc, lds4(vb + 12), x3);
            fma_col(acc, lds4(vb + 8), x2);
            fma_col(acc, lds4(vb + 4), x1);
            fma_col(acc, lds4(vb), x0);
          }
          const float* vh = v + n4 * 16;
#pragma unroll 2
          for (int t = grp; t < n1; t += 4)
            fma_col(acc, lds4(vh + t * 4), lds4(sX + srow_of(lc, n4 + t, 1, a.t.x_cap) * kTileLanes + lane0));
        } else {
#pragma unroll 2
          for (int t = grp; t < n4; t += 4) {
            const float* xp = sX + srow_of(lc, t, 4, a.t.x_cap) * kTileLanes + lane0;
            const float4 c = lds4(v + t * 4);
            const float4 x0 = lds4(xp), x1 = lds4(xp + kTileLanes), x2 = lds4(xp + 2 * kTileLanes),
                         x3 = lds4(xp + 3 * kTileLanes);
            const float a0[4] = {x0.x, x0.y, x0.z, x0.w}, a1[4] = {x1.x, x1.y, x1.z, x1.w},
                        a2[4] = {x2.x, x2.y, x2.z, x2.w}, a3[4] = {x3.x, x3.y, x3.z, x3.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
              acc[0][i] = fmaf(c.x, a0[i], fmaf(c.y, a1[i], fmaf(c.z, a2[i], fmaf(c.w, a3[i], acc[0][i]))));
          }
          const float* vh = v + n4 * 4;
          const int nqd = n1 / 4;
#pragma unroll 2
          for (int qd = grp; qd < nqd; qd += 4) {
            const int16_t* lq = lc + n4 + 4 * qd;
            const float4 c = lds4(vh + 4 * qd);
            const float4 x0 = lds4(sX + srow_of(lq, 0, 1, a.t.x_cap) * kTileLanes + lane0),
                         x1 = lds4(sX + srow_of(lq, 1, 1, a.t.x_cap) * kTileLanes + lane0),
                         x2 = lds4(sX + srow_of(lq, 2, 1, a.t.x_cap) * kTileLanes + lane0),
                         x3 = lds4(sX + srow_of(lq, 3, 1, a.t.x_cap) * kTileLanes + lane0);
            const float a0[4] = {x0.x, x0.y, x0.z, x0.w}, a1[4] = {x1.x, x1.y, x1.z, x1.w},
                        a2[4] = {x2.x, x2.y, x2.z, x2.w}, a3[4] = {x3.x, x3.y, x3.z, x3.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
              acc[0][i] = fmaf(c.x, a0[i], fmaf(c.y, a1[i], fmaf(c.z, a2[i], fmaf(c.w, a3[i], acc[0][i]))));
          }
        }
        if (oI == 4) {
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              acc[r][i] += __shfl_xor_sync(0xffffffffu, acc[r][i], 8);
              acc[r][i] += __shfl_xor_sync(0xffffffffu, acc[r][i], 16);
            }
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[0][i] += __shfl_xor_sync(0xffffffffu, acc[0][i], 8);
            acc[0][i] += __shfl_xor_sync(0xffffffffu, acc[0][i], 16);
          }
        }
        if (grp < oI) {
          float br[4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
            br[i] = grp == 0 ? acc[0][i] : grp == 1 ? acc[1][i] : grp == 2 ? acc[2][i] : acc[3][i];
          const int pr = prow + grp;
          const float4 ro = lds4(sX + (xown + grp) * kTileLanes + lane0);
          const float4 po = lds4(sP + pr * kTileLanes + lane0);
          const float4 so = lds4(sY + pr * kTileLanes + lane0);
          const float rv[4] = {ro.x, ro.y, ro.z, ro.w}, pv[4] = {po.x, po.y, po.z, po.w},
                      sv[4] = {so.x, so.y, so.z, so.w};
          float pn[4], yn[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const bool fresh = (cb[i] == 0.f);
            pn[i] = fresh ? rv[i] : fmaf(cb[i], pv[i], rv[i]);
            yn[i] = fresh ? br[i] : fmaf(cb[i], sv[i], br[i]);
            dot[i] = fmaf(pn[i], yn[i], dot[i]);
          }
          const size_t base = (size_t)(r0 + pr) * a.W + qlane + lane0;
          *reinterpret_cast<float4*>(a.P + base) = make_float4(pn[0], pn[1], pn[2], pn[3]);
          *reinterpret_cast<float4*>(a.Y + base) = make_float4(yn[0], yn[1], yn[2], yn[3]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty_bar[s]);    // this warp is done with the stage
    }
    if (!ok && lane == 0) atomicExch(a.err, 1);
  }
  // per-lane dot: groups, then consumer warps in order, then the grid reduction
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    dot[i] += __shfl_xor_sync(0xffffffffu, dot[i], 8);
    dot[i] += __shfl_xor_sync(0xffffffffu, dot[i], 16);
  }
  if (warp < kTileWarps && grp == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) sred[warp][lane0 + i] = (double)dot[i];
  }
  __syncthreads();
  double sum = 0.0;
  if (threadIdx.x < a.W && threadIdx.x / kTileLanes == q) {
#pragma unroll
    for (int w = 0; w < kTileWarps; ++w) sum += sred[w][threadIdx.x % kTileLanes];
  }
  __syncthreads();
  cta_sums_commit(sum, a.red, sred);
}

// Double-float SpMM: Y = S X (SP_DOT: X = q in double-float, Y double-float,
// per-lane dot X.Y) or the refinement residual r = u - S v0 (SP_RESID: X = v0
// single, u double-float; r rounded to FP32 into Y and P, Z zeroed, r.r).
template <typename TX>
struct SpmmDfArgs {
  Layout g;
  const float2* val;
  const TX* X;
  float2* Y;          // SP_DOT output
  const float2* U;    // SP_RESID right-hand side
  float* R;           // SP_RESID residual (FP32)
  float* P;           // SP_RESID CG direction
  float* Z;           // SP_RESID CG solution (zeroed)
  RedArgs red;
};

template <typename TX, int LW, int MODE>
__global__ void __launch_bounds__(kThreads) k_spmm_df(const SpmmDfArgs<TX> a) {
  constexpr int L = spmm_lanes<float2, TX, LW>();
  constexpr int G = L / LW;
  const int W = a.red.W;
  const int lane = threadIdx.x & 31;
  const bool writer = lane < 32 / G;
  const int lane0 = (lane % (32 / G)) * L;
  const int warp = threadIdx.x >> 5;
  dfacc dacc[L];
  float facc[L];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    acc_zero(dacc[i]);
    facc[i] = 0.f;
  }
  const int gw = blockIdx.x * kWarps + warp;
  const int a1 = a.g.warp_atoms[gw + 1];
  for (int I = a.g.warp_atoms[gw]; I < a1; ++I) {
    dfacc acc[4][L];
    int oI, r0;
    atom_row_product_split<DfOps<TX, L>, L, G>(a.g, a.val, a.X, W, I, acc, oI, r0);
    if (!writer) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (r >= oI) break;
      const size_t base = (size_t)(r0 + r) * W + lane0;
      if constexpr (MODE == SP_DOT) {
        float2 y[L], xo[L];
#pragma unroll
        for (int i = 0; i < L; ++i) y[i] = df_to_float2(acc_value(acc[r][i]));
        ld_x<float2, L>(reinterpret_cast<const float2*>(a.X) + base, xo);
        float* yf = reinterpret_cast<float*>(a.Y + base);
#pragma unroll
        for (int i = 0; i < L; ++i) {
          reinterpret_cast<float2*>(yf)[i] = y[i];
          acc_fma(dacc[i], xo[i], y[i]);
        }
      } else {
        float2 uu[L];
        ld_x<float2, L>(a.U + base, uu);
        float rr[L], zz[L];
#pragma unroll
        for (int i = 0; i < L; ++i) {
          const df res = df_sub(df_from_float2(uu[i]), acc_value(acc[r][i]));
          rr[i] = res.hi + res.lo;
          zz[i] = 0.f;
          facc[i] = fmaf(rr[i], rr[i], facc[i]);
        }
        st_lanes<float, L>(a.R + base, rr);
        st_lanes<float, L>(a.P + base, rr);
        st_lanes<float, L>(a.Z + base, zz);
      }
    }
  }
  double d[L];
#pragma unroll
  for (int i = 0; i < L; ++i) d[i] = (MODE == SP_DOT) ? df_to_double(acc_value(dacc[i])) : (double)facc[i];
  lane_reduce_commit_at<L>(d, a.red, lane0, writer);
}

// ===========================================================================
// Vector kernels over all rows (warp per row, L lanes per thread)
// ===========================================================================
struct VecArgs {
  int M;
  double* q;
  double* ring0;
  double* ring1;
  double* u;       // holds w = A q on entry of the update kernel, u afterwards
  void* r;
  void* p;
  void* Bp;
  void* x;         // CG solution of the current pass (v, or v0 in mixed mode)
  void* x2;        // mixed mode: refinement correction d
  const int* step;
  RedArgs red;
};

__device__ __forceinline__ int vec_warp_id() { return blockIdx.x * kWarps + (threadIdx.x >> 5); }
__device__ __forceinline__ int vec_warp_count() { return gridDim.x * kWarps; }

// K_U: three-term update (or seed / idle), start of the B-solve, ||u||^2.
template <typename T, int L>
__global__ void __launch_bounds__(kThreads) k_update(const VecArgs a) {
  const int W = a.red.W;
  const int lane0 = (threadIdx.x & 31) * L;
  const LaneCtl& c = a.red.c;
  int st[L], jr[L];
  double al[L], bp[L];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const int l = lane0 + i;
    st[i] = c.state[l];
    al[i] = c.alpha[l];
    bp[i] = c.beta_prev[l];
#ifdef GSK_DEBUG
    // the job index, then its row of e_j, each checked before use
    jr[i] = -1;
    if (st[i] == LS_SEED) {
      const int jb = c.job[l];
      if (GSK_IDX_OK(jb >= 0 && jb < a.red.jobs.n_jobs, 21, jb)) {
        jr[i] = a.red.jobs.col_row[jb];
        if (!GSK_IDX_OK(jr[i] >= 0 && jr[i] < a.M, 22, jb)) jr[i] = -1;
      }
    }
#else
    jr[i] = (st[i] == LS_SEED) ? a.red.jobs.col_row[c.job[l]] : -1;
#endif
  }
  const int slot = (*a.step) & 1;
  const double* Bq = slot ? a.ring1 : a.ring0;
  const double* Bqm = slot ? a.ring0 : a.ring1;
  T* r = static_cast<T*>(a.r);
  T* p = static_cast<T*>(a.p);
  T* x = static_cast<T*>(a.x);
  T acc[L];
#pragma unroll
  for (int i = 0; i < L; ++i) acc[i] = T(0);
  for (int row = vec_warp_id(); row < a.M; row += vec_warp_count()) {
    const size_t base = (size_t)row * W + lane0;
    double w[L], b1[L], b2[L], uu[L];
    ld_lanes<double, L>(a.u + base, w);
    ld_lanes<double, L>(Bq + base, b1);
    ld_lanes<double, L>(Bqm + base, b2);
    T ut[L], zero[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
      if (st[i] == LS_ACTIVE)
        uu[i] = fma(-al[i], b1[i], fma(-bp[i], b2[i], w[i]));
      else if (st[i] == LS_SEED)
        uu[i] = (row == jr[i]) ? 1.0 : 0.0;
      else
        uu[i] = 0.0;
      ut[i] = T(uu[i]);
      zero[i] = T(0);
      acc[i] = fmadd<T>(ut[i], ut[i], acc[i]);
    }
    st_lanes<double, L>(a.u + base, uu);
    st_lanes<T, L>(r + base, ut);
    st_lanes<T, L>(p + base, ut);
    st_lanes<T, L>(x + base, zero);
  }
  double d[L];
#pragma unroll
  for (int i = 0; i < L; ++i) d[i] = double(acc[i]);
  lane_reduce_commit<L>(d, a.red);
}

// K_C: x += a p, r -= a Bp, r.r. Each thread owns 4 consecutive lanes
// (16-byte loads for FP32); a warp covers 128 / W rows per pass, and the
// per-lane sums of the rows a warp covers are combined by shuffles.
template <typename T, int LW>
__global__ void __launch_bounds__(kThreads) k_cg_update(const VecArgs a) {
  constexpr int L = 4;
  constexpr int RPW = 4 / LW;            // rows per warp pass (W = 32 * LW)
  const int W = a.red.W;
  const int lane = threadIdx.x & 31;
  const int sub = lane / (32 / RPW);     // which of the warp's rows
  const int lane0 = (lane % (32 / RPW)) * L;
  T ca[L];
#pragma unroll
  for (int i = 0; i < L; ++i) ca[i] = T(a.red.c.cg_a[lane0 + i]);
  T* r = static_cast<T*>(a.r);
  const T* p = static_cast<const T*>(a.p);
  const T* Bp = static_cast<const T*>(a.Bp);
  T* x = static_cast<T*>(a.x);
  T acc[L];
#pragma unroll
  for (int i = 0; i < L; ++i) acc[i] = T(0);
  for (int row0 = vec_warp_id() * RPW; row0 < a.M; row0 += vec_warp_count() * RPW) {
    const int row = row0 + sub;
    if (row < a.M) {
      const size_t base = (size_t)row * W + lane0;
      T pv[L], bv[L], xv[L], rv[L];
      ld_lanes<T, L>(p + base, pv);
      ld_lanes<T, L>(Bp + base, bv);
      ld_lanes<T, L>(x + base, xv);
      ld_lanes<T, L>(r + base, rv);
#pragma unroll
      for (int i = 0; i < L; ++i) {
        xv[i] = fmadd<T>(ca[i], pv[i], xv[i]);
        rv[i] = fmadd<T>(-ca[i], bv[i], rv[i]);
        acc[i] = fmadd<T>(rv[i], rv[i], acc[i]);
      }
      st_lanes<T, L>(x + base, xv);
      st_lanes<T, L>(r + base, rv);
    }
  }
  double d[L];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    d[i] = double(acc[i]);
    for (int m = 32 / RPW; m < 32; m <<= 1) d[i] += __shfl_xor_sync(0xffffffffu, d[i], m);
  }
  lane_reduce_commit_at<L>(d, a.red, lane0, sub == 0);
}

// v = x (FP64 mode) or v0 + d (mixed mode)
template <typename T, int L, bool MIXED>
__device__ __forceinline__ void load_v(const VecArgs& a, size_t base, double (&v)[L]) {
  T xv[L];
  ld_lanes<T, L>(static_cast<const T*>(a.x) + base, xv);
#pragma unroll
  for (int i = 0; i < L; ++i) v[i] = double(xv[i]);
  if constexpr (MIXED) {
    T dv[L];
    ld_lanes<T, L>(static_cast<const T*>(a.x2) + base, dv);
#pragma unroll
    for (int i = 0; i < L; ++i) v[i] += double(dv[i]);
  }
}

// K_D: u.v
template <typename T, int L, bool MIXED>
__global__ void __launch_bounds__(kThreads) k_dot_uv(const VecArgs a) {
  const int W = a.red.W;
  const int lane0 = (threadIdx.x & 31) * L;
  double acc[L];
#pragma unroll
  for (int i = 0; i < L; ++i) acc[i] = 0.0;
  for (int row = vec_warp_id(); row < a.M; row += vec_warp_count()) {
    const size_t base = (size_t)row * W + lane0;
    double uv[L], v[L];
    ld_lanes<double, L>(a.u + base, uv);
    load_v<T, L, MIXED>(a, base, v);
#pragma unroll
    for (int i = 0; i < L; ++i) acc[i] = fma(uv[i], v[i], acc[i]);
  }
  lane_reduce_commit<L>(acc, a.red);
}

// K_F: q = v / beta, Bq_new = u / beta, Bq_prev slot cleared for lanes that restart.
template <typename T, int L, bool MIXED>
__global__ void __launch_bounds__(kThreads) k_finish(const VecArgs a) {
  const int W = a.red.W;
  const int lane0 = (threadIdx.x & 31) * L;
  const LaneCtl& c = a.red.c;
  double ib[L];
  bool keep[L];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const int l = lane0 + i;
    ib[i] = c.inv_beta[l];
    keep[i] = (c.state[l] == LS_ACTIVE && c.n[l] >= 1 && ib[i] != 0.0);
  }
  const int slot = (*a.step) & 1;             // step already advanced by FIN_BETA
  double* Bq_new = slot ? a.ring1 : a.ring0;
  double* Bq_old = slot ? a.ring0 : a.ring1;
  for (int row = vec_warp_id(); row < a.M; row += vec_warp_count()) {
    const size_t base = (size_t)row * W + lane0;
    double uv[L], v[L], qn[L], bn[L];
    ld_lanes<double, L>(a.u + base, uv);
    load_v<T, L, MIXED>(a, base, v);
#pragma unroll
    for (int i = 0; i < L; ++i) {
      qn[i] = (ib[i] != 0.0) ? v[i] * ib[i] : 0.0;
      bn[i] = (ib[i] != 0.0) ? uv[i] * ib[i] : 0.0;
    }
    st_lanes<double, L>(a.q + base, qn);
    st_lanes<double, L>(Bq_new + base, bn);
    bool any_clear = false;
#pragma unroll
    for (int i = 0; i < L; ++i) any_clear |= !keep[i];
    if (any_clear) {
      double old[L];
      ld_lanes<double, L>(Bq_old + base, old);
#pragma unroll
      for (int i = 0; i < L; ++i)
        if (!keep[i]) old[i] = 0.0;
      st_lanes<double, L>(Bq_old + base, old);
    }
  }
}

// ---- double-float Lanczos vectors (mixed mode with FP32-pair refinement) ----
// K_U (double-float): u = w - alpha Bq - beta Bq_prev, FP32 start of the B-solve, r.r
template <int L>
__global__ void __launch_bounds__(kThreads) k_update_df(const VecArgs a) {
  const int W = a.red.W;
  const int lane0 = (threadIdx.x & 31) * L;
  const LaneCtl& c = a.red.c;
  int st[L], jr[L];
  df al[L], bp[L];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const int l = lane0 + i;
    st[i] = c.state[l];
    al[i] = df_from_double(c.alpha[l]);
    bp[i] = df_from_double(c.beta_prev[l]);
#ifdef GSK_DEBUG
    // the job index, then its row of e_j, each checked before use
    jr[i] = -1;
    if (st[i] == LS_SEED) {
      const int jb = c.job[l];
      if (GSK_IDX_OK(jb >= 0 && jb < a.red.jobs.n_jobs, 21, jb)) {
        jr[i] = a.red.jobs.col_row[jb];
        if (!GSK_IDX_OK(jr[i] >= 0 && jr[i] < a.M, 22, jb)) jr[i] = -1;
      }
    }
#else
    jr[i] = (st[i] == LS_SEED) ? a.red.jobs.col_row[c.job[l]] : -1;
#endif
  }
  const int slot = (*a.step) & 1;
  const float2* Bq = reinterpret_cast<const float2*>(slot ? a.ring1 : a.ring0);
  const float2* Bqm = reinterpret_cast<const float2*>(slot ? a.ring0 : a.ring1);
  float2* u = reinterpret_cast<float2*>(a.u);
  float* r = static_cast<float*>(a.r);
  float* p = static_cast<float*>(a.p);
  float* x = static_cast<float*>(a.x);
  float acc[L];
#pragma unroll
  for (int i = 0; i < L; ++i) acc[i] = 0.f;
  for (int row = vec_warp_id(); row < a.M; row += vec_warp_count()) {
    const size_t base = (size_t)row * W + lane0;
    float2 w[L], b1[L], b2[L];
    ld_x<float2, L>(u + base, w);
    ld_x<float2, L>(Bq + base, b1);
    ld_x<float2, L>(Bqm + base, b2);
    float ut[L], zero[L];
    float2 uo[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
      df uu;
      if (st[i] == LS_ACTIVE)
        uu = df_sub(df_sub(df_from_float2(w[i]), df_mul(al[i], df_from_float2(b1[i]))),
                    df_mul(bp[i], df_from_float2(b2[i])));
      else if (st[i] == LS_SEED)
        uu = df{(row == jr[i]) ? 1.f : 0.f, 0.f};
      else
        uu = df{0.f, 0.f};
      uo[i] = df_to_float2(uu);
      ut[i] = uu.hi;
      zero[i] = 0.f;
      acc[i] = fmaf(ut[i], ut[i], acc[i]);
    }
#pragma unroll
    for (int i = 0; i < L; ++i) u[base + i] = uo[i];
    st_lanes<float, L>(r + base, ut);
    st_lanes<float, L>(p + base, ut);
    st_lanes<float, L>(x + base, zero);
  }
  double d[L];
#pragma unroll
  for (int i = 0; i < L; ++i) d[i] = (double)acc[i];
  lane_reduce_commit<L>(d, a.red);
}

// v = v0 + d exactly as a double-float
template <int L>
__device__ __forceinline__ void load_v_df(const VecArgs& a, size_t base, df (&v)[L]) {
  float v0[L], dd[L];
  ld_lanes<float, L>(static_cast<const float*>(a.x) + base, v0);
  ld_lanes<float, L>(static_cast<const float*>(a.x2) + base, dd);
#pragma unroll
  for (int i = 0; i < L; ++i) v[i] = two_sum(v0[i], dd[i]);
}

// K_D (double-float): u.v
template <int L>
__global__ void __launch_bounds__(kThreads) k_dot_uv_df(const VecArgs a) {
  const int W = a.red.W;
  const int lane0 = (threadIdx.x & 31) * L;
  const float2* u = reinterpret_cast<const float2*>(a.u);
  dfacc acc[L];
#pragma unroll
  for (int i = 0; i < L; ++i) acc_zero(acc[i]);
  for (int row = vec_warp_id(); row < a.M; row += vec_warp_count()) {
    const size_t base = (size_t)row * W + lane0;
    float2 uu[L];
    ld_x<float2, L>(u + base, uu);
    df v[L];
    load_v_df<L>(a, base, v);
#pragma unroll
    for (int i = 0; i < L; ++i) acc_fma(acc[i], uu[i], df_to_float2(v[i]));
  }
  double d[L];
#pragma unroll
  for (int i = 0; i < L; ++i) d[i] = df_to_double(acc_value(acc[i]));
  lane_reduce_commit<L>(d, a.red);
}

// K_F (double-float): q = v / beta, Bq_new = u / beta, previous slot cleared on restart
template <int L>
__global__ void __launch_bounds__(kThreads) k_finish_df(const VecArgs a) {
  const int W = a.red.W;
  const int lane0 = (threadIdx.x & 31) * L;
  const LaneCtl& c = a.red.c;
  df ib[L];
  bool keep[L], zero_out[L];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const int l = lane0 + i;
    const double b = c.inv_beta[l];
    ib[i] = df_from_double(b);
    zero_out[i] = (b == 0.0);
    keep[i] = (c.state[l] == LS_ACTIVE && c.n[l] >= 1 && b != 0.0);
  }
  const int slot = (*a.step) & 1;
  float2* Bq_new = reinterpret_cast<float2*>(slot ? a.ring1 : a.ring0);
  float2* Bq_old = reinterpret_cast<float2*>(slot ? a.ring0 : a.ring1);
  const float2* u = reinterpret_cast<const float2*>(a.u);
  float2* q = reinterpret_cast<float2*>(a.q);
  bool any_clear = false;
#pragma unroll
  for (int i = 0; i < L; ++i) any_clear |= !keep[i];
  for (int row = vec_warp_id(); row < a.M; row += vec_warp_count()) {
    const size_t base = (size_t)row * W + lane0;
    float2 uu[L];
    ld_x<float2, L>(u + base, uu);
    df v[L];
    load_v_df<L>(a, base, v);
#pragma unroll
    for (int i = 0; i < L; ++i) {
      q[base + i] = zero_out[i] ? make_float2(0.f, 0.f) : df_to_float2(df_mul(v[i], ib[i]));
      Bq_new[base + i] = zero_out[i] ? make_float2(0.f, 0.f) : df_to_float2(df_mul(df_from_float2(uu[i]), ib[i]));
    }
    if (any_clear) {
#pragma unroll
      for (int i = 0; i < L; ++i)
        if (!keep[i]) Bq_old[base + i] = make_float2(0.f, 0.f);
    }
  }
}

// ===========================================================================
// K4: per-shift recurrences on the pattern rows of each lane's column
// ===========================================================================
struct ShiftArgs {
  LaneCtl c;
  Jobs jobs;
  int W, S, Pmax, nsplit;
  const double* eps;        // S: Re z_k
  const double* zim;        // S: Im z_k (used when col_eta == 0)
  int col_eta;              // 1: column c uses Re z_k + i*eta[c]
  const int64_t* job_off;   // n_jobs + 1
  const int32_t* prow;      // pattern rows (library order), job_off layout
  double2* pbuf;            // [W][Pmax][S]
  double2* xbuf;            // [W][Pmax][S]
  double2* dg;              // [W][2][S][2]  (d, g) per step parity
  const double* q;          // q_n (M x W): FP64, or double-float pairs when q_df
  int q_df;
  double2* G;               // output, job_off layout x S
  int32_t* out_iters;
  int32_t* out_status;
  double* out_resid;
  double tol;
  int max_iter;
#ifdef GSK_DEBUG
  int M;                    // rows of q (pattern rows are checked against it)
#endif
};

__global__ void __launch_bounds__(kThreads) k_shift(const ShiftArgs a) {
  const int lane = blockIdx.x;
  const int split = blockIdx.y;
  const LaneCtl& c = a.c;
  if (c.state[lane] != LS_ACTIVE) return;
  __shared__ double2 s_l[kMaxShifts];
  __shared__ double2 s_z[kMaxShifts];
  __shared__ double s_red[kThreads / 32];
  __shared__ int s_bad;
  const int S = a.S;
  const int job = c.job[lane];
#ifdef GSK_DEBUG
  if (!GSK_IDX_OK(job >= 0 && job < a.jobs.n_jobs, 21, job)) return;
  if (!GSK_IDX_OK(a.job_off[job + 1] - a.job_off[job] <= a.Pmax && a.job_off[job] <= a.job_off[job + 1], 23, job))
    return;
#endif
  const int nprev = c.n[lane];
  const int n = nprev + 1;                 // step processed now
  const int brk = c.brk[lane];
  const int64_t off = a.job_off[job];
  const int P = (int)(a.job_off[job + 1] - off);
  const double alpha = c.alpha[lane];
  const double bp = c.beta_prev[lane];
  const double b0 = c.beta0[lane];
  const double unorm = c.unorm[lane];
  const double eta = a.jobs.eta[job];
  double2* dg = a.dg + (size_t)lane * 4 * S;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  double rmax = 0.0;
  if (!brk) {
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
      const double2 sigma = make_double2(a.eps[k], a.col_eta ? eta : a.zim[k]);
      double2 l, d, g;
      if (n == 1) {
        l = make_double2(0.0, 0.0);
        d = make_double2(sigma.x - alpha, sigma.y);
        g = make_double2(b0, 0.0);
      } else {
        const double2 dprev = dg[((nprev & 1) * S + k) * 2 + 0];
        const double2 gprev = dg[((nprev & 1) * S + k) * 2 + 1];
        l = cdiv(make_double2(-bp, 0.0), dprev);
        d = make_double2(sigma.x - alpha + l.x * bp, sigma.y + l.y * bp);
        g = cmul(make_double2(-l.x, -l.y), gprev);
      }
      const double2 zeta = cdiv(g, d);
      if (split == 0) {
        dg[((n & 1) * S + k) * 2 + 0] = d;
        dg[((n & 1) * S + k) * 2 + 1] = g;
      }
      s_l[k] = l;
      s_z[k] = zeta;
      const double res = cabs2(zeta) * unorm;
      if (!isfinite(res)) s_bad = 1;       // benign race: every writer stores 1
      rmax = fmax(rmax, res);
    }
  }
  // block max of the residual estimates
  for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = rmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_red[w]);
    s_red[0] = m;
  }
  __syncthreads();
  rmax = s_red[0];
  const bool bad = brk || s_bad;
  const bool conv = !bad && rmax <= a.tol;
  const bool fin = bad || conv || n >= a.max_iter;
  const int rows_per = (P + a.nsplit - 1) / a.nsplit;
  const int i0 = split * rows_per;
  const int i1 = min(P, i0 + rows_per);
  double2* pb = a.pbuf + (size_t)lane * a.Pmax * S;
  double2* xb = a.xbuf + (size_t)lane * a.Pmax * S;
  double2* Gj = a.G + (size_t)off * S;
  const int total = (i1 - i0) * S;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int i = i0 + t / S;
    const int k = t - (t / S) * S;
    const size_t e = (size_t)i * S + k;
    double2 xv;
    if (!bad) {
#ifdef GSK_DEBUG
      const int pr = a.prow[off + i];
      const size_t qidx = (size_t)(GSK_IDX_OK(pr >= 0 && pr < a.M, 24, off + i) ? pr : 0) * a.W + lane;
#else
      const size_t qidx = (size_t)a.prow[off + i] * a.W + lane;
#endif
      double qi;
      if (a.q_df) {
        const float2 qq = reinterpret_cast<const float2*>(a.q)[qidx];
        qi = (double)qq.x + (double)qq.y;
      } else {
        qi = a.q[qidx];
      }
      double2 pv;
      if (n == 1) {
        pv = make_double2(qi, 0.0);
        xv = cmul(s_z[k], pv);
      } else {
        const double2 po = pb[e];
        const double2 lp = cmul(s_l[k], po);
        pv = make_double2(qi - lp.x, -lp.y);
        xv = cadd(xb[e], cmul(s_z[k], pv));
      }
      pb[e] = pv;
      xb[e] = xv;
    } else {
      xv = (nprev >= 1) ? xb[e] : make_double2(0.0, 0.0);
    }
    if (fin) Gj[e] = xv;
  }
  if (fin && split == 0 && threadIdx.x == 0) {
    a.out_iters[job] = bad ? nprev : n;
    a.out_status[job] = bad ? GSK_BREAKDOWN : (conv ? GSK_CONVERGED : GSK_NOT_CONVERGED);
    a.out_resid[job] = bad ? (double)NAN : rmax;
    c.done[lane] = 1;
    c.cg_on[lane] = 0;
  }
}

// ===========================================================================
// Prime / wrap-up
// ===========================================================================
struct PrimeArgs {
  LaneCtl c;
  Jobs jobs;
  GraphCtl gc;
  int W;
};

__global__ void k_prime(const PrimeArgs a) {
  const int l = threadIdx.x;
  const LaneCtl& c = a.c;
  if (l < a.W) {
    if (l < a.jobs.n_jobs) {
      c.job[l] = a.jobs.queue[l];
      c.state[l] = LS_SEED;
#ifdef GSK_DEBUG
      if (!GSK_IDX_OK(c.job[l] >= 0 && c.job[l] < a.jobs.n_jobs, 20, l)) {
        c.job[l] = -1;
        c.state[l] = LS_IDLE;
      }
#endif
    } else {
      c.job[l] = -1;
      c.state[l] = LS_IDLE;
    }
    c.n[l] = 0;
    c.done[l] = 0;
    c.brk[l] = 0;
    c.alpha[l] = 0.0;
    c.beta_prev[l] = 0.0;
    c.beta0[l] = 0.0;
    c.inv_beta[l] = 0.0;
    c.cg_on[l] = 0;
    c.cg_a[l] = 0.0;
    c.cg_b[l] = 0.0;
  }
  if (l == 0) {
    *c.queue_head = min(a.W, a.jobs.n_jobs);
    *c.step = 0;
    *c.cg_iter = 0;
    *c.cg_total = 0;
    *c.red_counter = 0u;
    *c.unfinished = a.jobs.n_jobs;
    if (a.gc.use_graph) cudaGraphSetConditional(a.gc.h_outer, a.jobs.n_jobs > 0 ? 1u : 0u);
  }
}

// Columns still running when the step cap stopped the loop: write their last
// iterate with GSK_TIMEOUT; columns never started: zero G, GSK_TIMEOUT.
struct WrapArgs {
  LaneCtl c;
  Jobs jobs;
  int W, S, Pmax;
  const int64_t* job_off;
  const double2* xbuf;
  double2* G;
  int32_t* out_iters;
  int32_t* out_status;
  double* out_resid;
};

__global__ void k_wrapup(const WrapArgs a) {
  const int lane = blockIdx.x;
  if (lane < a.W) {
    const LaneCtl& c = a.c;
    if (c.state[lane] == LS_ACTIVE && !c.done[lane]) {
      const int job = c.job[lane];
#ifdef GSK_DEBUG
      if (!GSK_IDX_OK(job >= 0 && job < a.jobs.n_jobs, 21, job)) return;
      if (!GSK_IDX_OK(a.job_off[job + 1] - a.job_off[job] <= a.Pmax, 23, job)) return;
#endif
      const int64_t off = a.job_off[job];
      const int P = (int)(a.job_off[job + 1] - off);
      const double2* xb = a.xbuf + (size_t)lane * a.Pmax * a.S;
      const bool have_x = c.n[lane] >= 1;
      for (int t = threadIdx.x; t < P * a.S; t += blockDim.x)
        a.G[(size_t)off * a.S + t] = have_x ? xb[t] : make_double2(0.0, 0.0);
      if (threadIdx.x == 0) {
        a.out_iters[job] = c.n[lane];
        a.out_status[job] = GSK_TIMEOUT;
        a.out_resid[job] = (double)NAN;
      }
    }
  }
}

__global__ void k_unstarted(Jobs jobs, const int64_t* job_off, int S, double2* G, int32_t* out_status,
                            int32_t* out_iters, double* out_resid) {
  for (int j = blockIdx.x; j < jobs.n_jobs; j += gridDim.x) {
    if (out_status[j] >= 0) continue;
    const int64_t off = job_off[j];
    const int64_t cnt = (job_off[j + 1] - off) * S;
    for (int64_t t = threadIdx.x; t < cnt; t += blockDim.x) G[off * S + t] = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
      out_status[j] = GSK_TIMEOUT;
      out_iters[j] = 0;
      out_resid[j] = (double)NAN;
    }
  }
}

// ===========================================================================
// Host orchestration
// ===========================================================================
namespace {

#define GSK_CUDA_TRY(expr)                 \
  do {                                     \
    cudaError_t _e = (expr);               \
    if (_e != cudaSuccess) return _e;      \
  } while (0)

struct GraphBuilder {
  cudaGraph_t g;
  cudaGraphNode_t last{};
  bool has_last = false;
  cudaError_t err = cudaSuccess;

  explicit GraphBuilder(cudaGraph_t graph) : g(graph) {}

  template <typename A>
  void kernel(void (*f)(A), dim3 grid, dim3 block, const A& arg, unsigned smem = 0) {
    if (err != cudaSuccess) return;
    cudaKernelNodeParams p = {};
    p.func = reinterpret_cast<void*>(f);
    p.gridDim = grid;
    p.blockDim = block;
    p.sharedMemBytes = smem;
    void* args[1] = {const_cast<A*>(&arg)};
    p.kernelParams = args;
    p.extra = nullptr;
    cudaGraphNode_t n;
    err = cudaGraphAddKernelNode(&n, g, has_last ? &last : nullptr, has_last ? 1 : 0, &p);
    if (err == cudaSuccess) {
      last = n;
      has_last = true;
    }
  }

  // Appends a WHILE node driven by handle h; returns its body graph.
  cudaGraph_t while_node(cudaGraphConditionalHandle h) {
    if (err != cudaSuccess) return nullptr;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t n;
    err = cudaGraphAddNode(&n, g, has_last ? &last : nullptr, nullptr, has_last ? 1 : 0, &cp);
    if (err != cudaSuccess) return nullptr;
    last = n;
    has_last = true;
    return cp.conditional.phGraph_out[0];
  }
};

// Everything one solve launches, with the launch shapes.
struct Plan {
  int W = 64;
  int L = 2;
  bool mixed = false;
  bool df = false;       // mixed mode with double-float refinement / Lanczos vectors
  bool refine = true;
  int grid_rows = 1;     // SpMM CTAs (== lay.n_ctas)
  int grid_vec = 1;      // vector-kernel CTAs
  int nsplit = 1;
  // kernel argument blocks
  SpmmArgs<double, double, double> spA;
  SpmmArgs<double, double, double> spB64;
  SpmmArgs<float, float, float> spB32[2];
  SpmmArgs<double, float, float> spR;
  SpmmDfArgs<float2> spAdf;
  SpmmDfArgs<float> spRdf;
  int spmm_kind = GSK_SPMM_GATHER;    // kernel of the FP32 inner-CG products
  int grid_staged = 1;
  unsigned staged_smem = 0;
  SpmmStagedArgs spS;
  VecArgs upd, cgu[2], dot, fin;
  ShiftArgs sh;
  PrimeArgs prime;
  WrapArgs wrap;
};

template <int L>
struct Kernels {
  // FP64 mode
  static constexpr auto spmm64 = k_spmm<double, double, double, double, L, SP_DOT>;
  static constexpr auto spmm64cg = k_spmm<double, double, double, double, L, SP_CG>;
  static constexpr auto upd64 = k_update<double, L>;
  static constexpr auto cgu64 = k_cg_update<double, L>;
  static constexpr auto dot64 = k_dot_uv<double, L, false>;
  static constexpr auto fin64 = k_finish<double, L, false>;
  // mixed mode
  static constexpr auto spmm32cg = k_spmm<float, float, float, float, L, SP_CG>;
  static constexpr auto resid = k_spmm<double, float, float, double, L, SP_RESID>;
  static constexpr auto upd32 = k_update<float, L>;
  static constexpr auto cgu32 = k_cg_update<float, L>;
  static constexpr auto dotm = k_dot_uv<float, L, true>;
  static constexpr auto finm = k_finish<float, L, true>;
  // mixed mode, double-float refinement
  static constexpr auto spmm_df = k_spmm_df<float2, L, SP_DOT>;
  static constexpr auto resid_df = k_spmm_df<float, L, SP_RESID>;
  static constexpr auto upd_df = k_update_df<L>;
  static constexpr auto dot_df = k_dot_uv_df<L>;
  static constexpr auto fin_df = k_finish_df<L>;
};

// Launch of one kernel either into a graph (builder) or onto a stream.
struct Launcher {
  GraphBuilder* gb = nullptr;
  cudaStream_t stream = nullptr;
  template <typename A>
  cudaError_t operator()(void (*f)(A), dim3 grid, dim3 block, const A& arg, unsigned smem = 0) {
    if (gb) {
      gb->kernel(f, grid, block, arg, smem);
      return gb->err;
    }
    f<<<grid, block, smem, stream>>>(arg);
    return cudaGetLastError();
  }
};


template <int L>
cudaError_t launch_cg_iteration(const Plan& P, Launcher& la, int pass) {
  using K = Kernels<L>;
  const dim3 blk(kThreads);
  if (!P.mixed) {
    GSK_CUDA_TRY(la(K::spmm64cg, dim3(P.grid_rows), blk, P.spB64));
    GSK_CUDA_TRY(la(K::cgu64, dim3(P.grid_vec), blk, P.cgu[0]));
  } else {
    if (P.spmm_kind == GSK_SPMM_STAGED)
      GSK_CUDA_TRY(la(k_spmm_staged, dim3(P.grid_staged), dim3(kStagedThreads), P.spS, P.staged_smem));
    else
      GSK_CUDA_TRY(la(K::spmm32cg, dim3(P.grid_rows), blk, P.spB32[pass]));
    GSK_CUDA_TRY(la(K::cgu32, dim3(P.grid_vec), blk, P.cgu[pass]));
  }
  return cudaSuccess;
}

template <int L>
cudaError_t launch_step_head(const Plan& P, Launcher& la) {
  using K = Kernels<L>;
  const dim3 blk(kThreads);
  if (P.df) {
    GSK_CUDA_TRY(la(K::spmm_df, dim3(P.grid_rows), blk, P.spAdf));
    GSK_CUDA_TRY(la(K::upd_df, dim3(P.grid_vec), blk, P.upd));
  } else {
    GSK_CUDA_TRY(la(K::spmm64, dim3(P.grid_rows), blk, P.spA));
    if (!P.mixed)
      GSK_CUDA_TRY(la(K::upd64, dim3(P.grid_vec), blk, P.upd));
    else
      GSK_CUDA_TRY(la(K::upd32, dim3(P.grid_vec), blk, P.upd));
  }
  GSK_CUDA_TRY(la(k_shift, dim3(P.W, P.nsplit), blk, P.sh));
  return cudaSuccess;
}

template <int L>
cudaError_t launch_step_tail(const Plan& P, Launcher& la) {
  using K = Kernels<L>;
  const dim3 blk(kThreads);
  if (P.df) {
    GSK_CUDA_TRY(la(K::dot_df, dim3(P.grid_vec), blk, P.dot));
    GSK_CUDA_TRY(la(K::fin_df, dim3(P.grid_vec), blk, P.fin));
  } else if (!P.mixed) {
    GSK_CUDA_TRY(la(K::dot64, dim3(P.grid_vec), blk, P.dot));
    GSK_CUDA_TRY(la(K::fin64, dim3(P.grid_vec), blk, P.fin));
  } else {
    GSK_CUDA_TRY(la(K::dotm, dim3(P.grid_vec), blk, P.dot));
    GSK_CUDA_TRY(la(K::finm, dim3(P.grid_vec), blk, P.fin));
  }
  return cudaSuccess;
}

template <int L>
cudaError_t launch_resid(const Plan& P, Launcher& la) {
  using K = Kernels<L>;
  if (P.df) return la(K::resid_df, dim3(P.grid_rows), dim3(kThreads), P.spRdf);
  return la(K::resid, dim3(P.grid_rows), dim3(kThreads), P.spR);
}

// Builds the whole solve as one graph: prime -> WHILE(outer) { head, WHILE(cg1),
// [resid, WHILE(cg2)], tail } -> wrap-up.
template <int L>
cudaError_t build_graph(Plan& P, cudaGraphExec_t* exec) {
  cudaGraph_t top;
  GSK_CUDA_TRY(cudaGraphCreate(&top, 0));
  cudaError_t err = cudaSuccess;
  do {
    cudaGraphConditionalHandle h_outer, h_in1, h_in2 = 0;
    err = cudaGraphConditionalHandleCreate(&h_outer, top, 0, 0);
    if (err) break;
    GraphBuilder gtop(top);
    // handles of the inner loops live in the outer body graph: created after it exists
    GraphCtl gc{};
    gc.use_graph = 1;
    gc.h_outer = h_outer;
    gc.max_inner = P.upd.red.gc.max_inner;
    gc.step_cap = P.upd.red.gc.step_cap;
    P.prime.gc = gc;
    Launcher lt{&gtop, nullptr};
    err = lt(k_prime, dim3(1), dim3(kMaxW), P.prime);
    if (err) break;
    cudaGraph_t body = gtop.while_node(h_outer);
    if ((err = gtop.err)) break;
    err = cudaGraphConditionalHandleCreate(&h_in1, body, 0, 0);
    if (err) break;
    if (P.mixed && P.refine) {
      err = cudaGraphConditionalHandleCreate(&h_in2, body, 0, 0);
      if (err) break;
    }
    gc.h_inner1 = h_in1;
    gc.h_inner2 = h_in2;
    // propagate graph control into every argument block
    RedArgs* reds[] = {&P.spA.red, &P.spB64.red, &P.spB32[0].red, &P.spB32[1].red, &P.spR.red,
                       &P.spAdf.red, &P.spRdf.red, &P.spS.red,
                       &P.upd.red, &P.cgu[0].red, &P.cgu[1].red,
                       &P.dot.red, &P.fin.red};
    for (RedArgs* r : reds) r->gc = gc;
    GraphBuilder gb(body);
    Launcher lb{&gb, nullptr};
    err = launch_step_head<L>(P, lb);
    if (err) break;
    cudaGraph_t in1 = gb.while_node(h_in1);
    if ((err = gb.err)) break;
    {
      GraphBuilder gi(in1);
      Launcher li{&gi, nullptr};
      err = launch_cg_iteration<L>(P, li, 0);
      if (err) break;
    }
    if (P.mixed && P.refine) {
      err = launch_resid<L>(P, lb);
      if (err) break;
      cudaGraph_t in2 = gb.while_node(h_in2);
      if ((err = gb.err)) break;
      GraphBuilder gi(in2);
      Launcher li{&gi, nullptr};
      err = launch_cg_iteration<L>(P, li, 1);
      if (err) break;
    }
    err = launch_step_tail<L>(P, lb);
    if (err) break;
    err = lt(k_wrapup, dim3(P.W), dim3(kThreads), P.wrap);
    if (err) break;
    err = cudaGraphInstantiate(exec, top, 0);
  } while (0);
  cudaGraphDestroy(top);
  return err;
}

// Host-driven loop with the same kernels (no graph): reads the loop flags back.
template <int L>
cudaError_t run_host_loop(Plan& P, cudaStream_t s, int* h_flag, const int* d_unfinished) {
  Launcher la{nullptr, s};
  GSK_CUDA_TRY(la(k_prime, dim3(1), dim3(kMaxW), P.prime));
  auto flag = [&](int* out) -> cudaError_t {
    GSK_CUDA_TRY(cudaMemcpyAsync(out, d_unfinished, sizeof(int), cudaMemcpyDeviceToHost, s));
    return cudaStreamSynchronize(s);
  };
  const int max_inner = P.upd.red.gc.max_inner;
  for (int step = 0; step < P.upd.red.gc.step_cap; ++step) {
    GSK_CUDA_TRY(launch_step_head<L>(P, la));
    // the update kernel leaves the number of lanes needing CG in *unfinished
    GSK_CUDA_TRY(flag(h_flag));
    for (int it = 0; it < max_inner && *h_flag > 0; ++it) {
      GSK_CUDA_TRY(launch_cg_iteration<L>(P, la, 0));
      GSK_CUDA_TRY(flag(h_flag));
    }
    if (P.mixed && P.refine) {
      GSK_CUDA_TRY(launch_resid<L>(P, la));
      GSK_CUDA_TRY(flag(h_flag));
      for (int it = 0; it < max_inner && *h_flag > 0; ++it) {
        GSK_CUDA_TRY(launch_cg_iteration<L>(P, la, 1));
        GSK_CUDA_TRY(flag(h_flag));
      }
    }
    GSK_CUDA_TRY(launch_step_tail<L>(P, la));
    GSK_CUDA_TRY(flag(h_flag));
    if (*h_flag == 0) break;
  }
  return la(k_wrapup, dim3(P.W), dim3(kThreads), P.wrap);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

// ===========================================================================
// gsk_solve
// ===========================================================================
int solve_impl(gsk_ctx* h, int32_t S, const double* z, const double* eta, int32_t n_cols,
               const int32_t* cols, const gsk_options* opt_in, double* G_out, int32_t* iters,
               int32_t* status, double* resid) {
  gsk_options opt;
  gsk_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (S < 1 || S > kMaxShifts || n_cols < 0 || !z || (n_cols > 0 && (!cols || !G_out)))
    return GSK_EINVAL;
  if (opt.precision != GSK_FP64 && opt.precision != GSK_MIXED && opt.precision != GSK_MIXED_DF)
    return GSK_EINVAL;
  if (!(opt.tol > 0.0) || opt.max_iter < 1) return GSK_EINVAL;
  if (opt.batch_w != 0 && opt.batch_w != 32 && opt.batch_w != 64 && opt.batch_w != 128) return GSK_EINVAL;
  if (opt.precision == GSK_FP64 && opt.batch_w == 128) return GSK_ENOTSUP;
  if (opt.max_inner < 1) opt.max_inner = 200;
  for (int k = 0; k < S; ++k)
    if (!isfinite(z[2 * k]) || !isfinite(z[2 * k + 1])) return GSK_EINVAL;
  if (!eta)
    for (int k = 0; k < S; ++k)
      if (!(z[2 * k + 1] > 0.0)) return GSK_EINVAL;
  if (n_cols == 0) return GSK_OK;
  const int M = h->M;
  {
    std::vector<char> seen(M, 0);
    for (int c = 0; c < n_cols; ++c) {
      if (cols[c] < 0 || cols[c] >= M || seen[cols[c]]) return GSK_EINVAL;
      seen[cols[c]] = 1;
      if (eta && !(eta[c] > 0.0 && isfinite(eta[c]))) return GSK_EINVAL;
    }
  }
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  cudaStream_t stream = static_cast<cudaStream_t>(opt.stream);

  Plan P;
  P.mixed = (opt.precision != GSK_FP64);
  P.df = (opt.precision == GSK_MIXED_DF);
  P.refine = P.mixed && opt.refine != 0;
  int W = opt.batch_w;
  if (W == 0 && h->tuned_w[opt.precision] != 0) W = h->tuned_w[opt.precision];
  if (W == 0) {
    // lanes in flight: enough columns to fill the batch, favouring wide batches
    W = (n_cols > 64 && P.mixed) ? 128 : 64;
    if (n_cols <= 32) W = 32;
    if (!P.mixed && W > 64) W = 64;
  }
  P.W = W;
  P.L = W / 32;
  P.grid_rows = h->lay.n_ctas;
  P.grid_vec = std::max(1, std::min((M + kWarps - 1) / kWarps, h->num_sms * 6));

  // ---- job arrays (host) ----
  std::vector<int64_t> job_off(n_cols + 1, 0);
  for (int c = 0; c < n_cols; ++c) {
    const int j = cols[c];
    job_off[c + 1] = job_off[c] + (h->row_ptr[j + 1] - h->row_ptr[j]);
  }
  const int64_t n_elem = job_off[n_cols];
  int Pmax = 0;
  for (int c = 0; c < n_cols; ++c) Pmax = std::max<int>(Pmax, (int)(job_off[c + 1] - job_off[c]));
  std::vector<int32_t> prow(n_elem), col_row(n_cols), queue(n_cols);
  std::vector<double> jeta(n_cols);
  for (int c = 0; c < n_cols; ++c) {
    const int j = cols[c];
    col_row[c] = h->row_lib[j];
    jeta[c] = eta ? eta[c] : z[1];
    int64_t t = job_off[c];
    for (int64_t e = h->row_ptr[j]; e < h->row_ptr[j + 1]; ++e) prow[t++] = h->row_lib[h->col_idx[e]];
    queue[c] = c;
  }
  if (opt.sched == GSK_SCHED_LEARNED) {
    const int rc = learned_order(h, n_cols, cols, jeta.data(), stream, queue);
    if (rc != GSK_OK) return rc;
  } else if (opt.sched != GSK_SCHED_FIFO) {
    return GSK_EINVAL;
  }
  std::vector<double> eps(2 * S);
  for (int k = 0; k < S; ++k) {
    eps[k] = z[2 * k];
    eps[S + k] = z[2 * k + 1];
  }

  // ---- device workspace ----
  const size_t MW = (size_t)M * W;
  const size_t b64 = align_up(MW * sizeof(double), 256);
  const size_t b32 = align_up(MW * sizeof(float), 256);
  const size_t bcg = P.mixed ? b32 : b64;
  const size_t vec_bytes = 4 * b64 + 5 * bcg;
  if (h->ws_vec.ensure(vec_bytes) != cudaSuccess) return GSK_ENOMEM;
  char* vb = h->ws_vec.as<char>();
  double* q = reinterpret_cast<double*>(vb);
  double* ring0 = reinterpret_cast<double*>(vb + b64);
  double* ring1 = reinterpret_cast<double*>(vb + 2 * b64);
  double* u = reinterpret_cast<double*>(vb + 3 * b64);
  char* cgb = vb + 4 * b64;
  void* x = cgb;
  void* x2 = cgb + bcg;
  void* r = cgb + 2 * bcg;
  void* p = cgb + 3 * bcg;
  void* Bp = cgb + 4 * bcg;

  // kernel of the FP32 inner-CG products (mixed modes) and its launch shape
  if (opt.spmm_kernel < GSK_SPMM_AUTO || opt.spmm_kernel > GSK_SPMM_STAGED) return GSK_EINVAL;
  {
    int kind = opt.spmm_kernel;
    if (!P.mixed || h->tiles.n_tiles == 0) {
      if (kind == GSK_SPMM_STAGED) return GSK_ENOTSUP;
      kind = GSK_SPMM_GATHER;
    }
    if (kind == GSK_SPMM_AUTO) {
      // the autotuner's pick for this lane width, else the measured rule: the
      // staged kernel at 32 lanes, the gather kernel at 64 and 128
      const int wi = W == 32 ? 0 : W == 64 ? 1 : 2;
      kind = h->tuned_kernel[opt.precision][wi] != 0 ? h->tuned_kernel[opt.precision][wi]
                                                     : (W == 32 ? GSK_SPMM_STAGED : GSK_SPMM_GATHER);
    }
    if (kind == GSK_SPMM_STAGED) {
      const int nq = W / kTileLanes;
      P.grid_staged = std::min(h->tiles.n_tiles * nq, h->num_sms);
      P.grid_staged = std::max(nq, P.grid_staged - P.grid_staged % nq);
      P.staged_smem = 2u * StageLayout(h->tiles).bytes;
      if (cudaFuncSetAttribute(k_spmm_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.staged_smem) !=
          cudaSuccess)
        return GSK_ECUDA;
    }
    P.spmm_kind = kind;
  }

  // lane control block
  const int n_red = std::max(std::max(P.grid_rows, P.grid_vec), P.grid_staged);
  if (n_red > kMaxRedCtas) return GSK_ENOTSUP;
  const int n_grp_max = (kMaxRedCtas + kRedGroup - 1) / kRedGroup;
  const size_t lane_bytes = 64 * kMaxW * sizeof(double) + (size_t)n_red * kMaxW * sizeof(double) +
                            (size_t)n_grp_max * kMaxW * sizeof(double) + n_grp_max * sizeof(unsigned) + 256;
  if (h->ws_lane.ensure(lane_bytes) != cudaSuccess) return GSK_ENOMEM;
  char* lb = h->ws_lane.as<char>();
  LaneCtl c{};
  {
    size_t o = 0;
    auto take_i = [&]() { int* ptr = reinterpret_cast<int*>(lb + o); o += kMaxW * sizeof(double); return ptr; };
    auto take_d = [&]() { double* ptr = reinterpret_cast<double*>(lb + o); o += kMaxW * sizeof(double); return ptr; };
    c.job = take_i(); c.state = take_i(); c.n = take_i(); c.done = take_i(); c.brk = take_i();
    c.alpha = take_d(); c.beta_prev = take_d(); c.beta0 = take_d(); c.unorm = take_d();
    c.inv_beta = take_d(); c.rr = take_d(); c.rr_target = take_d(); c.cg_a = take_d();
    c.cg_b = take_d(); c.cg_on = take_i(); c.red_out = take_d();
    int* scal = take_i();
    c.queue_head = scal + 0; c.cg_iter = scal + 1; c.step = scal + 2; c.unfinished = scal + 3;
    c.cg_total = scal + 4;
    c.red_counter = reinterpret_cast<unsigned int*>(scal + 5);
    c.err = scal + 8;
    c.partials = reinterpret_cast<double*>(lb + o);
    o += (size_t)n_red * kMaxW * sizeof(double);
    c.grp_partials = reinterpret_cast<double*>(lb + o);
    o += (size_t)n_grp_max * kMaxW * sizeof(double);
    c.grp_counter = reinterpret_cast<unsigned int*>(lb + o);
  }

  // job arrays
  const size_t jb_bytes = align_up((n_cols + 1) * sizeof(int64_t), 256) +
                          align_up(n_elem * sizeof(int32_t), 256) +
                          3 * align_up(n_cols * sizeof(int32_t), 256) +
                          align_up(n_cols * sizeof(double), 256) * 2 +
                          align_up(2 * S * sizeof(double), 256) +
                          align_up(n_cols * sizeof(int32_t), 256);
  if (h->ws_jobs.ensure(jb_bytes) != cudaSuccess) return GSK_ENOMEM;
  char* jbp = h->ws_jobs.as<char>();
  size_t jo = 0;
  auto jtake = [&](size_t bytes) { void* ptr = jbp + jo; jo += align_up(bytes, 256); return ptr; };
  int64_t* d_job_off = static_cast<int64_t*>(jtake((n_cols + 1) * sizeof(int64_t)));
  int32_t* d_prow = static_cast<int32_t*>(jtake(n_elem * sizeof(int32_t)));
  int32_t* d_col_row = static_cast<int32_t*>(jtake(n_cols * sizeof(int32_t)));
  int32_t* d_queue = static_cast<int32_t*>(jtake(n_cols * sizeof(int32_t)));
  int32_t* d_status = static_cast<int32_t*>(jtake(n_cols * sizeof(int32_t)));
  double* d_eta = static_cast<double*>(jtake(n_cols * sizeof(double)));
  double* d_resid = static_cast<double*>(jtake(n_cols * sizeof(double)));
  double* d_eps = static_cast<double*>(jtake(2 * S * sizeof(double)));
  int32_t* d_iters = static_cast<int32_t*>(jtake(n_cols * sizeof(int32_t)));

  // shift state
  const size_t sh_bytes = 2 * align_up((size_t)W * Pmax * S * sizeof(double2), 256) +
                          align_up((size_t)W * 4 * S * sizeof(double2), 256);
  if (h->ws_shift.ensure(sh_bytes) != cudaSuccess) return GSK_ENOMEM;
  double2* pbuf = h->ws_shift.as<double2>();
  double2* xbuf = reinterpret_cast<double2*>(h->ws_shift.as<char>() + align_up((size_t)W * Pmax * S * sizeof(double2), 256));
  double2* dgb = reinterpret_cast<double2*>(h->ws_shift.as<char>() + 2 * align_up((size_t)W * Pmax * S * sizeof(double2), 256));

  // output staging for host G buffers
  cudaPointerAttributes pa{};
  bool g_on_device = false;
  if (cudaPointerGetAttributes(&pa, G_out) == cudaSuccess)
    g_on_device = (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  double2* Gd = reinterpret_cast<double2*>(G_out);
  const size_t g_bytes = (size_t)n_elem * S * sizeof(double2);
  if (!g_on_device) {
    if (h->ws_gstage.ensure(g_bytes) != cudaSuccess) return GSK_ENOMEM;
    Gd = h->ws_gstage.as<double2>();
  }

  // uploads
  cudaError_t e = cudaSuccess;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream);
  };
  up(d_job_off, job_off.data(), (n_cols + 1) * sizeof(int64_t));
  up(d_prow, prow.data(), n_elem * sizeof(int32_t));
  up(d_col_row, col_row.data(), n_cols * sizeof(int32_t));
  up(d_queue, queue.data(), n_cols * sizeof(int32_t));
  up(d_eta, jeta.data(), n_cols * sizeof(double));
  up(d_eps, eps.data(), 2 * S * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0xff, n_cols * sizeof(int32_t), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(vb, 0, vec_bytes, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(lb, 0, lane_bytes, stream);
  if (e != cudaSuccess) return GSK_ECUDA;

  // ---- argument blocks ----
  Jobs jobs{n_cols, d_queue, d_col_row, d_eta};
  GraphCtl gc{};
  gc.use_graph = 0;
  gc.max_inner = opt.max_inner;
  const int per_lane = (n_cols + W - 1) / W + 1;
  gc.step_cap = (int)std::min<int64_t>((int64_t)(opt.max_iter + 2) * per_lane, 2000000000LL);
  const double itol = (opt.inner_tol > 0.0) ? opt.inner_tol : (P.mixed ? 3e-6 : 1e-12);
  RedArgs rb{};
  rb.c = c;
  rb.jobs = jobs;
  rb.gc = gc;
  rb.W = W;
  rb.inner_tol2 = itol * itol;
  rb.max_iter = opt.max_iter;
  auto red = [&](int fin) { RedArgs x = rb; x.fin = fin; return x; };

  const Layout& g = h->lay;
  P.spA = {g, h->d_A64.as<double>(), q, u, nullptr, nullptr, nullptr, red(FIN_ALPHA)};
  P.spB64 = {g, h->d_B64.as<double>(), static_cast<double*>(r), static_cast<double*>(Bp), nullptr,
             static_cast<double*>(p), nullptr, red(FIN_CG_A)};
  for (int ps = 0; ps < 2; ++ps)
    P.spB32[ps] = {g, h->d_B32.as<float>(), static_cast<float*>(r), static_cast<float*>(Bp), nullptr,
                   static_cast<float*>(p), nullptr, red(FIN_CG_A)};
  P.spR = {g, h->d_B64.as<double>(), static_cast<float*>(x), static_cast<float*>(r), u, static_cast<float*>(p), static_cast<float*>(x2), red(FIN_RESID)};
  P.spAdf = {g, h->d_A2.as<float2>(), reinterpret_cast<const float2*>(q), reinterpret_cast<float2*>(u), nullptr,
             nullptr, nullptr, nullptr, red(FIN_ALPHA)};
  P.spRdf = {g, h->d_B2.as<float2>(), static_cast<const float*>(x), nullptr, reinterpret_cast<const float2*>(u),
             static_cast<float*>(r), static_cast<float*>(p), static_cast<float*>(x2), red(FIN_RESID)};
  if (P.spmm_kind == GSK_SPMM_STAGED) {
    P.spS.g = g;
    P.spS.t = h->tiles;
    P.spS.val = h->d_B32.as<float>();
    P.spS.X = static_cast<const float*>(r);
    P.spS.P = static_cast<float*>(p);
    P.spS.Y = static_cast<float*>(Bp);
    P.spS.W = W;
    P.spS.nq = W / kTileLanes;
    P.spS.err = c.err;
    P.spS.red = red(FIN_CG_A);
  }
  VecArgs va{};
  va.M = M; va.q = q; va.ring0 = ring0; va.ring1 = ring1; va.u = u;
  va.r = r; va.p = p; va.Bp = Bp; va.x = x; va.x2 = x2; va.step = c.step;
  P.upd = va; P.upd.red = red(FIN_UNORM);
  for (int ps = 0; ps < 2; ++ps) {
    P.cgu[ps] = va;
    P.cgu[ps].x = ps == 0 ? x : x2;
    P.cgu[ps].red = red(FIN_CG_RR);
    P.cgu[ps].red.max_iter = ps == 0 ? opt.max_iter : -1;
  }
  P.dot = va; P.dot.red = red(FIN_BETA);
  P.fin = va; P.fin.red = red(FIN_SUM);
  P.nsplit = std::max(1, std::min(8, (h->num_sms * 2) / W));
  P.sh = ShiftArgs{c, jobs, W, S, Pmax, P.nsplit, d_eps, d_eps + S, eta ? 1 : 0, d_job_off, d_prow, pbuf, xbuf, dgb, q, P.df ? 1 : 0, Gd,
                   d_iters, d_status, d_resid, opt.tol, opt.max_iter};
#ifdef GSK_DEBUG
  P.sh.M = h->M;
#endif
  P.prime = PrimeArgs{c, jobs, gc, W};
  P.wrap = WrapArgs{c, jobs, W, S, Pmax, d_job_off, xbuf, Gd, d_iters, d_status, d_resid};

#ifdef GSK_DEBUG
  {
    const int zero[4] = {0, 0, 0, 0};
    if (cudaMemcpyToSymbolAsync(g_dbg, zero, sizeof(zero), 0, cudaMemcpyHostToDevice, stream) != cudaSuccess)
      return GSK_ECUDA;
  }
#endif
  // ---- run ----
  auto run = [&](auto Ltag) -> cudaError_t {
    constexpr int LL = decltype(Ltag)::value;
    if (opt.use_graph) {
      cudaGraphExec_t ex = nullptr;
      cudaError_t ge = build_graph<LL>(P, &ex);
      if (ge == cudaSuccess) {
        ge = cudaGraphLaunch(ex, stream);
        cudaGraphExecDestroy(ex);
        return ge;
      }
      cudaGetLastError();
      return ge;
    }
    int* hflag = nullptr;
    GSK_CUDA_TRY(cudaMallocHost(&hflag, sizeof(int)));
    cudaError_t he = run_host_loop<LL>(P, stream, hflag, c.unfinished);
    cudaFreeHost(hflag);
    return he;
  };
  if (P.L == 1)
    e = run(std::integral_constant<int, 1>{});
  else if (P.L == 2)
    e = run(std::integral_constant<int, 2>{});
  else
    e = run(std::integral_constant<int, 4>{});
  if (e != cudaSuccess) return GSK_ECUDA;
  k_unstarted<<<std::min(n_cols, 1024), 128, 0, stream>>>(jobs, d_job_off, S, Gd, d_status, d_iters, d_resid);
  if (cudaGetLastError() != cudaSuccess) return GSK_ECUDA;

  // ---- results ----
  if (!g_on_device) e = cudaMemcpyAsync(G_out, Gd, g_bytes, cudaMemcpyDeviceToHost, stream);
  std::vector<int32_t> h_it(n_cols), h_st(n_cols);
  std::vector<double> h_rs(n_cols);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_it.data(), d_iters, n_cols * sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_st.data(), d_status, n_cols * sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_rs.data(), d_resid, n_cols * sizeof(double), cudaMemcpyDeviceToHost, stream);
  int h_cnt[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_cnt, c.queue_head, 9 * sizeof(int), cudaMemcpyDeviceToHost, stream);
  int h_dbg[4] = {0, 0, 0, 0};
#ifdef GSK_DEBUG
  if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(h_dbg, g_dbg, sizeof(h_dbg), 0, cudaMemcpyDeviceToHost, stream);
#endif
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return GSK_ECUDA;
  h->last.debug_code = h_dbg[0];
  h->last.debug_index = ((int64_t)h_dbg[2] << 32) | (int64_t)(uint32_t)h_dbg[1];
  if (h_dbg[0] != 0) return GSK_EBOUNDS;      // bounds-checked build: an index check failed
  if (h_cnt[8] != 0) return GSK_ETIMEOUT;     // a bounded wait of the staged SpMM gave up
  {
    // scal layout: queue_head, cg_iter, step, unfinished, cg_total
    const int64_t steps = h_cnt[2], cgt = h_cnt[4];
    h->last.outer_steps = steps;
    h->last.cg_iterations = cgt;
    const int64_t per_step = 3 + 2 + ((P.mixed && P.refine) ? 1 : 0);
    h->last.kernel_launches = 3 + steps * per_step + cgt * 2;
    h->last.batch_w = W;
    h->last.used_graph = opt.use_graph ? 1 : 0;
    h->last.spmm_kernel = P.spmm_kind;
  }
  if (iters) memcpy(iters, h_it.data(), n_cols * sizeof(int32_t));
  if (status) memcpy(status, h_st.data(), n_cols * sizeof(int32_t));
  if (resid) memcpy(resid, h_rs.data(), n_cols * sizeof(double));
  return GSK_OK;
}

}  // namespace gsk

// ===========================================================================
// Standalone block SpMM (same kernel and launch shape as inside the solve)
// ===========================================================================
namespace gsk {

#ifdef GSK_DEBUG
// Clear the record of failed index checks (before a call's kernels).
int dbg_reset(cudaStream_t s) {
  const int zero[4] = {0, 0, 0, 0};
  return cudaMemcpyToSymbolAsync(g_dbg, zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s) == cudaSuccess ? GSK_OK
                                                                                                       : GSK_ECUDA;
}
// Wait for the call's kernels and report the first failed index check.
int dbg_collect(gsk_ctx* h, cudaStream_t s) {
  int d[4] = {0, 0, 0, 0};
  if (cudaMemcpyFromSymbolAsync(d, g_dbg, sizeof(d), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return GSK_ECUDA;
  h->last.debug_code = d[0];
  h->last.debug_index = ((int64_t)d[2] << 32) | (int64_t)(uint32_t)d[1];
  return d[0] != 0 ? GSK_EBOUNDS : GSK_OK;
}
#endif

int spmm_impl(gsk_ctx* h, int32_t which, int32_t precision, int32_t W, const void* X, void* Y, int32_t n_rep,
              void* stream) {
  if (which < 0 || which > 2 || (precision != GSK_FP64 && precision != GSK_MIXED) || n_rep < 0 || !X || !Y)
    return GSK_EINVAL;
  if (W != 32 && W != 64 && W != 128) return GSK_EINVAL;
  if (precision == GSK_FP64 && W == 128) return GSK_ENOTSUP;
  if (which == 2 && (precision != GSK_MIXED || h->tiles.n_tiles == 0)) return GSK_ENOTSUP;
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
#ifdef GSK_DEBUG
  if (dbg_reset(s) != GSK_OK) return GSK_ECUDA;
#endif
  const int nq = W / kTileLanes;
  int grid_t = std::min(h->tiles.n_tiles * nq, h->num_sms);
  grid_t = std::max(nq, grid_t - grid_t % nq);
  const int grid = which == 2 ? std::max(h->lay.n_ctas, grid_t) : h->lay.n_ctas;
  const int n_grp_max = (kMaxRedCtas + kRedGroup - 1) / kRedGroup;
  const size_t lane_bytes = 64 * kMaxW * sizeof(double) + (size_t)grid * kMaxW * sizeof(double) +
                            (size_t)n_grp_max * kMaxW * sizeof(double) + n_grp_max * sizeof(unsigned) + 256;
  if (grid > kMaxRedCtas) return GSK_ENOTSUP;
  if (h->ws_lane.ensure(lane_bytes) != cudaSuccess) return GSK_ENOMEM;
  // direction vector of the CG form of the product (B): M x W, zero coefficient
  const size_t esz = precision == GSK_FP64 ? sizeof(double) : sizeof(float);
  if (which >= 1 && h->ws_misc.ensure((size_t)h->M * W * esz + 256) != cudaSuccess) return GSK_ENOMEM;
  char* lb = h->ws_lane.as<char>();
  if (cudaMemsetAsync(lb, 0, lane_bytes, s) != cudaSuccess) return GSK_ECUDA;
  LaneCtl c{};
  c.red_out = reinterpret_cast<double*>(lb);
  c.cg_b = reinterpret_cast<double*>(lb + kMaxW * sizeof(double));             // all zero
  c.red_counter = reinterpret_cast<unsigned int*>(lb + 2 * kMaxW * sizeof(double));
  c.partials = reinterpret_cast<double*>(lb + 3 * kMaxW * sizeof(double));
  c.grp_partials = c.partials + (size_t)grid * kMaxW;
  c.grp_counter = reinterpret_cast<unsigned int*>(c.grp_partials + (size_t)n_grp_max * kMaxW);
  RedArgs r{};
  r.c = c;
  r.fin = FIN_SUM;
  r.W = W;
  const dim3 blk(kThreads), grd(grid);
  void* P = which >= 1 ? h->ws_misc.ptr : nullptr;
  if (which == 2) {
    // staged kernel: the caller's X and Y plus the internal direction vector
    c.err = reinterpret_cast<int*>(lb + 2 * kMaxW * sizeof(double)) + 4;
    r.c = c;
    SpmmStagedArgs T;
    T.g = h->lay;
    T.t = h->tiles;
    T.val = h->d_B32.as<float>();
    T.X = static_cast<const float*>(X);
    T.P = static_cast<float*>(P);
    T.Y = static_cast<float*>(Y);
    T.W = W;
    T.nq = nq;
    T.err = c.err;
    T.red = r;
    const unsigned smem = 2u * StageLayout(h->tiles).bytes;
    if (cudaFuncSetAttribute(k_spmm_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return GSK_ECUDA;
    for (int i = 0; i < n_rep; ++i) {
      k_spmm_staged<<<dim3(grid_t), dim3(kStagedThreads), smem, s>>>(T);
      if (cudaGetLastError() != cudaSuccess) return GSK_ECUDA;
    }
    int herr = 0;
    if (cudaMemcpyAsync(&herr, c.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return GSK_ECUDA;
#ifdef GSK_DEBUG
    {
      const int dr = dbg_collect(h, s);
      if (dr != GSK_OK) return dr;
    }
#endif
    return herr ? GSK_ETIMEOUT : GSK_OK;
  }
  for (int i = 0; i < n_rep; ++i) {
    if (precision == GSK_FP64) {
      SpmmArgs<double, double, double> a{h->lay, (which ? h->d_B64 : h->d_A64).as<double>(),
                                         static_cast<const double*>(X), static_cast<double*>(Y),
                                         nullptr, static_cast<double*>(P), nullptr, r};
      if (which == 1) {
        if (W == 32) k_spmm<double, double, double, double, 1, SP_CG><<<grd, blk, 0, s>>>(a);
        else k_spmm<double, double, double, double, 2, SP_CG><<<grd, blk, 0, s>>>(a);
      } else {
        if (W == 32) k_spmm<double, double, double, double, 1, SP_DOT><<<grd, blk, 0, s>>>(a);
        else k_spmm<double, double, double, double, 2, SP_DOT><<<grd, blk, 0, s>>>(a);
      }
    } else {
      SpmmArgs<float, float, float> a{h->lay, (which ? h->d_B32 : h->d_A32).as<float>(),
                                      static_cast<const float*>(X), static_cast<float*>(Y),
                                      nullptr, static_cast<float*>(P), nullptr, r};
      if (which == 1) {
        if (W == 32) k_spmm<float, float, float, float, 1, SP_CG><<<grd, blk, 0, s>>>(a);
        else if (W == 64) k_spmm<float, float, float, float, 2, SP_CG><<<grd, blk, 0, s>>>(a);
        else k_spmm<float, float, float, float, 4, SP_CG><<<grd, blk, 0, s>>>(a);
      } else {
        if (W == 32) k_spmm<float, float, float, float, 1, SP_DOT><<<grd, blk, 0, s>>>(a);
        else if (W == 64) k_spmm<float, float, float, float, 2, SP_DOT><<<grd, blk, 0, s>>>(a);
        else k_spmm<float, float, float, float, 4, SP_DOT><<<grd, blk, 0, s>>>(a);
      }
    }
    if (cudaGetLastError() != cudaSuccess) return GSK_ECUDA;
  }
#ifdef GSK_DEBUG
  return dbg_collect(h, s);     // the bounds-checked build waits here to report failed checks
#else
  return GSK_OK;
#endif
}

// Bytes of the reduction workspace that spmm64_dot needs (zero it once
// before the first call; its counters are reset by their last user).
size_t spmm64_ws_bytes(const gsk_ctx* h) {
  const int n_grp_max = (kMaxRedCtas + kRedGroup - 1) / kRedGroup;
  return 256 + (size_t)h->lay.n_ctas * kMaxW * sizeof(double) + (size_t)n_grp_max * kMaxW * sizeof(double) +
         n_grp_max * sizeof(unsigned) + 256;
}

// Y = S X on W = 32 or 64 FP64 lanes (S = A for which = 0, B for which = 1)
// with the per-lane dot X.Y written to dots[0..W) (device): the solver's
// block SpMM kernel in its plain-product form, for callers outside the
// shifted solve (the multiple Arnoldi path).
int spmm64_dot(gsk_ctx* h, int which, int W, const double* X, double* Y, double* dots, void* ws, cudaStream_t s) {
  if ((W != 32 && W != 64) || !X || !Y || !dots || !ws) return GSK_EINVAL;
  const int grid = h->lay.n_ctas;
  if (grid > kMaxRedCtas) return GSK_ENOTSUP;
  const int n_grp_max = (kMaxRedCtas + kRedGroup - 1) / kRedGroup;
  char* b = static_cast<char*>(ws);
  LaneCtl c{};
  c.red_out = dots;
  c.red_counter = reinterpret_cast<unsigned int*>(b);
  c.partials = reinterpret_cast<double*>(b + 256);
  c.grp_partials = c.partials + (size_t)grid * kMaxW;
  c.grp_counter = reinterpret_cast<unsigned int*>(c.grp_partials + (size_t)n_grp_max * kMaxW);
  RedArgs r{};
  r.c = c;
  r.fin = FIN_SUM;
  r.W = W;
  SpmmArgs<double, double, double> a{h->lay, (which ? h->d_B64 : h->d_A64).as<double>(), X, Y,
                                     nullptr, nullptr, nullptr, r};
  if (W == 32) k_spmm<double, double, double, double, 1, SP_DOT><<<grid, kThreads, 0, s>>>(a);
  else k_spmm<double, double, double, double, 2, SP_DOT><<<grid, kThreads, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? GSK_OK : GSK_ECUDA;
}

}  // namespace gsk

namespace gsk {

int autotune_impl(gsk_ctx* h, int32_t S, const double* z, const double* eta, int32_t n_cols, const int32_t* cols,
                  const gsk_options* opt_in, int32_t* best_w) {
  if (!best_w || n_cols < 1 || !cols) return GSK_EINVAL;
  gsk_options opt;
  gsk_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.precision < GSK_FP64 || opt.precision > GSK_MIXED_DF) return GSK_EINVAL;
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(opt.stream);
  TuneRecord& rec = h->tune[opt.precision];
  rec = TuneRecord{};
  // on-disk cache keyed by the pencil, the request and the GPU
  char key[512];
  {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) return GSK_ECUDA;
    for (char* c = prop.name; *c; ++c)
      if (*c == ' ' || *c == '\t') *c = '_';
    snprintf(key, sizeof(key), "M=%d nnz=%lld natoms=%d precision=%d shifts=%d cols=%d gpu=%s sms=%d", h->M,
             (long long)h->nnz, h->n_atoms, opt.precision, S, n_cols, prop.name, prop.multiProcessorCount);
  }
  const char* path = getenv("GSK_TUNE_CACHE");
  if (path && *path) {
    std::ifstream in(path);
    std::string line;
    while (std::getline(in, line)) {
      const size_t bar = line.find(" | ");
      if (bar == std::string::npos || line.compare(0, bar, key) != 0 || bar != strlen(key)) continue;
      int w = 0, k = 0;
      if (sscanf(line.c_str() + bar + 3, "W=%d kernel=%d", &w, &k) == 2 && (w == 32 || w == 64 || w == 128) &&
          (k == GSK_SPMM_GATHER || k == GSK_SPMM_STAGED) && !(k == GSK_SPMM_STAGED && h->tiles.n_tiles == 0)) {
        h->tuned_w[opt.precision] = w;
        h->tuned_kernel[opt.precision][w == 32 ? 0 : w == 64 ? 1 : 2] = k;
        rec.w = w;
        rec.kernel = k;
        rec.from_cache = 1;
        *best_w = w;
        return GSK_OK;
      }
    }
  }
  const int cands[3] = {32, 64, 128};
  const int n_cand = (opt.precision == GSK_FP64) ? 2 : 3;
  std::vector<int> kernels{GSK_SPMM_GATHER};
  if (opt.precision != GSK_FP64 && h->tiles.n_tiles > 0) kernels.push_back(GSK_SPMM_STAGED);
  double best = 1e300;
  int pick_w = 64, pick_k = GSK_SPMM_GATHER;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GSK_ECUDA;
  int rc = GSK_OK;
  for (int ci = 0; ci < n_cand && rc == GSK_OK; ++ci) {
    const int W = cands[ci];
    const int n = std::min(n_cols, W);
    // device buffer for the truncated solve's G
    int64_t elems = 0;
    for (int c = 0; c < n; ++c) elems += h->row_ptr[cols[c] + 1] - h->row_ptr[cols[c]];
    if (h->ws_tune.ensure((size_t)elems * S * 16 + 256) != cudaSuccess) {
      rc = GSK_ENOMEM;
      break;
    }
    double best_k = 1e300;
    for (int kern : kernels) {
      gsk_options o = opt;
      o.batch_w = W;
      o.spmm_kernel = kern;
      o.max_iter = 24;
      o.tol = 1e-30;
      o.sched = GSK_SCHED_FIFO;
      double ms_per_step = 0.0;
      for (int rep = 0; rep < 2 && rc == GSK_OK; ++rep) {     // the first run warms up
        cudaEventRecord(e0, s);
        rc = solve_impl(h, S, z, eta, n, cols, &o, h->ws_tune.as<double>(), nullptr, nullptr, nullptr);
        cudaEventRecord(e1, s);
        if (rc != GSK_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          rc = GSK_ECUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_per_step = ms / std::max<int64_t>(1, h->last.outer_steps);
      }
      if (rc != GSK_OK) break;
      // estimated time of the whole set in units of a column's mean step count;
      // the factor 2 covers the longest column of a set with mixed damping
      const double est = ms_per_step * std::max((double)n_cols / W, 2.0);
      if (rec.n_cand < (int)(sizeof(rec.cand_w) / sizeof(rec.cand_w[0]))) {
        rec.cand_w[rec.n_cand] = W;
        rec.cand_kernel[rec.n_cand] = kern;
        rec.cand_ms_per_step[rec.n_cand] = ms_per_step;
        rec.cand_estimate[rec.n_cand] = est;
        ++rec.n_cand;
      }
      if (est < best_k) {
        best_k = est;
        h->tuned_kernel[opt.precision][ci] = kern;
      }
      if (est < best) {
        best = est;
        pick_w = W;
        pick_k = kern;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GSK_OK) return rc;
  h->tuned_w[opt.precision] = pick_w;
  rec.w = pick_w;
  rec.kernel = pick_k;
  if (path && *path) {
    std::ofstream out(path, std::ios::app);
    if (out) out << key << " | W=" << pick_w << " kernel=" << pick_k << "\n";
  }
  *best_w = pick_w;
  return GSK_OK;
}

}  // namespace gsk

// ===========================================================================
// Self-test of the bounds-checked build's recording path
// ===========================================================================
namespace gsk {
#ifdef GSK_DEBUG
__global__ void k_dbg_selftest(int code, long long idx) {
  if (threadIdx.x == 0) (void)GSK_IDX_OK(false, code, idx);     // a check that fails, guarding no access
}
#endif
}  // namespace gsk

extern "C" int gsk_debug_selftest(int32_t* code, int64_t* index) {
  if (!code || !index) return GSK_EINVAL;
#ifdef GSK_DEBUG
  if (gsk::dbg_reset(0) != GSK_OK) return GSK_ECUDA;
  gsk::k_dbg_selftest<<<1, 32>>>(99, 12345678901LL);
  if (cudaGetLastError() != cudaSuccess) return GSK_ECUDA;
  int d[4] = {0, 0, 0, 0};
  if (cudaMemcpyFromSymbol(d, gsk::g_dbg, sizeof(d)) != cudaSuccess) return GSK_ECUDA;
  *code = d[0];
  *index = ((int64_t)d[2] << 32) | (int64_t)(uint32_t)d[1];
  return gsk::dbg_reset(0) == GSK_OK && cudaDeviceSynchronize() == cudaSuccess ? GSK_OK : GSK_ECUDA;
#else
  *code = 0;
  *index = 0;
  return GSK_ENOTSUP;
#endif
}
