// Shared device definitions of libgsk: block layout of the pencil, lane
// control block, vector load helpers and the deterministic two-level lane
// reduction used by every kernel that produces per-column inner products.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gsk.h"

namespace gsk {

constexpr int kThreads = 256;             // threads per CTA of the row kernels
constexpr int kWarps = kThreads / 32;
constexpr int kMaxW = 128;                // widest lane batch
constexpr int kMaxShifts = 1024;          // shifts per solve (shared-memory bound of the shift kernel)
constexpr int kRedGroup = 16;             // CTAs per first-level group of the grid reduction
constexpr int kMaxRedCtas = 4096;         // CTAs of a reducing kernel

// ---------------------------------------------------------------------------
// Block layout of A and B (identical pattern), atoms in the library's order.
// Atom I owns rows atom_roff[I] .. atom_roff[I] + atom_orb[I] - 1. Its
// neighbour entries nbr_ptr[I] .. nbr_ptr[I+1] list first the 4-orbital
// neighbours (up to nbr_mid[I]) then the 1-orbital ones; an entry stores the
// neighbour's first row. The values of atom I start at val_ptr[I] (a multiple
// of 4) and are, per 4-orbital neighbour, 4 columns of o_I values (column b
// holds rows a = 0..o_I-1), then per 1-orbital neighbour o_I values for a
// 4-orbital atom, or, for a 1-orbital atom, one value per neighbour with the
// 1-orbital neighbours padded to a multiple of 4 (padding: value 0, row of
// the atom itself).
// ---------------------------------------------------------------------------
struct Layout {
  int32_t n_atoms;
  int32_t M;
  int32_t chunk;                 // atoms per CTA in the row kernels
  int32_t n_ctas;                // CTAs of the row kernels
  const int32_t* atom_roff;      // n_atoms + 1
  const int8_t* atom_orb;        // n_atoms
  const int32_t* nbr_ptr;        // n_atoms + 1
  const int32_t* nbr_mid;        // n_atoms
  const int32_t* nbr_roff;       // neighbour entries
  const int64_t* val_ptr;        // n_atoms
  const int32_t* warp_atoms;     // n_ctas * kWarps + 1: atoms [warp_atoms[w], warp_atoms[w+1]) of warp w
#ifdef GSK_DEBUG
  int32_t n_nbr;                 // neighbour entries (the length of nbr_roff)
  int64_t n_vals;                // values of the block layout (the length of each value copy)
#endif
};

// Tiles of the staged SpMM (k_spmm_staged). Atoms are cut, in library order,
// into tiles of consecutive atoms; a tile's CTA copies into shared memory the
// rows of every neighbour atom of the tile (its row union, contiguous row
// runs cut into pieces of at most kPieceRows rows), the tile's matrix values, local
// neighbour indices and atom descriptors, and the tile's own rows of the CG
// direction and of B p. Each consumer warp then runs a fixed, cost-balanced
// list of the tile's atoms out of shared memory.
constexpr int kTileLanes = 32;         // lanes per CTA (a W-lane batch uses W / 32 CTAs per tile)
constexpr int kTileWarps = 12;         // consumer warps of the staged kernel (atom lists per tile)
constexpr int kPieceRows = 16;         // longest row-run piece (one copy of up to 2 KB per 32 lanes)
struct TileHead {                      // one per tile, 64 bytes
  int32_t r0;                          // first own row (library order)
  int32_t n_own;                       // own rows
  int32_t n_atoms;                     // atoms
  int32_t nbox;                        // row-run pieces of the row union
  int32_t b0;                          // first piece
  int32_t l0;                          // first local index (a multiple of 8)
  int32_t nloc;                        // local indices (a multiple of 8)
  int32_t d0;                          // first atom descriptor
  int64_t v0;                          // first matrix value (a multiple of 4)
  int32_t nval;                        // matrix values (a multiple of 4)
  int32_t xrows;                       // shared rows of the row union
  uint8_t wptr[16];                    // warp w runs descriptors [wptr[w], wptr[w+1]) (kTileWarps + 1 used)
};
static_assert(sizeof(TileHead) == 64, "TileHead is 64 bytes");
static_assert(kTileWarps < 16, "the warp lists of a tile fit its header");
// Atom descriptor (int4): x = orbitals | own row in the tile << 8 | shared
// row of the atom's first row << 16; y = 4-orbital neighbours | 1-orbital
// neighbour entries << 16; z = first value (from the tile's first);
// w = first local index (from the tile's first).
struct TileArgs {
  int32_t n_tiles;
  int32_t x_cap;                 // shared rows of the row union
  int32_t own_cap;               // shared rows of each own-row buffer (P, Y)
  int32_t v_cap;                 // shared matrix values (floats)
  int32_t l_cap;                 // shared local indices (int16)
  int32_t d_cap;                 // shared atom descriptors
  const TileHead* head;          // n_tiles
  const int2* box;               // row-run pieces: (first global row, first shared row | rows << 16)
  const int16_t* loc;            // shared row of each neighbour entry's first row, tile by tile
  const int4* desc;              // atom descriptors, tile by tile, in warp order
  const int32_t* order;          // library atom of each descriptor
#ifdef GSK_DEBUG
  int32_t n_box, n_loc, n_desc;  // lengths of box, loc and desc
  int64_t n_vals;                // length of the value copy the tiles index
#endif
};

// Lane states of the batched solver.
enum LaneState : int { LS_IDLE = 0, LS_SEED = 1, LS_ACTIVE = 2 };

// Finalisation applied by the last CTA of a reducing kernel to the per-lane sums.
enum Fin : int {
  FIN_ALPHA = 0,     // alpha_n = q.(A q)
  FIN_UNORM = 1,     // ||u||^2 -> unorm, start of a B-solve
  FIN_CG_A = 2,      // p.(B p) -> CG step length
  FIN_CG_RR = 3,     // r.r -> CG direction update, convergence
  FIN_RESID = 4,     // ||u - B v0||^2 -> start of the refinement B-solve
  FIN_BETA = 5,      // u.v -> beta_n, lane bookkeeping, refill from the queue
  FIN_SUM = 6,       // plain sums into red_out
};

// Per-lane control block in device memory (structure of arrays, kMaxW each)
// plus solve-wide counters. All fields are written only by the single last
// CTA of a reducing kernel, by the prime kernel, or by split 0 of the shift
// kernel, so no two writers race.
struct LaneCtl {
  int* job;            // job index of the lane, -1 when idle
  int* state;          // LaneState
  int* n;              // completed Lanczos steps of the current column
  int* done;           // set by the shift kernel when the column finished this step
  int* brk;            // breakdown seen (beta^2 <= 0, non-finite, inner solve failed)
  double* alpha;       // alpha_n of the current step
  double* beta_prev;   // beta_{n-1} (off-diagonal entering step n)
  double* beta0;       // ||b||_B of the seed
  double* unorm;       // ||u_n||_2
  double* inv_beta;    // scale applied by the finish kernel (0 zeroes the lane)
  double* rr;          // CG: current r.r
  double* rr_target;   // CG: stop when r.r <= rr_target
  double* cg_a;        // CG step length
  double* cg_b;        // CG direction coefficient
  int* cg_on;          // CG still iterating for this lane
  double* red_out;     // FIN_SUM results
  // solve-wide
  int* queue_head;     // next queue slot to hand out
  int* cg_iter;        // CG iterations of the current B-solve pass
  int* step;           // outer steps executed
  int* unfinished;     // lanes busy + jobs queued
  int* cg_total;       // total CG iterations (all passes), for statistics
  int* err;            // set by a kernel whose bounded wait gave up
  unsigned int* red_counter;   // arrival counter of the second reduction level
  unsigned int* grp_counter;   // arrival counters of the first level (kMaxRedCtas / kRedGroup)
  double* partials;            // per-CTA partial sums (CTA * W + lane)
  double* grp_partials;        // per-group partial sums (group * W + lane)
};

// Read-only description of the job list of one solve.
struct Jobs {
  int32_t n_jobs;
  const int32_t* queue;       // queue order -> job index
  const int32_t* col_row;     // job -> row (library order) of e_j
  const double* eta;          // job -> damping of its shifts
};

// Graph control: conditional handles set from device code (0 when the solve
// is driven from the host).
struct GraphCtl {
  int use_graph;
  cudaGraphConditionalHandle h_outer;
  cudaGraphConditionalHandle h_inner1;
  cudaGraphConditionalHandle h_inner2;
  int max_inner;
  int step_cap;
};

// ---------------------------------------------------------------------------
// Vector helpers: L consecutive lanes of one row.
// ---------------------------------------------------------------------------
template <typename T, int L>
struct LaneVec;
template <> struct LaneVec<float, 1> { using V = float; };
template <> struct LaneVec<float, 2> { using V = float2; };
template <> struct LaneVec<float, 4> { using V = float4; };
template <> struct LaneVec<double, 1> { using V = double; };
template <> struct LaneVec<double, 2> { using V = double2; };

template <typename T, int L>
__device__ __forceinline__ void ld_lanes(const T* __restrict__ p, T (&o)[L]) {
  if constexpr (L == 4 && sizeof(T) == 8) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  } else {
    using V = typename LaneVec<T, L>::V;
    const V v = *reinterpret_cast<const V*>(p);
    const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int i = 0; i < L; ++i) o[i] = e[i];
  }
}

template <typename T, int L>
__device__ __forceinline__ void st_lanes(T* __restrict__ p, const T (&o)[L]) {
  if constexpr (L == 4 && sizeof(T) == 8) {
    reinterpret_cast<double2*>(p)[0] = make_double2(o[0], o[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(o[2], o[3]);
  } else {
    using V = typename LaneVec<T, L>::V;
    V v;
    T* e = reinterpret_cast<T*>(&v);
#pragma unroll
    for (int i = 0; i < L; ++i) e[i] = o[i];
    *reinterpret_cast<V*>(p) = v;
  }
}

// Four consecutive matrix values (16-byte aligned for float, 32 for double).
template <typename T>
struct Quad { T x, y, z, w; };

__device__ __forceinline__ Quad<float> ld_quad(const float* __restrict__ p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Quad<double> ld_quad(const double* __restrict__ p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return {a.x, a.y, b.x, b.y};
}

// ---------------------------------------------------------------------------
// Complex helpers (double2 = re, im). Division by Smith's method
// (R. L. Smith, CACM 5(8), 1962), which avoids overflow of c^2 + d^2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x;
    const double den = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  } else {
    const double r = b.x / b.y;
    const double den = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
  }
}
__device__ __forceinline__ double cabs2(double2 a) { return hypot(a.x, a.y); }

// ---------------------------------------------------------------------------
// Per-lane reduction: every thread holds partial sums for its L lanes
// (lanes lane0 .. lane0+L-1). The CTA folds its warps in a fixed order and
// writes one partial per lane; the last CTA to arrive folds all partials in
// CTA order and applies the finalisation. Deterministic: the summation order
// never depends on timing.
// ---------------------------------------------------------------------------
struct RedArgs {
  LaneCtl c;
  Jobs jobs;
  GraphCtl gc;
  int fin;
  int W;
  double inner_tol2;     // squared relative tolerance of the B-solve pass
  int max_iter;
};

__device__ void finalize_lane(const RedArgs& r, int lane, double s);
__device__ void finalize_all(const RedArgs& r);

// Fixed-order sum over CTAs [b0, b1) of src[b * W + l] for every lane l, by
// all threads of the CTA (parts = blockDim / W partial sums per lane, four
// independent loads in flight per thread), folded into out[l] by thread l.
__device__ __forceinline__ double fold_rows(const double* __restrict__ src, int b0, int b1, int W,
                                            double (*sm)[kMaxW]) {
  const int parts = kThreads / W;
  const int l = threadIdx.x % W;
  const int pidx = threadIdx.x / W;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  const bool in = threadIdx.x < kThreads;      // threads beyond kThreads (producer warps) add nothing
  int b = in ? b0 + pidx : b1;
  for (; b + 3 * parts < b1; b += 4 * parts) {
    s0 += __ldcg(&src[(size_t)b * W + l]);
    s1 += __ldcg(&src[(size_t)(b + parts) * W + l]);
    s2 += __ldcg(&src[(size_t)(b + 2 * parts) * W + l]);
    s3 += __ldcg(&src[(size_t)(b + 3 * parts) * W + l]);
  }
  for (; b < b1; b += parts) s0 += __ldcg(&src[(size_t)b * W + l]);
  __syncthreads();
  if (in) sm[pidx][l] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < W)
    for (int p = 0; p < parts; ++p) t += sm[p][threadIdx.x];
  return t;
}

// Two-level deterministic reduction across the grid, from per-CTA sums:
// thread t < W holds this CTA's sum for lane t in s. Each CTA writes its
// per-lane partial; the last CTA to arrive in each group of kRedGroup CTAs
// folds the group (fixed order); the last group to arrive folds the group
// sums and runs the finalisation. Counters are reset by their last user.
// sm is the CTA's fold scratch (kWarps x kMaxW doubles).
__device__ __forceinline__ void cta_sums_commit(double s, const RedArgs& r, double (*sm)[kMaxW]) {
  __shared__ bool is_last;
  const int W = r.W;
  if (threadIdx.x < W) r.c.partials[(size_t)blockIdx.x * W + threadIdx.x] = s;
  __threadfence();
  __syncthreads();
  const int grp = blockIdx.x / kRedGroup;
  const int n_grp = (gridDim.x + kRedGroup - 1) / kRedGroup;
  const int g0 = grp * kRedGroup;
  const int g1 = min((int)gridDim.x, g0 + kRedGroup);
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&r.c.grp_counter[grp], 1u);
    is_last = (prev == (unsigned)(g1 - g0 - 1));
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const double gs = fold_rows(r.c.partials, g0, g1, W, sm);
  if (threadIdx.x < W) r.c.grp_partials[(size_t)grp * W + threadIdx.x] = gs;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    r.c.grp_counter[grp] = 0u;
    const unsigned prev = atomicAdd(r.c.red_counter, 1u);
    is_last = (prev == (unsigned)(n_grp - 1));
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const double t = fold_rows(r.c.grp_partials, 0, n_grp, W, sm);
  if (threadIdx.x < W) finalize_lane(r, threadIdx.x, t);
  __syncthreads();
  if (threadIdx.x == 0) {
    finalize_all(r);
    *r.c.red_counter = 0u;
  }
}

// Per-lane reduction of a CTA followed by the grid commit. mine[i] is this
// thread's partial for lane lane0 + i; within a warp the threads with
// writer = true cover every lane exactly once; warps are folded in order.
template <int L>
__device__ __forceinline__ void lane_reduce_commit_at(const double (&mine)[L], const RedArgs& r, int lane0,
                                                      bool writer) {
  __shared__ double sm[kWarps][kMaxW];
  const int W = r.W;
  const int warp = threadIdx.x >> 5;
  if (writer) {
#pragma unroll
    for (int i = 0; i < L; ++i) sm[warp][lane0 + i] = mine[i];
  }
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < W) {
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += sm[w][threadIdx.x];
  }
  __syncthreads();
  cta_sums_commit(s, r, sm);
}

template <int L>
__device__ __forceinline__ void lane_reduce_commit(const double (&mine)[L], const RedArgs& r) {
  lane_reduce_commit_at<L>(mine, r, (threadIdx.x & 31) * L, true);
}

}  // namespace gsk
