// Multiple Arnoldi projection on the GPU (Sec. III-B, Eq. EQ-LS-MULTIPLE,
// EQ-EIG-GREEN-KRYLOV and EQ-PROJ-PHYS-QUANT-KRYLOV), batched over columns.
//
// For a batch of up to 32 columns j the two Krylov sequences of A, from e_j
// and from B^-1 e_j, run side by side as 64 lanes of one Lanczos process
// (lane c: K(A; e_j), lane 32 + c: K(A; B^-1 e_j)) with full
// reorthogonalisation (classical Gram-Schmidt, two passes) on the solver's
// FP64 block SpMM. B^-1 e_j comes from a batched CG on B. The second sequence
// is then projected twice onto the orthogonal complement of the first and
// orthonormalised by its Gram matrix (eigenvalues = squared sines of the
// principal angles between the two subspaces; directions whose sine is below
// 1e-7 are dropped). The reduced pencil (Q^T A Q, Q^T B Q) is formed from
// explicit Gram matrices and solved per column (Cholesky of Q^T B Q, cyclic
// Jacobi on the symmetric reduced matrix, one warp per column), which gives the Ritz values eps_m
// and B-orthonormal Ritz vectors v_m = Q y_m. The outputs on the pattern P(j)
// are rho_ij = sum_m f(eps_m) (v_m)_i (v_m)_j and, for given shifts,
// G_ij(z_k) = sum_m (v_m)_i (v_m)_j / (z_k - eps_m).
//
// Vectors live in [M][64] arrays (row-major, lane fastest) in the library's
// row order, so the SpMM kernel applies to them unchanged. Every reduction is
// a fixed-order sum: per-CTA partials over fixed row chunks, folded in chunk
// order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "gsk_common.cuh"
#include "gsk_ctx.h"

namespace {

constexpr int kL = 64;                 // lane stride of the Lanczos arrays
constexpr int kC = 32;                 // columns per batch
constexpr int kMaxM = 16;              // vectors per Krylov sequence (nu <= 32)
constexpr int kMaxN = 2 * kMaxM;       // reduced dimension
constexpr int kLD = kMaxN + 1;         // leading dimension of shared-memory matrices
constexpr double kRankTol2 = 1e-14;    // drop squared sines of principal angles below this
constexpr double kBreakTol = 1e-13;    // Krylov breakdown relative to ||A||_inf
constexpr int kMaxSweeps = 40;         // Jacobi sweeps (convergence is quadratic; ~8 suffice)
constexpr int kCgMax = 2000;           // CG iterations for B^-1 e_j
constexpr int kCgCheck = 8;            // CG iterations between host convergence checks
// Padding value of the Ritz-value output: the IEEE 754 binary64 quiet NaN (all exponent bits and
// the top fraction bit set), built from its bit pattern so no library routine runs for it.
__device__ __forceinline__ double quiet_nan() { return __longlong_as_double(0x7ff8000000000000LL); }
#define kQuietNaN quiet_nan()

// A list of vectors: vector a is p[a][r * ld + off[a] + c] for row r, column c.
struct VecSet {
  const double* p[kMaxN];
  int off[kMaxN];
  int n;
  int ld;
};
struct VecSetW {
  double* p[kMaxN];
  int off[kMaxN];
  int n;
  int ld;
};

// ---------------------------------------------------------------------------
// Gram matrices: D[(a * ny + b) * C + c] = sum_r X_a[r, c] * Y_b[r, c]
// ---------------------------------------------------------------------------
constexpr int kGramCols = 4;       // columns per CTA
constexpr int kGramRows = 16;      // rows per shared-memory tile
constexpr int kGramThreads = 256;
constexpr int kGramAcc = 16;       // most accumulators per thread: kGramCols * nx * ny <= 4096

// Partial sums over one chunk of rows (blockIdx.x) for 4 columns (blockIdx.y):
// part[chunk][(a * ny + b) * C + c]. The CTA's n_ent = 4 nx ny entries are
// spread so that no FP64 instruction is issued for nothing: with ACC == 1,
// R = 256 / n_ent row groups of n_ent threads each take every R-th row of a
// tile (one entry per thread) and are folded in group order at the end;
// with ACC > 1 (n_ent > 256) every thread holds ACC entries over all rows.
template <int ACC>
__global__ void __launch_bounds__(kGramThreads) k_gram(VecSet X, VecSet Y, int M, int C, int rows_per_chunk,
                                                       double* __restrict__ part) {
  __shared__ double xs[kGramRows][kMaxN * kGramCols];
  __shared__ double ys[kGramRows][kMaxN * kGramCols];
  __shared__ double fold[kGramThreads];
  const int nx = X.n, ny = Y.n;
  const int c0 = blockIdx.y * kGramCols;
  const int r0 = blockIdx.x * rows_per_chunk;
  const int r1 = min(M, r0 + rows_per_chunk);
  const int n_ent = kGramCols * nx * ny;
  const int tid = threadIdx.x;
  const int R = ACC == 1 ? kGramThreads / n_ent : 1;       // row groups
  const int rg = ACC == 1 ? tid / n_ent : 0;               // this thread's row group
  const bool live = ACC == 1 ? rg < R : true;
  int xi[ACC], yi[ACC];
  bool on[ACC];
  double acc[ACC];
#pragma unroll
  for (int s = 0; s < ACC; ++s) {
    const int e = ACC == 1 ? tid % n_ent : tid + kGramThreads * s;
    on[s] = live && e < n_ent;
    const int b = e % ny, t = e / ny, a = t % nx, q = t / nx;
    xi[s] = on[s] ? a * kGramCols + q : 0;
    yi[s] = on[s] ? b * kGramCols + q : 0;
    acc[s] = 0.0;
  }
  const int nv = nx + ny;
  for (int rt = r0; rt < r1; rt += kGramRows) {
    const int nr = min(kGramRows, r1 - rt);
    __syncthreads();
    for (int it = tid; it < kGramRows * nv * kGramCols; it += kGramThreads) {
      const int q = it % kGramCols;
      const int v = (it / kGramCols) % nv;
      const int i = it / (kGramCols * nv);
      double val = 0.0;
      if (i < nr && c0 + q < C) {
        const size_t row = (size_t)(rt + i);
        val = v < nx ? X.p[v][row * X.ld + X.off[v] + c0 + q] : Y.p[v - nx][row * Y.ld + Y.off[v - nx] + c0 + q];
      }
      if (v < nx) xs[i][v * kGramCols + q] = val;
      else ys[i][(v - nx) * kGramCols + q] = val;
    }
    __syncthreads();
    if (live) {
      for (int i = rg; i < nr; i += R) {
#pragma unroll
        for (int s = 0; s < ACC; ++s)
          if (on[s]) acc[s] = fma(xs[i][xi[s]], ys[i][yi[s]], acc[s]);
      }
    }
  }
  const size_t base = (size_t)blockIdx.x * nx * ny * C;
  if constexpr (ACC == 1) {
    // fold the row groups of each entry in group order
    __syncthreads();
    fold[tid] = live && on[0] ? acc[0] : 0.0;
    __syncthreads();
    if (tid < n_ent) {
      double t = 0.0;
      for (int g = 0; g < R; ++g) t += fold[g * n_ent + tid];
      const int e = tid;
      const int b = e % ny, tt = e / ny, a = tt % nx, q = tt / nx;
      if (c0 + q < C) part[base + (size_t)(a * ny + b) * C + c0 + q] = t;
    }
  } else {
#pragma unroll
    for (int s = 0; s < ACC; ++s) {
      const int e = tid + kGramThreads * s;
      if (e < n_ent) {
        const int b = e % ny, t = e / ny, a = t % nx, q = t / nx;
        if (c0 + q < C) part[base + (size_t)(a * ny + b) * C + c0 + q] = acc[s];
      }
    }
  }
}

// D[idx] = sum over chunks, in chunk order, of part[chunk][idx].
__global__ void k_gram_fold(int n_chunks, int n_out, const double* __restrict__ part, double* __restrict__ D) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n_out; idx += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int ch = 0; ch < n_chunks; ++ch) s += part[(size_t)ch * n_out + idx];
    D[idx] = s;
  }
}

// Z_b[r, c] = beta * Y_b[r, c] + gamma * sum_a X_a[r, c] * K[(a * nz + b) * C + c],
// for nx <= NX. One thread per (row, column); it reads every X_a of its
// element before it writes, so Z may alias X or Y element for element.
template <int NX>
__global__ void __launch_bounds__(256) k_combine(VecSet X, VecSet Y, VecSetW Z, const double* __restrict__ K,
                                                 int C, int M, double beta, double gamma) {
  const int64_t total = (int64_t)M * C;
  const int nx = X.n, nz = Z.n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % C);
    const size_t r = (size_t)(t / C);
    double x[NX];
#pragma unroll
    for (int a = 0; a < NX; ++a) x[a] = a < nx ? X.p[a][r * X.ld + X.off[a] + c] : 0.0;
    for (int b = 0; b < nz; ++b) {
      double s = 0.0;
#pragma unroll
      for (int a = 0; a < NX; ++a)
        if (a < nx) s = fma(x[a], K[(size_t)(a * nz + b) * C + c], s);
      double v = gamma * s;
      if (beta != 0.0) v = fma(beta, Y.p[b][r * Y.ld + Y.off[b] + c], v);
      Z.p[b][r * Z.ld + Z.off[b] + c] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// CG on B for B^-1 e_j, 32 lanes in [M][32] arrays
// ---------------------------------------------------------------------------
__global__ void k_cg_seed(int nb, const int32_t* __restrict__ jrow, double* r, double* p, double* u0) {
  const int c = threadIdx.x;
  if (c < nb) {
    r[(size_t)jrow[c] * kC + c] = 1.0;
    p[(size_t)jrow[c] * kC + c] = 1.0;
    u0[(size_t)jrow[c] * kL + c] = 1.0;
  }
}

// x += a p, r -= a q with a = rr / pq on active lanes.
__global__ void k_cg_xr(int M, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                        const double* __restrict__ q, const double* __restrict__ rr, const double* __restrict__ pq,
                        const int* __restrict__ active) {
  const int64_t total = (int64_t)M * kC;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % kC);
    if (!active[c]) continue;
    const double a = rr[c] / pq[c];
    x[t] = fma(a, p[t], x[t]);
    r[t] = fma(-a, q[t], r[t]);
  }
}

// p = r + b p on active lanes.
__global__ void k_cg_p(int M, double* __restrict__ p, const double* __restrict__ r, const double* __restrict__ bta,
                       const int* __restrict__ active) {
  const int64_t total = (int64_t)M * kC;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % kC);
    if (active[c]) p[t] = fma(bta[c], p[t], r[t]);
  }
}

// Per lane: b = rr_new / rr, rr = rr_new, stop at rr_new <= tol2 (or a
// non-positive curvature p.Bp); n_active = number of lanes still iterating.
__global__ void k_cg_lane(double* rr, const double* __restrict__ rr_new, const double* __restrict__ pq,
                          double* bta, int* active, double tol2, int* n_active) {
  const int c = threadIdx.x;
  int on = 0;
  if (c < kC) {
    if (active[c]) {
      const double rn = rr_new[c];
      if (!(pq[c] > 0.0) || !isfinite(rn)) {
        active[c] = 0;
      } else {
        bta[c] = rn / rr[c];
        rr[c] = rn;
        if (rn <= tol2) active[c] = 0;
      }
    }
    on = active[c];
  }
  on = __reduce_add_sync(0xffffffffu, on);
  if (c == 0) *n_active = on;
}

// K[c] = 1 / ||x_c|| (0 for a zero vector): the scale that seeds the second sequence.
__global__ void k_inv_norm(const double* __restrict__ n2, double* __restrict__ K, int C) {
  const int c = threadIdx.x;
  if (c < C) K[c] = n2[c] > 0.0 ? 1.0 / sqrt(n2[c]) : 0.0;
}

// ---------------------------------------------------------------------------
// Lanczos lane scalars
// ---------------------------------------------------------------------------
// K3 = [-alpha, -beta_prev] per lane: w = A u_k - alpha u_k - beta_prev u_{k-1}.
__global__ void k_coef3(const double* __restrict__ alpha, const double* __restrict__ beta_prev, double* K3) {
  const int l = threadIdx.x;
  if (l < kL) {
    K3[l] = -alpha[l];
    K3[kL + l] = -beta_prev[l];
  }
}

// beta_k = ||w||; a lane that is below the breakdown level (or already ended)
// stops: its next vector is zero. Otherwise inv = 1 / beta_k and the lane's
// keep bit for vector k + 1 is set.
__global__ void k_lanczos_lane(int k, const double* __restrict__ n2, double scale, double* beta_prev,
                               double* inv, unsigned* keep) {
  const int l = threadIdx.x;
  if (l >= kL) return;
  const double b = sqrt(fmax(n2[l], 0.0));
  const bool alive = (keep[l] >> k) & 1u;
  if (alive && b > kBreakTol * scale && isfinite(b)) {
    inv[l] = 1.0 / b;
    beta_prev[l] = b;
    keep[l] |= 1u << (k + 1);
  } else {
    inv[l] = 0.0;
    beta_prev[l] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Small dense eigenproblems in shared memory: one warp per column, n <= 32,
// lane x owns index x of every row or column operation; ordering between the
// steps is by __syncwarp only.
// ---------------------------------------------------------------------------
// Sum over the warp in a fixed order (tree on lane 0, then broadcast), so every
// lane holds the same value.
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

// Cyclic Jacobi (row-by-row pair order): each rotation J(p, q) zeroing H[p][q]
// is computed by every lane from the same three entries and applied as
// H <- J^T H J (rows p, q, then columns p, q) and Z <- Z J, lane x taking
// element x; an off-diagonal below 1e-17 sqrt|H_pp H_qq| is set to zero
// instead (threshold Jacobi). Sweeps stop when the off-diagonal mass is below
// 1e-30 of the total, or after kMaxSweeps.
__device__ void warp_jacobi(double (*H)[kLD], double (*Z)[kLD], int n) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < n; ++i)
    if (lane < n) Z[i][lane] = (i == lane) ? 1.0 : 0.0;
  __syncwarp();
  if (n <= 1) return;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    if (lane < n)
      for (int i = 0; i < n; ++i) {
        const double v = H[i][lane];
        tot += v * v;
        if (i != lane) off += v * v;
      }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if (!(off > 1e-30 * tot)) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = H[p][q];               // the same values in every lane
        const double app = H[p][p], aqq = H[q][q];
        if (apq == 0.0) continue;
        if (fabs(apq) <= 1e-17 * sqrt(fabs(app * aqq))) {
          // negligible: setting it to zero moves the eigenvalues by O(apq^2 / gap)
          __syncwarp();
          if (lane == 0) {
            H[p][q] = 0.0;
            H[q][p] = 0.0;
          }
          __syncwarp();
          continue;
        }
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = fabs(tau) > 1e150 ? 0.5 / tau
                                            : (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        __syncwarp();
        if (lane < n) {
          const double hp = H[p][lane], hq = H[q][lane];
          H[p][lane] = c * hp - s * hq;
          H[q][lane] = s * hp + c * hq;
        }
        __syncwarp();
        if (lane < n) {
          const double hp = H[lane][p], hq = H[lane][q];
          H[lane][p] = c * hp - s * hq;
          H[lane][q] = s * hp + c * hq;
          const double zp = Z[lane][p], zq = Z[lane][q];
          Z[lane][p] = c * zp - s * zq;
          Z[lane][q] = s * zp + c * zq;
        }
        __syncwarp();
      }
    }
  }
}

// Orthonormalisation of the projected second sequence by its Gram matrix
// G = U2^T U2 (m x m per column): G = Z diag(lambda) Z^T, the kept directions
// (lambda >= kRankTol2) give T[:, i] = Z[:, i] / sqrt(lambda_i), the others a
// zero column; keep2 gets one bit per kept direction. One warp per column.
__global__ void __launch_bounds__(32) k_svqb(int m, const double* __restrict__ G, double* __restrict__ T,
                                             unsigned* __restrict__ keep2) {
  __shared__ double H[kMaxN][kLD], Z[kMaxN][kLD];
  const int c = blockIdx.x, lane = threadIdx.x;
  for (int a = 0; a < m; ++a)
    if (lane < m) H[a][lane] = 0.5 * (G[(size_t)(a * m + lane) * kC + c] + G[(size_t)(lane * m + a) * kC + c]);
  __syncwarp();
  warp_jacobi(H, Z, m);
  __syncwarp();
  for (int a = 0; a < m; ++a)
    if (lane < m) {
      const double lam = H[lane][lane];
      T[(size_t)(a * m + lane) * kC + c] = lam >= kRankTol2 ? Z[a][lane] / sqrt(lam) : 0.0;
    }
  const unsigned bits = __ballot_sync(0xffffffffu, lane < m && H[lane < m ? lane : 0][lane < m ? lane : 0] >= kRankTol2);
  if (lane == 0) keep2[c] = bits;
}

// Per-column outputs of the reduced solve.
struct ReducedOut {
  double* eps;      // [c][kMaxN]: Ritz values ascending, NaN beyond the rank
  double* w;        // [c][kMaxN]: (v_m)_j^2
  double* q;        // [c][kMaxN]: (v_m)_j (B v_m)_j
  double* y;        // [c][kMaxN]: (v_m)_j
  double* Y;        // [c][kMaxN][kMaxN]: Ritz coefficients, row a (full index), column m
  double* t;        // [c][kMaxN]: sum_m Y[a][m] f(eps_m) (v_m)_j
  int* rank;        // [c]
  int* status;      // [c]: 0 ok, 1 Q^T B Q not positive definite
};

// Reduced pencil of column c (one warp): At, Bt (n x n, n = 2m, layout
// [(a*n+b)*kC + c]) on the kept indices (keep1: first sequence, lane c;
// keep2: second). Cholesky Bt = L L^T, H = L^-1 At L^-T, Jacobi H = Z D Z^T,
// Ritz coefficients Y = L^-T Z, eigenpairs sorted by ascending value.
__global__ void __launch_bounds__(32) k_reduced(int m, const double* __restrict__ At, const double* __restrict__ Bt,
                                                const unsigned* __restrict__ keep1, const unsigned* __restrict__ keep2,
                                                const double* const* __restrict__ U, const double* const* __restrict__ BQ,
                                                const int32_t* __restrict__ jrow, int nb, double mu, double kT,
                                                ReducedOut out) {
  __shared__ double Am[kMaxN][kLD], Lm[kMaxN][kLD], H[kMaxN][kLD], Z[kMaxN][kLD];
  __shared__ double eps[kMaxN], yv[kMaxN], bv[kMaxN], fv[kMaxN], qj[kMaxN], bj[kMaxN];
  __shared__ int kidx[kMaxN], rk[kMaxN];
  const int c = blockIdx.x, lane = threadIdx.x;
  const int n = 2 * m;
  if (c >= nb) return;
  // kept indices in ascending order: lane a < n is kept or not, prefix count by ballot
  const bool kept = lane < n && (lane < m ? ((keep1[c] >> lane) & 1u) : ((keep2[c] >> (lane - m)) & 1u));
  const unsigned kb = __ballot_sync(0xffffffffu, kept);
  const int r = __popc(kb);
  if (kept) kidx[__popc(kb & ((1u << lane) - 1u))] = lane;
  __syncwarp();
  for (int i = 0; i < r; ++i)
    if (lane < r) {
      const int a = kidx[i], b = kidx[lane];
      Am[i][lane] = 0.5 * (At[(size_t)(a * n + b) * kC + c] + At[(size_t)(b * n + a) * kC + c]);
      H[i][lane] = 0.5 * (Bt[(size_t)(a * n + b) * kC + c] + Bt[(size_t)(b * n + a) * kC + c]);
    }
  if (lane < r) {
    const int a = kidx[lane];
    const size_t e = (size_t)jrow[c] * kL + (a < m ? c : kC + c);
    qj[lane] = U[a % m][e];
    bj[lane] = BQ[a % m][e];
  }
  __syncwarp();
  // Cholesky of the kept block of Q^T B Q (in H), lower factor in Lm
  int fail = 0;
  for (int k = 0; k < r; ++k) {
    double v = H[k][k];
    for (int i = 0; i < k; ++i) v -= Lm[k][i] * Lm[k][i];
    if (!(v > 0.0)) {
      fail = 1;
      v = 1.0;
    }
    const double lkk = sqrt(v);                    // every lane computes the same pivot
    __syncwarp();
    if (lane == k) Lm[k][k] = lkk;
    if (lane > k && lane < r) {
      double w = H[lane][k];
      for (int jj = 0; jj < k; ++jj) w -= Lm[lane][jj] * Lm[k][jj];
      Lm[lane][k] = w / lkk;
    }
    __syncwarp();
  }
  // W = L^-1 At (into Z; lane = column), then H = L^-1 W^T (lane = row of H)
  if (lane < r)
    for (int i = 0; i < r; ++i) {
      double v = Am[i][lane];
      for (int k = 0; k < i; ++k) v -= Lm[i][k] * Z[k][lane];
      Z[i][lane] = v / Lm[i][i];
    }
  __syncwarp();
  if (lane < r)
    for (int i = 0; i < r; ++i) {
      double v = Z[lane][i];
      for (int k = 0; k < i; ++k) v -= Lm[i][k] * H[lane][k];
      H[lane][i] = v / Lm[i][i];
    }
  __syncwarp();
  for (int a = 0; a < r; ++a)
    if (lane < r && a < lane) {
      const double v = 0.5 * (H[a][lane] + H[lane][a]);
      H[a][lane] = v;
      H[lane][a] = v;
    }
  __syncwarp();
  warp_jacobi(H, Z, r);
  __syncwarp();
  // Y = L^-T Z (into Am; lane = column), rank of each eigenvalue
  if (lane < r) {
    for (int i = r - 1; i >= 0; --i) {
      double v = Z[i][lane];
      for (int k = i + 1; k < r; ++k) v -= Lm[k][i] * Am[k][lane];
      Am[i][lane] = v / Lm[i][i];
    }
    const double d = H[lane][lane];
    int k = 0;
    for (int jj = 0; jj < r; ++jj) {
      const double e = H[jj][jj];
      k += (e < d) || (e == d && jj < lane);
    }
    rk[lane] = k;
  }
  __syncwarp();
  if (lane < r) {
    const int s = rk[lane];
    eps[s] = H[lane][lane];
    double yy = 0.0, bb = 0.0;
    for (int a = 0; a < r; ++a) {
      yy = fma(qj[a], Am[a][lane], yy);
      bb = fma(bj[a], Am[a][lane], bb);
    }
    yv[s] = yy;
    bv[s] = bb;
    const double x = (H[lane][lane] - mu) / kT;
    const double ex = exp(-fabs(x));
    fv[s] = (x > 0.0) ? ex / (1.0 + ex) : 1.0 / (1.0 + ex);
  }
  __syncwarp();
  const size_t cb = (size_t)c * kMaxN;
  {
    const bool ok = lane < r;
    out.eps[cb + lane] = ok ? eps[lane] : kQuietNaN;
    out.w[cb + lane] = ok ? yv[lane] * yv[lane] : 0.0;
    out.q[cb + lane] = ok ? yv[lane] * bv[lane] : 0.0;
    out.y[cb + lane] = ok ? yv[lane] : 0.0;
  }
  // Y in the full index space (rows a = kidx[i]), columns in sorted order
  for (int a = 0; a < kMaxN; ++a) out.Y[(cb + a) * kMaxN + lane] = 0.0;
  __syncwarp();
  if (lane < r)
    for (int i = 0; i < r; ++i) out.Y[(cb + kidx[i]) * kMaxN + rk[lane]] = Am[i][lane];
  double tv = 0.0;
  if (lane < r)
    for (int col = 0; col < r; ++col) tv = fma(Am[lane][col], fv[rk[col]] * yv[rk[col]], tv);
  out.t[cb + lane] = 0.0;
  __syncwarp();
  if (lane < r) out.t[cb + kidx[lane]] = tv;
  if (lane == 0) {
    out.rank[c] = r;
    out.status[c] = fail;
  }
}

// rho and G on the pattern: one CTA per column, one warp per pattern entry.
// Lane a holds Q_a(i); rho_i = sum_a Q_a(i) t_a; lane m forms
// u_m = (v_m)_i (v_m)_j; G_ik = sum_m u_m / (z_k - eps_m).
constexpr int kOutShiftChunk = 64;
__global__ void __launch_bounds__(256) k_ma_output(int m, const double* const* __restrict__ U,
                                                   const int32_t* __restrict__ prow, const int64_t* __restrict__ poff,
                                                   ReducedOut ro, int S, const double2* __restrict__ z,
                                                   double* __restrict__ rho, double2* __restrict__ G) {
  __shared__ double Ys[kMaxN][kMaxN + 1];
  __shared__ double ts[kMaxN], ys[kMaxN], es[kMaxN];
  __shared__ double2 inv[kOutShiftChunk][kMaxN + 1];
  __shared__ double us[8][kMaxN];
  const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = 2 * m;
  const size_t cb = (size_t)c * kMaxN;
  const int r = ro.rank[c];
  for (int i = tid; i < kMaxN * kMaxN; i += blockDim.x) Ys[i / kMaxN][i % kMaxN] = ro.Y[cb * kMaxN + i];
  for (int i = tid; i < kMaxN; i += blockDim.x) {
    ts[i] = ro.t[cb + i];
    ys[i] = ro.y[cb + i];
    es[i] = i < r ? ro.eps[cb + i] : 0.0;
  }
  __syncthreads();
  const int64_t e0 = poff[c], e1 = poff[c + 1];
  const int n_chunks = (G && S > 0) ? (S + kOutShiftChunk - 1) / kOutShiftChunk : 0;
  // rho, and u_m per entry kept in a register for the G pass below
  for (int64_t e = e0 + warp; e < e1; e += blockDim.x >> 5) {
    const size_t row = (size_t)prow[e];
    const double qa = lane < n ? U[lane % m][row * kL + (lane < m ? c : kC + c)] : 0.0;
    double s = qa * (lane < kMaxN ? ts[lane] : 0.0);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rho[e] = s;
  }
  for (int ch = 0; ch < n_chunks; ++ch) {
    const int k0 = ch * kOutShiftChunk, nk = min(kOutShiftChunk, S - k0);
    __syncthreads();
    for (int i = tid; i < nk * kMaxN; i += blockDim.x) {
      const int k = i / kMaxN, mm = i % kMaxN;
      inv[k][mm] = mm < r ? gsk::cdiv(make_double2(1.0, 0.0), make_double2(z[k0 + k].x - es[mm], z[k0 + k].y))
                          : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int64_t e = e0 + warp; e < e1; e += blockDim.x >> 5) {
      const size_t row = (size_t)prow[e];
      const double qa = lane < n ? U[lane % m][row * kL + (lane < m ? c : kC + c)] : 0.0;
      double v = 0.0;                                   // (v_m)_i for m = lane
      for (int a = 0; a < n; ++a) v = fma(__shfl_sync(0xffffffffu, qa, a), Ys[a][lane], v);
      us[warp][lane] = lane < r ? v * ys[lane] : 0.0;
      __syncwarp();
      for (int k = lane; k < nk; k += 32) {
        double gr = 0.0, gi = 0.0;
        for (int mm = 0; mm < r; ++mm) {
          const double um = us[warp][mm];
          gr = fma(um, inv[k][mm].x, gr);
          gi = fma(um, inv[k][mm].y, gi);
        }
        G[(size_t)e * S + k0 + k] = make_double2(gr, gi);
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Ws {
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  T* take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
    return p;
  }
};

VecSet make_set(const std::vector<const double*>& p, const std::vector<int>& off, int ld) {
  VecSet s{};
  s.n = (int)p.size();
  s.ld = ld;
  for (int i = 0; i < s.n; ++i) {
    s.p[i] = p[i];
    s.off[i] = off[i];
  }
  return s;
}
VecSetW make_setw(const std::vector<double*>& p, const std::vector<int>& off, int ld) {
  VecSetW s{};
  s.n = (int)p.size();
  s.ld = ld;
  for (int i = 0; i < s.n; ++i) {
    s.p[i] = p[i];
    s.off[i] = off[i];
  }
  return s;
}

struct Runner {
  gsk_ctx* h;
  int M;
  int grid_vec;
  double* part;       // Gram partials
  size_t part_cap;    // doubles
  bool ok = true;

  void gram(const VecSet& X, const VecSet& Y, int C, double* D) {
    const int groups = (C + kGramCols - 1) / kGramCols;
    int chunks = std::max(1, (h->num_sms * 4) / groups);
    const size_t n_out = (size_t)X.n * Y.n * C;
    chunks = (int)std::min<size_t>(chunks, part_cap / std::max<size_t>(n_out, 1));
    chunks = std::max(1, std::min(chunks, (M + kGramRows - 1) / kGramRows));
    const int rows = (M + chunks - 1) / chunks;
    chunks = (M + rows - 1) / rows;
    const int n_ent = kGramCols * X.n * Y.n;
    if (n_ent > kGramAcc * kGramThreads) {                // more entries than the widest variant holds
      ok = false;
      return;
    }
    const dim3 grid(chunks, groups);
    if (n_ent <= kGramThreads) k_gram<1><<<grid, kGramThreads>>>(X, Y, M, C, rows, part);
    else if (n_ent <= 2 * kGramThreads) k_gram<2><<<grid, kGramThreads>>>(X, Y, M, C, rows, part);
    else if (n_ent <= 4 * kGramThreads) k_gram<4><<<grid, kGramThreads>>>(X, Y, M, C, rows, part);
    else if (n_ent <= 8 * kGramThreads) k_gram<8><<<grid, kGramThreads>>>(X, Y, M, C, rows, part);
    else k_gram<16><<<grid, kGramThreads>>>(X, Y, M, C, rows, part);
    const int fb = (int)std::min<size_t>((n_out + 255) / 256, 1024);
    k_gram_fold<<<std::max(fb, 1), 256>>>(chunks, (int)n_out, part, D);
    ok = ok && cudaGetLastError() == cudaSuccess;
  }
  void combine(const VecSet& X, const VecSet& Y, const VecSetW& Z, const double* K, int C, double beta,
               double gamma) {
    if (X.n <= 1) k_combine<1><<<grid_vec, 256>>>(X, Y, Z, K, C, M, beta, gamma);
    else if (X.n <= 2) k_combine<2><<<grid_vec, 256>>>(X, Y, Z, K, C, M, beta, gamma);
    else if (X.n <= 4) k_combine<4><<<grid_vec, 256>>>(X, Y, Z, K, C, M, beta, gamma);
    else if (X.n <= 8) k_combine<8><<<grid_vec, 256>>>(X, Y, Z, K, C, M, beta, gamma);
    else if (X.n <= 16) k_combine<16><<<grid_vec, 256>>>(X, Y, Z, K, C, M, beta, gamma);
    else k_combine<kMaxN><<<grid_vec, 256>>>(X, Y, Z, K, C, M, beta, gamma);
    ok = ok && cudaGetLastError() == cudaSuccess;
  }
};

}  // namespace

extern "C" {

int gsk_marnoldi(gsk_handle h, int32_t n_cols, const int32_t* cols, int32_t nu, double mu, double kT,
                 double* rho, int32_t n_shifts, const double* z, double* G, double* ritz, double* weight,
                 double* charge, int32_t* rank) {
  if (!h || n_cols < 0 || (n_cols > 0 && (!cols || !rho))) return GSK_EINVAL;
  if (nu < 2 || nu > kMaxN || (nu & 1)) return GSK_EINVAL;
  if (!(kT > 0.0) || !isfinite(kT) || !isfinite(mu)) return GSK_EINVAL;
  if (n_shifts < 0 || (n_shifts > 0 && (!z || !G))) return GSK_EINVAL;
  for (int32_t c = 0; c < n_cols; ++c)
    if (cols[c] < 0 || cols[c] >= h->M) return GSK_EINVAL;
  for (int32_t k = 0; k < 2 * n_shifts; ++k)
    if (!isfinite(z[k])) return GSK_EINVAL;
  if (n_cols == 0) return GSK_OK;
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  const int m = nu / 2;
  const int M = h->M;
  // ||A||_inf for the breakdown test
  double scale = 0.0;
  for (int32_t i = 0; i < M; ++i) scale = std::max(scale, fabs(h->a_diag[i]) + h->a_rowabs[i]);
  scale = std::max(scale, 1e-300);

  // ---- workspace ----
  const size_t vec64 = (size_t)M * kL, vec32 = (size_t)M * kC;
  const size_t part_cap = (size_t)std::max(h->num_sms * 4, 64) * kC * kMaxN * kMaxN / 2;
  size_t max_pat = 0;
  {
    for (int32_t c0 = 0; c0 < n_cols; c0 += kC) {
      size_t s = 0;
      for (int32_t c = c0; c < std::min(n_cols, c0 + kC); ++c) s += h->row_ptr[cols[c] + 1] - h->row_ptr[cols[c]];
      max_pat = std::max(max_pat, s);
    }
  }
  const size_t need = 256 * 64 + (3 * (size_t)m + 1) * vec64 * sizeof(double) + 4 * vec32 * sizeof(double) +
                      part_cap * sizeof(double) + 8 * (size_t)kMaxN * kMaxN * kL * sizeof(double) +
                      gsk::spmm64_ws_bytes(h) + max_pat * (sizeof(int32_t) + 8) + (size_t)n_shifts * 16 +
                      64 * 1024;
  if (h->ws_ma.ensure(need) != cudaSuccess) return GSK_ENOMEM;
  Ws w{h->ws_ma.as<char>(), 0};
  std::vector<double*> U(m), AU(m), BQ(m);
  for (int a = 0; a < m; ++a) U[a] = w.take<double>(vec64);
  for (int a = 0; a < m; ++a) AU[a] = w.take<double>(vec64);
  for (int a = 0; a < m; ++a) BQ[a] = w.take<double>(vec64);
  double* Wv = w.take<double>(vec64);
  double* cx = w.take<double>(vec32);
  double* cr = w.take<double>(vec32);
  double* cp = w.take<double>(vec32);
  double* cq = w.take<double>(vec32);
  double* part = w.take<double>(part_cap);
  double* K1 = w.take<double>((size_t)kMaxN * kMaxN * kL);     // Gram / coefficient matrices
  double* K2 = w.take<double>((size_t)kMaxN * kMaxN * kL);
  double* At = w.take<double>((size_t)kMaxN * kMaxN * kC);
  double* Bt = w.take<double>((size_t)kMaxN * kMaxN * kC);
  double* lane = w.take<double>(16 * kL);                       // per-lane scalars
  double* alpha = lane, *beta_prev = lane + kL, *inv = lane + 2 * kL, *n2 = lane + 3 * kL;
  double* rr = lane + 4 * kL, *rr_new = lane + 5 * kL, *pq = lane + 6 * kL, *bta = lane + 7 * kL;
  int* iscr = w.take<int>(4 * kL);
  int* active = iscr, *n_active = iscr + kL;
  unsigned* keep1 = w.take<unsigned>(kL);
  unsigned* keep2 = w.take<unsigned>(kL);
  int32_t* d_jrow = w.take<int32_t>(kC);
  const double** d_U = w.take<const double*>(kMaxM);
  const double** d_BQ = w.take<const double*>(kMaxM);
  ReducedOut ro{};
  ro.eps = w.take<double>((size_t)kC * kMaxN);
  ro.w = w.take<double>((size_t)kC * kMaxN);
  ro.q = w.take<double>((size_t)kC * kMaxN);
  ro.y = w.take<double>((size_t)kC * kMaxN);
  ro.Y = w.take<double>((size_t)kC * kMaxN * kMaxN);
  ro.t = w.take<double>((size_t)kC * kMaxN);
  ro.rank = w.take<int>(kC);
  ro.status = w.take<int>(kC);
  void* sws = w.take<char>(gsk::spmm64_ws_bytes(h));
  int32_t* d_prow = w.take<int32_t>(std::max<size_t>(max_pat, 1));
  int64_t* d_poff = w.take<int64_t>(kC + 1);
  double2* d_z = w.take<double2>(std::max(n_shifts, 1));
  if (w.off > h->ws_ma.bytes) return GSK_ENOMEM;

  cudaError_t ce = cudaMemset(sws, 0, gsk::spmm64_ws_bytes(h));
  if (ce == cudaSuccess) ce = cudaMemcpy(d_U, U.data(), m * sizeof(double*), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(d_BQ, BQ.data(), m * sizeof(double*), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess && n_shifts > 0) ce = cudaMemcpy(d_z, z, (size_t)n_shifts * 16, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) return GSK_ECUDA;

  Runner R{h, M, std::max(1, h->num_sms * 8), part, part_cap};
  std::vector<int64_t> pat_off(n_cols + 1, 0);
  for (int32_t c = 0; c < n_cols; ++c) pat_off[c + 1] = pat_off[c] + (h->row_ptr[cols[c] + 1] - h->row_ptr[cols[c]]);

  int rc = GSK_OK;
  for (int32_t c0 = 0; c0 < n_cols && rc == GSK_OK; c0 += kC) {
    const int nb = std::min<int>(kC, n_cols - c0);
    // rows of e_j and of the patterns (library order), pattern offsets of the batch
    std::vector<int32_t> jrow(kC, 0), prow;
    std::vector<int64_t> poff(kC + 1, 0);
    for (int c = 0; c < nb; ++c) {
      const int32_t j = cols[c0 + c];
      jrow[c] = h->row_lib[j];
      for (int64_t e = h->row_ptr[j]; e < h->row_ptr[j + 1]; ++e) prow.push_back(h->row_lib[h->col_idx[e]]);
      poff[c + 1] = (int64_t)prow.size();
    }
    for (int c = nb; c < kC; ++c) poff[c + 1] = poff[nb];
    ce = cudaMemcpy(d_jrow, jrow.data(), kC * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && !prow.empty())
      ce = cudaMemcpy(d_prow, prow.data(), prow.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(d_poff, poff.data(), (kC + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    // lane state: seed lanes c < nb of both sequences alive
    std::vector<unsigned> k1(kL, 0u);
    std::vector<int> act(kL, 0);
    std::vector<double> ones(kL, 1.0), zeros(kL, 0.0);
    for (int c = 0; c < nb; ++c) act[c] = 1;
    if (ce == cudaSuccess) ce = cudaMemcpy(active, act.data(), kL * sizeof(int), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(rr, ones.data(), kL * sizeof(double), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(beta_prev, zeros.data(), kL * sizeof(double), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset(U[0], 0, vec64 * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMemset(cx, 0, vec32 * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMemset(cr, 0, vec32 * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMemset(cp, 0, vec32 * sizeof(double));
    if (ce != cudaSuccess) return GSK_ECUDA;
    k_cg_seed<<<1, kC>>>(nb, d_jrow, cr, cp, U[0]);

    // ---- B^-1 e_j by CG (32 lanes) ----
    const VecSet setR = make_set({cr}, {0}, kC);
    const double cg_tol2 = 1e-30;          // ||r|| <= 1e-15 (||e_j|| = 1): the projection amplifies seed error
    int it = 0;
    for (; it < kCgMax; ++it) {
      if (gsk::spmm64_dot(h, 1, kC, cp, cq, pq, sws, 0) != GSK_OK) return GSK_ECUDA;
      k_cg_xr<<<R.grid_vec, 256>>>(M, cx, cr, cp, cq, rr, pq, active);
      R.gram(setR, setR, kC, rr_new);
      k_cg_lane<<<1, 32>>>(rr, rr_new, pq, bta, active, cg_tol2, n_active);
      k_cg_p<<<R.grid_vec, 256>>>(M, cp, cr, bta, active);
      if ((it + 1) % kCgCheck == 0) {
        int na = 0;
        if (cudaMemcpy(&na, n_active, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GSK_ECUDA;
        if (na == 0) break;
      }
    }
    if (!R.ok) return GSK_ECUDA;
    // second sequence seed: U0[:, 32 + c] = x_c / ||x_c||
    const VecSet setX = make_set({cx}, {0}, kC);
    R.gram(setX, setX, kC, n2);
    k_inv_norm<<<1, kC>>>(n2, K1, kC);
    R.combine(setX, setX, make_setw({U[0]}, {kC}, kL), K1, kC, 0.0, 1.0);
    for (int c = 0; c < nb; ++c) k1[c] = k1[kC + c] = 1u;
    if (cudaMemcpy(keep1, k1.data(), kL * sizeof(unsigned), cudaMemcpyHostToDevice) != cudaSuccess) return GSK_ECUDA;

    // ---- Lanczos, 64 lanes, full reorthogonalisation ----
    const VecSet setW = make_set({Wv}, {0}, kL);
    const VecSetW setWw = make_setw({Wv}, {0}, kL);
    for (int k = 0; k < m; ++k) {
      if (gsk::spmm64_dot(h, 0, kL, U[k], AU[k], alpha, sws, 0) != GSK_OK) return GSK_ECUDA;
      if (k == m - 1) break;
      k_coef3<<<1, kL>>>(alpha, beta_prev, K2);
      if (k == 0) R.combine(make_set({U[0]}, {0}, kL), make_set({AU[0]}, {0}, kL), setWw, K2, kL, 1.0, 1.0);
      else R.combine(make_set({U[k], U[k - 1]}, {0, 0}, kL), make_set({AU[k]}, {0}, kL), setWw, K2, kL, 1.0, 1.0);
      std::vector<const double*> up(U.begin(), U.begin() + k + 1);
      const VecSet setU = make_set(up, std::vector<int>(k + 1, 0), kL);
      for (int pass = 0; pass < 2; ++pass) {
        R.gram(setU, setW, kL, K1);
        R.combine(setU, setW, setWw, K1, kL, 1.0, -1.0);
      }
      R.gram(setW, setW, kL, n2);
      k_lanczos_lane<<<1, kL>>>(k, n2, scale, beta_prev, inv, keep1);
      R.combine(setW, setW, make_setw({U[k + 1]}, {0}, kL), inv, kL, 0.0, 1.0);
    }
    if (!R.ok) return GSK_ECUDA;

    // ---- second sequence: project out the first (twice), orthonormalise ----
    std::vector<const double*> uc(U.begin(), U.end()), auc(AU.begin(), AU.end());
    const VecSet U1 = make_set(uc, std::vector<int>(m, 0), kL);
    const VecSet U2 = make_set(uc, std::vector<int>(m, kC), kL);
    const VecSet AU1 = make_set(auc, std::vector<int>(m, 0), kL);
    const VecSet AU2 = make_set(auc, std::vector<int>(m, kC), kL);
    const VecSetW U2w = make_setw(U, std::vector<int>(m, kC), kL);
    const VecSetW AU2w = make_setw(AU, std::vector<int>(m, kC), kL);
    for (int pass = 0; pass < 2; ++pass) {
      R.gram(U1, U2, kC, K1);
      R.combine(U1, U2, U2w, K1, kC, 1.0, -1.0);
      R.combine(AU1, AU2, AU2w, K1, kC, 1.0, -1.0);
    }
    R.gram(U2, U2, kC, K1);
    k_svqb<<<kC, 32>>>(m, K1, K2, keep2);
    R.combine(U2, U2, U2w, K2, kC, 0.0, 1.0);
    R.combine(AU2, AU2, AU2w, K2, kC, 0.0, 1.0);

    // ---- B Q and the reduced pencil ----
    for (int a = 0; a < m; ++a)
      if (gsk::spmm64_dot(h, 1, kL, U[a], BQ[a], n2, sws, 0) != GSK_OK) return GSK_ECUDA;
    std::vector<const double*> qp, aqp, bqp;
    std::vector<int> qo;
    for (int half = 0; half < 2; ++half)
      for (int a = 0; a < m; ++a) {
        qp.push_back(U[a]);
        aqp.push_back(AU[a]);
        bqp.push_back(BQ[a]);
        qo.push_back(half * kC);
      }
    const VecSet Q = make_set(qp, qo, kL), AQ = make_set(aqp, qo, kL), BQs = make_set(bqp, qo, kL);
    R.gram(Q, AQ, kC, At);
    R.gram(Q, BQs, kC, Bt);
    k_reduced<<<kC, 32>>>(m, At, Bt, keep1, keep2, d_U, d_BQ, d_jrow, nb, mu, kT, ro);
    k_ma_output<<<nb, 256>>>(m, d_U, d_prow, d_poff, ro, n_shifts, d_z, rho + pat_off[c0],
                             n_shifts > 0 ? reinterpret_cast<double2*>(G) + (size_t)pat_off[c0] * n_shifts : nullptr);
    if (!R.ok || cudaGetLastError() != cudaSuccess) return GSK_ECUDA;

    // ---- per-column scalars to the host ----
    std::vector<double> he((size_t)kC * kMaxN), hw((size_t)kC * kMaxN), hq((size_t)kC * kMaxN);
    std::vector<int> hr(kC), hs(kC);
    ce = cudaMemcpy(he.data(), ro.eps, he.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemcpy(hw.data(), ro.w, hw.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemcpy(hq.data(), ro.q, hq.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemcpy(hr.data(), ro.rank, kC * sizeof(int), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemcpy(hs.data(), ro.status, kC * sizeof(int), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return GSK_ECUDA;
    for (int c = 0; c < nb; ++c) {
      const size_t o = (size_t)(c0 + c) * nu;
      for (int s = 0; s < nu; ++s) {
        if (ritz) ritz[o + s] = he[(size_t)c * kMaxN + s];
        if (weight) weight[o + s] = hw[(size_t)c * kMaxN + s];
        if (charge) charge[o + s] = hq[(size_t)c * kMaxN + s];
      }
      if (rank) rank[c0 + c] = hs[c] ? -1 : hr[c];
    }
    if (it >= kCgMax) rc = GSK_ETIMEOUT;     // B^-1 e_j did not reach its tolerance
  }
  return rc;
}

}  // extern "C"
