// Trace quantities on the solved columns (Sec. II, Eq. TRACE-X and
// Eq. EQ-FD-FUNC; Sec. VII, ICOHP): per-shift traces of Im G X, the chemical
// potential that fixes the electron count, the atom pattern of A and the
// connectivity matrix C_IJ.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "gsk_common.cuh"
#include "gsk_ctx.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kTraceShifts = 32;     // shifts per CTA column of the trace kernel (one per lane)
constexpr int kTraceRows = 8;        // element rows per CTA (one per warp)
constexpr int kMuRounds = 48;        // 33-section rounds of the chemical-potential search

// partial[bx][k] = sum over this CTA's elements e of X[vpos[e]] * Im G[e][k].
// Warp y of the CTA walks elements e = bx*8 + y, +8*gridDim.x, ...; lane x
// holds shift k = 32*blockIdx.y + x, so a warp reads 32 consecutive complex
// numbers (512 B) of one element. The 8 warps are folded in a fixed order.
__global__ void k_shift_trace_partial(int64_t n_elem, int S, const double2* __restrict__ G,
                                      const int64_t* __restrict__ vpos, const double* __restrict__ val,
                                      double* __restrict__ partial) {
  __shared__ double sm[kTraceRows][kTraceShifts];
  const int k = blockIdx.y * kTraceShifts + threadIdx.x;
  double s = 0.0;
  if (k < S) {
    for (int64_t e = (int64_t)blockIdx.x * kTraceRows + threadIdx.y; e < n_elem;
         e += (int64_t)gridDim.x * kTraceRows)
      s = fma(val[vpos[e]], G[e * S + k].y, s);
  }
  sm[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && k < S) {
    double t = 0.0;
    for (int y = 0; y < kTraceRows; ++y) t += sm[y][threadIdx.x];
    partial[(int64_t)blockIdx.x * S + k] = t;
  }
}

// s[k] = sum over CTAs b (in order) of partial[b][k].
__global__ void k_shift_trace_final(int nb, int S, const double* __restrict__ partial, double* __restrict__ s) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += partial[(int64_t)b * S + k];
  s[k] = t;
}

// N(mu) = -(1/pi) sum_k w_k f_mu(e_k) s_k, f in overflow-free form; one lane.
__device__ double electron_count(int S, const double* eps, const double* w, const double* s, double mu,
                                 double kT) {
  double n = 0.0;
  for (int k = 0; k < S; ++k) {
    const double x = (eps[k] - mu) / kT;
    const double ex = exp(-fabs(x));
    const double f = (x > 0.0) ? ex / (1.0 + ex) : 1.0 / (1.0 + ex);
    n = fma(w[k] * f, s[k], n);
  }
  return -n / kPi;
}

// Root of N(mu) = n_elec on [lo, hi] by 33-section search: each round the 32
// lanes evaluate N at 32 interior points and the bracket shrinks to the first
// sub-interval whose right end reaches n_elec, so N(lo) < n_elec <= N(hi)
// holds throughout (a root of the continuous N stays inside). out[0] = mu,
// out[1] = N(mu), out[2] = 1 if the initial bracket holds, else 0.
__global__ void k_mu_search(int S, const double* __restrict__ eps, const double* __restrict__ w,
                            const double* __restrict__ s, double kT, double n_elec, double lo, double hi,
                            double* __restrict__ out) {
  const int lane = threadIdx.x;
  const double nlo = electron_count(S, eps, w, s, lo, kT);    // every lane, same value
  const double nhi = electron_count(S, eps, w, s, hi, kT);
  if (!(nlo < n_elec && n_elec <= nhi)) {
    if (lane == 0) {
      out[0] = 0.5 * (lo + hi);
      out[1] = 0.0;
      out[2] = 0.0;
    }
    return;
  }
  for (int r = 0; r < kMuRounds; ++r) {
    const double c = lo + (hi - lo) * (double)(lane + 1) / 33.0;
    const bool up = electron_count(S, eps, w, s, c, kT) >= n_elec;
    const unsigned ball = __ballot_sync(0xffffffffu, up);
    double nlo2, nhi2;
    if (ball == 0u) {
      nlo2 = __shfl_sync(0xffffffffu, c, 31);
      nhi2 = hi;
    } else {
      const int l0 = __ffs(ball) - 1;
      nhi2 = __shfl_sync(0xffffffffu, c, l0);
      const double cprev = __shfl_sync(0xffffffffu, c, l0 > 0 ? l0 - 1 : 0);
      nlo2 = l0 > 0 ? cprev : lo;
    }
    if (!(nlo2 > lo || nhi2 < hi)) break;     // the bracket cannot shrink further in FP64
    lo = nlo2;
    hi = nhi2;
  }
  const double mu = 0.5 * (lo + hi);
  const double n = electron_count(S, eps, w, s, mu, kT);
  if (lane == 0) {
    out[0] = mu;
    out[1] = n;
    out[2] = 1.0;
  }
}

// C[q] = sum over the gather list of output slot q (in list order) of
// rho[rix[p]] * A[vpos[p]]: each slot has its own fixed order, so the result
// does not depend on the launch shape.
__global__ void k_icohp(int64_t n_slots, const int64_t* __restrict__ optr, const int64_t* __restrict__ rix,
                        const int64_t* __restrict__ vpos, const double* __restrict__ rho,
                        const double* __restrict__ aval, double* __restrict__ C) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_slots;
       q += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int64_t p = optr[q]; p < optr[q + 1]; ++p) t = fma(rho[rix[p]], aval[vpos[p]], t);
    C[q] = t;
  }
}

bool cols_valid(const gsk_ctx* h, int32_t n_cols, const int32_t* cols) {
  for (int32_t c = 0; c < n_cols; ++c)
    if (cols[c] < 0 || cols[c] >= h->M) return false;
  return true;
}

// Value slots (block layout) of the pattern entries of the columns, in G's order.
void gather_vpos(const gsk_ctx* h, int32_t n_cols, const int32_t* cols, std::vector<int64_t>& vpos) {
  vpos.clear();
  for (int32_t c = 0; c < n_cols; ++c) {
    const int32_t j = cols[c];
    for (int64_t e = h->row_ptr[j]; e < h->row_ptr[j + 1]; ++e) vpos.push_back(h->csr_vpos[e]);
  }
}

void ensure_atom_pattern(gsk_ctx* h) {
  if (!h->apat_ptr.empty()) return;
  const int32_t N = h->n_atoms;
  std::vector<int32_t> first(N, 0);          // first row of each caller atom
  for (int32_t i = h->M - 1; i >= 0; --i) first[h->atom_of_row[i]] = i;
  h->apat_ptr.assign(N + 1, 0);
  h->apat_idx.clear();
  std::vector<int32_t> nb;
  for (int32_t J = 0; J < N; ++J) {
    nb.clear();
    for (int32_t j = first[J]; j < h->M && h->atom_of_row[j] == J; ++j)
      for (int64_t e = h->row_ptr[j]; e < h->row_ptr[j + 1]; ++e) nb.push_back(h->atom_of_row[h->col_idx[e]]);
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    h->apat_idx.insert(h->apat_idx.end(), nb.begin(), nb.end());
    h->apat_ptr[J + 1] = (int64_t)h->apat_idx.size();
  }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Per-shift traces s_k into device memory. ws_misc holds, in order: `front`
// bytes for the caller (returned in *d_front), s (S doubles, *d_s), the
// value slots of the pattern entries and the per-CTA partial sums. Returns a
// GSK_ status; the work is queued on the legacy default stream.
int shift_trace_device(gsk_ctx* h, int32_t n_cols, const int32_t* cols, int32_t S, const double* G,
                       int32_t which, size_t front, char** d_front, double** d_s) {
  std::vector<int64_t> vpos;
  gather_vpos(h, n_cols, cols, vpos);
  const int64_t n = (int64_t)vpos.size();
  const int shift_blocks = (S + kTraceShifts - 1) / kTraceShifts;
  int nb = (int)std::min<int64_t>((n + kTraceRows - 1) / kTraceRows,
                                  std::max<int64_t>(1, (int64_t)h->num_sms * 8 / shift_blocks));
  nb = std::max(nb, 1);
  const size_t o_s = align256(front);
  const size_t o_v = o_s + align256((size_t)S * sizeof(double));
  const size_t o_p = o_v + align256((size_t)std::max<int64_t>(n, 1) * sizeof(int64_t));
  const size_t need = o_p + (size_t)nb * S * sizeof(double);
  if (h->ws_misc.ensure(need) != cudaSuccess) return GSK_ENOMEM;
  char* base = h->ws_misc.as<char>();
  *d_front = base;
  *d_s = reinterpret_cast<double*>(base + o_s);
  int64_t* d_vpos = reinterpret_cast<int64_t*>(base + o_v);
  double* d_part = reinterpret_cast<double*>(base + o_p);
  if (n == 0) {
    if (cudaMemset(*d_s, 0, (size_t)S * sizeof(double)) != cudaSuccess) return GSK_ECUDA;
    return GSK_OK;
  }
  if (cudaMemcpy(d_vpos, vpos.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess)
    return GSK_ECUDA;
  const double* val = which == 0 ? h->d_A64.as<double>() : h->d_B64.as<double>();
  const dim3 grid((unsigned)nb, (unsigned)shift_blocks);
  k_shift_trace_partial<<<grid, dim3(kTraceShifts, kTraceRows)>>>(n, S, reinterpret_cast<const double2*>(G),
                                                                   d_vpos, val, d_part);
  k_shift_trace_final<<<(S + 127) / 128, 128>>>(nb, S, d_part, *d_s);
  return cudaGetLastError() == cudaSuccess ? GSK_OK : GSK_ECUDA;
}

bool finite_n(const double* v, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(v[i])) return false;
  return true;
}

}  // namespace

extern "C" {

int gsk_shift_trace(gsk_handle h, int32_t n_cols, const int32_t* cols, int32_t n_shifts, const double* G,
                    int32_t which, double* s) {
  if (!h || n_cols < 0 || n_shifts < 1 || !s || (which != 0 && which != 1)) return GSK_EINVAL;
  if (n_cols > 0 && (!cols || !G)) return GSK_EINVAL;
  if (!cols_valid(h, n_cols, cols)) return GSK_EINVAL;
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  char* d_front = nullptr;
  double* d_s = nullptr;
  const int rc = shift_trace_device(h, n_cols, cols, n_shifts, G, which, 0, &d_front, &d_s);
  if (rc != GSK_OK) return rc;
  return cudaMemcpy(s, d_s, (size_t)n_shifts * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess
             ? GSK_OK : GSK_ECUDA;
}

// mu search on the GPU from per-shift traces already in device memory
// (d_front holds room for eps, w and the 3 outputs, d_s the traces).
static int mu_search_device(int32_t n_shifts, const double* eps, const double* w, const double* d_s, char* d_front,
                            double kT, double n_elec, double mu_lo, double mu_hi, double* mu, double* count) {
  double* d_eps = reinterpret_cast<double*>(d_front);
  double* d_w = d_eps + n_shifts;
  double* d_out = d_w + n_shifts;
  cudaError_t e = cudaMemcpy(d_eps, eps, (size_t)n_shifts * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_w, w, (size_t)n_shifts * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return GSK_ECUDA;
  k_mu_search<<<1, 32>>>(n_shifts, d_eps, d_w, d_s, kT, n_elec, mu_lo, mu_hi, d_out);
  double out[3];
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(out), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return GSK_ECUDA;
  if (out[2] != 1.0) return GSK_EINVAL;      // n_elec not bracketed by [mu_lo, mu_hi]
  *mu = out[0];
  if (count) *count = out[1];
  return GSK_OK;
}

static bool mu_args_ok(int32_t n_shifts, const double* eps, const double* w, double kT, double n_elec, double mu_lo,
                       double mu_hi, const double* mu) {
  if (n_shifts < 1 || !eps || !w || !mu) return false;
  if (!(kT > 0.0) || !isfinite(kT) || !isfinite(n_elec) || !isfinite(mu_lo) || !isfinite(mu_hi) || !(mu_lo < mu_hi))
    return false;
  return finite_n(eps, n_shifts) && finite_n(w, n_shifts);
}

int gsk_mu_from_traces(gsk_handle h, int32_t n_shifts, const double* eps, const double* w, const double* s,
                       double kT, double n_elec, double mu_lo, double mu_hi, double* mu, double* count) {
  if (!h || !s || !mu_args_ok(n_shifts, eps, w, kT, n_elec, mu_lo, mu_hi, mu)) return GSK_EINVAL;
  if (!finite_n(s, n_shifts)) return GSK_EINVAL;
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  const size_t front = align256((2 * (size_t)n_shifts + 4) * sizeof(double));
  if (h->ws_misc.ensure(front + (size_t)n_shifts * sizeof(double)) != cudaSuccess) return GSK_ENOMEM;
  char* base = h->ws_misc.as<char>();
  double* d_s = reinterpret_cast<double*>(base + front);
  if (cudaMemcpy(d_s, s, (size_t)n_shifts * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) return GSK_ECUDA;
  return mu_search_device(n_shifts, eps, w, d_s, base, kT, n_elec, mu_lo, mu_hi, mu, count);
}

int gsk_find_mu(gsk_handle h, int32_t n_cols, const int32_t* cols, int32_t n_shifts, const double* eps,
                const double* w, const double* G, double kT, double n_elec, double mu_lo, double mu_hi,
                double* mu, double* count) {
  if (!h || n_cols < 1 || !cols || !G || !mu_args_ok(n_shifts, eps, w, kT, n_elec, mu_lo, mu_hi, mu))
    return GSK_EINVAL;
  if (!cols_valid(h, n_cols, cols)) return GSK_EINVAL;
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  char* d_front = nullptr;
  double* d_s = nullptr;
  const size_t front = (2 * (size_t)n_shifts + 4) * sizeof(double);
  const int rc = shift_trace_device(h, n_cols, cols, n_shifts, G, 1, front, &d_front, &d_s);
  if (rc != GSK_OK) return rc;
  return mu_search_device(n_shifts, eps, w, d_s, d_front, kT, n_elec, mu_lo, mu_hi, mu, count);
}

int gsk_atom_pattern(gsk_handle h, int64_t* aptr, int32_t* aidx) {
  if (!h || !aptr) return GSK_EINVAL;
  ensure_atom_pattern(h);
  std::copy(h->apat_ptr.begin(), h->apat_ptr.end(), aptr);
  if (aidx) std::copy(h->apat_idx.begin(), h->apat_idx.end(), aidx);
  return GSK_OK;
}

int gsk_icohp(gsk_handle h, int32_t n_cols, const int32_t* cols, const double* rho, double* C, void* stream) {
  if (!h || n_cols < 0 || !C || (n_cols > 0 && (!cols || !rho))) return GSK_EINVAL;
  if (!cols_valid(h, n_cols, cols)) return GSK_EINVAL;
  ensure_atom_pattern(h);
  const int64_t n_slots = (int64_t)h->apat_idx.size();
  // gather lists: for every atom-pattern slot, the (rho entry, A value slot)
  // pairs of the given columns that fall in it, in (column, entry) order
  std::vector<int64_t> slot_of;                     // per pattern entry of the columns
  std::vector<int64_t> optr(n_slots + 1, 0);
  int64_t n_pairs = 0;
  for (int32_t c = 0; c < n_cols; ++c) {
    const int32_t j = cols[c];
    const int32_t J = h->atom_of_row[j];
    const int32_t* a0 = h->apat_idx.data() + h->apat_ptr[J];
    const int32_t* a1 = h->apat_idx.data() + h->apat_ptr[J + 1];
    for (int64_t e = h->row_ptr[j]; e < h->row_ptr[j + 1]; ++e) {
      const int32_t I = h->atom_of_row[h->col_idx[e]];
      const int64_t q = h->apat_ptr[J] + (std::lower_bound(a0, a1, I) - a0);
      slot_of.push_back(q);
      ++optr[q + 1];
      ++n_pairs;
    }
  }
  for (int64_t q = 0; q < n_slots; ++q) optr[q + 1] += optr[q];
  std::vector<int64_t> rix(std::max<int64_t>(n_pairs, 1)), vpos(std::max<int64_t>(n_pairs, 1));
  {
    std::vector<int64_t> fill(optr.begin(), optr.end() - 1);
    int64_t t = 0;
    for (int32_t c = 0; c < n_cols; ++c) {
      const int32_t j = cols[c];
      for (int64_t e = h->row_ptr[j]; e < h->row_ptr[j + 1]; ++e, ++t) {
        const int64_t p = fill[slot_of[t]]++;
        rix[p] = t;                                   // rho is laid out like G: entry t of the column set
        vpos[p] = h->csr_vpos[e];
      }
    }
  }
  if (n_slots == 0) return GSK_OK;
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  const size_t o_r = align256((size_t)(n_slots + 1) * sizeof(int64_t));
  const size_t o_v = o_r + align256(rix.size() * sizeof(int64_t));
  const size_t need = o_v + vpos.size() * sizeof(int64_t);
  if (h->ws_misc.ensure(need) != cudaSuccess) return GSK_ENOMEM;
  char* base = h->ws_misc.as<char>();
  int64_t* d_optr = reinterpret_cast<int64_t*>(base);
  int64_t* d_rix = reinterpret_cast<int64_t*>(base + o_r);
  int64_t* d_vpos = reinterpret_cast<int64_t*>(base + o_v);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the host lists are pageable and die with this call: copy synchronously
  cudaError_t e = cudaMemcpy(d_optr, optr.data(), optr.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_rix, rix.data(), rix.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_vpos, vpos.data(), vpos.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return GSK_ECUDA;
  const int64_t blocks = std::min<int64_t>((n_slots + 255) / 256, (int64_t)h->num_sms * 8);
  k_icohp<<<(unsigned)blocks, 256, 0, st>>>(n_slots, d_optr, d_rix, d_vpos, rho, h->d_A64.as<double>(), C);
  return cudaGetLastError() == cudaSuccess ? GSK_OK : GSK_ECUDA;
}

}  // extern "C"
