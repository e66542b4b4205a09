// C ABI entry points of libgsk: handle creation (validation and the atom-block
// layout of A and B), pattern offsets, density matrix, traces, error strings.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "gsk_common.cuh"
#include "gsk_ctx.h"

using gsk::DevBuf;

namespace {

constexpr double kPi = 3.14159265358979323846;

// 3 x 10-bit interleave (Morton code) of a quantised position.
uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

bool finite_all(const double* v, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(v[i])) return false;
  return true;
}

int check_csr(const gsk_csr* m, int32_t M) {
  if (!m || m->n_rows != M || !m->row_ptr || !m->col_idx || !m->val) return GSK_EINVAL;
  if (m->row_ptr[0] != 0) return GSK_EINVAL;
  for (int32_t i = 0; i < M; ++i) {
    const int64_t a = m->row_ptr[i], b = m->row_ptr[i + 1];
    if (b < a) return GSK_EINVAL;
    for (int64_t e = a; e < b; ++e) {
      const int32_t c = m->col_idx[e];
      if (c < 0 || c >= M) return GSK_EINVAL;
      if (e > a && c <= m->col_idx[e - 1]) return GSK_EINVAL;
    }
  }
  if (!finite_all(m->val, m->row_ptr[M])) return GSK_EINVAL;
  return GSK_OK;
}

// Structural and numerical symmetry: for every (i, j) the entry (j, i) exists
// and agrees to a relative 1e-12.
bool symmetric(const gsk_csr* m) {
  const int32_t M = m->n_rows;
  for (int32_t i = 0; i < M; ++i) {
    for (int64_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; ++e) {
      const int32_t j = m->col_idx[e];
      if (j <= i) continue;
      const int32_t* lo = m->col_idx + m->row_ptr[j];
      const int32_t* hi = m->col_idx + m->row_ptr[j + 1];
      const int32_t* f = std::lower_bound(lo, hi, i);
      if (f == hi || *f != i) return false;
      const double a = m->val[e], b = m->val[m->row_ptr[j] + (f - lo)];
      if (fabs(a - b) > 1e-12 * std::max(fabs(a), fabs(b)) + 1e-300) return false;
    }
  }
  return true;
}

template <typename T>
cudaError_t upload(DevBuf& d, const std::vector<T>& h) {
  const size_t bytes = std::max<size_t>(h.size() * sizeof(T), 16);
  cudaError_t e = d.ensure(bytes);
  if (e != cudaSuccess) return e;
  if (!h.empty()) e = cudaMemcpy(d.ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// ---------------------------------------------------------------------------
// density and trace kernels
// ---------------------------------------------------------------------------
__global__ void k_fermi_weights(int S, const double* eps, const double* w, double mu, double kT,
                                double* coef) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S) return;
  // f(e) = 1/(1+exp(x)), x = (e-mu)/kT, with exp of a non-positive argument only
  const double x = (eps[k] - mu) / kT;
  const double ex = exp(-fabs(x));
  const double f = (x > 0.0) ? ex / (1.0 + ex) : 1.0 / (1.0 + ex);
  coef[k] = -w[k] * f / kPi;
}

// rho[e] = sum_k coef[k] * Im G[e][k]; one warp per element, fixed-order shuffle sum.
__global__ void k_density(int64_t n_elem, int S, const double* coef, const double2* G, double* rho) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = warp; e < n_elem; e += nwarps) {
    double s = 0.0;
    for (int k = lane; k < S; k += 32) s = fma(coef[k], G[e * S + k].y, s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rho[e] = s;
  }
}

// partial[b] = sum over this CTA's elements of rho[e] * val[vpos[e]]
__global__ void k_trace_partial(int64_t n, const double* rho, const int64_t* vpos, const double* val,
                                double* partial) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s = fma(rho[e], val[vpos[e]], s);
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void k_trace_final(int nb, const double* partial, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[b];
    *out = s;
  }
}

// Fixed device scratch of gsk_density_noalloc: eps, w and the Fermi-weighted
// coefficients of one call (3 * GSK_NOALLOC_MAX_SHIFTS doubles). Host code
// must not pass the symbol itself to a kernel: in host code it names a host
// stand-in, so the device address is looked up with cudaGetSymbolAddress.
__device__ __align__(256) double g_noalloc_scratch[3 * GSK_NOALLOC_MAX_SHIFTS];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once per device).
cudaError_t noalloc_scratch(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" {

int gsk_density_noalloc(int64_t n_elem, int32_t n_shifts, const double* eps, const double* w, double mu,
                        double kT, const double* G, double* rho, void* stream) {
  if (n_elem < 0 || n_shifts < 1 || n_shifts > GSK_NOALLOC_MAX_SHIFTS || !eps || !w || !(kT > 0.0) ||
      !isfinite(mu))
    return GSK_EINVAL;
  if (n_elem > 0 && (!G || !rho)) return GSK_EINVAL;
  if (!finite_all(eps, n_shifts) || !finite_all(w, n_shifts)) return GSK_EINVAL;
  if (n_elem == 0) return GSK_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return GSK_ECUDA;
  double* scratch = nullptr;
  if (noalloc_scratch(dev, &scratch) != cudaSuccess) return GSK_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* d_eps = scratch;
  double* d_w = scratch + n_shifts;
  double* d_coef = scratch + 2 * n_shifts;
  cudaError_t e = cudaMemcpyAsync(d_eps, eps, n_shifts * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_w, w, n_shifts * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return GSK_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GSK_ECUDA;
  k_fermi_weights<<<(n_shifts + 127) / 128, 128, 0, s>>>(n_shifts, d_eps, d_w, mu, kT, d_coef);
  const int64_t blocks = std::min<int64_t>((n_elem + 7) / 8, (int64_t)sms * 16);
  k_density<<<(unsigned)blocks, 256, 0, s>>>(n_elem, n_shifts, d_coef, reinterpret_cast<const double2*>(G), rho);
  return cudaGetLastError() == cudaSuccess ? GSK_OK : GSK_ECUDA;
}

void gsk_default_options(gsk_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = GSK_FP64;
  opt->tol = 1e-8;
  opt->max_iter = 20000;
  opt->batch_w = 0;
  opt->refine = 1;
  opt->sched = GSK_SCHED_FIFO;
  opt->inner_tol = 0.0;
  opt->max_inner = 200;
  opt->use_graph = 1;
  opt->stream = nullptr;
}

const char* gsk_strerror(int code) {
  switch (code) {
    case GSK_OK: return "ok";
    case GSK_EINVAL: return "invalid argument (shape, index, pointer, option or non-finite value)";
    case GSK_ENOTSPD: return "B fails the positive-diagonal / strict diagonal dominance check";
    case GSK_ENOMEM: return "out of memory";
    case GSK_ECUDA: return "CUDA runtime error";
    case GSK_ETIMEOUT: return "bounded device wait gave up";
    case GSK_ENOTSUP: return "option combination not supported";
    case GSK_EBOUNDS: return "bounds-checked build: an index check failed (see gsk_stats.debug_code)";
    default: return "unknown gsk status";
  }
}

int gsk_create(const gsk_csr* A, const gsk_csr* B, const gsk_orbmap* map, gsk_handle* out) {
  if (!out) return GSK_EINVAL;
  *out = nullptr;
  if (!A || !B || !map || A->n_rows <= 0 || map->n_atoms <= 0 || !map->orb_offset || !map->orb_count)
    return GSK_EINVAL;
  const int32_t M = A->n_rows;
  const int32_t N = map->n_atoms;
  int rc = check_csr(A, M);
  if (rc == GSK_OK) rc = check_csr(B, M);
  if (rc != GSK_OK) return rc;
  if (A->row_ptr[M] != B->row_ptr[M]) return GSK_EINVAL;
  for (int32_t i = 0; i <= M; ++i)
    if (A->row_ptr[i] != B->row_ptr[i]) return GSK_EINVAL;
  const int64_t nnz = A->row_ptr[M];
  for (int64_t e = 0; e < nnz; ++e)
    if (A->col_idx[e] != B->col_idx[e]) return GSK_EINVAL;
  // orbital map tiles the rows
  int64_t next = 0;
  for (int32_t I = 0; I < N; ++I) {
    const int c = map->orb_count[I];
    if ((c != 1 && c != 4) || map->orb_offset[I] != next) return GSK_EINVAL;
    next += c;
  }
  if (next != M) return GSK_EINVAL;
  if (map->pos && !finite_all(map->pos, 3 * (int64_t)N)) return GSK_EINVAL;
  if (!symmetric(A) || !symmetric(B)) return GSK_EINVAL;
  // B: positive diagonal and strict diagonal dominance (sufficient for SPD)
  std::vector<double> a_diag(M, 0.0), b_diag(M, 0.0), a_rowabs(M, 0.0), b_rowabs(M, 0.0);
  for (int32_t i = 0; i < M; ++i) {
    for (int64_t e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e) {
      if (A->col_idx[e] == i) {
        a_diag[i] = A->val[e];
        b_diag[i] = B->val[e];
      } else {
        a_rowabs[i] += fabs(A->val[e]);
        b_rowabs[i] += fabs(B->val[e]);
      }
    }
    if (!(b_diag[i] > 0.0) || !(b_diag[i] > b_rowabs[i])) return GSK_ENOTSPD;
  }

  gsk_ctx* h = new (std::nothrow) gsk_ctx();
  if (!h) return GSK_ENOMEM;
  auto fail = [&](int code) {
    delete h;
    return code;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess) return fail(GSK_ECUDA);
  if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
    return fail(GSK_ECUDA);
  h->M = M;
  h->n_atoms = N;
  h->nnz = nnz;
  h->row_ptr.assign(A->row_ptr, A->row_ptr + M + 1);
  h->col_idx.assign(A->col_idx, A->col_idx + nnz);
  h->a_diag = std::move(a_diag);
  h->b_diag = std::move(b_diag);
  h->a_rowabs = std::move(a_rowabs);
  h->b_rowabs = std::move(b_rowabs);

  // ---- atom order: Morton curve over positions (identity without them) ----
  std::vector<int32_t> perm(N);
  std::iota(perm.begin(), perm.end(), 0);
  if (map->pos) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int32_t I = 0; I < N; ++I)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], map->pos[3 * I + d]);
        hi[d] = std::max(hi[d], map->pos[3 * I + d]);
      }
    std::vector<uint32_t> code(N);
    for (int32_t I = 0; I < N; ++I) {
      uint32_t q[3];
      for (int d = 0; d < 3; ++d) {
        const double span = hi[d] - lo[d];
        const double t = span > 0 ? (map->pos[3 * I + d] - lo[d]) / span : 0.0;
        q[d] = (uint32_t)std::min(1023.0, std::max(0.0, floor(t * 1024.0)));
      }
      code[I] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
    }
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return code[a] < code[b]; });
    h->pos_lib.resize(3 * (size_t)N);
    for (int32_t I = 0; I < N; ++I)
      for (int d = 0; d < 3; ++d) h->pos_lib[3 * (size_t)I + d] = map->pos[3 * (size_t)perm[I] + d];
  }
  std::vector<int32_t> inv(N);
  for (int32_t I = 0; I < N; ++I) inv[perm[I]] = I;
  std::vector<int8_t> orb(N);
  std::vector<int32_t> roff(N + 1, 0);
  for (int32_t I = 0; I < N; ++I) {
    orb[I] = map->orb_count[perm[I]];
    roff[I + 1] = roff[I] + orb[I];
  }
  std::vector<int32_t> atom_of_row(M);
  for (int32_t Ic = 0; Ic < N; ++Ic)
    for (int a = 0; a < map->orb_count[Ic]; ++a) atom_of_row[map->orb_offset[Ic] + a] = Ic;
  h->row_lib.resize(M);
  for (int32_t i = 0; i < M; ++i) {
    const int32_t Ic = atom_of_row[i];
    h->row_lib[i] = roff[inv[Ic]] + (i - map->orb_offset[Ic]);
  }

  // ---- neighbour lists (library atoms), 4-orbital neighbours first ----
  std::vector<int32_t> nbr_ptr(N + 1, 0), nbr_mid(N), nbr_roff;
  std::vector<int32_t> nbr_atom;       // library atom of each entry (-1: padding)
  std::vector<int64_t> val_ptr(N);
  nbr_roff.reserve((size_t)nnz / 2 + 16);
  nbr_atom.reserve((size_t)nnz / 2 + 16);
  int64_t nval = 0;
  std::vector<int32_t> tmp4, tmp1;
  for (int32_t I = 0; I < N; ++I) {
    const int32_t Ic = perm[I];
    tmp4.clear();
    tmp1.clear();
    for (int a = 0; a < orb[I]; ++a) {
      const int32_t row = map->orb_offset[Ic] + a;
      for (int64_t e = A->row_ptr[row]; e < A->row_ptr[row + 1]; ++e) {
        const int32_t J = inv[atom_of_row[A->col_idx[e]]];
        (orb[J] == 4 ? tmp4 : tmp1).push_back(J);
      }
    }
    for (auto* t : {&tmp4, &tmp1}) {
      std::sort(t->begin(), t->end());
      t->erase(std::unique(t->begin(), t->end()), t->end());
    }
    val_ptr[I] = nval;
    for (int32_t J : tmp4) {
      nbr_atom.push_back(J);
      nbr_roff.push_back(roff[J]);
    }
    nbr_mid[I] = (int32_t)nbr_atom.size();
    for (int32_t J : tmp1) {
      nbr_atom.push_back(J);
      nbr_roff.push_back(roff[J]);
    }
    int64_t n1 = (int64_t)tmp1.size();
    if (orb[I] == 1) {
      const int64_t pad = (4 - n1 % 4) % 4;
      for (int64_t t = 0; t < pad; ++t) {
        nbr_atom.push_back(-1);
        nbr_roff.push_back(roff[I]);
      }
      n1 += pad;
      nval += 4 * (int64_t)tmp4.size() + n1;
    } else {
      nval += 16 * (int64_t)tmp4.size() + 4 * n1;
    }
    nbr_ptr[I + 1] = (int32_t)nbr_atom.size();
    if (nbr_atom.size() > (size_t)INT32_MAX - 64) return fail(GSK_ENOTSUP);
  }
  h->n_nbr = (int32_t)nbr_atom.size();
  h->n_vals = nval;

  // ---- values in the block layout; caller CSR entry -> value slot ----
  std::vector<double> va(nval, 0.0), vbv(nval, 0.0);
  h->csr_vpos.assign(nnz, -1);
  for (int32_t I = 0; I < N; ++I) {
    const int32_t Ic = perm[I];
    const int oI = orb[I];
    const int32_t e0 = nbr_ptr[I], em = nbr_mid[I];
    for (int a = 0; a < oI; ++a) {
      const int32_t row = map->orb_offset[Ic] + a;
      for (int64_t e = A->row_ptr[row]; e < A->row_ptr[row + 1]; ++e) {
        const int32_t col = A->col_idx[e];
        const int32_t Jc = atom_of_row[col];
        const int32_t J = inv[Jc];
        const int b = col - map->orb_offset[Jc];
        int64_t slot;
        if (orb[J] == 4) {
          const int32_t* f = std::lower_bound(nbr_atom.data() + e0, nbr_atom.data() + em, J);
          const int64_t t = f - (nbr_atom.data() + e0);
          slot = val_ptr[I] + t * 4 * oI + (int64_t)b * oI + a;
        } else {
          const int32_t* f = std::lower_bound(nbr_atom.data() + em, nbr_atom.data() + nbr_ptr[I + 1], J,
                                              [](int32_t x, int32_t y) { return (uint32_t)x < (uint32_t)y; });
          const int64_t t = f - (nbr_atom.data() + em);
          const int64_t n4 = em - e0;
          slot = val_ptr[I] + n4 * 4 * oI + t * oI + a;
        }
        va[slot] = A->val[e];
        vbv[slot] = B->val[e];
        h->csr_vpos[e] = slot;
      }
    }
  }
  // FP32 copies for the mixed-precision inner solve
  std::vector<float> va32(nval), vb32(nval);
  std::vector<float> va2(2 * nval), vb2(2 * nval);     // double-float pairs (hi, lo)
  for (int64_t t = 0; t < nval; ++t) {
    va32[t] = (float)va[t];
    vb32[t] = (float)vbv[t];
    va2[2 * t] = va32[t];
    va2[2 * t + 1] = (float)(va[t] - (double)va32[t]);
    vb2[2 * t] = vb32[t];
    vb2[2 * t + 1] = (float)(vbv[t] - (double)vb32[t]);
  }

  std::vector<float> rowfeat;
  gsk::build_row_features(A, B, map, rowfeat);

  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload(h->d_rowfeat, rowfeat);
  if (e == cudaSuccess) e = upload(h->d_atom_roff, roff);
  if (e == cudaSuccess) e = upload(h->d_atom_orb, orb);
  if (e == cudaSuccess) e = upload(h->d_nbr_ptr, nbr_ptr);
  if (e == cudaSuccess) e = upload(h->d_nbr_mid, nbr_mid);
  if (e == cudaSuccess) e = upload(h->d_nbr_roff, nbr_roff);
  if (e == cudaSuccess) e = upload(h->d_val_ptr, val_ptr);
  if (e == cudaSuccess) e = upload(h->d_A64, va);
  if (e == cudaSuccess) e = upload(h->d_B64, vbv);
  if (e == cudaSuccess) e = upload(h->d_A32, va32);
  if (e == cudaSuccess) e = upload(h->d_B32, vb32);
  if (e == cudaSuccess) e = upload(h->d_A2, va2);
  if (e == cudaSuccess) e = upload(h->d_B2, vb2);
  if (e == cudaErrorMemoryAllocation) return fail(GSK_ENOMEM);
  if (e != cudaSuccess) return fail(GSK_ECUDA);

  gsk::Layout& L = h->lay;
  L.n_atoms = N;
  L.M = M;
  L.n_ctas = std::max(1, std::min((N + gsk::kWarps - 1) / gsk::kWarps, h->num_sms * 6));
  L.chunk = (N + L.n_ctas - 1) / L.n_ctas;
  // Static balance of the SpMM traversal: the atoms are cut into one
  // contiguous segment per warp of about equal cost, the cost of an atom being
  // its multiply-adds per lane plus a load overhead per neighbour block. The
  // cut is fixed at creation, so every product sums in the same order.
  {
    const int n_w = L.n_ctas * gsk::kWarps;
    std::vector<double> cost(N);
    double total = 0.0;
    for (int32_t I = 0; I < N; ++I) {
      const int n4 = nbr_mid[I] - nbr_ptr[I];
      const int n1 = nbr_ptr[I + 1] - nbr_mid[I];
      const double fma = (double)orb[I] * (4.0 * n4 + n1);
      const double blocks = (orb[I] == 4) ? (double)(n4 + n1) : (double)n4 + n1 / 4.0;
      cost[I] = fma + 8.0 * blocks;
      total += cost[I];
    }
    std::vector<int32_t> cut(n_w + 1, N);
    cut[0] = 0;
    double acc = 0.0;
    int w = 1;
    for (int32_t I = 0; I < N && w < n_w; ++I) {
      acc += cost[I];
      while (w < n_w && acc >= total * w / n_w) cut[w++] = I + 1;
    }
    for (; w < n_w; ++w) cut[w] = N;
    if (upload(h->d_warp_atoms, cut) != cudaSuccess) return fail(GSK_ECUDA);
    L.warp_atoms = h->d_warp_atoms.as<int32_t>();
  }
  // tiles of the staged SpMM; an atom too large for one tile leaves them unbuilt
  {
    const int trc = gsk::build_tiles(h, roff, orb, nbr_ptr, nbr_mid, nbr_atom, val_ptr, nval);
    if (trc == GSK_ENOMEM || trc == GSK_ECUDA) return fail(trc);
    if (trc != GSK_OK) h->tiles.n_tiles = 0;
  }
  L.atom_roff = h->d_atom_roff.as<int32_t>();
  L.atom_orb = h->d_atom_orb.as<int8_t>();
  L.nbr_ptr = h->d_nbr_ptr.as<int32_t>();
  L.nbr_mid = h->d_nbr_mid.as<int32_t>();
  L.nbr_roff = h->d_nbr_roff.as<int32_t>();
  L.val_ptr = h->d_val_ptr.as<int64_t>();
#ifdef GSK_DEBUG
  L.n_nbr = h->n_nbr;
  L.n_vals = h->n_vals;
#endif
  h->atom_perm = std::move(perm);
  h->atom_of_row = std::move(atom_of_row);
  h->orb_lib = std::move(orb);
  *out = h;
  return GSK_OK;
}

int gsk_destroy(gsk_handle h) {
  if (!h) return GSK_OK;
  int dev = -1;
  cudaGetDevice(&dev);
  cudaSetDevice(h->device);
  delete h;
  if (dev >= 0) cudaSetDevice(dev);
  return GSK_OK;
}

int gsk_autotune(gsk_handle h, int32_t n_shifts, const double* z, const double* eta, int32_t n_cols,
                 const int32_t* cols, const gsk_options* opt, int32_t* best_w) {
  if (!h) return GSK_EINVAL;
  return gsk::autotune_impl(h, n_shifts, z, eta, n_cols, cols, opt, best_w);
}

int gsk_autotune_result(gsk_handle h, int32_t precision, int32_t* w, int32_t* kernel, int32_t* from_cache,
                        int32_t* n_cand, int32_t* cand_w, int32_t* cand_kernel, double* cand_ms_per_step) {
  if (!h || precision < GSK_FP64 || precision > GSK_MIXED_DF) return GSK_EINVAL;
  const gsk::TuneRecord& r = h->tune[precision];
  if (w) *w = r.w;
  if (kernel) *kernel = r.kernel;
  if (from_cache) *from_cache = r.from_cache;
  if (n_cand) *n_cand = r.n_cand;
  for (int i = 0; i < r.n_cand; ++i) {
    if (cand_w) cand_w[i] = r.cand_w[i];
    if (cand_kernel) cand_kernel[i] = r.cand_kernel[i];
    if (cand_ms_per_step) cand_ms_per_step[i] = r.cand_ms_per_step[i];
  }
  return GSK_OK;
}

int gsk_row_order(gsk_handle h, int32_t* row_lib) {
  if (!h || !row_lib) return GSK_EINVAL;
  memcpy(row_lib, h->row_lib.data(), (size_t)h->M * sizeof(int32_t));
  return GSK_OK;
}

int gsk_spmm(gsk_handle h, int32_t which, int32_t precision, int32_t W, const void* X, void* Y, int32_t n_rep,
             void* stream) {
  if (!h) return GSK_EINVAL;
  return gsk::spmm_impl(h, which, precision, W, X, Y, n_rep, stream);
}

int gsk_last_stats(gsk_handle h, gsk_stats* out) {
  if (!h || !out) return GSK_EINVAL;
  *out = h->last;
  return GSK_OK;
}

int gsk_dims(gsk_handle h, int32_t* M, int64_t* nnz) {
  if (!h) return GSK_EINVAL;
  if (M) *M = h->M;
  if (nnz) *nnz = h->nnz;
  return GSK_OK;
}

int gsk_pattern_offsets(gsk_handle h, int32_t n_cols, const int32_t* cols, int64_t* offsets) {
  if (!h || n_cols < 0 || !offsets || (n_cols > 0 && !cols)) return GSK_EINVAL;
  offsets[0] = 0;
  for (int32_t c = 0; c < n_cols; ++c) {
    const int32_t j = cols[c];
    if (j < 0 || j >= h->M) return GSK_EINVAL;
    offsets[c + 1] = offsets[c] + (h->row_ptr[j + 1] - h->row_ptr[j]);
  }
  return GSK_OK;
}

int gsk_solve(gsk_handle h, int32_t n_shifts, const double* z, const double* eta, int32_t n_cols,
              const int32_t* cols, const gsk_options* opt, double* G, int32_t* iters, int32_t* status,
              double* resid) {
  if (!h) return GSK_EINVAL;
  return gsk::solve_impl(h, n_shifts, z, eta, n_cols, cols, opt, G, iters, status, resid);
}

int gsk_density(gsk_handle h, int64_t n_elem, int32_t n_shifts, const double* eps, const double* w,
                double mu, double kT, const double* G, double* rho, void* stream) {
  if (!h || n_elem < 0 || n_shifts < 1 || !eps || !w || !(kT > 0.0) || !isfinite(mu)) return GSK_EINVAL;
  if (n_elem > 0 && (!G || !rho)) return GSK_EINVAL;
  if (!finite_all(eps, n_shifts) || !finite_all(w, n_shifts)) return GSK_EINVAL;
  if (n_elem == 0) return GSK_OK;
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->ws_misc.ensure(3 * (size_t)n_shifts * sizeof(double) + 256) != cudaSuccess) return GSK_ENOMEM;
  double* d_eps = h->ws_misc.as<double>();
  double* d_w = d_eps + n_shifts;
  double* d_coef = d_w + n_shifts;
  cudaError_t e = cudaMemcpyAsync(d_eps, eps, n_shifts * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_w, w, n_shifts * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return GSK_ECUDA;
  k_fermi_weights<<<(n_shifts + 127) / 128, 128, 0, s>>>(n_shifts, d_eps, d_w, mu, kT, d_coef);
  const int64_t blocks = std::min<int64_t>((n_elem + 7) / 8, (int64_t)h->num_sms * 16);
  k_density<<<(unsigned)blocks, 256, 0, s>>>(n_elem, n_shifts, d_coef, reinterpret_cast<const double2*>(G), rho);
  return cudaGetLastError() == cudaSuccess ? GSK_OK : GSK_ECUDA;
}

int gsk_trace(gsk_handle h, int32_t n_cols, const int32_t* cols, const double* rho, int32_t which,
              double* out) {
  if (!h || n_cols < 0 || !out || (which != 0 && which != 1) || (n_cols > 0 && (!cols || !rho)))
    return GSK_EINVAL;
  *out = 0.0;
  std::vector<int64_t> vpos;
  for (int32_t c = 0; c < n_cols; ++c) {
    const int32_t j = cols[c];
    if (j < 0 || j >= h->M) return GSK_EINVAL;
    for (int64_t e = h->row_ptr[j]; e < h->row_ptr[j + 1]; ++e) vpos.push_back(h->csr_vpos[e]);
  }
  if (vpos.empty()) return GSK_OK;
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  const int nb = 256;
  const size_t need = vpos.size() * sizeof(int64_t) + (nb + 1) * sizeof(double) + 256;
  if (h->ws_misc.ensure(need) != cudaSuccess) return GSK_ENOMEM;
  int64_t* d_vpos = h->ws_misc.as<int64_t>();
  double* d_part = reinterpret_cast<double*>(d_vpos + vpos.size());
  cudaError_t e = cudaMemcpy(d_vpos, vpos.data(), vpos.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return GSK_ECUDA;
  const double* val = which == 0 ? h->d_A64.as<double>() : h->d_B64.as<double>();
  k_trace_partial<<<nb, 256>>>((int64_t)vpos.size(), rho, d_vpos, val, d_part);
  k_trace_final<<<1, 32>>>(nb, d_part, d_part + nb);
  e = cudaMemcpy(out, d_part + nb, sizeof(double), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? GSK_OK : GSK_ECUDA;
}

}  // extern "C"
