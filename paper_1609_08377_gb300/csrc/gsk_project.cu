// Real-space projection (Sec. III-B): each column j is solved on the pencil
// restricted to the region of kappa atoms or more around its atom (all atoms
// within the distance of the kappa-th nearest one, J included, minimum image
// in a periodic box), by the multiple Arnoldi projection of gsk_marnoldi.
//
// The columns of a batch of 32 have independent restricted pencils; they are
// placed side by side as one block-diagonal pencil (a temporary handle), whose
// columns gsk_marnoldi solves together. A column's Krylov vectors stay inside
// its own block, so the batch computes exactly the 32 projected problems.
// rho comes back on the full pattern P(j), zero for rows outside the region.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "gsk_common.cuh"
#include "gsk_ctx.h"

namespace {

constexpr int kBatch = 32;

// rho[e] = idx[e] >= 0 ? local[idx[e]] : 0
__global__ void k_scatter_rho(int64_t n, const int64_t* __restrict__ idx, const double* __restrict__ local,
                              double* __restrict__ rho) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = idx[e];
    rho[e] = k >= 0 ? local[k] : 0.0;
  }
}

// Host copies of the values (caller CSR order is reached through csr_vpos),
// the caller-order positions and the first row of every caller atom.
int ensure_host_side(gsk_ctx* h) {
  if (h->host_A64.empty()) {
    h->host_A64.resize(h->n_vals);
    h->host_B64.resize(h->n_vals);
    if (cudaMemcpy(h->host_A64.data(), h->d_A64.ptr, h->n_vals * sizeof(double), cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(h->host_B64.data(), h->d_B64.ptr, h->n_vals * sizeof(double), cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
      h->host_A64.clear();
      h->host_B64.clear();
      return GSK_ECUDA;
    }
  }
  if (h->pos_caller.empty() && !h->pos_lib.empty()) {
    h->pos_caller.resize(3 * (size_t)h->n_atoms);
    for (int32_t I = 0; I < h->n_atoms; ++I)
      for (int d = 0; d < 3; ++d) h->pos_caller[3 * (size_t)h->atom_perm[I] + d] = h->pos_lib[3 * (size_t)I + d];
  }
  if (h->atom_first_row.empty()) {
    h->atom_first_row.assign(h->n_atoms + 1, 0);
    for (int32_t i = h->M - 1; i >= 0; --i) h->atom_first_row[h->atom_of_row[i]] = i;
    h->atom_first_row[h->n_atoms] = h->M;
  }
  return GSK_OK;
}

// Uniform grid of cells over the atoms (periodic box, or the atoms' bounding
// box without one), about 8 atoms per cell, for the region search.
struct CellGrid {
  int n[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, side[3] = {1, 1, 1};
  bool periodic = false;
  std::vector<int32_t> start, atoms;      // cell c holds atoms[start[c] .. start[c+1])

  int coord(double x, int d) const {
    double t = x - lo[d];
    if (periodic) t -= side[d] * n[d] * floor(t / (side[d] * n[d]));
    int k = (int)floor(t / side[d]);
    return std::min(std::max(k, 0), n[d] - 1);
  }
  void build(const double* pos, int32_t N, const double* box) {
    periodic = box != nullptr;
    double ext[3];
    for (int d = 0; d < 3; ++d) {
      if (periodic) {
        lo[d] = 0.0;
        ext[d] = box[d];
      } else {
        double a = 1e300, b = -1e300;
        for (int32_t i = 0; i < N; ++i) {
          a = std::min(a, pos[3 * (size_t)i + d]);
          b = std::max(b, pos[3 * (size_t)i + d]);
        }
        lo[d] = a;
        ext[d] = std::max(b - a, 1e-9);
      }
    }
    const double c = cbrt(ext[0] * ext[1] * ext[2] * 8.0 / std::max(N, 1));
    for (int d = 0; d < 3; ++d) {
      n[d] = std::max(1, std::min(1024, (int)floor(ext[d] / std::max(c, 1e-9))));
      side[d] = ext[d] / n[d];
    }
    const size_t nc = (size_t)n[0] * n[1] * n[2];
    std::vector<int32_t> cell(N);
    start.assign(nc + 1, 0);
    for (int32_t i = 0; i < N; ++i) {
      const int cx = coord(pos[3 * (size_t)i], 0), cy = coord(pos[3 * (size_t)i + 1], 1),
                cz = coord(pos[3 * (size_t)i + 2], 2);
      cell[i] = (cz * n[1] + cy) * n[0] + cx;
      ++start[cell[i] + 1];
    }
    for (size_t k = 0; k < nc; ++k) start[k + 1] += start[k];
    atoms.assign(N, 0);
    std::vector<int32_t> fill(start.begin(), start.end() - 1);
    for (int32_t i = 0; i < N; ++i) atoms[fill[cell[i]]++] = i;
  }
  // Atoms of every cell within Chebyshev cell distance S of cell (cx, cy, cz).
  void gather(int cx, int cy, int cz, int S, std::vector<int32_t>& out) const {
    out.clear();
    int lo3[3], hi3[3];
    const int cc[3] = {cx, cy, cz};
    for (int d = 0; d < 3; ++d) {
      if (periodic && 2 * S + 1 >= n[d]) {        // the whole dimension, each cell once
        lo3[d] = 0;
        hi3[d] = n[d] - 1;
      } else if (periodic) {
        lo3[d] = cc[d] - S;
        hi3[d] = cc[d] + S;
      } else {
        lo3[d] = std::max(0, cc[d] - S);
        hi3[d] = std::min(n[d] - 1, cc[d] + S);
      }
    }
    for (int z = lo3[2]; z <= hi3[2]; ++z)
      for (int y = lo3[1]; y <= hi3[1]; ++y)
        for (int x = lo3[0]; x <= hi3[0]; ++x) {
          const int wx = ((x % n[0]) + n[0]) % n[0], wy = ((y % n[1]) + n[1]) % n[1], wz = ((z % n[2]) + n[2]) % n[2];
          const size_t k = ((size_t)wz * n[1] + wy) * n[0] + wx;
          out.insert(out.end(), atoms.begin() + start[k], atoms.begin() + start[k + 1]);
        }
  }
};

// Squared (minimum-image) distance between atoms a and J.
inline double dist2(const double* p, int32_t a, int32_t J, const double* box) {
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    double x = p[3 * (size_t)a + d] - p[3 * (size_t)J + d];
    if (box) x -= box[d] * nearbyint(x / box[d]);
    s += x * x;
  }
  return s;
}

// Atoms within the distance of the kappa-th nearest atom to J (ascending
// index), found on the cell grid: cells are gathered in growing cubes around
// J's cell until they hold kappa atoms; the kappa-th smallest distance D among
// those bounds the true one, so one more gather of every cell within
// ceil(D / cell side) + 1 holds every atom of the region, and the kappa-th
// smallest distance there is exact.
void region_of(const gsk_ctx* h, const CellGrid& g, int32_t J, int32_t kappa, const double* box,
               std::vector<double>& d2, std::vector<int32_t>& cand, std::vector<int32_t>& out) {
  const int32_t N = h->n_atoms;
  const double* p = h->pos_caller.data();
  const int32_t k = std::min(kappa, N);
  const int cx = g.coord(p[3 * (size_t)J], 0), cy = g.coord(p[3 * (size_t)J + 1], 1),
            cz = g.coord(p[3 * (size_t)J + 2], 2);
  const int max_s = std::max(g.n[0], std::max(g.n[1], g.n[2]));
  int S = 1;
  for (;; ++S) {
    g.gather(cx, cy, cz, S, cand);
    if ((int32_t)cand.size() >= k || S >= max_s) break;
  }
  auto kth = [&]() {
    d2.resize(cand.size());
    for (size_t t = 0; t < cand.size(); ++t) d2[t] = dist2(p, cand[t], J, box);
    std::vector<double> tmp(d2);
    std::nth_element(tmp.begin(), tmp.begin() + (k - 1), tmp.end());
    return tmp[k - 1];
  };
  double cut = kth();
  const double cmin = std::min(g.side[0], std::min(g.side[1], g.side[2]));
  const int S2 = (int)ceil(sqrt(cut) / cmin) + 1;
  if (S2 > S) {
    g.gather(cx, cy, cz, std::min(S2, max_s), cand);
    cut = kth();
  }
  out.clear();
  for (size_t t = 0; t < cand.size(); ++t)
    if (d2[t] <= cut) out.push_back(cand[t]);
  std::sort(out.begin(), out.end());
}

}  // namespace

extern "C" {

int gsk_marnoldi_projected(gsk_handle h, const double* box, int32_t kappa, int32_t n_cols, const int32_t* cols,
                           int32_t nu, double mu, double kT, double* rho, double* ritz, double* weight,
                           double* charge, int32_t* rank, int32_t* m_local) {
  if (!h || kappa < 1 || n_cols < 0 || (n_cols > 0 && (!cols || !rho))) return GSK_EINVAL;
  if (h->pos_lib.empty()) return GSK_EINVAL;          // the region needs atom positions
  if (box)
    for (int d = 0; d < 3; ++d)
      if (!(box[d] > 0.0) || !isfinite(box[d])) return GSK_EINVAL;
  for (int32_t c = 0; c < n_cols; ++c)
    if (cols[c] < 0 || cols[c] >= h->M) return GSK_EINVAL;
  if (n_cols == 0) return GSK_OK;
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  int rc = ensure_host_side(h);
  if (rc != GSK_OK) return rc;

  std::vector<int32_t> glob2loc(h->M, -1);
  std::vector<double> d2;
  std::vector<int32_t> atoms, cand;
  CellGrid grid;
  grid.build(h->pos_caller.data(), h->n_atoms, box);
  int64_t full_off = 0;                                 // start of the batch in the full rho layout
  for (int32_t c0 = 0; c0 < n_cols; c0 += kBatch) {
    const int nb = std::min<int>(kBatch, n_cols - c0);
    // block-diagonal pencil of the batch's restricted problems
    std::vector<int64_t> rp(1, 0);
    std::vector<int32_t> ci, loc_off;
    std::vector<double> va, vb;
    std::vector<int8_t> loc_cnt;
    std::vector<int32_t> lcols(nb);
    std::vector<int64_t> scatter;                       // full entry -> local rho index or -1
    int32_t base = 0;
    int64_t lpat = 0;                                   // start of this column in the local rho layout
    for (int c = 0; c < nb; ++c) {
      const int32_t j = cols[c0 + c];
      const int32_t J = h->atom_of_row[j];
      region_of(h, grid, J, kappa, box, d2, cand, atoms);
      int32_t nloc = 0;
      for (int32_t a : atoms) {
        const int32_t f = h->atom_first_row[a], cnt = h->atom_first_row[a + 1] - f;
        loc_off.push_back(base + nloc);
        loc_cnt.push_back((int8_t)cnt);
        for (int32_t t = 0; t < cnt; ++t) glob2loc[f + t] = nloc + t;
        nloc += cnt;
      }
      if (m_local) m_local[c0 + c] = nloc;
      // rows of the restricted pencil (global order = local order)
      for (int32_t a : atoms) {
        const int32_t f = h->atom_first_row[a], cnt = h->atom_first_row[a + 1] - f;
        for (int32_t gi = f; gi < f + cnt; ++gi) {
          for (int64_t e = h->row_ptr[gi]; e < h->row_ptr[gi + 1]; ++e) {
            const int32_t l = glob2loc[h->col_idx[e]];
            if (l < 0) continue;
            ci.push_back(base + l);
            va.push_back(h->host_A64[h->csr_vpos[e]]);
            vb.push_back(h->host_B64[h->csr_vpos[e]]);
          }
          rp.push_back((int64_t)ci.size());
        }
      }
      lcols[c] = base + glob2loc[j];
      // where each entry of the full P(j) lands in the local layout
      int64_t kept = 0;
      for (int64_t e = h->row_ptr[j]; e < h->row_ptr[j + 1]; ++e)
        scatter.push_back(glob2loc[h->col_idx[e]] >= 0 ? lpat + kept++ : -1);
      lpat += kept;
      for (int32_t a : atoms) {
        const int32_t f = h->atom_first_row[a], cnt = h->atom_first_row[a + 1] - f;
        for (int32_t t = 0; t < cnt; ++t) glob2loc[f + t] = -1;
      }
      base += nloc;
    }
    gsk_csr Ac{base, rp.data(), ci.data(), va.data()};
    gsk_csr Bc{base, rp.data(), ci.data(), vb.data()};
    gsk_orbmap om{(int32_t)loc_off.size(), loc_off.data(), loc_cnt.data(), nullptr};
    gsk_handle t = nullptr;
    rc = gsk_create(&Ac, &Bc, &om, &t);
    if (rc != GSK_OK) return rc;
    const int64_t n_full = (int64_t)scatter.size();
    const size_t need = ((size_t)std::max<int64_t>(lpat, 1) * sizeof(double) + 255) / 256 * 256 +
                        (size_t)std::max<int64_t>(n_full, 1) * sizeof(int64_t);
    if (h->ws_proj.ensure(need) != cudaSuccess) {
      gsk_destroy(t);
      return GSK_ENOMEM;
    }
    double* d_local = h->ws_proj.as<double>();
    int64_t* d_idx = reinterpret_cast<int64_t*>(h->ws_proj.as<char>() +
                                                ((size_t)std::max<int64_t>(lpat, 1) * sizeof(double) + 255) / 256 * 256);
    rc = gsk_marnoldi(t, nb, lcols.data(), nu, mu, kT, d_local, 0, nullptr, nullptr,
                      ritz ? ritz + (size_t)c0 * nu : nullptr, weight ? weight + (size_t)c0 * nu : nullptr,
                      charge ? charge + (size_t)c0 * nu : nullptr, rank ? rank + c0 : nullptr);
    if (rc == GSK_OK && cudaSetDevice(h->device) != cudaSuccess) rc = GSK_ECUDA;
    if (rc == GSK_OK &&
        cudaMemcpy(d_idx, scatter.data(), n_full * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = GSK_ECUDA;
    if (rc == GSK_OK) {
      const int64_t blocks = std::min<int64_t>((n_full + 255) / 256, (int64_t)h->num_sms * 8);
      k_scatter_rho<<<(unsigned)std::max<int64_t>(blocks, 1), 256>>>(n_full, d_idx, d_local, rho + full_off);
      if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = GSK_ECUDA;
    }
    gsk_destroy(t);
    if (rc != GSK_OK) return rc;
    full_off += n_full;
  }
  return GSK_OK;
}

}  // extern "C"
