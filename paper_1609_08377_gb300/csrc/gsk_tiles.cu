// Tiles of the staged block SpMM (host side).
//
// The inner CG products of the shifted solve (Sec. III-B: v = B^{-1} u at
// every Lanczos step) multiply B by 32..128 lane vectors. A plain gather reads
// every neighbour row once per atom that touches it -- about 53 times per row
// at the workloads' density and cutoff -- from L2, with one load chain per
// block and little memory-level parallelism. Here consecutive atoms of the
// space-filling-curve order form a tile whose neighbour-row union is copied
// into shared memory once, asynchronously, so a row is read from L2 about 12
// times per product and the arithmetic runs out of shared memory.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gsk_ctx.h"

namespace gsk {

namespace {

template <typename T>
cudaError_t upload_vec(DevBuf& b, const std::vector<T>& v) {
  const size_t bytes = std::max<size_t>(v.size() * sizeof(T), 16);
  cudaError_t e = b.ensure(bytes);
  if (e != cudaSuccess) return e;
  if (v.empty()) return cudaMemset(b.ptr, 0, bytes);
  return cudaMemcpy(b.ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

int plan_tiles(const std::vector<int32_t>& roff, const std::vector<int8_t>& orb,
               const std::vector<int32_t>& nbr_ptr, const std::vector<int32_t>& nbr_mid,
               const std::vector<int32_t>& nbr_atom, const std::vector<int64_t>& val_ptr, int64_t n_vals,
               TilePlan& P) {
  const int32_t N = (int32_t)orb.size();
  // shared-memory capacities of one CTA (32 lanes of FP32 = 128 B per row)
  P.x_cap = 448;
  P.own_cap = 64;
  P.v_cap = 5120;
  P.l_cap = 1536;
  P.d_cap = 64;                         // atoms per tile (and descriptors in shared memory)
  auto val_end = [&](int32_t I) { return I + 1 < N ? val_ptr[I + 1] : n_vals; };
  auto atom_of = [&](int32_t e, int32_t I) { return nbr_atom[e] < 0 ? I : nbr_atom[e]; };
  P.tile_atom.assign(1, 0);
  P.head.clear();
  P.box.clear();
  P.loc.clear();
  P.desc.clear();
  P.desc_atom.clear();
  std::vector<int32_t> uni, merged, nb;
  std::vector<int32_t> srow(N, -1);     // shared row of an atom's first row (current tile)

  int32_t t0 = 0;
  while (t0 < N) {
    uni.clear();
    int32_t t1 = t0;
    int x_rows = 0;
    while (t1 < N && t1 - t0 < P.d_cap) {
      // candidate union: current union + atom t1 + its neighbours
      nb.clear();
      nb.push_back(t1);
      for (int32_t e = nbr_ptr[t1]; e < nbr_ptr[t1 + 1]; ++e) nb.push_back(atom_of(e, t1));
      std::sort(nb.begin(), nb.end());
      nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
      merged.clear();
      std::set_union(uni.begin(), uni.end(), nb.begin(), nb.end(), std::back_inserter(merged));
      int rows = 0;
      for (int32_t J : merged) rows += orb[J];
      const int own_rows = roff[t1 + 1] - roff[t0];
      const int64_t nval = val_end(t1) - val_ptr[t0];
      const int32_t nloc = nbr_ptr[t1 + 1] - nbr_ptr[t0];
      const bool fits = rows <= P.x_cap && own_rows <= P.own_cap && nval <= P.v_cap &&
                        ((nloc + 7) / 8) * 8 <= P.l_cap;
      if (!fits) {
        if (t1 == t0) return GSK_ENOTSUP;     // one atom alone exceeds a capacity
        break;
      }
      uni.swap(merged);
      x_rows = rows;
      ++t1;
    }
    TileHead hd;
    memset(&hd, 0, sizeof(hd));
    hd.r0 = roff[t0];
    hd.n_own = roff[t1] - roff[t0];
    hd.n_atoms = t1 - t0;
    hd.b0 = (int32_t)P.box.size();
    hd.l0 = (int32_t)P.loc.size();
    hd.d0 = (int32_t)P.desc.size();
    hd.v0 = val_ptr[t0];
    hd.nval = (int32_t)(val_end(t1 - 1) - val_ptr[t0]);
    hd.xrows = x_rows;
    // row runs of the union -> boxes and shared rows
    int srow_next = 0;
    size_t a = 0;
    while (a < uni.size()) {
      size_t b = a + 1;
      while (b < uni.size() && uni[b] == uni[b - 1] + 1) ++b;
      const int r0 = roff[uni[a]];
      const int n = roff[uni[b - 1] + 1] - r0;
      for (size_t k = a; k < b; ++k) srow[uni[k]] = srow_next + (roff[uni[k]] - r0);
      // pieces of at most kPieceRows rows tile the run exactly
      for (int off = 0; off < n; off += kPieceRows)
        P.box.push_back(make_int2(r0 + off, (srow_next + off) | (std::min(kPieceRows, n - off) << 16)));
      srow_next += n;
      a = b;
    }
    hd.nbox = (int32_t)P.box.size() - hd.b0;
    // local indices of the neighbour entries, padded to 8 (16-byte bulk copies)
    for (int32_t I = t0; I < t1; ++I)
      for (int32_t e = nbr_ptr[I]; e < nbr_ptr[I + 1]; ++e) P.loc.push_back((int16_t)srow[atom_of(e, I)]);
    while (P.loc.size() % 8) P.loc.push_back(0);
    hd.nloc = (int32_t)P.loc.size() - hd.l0;
    // cost-balanced atom lists of the warps (longest processing time first)
    {
      std::vector<std::pair<double, int32_t>> cost;
      for (int32_t I = t0; I < t1; ++I) {
        const int n4 = nbr_mid[I] - nbr_ptr[I];
        const int n1 = nbr_ptr[I + 1] - nbr_mid[I];
        const double fma = (double)orb[I] * (4.0 * n4 + n1);
        const double blocks = (orb[I] == 4) ? (double)(n4 + n1) : (double)n4 + n1 / 4.0;
        cost.push_back({fma + 8.0 * blocks, I});
      }
      std::stable_sort(cost.begin(), cost.end(),
                       [](const std::pair<double, int32_t>& x, const std::pair<double, int32_t>& y) {
                         return x.first > y.first;
                       });
      double load[kTileWarps] = {0};
      std::vector<int32_t> lists[kTileWarps];
      for (const auto& c : cost) {
        int w = 0;
        for (int k = 1; k < kTileWarps; ++k)
          if (load[k] < load[w]) w = k;
        load[w] += c.first;
        lists[w].push_back(c.second);
      }
      // warp slots take the lists heaviest first on even tiles and lightest
      // first on odd ones: a warp runs at most one tile ahead of the slowest
      // (two stages), so alternating evens out each warp's load over a pair of
      // tiles instead of giving the same warps the 4-orbital atoms every time
      int order[kTileWarps];
      for (int w = 0; w < kTileWarps; ++w) order[w] = w;
      std::stable_sort(order, order + kTileWarps, [&](int x, int y) { return load[x] > load[y]; });
      if (P.head.size() & 1) std::reverse(order, order + kTileWarps);
      int nd = 0;
      for (int slot = 0; slot < kTileWarps; ++slot) {
        std::vector<int32_t>& lst = lists[order[slot]];
        std::sort(lst.begin(), lst.end());
        hd.wptr[slot] = (uint8_t)nd;
        for (int32_t I : lst) {
          const int n4 = nbr_mid[I] - nbr_ptr[I];
          const int n1 = nbr_ptr[I + 1] - nbr_mid[I];
          int4 d;
          d.x = orb[I] | ((roff[I] - roff[t0]) << 8) | (srow[I] << 16);
          d.y = n4 | (n1 << 16);
          d.z = (int32_t)(val_ptr[I] - val_ptr[t0]);
          d.w = nbr_ptr[I] - nbr_ptr[t0];
          P.desc.push_back(d);
          P.desc_atom.push_back(I);
          ++nd;
        }
      }
      hd.wptr[kTileWarps] = (uint8_t)nd;
    }
    for (size_t k = 0; k < uni.size(); ++k) srow[uni[k]] = -1;
    P.head.push_back(hd);
    P.tile_atom.push_back(t1);
    t0 = t1;
  }
  P.n_tiles = (int32_t)P.head.size();
  return GSK_OK;
}

int build_tiles(gsk_ctx* h, const std::vector<int32_t>& roff, const std::vector<int8_t>& orb,
                const std::vector<int32_t>& nbr_ptr, const std::vector<int32_t>& nbr_mid,
                const std::vector<int32_t>& nbr_atom, const std::vector<int64_t>& val_ptr, int64_t n_vals) {
  TilePlan P;
  const int rc = plan_tiles(roff, orb, nbr_ptr, nbr_mid, nbr_atom, val_ptr, n_vals, P);
  if (rc != GSK_OK) return rc;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload_vec(h->d_tile_head, P.head);
  if (e == cudaSuccess) e = upload_vec(h->d_box, P.box);
  if (e == cudaSuccess) e = upload_vec(h->d_loc, P.loc);
  if (e == cudaSuccess) e = upload_vec(h->d_desc, P.desc);
  if (e == cudaSuccess) e = upload_vec(h->d_order, P.desc_atom);
  if (e == cudaErrorMemoryAllocation) return GSK_ENOMEM;
  if (e != cudaSuccess) return GSK_ECUDA;
  TileArgs& t = h->tiles;
  t.n_tiles = P.n_tiles;
  t.x_cap = P.x_cap;
  t.own_cap = P.own_cap;
  t.v_cap = P.v_cap;
  t.l_cap = P.l_cap;
  t.d_cap = P.d_cap;
  t.head = h->d_tile_head.as<TileHead>();
  t.box = h->d_box.as<int2>();
  t.loc = h->d_loc.as<int16_t>();
  t.desc = h->d_desc.as<int4>();
  t.order = h->d_order.as<int32_t>();
#ifdef GSK_DEBUG
  t.n_box = (int32_t)P.box.size();
  t.n_loc = (int32_t)P.loc.size();
  t.n_desc = (int32_t)P.desc.size();
  t.n_vals = n_vals;
#endif
  h->tile_boxes = (int64_t)P.box.size();
  return GSK_OK;
}

}  // namespace gsk
