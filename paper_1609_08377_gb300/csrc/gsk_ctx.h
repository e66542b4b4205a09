// Host-side handle of libgsk (shared by the translation units of the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "gsk_common.cuh"

namespace gsk {

// Result of one gsk_autotune call: the pick and every candidate measured.
struct TuneRecord {
  int w = 0, kernel = 0, from_cache = 0, n_cand = 0;
  int cand_w[8] = {0}, cand_kernel[8] = {0};
  double cand_ms_per_step[8] = {0}, cand_estimate[8] = {0};
};

// Device buffer that grows on demand and is owned by the handle.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&ptr, need);
    if (e == cudaSuccess) bytes = need;
    return e;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
  }
  template <typename T>
  T* as() const { return static_cast<T*>(ptr); }
};

}  // namespace gsk

struct gsk_ctx {
  int device = 0;
  int32_t M = 0;
  int32_t n_atoms = 0;
  int64_t nnz = 0;        // stored entries of A (caller's pattern)
  int64_t n_vals = 0;     // values in the block layout (with padding)
  int32_t n_nbr = 0;      // neighbour entries of the block layout
  int num_sms = 0;

  // host-side maps
  std::vector<int64_t> row_ptr;     // caller's CSR pattern of A
  std::vector<int32_t> col_idx;
  std::vector<int32_t> row_lib;     // caller row -> library row
  std::vector<int64_t> csr_vpos;    // caller CSR entry -> value slot (block layout)
  std::vector<int32_t> atom_perm;   // library atom -> caller atom
  std::vector<int8_t> orb_lib;      // library atom -> orbital count
  std::vector<double> pos_lib;      // library atom -> xyz (empty without positions)
  std::vector<double> a_diag, b_diag, a_rowabs, b_rowabs;   // per caller row
  std::vector<int32_t> atom_of_row;   // caller row -> caller atom
  std::vector<int64_t> apat_ptr;      // caller atom pattern of A (CSR over atoms; built on first use)
  std::vector<int32_t> apat_idx;
  std::vector<double> host_A64, host_B64;   // block-layout values on the host (projection; on first use)
  std::vector<double> pos_caller;          // caller-order positions (projection; on first use)
  std::vector<int32_t> atom_first_row;     // first row of every caller atom, and M (projection)

  // device block layout
  gsk::Layout lay{};
  gsk::DevBuf d_atom_roff, d_atom_orb, d_nbr_ptr, d_nbr_mid, d_nbr_roff, d_val_ptr, d_warp_atoms;
  gsk::DevBuf d_A64, d_B64, d_A32, d_B32, d_A2, d_B2;   // FP64, FP32, FP32 pairs (hi, lo)

  // tiles of the staged SpMM (built at creation; n_tiles == 0: not available)
  gsk::TileArgs tiles{};
  gsk::DevBuf d_tile_head, d_box, d_loc, d_desc, d_order;
  int64_t tile_boxes = 0;  // row-run pieces of all row unions (statistics)

  gsk_stats last{};

  // learned scheduler
  gsk::DevBuf d_rowfeat;          // M x 14 static per-row features
  gsk::DevBuf d_sched_params;     // GSK_MLP_NPARAM floats
  gsk::DevBuf d_sched_norm;       // 2 * GSK_MLP_IN floats
  gsk::DevBuf ws_sched;           // feature / prediction scratch
  bool sched_ready = false;

  // autotuned lane width per precision mode (0: not tuned) and inner-CG
  // product kernel per precision mode and lane width 32 / 64 / 128 (0: not tuned)
  int tuned_w[3] = {0, 0, 0};
  int tuned_kernel[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  gsk::TuneRecord tune[3];     // the autotuner's last result per precision mode

  // solver workspace (grown on demand)
  gsk::DevBuf ws_vec;      // Lanczos / CG vectors
  gsk::DevBuf ws_lane;     // lane control block
  gsk::DevBuf ws_jobs;     // job arrays
  gsk::DevBuf ws_shift;    // shift recurrence state
  gsk::DevBuf ws_gstage;   // staging of G for host output buffers
  gsk::DevBuf ws_misc;     // density / trace scratch
  gsk::DevBuf ws_tune;     // G of the autotuner's truncated solves
  gsk::DevBuf ws_ma;       // multiple Arnoldi: vectors, Grams, small matrices
  gsk::DevBuf ws_proj;     // real-space projection: local rho and scatter map

  ~gsk_ctx() {
    gsk::DevBuf* all[] = {&d_atom_roff, &d_atom_orb, &d_nbr_ptr, &d_nbr_mid, &d_nbr_roff, &d_val_ptr, &d_warp_atoms,
                          &d_A64, &d_B64, &d_A32, &d_B32, &d_A2, &d_B2, &ws_vec, &ws_lane, &ws_jobs,
                          &ws_shift, &ws_gstage, &ws_misc, &d_rowfeat, &d_sched_params, &d_sched_norm, &ws_sched, &ws_tune, &ws_ma, &ws_proj,
                          &d_tile_head, &d_box, &d_loc, &d_desc, &d_order};
    for (auto* b : all) b->release();
  }
};

namespace gsk {
inline size_t align_up_sz(size_t x, size_t a) { return (x + a - 1) / a * a; }
void build_row_features(const gsk_csr* A, const gsk_csr* B, const gsk_orbmap* map, std::vector<float>& out);
int learned_order(gsk_ctx* h, int32_t n_cols, const int32_t* cols, const double* eta_cols, cudaStream_t s,
                  std::vector<int32_t>& queue);
int solve_impl(gsk_ctx* h, int32_t S, const double* z, const double* eta, int32_t n_cols,
               const int32_t* cols, const gsk_options* opt, double* G, int32_t* iters,
               int32_t* status, double* resid);
int autotune_impl(gsk_ctx* h, int32_t S, const double* z, const double* eta, int32_t n_cols, const int32_t* cols,
                  const gsk_options* opt, int32_t* best_w);
int spmm_impl(gsk_ctx* h, int32_t which, int32_t precision, int32_t W, const void* X, void* Y, int32_t n_rep,
              void* stream);
size_t spmm64_ws_bytes(const gsk_ctx* h);
// Host plan of the staged SpMM's tiles (see TileArgs), from the host copy of
// the block layout (atoms in library order).
struct TilePlan {
  int32_t n_tiles = 0, x_cap = 0, own_cap = 0, v_cap = 0, l_cap = 0, d_cap = 0;
  std::vector<int32_t> tile_atom;     // n_tiles + 1 (atom ranges, for checks)
  std::vector<TileHead> head;
  std::vector<int2> box;
  std::vector<int16_t> loc;
  std::vector<int4> desc;
  std::vector<int32_t> desc_atom;     // library atom of each descriptor (for checks)
};
// Returns GSK_OK, or GSK_ENOTSUP when one atom alone exceeds a capacity.
int plan_tiles(const std::vector<int32_t>& roff, const std::vector<int8_t>& orb,
               const std::vector<int32_t>& nbr_ptr, const std::vector<int32_t>& nbr_mid,
               const std::vector<int32_t>& nbr_atom, const std::vector<int64_t>& val_ptr, int64_t n_vals,
               TilePlan& plan);
// Tiles of the staged SpMM uploaded to the handle. Returns GSK_OK,
// GSK_ENOTSUP (see plan_tiles), GSK_ENOMEM or GSK_ECUDA.
int build_tiles(gsk_ctx* h, const std::vector<int32_t>& roff, const std::vector<int8_t>& orb,
                const std::vector<int32_t>& nbr_ptr, const std::vector<int32_t>& nbr_mid,
                const std::vector<int32_t>& nbr_atom, const std::vector<int64_t>& val_ptr, int64_t n_vals);

int spmm64_dot(gsk_ctx* h, int which, int W, const double* X, double* Y, double* dots, void* ws, cudaStream_t s);
}
