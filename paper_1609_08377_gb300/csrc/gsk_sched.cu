// Learned column scheduler of libgsk: per-column features, a 16 -> 64 -> 64 -> 1
// tanh MLP (FP32) that predicts log(Lanczos steps) of a column, its training
// (forward, backward, Adam) and its use as the work-queue order of gsk_solve
// (longest predicted column first). Motivation: the load imbalance from
// structural disorder reported for the polymer runs (Sec. IV-C of the paper).
//
// Parameter layout (one flat FP32 vector): W1 [64][16], b1 [64], W2 [64][64],
// b2 [64], w3 [64], b3 [1]. Feature normalisation: 32 floats, mean[16] then
// std[16]; the network sees (x - mean) / std.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "gsk_common.cuh"
#include "gsk_ctx.h"

namespace {

constexpr int NI = GSK_MLP_IN;
constexpr int NH = GSK_MLP_HIDDEN;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + NH * NI;
constexpr int OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH;
constexpr int OFF_B3 = OFF_W3 + NH;
constexpr int NPARAM = OFF_B3 + 1;
static_assert(NPARAM == GSK_MLP_NPARAM, "parameter count");
constexpr int TILE = 32;          // samples per tile of the MLP kernels
constexpr int kTrainCtas = 128;   // CTAs of the gradient kernel

// Features of the requested columns: log(eta), 0.1/eta, then the 14 static
// per-row descriptors computed at handle creation.
__global__ void k_features(int n, const int32_t* cols, const double* eta, const float* rowfeat, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double e = eta[c];
  float* o = out + (size_t)c * NI;
  o[0] = (float)log(e);
  o[1] = (float)(0.1 / e);
  const float* r = rowfeat + (size_t)cols[c] * (NI - 2);
#pragma unroll
  for (int k = 0; k < NI - 2; ++k) o[2 + k] = r[k];
}

// Forward pass of one tile of samples by a CTA of NH threads (thread i = hidden
// unit i). Leaves x, h1, h2 of the tile in shared memory and returns y for
// sample s in y[s] (valid after the call for s < cnt).
struct TileSmem {
  float W1[NH * NI];
  float W2[NH * NH];
  float b1[NH], b2[NH], w3[NH];
  float x[TILE][NI];
  float h1[TILE][NH];
  float h2[TILE][NH];
  float y[TILE];
  float red[TILE][2];
};

__device__ void load_params(TileSmem& sm, const float* p) {
  for (int t = threadIdx.x; t < NH * NI; t += blockDim.x) sm.W1[t] = p[OFF_W1 + t];
  for (int t = threadIdx.x; t < NH * NH; t += blockDim.x) sm.W2[t] = p[OFF_W2 + t];
  for (int t = threadIdx.x; t < NH; t += blockDim.x) {
    sm.b1[t] = p[OFF_B1 + t];
    sm.b2[t] = p[OFF_B2 + t];
    sm.w3[t] = p[OFF_W3 + t];
  }
}

__device__ void tile_forward(TileSmem& sm, const float* feat, const float* norm, int s0, int cnt, float b3) {
  const int i = threadIdx.x;
  for (int t = threadIdx.x; t < TILE * NI; t += blockDim.x) {
    const int s = t / NI, k = t % NI;
    sm.x[s][k] = (s < cnt) ? (feat[(size_t)(s0 + s) * NI + k] - norm[k]) / norm[NI + k] : 0.f;
  }
  __syncthreads();
  for (int s = 0; s < TILE; ++s) {
    float z = sm.b1[i];
#pragma unroll
    for (int k = 0; k < NI; ++k) z = fmaf(sm.W1[i * NI + k], sm.x[s][k], z);
    sm.h1[s][i] = tanhf(z);
  }
  __syncthreads();
  for (int s = 0; s < TILE; ++s) {
    float z = sm.b2[i];
#pragma unroll 8
    for (int k = 0; k < NH; ++k) z = fmaf(sm.W2[i * NH + k], sm.h1[s][k], z);
    sm.h2[s][i] = tanhf(z);
  }
  __syncthreads();
  // y[s] = w3 . h2[s] + b3: warp w sums samples s = w, w + 2, ... (fixed order)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s = warp; s < TILE; s += NH / 32) {
    float acc = sm.w3[lane] * sm.h2[s][lane] + sm.w3[lane + 32] * sm.h2[s][lane + 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sm.y[s] = acc + b3;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NH) k_mlp_forward(int n, const float* feat, const float* norm, const float* p,
                                                     float* y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem& sm = *reinterpret_cast<TileSmem*>(smem_raw);
  load_params(sm, p);
  const float b3 = p[OFF_B3];
  __syncthreads();
  for (int s0 = blockIdx.x * TILE; s0 < n; s0 += gridDim.x * TILE) {
    const int cnt = min(TILE, n - s0);
    tile_forward(sm, feat, norm, s0, cnt, b3);
    if ((int)threadIdx.x < cnt) y[s0 + threadIdx.x] = sm.y[threadIdx.x];
    __syncthreads();
  }
}

// Per-CTA partial gradients of L = (1/n) sum (y - t)^2 (and partial loss).
// Thread i owns row i of dW1 (16) and of dW2 (64) plus db1[i], db2[i], dw3[i].
__global__ void __launch_bounds__(NH) k_mlp_grad(int n, const float* feat, const float* norm, const float* target,
                                                  const float* p, float* partial /* kTrainCtas x (NPARAM + 1) */) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem& sm = *reinterpret_cast<TileSmem*>(smem_raw);
  __shared__ float dz2[TILE][NH];
  load_params(sm, p);
  const float b3 = p[OFF_B3];
  __syncthreads();
  const int i = threadIdx.x;
  float gW1[NI], gW2[NH];
#pragma unroll
  for (int k = 0; k < NI; ++k) gW1[k] = 0.f;
#pragma unroll
  for (int k = 0; k < NH; ++k) gW2[k] = 0.f;
  float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, lsum = 0.f;
  const float inv_n = 1.0f / (float)n;
  for (int s0 = blockIdx.x * TILE; s0 < n; s0 += gridDim.x * TILE) {
    const int cnt = min(TILE, n - s0);
    tile_forward(sm, feat, norm, s0, cnt, b3);
    // dy, loss (thread s handles sample s; lanes >= cnt contribute zero)
    if (i < TILE) {
      const float r = (i < cnt) ? sm.y[i] - target[s0 + i] : 0.f;
      sm.red[i][0] = 2.f * r * inv_n;
      sm.red[i][1] = r * r;
    }
    __syncthreads();
    for (int s = 0; s < cnt; ++s) {
      const float dy = sm.red[s][0];
      const float h2 = sm.h2[s][i];
      gw3 = fmaf(dy, h2, gw3);
      dz2[s][i] = dy * sm.w3[i] * (1.f - h2 * h2);
    }
    if (i == 0)
      for (int s = 0; s < cnt; ++s) {
        gb3 += sm.red[s][0];
        lsum += sm.red[s][1];
      }
    __syncthreads();
    for (int s = 0; s < cnt; ++s) {
      const float d2 = dz2[s][i];
      gb2 += d2;
#pragma unroll
      for (int k = 0; k < NH; ++k) gW2[k] = fmaf(d2, sm.h1[s][k], gW2[k]);
      // dz1[s][i] = (sum_m dz2[s][m] W2[m][i]) (1 - h1[s][i]^2)
      float a = 0.f;
#pragma unroll 8
      for (int m = 0; m < NH; ++m) a = fmaf(dz2[s][m], sm.W2[m * NH + i], a);
      const float h1 = sm.h1[s][i];
      const float d1 = a * (1.f - h1 * h1);
      gb1 += d1;
#pragma unroll
      for (int k = 0; k < NI; ++k) gW1[k] = fmaf(d1, sm.x[s][k], gW1[k]);
    }
    __syncthreads();
  }
  float* out = partial + (size_t)blockIdx.x * (NPARAM + 1);
#pragma unroll
  for (int k = 0; k < NI; ++k) out[OFF_W1 + i * NI + k] = gW1[k];
#pragma unroll
  for (int k = 0; k < NH; ++k) out[OFF_W2 + i * NH + k] = gW2[k];
  out[OFF_B1 + i] = gb1;
  out[OFF_B2 + i] = gb2;
  out[OFF_W3 + i] = gw3;
  if (i == 0) {
    out[OFF_B3] = gb3;
    out[NPARAM] = lsum;
  }
}

// Fixed-order sum of the partial gradients, then one Adam step (Kingma and Ba,
// ICLR 2015, with bias correction). grad (optional) receives the gradient,
// loss (optional) the mean squared error before the step.
__global__ void k_mlp_adam(int nparts, int n, const float* partial, float* p, float* m, float* v, int t, float lr,
                           float b1, float b2, float eps, float* grad, float* loss) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k <= NPARAM) {
    float g = 0.f;
    for (int b = 0; b < nparts; ++b) g += partial[(size_t)b * (NPARAM + 1) + k];
    if (k == NPARAM) {
      if (loss) *loss = g / (float)n;
      return;
    }
    if (grad) grad[k] = g;
    if (t > 0) {
      const float mk = b1 * m[k] + (1.f - b1) * g;
      const float vk = b2 * v[k] + (1.f - b2) * g * g;
      m[k] = mk;
      v[k] = vk;
      const float mh = mk / (1.f - powf(b1, (float)t));
      const float vh = vk / (1.f - powf(b2, (float)t));
      p[k] -= lr * mh / (sqrtf(vh) + eps);
    }
  }
}

size_t tile_smem() { return sizeof(TileSmem); }

}  // namespace

namespace gsk {

// Static per-row descriptors (features 2..15) of every row, caller order,
// from the caller's CSR matrices (called during gsk_create).
void build_row_features(const gsk_csr* A, const gsk_csr* B, const gsk_orbmap* map, std::vector<float>& out) {
  const int32_t M = A->n_rows;
  const int32_t n_atoms = map->n_atoms;
  out.assign((size_t)M * (NI - 2), 0.f);
  std::vector<int32_t> atom_of_row(M);
  for (int32_t I = 0; I < n_atoms; ++I)
    for (int a = 0; a < map->orb_count[I]; ++a) atom_of_row[map->orb_offset[I] + a] = I;
  std::vector<int32_t> seen(n_atoms, -1);
  for (int32_t I = 0; I < n_atoms; ++I) {
    int n4 = 0, n1 = 0;
    for (int a = 0; a < map->orb_count[I]; ++a) {
      const int32_t row = map->orb_offset[I] + a;
      for (int64_t e = A->row_ptr[row]; e < A->row_ptr[row + 1]; ++e) {
        const int32_t J = atom_of_row[A->col_idx[e]];
        if (J == I || seen[J] == I) continue;
        seen[J] = I;
        (map->orb_count[J] == 4 ? n4 : n1)++;
      }
    }
    for (int a = 0; a < map->orb_count[I]; ++a) {
      const int32_t j = map->orb_offset[I] + a;
      double aoff = 0.0, boff = 0.0, a2 = 0.0, aall = 0.0, ajj = 0.0, bjj = 0.0;
      for (int64_t e = A->row_ptr[j]; e < A->row_ptr[j + 1]; ++e) {
        aall += fabs(A->val[e]);
        if (A->col_idx[e] == j) {
          ajj = A->val[e];
          bjj = B->val[e];
          continue;
        }
        aoff += fabs(A->val[e]);
        boff += fabs(B->val[e]);
        a2 += A->val[e] * A->val[e];
      }
      float* o = out.data() + (size_t)j * (NI - 2);
      o[0] = (float)((A->row_ptr[j + 1] - A->row_ptr[j]) / 100.0);
      o[1] = (float)((n4 + n1) / 50.0);
      o[2] = (float)(n4 / 20.0);
      o[3] = (float)(n1 / 40.0);
      o[4] = map->orb_count[I] == 4 ? 1.f : 0.f;
      o[5] = (float)(a / 3.0);
      o[6] = (float)(ajj / 10.0);
      o[7] = (float)(aoff / 10.0);
      o[8] = (float)boff;
      o[9] = (float)(sqrt(a2) / 10.0);
      o[10] = (float)(ajj * ajj / 100.0);
      o[11] = (float)bjj;
      o[12] = (float)log1p(aall);
      o[13] = 1.f;
    }
  }
}

// Queue order of a learned-scheduled solve: longest predicted column first
// (ties in the given order). Returns a GSK code.
int learned_order(gsk_ctx* h, int32_t n_cols, const int32_t* cols, const double* eta_cols, cudaStream_t s,
                  std::vector<int32_t>& queue) {
  if (!h->sched_ready) return GSK_EINVAL;
  const size_t need = align_up_sz((size_t)n_cols * sizeof(int32_t), 256) + align_up_sz((size_t)n_cols * 8, 256) +
                      align_up_sz((size_t)n_cols * NI * sizeof(float), 256) +
                      align_up_sz((size_t)n_cols * sizeof(float), 256);
  if (h->ws_sched.ensure(need) != cudaSuccess) return GSK_ENOMEM;
  char* b = h->ws_sched.as<char>();
  int32_t* d_cols = reinterpret_cast<int32_t*>(b);
  b += align_up_sz((size_t)n_cols * sizeof(int32_t), 256);
  double* d_eta = reinterpret_cast<double*>(b);
  b += align_up_sz((size_t)n_cols * 8, 256);
  float* d_feat = reinterpret_cast<float*>(b);
  b += align_up_sz((size_t)n_cols * NI * sizeof(float), 256);
  float* d_y = reinterpret_cast<float*>(b);
  cudaError_t e = cudaMemcpyAsync(d_cols, cols, n_cols * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_eta, eta_cols, n_cols * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return GSK_ECUDA;
  k_features<<<(n_cols + 127) / 128, 128, 0, s>>>(n_cols, d_cols, d_eta, h->d_rowfeat.as<float>(), d_feat);
  const int grid = std::max(1, std::min((n_cols + TILE - 1) / TILE, h->num_sms * 4));
  k_mlp_forward<<<grid, NH, tile_smem(), s>>>(n_cols, d_feat, h->d_sched_norm.as<float>(),
                                             h->d_sched_params.as<float>(), d_y);
  if (cudaGetLastError() != cudaSuccess) return GSK_ECUDA;
  std::vector<float> y(n_cols);
  e = cudaMemcpyAsync(y.data(), d_y, n_cols * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return GSK_ECUDA;
  queue.resize(n_cols);
  std::iota(queue.begin(), queue.end(), 0);
  std::stable_sort(queue.begin(), queue.end(), [&](int32_t a, int32_t c) { return y[a] > y[c]; });
  return GSK_OK;
}

}  // namespace gsk

extern "C" {

int gsk_features(gsk_handle h, int32_t n_cols, const int32_t* cols, const double* eta, float* feat,
                 void* stream) {
  if (!h || n_cols < 0 || (n_cols > 0 && (!cols || !eta || !feat))) return GSK_EINVAL;
  if (n_cols == 0) return GSK_OK;
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  for (int32_t c = 0; c < n_cols; ++c)
    if (cols[c] < 0 || cols[c] >= h->M || !(eta[c] > 0.0) || !isfinite(eta[c])) return GSK_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t need = gsk::align_up_sz((size_t)n_cols * sizeof(int32_t), 256) + (size_t)n_cols * 8 + 256;
  if (h->ws_sched.ensure(need) != cudaSuccess) return GSK_ENOMEM;
  int32_t* d_cols = h->ws_sched.as<int32_t>();
  double* d_eta = reinterpret_cast<double*>(h->ws_sched.as<char>() +
                                            gsk::align_up_sz((size_t)n_cols * sizeof(int32_t), 256));
  cudaError_t e = cudaMemcpyAsync(d_cols, cols, n_cols * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_eta, eta, n_cols * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return GSK_ECUDA;
  k_features<<<(n_cols + 127) / 128, 128, 0, s>>>(n_cols, d_cols, d_eta, h->d_rowfeat.as<float>(), feat);
  if (cudaGetLastError() != cudaSuccess) return GSK_ECUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? GSK_OK : GSK_ECUDA;
}

int gsk_mlp_forward(int32_t n, const float* feat, const float* norm, const float* params, float* y, void* stream) {
  if (n < 0 || (n > 0 && (!feat || !norm || !params || !y))) return GSK_EINVAL;
  if (n == 0) return GSK_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GSK_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = std::max(1, std::min((n + TILE - 1) / TILE, std::max(1, sms) * 4));
  k_mlp_forward<<<grid, NH, tile_smem(), s>>>(n, feat, norm, params, y);
  return cudaGetLastError() == cudaSuccess ? GSK_OK : GSK_ECUDA;
}

size_t gsk_mlp_workspace_bytes(int32_t n) {
  (void)n;
  return (size_t)kTrainCtas * (NPARAM + 1) * sizeof(float);
}

int gsk_mlp_train_step(int32_t n, const float* feat, const float* norm, const float* target, float* params,
                       float* adam_m, float* adam_v, int32_t t, float lr, float* grad, float* loss, void* work,
                       void* stream) {
  if (n < 1 || !feat || !norm || !target || !params || !work || t < 0) return GSK_EINVAL;
  if (t > 0 && (!adam_m || !adam_v || !(lr > 0.f))) return GSK_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = std::max(1, std::min(kTrainCtas, (n + TILE - 1) / TILE));
  float* partial = static_cast<float*>(work);
  k_mlp_grad<<<grid, NH, tile_smem(), s>>>(n, feat, norm, target, params, partial);
  k_mlp_adam<<<(NPARAM + 1 + 255) / 256, 256, 0, s>>>(grid, n, partial, params, adam_m, adam_v, t, lr, 0.9f,
                                                     0.999f, 1e-8f, grad, loss);
  return cudaGetLastError() == cudaSuccess ? GSK_OK : GSK_ECUDA;
}

int gsk_set_sched_model(gsk_handle h, const float* params, const float* norm) {
  if (!h || !params || !norm) return GSK_EINVAL;
  for (int k = 0; k < NPARAM; ++k)
    if (!isfinite(params[k])) return GSK_EINVAL;
  for (int k = 0; k < 2 * NI; ++k)
    if (!isfinite(norm[k]) || (k >= NI && !(norm[k] > 0.f))) return GSK_EINVAL;
  if (cudaSetDevice(h->device) != cudaSuccess) return GSK_ECUDA;
  if (h->d_sched_params.ensure(NPARAM * sizeof(float)) != cudaSuccess) return GSK_ENOMEM;
  if (h->d_sched_norm.ensure(2 * NI * sizeof(float)) != cudaSuccess) return GSK_ENOMEM;
  if (cudaMemcpy(h->d_sched_params.ptr, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->d_sched_norm.ptr, norm, 2 * NI * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return GSK_ECUDA;
  h->sched_ready = true;
  return GSK_OK;
}

}  // extern "C"
