// mlp.cu -- training of the branching network on the GPU: forward on the
// tensor cores, softmax cross-entropy per decision node, backward (dW1 on the
// tensor cores as X^T * dH), Adam with FP32 master weights, BF16 packing.
//
// Training data are the decision traces of the plain search (scuba_trace):
// node k has rows [node_row[k], node_row[k] + node_nrows[k]) -- one row per
// variable unassigned at that decision -- and per-row targets counting the
// variable's occurrences in falsified clauses of the node's subtree. The loss
// of a node is the cross-entropy between the normalised targets and the
// softmax of the scores over its rows.
//
// Master parameter layout (FP32, NPARAM = 1153): W1[i][j] at i*64 + j
// (i < 16 features, j < 64 hidden), b1[j] at 1024 + j, w2[j] at 1088 + j,
// b2 at 1152.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <string>

#include "../../include/scuba.h"
#include "learn.cuh"
#include "scuba_internal.h"

namespace scuba {
namespace mlpk {

using learn::MlpWeights;
using learn::NFEAT;
using learn::NHID;
using learn::NPARAM;
constexpr int OFF_B1 = NFEAT * NHID, OFF_W2 = OFF_B1 + NHID, OFF_B2 = OFF_W2 + NHID;
constexpr uint32_t FULL = 0xffffffffu;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// He-style initialisation from a counter-based stream (Box-Muller).
__global__ void k_init(float* master, uint64_t seed) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  float std = 0.0f;
  if (p < OFF_B1) std = sqrtf(2.0f / NFEAT);
  else if (p >= OFF_W2 && p < OFF_B2) std = sqrtf(1.0f / NHID);
  const uint64_t r1 = mix64(seed * 0x9E3779B97F4A7C15ULL + 2 * (uint64_t)p + 1);
  const uint64_t r2 = mix64(seed * 0x9E3779B97F4A7C15ULL + 2 * (uint64_t)p + 2);
  const float u1 = ((r1 >> 11) + 0.5f) * (1.0f / 9007199254740992.0f);
  const float u2 = (r2 >> 11) * (1.0f / 9007199254740992.0f);
  master[p] = std * sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// Packed weight of parameter p (BF16 matrices transposed as the solver
// reads them, FP32 biases).
__device__ __forceinline__ void pack_one(const float* master, MlpWeights* W, int p) {
  if (p < OFF_B1) {
    const int i = p / NHID, j = p % NHID;
    W->w1t[j * NFEAT + i] = __float2bfloat16(master[p]);
  } else if (p < OFF_W2) {
    W->b1[p - OFF_B1] = master[p];
  } else if (p < OFF_B2) {
    W->w2[p - OFF_W2] = __float2bfloat16(master[p]);
  } else if (p == OFF_B2) {
    W->b2 = master[p];
    W->pad[0] = W->pad[1] = W->pad[2] = 0.0f;
  }
}

__global__ void k_pack(const float* master, MlpWeights* W) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NPARAM) pack_one(master, W, p);
}

// Stage rows [r, r+16) of x (clipped to [lo, hi)) into a shared 16x16 tile.
__device__ __forceinline__ void stage_tile(const __nv_bfloat16* x, int64_t r, int64_t lo,
                                           int64_t hi, __nv_bfloat16* tile, int lane) {
  for (int k = lane; k < 16 * NFEAT; k += 32) {
    const int64_t row = r + k / NFEAT;
    tile[k] = (row >= lo && row < hi) ? x[row * NFEAT + (k % NFEAT)] : __float2bfloat16(0.0f);
  }
  __syncwarp();
}

// Scores of all rows [0, rows): one warp per 16-row tile (grid-stride).
__global__ void k_forward(const __nv_bfloat16* x, int64_t rows, const MlpWeights* W,
                          float* scores) {
  __shared__ __nv_bfloat16 tiles[8][16 * NFEAT];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nt = (rows + 15) / 16;
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; t < nt;
       t += (int64_t)gridDim.x * (blockDim.x >> 5)) {
    stage_tile(x, 16 * t, 0, rows, tiles[wib], lane);
    float lo, hi;
    learn::mlp_tile_scores(W, tiles[wib], lane, lo, hi);
    const int g = lane >> 2;
    if ((lane & 3) == 0) {
      if (16 * t + g < rows) scores[16 * t + g] = lo;
      if (16 * t + g + 8 < rows) scores[16 * t + g + 8] = hi;
    }
    __syncwarp();
  }
}

// Per node: scores of its rows, softmax, cross-entropy against normalised
// targets, dS = softmax - target. One warp per node.
__global__ void k_node_loss(const int64_t* node_row, const int32_t* node_nrows,
                            const int32_t* node_closed, int64_t k0, int64_t k1,
                            const __nv_bfloat16* x, const MlpWeights* W, const float* target,
                            float* dS, float* loss) {
  __shared__ __nv_bfloat16 tiles[8][16 * NFEAT];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int64_t k = k0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; k < k1;
       k += (int64_t)gridDim.x * (blockDim.x >> 5)) {
    const int64_t r0 = node_row[k];
    const int32_t n = node_nrows[k];
    float tsum = 0.0f;
    for (int i = lane; i < n; i += 32) tsum += target[r0 + i];
    for (int d = 16; d > 0; d >>= 1) tsum += __shfl_xor_sync(FULL, tsum, d);
    const bool use = node_closed[k] && n > 1 && tsum > 0.0f;
    if (!use) {
      for (int i = lane; i < n; i += 32) dS[r0 + i] = 0.0f;
      continue;
    }
    // scores into dS (as scratch), then the max
    for (int64_t r = r0; r < r0 + n; r += 16) {
      stage_tile(x, r, r0, r0 + n, tiles[wib], lane);
      float lo, hi;
      learn::mlp_tile_scores(W, tiles[wib], lane, lo, hi);
      const int g = lane >> 2;
      if ((lane & 3) == 0) {
        if (r + g < r0 + n) dS[r + g] = lo;
        if (r + g + 8 < r0 + n) dS[r + g + 8] = hi;
      }
      __syncwarp();
    }
    float mx = -INFINITY;
    for (int i = lane; i < n; i += 32) mx = fmaxf(mx, dS[r0 + i]);
    for (int d = 16; d > 0; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, d));
    float se = 0.0f;
    for (int i = lane; i < n; i += 32) se += expf(dS[r0 + i] - mx);
    for (int d = 16; d > 0; d >>= 1) se += __shfl_xor_sync(FULL, se, d);
    const float lse = mx + logf(se);
    float ce = 0.0f;
    for (int i = lane; i < n; i += 32) {
      const float s = dS[r0 + i];
      const float t = target[r0 + i] / tsum;
      ce -= t * (s - lse);
      dS[r0 + i] = expf(s - lse) - t;
    }
    for (int d = 16; d > 0; d >>= 1) ce += __shfl_xor_sync(FULL, ce, d);
    if (lane == 0) {
      atomicAdd(&loss[0], ce);
      atomicAdd(&loss[1], 1.0f);
    }
  }
}

// Gradients of the summed node losses with respect to every parameter.
// One block per node; warps stride over its 16-row tiles. dW1 = X^T dH runs
// on the tensor cores: A = X^T tile (features x rows), B = dH tile (rows x
// 8 hidden units) staged through shared memory in BF16.
__global__ void __launch_bounds__(128) k_backward(const int64_t* node_row,
                                                  const int32_t* node_nrows, int64_t k0,
                                                  const __nv_bfloat16* x, const MlpWeights* W,
                                                  const float* dS, float* grad) {
  __shared__ __nv_bfloat16 xt[4][16 * NFEAT];
  __shared__ __nv_bfloat16 dh_t[4][16 * NHID];
  __shared__ float gacc[NPARAM];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int p = threadIdx.x; p < NPARAM; p += blockDim.x) gacc[p] = 0.0f;
  __syncthreads();
  const int64_t k = k0 + blockIdx.x;
  const int64_t r0 = node_row[k];
  const int32_t n = node_nrows[k];
  float cw1[NHID / 8][4];
#pragma unroll
  for (int q = 0; q < NHID / 8; q++) cw1[q][0] = cw1[q][1] = cw1[q][2] = cw1[q][3] = 0.0f;
  float gw2[16], gb1[16], gb2 = 0.0f;
#pragma unroll
  for (int q = 0; q < 16; q++) gw2[q] = gb1[q] = 0.0f;
  for (int64_t r = r0 + 16 * wib; r < r0 + n; r += 16 * nw) {
    stage_tile(x, r, r0, r0 + n, xt[wib], lane);
    float z[4 * (NHID / 8)];
    float lo, hi;
    learn::mlp_tile_scores(W, xt[wib], lane, lo, hi, z);
    const float ds_lo = (r + g < r0 + n) ? dS[r + g] : 0.0f;
    const float ds_hi = (r + g + 8 < r0 + n) ? dS[r + g + 8] : 0.0f;
    if (t == 0) gb2 += ds_lo + ds_hi;
#pragma unroll
    for (int q = 0; q < NHID / 8; q++) {
      const int j0 = 8 * q + 2 * t;
      const float w0 = __bfloat162float(W->w2[j0]), w1 = __bfloat162float(W->w2[j0 + 1]);
      const float z0 = z[4 * q], z1 = z[4 * q + 1], z2 = z[4 * q + 2], z3 = z[4 * q + 3];
      gw2[2 * q] += fmaxf(z0, 0.f) * ds_lo + fmaxf(z2, 0.f) * ds_hi;
      gw2[2 * q + 1] += fmaxf(z1, 0.f) * ds_lo + fmaxf(z3, 0.f) * ds_hi;
      const float d0 = z0 > 0.f ? ds_lo * w0 : 0.f, d1 = z1 > 0.f ? ds_lo * w1 : 0.f;
      const float d2 = z2 > 0.f ? ds_hi * w0 : 0.f, d3 = z3 > 0.f ? ds_hi * w1 : 0.f;
      gb1[2 * q] += d0 + d2;
      gb1[2 * q + 1] += d1 + d3;
      __nv_bfloat16* dr = dh_t[wib];
      dr[g * NHID + j0] = __float2bfloat16(d0);
      dr[g * NHID + j0 + 1] = __float2bfloat16(d1);
      dr[(g + 8) * NHID + j0] = __float2bfloat16(d2);
      dr[(g + 8) * NHID + j0 + 1] = __float2bfloat16(d3);
    }
    __syncwarp();
    // A = X^T: A[i][row] = x[row][i]
    const __nv_bfloat16* xs = xt[wib];
    uint32_t a[4];
    a[0] = learn::pack_bf16(xs[(2 * t) * NFEAT + g], xs[(2 * t + 1) * NFEAT + g]);
    a[1] = learn::pack_bf16(xs[(2 * t) * NFEAT + g + 8], xs[(2 * t + 1) * NFEAT + g + 8]);
    a[2] = learn::pack_bf16(xs[(2 * t + 8) * NFEAT + g], xs[(2 * t + 9) * NFEAT + g]);
    a[3] = learn::pack_bf16(xs[(2 * t + 8) * NFEAT + g + 8], xs[(2 * t + 9) * NFEAT + g + 8]);
    const __nv_bfloat16* dr = dh_t[wib];
#pragma unroll
    for (int q = 0; q < NHID / 8; q++) {
      uint32_t b[2];
      b[0] = learn::pack_bf16(dr[(2 * t) * NHID + 8 * q + g], dr[(2 * t + 1) * NHID + 8 * q + g]);
      b[1] = learn::pack_bf16(dr[(2 * t + 8) * NHID + 8 * q + g],
                              dr[(2 * t + 9) * NHID + 8 * q + g]);
      learn::mma16816(cw1[q], a, b);
    }
    __syncwarp();
  }
  // reduce into shared, then global
  for (int q = 0; q < NHID / 8; q++) {
    const int j0 = 8 * q + 2 * t;
    atomicAdd(&gacc[g * NHID + j0], cw1[q][0]);
    atomicAdd(&gacc[g * NHID + j0 + 1], cw1[q][1]);
    atomicAdd(&gacc[(g + 8) * NHID + j0], cw1[q][2]);
    atomicAdd(&gacc[(g + 8) * NHID + j0 + 1], cw1[q][3]);
    atomicAdd(&gacc[OFF_W2 + j0], gw2[2 * q]);
    atomicAdd(&gacc[OFF_W2 + j0 + 1], gw2[2 * q + 1]);
    atomicAdd(&gacc[OFF_B1 + j0], gb1[2 * q]);
    atomicAdd(&gacc[OFF_B1 + j0 + 1], gb1[2 * q + 1]);
  }
  if (t == 0) atomicAdd(&gacc[OFF_B2], gb2);
  __syncthreads();
  for (int p = threadIdx.x; p < NPARAM; p += blockDim.x)
    if (gacc[p] != 0.0f) atomicAdd(&grad[p], gacc[p]);
}

// One training step after a minibatch's gradient: Adam (Kingma and Ba,
// Algorithm 1; beta 0.9/0.999, eps 1e-8) on the mean gradient over the
// minibatch's nodes, then the packed weight of each parameter, the epoch's
// loss sums, and the other gradient buffer cleared for the next minibatch
// (the two buffers alternate, so nothing here reads what it clears).
__global__ void k_adam_pack(float* master, float* m, float* v, const float* grad,
                            float* grad_next, MlpWeights* W, float lr, int step,
                            float* epoch_loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM + 2) return;
  grad_next[p] = 0.0f;
  if (p >= NPARAM) {
    if (epoch_loss) epoch_loss[p - NPARAM] += grad[p];  // summed loss, nodes used
    return;
  }
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float nodes = grad[NPARAM + 1];
  const float s = nodes > 0.0f ? 1.0f / nodes : 0.0f;  // mean over nodes
  const float gr = grad[p] * s;
  m[p] = b1 * m[p] + (1.0f - b1) * gr;
  v[p] = b2 * v[p] + (1.0f - b2) * gr * gr;
  const float mh = m[p] / (1.0f - powf(b1, (float)step));
  const float vh = v[p] / (1.0f - powf(b2, (float)step));
  master[p] -= lr * mh / (sqrtf(vh) + eps);
  pack_one(master, W, p);
}

}  // namespace mlpk

namespace {

struct TrainScratch {
  void* dS = nullptr;
  size_t dS_cap = 0;
  void* grad = nullptr;  // 2 x (NPARAM + 2): gradient, loss sum, nodes used (ping-pong)
};

std::map<int, TrainScratch>& train_scratch() {
  static std::map<int, TrainScratch> m;
  return m;
}

int fail(const char* what, cudaError_t e) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return SCUBA_ERR_CUDA;
}

}  // namespace
}  // namespace scuba

using namespace scuba;

extern "C" int scuba_mlp_layout(int64_t* out) {
  if (!out) return SCUBA_ERR_ARG;
  out[0] = (int64_t)sizeof(learn::MlpWeights);
  out[1] = learn::NPARAM;
  out[2] = learn::NFEAT;
  out[3] = learn::NHID;
  return SCUBA_OK;
}

extern "C" int scuba_mlp_init(float* master, void* weights, uint64_t seed, void* stream) {
  if (!master || !weights) return SCUBA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  mlpk::k_init<<<(learn::NPARAM + 255) / 256, 256, 0, st>>>(master, seed);
  mlpk::k_pack<<<(learn::NPARAM + 255) / 256, 256, 0, st>>>(
      master, static_cast<learn::MlpWeights*>(weights));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SCUBA_OK : fail("scuba_mlp_init", e);
}

extern "C" int scuba_mlp_pack(const float* master, void* weights, void* stream) {
  if (!master || !weights) return SCUBA_ERR_ARG;
  mlpk::k_pack<<<(learn::NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      master, static_cast<learn::MlpWeights*>(weights));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SCUBA_OK : fail("scuba_mlp_pack", e);
}

extern "C" int scuba_mlp_forward(const uint16_t* x, int64_t rows, const void* weights,
                                 float* scores, void* stream) {
  if (rows < 0 || (rows > 0 && (!x || !weights || !scores))) return SCUBA_ERR_ARG;
  if (rows == 0) return SCUBA_OK;
  const int64_t tiles = (rows + 15) / 16;
  const int grid = (int)std::min<int64_t>((tiles + 7) / 8, 65535);
  mlpk::k_forward<<<grid, 256, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const __nv_bfloat16*>(x), rows,
      static_cast<const learn::MlpWeights*>(weights), scores);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SCUBA_OK : fail("scuba_mlp_forward", e);
}

// The loss and gradient kernels of nodes [k0, k1) into grad (cleared by
// the caller): per-node softmax cross-entropy, then the backward pass.
static void grad_kernels(const scuba_trace* tr, int64_t k0, int64_t k1, const void* weights,
                         float* grad, float* dS, cudaStream_t st) {
  const int64_t nodes = k1 - k0;
  if (nodes <= 0) return;
  const int lgrid = (int)std::min<int64_t>((nodes + 7) / 8, 65535);
  mlpk::k_node_loss<<<lgrid, 256, 0, st>>>(
      tr->node_row, tr->node_nrows, tr->node_closed, k0, k1,
      reinterpret_cast<const __nv_bfloat16*>(tr->x),
      static_cast<const learn::MlpWeights*>(weights), tr->target, dS, grad + learn::NPARAM);
  for (int64_t b = 0; b < nodes; b += 65535) {
    const int64_t cnt = std::min<int64_t>(65535, nodes - b);
    mlpk::k_backward<<<(unsigned)cnt, 128, 0, st>>>(
        tr->node_row, tr->node_nrows, k0 + b, reinterpret_cast<const __nv_bfloat16*>(tr->x),
        static_cast<const learn::MlpWeights*>(weights), dS, grad);
  }
}

static int grad_impl(const scuba_trace* tr, int64_t k0, int64_t k1, const void* weights,
                     float* grad, float* dS, cudaStream_t st) {
  cudaMemsetAsync(grad, 0, sizeof(float) * (learn::NPARAM + 2), st);
  grad_kernels(tr, k0, k1, weights, grad, dS, st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SCUBA_OK : fail("scuba_mlp_grad", e);
}

extern "C" int scuba_mlp_grad(const scuba_trace* tr, int64_t node_begin, int64_t node_end,
                              const void* weights, float* grad, float* dS, void* stream) {
  if (!tr || !weights || !grad || !dS || node_begin < 0 || node_end < node_begin)
    return SCUBA_ERR_ARG;
  return grad_impl(tr, node_begin, node_end, weights, grad, dS, (cudaStream_t)stream);
}

extern "C" int scuba_mlp_train(const scuba_trace* tr, int64_t nodes, float* master, float* adam_m,
                               float* adam_v, void* weights, int32_t epochs, int32_t batch_nodes,
                               float lr, float* epoch_loss, void* stream) {
  if (!tr || !master || !adam_m || !adam_v || !weights || epochs < 0 || batch_nodes < 1 ||
      nodes < 0 || nodes > tr->max_nodes || !(lr > 0.0f))
    return SCUBA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  TrainScratch& S = train_scratch()[dev];
  const size_t need = sizeof(float) * (size_t)std::max<int64_t>(tr->max_rows, 1);
  if (S.dS_cap < need) {
    if (S.dS) cudaFree(S.dS);
    S.dS = nullptr;
    S.dS_cap = 0;
    if (cudaMalloc(&S.dS, need) != cudaSuccess) return SCUBA_ERR_NOMEM;
    S.dS_cap = need;
  }
  const size_t gwords = learn::NPARAM + 2;
  if (!S.grad && cudaMalloc(&S.grad, sizeof(float) * 2 * gwords) != cudaSuccess)
    return SCUBA_ERR_NOMEM;
  float* gbuf = static_cast<float*>(S.grad);
  float* dS = static_cast<float*>(S.dS);
  cudaMemsetAsync(adam_m, 0, sizeof(float) * learn::NPARAM, st);
  cudaMemsetAsync(adam_v, 0, sizeof(float) * learn::NPARAM, st);
  cudaMemsetAsync(gbuf, 0, sizeof(float) * 2 * gwords, st);
  if (epoch_loss) cudaMemsetAsync(epoch_loss, 0, sizeof(float) * 2 * (size_t)epochs, st);
  // three launches per minibatch: loss, backward, Adam + packing (which also
  // clears the other gradient buffer for the next minibatch)
  int step = 0;
  for (int ep = 0; ep < epochs; ep++) {
    for (int64_t k0 = 0; k0 < nodes; k0 += batch_nodes) {
      const int64_t k1 = std::min<int64_t>(nodes, k0 + batch_nodes);
      float* grad = gbuf + (size_t)(step & 1) * gwords;
      float* grad_next = gbuf + (size_t)((step + 1) & 1) * gwords;
      grad_kernels(tr, k0, k1, weights, grad, dS, st);
      step++;
      mlpk::k_adam_pack<<<(learn::NPARAM + 2 + 255) / 256, 256, 0, st>>>(
          master, adam_m, adam_v, grad, grad_next, static_cast<learn::MlpWeights*>(weights),
          lr, step, epoch_loss ? epoch_loss + 2 * ep : nullptr);
    }
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SCUBA_OK : fail("scuba_mlp_train", e);
}
