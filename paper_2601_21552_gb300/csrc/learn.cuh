// learn.cuh -- device pieces shared by the learned-branching search and the
// training kernels: the weight layout of the incidence MLP and its forward
// pass on the tensor cores (mma.sync m16n8k16, BF16 in, FP32 accumulate).
//
// The network scores one variable from NFEAT features of the residual formula
// (the clause-variable incidence around that variable, its activity and its
// place among the input bits): score = w2 . relu(W1 x + b1) + b2, with
// NFEAT = 16 inputs and NHID = 64 hidden units. It only orders decisions; the
// search stays a complete DPLL, so verdicts do not depend on it.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace scuba {
namespace learn {

constexpr int NFEAT = 16;
constexpr int NHID = 64;
constexpr int MAX_TRACE_DEPTH = 8;

// Packed weights in device memory (byte layout published in scuba.h).
struct MlpWeights {
  __nv_bfloat16 w1t[NHID * NFEAT];  // W1 transposed: w1t[j*NFEAT + i] = W1[i][j]
  __nv_bfloat16 w2[NHID];
  float b1[NHID];
  float b2;
  float pad[3];
};
static_assert(sizeof(MlpWeights) == 2048 + 128 + 256 + 16, "weight layout");

// Number of FP32 master parameters (W1, b1, w2, b2), in this order.
constexpr int NPARAM = NFEAT * NHID + NHID + NHID + 1;

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  uint32_t a = (uint32_t)__bfloat16_as_ushort(lo);
  uint32_t b = (uint32_t)__bfloat16_as_ushort(hi);
  return a | (b << 16);
}

// D = A(16x16, row-major) * B(16x8, col-major) + C, BF16 inputs, FP32 accumulate.
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment for rows [r0, r0+16) of a row-major [rows x NFEAT] BF16 tile.
// Lane layout of m16n8k16: g = lane/4 selects the row pair (g, g+8), t = lane%4
// the column pairs (2t, 2t+1) and (2t+8, 2t+9).
__device__ __forceinline__ void load_a(const __nv_bfloat16* x, int lane, uint32_t a[4]) {
  const int g = lane >> 2, t = lane & 3;
  const __nv_bfloat16* r0 = x + g * NFEAT;
  const __nv_bfloat16* r1 = x + (g + 8) * NFEAT;
  a[0] = pack_bf16(r0[2 * t], r0[2 * t + 1]);
  a[1] = pack_bf16(r1[2 * t], r1[2 * t + 1]);
  a[2] = pack_bf16(r0[2 * t + 8], r0[2 * t + 9]);
  a[3] = pack_bf16(r1[2 * t + 8], r1[2 * t + 9]);
}

// B fragment for hidden units [8n, 8n+8): B[k][col] = W1[k][8n+col].
__device__ __forceinline__ void load_b(const MlpWeights* W, int n, int lane, uint32_t b[2]) {
  const int g = lane >> 2, t = lane & 3;
  const __nv_bfloat16* col = W->w1t + (8 * n + g) * NFEAT;
  b[0] = pack_bf16(col[2 * t], col[2 * t + 1]);
  b[1] = pack_bf16(col[2 * t + 8], col[2 * t + 9]);
}

// Scores of the 16 rows of one tile. Every lane ends with the scores of rows
// g and g+8 (lane/4 = g). z (optional) receives the pre-activations in the
// mma output layout: z[4n + k] for hidden pair (8n + 2t, 8n + 2t + 1) of rows
// g (k = 0, 1) and g+8 (k = 2, 3).
__device__ __forceinline__ void mlp_tile_scores(const MlpWeights* W, const __nv_bfloat16* xtile,
                                                int lane, float& s_lo, float& s_hi,
                                                float* z = nullptr) {
  uint32_t a[4];
  load_a(xtile, lane, a);
  const int t = lane & 3;
  float p_lo = 0.f, p_hi = 0.f;
#pragma unroll
  for (int n = 0; n < NHID / 8; n++) {
    uint32_t b[2];
    load_b(W, n, lane, b);
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    mma16816(c, a, b);
    const int j0 = 8 * n + 2 * t, j1 = j0 + 1;
    const float z0 = c[0] + W->b1[j0], z1 = c[1] + W->b1[j1];
    const float z2 = c[2] + W->b1[j0], z3 = c[3] + W->b1[j1];
    if (z) {
      z[4 * n + 0] = z0;
      z[4 * n + 1] = z1;
      z[4 * n + 2] = z2;
      z[4 * n + 3] = z3;
    }
    const float w0 = __bfloat162float(W->w2[j0]), w1 = __bfloat162float(W->w2[j1]);
    p_lo += fmaxf(z0, 0.f) * w0 + fmaxf(z1, 0.f) * w1;
    p_hi += fmaxf(z2, 0.f) * w0 + fmaxf(z3, 0.f) * w1;
  }
  p_lo += __shfl_xor_sync(0xffffffffu, p_lo, 1);
  p_lo += __shfl_xor_sync(0xffffffffu, p_lo, 2);
  p_hi += __shfl_xor_sync(0xffffffffu, p_hi, 1);
  p_hi += __shfl_xor_sync(0xffffffffu, p_hi, 2);
  s_lo = p_lo + W->b2;
  s_hi = p_hi + W->b2;
}

}  // namespace learn
}  // namespace scuba
