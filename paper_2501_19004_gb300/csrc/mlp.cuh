// Warp-level BF16 tensor-core MLP (8 -> 32 -> 32 -> 1) shared by the
// predictor's inference (in the bucket selection) and training kernels.
// One warp evaluates 16 rows with mma.sync.m16n8k16 (bf16 x bf16 -> fp32):
// lane = 4 * g + t holds rows g and g + 8; a C fragment of n-tile j holds
// columns 8j + 2t and 8j + 2t + 1; two adjacent n-tiles of a layer's output
// form the A fragment of one 16-wide k-step of the next layer.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

namespace lv {

// parameter layout (floats)
constexpr int kW1 = 0;              // W1[8][32]
constexpr int kB1 = kW1 + 8 * 32;   // b1[32]
constexpr int kW2 = kB1 + 32;       // W2[32][32]
constexpr int kB2 = kW2 + 32 * 32;  // b2[32]
constexpr int kW3 = kB2 + 32;       // w3[32]
constexpr int kB3 = kW3 + 32;       // b3
constexpr int kMlpParams = kB3 + 1;  // 1377
constexpr int kFeatures = 8;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
  return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct MlpFrags {
  uint32_t b1f[4][2];     // layer 1 B fragments per n-tile (k rows 8..15 are zero)
  uint32_t b2f[2][4][2];  // layer 2 B fragments [k-step][n-tile]
  float bias1[4][2], bias2[4][2], w3[4][2];
  float b3;
};

__device__ __forceinline__ void mlp_load_frags(const float *p, MlpFrags &f, int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int n = 8 * j + g;
    f.b1f[j][0] = pack_bf16(p[kW1 + (2 * t) * 32 + n], p[kW1 + (2 * t + 1) * 32 + n]);
    f.b1f[j][1] = 0u;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int k0 = 16 * s + 2 * t;
      f.b2f[s][j][0] = pack_bf16(p[kW2 + k0 * 32 + n], p[kW2 + (k0 + 1) * 32 + n]);
      f.b2f[s][j][1] = pack_bf16(p[kW2 + (k0 + 8) * 32 + n], p[kW2 + (k0 + 9) * 32 + n]);
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int c = 8 * j + 2 * t + e;
      f.bias1[j][e] = p[kB1 + c];
      f.bias2[j][e] = p[kB2 + c];
      f.w3[j][e] = bf16r(p[kW3 + c]);
    }
  }
  f.b3 = p[kB3];
}

// Forward pass of 16 rows.  x0/x1: features 2t, 2t+1 of rows g and g+8.
// h1/h2: bf16-rounded ReLU outputs in C-fragment layout; l0/l1: logits of
// rows g and g+8 (valid in every lane of the quad).
__device__ __forceinline__ void mlp_tile_forward(const MlpFrags &f, const float (&x0)[2], const float (&x1)[2],
                                                 float (&h1)[4][4], float (&h2)[4][4], float &l0, float &l1, int t) {
  (void)t;
  const uint32_t a1[4] = {pack_bf16(x0[0], x0[1]), pack_bf16(x1[0], x1[1]), 0u, 0u};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float acc[4] = {f.bias1[j][0], f.bias1[j][1], f.bias1[j][0], f.bias1[j][1]};
    mma_bf16(acc, a1, f.b1f[j]);
#pragma unroll
    for (int e = 0; e < 4; ++e) h1[j][e] = bf16r(fmaxf(acc[e], 0.f));
  }
  uint32_t a2[2][4];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    a2[s][0] = pack_bf16(h1[2 * s][0], h1[2 * s][1]);
    a2[s][1] = pack_bf16(h1[2 * s][2], h1[2 * s][3]);
    a2[s][2] = pack_bf16(h1[2 * s + 1][0], h1[2 * s + 1][1]);
    a2[s][3] = pack_bf16(h1[2 * s + 1][2], h1[2 * s + 1][3]);
  }
  float p0 = 0.f, p1 = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float acc[4] = {f.bias2[j][0], f.bias2[j][1], f.bias2[j][0], f.bias2[j][1]};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const uint32_t a[4] = {a2[s][0], a2[s][1], a2[s][2], a2[s][3]};
      mma_bf16(acc, a, f.b2f[s][j]);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) h2[j][e] = bf16r(fmaxf(acc[e], 0.f));
    p0 += h2[j][0] * f.w3[j][0] + h2[j][1] * f.w3[j][1];
    p1 += h2[j][2] * f.w3[j][0] + h2[j][3] * f.w3[j][1];
  }
  p0 += __shfl_xor_sync(0xFFFFFFFFu, p0, 1);
  p1 += __shfl_xor_sync(0xFFFFFFFFu, p1, 1);
  p0 += __shfl_xor_sync(0xFFFFFFFFu, p0, 2);
  p1 += __shfl_xor_sync(0xFFFFFFFFu, p1, 2);
  l0 = p0 + f.b3;
  l1 = p1 + f.b3;
}

}  // namespace lv
