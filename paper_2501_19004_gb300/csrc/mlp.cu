// Learned vertex-activity predictor: an 8 -> 32 -> 32 -> 1 MLP with BF16
// operands and FP32 accumulation on the tensor cores (mma.sync m16n8k16).
// The paper has no counterpart; the predictor decides which flagged vertices
// of a bucket to evaluate in the local-moving phase (Algorithm 5).
//
// Parameters (fp32, kMlpParams floats): W1[8][32], b1[32], W2[32][32],
// b2[32], w3[32], b3 -- W[k][n] maps input k to output n.  Arithmetic, the
// same in every kernel here: x, W1, W2, w3 and the ReLU outputs h1, h2 are
// rounded to bf16 (round to nearest even); products are accumulated in
// fp32; biases stay fp32.  p = sigmoid(logit).
//
// Kernels
//   k_mlp_forward   16 samples per warp: logits (inference, tests);
//   k_mlp_grad      128 samples per block: forward on the tensor cores,
//                   backward of the mean binary cross-entropy (dlogit =
//                   (p - y)/N, ReLU masks), dh1 = dz2 W2^T on the tensor cores,
//                   weight gradients dW2 = h1^T dz2 and dW1 = x^T dz1 as
//                   tensor-core contractions over the samples (bf16 operands),
//                   bias gradients in fp32; every block sums its tiles in
//                   shared memory and writes one partial gradient;
//   k_mlp_reduce    adds the blocks' partials into `grad` in block order, so
//                   a gradient (and a training run) is the same bit for bit
//                   on every run;
//   k_mlp_adam      Adam update of the fp32 parameters.
#include <cuda_bf16.h>

#include "internal.h"
#include "mlp.cuh"

namespace lv {

int64_t mlp_param_count() { return kMlpParams; }

namespace {

constexpr int kGradSamples = 128;  // samples per block of k_mlp_grad (8 warps x 16)

// ------------------------------------------------------------- k_mlp_forward
__global__ void __launch_bounds__(256) k_mlp_forward(const float *params, const float *X, int64_t n, float *logit) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  MlpFrags f;
  mlp_load_frags(params, f, lane);
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 16 < n; tile += warps) {
    const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
    float x0[2] = {0.f, 0.f}, x1[2] = {0.f, 0.f};
    if (r0 < n) {
      x0[0] = X[r0 * 8 + 2 * t];
      x0[1] = X[r0 * 8 + 2 * t + 1];
    }
    if (r1 < n) {
      x1[0] = X[r1 * 8 + 2 * t];
      x1[1] = X[r1 * 8 + 2 * t + 1];
    }
    float h1[4][4], h2[4][4], l0, l1;
    mlp_tile_forward(f, x0, x1, h1, h2, l0, l1, t);
    if (t == 0) {
      if (r0 < n) logit[r0] = l0;
      if (r1 < n) logit[r1] = l1;
    }
  }
}

// --------------------------------------------------------------- k_mlp_grad
// Shared tiles per block (row = sample): x (bf16, 16 columns, 8 used), h1 and
// dz2 and dz1 (bf16, 32 columns); bias-gradient partials in fp32.
// Per-warp bias partials of a tile (each written by one lane), and the
// block's running gradient over its tiles (acc, loss).
struct GradSmem {
  __nv_bfloat16 x[kGradSamples][16];
  __nv_bfloat16 h1[kGradSamples][32];
  __nv_bfloat16 dz2[kGradSamples][32];
  __nv_bfloat16 dz1[kGradSamples][32];
  float db1[8][32], db2[8][32], dw3[8][32], db3[8], wloss[8];
  float acc[kMlpParams];
  float loss;
};

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16 *a, const __nv_bfloat16 *b) {
  __nv_bfloat162 v;
  v.x = *a;
  v.y = *b;
  return *reinterpret_cast<uint32_t *>(&v);
}

__global__ void __launch_bounds__(256) k_mlp_grad(const float *params, const float *X, const float *Y, int64_t n,
                                                  float scale, float *partial) {
  __shared__ GradSmem sm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  MlpFrags f;
  mlp_load_frags(params, f, lane);
  // W2 as a B operand of dh1 = dz2 W2^T: B[k = out][n = in] = W2[in][out]
  uint32_t bT[2][4][2];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nn = 8 * j + g;
      const int k0 = 16 * s + 2 * t;
      bT[s][j][0] = pack_bf16(params[kW2 + nn * 32 + k0], params[kW2 + nn * 32 + k0 + 1]);
      bT[s][j][1] = pack_bf16(params[kW2 + nn * 32 + k0 + 8], params[kW2 + nn * 32 + k0 + 9]);
    }
  for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) sm.acc[p] = 0.f;
  if (threadIdx.x == 0) sm.loss = 0.f;
  __syncthreads();
  for (int64_t base = (int64_t)blockIdx.x * kGradSamples; base < n; base += (int64_t)gridDim.x * kGradSamples) {
    // ---- per warp: 16 samples forward and backward to dz1 ----
    const int rl0 = warp * 16 + g, rl1 = rl0 + 8;  // rows within the block tile
    const int64_t r0 = base + rl0, r1 = base + rl1;
    const bool v0 = r0 < n, v1 = r1 < n;
    float x0[2] = {0.f, 0.f}, x1[2] = {0.f, 0.f};
    if (v0) {
      x0[0] = X[r0 * 8 + 2 * t];
      x0[1] = X[r0 * 8 + 2 * t + 1];
    }
    if (v1) {
      x1[0] = X[r1 * 8 + 2 * t];
      x1[1] = X[r1 * 8 + 2 * t + 1];
    }
    sm.x[rl0][2 * t] = __float2bfloat16_rn(x0[0]);
    sm.x[rl0][2 * t + 1] = __float2bfloat16_rn(x0[1]);
    sm.x[rl1][2 * t] = __float2bfloat16_rn(x1[0]);
    sm.x[rl1][2 * t + 1] = __float2bfloat16_rn(x1[1]);
    sm.x[rl0][8 + 2 * t] = __float2bfloat16_rn(0.f);
    sm.x[rl0][9 + 2 * t] = __float2bfloat16_rn(0.f);
    sm.x[rl1][8 + 2 * t] = __float2bfloat16_rn(0.f);
    sm.x[rl1][9 + 2 * t] = __float2bfloat16_rn(0.f);
    float h1[4][4], h2[4][4], l0, l1;
    mlp_tile_forward(f, x0, x1, h1, h2, l0, l1, t);
    const float y0 = v0 ? Y[r0] : 0.f, y1 = v1 ? Y[r1] : 0.f;
    const float p0 = 1.f / (1.f + __expf(-l0)), p1 = 1.f / (1.f + __expf(-l1));
    const float d0 = v0 ? (p0 - y0) * scale : 0.f, d1 = v1 ? (p1 - y1) * scale : 0.f;
    {
      // binary cross-entropy from the logit: max(l,0) - l*y + log(1 + exp(-|l|));
      // lanes with t == 0 hold the rows, summed over the 8 groups
      float ls = 0.f;
      if (t == 0 && v0) ls += fmaxf(l0, 0.f) - l0 * y0 + log1pf(__expf(-fabsf(l0)));
      if (t == 0 && v1) ls += fmaxf(l1, 0.f) - l1 * y1 + log1pf(__expf(-fabsf(l1)));
      float db = t == 0 ? d0 + d1 : 0.f;
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        ls += __shfl_xor_sync(0xFFFFFFFFu, ls, o);
        db += __shfl_xor_sync(0xFFFFFFFFu, db, o);
      }
      if (lane == 0) {
        sm.wloss[warp] = ls * scale;
        sm.db3[warp] = db;
      }
    }
    // dz2 = dlogit * w3 * [z2 > 0]; dw3 = sum dlogit * h2; db2 = sum dz2
    uint32_t adz2[2][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 8 * j + 2 * t;
      float dz[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float dl = e < 2 ? d0 : d1;
        dz[e] = h2[j][e] > 0.f ? dl * f.w3[j][e & 1] : 0.f;
      }
      // partial sums over this thread's two rows, then over the 8 groups
      float s_w3a = d0 * h2[j][0] + d1 * h2[j][2], s_w3b = d0 * h2[j][1] + d1 * h2[j][3];
      float s_b2a = dz[0] + dz[2], s_b2b = dz[1] + dz[3];
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        s_w3a += __shfl_xor_sync(0xFFFFFFFFu, s_w3a, o);
        s_w3b += __shfl_xor_sync(0xFFFFFFFFu, s_w3b, o);
        s_b2a += __shfl_xor_sync(0xFFFFFFFFu, s_b2a, o);
        s_b2b += __shfl_xor_sync(0xFFFFFFFFu, s_b2b, o);
      }
      if (g == 0) {
        sm.dw3[warp][c] = s_w3a;
        sm.dw3[warp][c + 1] = s_w3b;
        sm.db2[warp][c] = s_b2a;
        sm.db2[warp][c + 1] = s_b2b;
      }
      sm.dz2[rl0][c] = __float2bfloat16_rn(dz[0]);
      sm.dz2[rl0][c + 1] = __float2bfloat16_rn(dz[1]);
      sm.dz2[rl1][c] = __float2bfloat16_rn(dz[2]);
      sm.dz2[rl1][c + 1] = __float2bfloat16_rn(dz[3]);
      // C fragments of n-tiles (2s, 2s+1) form the A fragment of k-step s
      const int s = j >> 1, hi = j & 1;
      adz2[s][2 * hi + 0] = pack_bf16(dz[0], dz[1]);
      adz2[s][2 * hi + 1] = pack_bf16(dz[2], dz[3]);
    }
    // dh1 = dz2 W2^T on the tensor cores; dz1 = dh1 * [z1 > 0]; db1 = sum dz1
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const uint32_t a[4] = {adz2[s][0], adz2[s][1], adz2[s][2], adz2[s][3]};
        mma_bf16(acc, a, bT[s][j]);
      }
      const int c = 8 * j + 2 * t;
      float dz[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) dz[e] = h1[j][e] > 0.f ? acc[e] : 0.f;
      float s_a = dz[0] + dz[2], s_b = dz[1] + dz[3];
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        s_a += __shfl_xor_sync(0xFFFFFFFFu, s_a, o);
        s_b += __shfl_xor_sync(0xFFFFFFFFu, s_b, o);
      }
      if (g == 0) {
        sm.db1[warp][c] = s_a;
        sm.db1[warp][c + 1] = s_b;
      }
      sm.dz1[rl0][c] = __float2bfloat16_rn(dz[0]);
      sm.dz1[rl0][c + 1] = __float2bfloat16_rn(dz[1]);
      sm.dz1[rl1][c] = __float2bfloat16_rn(dz[2]);
      sm.dz1[rl1][c + 1] = __float2bfloat16_rn(dz[3]);
      sm.h1[rl0][c] = __float2bfloat16_rn(h1[j][0]);
      sm.h1[rl0][c + 1] = __float2bfloat16_rn(h1[j][1]);
      sm.h1[rl1][c] = __float2bfloat16_rn(h1[j][2]);
      sm.h1[rl1][c + 1] = __float2bfloat16_rn(h1[j][3]);
    }
    __syncthreads();
    // ---- weight gradients: contractions over the block's 128 samples ----
    // warps 0..7: dW2 (32 x 32) tile (mt = warp >> 2, nt = warp & 3);
    // warps 0..3 also: dW1 (16 x 32, rows 0..7 real) tile nt = warp.
    {
      const int mt = warp >> 2, nt = warp & 3;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < kGradSamples / 16; ++ks) {
        const int k0 = 16 * ks + 2 * t;
        const int m0 = 16 * mt + g;
        // A[m][k] = h1[sample k][feature m]
        const uint32_t a[4] = {ld_pair(&sm.h1[k0][m0], &sm.h1[k0 + 1][m0]),
                               ld_pair(&sm.h1[k0][m0 + 8], &sm.h1[k0 + 1][m0 + 8]),
                               ld_pair(&sm.h1[k0 + 8][m0], &sm.h1[k0 + 9][m0]),
                               ld_pair(&sm.h1[k0 + 8][m0 + 8], &sm.h1[k0 + 9][m0 + 8])};
        // B[k][n] = dz2[sample k][feature n]
        const int n0 = 8 * nt + g;
        const uint32_t b[2] = {ld_pair(&sm.dz2[k0][n0], &sm.dz2[k0 + 1][n0]),
                               ld_pair(&sm.dz2[k0 + 8][n0], &sm.dz2[k0 + 9][n0])};
        mma_bf16(acc, a, b);
      }
      const int row = 16 * mt + g, col = 8 * nt + 2 * t;  // every element has one owner lane
      sm.acc[kW2 + row * 32 + col] += acc[0];
      sm.acc[kW2 + row * 32 + col + 1] += acc[1];
      sm.acc[kW2 + (row + 8) * 32 + col] += acc[2];
      sm.acc[kW2 + (row + 8) * 32 + col + 1] += acc[3];
    }
    if (warp < 4) {
      const int nt = warp;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < kGradSamples / 16; ++ks) {
        const int k0 = 16 * ks + 2 * t;
        const uint32_t a[4] = {ld_pair(&sm.x[k0][g], &sm.x[k0 + 1][g]), ld_pair(&sm.x[k0][g + 8], &sm.x[k0 + 1][g + 8]),
                               ld_pair(&sm.x[k0 + 8][g], &sm.x[k0 + 9][g]),
                               ld_pair(&sm.x[k0 + 8][g + 8], &sm.x[k0 + 9][g + 8])};
        const int n0 = 8 * nt + g;
        const uint32_t b[2] = {ld_pair(&sm.dz1[k0][n0], &sm.dz1[k0 + 1][n0]),
                               ld_pair(&sm.dz1[k0 + 8][n0], &sm.dz1[k0 + 9][n0])};
        mma_bf16(acc, a, b);
      }
      const int row = g, col = 8 * nt + 2 * t;  // rows 8..15 are the zero padding
      sm.acc[kW1 + row * 32 + col] += acc[0];
      sm.acc[kW1 + row * 32 + col + 1] += acc[1];
    }
    // bias partials of the tile, warps summed in order
    if (threadIdx.x < 32) {
      float b1 = 0.f, b2 = 0.f, w3 = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        b1 += sm.db1[w][threadIdx.x];
        b2 += sm.db2[w][threadIdx.x];
        w3 += sm.dw3[w][threadIdx.x];
      }
      sm.acc[kB1 + threadIdx.x] += b1;
      sm.acc[kB2 + threadIdx.x] += b2;
      sm.acc[kW3 + threadIdx.x] += w3;
    }
    if (threadIdx.x == 32) {
      float b3 = 0.f, ls = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        b3 += sm.db3[w];
        ls += sm.wloss[w];
      }
      sm.acc[kB3] += b3;
      sm.loss += ls;
    }
    __syncthreads();
  }
  float *out = partial + (int64_t)blockIdx.x * (kMlpParams + 1);
  for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) out[p] = sm.acc[p];
  if (threadIdx.x == 0) out[kMlpParams] = sm.loss;
}

// grad[p] += sum over blocks b (in order) of partial[b][p]; likewise the loss.
__global__ void k_mlp_reduce(const float *partial, int blocks, float *grad, float *loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kMlpParams) return;
  float sum = 0.f;
  for (int b = 0; b < blocks; ++b) sum += partial[(int64_t)b * (kMlpParams + 1) + p];
  if (p < kMlpParams) grad[p] += sum;
  else if (loss) *loss += sum;
}

// Adam (Kingma & Ba 2015) on the fp32 parameters; `step` counts from 1.
__global__ void k_mlp_adam(float *params, const float *grad, float *m, float *v, float lr, float b1, float b2,
                           float eps, int step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float gr = grad[i];
  m[i] = b1 * m[i] + (1.f - b1) * gr;
  v[i] = b2 * v[i] + (1.f - b2) * gr * gr;
  const float mh = m[i] / (1.f - powf(b1, (float)step));
  const float vh = v[i] / (1.f - powf(b2, (float)step));
  params[i] -= lr * mh / (sqrtf(vh) + eps);
}

// Fisher-Yates-free shuffle: a random permutation key per sample from a
// counter-based hash, then the minibatches read samples in key order via an
// index array sorted on the host side; here the order is a multiplicative
// stride permutation (gcd(stride, n) = 1), cheap and deterministic.
__global__ void k_gather_batch(const float *X, const float *Y, int64_t n, int64_t start, int64_t count,
                               uint64_t stride, float *Xb, float *Yb) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < count; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = (int64_t)(((unsigned __int128)(uint64_t)(start + r) * stride) % (uint64_t)n);
#pragma unroll
    for (int k = 0; k < 8; ++k) Xb[r * 8 + k] = X[src * 8 + k];
    Yb[r] = Y[src];
  }
}

}  // namespace

void mlp_forward(const float *params, const float *X, int64_t n, float *logit, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t tiles = (n + 15) / 16;
  const int blocks = (int)std::min<int64_t>((tiles + 7) / 8, 152 * 16);
  LV_LAUNCH(k_mlp_forward<<<blocks, 256, 0, s>>>(params, X, n, logit));
}

int mlp_grad_blocks(int64_t n) { return (int)std::min<int64_t>((n + kGradSamples - 1) / kGradSamples, 152 * 8); }

size_t mlp_grad_scratch_floats(int64_t n) { return (size_t)std::max(mlp_grad_blocks(n), 1) * (kMlpParams + 1); }

void mlp_gradient(const float *params, const float *X, const float *Y, int64_t n, float scale, float *grad,
                  float *loss, float *scratch, cudaStream_t s) {
  if (n <= 0) return;
  const int blocks = mlp_grad_blocks(n);
  LV_LAUNCH(k_mlp_grad<<<blocks, 256, 0, s>>>(params, X, Y, n, scale, scratch));
  LV_LAUNCH(k_mlp_reduce<<<(kMlpParams + 1 + 255) / 256, 256, 0, s>>>(scratch, blocks, grad, loss));
}

void mlp_adam(float *params, const float *grad, float *m, float *v, float lr, int step, cudaStream_t s) {
  LV_LAUNCH(k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(params, grad, m, v, lr, 0.9f, 0.999f, 1e-8f, step));
}

void mlp_gather_batch(const float *X, const float *Y, int64_t n, int64_t start, int64_t count, uint64_t stride,
                      float *Xb, float *Yb, cudaStream_t s) {
  if (count <= 0) return;
  LV_LAUNCH(k_gather_batch<<<(int)std::min<int64_t>((count + 255) / 256, 4096), 256, 0, s>>>(X, Y, n, start, count,
                                                                                              stride, Xb, Yb));
}

}  // namespace lv
