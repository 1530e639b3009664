// mlp_kernels.cu -- the learned near-contact correction: a 14 -> 64 -> 64 -> 6
// tanh network on the BF16 tensor cores (mma.sync m16n8k16, FP32
// accumulation), its training (forward, backward, Adam) and its use inside
// the coupled step for cell pairs closer than a gap cut-off.
//
// The paper gives no such term; it explains why one is missing (no fluid
// node between two cells closer than the lattice resolves, and no analytic
// lubrication force added, Sec. II).  The network is trained on what the
// method itself computes at a finer resolution.
//
// Tiles: one warp takes 16 samples.  The accumulator fragment of one layer is
// the A operand of the next (16 x 8 column tiles pair up into 16 x 16 k
// steps), so the forward pass stays in registers.  The backward pass stages
// the transposed activations and deltas of its 16 samples in shared memory
// for the weight-gradient products, whose contraction runs over the samples.
//
// Parameter layout (FP32 master copy, row-major): W1 64 x 14, b1 64,
// W2 64 x 64, b2 64, W3 6 x 64, b3 6 (5510 values).  Normalisation: inputs
// x~ = (x - mx) / sx, outputs y = y~ sy + my.
#include <mutex>

#include "../../include/bloodlb.h"
#include "bl_internal.cuh"

namespace bl {

constexpr int NI = 14, NH = 64, NO = 6;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH, NPAR = OFF_B3 + NO;
static_assert(NPAR == 5510, "parameter count");

// BF16 operand copies, rows padded by 8 elements against bank conflicts:
// W1p 64 x (16+8), W2p 64 x (64+8), W3p 8 x (64+8) as [n][k] (B operands of
// the forward pass); W2t 64 x (64+8), W3t 64 x (16+8) as [k][n] (B operands
// of the delta products)
constexpr int S1 = 24, S2 = 72, S3 = 72, S2T = 72, S3T = 24;
constexpr int P_W1 = 0, P_W2 = P_W1 + 64 * S1, P_W3 = P_W2 + 64 * S2, P_W2T = P_W3 + 8 * S3,
              P_W3T = P_W2T + 64 * S2T, P_TOTAL = P_W3T + 64 * S3T;

struct MlpDev {
  const __nv_bfloat16 *wp;  // P_TOTAL packed operands
  const float *theta;       // biases read from here
  const float *norm;        // mx[14], sx[14], my[6], sy[6]
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 32-bit word holding elements (k, k+1) of row n of a [n][k] BF16 array
__device__ __forceinline__ uint32_t ld2(const __nv_bfloat16 *base, int stride, int n, int k) {
  return *reinterpret_cast<const uint32_t *>(base + n * stride + k);
}

// packs the BF16 operand copies from the FP32 master parameters
__global__ void k_mlp_pack(const float *theta, __nv_bfloat16 *wp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P_TOTAL) return;
  float v = 0.f;
  if (i < P_W2) {
    const int n = i / S1, k = i % S1;
    if (k < NI) v = theta[OFF_W1 + n * NI + k];
  } else if (i < P_W3) {
    const int j = i - P_W2, n = j / S2, k = j % S2;
    if (k < NH) v = theta[OFF_W2 + n * NH + k];
  } else if (i < P_W2T) {
    const int j = i - P_W3, n = j / S3, k = j % S3;
    if (n < NO && k < NH) v = theta[OFF_W3 + n * NH + k];
  } else if (i < P_W3T) {
    const int j = i - P_W2T, kk = j / S2T, n = j % S2T;  // row kk = input unit of W2, col n = output unit
    if (n < NH) v = theta[OFF_W2 + n * NH + kk];
  } else {
    const int j = i - P_W3T, kk = j / S3T, o = j % S3T;  // row kk = hidden unit, col o = output
    if (o < NO) v = theta[OFF_W3 + o * NH + kk];
  }
  wp[i] = __float2bfloat16_rn(v);
}

// Forward pass of one warp tile (16 samples, rows r0.. of x).  Lane (g, t) =
// (lane / 4, lane % 4).  Leaves the activations in accumulator layout:
// h1[j], h2[j] for column tiles j = 0..7 (units 8j..8j+7), y for outputs.
struct Tile {
  float h1[8][4], h2[8][4], y[4];
};

__device__ __forceinline__ void tile_forward(const __nv_bfloat16 *wp, const float *theta, const float (&xs)[8],
                                             Tile &T) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t a[4] = {pack_bf16(xs[0], xs[1]), pack_bf16(xs[2], xs[3]), pack_bf16(xs[4], xs[5]),
                   pack_bf16(xs[6], xs[7])};
  // layer 1: x~ W1^T + b1, tanh
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float b0 = theta[OFF_B1 + 8 * j + 2 * t], b1 = theta[OFF_B1 + 8 * j + 2 * t + 1];
    T.h1[j][0] = b0;
    T.h1[j][1] = b1;
    T.h1[j][2] = b0;
    T.h1[j][3] = b1;
    mma16816(T.h1[j], a, ld2(wp + P_W1, S1, 8 * j + g, 2 * t), ld2(wp + P_W1, S1, 8 * j + g, 2 * t + 8));
#pragma unroll
    for (int e = 0; e < 4; ++e) T.h1[j][e] = tanhf(T.h1[j][e]);
  }
  // layer 2
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float b0 = theta[OFF_B2 + 8 * j + 2 * t], b1 = theta[OFF_B2 + 8 * j + 2 * t + 1];
    T.h2[j][0] = b0;
    T.h2[j][1] = b1;
    T.h2[j][2] = b0;
    T.h2[j][3] = b1;
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const uint32_t ak[4] = {pack_bf16(T.h1[2 * kk][0], T.h1[2 * kk][1]), pack_bf16(T.h1[2 * kk][2], T.h1[2 * kk][3]),
                            pack_bf16(T.h1[2 * kk + 1][0], T.h1[2 * kk + 1][1]),
                            pack_bf16(T.h1[2 * kk + 1][2], T.h1[2 * kk + 1][3])};
#pragma unroll
    for (int j = 0; j < 8; ++j)
      mma16816(T.h2[j], ak, ld2(wp + P_W2, S2, 8 * j + g, 16 * kk + 2 * t),
               ld2(wp + P_W2, S2, 8 * j + g, 16 * kk + 2 * t + 8));
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) T.h2[j][e] = tanhf(T.h2[j][e]);
  // layer 3 (outputs 6, 7 of the tile are padding)
  const float c0 = 2 * t < NO ? theta[OFF_B3 + 2 * t] : 0.f, c1 = 2 * t + 1 < NO ? theta[OFF_B3 + 2 * t + 1] : 0.f;
  T.y[0] = c0;
  T.y[1] = c1;
  T.y[2] = c0;
  T.y[3] = c1;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const uint32_t ak[4] = {pack_bf16(T.h2[2 * kk][0], T.h2[2 * kk][1]), pack_bf16(T.h2[2 * kk][2], T.h2[2 * kk][3]),
                            pack_bf16(T.h2[2 * kk + 1][0], T.h2[2 * kk + 1][1]),
                            pack_bf16(T.h2[2 * kk + 1][2], T.h2[2 * kk + 1][3])};
    mma16816(T.y, ak, ld2(wp + P_W3, S3, g, 16 * kk + 2 * t), ld2(wp + P_W3, S3, g, 16 * kk + 2 * t + 8));
  }
}

// the standardised inputs of this lane's A-fragment positions: rows g, g+8
// of the tile, columns 2t, 2t+1, 2t+8, 2t+9 (columns >= 14 are zero)
__device__ __forceinline__ void load_x(const float *x, int B, int r0, const float *norm, float (&xs)[8]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int rows[2] = {r0 + g, r0 + g + 8};
  const int cols[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
  // order of the A fragment: (g, c0) (g, c1) (g+8, c0) (g+8, c1) (g, c2) (g, c3) (g+8, c2) (g+8, c3)
  const int rsel[8] = {0, 0, 1, 1, 0, 0, 1, 1}, csel[8] = {0, 1, 0, 1, 2, 3, 2, 3};
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int r = rows[rsel[e]], c = cols[csel[e]];
    xs[e] = (r < B && c < NI) ? (x[(size_t)r * NI + c] - norm[c]) / norm[NI + c] : 0.f;
  }
}

// inference on raw features: y = network(x) in raw output units (B x 6);
// with Bdev the row count is min(*Bdev, B), read on the device
__global__ void __launch_bounds__(128) k_mlp_forward(MlpDev m, const float *x, int B, const int *Bdev, float *y) {
  __shared__ __align__(16) __nv_bfloat16 wp[P_TOTAL];
  if (Bdev) B = min(*Bdev, B);
  for (int i = threadIdx.x; i < P_W2T; i += blockDim.x) wp[i] = m.wp[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int r0 = (blockIdx.x * 4 + (threadIdx.x >> 5)) * 16; r0 < B; r0 += gridDim.x * 64) {
    float xs[8];
    load_x(x, B, r0, m.norm, xs);
    Tile T;
    tile_forward(wp, m.theta, xs, T);
    const float *my = m.norm + 2 * NI, *sy = m.norm + 2 * NI + NO;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = r0 + g + (e >= 2 ? 8 : 0), c = 2 * t + (e & 1);
      if (r < B && c < NO) y[(size_t)r * NO + c] = T.y[e] * sy[c] + my[c];
    }
  }
}

// Loss and gradient of the mean squared error of the standardised outputs
// over B samples (targets in raw units).  Each block adds its tiles into
// shared FP32 sums and writes one partial row of NPAR + 1 values (gradient,
// then the loss sum); k_mlp_reduce adds the partial rows in block order.
constexpr int DS = 24;  // row stride of the transposed [unit][sample] BF16 stages

__global__ void __launch_bounds__(128) k_mlp_grad(MlpDev m, const float *x, const float *yt, int B,
                                                  float *partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16 *wp = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
  float *gs = reinterpret_cast<float *>(smem_raw + sizeof(__nv_bfloat16) * P_TOTAL);  // NPAR + 1 sums
  __nv_bfloat16 *stg = reinterpret_cast<__nv_bfloat16 *>(gs + NPAR + 2);              // per warp stages
  for (int i = threadIdx.x; i < P_TOTAL; i += blockDim.x) wp[i] = m.wp[i];
  for (int i = threadIdx.x; i < NPAR + 1; i += blockDim.x) gs[i] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, wid = threadIdx.x >> 5;
  // per-warp transposed stages, [unit][sample]: xT 16 rows, h1T 64, h2T 64,
  // d1T 64, d2T 64, d3T 16 (rows >= 6 zero)
  __nv_bfloat16 *st = stg + (size_t)wid * (16 + 64 * 4 + 16) * DS;
  __nv_bfloat16 *xT = st, *h1T = xT + 16 * DS, *h2T = h1T + 64 * DS, *d1T = h2T + 64 * DS, *d2T = d1T + 64 * DS,
                *d3T = d2T + 64 * DS;
  const float inv_b = 1.0f / (float)B;
  const float *my = m.norm + 2 * NI, *sy = m.norm + 2 * NI + NO;
  float loss = 0.f;
  for (int r0 = (blockIdx.x * 4 + wid) * 16; r0 < B; r0 += gridDim.x * 64) {
    float xs[8];
    load_x(x, B, r0, m.norm, xs);
    Tile T;
    tile_forward(wp, m.theta, xs, T);
    // d3 = 2 (y~ - t~) / B on valid rows and outputs
    float d3[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = r0 + g + (e >= 2 ? 8 : 0), c = 2 * t + (e & 1);
      float d = 0.f;
      if (r < B && c < NO) {
        const float res = T.y[e] - (yt[(size_t)r * NO + c] - my[c]) / sy[c];
        loss += res * res;
        d = 2.0f * res * inv_b;
      }
      d3[e] = d;
    }
    // d2 = (d3 W3) * (1 - h2^2): A = d3 (k = outputs, 8..15 zero), B = W3t
    const uint32_t a3[4] = {pack_bf16(d3[0], d3[1]), pack_bf16(d3[2], d3[3]), 0u, 0u};
    float d2[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      d2[j][0] = d2[j][1] = d2[j][2] = d2[j][3] = 0.f;
      mma16816(d2[j], a3, ld2(wp + P_W3T, S3T, 8 * j + g, 2 * t), 0u);
#pragma unroll
      for (int e = 0; e < 4; ++e) d2[j][e] *= 1.0f - T.h2[j][e] * T.h2[j][e];
    }
    // d1 = (d2 W2) * (1 - h1^2): B = W2t
    float d1[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) d1[j][0] = d1[j][1] = d1[j][2] = d1[j][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const uint32_t ak[4] = {pack_bf16(d2[2 * kk][0], d2[2 * kk][1]), pack_bf16(d2[2 * kk][2], d2[2 * kk][3]),
                              pack_bf16(d2[2 * kk + 1][0], d2[2 * kk + 1][1]),
                              pack_bf16(d2[2 * kk + 1][2], d2[2 * kk + 1][3])};
#pragma unroll
      for (int j = 0; j < 8; ++j)
        mma16816(d1[j], ak, ld2(wp + P_W2T, S2T, 8 * j + g, 16 * kk + 2 * t),
                 ld2(wp + P_W2T, S2T, 8 * j + g, 16 * kk + 2 * t + 8));
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) d1[j][e] *= 1.0f - T.h1[j][e] * T.h1[j][e];
    // stage the transposed operands: element (sample s, unit u) -> [u][s]
    __syncwarp();
    {
      const int sr[2] = {g, g + 8};
      const float xv[8] = {xs[0], xs[1], xs[2], xs[3], xs[4], xs[5], xs[6], xs[7]};
      const int rsel[8] = {0, 0, 1, 1, 0, 0, 1, 1}, cols[8] = {2 * t, 2 * t + 1, 2 * t, 2 * t + 1,
                                                                2 * t + 8, 2 * t + 9, 2 * t + 8, 2 * t + 9};
#pragma unroll
      for (int e = 0; e < 8; ++e) xT[cols[e] * DS + sr[rsel[e]]] = __float2bfloat16_rn(xv[e]);
#pragma unroll
      for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int s = sr[e >> 1], u = 8 * j + 2 * t + (e & 1);
          h1T[u * DS + s] = __float2bfloat16_rn(T.h1[j][e]);
          h2T[u * DS + s] = __float2bfloat16_rn(T.h2[j][e]);
          d1T[u * DS + s] = __float2bfloat16_rn(d1[j][e]);
          d2T[u * DS + s] = __float2bfloat16_rn(d2[j][e]);
        }
#pragma unroll
      for (int e = 0; e < 4; ++e) d3T[(2 * t + (e & 1)) * DS + sr[e >> 1]] = __float2bfloat16_rn(d3[e]);
#pragma unroll
      for (int e = 0; e < 4; ++e) d3T[(8 + 2 * t + (e & 1)) * DS + sr[e >> 1]] = __float2bfloat16_rn(0.f);
    }
    __syncwarp();
    // weight gradients dW = dT^T-products over the 16 samples: A = dT [unit][sample]
    // (16 x 16 per m tile), B = hT [unit][sample] read as (k = sample, n = unit)
    auto afrag = [&](const __nv_bfloat16 *src, int m0, uint32_t (&a)[4]) {
      a[0] = ld2(src, DS, m0 + g, 2 * t);
      a[1] = ld2(src, DS, m0 + g + 8, 2 * t);
      a[2] = ld2(src, DS, m0 + g, 2 * t + 8);
      a[3] = ld2(src, DS, m0 + g + 8, 2 * t + 8);
    };
    auto acc = [&](int off, int ncols, int m0, int n0, const float (&c)[4], int mrows) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = m0 + g + (e >= 2 ? 8 : 0), col = n0 + 2 * t + (e & 1);
        if (r < mrows && col < ncols) atomicAdd(&gs[off + r * ncols + col], c[e]);
      }
    };
    // dW1 (64 x 14): m tiles of d1T, n tiles of xT (2 tiles, 16 columns)
#pragma unroll
    for (int mi = 0; mi < 4; ++mi) {
      uint32_t a[4];
      afrag(d1T, 16 * mi, a);
#pragma unroll
      for (int nj = 0; nj < 2; ++nj) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(c, a, ld2(xT, DS, 8 * nj + g, 2 * t), ld2(xT, DS, 8 * nj + g, 2 * t + 8));
        acc(OFF_W1, NI, 16 * mi, 8 * nj, c, NH);
      }
    }
    // dW2 (64 x 64): d2T x h1T
#pragma unroll
    for (int mi = 0; mi < 4; ++mi) {
      uint32_t a[4];
      afrag(d2T, 16 * mi, a);
#pragma unroll
      for (int nj = 0; nj < 8; ++nj) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(c, a, ld2(h1T, DS, 8 * nj + g, 2 * t), ld2(h1T, DS, 8 * nj + g, 2 * t + 8));
        acc(OFF_W2, NH, 16 * mi, 8 * nj, c, NH);
      }
    }
    // dW3 (6 x 64): d3T x h2T
    {
      uint32_t a[4];
      afrag(d3T, 0, a);
#pragma unroll
      for (int nj = 0; nj < 8; ++nj) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(c, a, ld2(h2T, DS, 8 * nj + g, 2 * t), ld2(h2T, DS, 8 * nj + g, 2 * t + 8));
        acc(OFF_W3, NH, 0, 8 * nj, c, NO);
      }
    }
    // bias gradients: sums over the samples (FP32 deltas)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        float s1 = d1[j][e] + d1[j][e + 2], s2 = d2[j][e] + d2[j][e + 2];
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
          s1 += __shfl_xor_sync(0xffffffffu, s1, o);
          s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (g == 0) {
          atomicAdd(&gs[OFF_B1 + 8 * j + 2 * t + e], s1);
          atomicAdd(&gs[OFF_B2 + 8 * j + 2 * t + e], s2);
        }
      }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float s3 = d3[e] + d3[e + 2];
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) s3 += __shfl_xor_sync(0xffffffffu, s3, o);
      if (g == 0 && 2 * t + e < NO) atomicAdd(&gs[OFF_B3 + 2 * t + e], s3);
    }
    __syncwarp();
  }
  // the block's loss sum, then its partial row
  loss = warp_sum(loss);
  if (lane == 0) atomicAdd(&gs[NPAR], loss * inv_b);
  __syncthreads();
  for (int i = threadIdx.x; i < NPAR + 1; i += blockDim.x) partial[(size_t)blockIdx.x * (NPAR + 1) + i] = gs[i];
}

// sums the partial rows in block order (a fixed order: the same data give
// the same gradient bit for bit)
__global__ void k_mlp_reduce(const float *partial, int nblocks, float *grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPAR + 1) return;
  float s = 0.f;
  for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * (NPAR + 1) + i];
  grad[i] = s;
}

// Adam on the FP32 master parameters (step count k >= 1)
__global__ void k_mlp_adam(float *theta, const float *grad, float *m1, float *m2, float lr, float b1, float b2,
                           float eps, int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPAR) return;
  const float gi = grad[i];
  const float a = b1 * m1[i] + (1.0f - b1) * gi, v = b2 * m2[i] + (1.0f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = v;
  const float ah = a / (1.0f - powf(b1, (float)k)), vh = v / (1.0f - powf(b2, (float)k));
  theta[i] -= lr * ah / (sqrtf(vh) + eps);
}

}  // namespace bl

// ---------------------------------------------------------------------------
// C ABI

using namespace bl;

struct bl_mlp {
  cudaStream_t stream;
  float *theta, *grad, *m1, *m2, *norm, *partial;
  __nv_bfloat16 *wp;
  int nblocks;
  int k;  // Adam steps taken
  char err[128];
};

static const int MLP_BLOCKS = 152;

static size_t grad_smem() {
  return sizeof(__nv_bfloat16) * P_TOTAL + sizeof(float) * (NPAR + 2) +
         sizeof(__nv_bfloat16) * 4 * (16 + 64 * 4 + 16) * DS;
}

static int mlp_pack(bl_mlp *m) {
  k_mlp_pack<<<(P_TOTAL + 255) / 256, 256, 0, m->stream>>>(m->theta, m->wp);
  return cudaGetLastError() == cudaSuccess ? BL_OK : BL_ECUDA;
}

extern "C" int bl_mlp_create(bl_mlp **out, void *cuda_stream) {
  if (!out) return BL_EINVAL;
  *out = nullptr;
  bl_mlp *m = new bl_mlp();
  m->stream = (cudaStream_t)cuda_stream;
  m->nblocks = MLP_BLOCKS;
  bool ok = cudaMalloc(&m->theta, sizeof(float) * NPAR) == cudaSuccess &&
            cudaMalloc(&m->grad, sizeof(float) * (NPAR + 1)) == cudaSuccess &&
            cudaMalloc(&m->m1, sizeof(float) * NPAR) == cudaSuccess &&
            cudaMalloc(&m->m2, sizeof(float) * NPAR) == cudaSuccess &&
            cudaMalloc(&m->norm, sizeof(float) * 40) == cudaSuccess &&
            cudaMalloc(&m->partial, sizeof(float) * (NPAR + 1) * MLP_BLOCKS) == cudaSuccess &&
            cudaMalloc(&m->wp, sizeof(__nv_bfloat16) * P_TOTAL) == cudaSuccess;
  if (ok) {
    cudaMemsetAsync(m->theta, 0, sizeof(float) * NPAR, m->stream);
    cudaMemsetAsync(m->m1, 0, sizeof(float) * NPAR, m->stream);
    cudaMemsetAsync(m->m2, 0, sizeof(float) * NPAR, m->stream);
    float norm[40];
    for (int i = 0; i < 40; ++i) norm[i] = (i < NI || (i >= 2 * NI && i < 2 * NI + NO)) ? 0.f : 1.f;
    ok = cudaMemcpyAsync(m->norm, norm, sizeof(norm), cudaMemcpyHostToDevice, m->stream) == cudaSuccess &&
         cudaStreamSynchronize(m->stream) == cudaSuccess && mlp_pack(m) == BL_OK &&
         cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()) ==
             cudaSuccess;
  }
  if (!ok) {
    bl_mlp_destroy(m);
    return BL_ENOMEM;
  }
  *out = m;
  return BL_OK;
}

extern "C" int bl_mlp_params_set(bl_mlp *m, const float *theta, const float *norm) {
  if (!m) return BL_EINVAL;
  if (theta && cudaMemcpyAsync(m->theta, theta, sizeof(float) * NPAR, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
    return BL_ECUDA;
  if (norm) {
    for (int i = 0; i < NI; ++i)
      if (!(norm[NI + i] > 0.f)) return BL_EINVAL;
    for (int i = 0; i < NO; ++i)
      if (!(norm[2 * NI + NO + i] > 0.f)) return BL_EINVAL;
    if (cudaMemcpyAsync(m->norm, norm, sizeof(float) * 40, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
      return BL_ECUDA;
  }
  if (theta) {
    m->k = 0;
    cudaMemsetAsync(m->m1, 0, sizeof(float) * NPAR, m->stream);
    cudaMemsetAsync(m->m2, 0, sizeof(float) * NPAR, m->stream);
  }
  if (mlp_pack(m) != BL_OK) return BL_ECUDA;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? BL_OK : BL_ECUDA;
}

extern "C" int bl_mlp_params_get(bl_mlp *m, float *theta, float *norm) {
  if (!m) return BL_EINVAL;
  if (theta && cudaMemcpyAsync(theta, m->theta, sizeof(float) * NPAR, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return BL_ECUDA;
  if (norm && cudaMemcpyAsync(norm, m->norm, sizeof(float) * 40, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return BL_ECUDA;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? BL_OK : BL_ECUDA;
}

static MlpDev mlp_dev(const bl_mlp *m) { return MlpDev{m->wp, m->theta, m->norm}; }

extern "C" int bl_mlp_forward(bl_mlp *m, const float *x, int B, float *y) {
  if (!m || B < 0 || (B > 0 && (!x || !y))) return BL_EINVAL;
  if (B == 0) return BL_OK;
  const int blocks = min((B + 63) / 64, 4 * MLP_BLOCKS);
  k_mlp_forward<<<blocks, 128, 0, m->stream>>>(mlp_dev(m), x, B, nullptr, y);
  return cudaGetLastError() == cudaSuccess ? BL_OK : BL_ECUDA;
}

extern "C" int bl_mlp_grad(bl_mlp *m, const float *x, const float *y, int B, float *loss, float *grad) {
  if (!m || B < 1 || !x || !y) return BL_EINVAL;
  k_mlp_grad<<<m->nblocks, 128, grad_smem(), m->stream>>>(mlp_dev(m), x, y, B, m->partial);
  k_mlp_reduce<<<(NPAR + 1 + 255) / 256, 256, 0, m->stream>>>(m->partial, m->nblocks, m->grad);
  if (cudaGetLastError() != cudaSuccess) return BL_ECUDA;
  if (loss && cudaMemcpyAsync(loss, m->grad + NPAR, sizeof(float), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return BL_ECUDA;
  if (grad && cudaMemcpyAsync(grad, m->grad, sizeof(float) * NPAR, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return BL_ECUDA;
  if ((loss || grad) && cudaStreamSynchronize(m->stream) != cudaSuccess) return BL_ECUDA;
  return BL_OK;
}

extern "C" int bl_mlp_adam(bl_mlp *m, float lr, float beta1, float beta2, float eps) {
  if (!m || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return BL_EINVAL;
  m->k++;
  k_mlp_adam<<<(NPAR + 255) / 256, 256, 0, m->stream>>>(m->theta, m->grad, m->m1, m->m2, lr, beta1, beta2, eps, m->k);
  if (cudaGetLastError() != cudaSuccess) return BL_ECUDA;
  return mlp_pack(m);
}

namespace bl {
void launch_mlp_forward_dev(const void *mlp, const float *x, const int *count, int cap, float *y, cudaStream_t st) {
  const bl_mlp *m = static_cast<const bl_mlp *>(mlp);
  const int blocks = min((cap + 63) / 64, 4 * MLP_BLOCKS);
  if (blocks > 0) k_mlp_forward<<<blocks, 128, 0, st>>>(mlp_dev(m), x, cap, count, y);
}
}  // namespace bl

extern "C" int bl_mlp_sync(bl_mlp *m) {
  if (!m) return BL_EINVAL;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? BL_OK : BL_ECUDA;
}

extern "C" void bl_mlp_destroy(bl_mlp *m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  void *p[] = {m->theta, m->grad, m->m1, m->m2, m->norm, m->partial, m->wp};
  for (void *q : p)
    if (q) cudaFree(q);
  delete m;
}
