// The learned warm start of the elliptic-relaxation solve: a per-node MLP
// 11 -> 64 -> 64 -> 64 -> 9 with GELU, BF16 weights and activations, FP32
// accumulation, trained with Adam by the kernels below.  (The paper warm-
// starts the solve from the previous step, sec. 3.2; the network is an
// addition; the FP64 solve it seeds still runs to the same residual.)
//
// Inputs per node: <U>, <V>, <W>, <uu>, <vv>, <ww>, <uv>, <uw>, <vw>,
// <omega>, wall distance; outputs wp_ij.  Both standardized with stored
// means and scales.  Matrix products on the tensor cores (mma.sync
// m16n8k16, BF16 x BF16 -> FP32); the weight gradients, a reduction over
// the batch, in FP32 in a fixed order (deterministic).
// Rounding points (shared with the CPU check): the standardized input, the
// weights, every hidden activation and every back-propagated gradient are
// rounded to BF16 before they enter a product.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "rng.cuh"

namespace pdfgb {

constexpr int kIn = 11, kHid = 64, kOut = 9;
// flat parameter layout: W0[64][11] b0[64] W1[64][64] b1[64] W2[64][64] b2[64] W3[9][64] b3[9]
__host__ __device__ constexpr int kOffW_(int l) { return l == 0 ? 0 : l == 1 ? 768 : l == 2 ? 4928 : 9088; }
__host__ __device__ constexpr int kOffB_(int l) { return l == 0 ? 704 : l == 1 ? 4864 : l == 2 ? 9024 : 9664; }
constexpr int kNParam = 9673;
__host__ __device__ constexpr int kRealN_(int l) { return l == 3 ? 9 : 64; }
__host__ __device__ constexpr int kRealK_(int l) { return l == 0 ? 11 : 64; }
__host__ __device__ constexpr int kPadN_(int l) { return l == 3 ? 16 : 64; }
__host__ __device__ constexpr int kPadK_(int l) { return l == 0 ? 16 : 64; }
// packed BF16 weights: W_l [PadN][PadK] then WT_l [PadK][PadN]
__host__ __device__ constexpr int kOffWb_(int l) { return l == 0 ? 0 : l == 1 ? 1024 : l == 2 ? 5120 : 9216; }
__host__ __device__ constexpr int kOffWT_(int l) { return l == 0 ? 10240 : l == 1 ? 11264 : l == 2 ? 15360 : 19456; }
constexpr int kNWb = 20480;
__host__ __device__ constexpr int kOffBias_(int l) { return 64 * l; }  // padded biases, 208 floats
constexpr int kNBias = 208;
constexpr int kThreads = 128;   // 4 warps, 16 rows each per pass
constexpr int kRows = 64;

}  // namespace pdfgb

struct pdf_mlp {
  float* w = nullptr;        // [kNParam] FP32 master parameters
  float* m = nullptr;        // Adam first moments
  float* v = nullptr;        // Adam second moments
  float* grad = nullptr;     // [kNParam]
  __nv_bfloat16* wb = nullptr;  // packed BF16 weights
  float* bias = nullptr;     // [208] padded biases (FP32)
  float* norm = nullptr;     // in_mean[16] in_inv[16] out_mean[16] out_scale[16]
  float* part = nullptr;     // per-CTA partial gradients
  float* loss_part = nullptr;
  float* host = nullptr;     // pinned scalars
  int max_ctas = 0;
  int64_t t = 0;             // Adam step count
};

namespace pdfgb {

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// One layer for a warp's 16 rows: C[16][8*NT] = A[16][16*KT] * W^T, with A
// in fragment registers (KT k-tiles) and W [N][K] row-major in shared memory
// (ld = padded K).
template <int KT, int NT>
__device__ __forceinline__ void layer_mma(const uint32_t (&A)[KT][4], const __nv_bfloat16* W, int ld,
                                          float (&C)[NT][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int n = 0; n < NT; ++n) {
    C[n][0] = C[n][1] = C[n][2] = C[n][3] = 0.f;
    const __nv_bfloat16* row = W + (n * 8 + g) * ld;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(row + k * 16 + 2 * t);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(row + k * 16 + 8 + 2 * t);
      mma_bf16(C[n], A[k], b0, b1);
    }
  }
}

// Accumulator tiles (pairs of n-tiles) -> A fragments of the next product.
template <int NT>
__device__ __forceinline__ void c_to_a(const float (&C)[NT][4], uint32_t (&A)[NT / 2][4]) {
#pragma unroll
  for (int q = 0; q < NT / 2; ++q) {
    A[q][0] = pack_bf16(C[2 * q][0], C[2 * q][1]);
    A[q][1] = pack_bf16(C[2 * q][2], C[2 * q][3]);
    A[q][2] = pack_bf16(C[2 * q + 1][0], C[2 * q + 1][1]);
    A[q][3] = pack_bf16(C[2 * q + 1][2], C[2 * q + 1][3]);
  }
}

// Standardized input rows -> A fragments of layer 0 (K padded to 16).
__device__ __forceinline__ void load_input(const float* __restrict__ X, int64_t n, int64_t row0,
                                           const float* norm, uint32_t (&A)[1][4], __nv_bfloat16* a0s /*[16][16] or null*/) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float v[2][4];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t r = row0 + g + 8 * h;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = (j < 2 ? 2 * t + j : 8 + 2 * t + (j - 2));
      float x = 0.f;
      if (r < n && col < kIn) x = (X[r * kIn + col] - norm[col]) * norm[16 + col];
      v[h][j] = x;
    }
  }
  A[0][0] = pack_bf16(v[0][0], v[0][1]);
  A[0][1] = pack_bf16(v[1][0], v[1][1]);
  A[0][2] = pack_bf16(v[0][2], v[0][3]);
  A[0][3] = pack_bf16(v[1][2], v[1][3]);
  if (a0s) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = g + ((q & 1) ? 8 : 0), col = 2 * t + ((q & 2) ? 8 : 0);
      *reinterpret_cast<uint32_t*>(a0s + row * 16 + col) = A[0][q];
    }
  }
}

__device__ __forceinline__ void stage_weights(const __nv_bfloat16* __restrict__ wb, const float* __restrict__ bias,
                                              const float* __restrict__ norm, __nv_bfloat16* s_w, float* s_b,
                                              float* s_norm, int n_wb) {
  for (int i = threadIdx.x; i < n_wb / 2; i += blockDim.x)
    reinterpret_cast<uint32_t*>(s_w)[i] = reinterpret_cast<const uint32_t*>(wb)[i];
  for (int i = threadIdx.x; i < kNBias; i += blockDim.x) s_b[i] = bias[i];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) s_norm[i] = norm[i];
  __syncthreads();
}

// Inference: Y[n][9] (de-standardized) from X[n][11].
__global__ void __launch_bounds__(kThreads) k_mlp_fwd(const __nv_bfloat16* __restrict__ wb,
                                                       const float* __restrict__ bias, const float* __restrict__ norm,
                                                       const float* __restrict__ X, int64_t n, float* __restrict__ Y) {
  __shared__ __align__(16) __nv_bfloat16 s_w[10240];
  __shared__ float s_b[kNBias], s_norm[64];
  stage_weights(wb, bias, norm, s_w, s_b, s_norm, kOffWT_(0));
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
  const int64_t chunks = (n + 15) / 16;
  for (int64_t c = (int64_t)blockIdx.x * 4 + w; c < chunks; c += (int64_t)gridDim.x * 4) {
    const int64_t row0 = c * 16;
    uint32_t A0[1][4];
    load_input(X, n, row0, s_norm, A0, nullptr);
    float C[8][4];
    uint32_t A[4][4];
    layer_mma<1, 8>(A0, s_w + kOffWb_(0), 16, C);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) C[j][e] = gelu(C[j][e] + s_b[kOffBias_(0) + j * 8 + 2 * t + (e & 1)]);
    c_to_a<8>(C, A);
#pragma unroll
    for (int l = 1; l <= 2; ++l) {
      layer_mma<4, 8>(A, s_w + kOffWb_(l), 64, C);
#pragma unroll
      for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) C[j][e] = gelu(C[j][e] + s_b[kOffBias_(l) + j * 8 + 2 * t + (e & 1)]);
      c_to_a<8>(C, A);
    }
    float O[2][4];
    layer_mma<4, 2>(A, s_w + kOffWb_(3), 64, O);
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = j * 8 + 2 * t + (e & 1);
        const int64_t r = row0 + g + ((e & 2) ? 8 : 0);
        if (col < kOut && r < n)
          Y[r * kOut + col] = (O[j][e] + s_b[kOffBias_(3) + col]) * s_norm[48 + col] + s_norm[32 + col];
      }
  }
}

// Training pass: forward, backward, per-CTA partial gradients of the mean
// squared error (over the batch and the 9 standardized outputs).
struct TrainSmem {
  __nv_bfloat16 w[kNWb];              // W_l and WT_l
  float b[kNBias];
  float norm[64];
  __nv_bfloat16 a0[kRows][16];        // layer inputs (BF16)
  __nv_bfloat16 a1[kRows][64], a2[kRows][64], a3[kRows][64];
  float z0[kRows][64], z1[kRows][64], z2[kRows][64];  // pre-activations
  __nv_bfloat16 d0[kRows][64], d1[kRows][64], d2[kRows][64], d3[kRows][16];  // dz_l (BF16)
  float acc[kNParam];                 // this CTA's gradient
  float loss[4];
};

__device__ __forceinline__ void store_c(const float (&C)[8][4], float (*z)[64], int rbase) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) z[rbase + g + ((e & 2) ? 8 : 0)][j * 8 + 2 * t + (e & 1)] = C[j][e];
}

__device__ __forceinline__ void store_a(const uint32_t (&A)[4][4], __nv_bfloat16 (*a)[64], int rbase) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int row = rbase + g + ((r & 1) ? 8 : 0), col = q * 16 + 2 * t + ((r & 2) ? 8 : 0);
      *reinterpret_cast<uint32_t*>(&a[row][col]) = A[q][r];
    }
}

__global__ void __launch_bounds__(kThreads) k_mlp_train(const __nv_bfloat16* __restrict__ wb,
                                                         const float* __restrict__ bias, const float* __restrict__ norm,
                                                         const float* __restrict__ X, const float* __restrict__ Yt,
                                                         int64_t n, float* __restrict__ part,
                                                         float* __restrict__ loss_part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  stage_weights(wb, bias, norm, S.w, S.b, S.norm, kNWb);
  for (int i = threadIdx.x; i < kNParam; i += kThreads) S.acc[i] = 0.f;
  if (threadIdx.x < 4) S.loss[threadIdx.x] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
  const float inv_count = 1.0f / (float)(n * kOut);
  float my_loss = 0.f;
  const int64_t blocks = (n + kRows - 1) / kRows;
  for (int64_t blk = blockIdx.x; blk < blocks; blk += gridDim.x) {
    const int64_t row0 = blk * kRows + w * 16;
    const int rb = w * 16;
    // ---- forward, keeping layer inputs and pre-activations
    uint32_t A0[1][4];
    load_input(X, n, row0, S.norm, A0, &S.a0[rb][0]);
    float C[8][4];
    uint32_t A[4][4];
    layer_mma<1, 8>(A0, S.w + kOffWb_(0), 16, C);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) C[j][e] += S.b[kOffBias_(0) + j * 8 + 2 * t + (e & 1)];
    store_c(C, S.z0, rb);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) C[j][e] = gelu(C[j][e]);
    c_to_a<8>(C, A);
    store_a(A, S.a1, rb);
    layer_mma<4, 8>(A, S.w + kOffWb_(1), 64, C);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) C[j][e] += S.b[kOffBias_(1) + j * 8 + 2 * t + (e & 1)];
    store_c(C, S.z1, rb);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) C[j][e] = gelu(C[j][e]);
    c_to_a<8>(C, A);
    store_a(A, S.a2, rb);
    layer_mma<4, 8>(A, S.w + kOffWb_(2), 64, C);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) C[j][e] += S.b[kOffBias_(2) + j * 8 + 2 * t + (e & 1)];
    store_c(C, S.z2, rb);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) C[j][e] = gelu(C[j][e]);
    c_to_a<8>(C, A);
    store_a(A, S.a3, rb);
    float O[2][4];
    layer_mma<4, 2>(A, S.w + kOffWb_(3), 64, O);
    // ---- output gradient dL/dy = 2 (y - t) / (n 9), rows past n and padded columns 0
    float D[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = j * 8 + 2 * t + (e & 1);
        const int64_t r = row0 + g + ((e & 2) ? 8 : 0);
        float d = 0.f;
        if (col < kOut && r < n) {
          const float y = O[j][e] + S.b[kOffBias_(3) + col];
          const float tt = (Yt[r * kOut + col] - S.norm[32 + col]) / S.norm[48 + col];
          const float diff = y - tt;
          my_loss += diff * diff;
          d = 2.0f * diff * inv_count;
        }
        D[j][e] = d;
      }
    uint32_t G3[1][4];
    c_to_a<2>(D, G3);
    {
      // dz3 (BF16) to shared memory
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = rb + g + ((r & 1) ? 8 : 0), col = 2 * t + ((r & 2) ? 8 : 0);
        *reinterpret_cast<uint32_t*>(&S.d3[row][col]) = G3[0][r];
      }
    }
    // ---- back through layers 3..1: da = dz W (B operand from WT), dz = da * gelu'(z)
    float Cd[8][4];
    layer_mma<1, 8>(G3, S.w + kOffWT_(3), 16, Cd);  // WT3 [64][16]: da2 [16][64]
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        Cd[j][e] *= gelu_grad(S.z2[rb + g + ((e & 2) ? 8 : 0)][j * 8 + 2 * t + (e & 1)]);
    uint32_t G[4][4];
    c_to_a<8>(Cd, G);
    store_a(G, S.d2, rb);
    layer_mma<4, 8>(G, S.w + kOffWT_(2), 64, Cd);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        Cd[j][e] *= gelu_grad(S.z1[rb + g + ((e & 2) ? 8 : 0)][j * 8 + 2 * t + (e & 1)]);
    c_to_a<8>(Cd, G);
    store_a(G, S.d1, rb);
    layer_mma<4, 8>(G, S.w + kOffWT_(1), 64, Cd);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        Cd[j][e] *= gelu_grad(S.z0[rb + g + ((e & 2) ? 8 : 0)][j * 8 + 2 * t + (e & 1)]);
    c_to_a<8>(Cd, G);
    store_a(G, S.d0, rb);
    __syncthreads();
    // ---- weight gradients of this block of 64 rows, FP32, fixed order
    for (int i = threadIdx.x; i < kNParam; i += kThreads) {
      int l = 3;
      while (l > 0 && i < kOffW_(l)) --l;
      float s = 0.f;
      if (i < kOffB_(l)) {  // weight W_l[o][k]
        const int o = (i - kOffW_(l)) / kRealK_(l), k = (i - kOffW_(l)) % kRealK_(l);
        for (int r = 0; r < kRows; ++r) {
          float dz, a;
          if (l == 0) { dz = __bfloat162float(S.d0[r][o]); a = __bfloat162float(S.a0[r][k]); }
          else if (l == 1) { dz = __bfloat162float(S.d1[r][o]); a = __bfloat162float(S.a1[r][k]); }
          else if (l == 2) { dz = __bfloat162float(S.d2[r][o]); a = __bfloat162float(S.a2[r][k]); }
          else { dz = __bfloat162float(S.d3[r][o]); a = __bfloat162float(S.a3[r][k]); }
          s = fmaf(dz, a, s);
        }
      } else {  // bias b_l[o]
        const int o = i - kOffB_(l);
        for (int r = 0; r < kRows; ++r) {
          s += __bfloat162float(l == 0 ? S.d0[r][o] : (l == 1 ? S.d1[r][o] : (l == 2 ? S.d2[r][o] : S.d3[r][o])));
        }
      }
      S.acc[i] += s;
    }
    __syncthreads();
  }
  // loss: warp sums, then warps in order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_xor_sync(0xffffffffu, my_loss, o);
  if (lane == 0) S.loss[w] = my_loss;
  __syncthreads();
  for (int i = threadIdx.x; i < kNParam; i += kThreads) part[(int64_t)blockIdx.x * kNParam + i] = S.acc[i];
  if (threadIdx.x == 0) loss_part[blockIdx.x] = ((S.loss[0] + S.loss[1]) + S.loss[2]) + S.loss[3];
}

// Sum the per-CTA partials in CTA order; optionally one Adam step.
__global__ void k_mlp_reduce_adam(const float* __restrict__ part, int nparts, const float* __restrict__ loss_part,
                                  float* __restrict__ grad, float* __restrict__ w, float* __restrict__ m,
                                  float* __restrict__ v, float lr, float b1t, float b2t, int update,
                                  float* __restrict__ loss_out, int64_t n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && loss_out) {
    float s = 0.f;
    for (int c = 0; c < nparts; ++c) s += loss_part[c];
    *loss_out = s / (float)(n * kOut);
  }
  if (i >= kNParam) return;
  float s = 0.f;
  for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * kNParam + i];
  grad[i] = s;
  if (!update) return;
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  const float mi = beta1 * m[i] + (1.f - beta1) * s;
  const float vi = beta2 * v[i] + (1.f - beta2) * s * s;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / b1t) / (sqrtf(vi / b2t) + eps);
}

// FP32 master parameters -> packed BF16 weights (and transposes), padded biases.
__global__ void k_mlp_pack(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, float* __restrict__ bias) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kNWb) {
    const bool tr = i >= kOffWT_(0);
    int l = 3;
    while (l > 0 && i < (tr ? kOffWT_(l) : kOffWb_(l))) --l;
    const int rel = i - (tr ? kOffWT_(l) : kOffWb_(l));
    int o, k;
    if (!tr) { o = rel / kPadK_(l); k = rel % kPadK_(l); }
    else { k = rel / kPadN_(l); o = rel % kPadN_(l); }
    float val = 0.f;
    if (o < kRealN_(l) && k < kRealK_(l)) val = w[kOffW_(l) + o * kRealK_(l) + k];
    wb[i] = __float2bfloat16_rn(val);
  }
  if (i < kNBias) {
    int l = 3;
    while (l > 0 && i < kOffBias_(l)) --l;
    const int o = i - kOffBias_(l);
    bias[i] = o < kRealN_(l) ? w[kOffB_(l) + o] : 0.f;
  }
}

// He-normal initial weights from the library's Philox draws (purpose 3), zero biases.
__global__ void k_mlp_init(uint64_t seed, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParam) return;
  m[i] = 0.f;
  v[i] = 0.f;
  int l = 3;
  while (l > 0 && i < kOffW_(l)) --l;
  if (i >= kOffB_(l)) { w[i] = 0.f; return; }
  float g[4];
  gauss4(seed, (uint32_t)i, 0u, 0u, 3u, g);
  w[i] = g[0] * sqrtf(2.0f / (float)kRealK_(l));
}

// Features and targets of every node.  The network corrects the local
// model of the elliptic relaxation: its inputs are the nodal right-hand
// side rhs_ij of eq. elliptic-relaxation-Lagrangian (the solution where the
// elliptic term vanishes), the wall distance over L and log(L^2 / h^2)
// (L^2 of the C_xi = 1 class, h^2 the mean area of the node's elements),
// and its target is the correction wp_ij - rhs_ij that the elliptic term
// makes.
__global__ void k_mlp_features(int32_t n_nodes, const double* __restrict__ rhs, const double* __restrict__ L2,
                               const double* __restrict__ wall_d, const int32_t* __restrict__ nse_off,
                               const int32_t* __restrict__ nse, const ElemGeo* __restrict__ geo,
                               const double* __restrict__ wp, float* __restrict__ X, float* __restrict__ Y) {
  for (int32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x) {
    float* x = X + (int64_t)n * kIn;
    for (int q = 0; q < 9; ++q) x[q] = (float)rhs[(int64_t)q * n_nodes + n];
    const double l2 = fmax(L2[(int64_t)2 * n_nodes + n], 1e-300);
    double area = 0.0;
    const int32_t b = nse_off[n], c = nse_off[n + 1] - b;
    for (int32_t i = b; i < b + c; ++i) area += 0.5 * geo[nse[i]].two_area;
    const double h2 = c > 0 ? area / (double)c : 1.0;
    x[9] = (float)(wall_d[n] / sqrt(l2));
    x[10] = (float)log(l2 / h2);
    if (wp && Y)
      for (int q = 0; q < kOut; ++q)
        Y[(int64_t)n * kOut + q] = (float)(wp[(int64_t)q * n_nodes + n] - rhs[(int64_t)q * n_nodes + n]);
  }
}

// A training batch: row i of (Xb, Yb) is row r_i of (X, Y), r_i drawn
// uniformly from [0, n) by Philox4x32-10 (key seed, counter (i, step, 0, 4)):
// the top 32 bits of word 0 times n, shifted down.
__global__ void k_mlp_batch(const float* __restrict__ X, const float* __restrict__ Y, int64_t n, uint64_t seed,
                            uint32_t step, int64_t batch, float* __restrict__ Xb, float* __restrict__ Yb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < batch; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)i, step, 0u, 4u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const int64_t r = (int64_t)(((uint64_t)c[0] * (uint64_t)n) >> 32);
    for (int q = 0; q < kIn; ++q) Xb[i * kIn + q] = X[r * kIn + q];
    for (int q = 0; q < kOut; ++q) Yb[i * kOut + q] = Y[r * kOut + q];
  }
}

// wp = rhs + the network's correction.
__global__ void k_mlp_to_wp(int32_t n_nodes, const float* __restrict__ Y, const double* __restrict__ rhs,
                            double* __restrict__ wp) {
  for (int32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x)
    for (int q = 0; q < kOut; ++q)
      wp[(int64_t)q * n_nodes + n] = rhs[(int64_t)q * n_nodes + n] + (double)Y[(int64_t)n * kOut + q];
}

// Standardization from data: means and 1/std of inputs, means and std of targets.
__global__ void k_mlp_fit_norm(const float* __restrict__ X, const float* __restrict__ Y, int64_t n,
                               float* __restrict__ norm) {
  const int c = threadIdx.x;  // one column per thread: 11 inputs then 9 outputs
  if (c >= kIn + kOut) return;
  const bool inp = c < kIn;
  const int col = inp ? c : c - kIn;
  const int ld = inp ? kIn : kOut;
  const float* src = inp ? X : Y;
  double s = 0.0, s2 = 0.0;
  for (int64_t r = 0; r < n; ++r) s += src[r * ld + col];
  const double mean = s / (double)n;
  for (int64_t r = 0; r < n; ++r) { const double d = src[r * ld + col] - mean; s2 += d * d; }
  double sd = sqrt(s2 / (double)n);
  if (!(sd > 1e-20)) sd = 1.0;
  if (inp) { norm[col] = (float)mean; norm[16 + col] = (float)(1.0 / sd); }
  else { norm[32 + col] = (float)mean; norm[48 + col] = (float)sd; }
}

static size_t train_smem() { return sizeof(TrainSmem); }

}  // namespace pdfgb

using namespace pdfgb;

extern "C" pdf_status pdf_mlp_create(uint64_t seed, pdf_mlp** out) {
  if (!out) return fail(PDF_EINVAL, "pdf_mlp_create: out is NULL");
  *out = nullptr;
  pdf_mlp* M = new (std::nothrow) pdf_mlp();
  if (!M) return fail(PDF_ENOMEM, "pdf_mlp_create: host allocation");
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  M->max_ctas = sms * 2;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t b) { if (e == cudaSuccess) e = cudaMalloc(p, b); };
  A((void**)&M->w, sizeof(float) * kNParam);
  A((void**)&M->m, sizeof(float) * kNParam);
  A((void**)&M->v, sizeof(float) * kNParam);
  A((void**)&M->grad, sizeof(float) * kNParam);
  A((void**)&M->wb, sizeof(__nv_bfloat16) * kNWb);
  A((void**)&M->bias, sizeof(float) * kNBias);
  A((void**)&M->norm, sizeof(float) * 64);
  A((void**)&M->part, sizeof(float) * kNParam * (size_t)M->max_ctas);
  A((void**)&M->loss_part, sizeof(float) * M->max_ctas);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&M->host, sizeof(float) * 16);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem());
  if (e == cudaSuccess) {
    std::vector<float> nrm(64, 0.f);
    for (int i = 0; i < 16; ++i) { nrm[16 + i] = 1.f; nrm[48 + i] = 1.f; }
    e = cudaMemcpy(M->norm, nrm.data(), sizeof(float) * 64, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    k_mlp_init<<<(kNParam + 255) / 256, 256>>>(seed, M->w, M->m, M->v);
    k_mlp_pack<<<(kNWb + 255) / 256, 256>>>(M->w, M->wb, M->bias);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    pdf_mlp_destroy(M);
    return cuda_fail(e, "pdf_mlp_create");
  }
  *out = M;
  return PDF_OK;
}

extern "C" pdf_status pdf_mlp_destroy(pdf_mlp* M) {
  if (!M) return PDF_OK;
  cudaFree(M->w); cudaFree(M->m); cudaFree(M->v); cudaFree(M->grad); cudaFree(M->wb); cudaFree(M->bias);
  cudaFree(M->norm); cudaFree(M->part); cudaFree(M->loss_part);
  if (M->host) cudaFreeHost(M->host);
  delete M;
  return PDF_OK;
}

extern "C" pdf_status pdf_mlp_params(pdf_mlp* M, const float* set, float* get, const float* set_norm,
                                     float* get_norm) {
  if (!M) return fail(PDF_EINVAL, "pdf_mlp_params: NULL network");
  if (get) PDF_CUDA(cudaMemcpy(get, M->w, sizeof(float) * kNParam, cudaMemcpyDefault));
  if (get_norm) PDF_CUDA(cudaMemcpy(get_norm, M->norm, sizeof(float) * 64, cudaMemcpyDefault));
  if (set) {
    PDF_CUDA(cudaMemcpy(M->w, set, sizeof(float) * kNParam, cudaMemcpyDefault));
    PDF_CUDA(cudaMemset(M->m, 0, sizeof(float) * kNParam));
    PDF_CUDA(cudaMemset(M->v, 0, sizeof(float) * kNParam));
    M->t = 0;
  }
  if (set_norm) PDF_CUDA(cudaMemcpy(M->norm, set_norm, sizeof(float) * 64, cudaMemcpyDefault));
  if (set) {
    PDF_KERNEL("k_mlp_pack", (cudaStream_t)0, k_mlp_pack<<<(kNWb + 255) / 256, 256>>>(M->w, M->wb, M->bias));
    PDF_CUDA(cudaDeviceSynchronize());
  }
  return PDF_OK;
}

extern "C" pdf_status pdf_mlp_fit_norm(pdf_mlp* M, const float* X, const float* Y, int64_t n, void* stream) {
  if (!M || !X || !Y || n < 1) return fail(PDF_EINVAL, "pdf_mlp_fit_norm: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  PDF_KERNEL("k_mlp_fit_norm", st, k_mlp_fit_norm<<<1, 32, 0, st>>>(X, Y, n, M->norm));
  return PDF_OK;
}

extern "C" pdf_status pdf_mlp_forward(const pdf_mlp* M, const float* X, int64_t n, float* Y, void* stream) {
  if (!M || n < 0 || (n > 0 && (!X || !Y))) return fail(PDF_EINVAL, "pdf_mlp_forward: bad arguments");
  if (n == 0) return PDF_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t chunks = (n + 15) / 16;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((chunks + 3) / 4, 4096));
  PDF_KERNEL("k_mlp_fwd", st, k_mlp_fwd<<<blocks, kThreads, 0, st>>>(M->wb, M->bias, M->norm, X, n, Y));
  return PDF_OK;
}

static pdf_status mlp_pass(pdf_mlp* M, const float* X, const float* Y, int64_t n, float lr, int update,
                           float* loss, float* grad_out, cudaStream_t st) {
  if (!M || !X || !Y || n < 1) return fail(PDF_EINVAL, "pdf_mlp: bad arguments");
  const int64_t blocks64 = (n + kRows - 1) / kRows;
  const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(blocks64, M->max_ctas));
  PDF_KERNEL("k_mlp_train", st, k_mlp_train<<<ctas, kThreads, train_smem(), st>>>(M->wb, M->bias, M->norm, X, Y, n,
                                                                                    M->part, M->loss_part));
  float b1t = 1.f, b2t = 1.f;
  if (update) {
    M->t += 1;
    b1t = 1.f - powf(0.9f, (float)M->t);
    b2t = 1.f - powf(0.999f, (float)M->t);
  }
  PDF_KERNEL("k_mlp_reduce_adam", st, k_mlp_reduce_adam<<<(kNParam + 255) / 256, 256, 0, st>>>(
                                          M->part, ctas, M->loss_part, M->grad, M->w, M->m, M->v, lr, b1t, b2t, update,
                                          loss ? M->host : nullptr, n));
  if (update) PDF_KERNEL("k_mlp_pack", st, k_mlp_pack<<<(kNWb + 255) / 256, 256, 0, st>>>(M->w, M->wb, M->bias));
  if (grad_out) PDF_CUDA(cudaMemcpyAsync(grad_out, M->grad, sizeof(float) * kNParam, cudaMemcpyDefault, st));
  if (loss) {
    PDF_CUDA(cudaStreamSynchronize(st));
    *loss = M->host[0];
  }
  return PDF_OK;
}

extern "C" pdf_status pdf_mlp_grad(pdf_mlp* M, const float* X, const float* Y, int64_t n, float* grad,
                                   float* loss, void* stream) {
  return mlp_pass(M, X, Y, n, 0.f, 0, loss, grad, (cudaStream_t)stream);
}

extern "C" pdf_status pdf_mlp_train_step(pdf_mlp* M, const float* X, const float* Y, int64_t n, float lr,
                                         float* loss, void* stream) {
  return mlp_pass(M, X, Y, n, lr, 1, loss, nullptr, (cudaStream_t)stream);
}

extern "C" pdf_status pdf_mlp_batch(const float* X, const float* Y, int64_t n, uint64_t seed, uint32_t step,
                                    int64_t batch, float* Xb, float* Yb, void* stream) {
  if (!X || !Y || !Xb || !Yb || n < 1 || n > (int64_t)UINT32_MAX || batch < 1)
    return fail(PDF_EINVAL, "pdf_mlp_batch: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = (int)std::min<int64_t>((batch + 255) / 256, 4096);
  PDF_KERNEL("k_mlp_batch", st, k_mlp_batch<<<blocks, 256, 0, st>>>(X, Y, n, seed, step, batch, Xb, Yb));
  return PDF_OK;
}

extern "C" pdf_status pdf_mlp_features(pdf_particles* p, const pdf_mesh* m, const pdf_model_params* params,
                                       const double* wp, float* X, float* Y, void* stream) {
  if (!p || !m || p->mesh != m || !params || !X) return fail(PDF_EINVAL, "pdf_mlp_features: bad arguments");
  if (!p->have_stats) return fail(PDF_ESTATE, "pdf_mlp_features: call pdf_estimate_stats first");
  cudaStream_t st = (cudaStream_t)stream;
  const double *rhs = nullptr, *L2 = nullptr;
  pdf_status s = relax_fields(p, params, st, &rhs, &L2);
  if (s != PDF_OK) return s;
  const int32_t nn = m->d.n_nodes;
  PDF_KERNEL("k_mlp_features", st, k_mlp_features<<<(nn + 255) / 256, 256, 0, st>>>(
                                       nn, rhs, L2, m->rx.wall_d, m->d.nse_off, m->d.nse, m->d.geo, wp, X, Y));
  return PDF_OK;
}

extern "C" pdf_status pdf_mlp_guess(const pdf_mlp* M, pdf_particles* p, const pdf_mesh* m,
                                    const pdf_model_params* params, double* wp, float* scratch, void* stream) {
  if (!M || !p || !m || p->mesh != m || !params || !wp || !scratch)
    return fail(PDF_EINVAL, "pdf_mlp_guess: bad arguments");
  if (!p->have_stats) return fail(PDF_ESTATE, "pdf_mlp_guess: call pdf_estimate_stats first");
  cudaStream_t st = (cudaStream_t)stream;
  const double *rhs = nullptr, *L2 = nullptr;
  pdf_status s = relax_fields(p, params, st, &rhs, &L2);
  if (s != PDF_OK) return s;
  const int32_t nn = m->d.n_nodes;
  float* X = scratch;
  float* Y = scratch + (size_t)nn * kIn;
  PDF_KERNEL("k_mlp_features", st, k_mlp_features<<<(nn + 255) / 256, 256, 0, st>>>(
                                       nn, rhs, L2, m->rx.wall_d, m->d.nse_off, m->d.nse, m->d.geo, nullptr, X,
                                       nullptr));
  s = pdf_mlp_forward(M, X, nn, Y, stream);
  if (s != PDF_OK) return s;
  PDF_KERNEL("k_mlp_to_wp", st, k_mlp_to_wp<<<(nn + 255) / 256, 256, 0, st>>>(nn, Y, rhs, wp));
  return PDF_OK;
}
