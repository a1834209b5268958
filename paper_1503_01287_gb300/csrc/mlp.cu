// The small network of the learned weights: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3,
// x in R^16, two hidden layers of 64, one output, trained on the mean squared error.
//
// Forward and backward passes run 64 samples per CTA.  The three matrix
// products of each layer (H = X W^T, dW = dZ^T H, dX = dZ W) are BF16
// tensor-core MMAs (mma.sync m16n8k16, FP32 accumulate) on operands staged in
// shared memory; weight gradients are summed over CTAs with FP32 atomics; the
// FP32 master weights are updated by Adam.
#include <cuda_bf16.h>

#include <cstdio>
#include <vector>

#include "amg_internal.cuh"

namespace amgp2 {

namespace {

constexpr int NI = 16, NH = 64, TILE = 64;
constexpr int OW1 = 0, OB1 = OW1 + NH * NI, OW2 = OB1 + NH, OB2 = OW2 + NH * NH,
              OW3 = OB2 + NH, OB3 = OW3 + NH, NPARAM = OB3 + 1;

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One 16 x 8 output tile (rows m0.., columns n0..) of C = A B over K (multiple
// of 16), A(m, k) and B(k, n) read through accessors (bf16 values in shared
// memory).  Fragment layout of m16n8k16: lane = 4 g + t; A holds rows g, g+8 at
// columns 2t, 2t+1 (+8); B holds rows 2t, 2t+1 (+8) at column g; C holds rows
// g, g+8 at columns 2t, 2t+1.
template <class FA, class FB>
__device__ __forceinline__ void mma_tile(FA A, FB Bm, int m0, int n0, int K, float c[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4], b[2];
    a[0] = pack2(A(m0 + g, k0 + 2 * t), A(m0 + g, k0 + 2 * t + 1));
    a[1] = pack2(A(m0 + g + 8, k0 + 2 * t), A(m0 + g + 8, k0 + 2 * t + 1));
    a[2] = pack2(A(m0 + g, k0 + 2 * t + 8), A(m0 + g, k0 + 2 * t + 9));
    a[3] = pack2(A(m0 + g + 8, k0 + 2 * t + 8), A(m0 + g + 8, k0 + 2 * t + 9));
    b[0] = pack2(Bm(k0 + 2 * t, n0 + g), Bm(k0 + 2 * t + 1, n0 + g));
    b[1] = pack2(Bm(k0 + 2 * t + 8, n0 + g), Bm(k0 + 2 * t + 9, n0 + g));
    mma16816(c, a, b);
  }
}

struct Smem {
  __nv_bfloat16 w1[NH * NI], w2[NH * NH], x[TILE * NI], h1[TILE * NH], dz2[TILE * NH],
      dz1[TILE * NH];
  float z1[TILE * NH], z2[TILE * NH];
  float w3[NH], b1[NH], b2[NH], y[TILE], dy[TILE];
};

// Forward (and, with BWD, backward) pass of the samples [64 blockIdx.x, +64).
// y: per-sample outputs (may be null); grad: gradient accumulator (BWD);
// loss: accumulator of sum (y - t)^2 / n (BWD with the squared-error loss);
// dyin: when given (BWD), the per-sample gradient dL/dy_i of any loss, used instead
// of the squared error (grad then accumulates sum_i dyin_i dy_i/dtheta).
template <bool BWD>
__global__ void __launch_bounds__(128) k_mlp(const float* __restrict__ theta,
                                             const float* __restrict__ X,
                                             const float* __restrict__ tgt, int n,
                                             float* __restrict__ yout, float* __restrict__ grad,
                                             float* __restrict__ loss,
                                             const float* __restrict__ dyin) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Smem& S = *reinterpret_cast<Smem*>(smraw);
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int s0 = blockIdx.x * TILE;
  for (int q = tid; q < NH * NI; q += nt) S.w1[q] = __float2bfloat16(theta[OW1 + q]);
  for (int q = tid; q < NH * NH; q += nt) S.w2[q] = __float2bfloat16(theta[OW2 + q]);
  for (int q = tid; q < NH; q += nt) {
    S.w3[q] = theta[OW3 + q];
    S.b1[q] = theta[OB1 + q];
    S.b2[q] = theta[OB2 + q];
  }
  for (int q = tid; q < TILE * NI; q += nt) {
    const int s = q / NI;
    S.x[q] = __float2bfloat16(s0 + s < n ? X[(int64_t)(s0 + s) * NI + q % NI] : 0.f);
  }
  __syncthreads();
  const int g = lane >> 2, t = lane & 3;
  // z1 = x W1^T + b1: 4 x 8 tiles of 16 x 8, K = 16
  for (int tile = warp; tile < 32; tile += nt / 32) {
    const int m0 = (tile / 8) * 16, n0 = (tile % 8) * 8;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    mma_tile([&](int m, int k) { return S.x[m * NI + k]; },
             [&](int k, int nn) { return S.w1[nn * NI + k]; }, m0, n0, NI, c);
    const int r[4] = {m0 + g, m0 + g, m0 + g + 8, m0 + g + 8};
    const int cc[4] = {n0 + 2 * t, n0 + 2 * t + 1, n0 + 2 * t, n0 + 2 * t + 1};
    for (int e = 0; e < 4; ++e) {
      const float z = c[e] + S.b1[cc[e]];
      S.z1[r[e] * NH + cc[e]] = z;
      S.h1[r[e] * NH + cc[e]] = __float2bfloat16(fmaxf(z, 0.f));
    }
  }
  __syncthreads();
  // z2 = h1 W2^T + b2, K = 64
  for (int tile = warp; tile < 32; tile += nt / 32) {
    const int m0 = (tile / 8) * 16, n0 = (tile % 8) * 8;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    mma_tile([&](int m, int k) { return S.h1[m * NH + k]; },
             [&](int k, int nn) { return S.w2[nn * NH + k]; }, m0, n0, NH, c);
    const int r[4] = {m0 + g, m0 + g, m0 + g + 8, m0 + g + 8};
    const int cc[4] = {n0 + 2 * t, n0 + 2 * t + 1, n0 + 2 * t, n0 + 2 * t + 1};
    for (int e = 0; e < 4; ++e) S.z2[r[e] * NH + cc[e]] = c[e] + S.b2[cc[e]];
  }
  __syncthreads();
  // y = relu(z2) . w3 + b3
  if (tid < TILE) {
    float acc = theta[OB3];
    for (int j = 0; j < NH; ++j) acc = fmaf(fmaxf(S.z2[tid * NH + j], 0.f), S.w3[j], acc);
    S.y[tid] = acc;
    if (yout && s0 + tid < n) yout[s0 + tid] = acc;
    if (BWD && dyin) {           // upstream gradient given per sample
      S.dy[tid] = (s0 + tid < n) ? dyin[s0 + tid] : 0.f;
    } else if (BWD) {            // mean squared error against tgt
      const float d = (s0 + tid < n) ? acc - tgt[s0 + tid] : 0.f;
      S.dy[tid] = 2.f * d / (float)n;
      atomicAdd(loss, d * d / (float)n);
    }
  }
  if (!BWD) return;
  __syncthreads();
  // output layer gradients and dz2 = dy w3 (z2 > 0)
  if (tid < NH) {
    float gw = 0.f, gb = 0.f;
    for (int s = 0; s < TILE; ++s) {
      const float z = S.z2[s * NH + tid];
      gw = fmaf(S.dy[s], fmaxf(z, 0.f), gw);
      const float dz = z > 0.f ? S.dy[s] * S.w3[tid] : 0.f;
      gb += dz;
      S.dz2[s * NH + tid] = __float2bfloat16(dz);
    }
    atomicAdd(&grad[OW3 + tid], gw);
    atomicAdd(&grad[OB2 + tid], gb);
    if (tid == 0) {
      float gb3 = 0.f;
      for (int s = 0; s < TILE; ++s) gb3 += S.dy[s];
      atomicAdd(&grad[OB3], gb3);
    }
  }
  __syncthreads();
  // dW2 = dz2^T h1 (m: out unit, k: sample, n: in unit) and dz1 = dz2 W2 (z1 > 0)
  for (int tile = warp; tile < 32; tile += nt / 32) {
    const int m0 = (tile / 8) * 16, n0 = (tile % 8) * 8;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    mma_tile([&](int m, int k) { return S.dz2[k * NH + m]; },
             [&](int k, int nn) { return S.h1[k * NH + nn]; }, m0, n0, TILE, c);
    atomicAdd(&grad[OW2 + (m0 + g) * NH + n0 + 2 * t], c[0]);
    atomicAdd(&grad[OW2 + (m0 + g) * NH + n0 + 2 * t + 1], c[1]);
    atomicAdd(&grad[OW2 + (m0 + g + 8) * NH + n0 + 2 * t], c[2]);
    atomicAdd(&grad[OW2 + (m0 + g + 8) * NH + n0 + 2 * t + 1], c[3]);
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    mma_tile([&](int m, int k) { return S.dz2[m * NH + k]; },
             [&](int k, int nn) { return S.w2[k * NH + nn]; }, m0, n0, NH, d);
    const int r[4] = {m0 + g, m0 + g, m0 + g + 8, m0 + g + 8};
    const int cc[4] = {n0 + 2 * t, n0 + 2 * t + 1, n0 + 2 * t, n0 + 2 * t + 1};
    for (int e = 0; e < 4; ++e) {
      const float v = S.z1[r[e] * NH + cc[e]] > 0.f ? d[e] : 0.f;
      S.z2[r[e] * NH + cc[e]] = v;    // z2 no longer needed: holds dz1 in FP32
      S.dz1[r[e] * NH + cc[e]] = __float2bfloat16(v);
    }
  }
  __syncthreads();
  if (tid < NH) {
    float gb = 0.f;
    for (int s = 0; s < TILE; ++s) gb += S.z2[s * NH + tid];
    atomicAdd(&grad[OB1 + tid], gb);
  }
  // dW1 = dz1^T x: 4 x 2 tiles, K = 64
  for (int tile = warp; tile < 8; tile += nt / 32) {
    const int m0 = (tile / 2) * 16, n0 = (tile % 2) * 8;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    mma_tile([&](int m, int k) { return S.dz1[k * NH + m]; },
             [&](int k, int nn) { return S.x[k * NI + nn]; }, m0, n0, TILE, c);
    atomicAdd(&grad[OW1 + (m0 + g) * NI + n0 + 2 * t], c[0]);
    atomicAdd(&grad[OW1 + (m0 + g) * NI + n0 + 2 * t + 1], c[1]);
    atomicAdd(&grad[OW1 + (m0 + g + 8) * NI + n0 + 2 * t], c[2]);
    atomicAdd(&grad[OW1 + (m0 + g + 8) * NI + n0 + 2 * t + 1], c[3]);
  }
}

__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ grad,
                       float* __restrict__ m, float* __restrict__ v, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

constexpr size_t kSmem = sizeof(Smem);

void set_smem() {
  max_dynamic_smem((const void*)k_mlp<true>, (int)kSmem);
  max_dynamic_smem((const void*)k_mlp<false>, (int)kSmem);
}

}  // namespace

int mlp_nparam() { return NPARAM; }

void mlp_forward(const float* theta, const float* X, int n, float* y, cudaStream_t s) {
  set_smem();
  if (n <= 0) return;
  k_mlp<false><<<(n + TILE - 1) / TILE, 128, kSmem, s>>>(theta, X, nullptr, n, y, nullptr,
                                                          nullptr, nullptr);
  AMG_LAUNCH_CHECK();
}

void mlp_gradient(const float* theta, const float* X, const float* t, int n, float* grad,
                  float* loss, cudaStream_t s) {
  set_smem();
  AMG_CUDA(cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), s));
  AMG_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), s));
  if (n <= 0) return;
  k_mlp<true><<<(n + TILE - 1) / TILE, 128, kSmem, s>>>(theta, X, t, n, nullptr, grad, loss,
                                                         nullptr);
  AMG_LAUNCH_CHECK();
}

void mlp_backward(const float* theta, const float* X, const float* dy, int n, float* grad,
                  cudaStream_t s) {
  set_smem();
  AMG_CUDA(cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), s));
  if (n <= 0) return;
  k_mlp<true><<<(n + TILE - 1) / TILE, 128, kSmem, s>>>(theta, X, nullptr, n, nullptr, grad,
                                                         nullptr, dy);
  AMG_LAUNCH_CHECK();
}

void mlp_adam(float* theta, const float* grad, float* m, float* v, int step, float lr,
              cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(theta, grad, m, v, NPARAM, lr, b1, b2, 1e-8f, c1,
                                              c2);
  AMG_LAUNCH_CHECK();
}

}  // namespace amgp2
