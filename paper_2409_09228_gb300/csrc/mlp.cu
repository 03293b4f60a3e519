// The learned path-length seed (mlp.cuh): its training kernels (forward and
// backward of the mean squared error on the tensor cores, Adam), inference,
// the p2r path-length iteration alone, and the p2r fit that seeds every
// layer's iteration from the network.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "fit.h"
#include "fused.cuh"
#include "internal.h"
#include "mlp.cuh"

using namespace fitimpl;
using mlpk::Image;
using mlpk::TrainImage;

struct fit_mlp {
  int device = 0;
  float* d_params = nullptr;  // [kParams] FP32 master
  float* d_m = nullptr;       // Adam first and second moments
  float* d_v = nullptr;
  TrainImage* d_img = nullptr;
  float* d_partials = nullptr;  // [partial_blocks][kPartial]
  int64_t partial_blocks = 0;
  float* d_curve = nullptr;  // loss per epoch
  int curve_cap = 0;
  int64_t step = 0;  // Adam steps taken
  float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
};

namespace {

constexpr int kRows = 64;        // samples per block of the gradient kernel
constexpr int kPartial = 4808;   // per-block partial: gradient [0, 4801), sum of
constexpr int kSse = 4801;       // squared errors, count of finite targets
constexpr int kCount = 4802;
constexpr int kMaxGradSamples = 65536;

// ---- the BF16 fragment image of the parameters ------------------------------

__device__ void build_image(const float* __restrict__ P, TrainImage* img, int tid, int nthr) {
  using namespace mlpk;
  uint32_t* w1 = &img->fwd.w1[0][0].x;
  for (int i = tid; i < 2 * 32 * 4; i += nthr) {
    const int e = i & 3, lane = (i >> 2) & 31, j = i >> 7;
    const int g = lane >> 2, c = lane & 3;
    const int row = (4 * j + e) * 8 + g;
    w1[i] = pack_bf16(P[kOffW1 + row * 8 + 2 * c], P[kOffW1 + row * 8 + 2 * c + 1]);
  }
  uint32_t* w2 = &img->fwd.w2[0][0][0].x;
  uint32_t* w2t = &img->w2t[0][0][0].x;
  for (int i = tid; i < 4 * 4 * 32 * 4; i += nthr) {
    const int e = i & 3, lane = (i >> 2) & 31, j = (i >> 7) & 3, kb = i >> 9;
    const int g = lane >> 2, c = lane & 3;
    const int nb = 2 * j + (e >> 1), k0 = kb * 16 + (e & 1) * 8 + 2 * c, n = nb * 8 + g;
    w2[i] = pack_bf16(P[kOffW2 + n * 64 + k0], P[kOffW2 + n * 64 + k0 + 1]);
    w2t[i] = pack_bf16(P[kOffW2 + k0 * 64 + n], P[kOffW2 + (k0 + 1) * 64 + n]);
  }
  uint32_t* w3 = &img->fwd.w3[0][0].x;
  for (int i = tid; i < 2 * 32 * 4; i += nthr) {
    const int e = i & 3, lane = (i >> 2) & 31, j = i >> 7;
    const int g = lane >> 2, c = lane & 3;
    const int k0 = (2 * j + (e >> 1)) * 16 + (e & 1) * 8 + 2 * c;
    w3[i] = g == 0 ? pack_bf16(P[kOffW3 + k0], P[kOffW3 + k0 + 1]) : 0u;
  }
  for (int i = tid; i < kHid; i += nthr) {
    img->fwd.b1[i] = P[kOffB1 + i];
    img->fwd.b2[i] = P[kOffB2 + i];
    img->w3f[i] = bf16_round(P[kOffW3 + i]);
  }
  if (tid == 0) {
    img->fwd.b3 = P[kOffB3];
    img->fwd.pad[0] = img->fwd.pad[1] = img->fwd.pad[2] = 0.f;
  }
}

__global__ void __launch_bounds__(1024) mlp_image_kernel(const float* __restrict__ P,
                                                         TrainImage* img) {
  build_image(P, img, threadIdx.x, blockDim.x);
}

// ---- inputs and targets -------------------------------------------------------

__global__ void __launch_bounds__(256)
    mlp_prepare_kernel(float kB, const float* __restrict__ par, int64_t ld,
                       const int32_t* __restrict__ q, const float* __restrict__ R,
                       const float* __restrict__ h_exact, int64_t n, float* __restrict__ x,
                       float* __restrict__ target) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float p[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = par[k * ld + i];
  const fitk::Trig<float> g = fitk::trig_of(p);
  const float qf = (float)q[i], Ri = R[i];
  float f[mlpk::kIn];
  mlpk::features(p, g.cphi, g.sphi, g.cth, qf, kB, Ri, f);
  float4* xo = reinterpret_cast<float4*>(x + i * mlpk::kIn);
  xo[0] = make_float4(f[0], f[1], f[2], f[3]);
  xo[1] = make_float4(f[4], f[5], f[6], f[7]);
  if (!target) return;
  // straight-line distance along the momentum to the cylinder, from inside
  const float kappa = -qf * kB * p[3];
  const float b0 = fmaf(p[0], g.cphi, p[1] * g.sphi);
  const float c0 = fmaf(p[0], p[0], fmaf(p[1], p[1], -Ri * Ri));
  const float disc = fmaf(b0, b0, -c0);
  float t = __int_as_float(0x7fc00000);
  if (c0 <= 0.f && disc >= 0.f && kappa != 0.f) {
    const float sq = sqrtf(disc);
    const float hl = b0 > 0.f ? -c0 / (b0 + sq) : sq - b0;
    t = (h_exact[i] - hl) / (0.5f * kappa * hl * hl);
  }
  target[i] = t;
}

// ---- inference ------------------------------------------------------------------

__global__ void __launch_bounds__(kBlock) mlp_forward_kernel(const Image* __restrict__ img,
                                                             const float* __restrict__ x,
                                                             int64_t n, float* __restrict__ y) {
  __shared__ Image W;
  __shared__ uint4 stage[kBlock / 32][64];
  mlpk::copy_image(W, img);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  float f[mlpk::kIn] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (i < n) {
    const float4* xi = reinterpret_cast<const float4*>(x + i * mlpk::kIn);
    const float4 u = __ldg(xi), v = __ldg(xi + 1);
    f[0] = u.x, f[1] = u.y, f[2] = u.z, f[3] = u.w, f[4] = v.x, f[5] = v.y, f[6] = v.z, f[7] = v.w;
  }
  const float out = mlpk::infer_warp(W, stage[threadIdx.x >> 5], f);
  if (i < n) y[i] = out;
}

// ---- training: forward + backward of one block of 64 samples ---------------------

// Shared memory of the gradient kernel.  The BF16 matrices staged for the
// weight-gradient contractions are [64 samples][64 columns] in 16-byte
// chunks of 8 columns, chunk index XOR (row % 8) so that eight consecutive
// rows of one chunk fall in different banks.
struct GradSmem {
  TrainImage W;
  uint4 xs[2][kRows];  // hi and lo halves of the inputs, one 16-byte row per sample
  uint4 dz2[kRows][8];
  uint4 a1[kRows][8];
  uint4 dz1[kRows][8];
  float red[3 * 64 + 3];  // db1, db2, dW3, db3, sum of squared errors, count
};

__device__ __forceinline__ uint32_t* swz(uint4 (*m)[8], int row, int chunk) {
  return &m[row][chunk ^ (row & 7)].x;
}

// Stores the four A-fragment registers of one k-block (rows g and g + 8 of the
// warp's tile, columns 16 kb .. 16 kb + 15) into a staged matrix.
__device__ __forceinline__ void stage_a(uint4 (*m)[8], int r0, int kb, int c,
                                        const uint32_t (&a)[4]) {
  swz(m, r0, 2 * kb)[c] = a[0];
  swz(m, r0 + 8, 2 * kb)[c] = a[1];
  swz(m, r0, 2 * kb + 1)[c] = a[2];
  swz(m, r0 + 8, 2 * kb + 1)[c] = a[3];
}

// Sum over the eight lanes with the same c (lane bits 2..4).
__device__ __forceinline__ float sum_over_g(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

// Block b takes samples (off + 64 b + r) mod n, r < 64, of the first cnt of
// the batch; each of the four warps a 16-sample tile.  Writes the block's
// partial gradient of (1/cnt) sum (y - t)^2, its sum of squared errors and
// its count of finite targets to partials[b].
__global__ void __launch_bounds__(kBlock) mlp_grad_kernel(const TrainImage* __restrict__ img,
                                                          const float* __restrict__ X,
                                                          const float* __restrict__ T, int64_t n,
                                                          int64_t off, int64_t cnt, float inv_cnt,
                                                          float* __restrict__ partials) {
  using namespace mlpk;
  __shared__ GradSmem S;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, c = lane & 3;
  copy_image(S.W, img);
  for (int i = tid; i < 3 * 64 + 3; i += kBlock) S.red[i] = 0.f;
  const int64_t base = (int64_t)blockIdx.x * kRows;
  if (tid < kRows) {
    float f[kIn] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (base + tid < cnt) {
      const float4* xi = reinterpret_cast<const float4*>(X + ((off + base + tid) % n) * kIn);
      const float4 u = __ldg(xi), v = __ldg(xi + 1);
      f[0] = u.x, f[1] = u.y, f[2] = u.z, f[3] = u.w, f[4] = v.x, f[5] = v.y, f[6] = v.z, f[7] = v.w;
    }
    stage_inputs(f, &S.xs[0][tid], &S.xs[1][tid]);
  }
  __syncthreads();

  // forward, keeping the pre-activations for the ReLU derivatives
  const int r0 = warp * 16 + g;  // this lane's rows r0 and r0 + 8
  uint32_t a[4];
  ldsm_x4(a, &S.xs[lane >> 4][warp * 16 + (lane & 15)]);
  float z1[8][4];
  layer1(S.W.fwd, a, lane, z1);
  uint32_t a1f[4][4];
  to_a_relu(z1, a1f);
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) stage_a(S.a1, r0, kb, c, a1f[kb]);
  float z2[8][4];
  layer2(S.W.fwd, a1f, lane, z2);
  uint32_t a2f[4][4];
  to_a_relu(z2, a2f);
  float o[4];
  layer3(S.W.fwd, a2f, lane, o);

  // output error (lanes c = 0 hold rows r0 and r0 + 8), broadcast over the quad
  float e0 = 0.f, e1 = 0.f, nval = 0.f;
  if (c == 0) {
    const int64_t b0 = base + r0, b1 = base + r0 + 8;
    if (b0 < cnt) {
      const float t = __ldg(T + (off + b0) % n);
      if (isfinite(t)) e0 = o[0] - t, nval += 1.f;
    }
    if (b1 < cnt) {
      const float t = __ldg(T + (off + b1) % n);
      if (isfinite(t)) e1 = o[2] - t, nval += 1.f;
    }
  }
  float sse = e0 * e0 + e1 * e1;
  const float dy0 = __shfl_sync(0xffffffffu, 2.f * e0 * inv_cnt, lane & ~3);
  const float dy1 = __shfl_sync(0xffffffffu, 2.f * e1 * inv_cnt, lane & ~3);
  float db3 = c == 0 ? dy0 + dy1 : 0.f;

  // layer 3 and 2: dW3 = sum dy a2, dz2 = dy W3 [z2 > 0], db2 = sum dz2
  float dz2[8][4], gw3[8][2], gb2[8][2];
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) {
    const uint32_t ra = a2f[nb >> 1][(nb & 1) ? 2 : 0], rb = a2f[nb >> 1][(nb & 1) ? 3 : 1];
    gw3[nb][0] = fmaf(dy0, bf16_lo(ra), dy1 * bf16_lo(rb));
    gw3[nb][1] = fmaf(dy0, bf16_hi(ra), dy1 * bf16_hi(rb));
    const float w0 = S.W.w3f[nb * 8 + 2 * c], w1 = S.W.w3f[nb * 8 + 2 * c + 1];
    dz2[nb][0] = z2[nb][0] > 0.f ? dy0 * w0 : 0.f;
    dz2[nb][1] = z2[nb][1] > 0.f ? dy0 * w1 : 0.f;
    dz2[nb][2] = z2[nb][2] > 0.f ? dy1 * w0 : 0.f;
    dz2[nb][3] = z2[nb][3] > 0.f ? dy1 * w1 : 0.f;
    gb2[nb][0] = dz2[nb][0] + dz2[nb][2];
    gb2[nb][1] = dz2[nb][1] + dz2[nb][3];
  }
  uint32_t dzf[4][4];
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    dzf[kb][0] = pack_bf16(dz2[2 * kb][0], dz2[2 * kb][1]);
    dzf[kb][1] = pack_bf16(dz2[2 * kb][2], dz2[2 * kb][3]);
    dzf[kb][2] = pack_bf16(dz2[2 * kb + 1][0], dz2[2 * kb + 1][1]);
    dzf[kb][3] = pack_bf16(dz2[2 * kb + 1][2], dz2[2 * kb + 1][3]);
    stage_a(S.dz2, r0, kb, c, dzf[kb]);
  }

  // layer 1: dA1 = dZ2 W2, dz1 = dA1 [z1 > 0], db1 = sum dz1
  float da1[8][4];
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) da1[nb][0] = da1[nb][1] = da1[nb][2] = da1[nb][3] = 0.f;
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint4 w = S.W.w2t[kb][j][lane];
      mma_acc(da1[2 * j], dzf[kb], w.x, w.y);
      mma_acc(da1[2 * j + 1], dzf[kb], w.z, w.w);
    }
  }
  float gb1[8][2];
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) {
#pragma unroll
    for (int k = 0; k < 4; ++k) da1[nb][k] = z1[nb][k] > 0.f ? da1[nb][k] : 0.f;
    gb1[nb][0] = da1[nb][0] + da1[nb][2];
    gb1[nb][1] = da1[nb][1] + da1[nb][3];
  }
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    const uint32_t d[4] = {pack_bf16(da1[2 * kb][0], da1[2 * kb][1]),
                           pack_bf16(da1[2 * kb][2], da1[2 * kb][3]),
                           pack_bf16(da1[2 * kb + 1][0], da1[2 * kb + 1][1]),
                           pack_bf16(da1[2 * kb + 1][2], da1[2 * kb + 1][3])};
    stage_a(S.dz1, r0, kb, c, d);
  }

  // bias and dW3 sums over the block's rows
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float v1 = sum_over_g(gb1[nb][e]), v2 = sum_over_g(gb2[nb][e]),
                  v3 = sum_over_g(gw3[nb][e]);
      if (g == 0) {
        atomicAdd(&S.red[nb * 8 + 2 * c + e], v1);
        atomicAdd(&S.red[64 + nb * 8 + 2 * c + e], v2);
        atomicAdd(&S.red[128 + nb * 8 + 2 * c + e], v3);
      }
    }
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    db3 += __shfl_xor_sync(0xffffffffu, db3, m);
    sse += __shfl_xor_sync(0xffffffffu, sse, m);
    nval += __shfl_xor_sync(0xffffffffu, nval, m);
  }
  if (lane == 0) {
    atomicAdd(&S.red[192], db3);
    atomicAdd(&S.red[193], sse);
    atomicAdd(&S.red[194], nval);
  }
  __syncthreads();

  // weight gradients, contracted over the block's 64 samples on the tensor
  // cores: dW2[j][i] = sum_s dz2[s][j] a1[s][i] and dW1[j][k] = sum_s dz1[s][j]
  // (hi + lo)[s][k]; warp w takes the output rows j = 16 w .. 16 w + 15.
  float gw2[8][4], gw1[2][4];
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) gw2[nb][0] = gw2[nb][1] = gw2[nb][2] = gw2[nb][3] = 0.f;
  gw1[0][0] = gw1[0][1] = gw1[0][2] = gw1[0][3] = 0.f;
  gw1[1][0] = gw1[1][1] = gw1[1][2] = gw1[1][3] = 0.f;
#pragma unroll
  for (int ks = 0; ks < kRows / 16; ++ks) {
    const int sa = ks * 16 + (lane & 7) + ((lane >> 4) & 1) * 8;  // A: dz^T, rows of samples
    const int ca = 2 * warp + ((lane >> 3) & 1);
    const int sb = ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;  // B: rows of samples
    uint32_t A2[4], A1[4];
    ldsm_x4_trans(A2, swz(S.dz2, sa, ca));
    ldsm_x4_trans(A1, swz(S.dz1, sa, ca));
#pragma unroll
    for (int np = 0; np < 4; ++np) {
      uint32_t Bq[4];
      ldsm_x4_trans(Bq, swz(S.a1, sb, 2 * np + (lane >> 4)));
      mma_acc(gw2[2 * np], A2, Bq[0], Bq[1]);
      mma_acc(gw2[2 * np + 1], A2, Bq[2], Bq[3]);
    }
    uint32_t Bx[4];
    ldsm_x4_trans(Bx, &S.xs[lane >> 4][sb]);
    mma_acc(gw1[0], A1, Bx[0], Bx[1]);
    mma_acc(gw1[1], A1, Bx[2], Bx[3]);
  }

  float* P = partials + (int64_t)blockIdx.x * kPartial;
  const int j0 = warp * 16 + g;
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) {
    const int i0 = nb * 8 + 2 * c;
    *reinterpret_cast<float2*>(&P[kOffW2 + j0 * 64 + i0]) = make_float2(gw2[nb][0], gw2[nb][1]);
    *reinterpret_cast<float2*>(&P[kOffW2 + (j0 + 8) * 64 + i0]) =
        make_float2(gw2[nb][2], gw2[nb][3]);
  }
  P[kOffW1 + j0 * 8 + 2 * c] = gw1[0][0] + gw1[1][0];
  P[kOffW1 + j0 * 8 + 2 * c + 1] = gw1[0][1] + gw1[1][1];
  P[kOffW1 + (j0 + 8) * 8 + 2 * c] = gw1[0][2] + gw1[1][2];
  P[kOffW1 + (j0 + 8) * 8 + 2 * c + 1] = gw1[0][3] + gw1[1][3];
  for (int i = tid; i < 64; i += kBlock) {
    P[kOffB1 + i] = S.red[i];
    P[kOffB2 + i] = S.red[64 + i];
    P[kOffW3 + i] = S.red[128 + i];
  }
  if (tid == 0) {
    P[kOffB3] = S.red[192];
    P[kSse] = S.red[193];
    P[kCount] = S.red[194];
  }
}

// Sum of the per-block partials (fixed order): gradient and mean loss.
__global__ void __launch_bounds__(256)
    mlp_reduce_kernel(const float* __restrict__ partials, int nblk, float inv_cnt,
                      float* __restrict__ grad, float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < mlpk::kParams) {
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += partials[(int64_t)b * kPartial + i];
    grad[i] = s;
  }
  if (i == 0) {
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += partials[(int64_t)b * kPartial + kSse];
    *loss = s * inv_cnt;
  }
}

// One Adam step (Kingma and Ba, 2015, Algorithm 1) with the gradient grad, or
// the sum of nblk partials when grad is NULL; bc1 = 1 - beta1^t and
// bc2 = 1 - beta2^t; one parameter per thread over the grid.  Block 0 adds
// curve_scale times the partials' squared errors to *curve.  The BF16 image
// is rebuilt from the new parameters by mlp_image_kernel afterwards.
constexpr int kAdamThreads = 256;
constexpr int kAdamBlocks = (mlpk::kParams + kAdamThreads - 1) / kAdamThreads;

__global__ void __launch_bounds__(kAdamThreads)
    mlp_adam_kernel(float* __restrict__ P, float* __restrict__ M, float* __restrict__ V,
                    const float* __restrict__ grad, const float* __restrict__ partials, int nblk,
                    float lr, float beta1, float beta2, float eps, float bc1, float bc2,
                    float* curve, float curve_scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < mlpk::kParams) {
    float gi;
    if (grad) {
      gi = grad[i];
    } else {
      gi = 0.f;
      for (int b = 0; b < nblk; ++b) gi += partials[(int64_t)b * kPartial + i];
    }
    const float m = fmaf(beta1, M[i], (1.f - beta1) * gi);
    const float v = fmaf(beta2, V[i], (1.f - beta2) * gi * gi);
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
  }
  if (curve && i == 0) {
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += partials[(int64_t)b * kPartial + kSse];
    *curve += s * curve_scale;
  }
}

// ---- the p2r path-length iteration alone ---------------------------------------

// One state per thread; every thread of the block stays to the end so that the
// warps can evaluate the network together.
template <bool SEED>
__global__ void __launch_bounds__(kBlock)
    path_length_kernel(const Image* __restrict__ img, float kB, int max_iter, float tol,
                       bool line_start, const float* __restrict__ par, int64_t ld,
                       const int32_t* __restrict__ q, const float* __restrict__ R, int64_t n,
                       float* __restrict__ h_out, int32_t* __restrict__ it_out) {
  __shared__ Image W;
  __shared__ uint4 stage[kBlock / 32][64];
  if (SEED) {
    mlpk::copy_image(W, img);
    __syncthreads();
  }
  const int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const bool valid = i < n;
  float p[6] = {1.f, 0.f, 0.f, 1.f, 0.f, 1.5707964f};
  float qf = 1.f, Ri = 2.f;
  if (valid) {
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k] = __ldg(par + k * ld + i);
    qf = (float)__ldg(q + i);
    Ri = __ldg(R + i);
  }
  const fitk::Trig<float> g = fitk::trig_of(p);
  float gs = 0.f;
  if (SEED) {
    float f[mlpk::kIn];
    mlpk::features(p, g.cphi, g.sphi, g.cth, qf, kB, Ri, f);
    gs = mlpk::infer_warp(W, stage[threadIdx.x >> 5], f);
  }
  if (!valid) return;
  unsigned it[1] = {0u};
  bool nc = false;
  fitk::PathR<float> w;
  const bool failed =
      fitk::path_r<float, SEED>(p, g, -qf * kB * p[3], Ri, max_iter, tol * Ri, line_start, it,
                                nc, w, gs);
  h_out[i] = failed ? __int_as_float(0x7fc00000) : w.h;
  if (it_out) it_out[i] = failed ? 0 : (int32_t)it[0];
}

// ---- the p2r fit with the learned seed -----------------------------------------

// One track per thread (not two, as in fit_fused_kernel): all 32 lanes of a
// warp evaluate the network together before every layer, so no thread leaves
// the layer loop early; a track that stops (surface not reached, non-finite
// update) only stops moving.  Outputs, status bits and counters as
// fit_fused_kernel<FIT_MODE_R>.
__global__ void __launch_bounds__(kBlock) fit_seeded_kernel(const __grid_constant__ FitArgs a,
                                                            const Image* __restrict__ img) {
  __shared__ Image W;
  __shared__ uint4 stage[kBlock / 32][64];
  mlpk::copy_image(W, img);
  __syncthreads();
  const int64_t t = a.t0 + (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const bool valid = t < a.t1;
  State<float> s;
  if (valid) {
    load_state(a, t, s);
  } else {
    const float p0[6] = {1.f, 0.f, 0.f, 1.f, 0.f, 1.5707964f};
#pragma unroll
    for (int k = 0; k < 6; ++k) s.p[k] = p0[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) s.c[k] = 0.f;
    s.qf = 1.f;
    s.chi2 = 0.f;
    s.g = fitk::trig_of(s.p);
  }
  const Geo& geo = a.geo;
  unsigned st = 0u, iters[1] = {0u};
  bool moving = valid;
  const int64_t ldh = a.ld_hit;
  for (int l = 0; l < a.nlayer; ++l) {
    if (!__any_sync(0xffffffffu, moving)) break;
    const float sf = geo.surf.s[l];
    float f[mlpk::kIn];
    mlpk::features(s.p, s.g.cphi, s.g.sphi, s.g.cth, s.qf, geo.kB, sf, f);
    const float gs = mlpk::infer_warp(W, stage[threadIdx.x >> 5], f);
    if (!moving) continue;
    float m[3], v[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) fitk::ld(m[k], a.hpos + (3 * l + k) * ldh + t);
#pragma unroll
    for (int k = 0; k < 6; ++k) fitk::ld(v[k], a.hcov + (6 * l + k) * ldh + t);
    bool nc = false;
    const bool failed = fitk::prop_r<float, true>(s.p, s.c, s.g, s.qf * -geo.kB, sf, geo.max_iter,
                                                  geo.tol * sf, false, iters, nc, gs);
    if (failed) {
      st |= FIT_ST_NO_INTERSECTION;
      if (a.chi2_layer)
        for (int r = l; r < a.nlayer; ++r) a.chi2_layer[(int64_t)r * a.ld_out + t] = 0.f;
      moving = false;
      continue;
    }
    const float phi_pred = s.p[4], th_pred = s.p[5];
    float x2 = fitk::update_r(s.p, s.c, m, v);
    const bool flip = fitk::normalise(s.p, s.c, s.qf, s.g, phi_pred, th_pred);
    const bool alive = fitk::finite_(x2);
    if (nc) st |= FIT_ST_NOT_CONVERGED;
    if (flip) st |= FIT_ST_CHARGE_FLIP;
    if (!alive) st |= FIT_ST_NONFINITE;
    x2 = alive ? x2 : 0.f;
    s.chi2 += x2;
    if (a.chi2_layer) a.chi2_layer[(int64_t)l * a.ld_out + t] = x2;
    if (!alive) {
      if (a.chi2_layer)
        for (int r = l + 1; r < a.nlayer; ++r) a.chi2_layer[(int64_t)r * a.ld_out + t] = 0.f;
      moving = false;
    }
  }
  if (valid) {
    unsigned st1[1] = {st};
    store_state(a, t, s, st1);
    if (st1[0]) count_status(st1[0], a.counters);
  }
  count_iterations(valid ? iters[0] : 0u, &a.counters[4]);
}

// ---- host helpers ------------------------------------------------------------------

uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Grows the partials buffer; earlier asynchronous calls may still read the old
// one, so the device is drained first.
int ensure_partials(fit_mlp* m, int64_t nblk) {
  if (nblk <= m->partial_blocks) return FIT_OK;
  if (m->d_partials) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "fit_mlp: synchronize");
    cudaFree(m->d_partials);
  }
  m->d_partials = nullptr;
  m->partial_blocks = 0;
  cudaError_t e = cudaMalloc(&m->d_partials, (size_t)nblk * kPartial * sizeof(float));
  if (e != cudaSuccess) return fail(FIT_ERR_NOMEM, std::string("fit_mlp: cudaMalloc: ") +
                                                       cudaGetErrorString(e));
  m->partial_blocks = nblk;
  return FIT_OK;
}

int upload_params(fit_mlp* m, const float* host) {
  cudaError_t e = cudaMemcpy(m->d_params, host, mlpk::kParams * sizeof(float),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, mlpk::kParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, mlpk::kParams * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, "fit_mlp: upload");
  m->step = 0;
  mlp_image_kernel<<<1, 1024>>>(m->d_params, m->d_img);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "fit_mlp: image");
  return FIT_OK;
}

int launch_adam(fit_mlp* m, const float* grad, int nblk, float lr, float* curve, float scale,
                cudaStream_t s) {
  m->step += 1;
  const double bc1 = 1.0 - std::pow((double)m->beta1, (double)m->step);
  const double bc2 = 1.0 - std::pow((double)m->beta2, (double)m->step);
  mlp_adam_kernel<<<kAdamBlocks, kAdamThreads, 0, s>>>(m->d_params, m->d_m, m->d_v, grad,
                                                        m->d_partials, nblk, lr, m->beta1, m->beta2,
                                                        m->eps, (float)bc1, (float)bc2, curve, scale);
  mlp_image_kernel<<<1, 1024, 0, s>>>(m->d_params, m->d_img);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FIT_OK : cuda_fail(e, "fit_mlp: Adam launch");
}

}  // namespace

namespace fitimpl {

void launch_seeded_fit(const FitArgs& a, const void* img, cudaStream_t s) {
  const int64_t nblk = (a.t1 - a.t0 + kBlock - 1) / kBlock;
  fit_seeded_kernel<<<(unsigned)nblk, kBlock, 0, s>>>(a, static_cast<const Image*>(img));
}

size_t mlp_image_bytes() { return sizeof(Image); }

}  // namespace fitimpl

extern "C" {

int fit_mlp_create(fit_mlp** out, int device, uint64_t seed) {
  g_last_error.clear();
  if (!out) return fail(FIT_ERR_ARG, "fit_mlp_create: NULL argument");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "fit_mlp_create: cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(FIT_ERR_ARG, "fit_mlp_create: no such device");
  DeviceGuard guard(device);
  fit_mlp* m = new fit_mlp();
  m->device = device;
  const size_t pb = mlpk::kParams * sizeof(float);
  if (cudaMalloc(&m->d_params, pb) != cudaSuccess || cudaMalloc(&m->d_m, pb) != cudaSuccess ||
      cudaMalloc(&m->d_v, pb) != cudaSuccess ||
      cudaMalloc(&m->d_img, sizeof(TrainImage)) != cudaSuccess) {
    fit_mlp_destroy(m);
    return fail(FIT_ERR_NOMEM, "fit_mlp_create: cudaMalloc");
  }
  // He-uniform weights (bound sqrt(6 / fan_in)), zero biases
  std::vector<float> P(mlpk::kParams, 0.f);
  uint64_t x = seed;
  auto uni = [&](float bound) {
    const double u = (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0);
    return (float)((2.0 * u - 1.0) * bound);
  };
  for (int i = 0; i < 512; ++i) P[mlpk::kOffW1 + i] = uni(std::sqrt(6.f / 8.f));
  for (int i = 0; i < 4096; ++i) P[mlpk::kOffW2 + i] = uni(std::sqrt(6.f / 64.f));
  for (int i = 0; i < 64; ++i) P[mlpk::kOffW3 + i] = uni(std::sqrt(6.f / 64.f));
  const int rc = upload_params(m, P.data());
  if (rc != FIT_OK) {
    fit_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return FIT_OK;
}

void fit_mlp_destroy(fit_mlp* m) {
  if (!m) return;
  {
    DeviceGuard guard(m->device);
    cudaDeviceSynchronize();
    cudaFree(m->d_params);
    cudaFree(m->d_m);
    cudaFree(m->d_v);
    cudaFree(m->d_img);
    cudaFree(m->d_partials);
    cudaFree(m->d_curve);
  }
  delete m;
}

int fit_mlp_set_params(fit_mlp* m, const float* params) {
  g_last_error.clear();
  if (!m || !params) return fail(FIT_ERR_ARG, "fit_mlp_set_params: NULL argument");
  DeviceGuard guard(m->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "fit_mlp_set_params");
  return upload_params(m, params);
}

int fit_mlp_get_params(const fit_mlp* m, float* params) {
  g_last_error.clear();
  if (!m || !params) return fail(FIT_ERR_ARG, "fit_mlp_get_params: NULL argument");
  DeviceGuard guard(m->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(params, m->d_params, mlpk::kParams * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? FIT_OK : cuda_fail(e, "fit_mlp_get_params");
}

int fit_mlp_prepare(float B, const float* par, int64_t ld, const int32_t* q, const float* R,
                    const float* h_exact, int64_t n, float* x, float* target, void* stream) {
  g_last_error.clear();
  if (n < 0 || ld < n) return fail(FIT_ERR_ARG, "fit_mlp_prepare: n < 0 or ld < n");
  if (n == 0) return FIT_OK;
  if (!par || !q || !R || !x || (!h_exact != !target))
    return fail(FIT_ERR_ARG, "fit_mlp_prepare: NULL argument (h_exact and target go together)");
  if (!aligned16(x)) return fail(FIT_ERR_ARG, "fit_mlp_prepare: x must be 16-byte aligned");
  if (!(B == B)) return fail(FIT_ERR_ARG, "fit_mlp_prepare: B is NaN");
  const int64_t nblk = (n + 255) / 256;
  if (nblk > 0x7fffffff) return fail(FIT_ERR_ARG, "fit_mlp_prepare: n too large");
  mlp_prepare_kernel<<<(unsigned)nblk, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      (float)(0.00299792458 * (double)B), par, ld, q, R, h_exact, n, x, target);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FIT_OK : cuda_fail(e, "fit_mlp_prepare: launch");
}

int fit_mlp_forward(const fit_mlp* m, const float* x, int64_t n, float* y, void* stream) {
  g_last_error.clear();
  if (!m || n < 0) return fail(FIT_ERR_ARG, "fit_mlp_forward: NULL network or n < 0");
  if (n == 0) return FIT_OK;
  if (!x || !y || !aligned16(x))
    return fail(FIT_ERR_ARG, "fit_mlp_forward: NULL or misaligned buffer");
  const int64_t nblk = (n + kBlock - 1) / kBlock;
  if (nblk > 0x7fffffff) return fail(FIT_ERR_ARG, "fit_mlp_forward: n too large");
  DeviceGuard guard(m->device);
  mlp_forward_kernel<<<(unsigned)nblk, kBlock, 0, static_cast<cudaStream_t>(stream)>>>(
      &m->d_img->fwd, x, n, y);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FIT_OK : cuda_fail(e, "fit_mlp_forward: launch");
}

int fit_mlp_gradient(fit_mlp* m, const float* x, const float* target, int64_t n, float* grad,
                     float* loss, void* stream) {
  g_last_error.clear();
  if (!m || !x || !target || !grad || !loss)
    return fail(FIT_ERR_ARG, "fit_mlp_gradient: NULL argument");
  if (n < 1 || n > kMaxGradSamples)
    return fail(FIT_ERR_ARG, "fit_mlp_gradient: n out of [1, 65536]");
  if (!aligned16(x)) return fail(FIT_ERR_ARG, "fit_mlp_gradient: x must be 16-byte aligned");
  DeviceGuard guard(m->device);
  const int nblk = (int)((n + kRows - 1) / kRows);
  int rc = ensure_partials(m, nblk);
  if (rc != FIT_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mlp_grad_kernel<<<nblk, kBlock, 0, s>>>(m->d_img, x, target, n, 0, n, 1.f / (float)n,
                                          m->d_partials);
  mlp_reduce_kernel<<<(mlpk::kParams + 255) / 256, 256, 0, s>>>(m->d_partials, nblk,
                                                                1.f / (float)n, grad, loss);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FIT_OK : cuda_fail(e, "fit_mlp_gradient: launch");
}

int fit_mlp_adam_step(fit_mlp* m, const float* grad, float lr, void* stream) {
  g_last_error.clear();
  if (!m || !grad) return fail(FIT_ERR_ARG, "fit_mlp_adam_step: NULL argument");
  if (!(lr >= 0.f)) return fail(FIT_ERR_ARG, "fit_mlp_adam_step: lr must be >= 0");
  DeviceGuard guard(m->device);
  return launch_adam(m, grad, 0, lr, nullptr, 0.f, static_cast<cudaStream_t>(stream));
}

int fit_mlp_train(fit_mlp* m, const float* x, const float* target, int64_t n,
                  const fit_mlp_train_config* cfg, float* loss_per_epoch, void* stream) {
  g_last_error.clear();
  if (!m || !x || !target || !cfg) return fail(FIT_ERR_ARG, "fit_mlp_train: NULL argument");
  if (cfg->epochs < 1 || cfg->batch < kRows || cfg->batch > kMaxGradSamples || n < cfg->batch)
    return fail(FIT_ERR_ARG, "fit_mlp_train: need epochs >= 1, 64 <= batch <= 65536, n >= batch");
  if (!(cfg->lr > 0.f) || !(cfg->lr_final >= 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
      !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps > 0.f))
    return fail(FIT_ERR_ARG, "fit_mlp_train: invalid learning rate or Adam setting");
  if (!aligned16(x)) return fail(FIT_ERR_ARG, "fit_mlp_train: x must be 16-byte aligned");
  DeviceGuard guard(m->device);
  const int nblk = (cfg->batch + kRows - 1) / kRows;
  int rc = ensure_partials(m, nblk);
  if (rc != FIT_OK) return rc;
  if (cfg->epochs > m->curve_cap) {
    if (m->d_curve) cudaDeviceSynchronize();
    cudaFree(m->d_curve);
    m->d_curve = nullptr;
    m->curve_cap = 0;
    if (cudaMalloc(&m->d_curve, cfg->epochs * sizeof(float)) != cudaSuccess)
      return fail(FIT_ERR_NOMEM, "fit_mlp_train: cudaMalloc");
    m->curve_cap = cfg->epochs;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(m->d_curve, 0, cfg->epochs * sizeof(float), s);
  if (e != cudaSuccess) return cuda_fail(e, "fit_mlp_train: memset");
  m->beta1 = cfg->beta1;
  m->beta2 = cfg->beta2;
  m->eps = cfg->eps;
  const int64_t steps = n / cfg->batch;
  const int64_t total = steps * cfg->epochs;
  const float scale = 1.f / (float)((double)cfg->batch * (double)steps);
  uint64_t rs = cfg->seed;
  int64_t t = 0;
  for (int ep = 0; ep < cfg->epochs; ++ep) {
    const int64_t start = (int64_t)(splitmix64(rs) % (uint64_t)n);
    for (int64_t k = 0; k < steps; ++k, ++t) {
      const double frac = total > 1 ? (double)t / (double)(total - 1) : 0.0;
      const float lr = (float)(cfg->lr_final + 0.5 * (cfg->lr - cfg->lr_final) *
                                                   (1.0 + std::cos(3.14159265358979323846 * frac)));
      mlp_grad_kernel<<<nblk, kBlock, 0, s>>>(m->d_img, x, target, n, (start + k * cfg->batch) % n,
                                              cfg->batch, 1.f / (float)cfg->batch, m->d_partials);
      rc = launch_adam(m, nullptr, nblk, lr, m->d_curve + ep, scale, s);
      if (rc != FIT_OK) return rc;
    }
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "fit_mlp_train: synchronize");
  if (loss_per_epoch) {
    e = cudaMemcpy(loss_per_epoch, m->d_curve, cfg->epochs * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "fit_mlp_train: copy losses");
  }
  return FIT_OK;
}

int fit_mlp_attach(fit_handle* h, const fit_mlp* m, void* stream) {
  g_last_error.clear();
  if (!h) return fail(FIT_ERR_ARG, "fit_mlp_attach: NULL handle");
  if (!m) {
    h->seeded = false;
    return FIT_OK;
  }
  if (m->device != h->device)
    return fail(FIT_ERR_ARG, "fit_mlp_attach: network and handle on different devices");
  DeviceGuard guard(h->device);
  if (!h->d_mlp) {
    cudaError_t e = cudaMalloc(&h->d_mlp, sizeof(Image));
    if (e != cudaSuccess) return fail(FIT_ERR_NOMEM, "fit_mlp_attach: cudaMalloc");
  }
  cudaError_t e = cudaMemcpyAsync(h->d_mlp, &m->d_img->fwd, sizeof(Image),
                                  cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "fit_mlp_attach: copy");
  h->seeded = true;
  return FIT_OK;
}

int fit_path_lengths(fit_handle* h, const float* par, int64_t ld, const int32_t* q,
                     const float* R, int64_t n, float* h_out, int32_t* iters_out, int seeded,
                     void* stream) {
  g_last_error.clear();
  if (!h) return fail(FIT_ERR_ARG, "fit_path_lengths: NULL handle");
  if (!h->has[FIT_MODE_R]) return fail(FIT_ERR_ARG, "fit_path_lengths: p2r not configured");
  if (seeded && !h->seeded) return fail(FIT_ERR_ARG, "fit_path_lengths: no network attached");
  if (n < 0 || ld < n) return fail(FIT_ERR_ARG, "fit_path_lengths: n < 0 or ld < n");
  if (n == 0) return FIT_OK;
  if (!par || !q || !R || !h_out) return fail(FIT_ERR_ARG, "fit_path_lengths: NULL argument");
  const int64_t nblk = (n + kBlock - 1) / kBlock;
  if (nblk > 0x7fffffff) return fail(FIT_ERR_ARG, "fit_path_lengths: n too large");
  DeviceGuard guard(h->device);
  const Geo& geo = h->geo[FIT_MODE_R];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Image* img = static_cast<const Image*>(h->d_mlp);
  if (seeded)
    path_length_kernel<true><<<(unsigned)nblk, kBlock, 0, s>>>(
        img, geo.kB, geo.max_iter, geo.tol, geo.line_start != 0, par, ld, q, R, n, h_out,
        iters_out);
  else
    path_length_kernel<false><<<(unsigned)nblk, kBlock, 0, s>>>(
        img, geo.kB, geo.max_iter, geo.tol, geo.line_start != 0, par, ld, q, R, n, h_out,
        iters_out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FIT_OK : cuda_fail(e, "fit_path_lengths: launch");
}

}  // extern "C"
