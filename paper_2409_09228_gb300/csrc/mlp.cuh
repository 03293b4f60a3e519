// Learned path-length seed for the p2r iteration: a multilayer perceptron
// 8 -> 64 -> 64 -> 1 (ReLU) whose output corrects the straight-line seed of
// the iterative helix-cylinder step (paper Sec. 3.2, "propagation to r" by
// discrete steps).  BF16 weights and activations, FP32 accumulation, on the
// tensor cores through warp-level mma.sync m16n8k16.
//
// Inputs (the track's parameters in the frame whose x axis points along its
// transverse position, the charge and the target radius R):
//   f0 = r0 / R          r0 = sqrt(x^2 + y^2)
//   f1 = z / R
//   f2 = R / (2 rho)     = kA B w R / 2, rho the transverse radius of curvature
//   f3 = cos psi         psi = phi - atan2(y, x), the momentum azimuth
//   f4 = sin psi         in the local frame
//   f5 = cos theta
//   f6 = q
//   f7 = R / 100 cm
// Output g: the network's estimate of (h - h_line) / (kappa h_line^2 / 2),
// where h is the exact transverse path length to the cylinder and h_line the
// straight-line distance along the momentum; the seed is
// h0 = h_line + g kappa h_line^2 / 2, which is h_line at kappa = 0.
//
// Each input x is fed as two BF16 numbers, hi = bf16(x) and lo = bf16(x - hi),
// against the same weight row (K = 16 = 8 hi + 8 lo columns), so the first
// layer sees the FP32 input to ~2^-16 relative.
//
// Parameter vector (FP32 master copy, 4801 floats):
//   W1 [64][8] at 0, b1 [64] at 512, W2 [64][64] at 576, b2 [64] at 4672,
//   W3 [64] at 4736, b3 at 4800; W[out][in].
#pragma once

#include <cstdint>

#include "track_math.cuh"

namespace mlpk {

constexpr int kIn = 8, kHid = 64;
constexpr int kOffW1 = 0, kOffB1 = 512, kOffW2 = 576, kOffB2 = 4672, kOffW3 = 4736, kOffB3 = 4800;
constexpr int kParams = 4801;

// BF16 weights in mma fragment order (the word a lane loads is its own
// fragment register), FP32 biases.  Lane l = 4 g + c holds, for an n-tile of
// 8 output columns, B[k = 2c, 2c+1][n = g] (register b0) and B[k = 2c+8,
// 2c+9][n = g] (b1).
struct Image {
  uint4 w1[2][32];     // layer 1, .x .. .w = n-tiles 4j .. 4j+3 (b0 = b1: hi and lo share W1)
  uint4 w2[4][4][32];  // layer 2, [k-block][j][lane] = {b0, b1 of n-tile 2j, b0, b1 of 2j+1}
  uint4 w3[2][32];     // layer 3 (one column, n = 0), {b0, b1 of k-block 2j, b0, b1 of 2j+1}
  float b1[kHid], b2[kHid];
  float b3, pad[3];
};

// The training kernels also need W2 transposed (dA1 = dZ2 W2) and W3 as the
// BF16-rounded FP32 values the forward pass used.
struct TrainImage {
  Image fwd;
  uint4 w2t[4][4][32];  // B[k = out j][n = in i] = W2[j][i], same packing as w2
  float w3f[kHid];
};

static_assert(sizeof(Image) % 16 == 0, "image copied as uint4");
static_assert(sizeof(TrainImage) % 16 == 0, "image copied as uint4");

// ---- BF16 conversion (round to nearest even) and packing ------------------

// Packs (lo, hi) into one register; the lower half holds lo (the element with
// the smaller column index in an mma fragment).
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
// The same with ReLU applied first.
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ float bf16_lo(uint32_t r) { return __uint_as_float(r << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t r) { return __uint_as_float(r & 0xffff0000u); }
__device__ __forceinline__ float bf16_round(float x) { return bf16_lo(pack_bf16(x, 0.f)); }

// ---- tensor-core and shared-memory matrix primitives ----------------------

// D = A B + C, A 16x16 (row), B 16x8 (col), BF16 in, FP32 accumulate.
// Fragments: a0 (row g, k 2c..2c+1), a1 (row g+8), a2 (row g, k 2c+8..),
// a3 (row g+8, k 2c+8..); c0 c1 (row g, n 2c, 2c+1), c2 c3 (row g+8).
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1,
                                    const float (&c)[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%10,%11,%12,%13};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]),
        "f"(c[2]), "f"(c[3]));
}
__device__ __forceinline__ void mma_acc(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                        uint32_t b1) {
  mma(d, a, b0, b1, d);
}

// Four 8x8 BF16 matrices from shared memory; lanes 8i..8i+7 give the row
// addresses of matrix i, register i receives (row lane/4, cols 2(lane%4), +1)
// of matrix i, or with trans the element pair (rows 2(lane%4), +1; col lane/4).
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* row) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* row) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// ---- inputs -----------------------------------------------------------------

// The eight inputs of one track (definitions at the top of this file);
// (cphi, sphi) = (cos, sin) of the momentum azimuth, cth = cos theta,
// kB = kA B.  A track at r0 = 0 takes psi = 0.
__device__ __forceinline__ void features(const float (&p)[6], float cphi, float sphi, float cth,
                                         float qf, float kB, float R, float (&f)[kIn]) {
  const float x = p[0], y = p[1];
  const float r2 = fmaf(x, x, y * y);
  const bool at0 = !(r2 > 0.f);
  const float ir = at0 ? 0.f : rsqrtf(r2);
  const float iR = __fdividef(1.f, R);
  f[0] = r2 * ir * iR;
  f[1] = p[2] * iR;
  f[2] = 0.5f * kB * p[3] * R;
  f[3] = at0 ? 1.f : fmaf(x, cphi, y * sphi) * ir;
  f[4] = at0 ? 0.f : fmaf(x, sphi, -(y * cphi)) * ir;
  f[5] = cth;
  f[6] = qf;
  f[7] = 0.01f * R;
}

// Writes the hi and lo BF16 halves of a lane's inputs as two 16-byte rows.
__device__ __forceinline__ void stage_inputs(const float (&f)[kIn], uint4* hi_row, uint4* lo_row) {
  uint32_t hi[4], lo[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    hi[k] = pack_bf16(f[2 * k], f[2 * k + 1]);
    lo[k] = pack_bf16(f[2 * k] - bf16_lo(hi[k]), f[2 * k + 1] - bf16_hi(hi[k]));
  }
  *hi_row = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *lo_row = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

// ---- forward pass of one 16-row tile ----------------------------------------

// Layer-1 accumulators (rows of the tile x 64 hidden units) -> A fragments of
// the next layer (4 k-blocks of 16 hidden units), ReLU and BF16 on the way.
__device__ __forceinline__ void to_a_relu(const float (&z)[8][4], uint32_t (&a)[4][4]) {
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    a[kb][0] = pack_bf16_relu(z[2 * kb][0], z[2 * kb][1]);
    a[kb][1] = pack_bf16_relu(z[2 * kb][2], z[2 * kb][3]);
    a[kb][2] = pack_bf16_relu(z[2 * kb + 1][0], z[2 * kb + 1][1]);
    a[kb][3] = pack_bf16_relu(z[2 * kb + 1][2], z[2 * kb + 1][3]);
  }
}

__device__ __forceinline__ void layer1(const Image& W, const uint32_t (&a)[4], int lane,
                                       float (&z)[8][4]) {
  const int c = lane & 3;
  const uint4 w0 = W.w1[0][lane], w1 = W.w1[1][lane];
  const uint32_t wb[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) {
    const float2 b = *reinterpret_cast<const float2*>(&W.b1[nb * 8 + 2 * c]);
    const float cin[4] = {b.x, b.y, b.x, b.y};
    mma(z[nb], a, wb[nb], wb[nb], cin);
  }
}

__device__ __forceinline__ void layer2(const Image& W, const uint32_t (&a)[4][4], int lane,
                                       float (&z)[8][4]) {
  const int c = lane & 3;
#pragma unroll
  for (int nb = 0; nb < 8; ++nb) {
    const float2 b = *reinterpret_cast<const float2*>(&W.b2[nb * 8 + 2 * c]);
    z[nb][0] = b.x;
    z[nb][1] = b.y;
    z[nb][2] = b.x;
    z[nb][3] = b.y;
  }
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint4 w = W.w2[kb][j][lane];
      mma_acc(z[2 * j], a[kb], w.x, w.y);
      mma_acc(z[2 * j + 1], a[kb], w.z, w.w);
    }
  }
}

// Output column 0: o[0] for row g, o[2] for row g + 8 (lanes with c = 0).
__device__ __forceinline__ void layer3(const Image& W, const uint32_t (&a)[4][4], int lane,
                                       float (&o)[4]) {
  const uint4 w0 = W.w3[0][lane], w1 = W.w3[1][lane];
  const uint32_t wb[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
  o[0] = o[1] = o[2] = o[3] = W.b3;
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) mma_acc(o, a[kb], wb[2 * kb], wb[2 * kb + 1]);
}

// The network on the 32 lanes' inputs f (one sample per lane); every lane of
// the warp must call it (warp-collective).  stage: this warp's 64 rows of
// 16 bytes in shared memory (hi rows 0..31, lo rows 32..63).  Returns the
// lane's own output.
__device__ __forceinline__ float infer_warp(const Image& W, uint4* stage, const float (&f)[kIn]) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  stage_inputs(f, &stage[lane], &stage[32 + lane]);
  __syncwarp();
  float out = 0.f;
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    uint32_t a[4];
    // lanes 0..15: hi rows of the tile (k 0..7), lanes 16..31: lo rows (k 8..15)
    ldsm_x4(a, &stage[(lane >> 4) * 32 + mt * 16 + (lane & 15)]);
    float z[8][4];
    layer1(W, a, lane, z);
    uint32_t a2[4][4];
    to_a_relu(z, a2);
    layer2(W, a2, lane, z);
    to_a_relu(z, a2);
    float o[4];
    layer3(W, a2, lane, o);
    // row r of the tile is lane 16 mt + r; its value sits on lane 4 (r % 8)
    const float v0 = __shfl_sync(0xffffffffu, o[0], (lane & 7) * 4);
    const float v2 = __shfl_sync(0xffffffffu, o[2], (lane & 7) * 4);
    if ((lane >> 4) == mt) out = (lane & 8) ? v2 : v0;
  }
  __syncwarp();
  return out;
}

// Copies an image (a multiple of 16 bytes) with the whole block.
template <class Img>
__device__ __forceinline__ void copy_image(Img& dst, const Img* __restrict__ src) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Img) / 16); i += blockDim.x) d[i] = __ldg(s + i);
}

}  // namespace mlpk
