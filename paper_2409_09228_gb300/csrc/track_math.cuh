// Per-track FP32 arithmetic of the fused propagate + update kernel.
//
// Everything here acts on one track held in registers: the parameters
// p = (x, y, z, w, phi, theta) and the packed lower triangle c[21] of the 6x6
// covariance.  The paper (Sec. 3, Sec. 3.2) names the steps -- helix
// propagation to a plane or a cylinder with sin/cos and up-to-6x6 matrix
// products, then a Kalman update with a small matrix inverse and trigonometric
// functions -- but prints no formula; the ones used here are the textbook
// helix and Kalman filter:
//
//   kappa = -q kA B w (1/cm); with u = kappa h / 2 and s(u) = sin(u)/u,
//   x' = x + h s(u) cos(phi + u),  y' = y + h s(u) sin(phi + u),
//   z' = z + h cot(theta),  phi' = phi + kappa h.
//   p2z: h = (Z - z) tan(theta).
//   p2r: h from an iteration that advances by straight-line steps to the
//        cylinder along the current direction (paper Sec. 3.2, "advancing the
//        track state ... in discrete steps"), until a step is below tol * R.
//   J = J_h + (d p'/d h) (grad h)^T, C' = J C J^T (sparse, see masks below).
//   Update with the hit's 2-D position on the surface (x, y for p2z; the
//   azimuthal direction at the hit and z for p2r).
#pragma once

#include <cstdint>

#include "fit.h"

namespace fitk {

constexpr float kA = 0.00299792458f;  // GeV / (T cm)
constexpr float kPi = 3.14159265358979f;
constexpr float kTwoPi = 6.28318530717959f;

__host__ __device__ constexpr int sym(int i, int j) {
  return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i;
}

// s(u) = sin(u)/u, its derivative s'(u), and cos(u).  For |u| <= 1.25 the
// Taylor series in u^2 (truncated after u^12; remainder < 2e-10) avoid the
// cancellation of (u cos u - sin u)/u^2 at small u, where the straight-line
// limit kappa -> 0 must stay exact.
__device__ __forceinline__ void sinc_d(float u, float& s, float& sp, float& cu) {
  const float u2 = u * u;
  if (fabsf(u) <= 1.25f) {
    s = fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, 1.6059044e-10f, -2.5052108e-08f),
                                                  2.7557319e-06f), -1.9841270e-04f), 8.3333333e-03f),
                      -1.6666667e-01f), 1.0f);
    sp = u * fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, 1.9270853e-09f, -2.5052108e-07f),
                                             2.2045855e-05f), -1.1904762e-03f), 3.3333333e-02f),
                  -3.3333333e-01f);
    cu = fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, 2.0876757e-09f, -2.7557319e-07f),
                                                   2.4801587e-05f), -1.3888889e-03f), 4.1666667e-02f),
                       -0.5f), 1.0f);
  } else {
    float sn;
    sincosf(u, &sn, &cu);
    s = sn / u;
    sp = (cu - s) / u;
  }
}

// Sparsity of the transport Jacobian: bit (6 i + k) is set when J[i][k] can be
// non-zero.  Rows/columns: x, y, z, w, phi, theta.
__host__ __device__ constexpr unsigned long long bit(int i, int k) { return 1ull << (6 * i + k); }
// p2z: grad h = (0, 0, -tan, 0, 0, (Z - z)/cos^2); the z row vanishes.
constexpr unsigned long long kMaskZ =
    bit(0, 0) | bit(0, 2) | bit(0, 3) | bit(0, 4) | bit(0, 5) |
    bit(1, 1) | bit(1, 2) | bit(1, 3) | bit(1, 4) | bit(1, 5) |
    bit(3, 3) |
    bit(4, 2) | bit(4, 3) | bit(4, 4) | bit(4, 5) |
    bit(5, 5);
// p2r: grad h has x, y, w, phi components.
constexpr unsigned long long kMaskR =
    bit(0, 0) | bit(0, 1) | bit(0, 3) | bit(0, 4) |
    bit(1, 0) | bit(1, 1) | bit(1, 3) | bit(1, 4) |
    bit(2, 0) | bit(2, 1) | bit(2, 2) | bit(2, 3) | bit(2, 4) | bit(2, 5) |
    bit(3, 3) |
    bit(4, 0) | bit(4, 1) | bit(4, 3) | bit(4, 4) |
    bit(5, 5);

// c <- J c J^T on the packed lower triangle, touching only the entries that
// MASK marks.  With the loops unrolled the mask tests fold at compile time.
template <unsigned long long MASK>
__device__ __forceinline__ void similarity(const float (&J)[6][6], float (&c)[21]) {
  float JC[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (MASK & bit(i, k)) acc = fmaf(J[i][k], c[sym(k, j)], acc);
      JC[i][j] = acc;
    }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float acc = 0.f;
      if ((MASK & (63ull << (6 * i))) && (MASK & (63ull << (6 * j)))) {  // zero rows give 0
#pragma unroll
        for (int k = 0; k < 6; ++k)
          if (MASK & bit(j, k)) acc = fmaf(JC[i][k], J[j][k], acc);
      }
      c[sym(i, j)] = acc;
    }
}

// Propagation to the plane z = Z.  Returns FIT_ST_* bits (0 on success); on
// failure p and c are untouched.
__device__ __forceinline__ unsigned prop_z(float (&p)[6], float (&c)[21], float dkdw, float Z) {
  float sth, cth;
  sincosf(p[5], &sth, &cth);
  const float dz = Z - p[2];
  const float tanth = sth / cth;
  const float h = dz * tanth;
  if (!(h > 0.f)) return FIT_ST_NO_INTERSECTION;
  const float kappa = dkdw * p[3];
  const float u = 0.5f * kappa * h;
  float s, sp, cu;
  sinc_d(u, s, sp, cu);
  const float su = u * s;
  float sm, cm;
  sincosf(p[4] + u, &sm, &cm);
  const float hs = h * s;
  const float dx = hs * cm, dy = hs * sm;
  const float c1 = cm * cu - sm * su;  // cos(phi')
  const float s1 = sm * cu + cm * su;  // sin(phi')
  const float hh = 0.5f * h * h * dkdw;
  const float hth = dz / (cth * cth);  // dh/dtheta
  float J[6][6];
  J[0][0] = 1.f;
  J[0][2] = -c1 * tanth;
  J[0][3] = hh * (sp * cm - s * sm);
  J[0][4] = -dy;
  J[0][5] = c1 * hth;
  J[1][1] = 1.f;
  J[1][2] = -s1 * tanth;
  J[1][3] = hh * (sp * sm + s * cm);
  J[1][4] = dx;
  J[1][5] = s1 * hth;
  J[3][3] = 1.f;
  J[4][2] = -kappa * tanth;
  J[4][3] = h * dkdw;
  J[4][4] = 1.f;
  J[4][5] = kappa * hth;
  J[5][5] = 1.f;
  similarity<kMaskZ>(J, c);
  p[0] += dx;
  p[1] += dy;
  p[2] = Z;
  p[4] += 2.f * u;
  return 0u;
}

// Propagation to the cylinder r = R by straight-line steps along the current
// direction.  Returns FIT_ST_* bits; NO_INTERSECTION leaves p and c untouched.
__device__ __forceinline__ unsigned prop_r(float (&p)[6], float (&c)[21], float dkdw, float R,
                                           int max_iter, float tol_abs, unsigned& iters) {
  float sph, cph;
  sincosf(p[4], &sph, &cph);
  const float x = p[0], y = p[1];
  const float R2 = R * R;
  const float kappa = dkdw * p[3];
  // The transverse circle (centre c, radius rho = 1/|kappa|) reaches radius
  // R only if |c| + rho >= R, which always holds when rho >= R.
  {
    const float rho = 1.f / fabsf(kappa);
    if (rho < R) {
      const float irs = 1.f / kappa;  // signed radius
      const float cx = fmaf(-sph, irs, x), cy = fmaf(cph, irs, y);
      if (sqrtf(fmaf(cx, cx, cy * cy)) + rho < R) return FIT_ST_NO_INTERSECTION;
    }
  }
  // First step: along the initial direction to the circle.
  float h;
  {
    const float b = x * cph + y * sph;
    const float c0 = fmaf(x, x, fmaf(y, y, -R2));
    const float disc = fmaf(b, b, -c0);
    if (!(disc >= 0.f)) return FIT_ST_NO_INTERSECTION;
    const float sq = sqrtf(disc);
    if (c0 <= 0.f) {
      h = (b > 0.f) ? -c0 / (b + sq) : sq - b;  // forward root from inside
    } else {
      if (!(b < 0.f)) return FIT_ST_NO_INTERSECTION;  // outside, moving away
      h = c0 / (sq - b);                               // nearer forward root
    }
  }
  unsigned st = FIT_ST_NOT_CONVERGED;
  float s = 1.f, sp = 0.f, sm = sph, cm = cph, px = x, py = y, c1 = cph, s1 = sph, d = 0.f;
  for (int it = 0; it < max_iter; ++it) {
    ++iters;
    const float u = 0.5f * kappa * h;
    float cu;
    sinc_d(u, s, sp, cu);
    const float su = u * s;
    sincosf(p[4] + u, &sm, &cm);
    const float hs = h * s;
    px = fmaf(hs, cm, x);
    py = fmaf(hs, sm, y);
    c1 = cm * cu - sm * su;
    s1 = sm * cu + cm * su;
    // Step along (c1, s1) to the circle: d^2 + 2 b d + c2 = 0, smaller root.
    const float b = px * c1 + py * s1;
    const float c2 = fmaf(px, px, fmaf(py, py, -R2));
    const float disc = fmaf(b, b, -c2);
    d = (disc >= 0.f) ? -c2 / (b + copysignf(sqrtf(disc), b)) : -c2 / (2.f * b);
    h += d;
    if (fabsf(d) <= tol_abs) {
      st = 0u;
      break;
    }
  }
  // The loop evaluated the helix at h - d; move along the tangent by d
  // (the neglected curvature term, kappa d^2 / 2, is below FP32 resolution
  // once |d| <= tol).
  px = fmaf(d, c1, px);
  py = fmaf(d, s1, py);
  float sth, cth;
  sincosf(p[5], &sth, &cth);
  const float cot = cth / sth;
  const float dx = px - x, dy = py - y;
  const float hh = 0.5f * h * h * dkdw;
  const float Xw = hh * (sp * cm - s * sm);
  const float Yw = hh * (sp * sm + s * cm);
  // grad h = -grad g / (dg/dh) with g = x'^2 + y'^2 - R^2.
  const float iD = 1.f / (px * c1 + py * s1);
  const float hx = -px * iD, hy = -py * iD;
  const float hw = -(px * Xw + py * Yw) * iD;
  const float hp = (px * dy - py * dx) * iD;
  float J[6][6];
  J[0][0] = py * s1 * iD;  // = 1 + c1 hx
  J[0][1] = c1 * hy;
  J[0][3] = fmaf(c1, hw, Xw);
  J[0][4] = fmaf(c1, hp, -dy);
  J[1][0] = s1 * hx;
  J[1][1] = px * c1 * iD;  // = 1 + s1 hy
  J[1][3] = fmaf(s1, hw, Yw);
  J[1][4] = fmaf(s1, hp, dx);
  J[2][0] = cot * hx;
  J[2][1] = cot * hy;
  J[2][2] = 1.f;
  J[2][3] = cot * hw;
  J[2][4] = cot * hp;
  J[2][5] = -h / (sth * sth);
  J[3][3] = 1.f;
  J[4][0] = kappa * hx;
  J[4][1] = kappa * hy;
  J[4][3] = fmaf(kappa, hw, h * dkdw);
  J[4][4] = fmaf(kappa, hp, 1.f);
  J[5][5] = 1.f;
  similarity<kMaskR>(J, c);
  p[0] = px;
  p[1] = py;
  p[2] = fmaf(h, cot, p[2]);
  p[4] = fmaf(kappa, h, p[4]);
  return st;
}

// Kalman update with a 2-D measurement: a and b are the columns of C H^T (the
// two measured directions), S = H C H^T + H V H^T, K = C H^T S^-1,
// p += K r, C -= K (H C), chi2 = r^T S^-1 r.
//
// FP32 note: a and b are strongly correlated and so is S, so K = [a b] S^-1
// cancels.  K is formed as [a S11 - b S01, b S00 - a S01] / det with the
// rounding error of each second product recovered by an FMA (and det by
// Kahan's 2x2 determinant); forming S^-1 first and multiplying loses up to
// ~1e-4 relative accuracy in the 1/pT variance after 20 layers.
__device__ __forceinline__ float kalman_2d(float (&p)[6], float (&c)[21], const float (&a)[6],
                                           const float (&b)[6], float S00, float S01, float S11,
                                           float r0, float r1) {
  const float w01 = S01 * S01;
  const float det = fmaf(S00, S11, -w01) - fmaf(S01, S01, -w01);
  const float id = 1.f / det;
  float k0[6], k1[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float t0 = b[i] * S01, t1 = a[i] * S01;
    k0[i] = (fmaf(a[i], S11, -t0) - fmaf(b[i], S01, -t0)) * id;
    k1[i] = (fmaf(b[i], S00, -t1) - fmaf(a[i], S01, -t1)) * id;
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] = fmaf(k0[i], r0, fmaf(k1[i], r1, p[i]));
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) c[sym(i, j)] -= fmaf(k0[i], a[j], k1[i] * b[j]);
  // chi2 = (S11 r0^2 - 2 S01 r0 r1 + S00 r1^2) / det
  return fmaf(S11 * r0, r0, fmaf(S00 * r1, r1, -2.f * S01 * r0 * r1)) * id;
}

// After an update: phi into (-pi, pi]; a negative w flips the charge.
__device__ __forceinline__ unsigned normalise(float (&p)[6], float (&c)[21], int& q) {
  const float k = floorf((kPi - p[4]) * (1.f / kTwoPi));
  p[4] = fmaf(k, kTwoPi, p[4]);
  if (p[3] < 0.f) {
    p[3] = -p[3];
    q = -q;
#pragma unroll
    for (int i = 0; i < 6; ++i)
      if (i != 3) c[sym(3, i)] = -c[sym(3, i)];
    return FIT_ST_CHARGE_FLIP;
  }
  return 0u;
}

// p2z update: H measures x and y.
__device__ __forceinline__ float update_z(float (&p)[6], float (&c)[21], const float (&m)[3],
                                          const float (&v)[6]) {
  float a[6], b[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    a[i] = c[sym(i, 0)];
    b[i] = c[sym(i, 1)];
  }
  return kalman_2d(p, c, a, b, a[0] + v[0], b[0] + v[1], b[1] + v[2], m[0] - p[0], m[1] - p[1]);
}

// p2r update: H measures the position along the cylinder's azimuthal
// direction t = (-sin phi_h, cos phi_h, 0) at the hit azimuth, and z.
__device__ __forceinline__ float update_r(float (&p)[6], float (&c)[21], const float (&m)[3],
                                          const float (&v)[6]) {
  const float ir = rsqrtf(fmaf(m[0], m[0], m[1] * m[1]));
  const float sh = m[1] * ir, ch = m[0] * ir;
  float a[6], b[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    a[i] = fmaf(ch, c[sym(i, 1)], -sh * c[sym(i, 0)]);
    b[i] = c[sym(i, 2)];
  }
  const float vtt = fmaf(sh * sh, v[0], fmaf(ch * ch, v[2], -2.f * sh * ch * v[1]));
  const float vtz = fmaf(ch, v[4], -sh * v[3]);
  const float S00 = fmaf(ch, a[1], -sh * a[0]) + vtt;
  const float S01 = a[2] + vtz;
  const float S11 = b[2] + v[5];
  const float r0 = fmaf(ch, m[1] - p[1], -sh * (m[0] - p[0]));
  const float r1 = m[2] - p[2];
  return kalman_2d(p, c, a, b, S00, S01, S11, r0, r1);
}

}  // namespace fitk
