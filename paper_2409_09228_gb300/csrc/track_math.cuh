// Per-track FP32 arithmetic of the fused propagate + update kernel.
//
// Everything here acts on tracks held in registers: the parameters
// p = (x, y, z, w, phi, theta) and the packed lower triangle c[21] of the 6x6
// covariance.  Each function is a template over the lane type T (lanes.cuh):
// float for one track, F2 for two tracks whose FP32 work shares packed
// instructions.  The paper (Sec. 3, Sec. 3.2) names the steps -- helix
// propagation to a plane or a cylinder with sin/cos and up-to-6x6 matrix
// products, then a Kalman update with a small matrix inverse and
// trigonometric functions -- but prints no formula; the ones used here are the
// textbook helix and Kalman filter:
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
//
// The cosine and sine of phi and theta travel with the track (struct Trig):
// a propagation turns phi by kappa h, an update changes phi and theta by the
// gain times the residual, and both are applied as rotations of the carried
// (cos, sin) pairs, so a layer needs no trigonometric function call.
#pragma once

#include <cstdint>

#include "fit.h"
#include "lanes.cuh"

namespace fitk {

constexpr float kA = 0.00299792458f;  // GeV / (T cm)
constexpr float kPi = 3.14159265358979f;
constexpr float kTwoPi = 6.28318530717959f;

// pi, 2 pi and 1/(2 pi) in the lane type's precision.
template <class T>
__device__ __forceinline__ T pi_() { return T(kPi); }
template <>
__device__ __forceinline__ double pi_<double>() { return 3.141592653589793; }
template <class T>
__device__ __forceinline__ T two_pi_() { return T(kTwoPi); }
template <>
__device__ __forceinline__ double two_pi_<double>() { return 6.283185307179586; }
template <class T>
__device__ __forceinline__ T inv_two_pi_() { return T(1.f / kTwoPi); }
template <>
__device__ __forceinline__ double inv_two_pi_<double>() { return 0.15915494309189535; }

__host__ __device__ constexpr int sym(int i, int j) {
  return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i;
}

// sin and cos of x for |x| < 2^12 (the propagator's angles stay within a few
// pi).  Cody & Waite's reduction x = j pi/2 + r with pi/2 split into the
// nearest float and its remainder (W. J. Cody, W. Waite, "Software Manual for
// the Elementary Functions", 1980), then the Taylor series of sin and cos on
// |r| <= pi/4 truncated after r^9 and r^10 (remainders < 2e-9), and the
// quadrant j mod 4 applied by swapping and sign flips.
__device__ __forceinline__ void sincos_cw(float x, float& s, float& c) {
  const float j = rintf(x * 0.636619772f);
  float r = fmaf(j, -1.57079637f, x);  // float(pi/2)
  r = fmaf(j, 4.37113883e-08f, r);     // pi/2 - float(pi/2) = -4.37113883e-08
  const float r2 = r * r;
  const float sr = fmaf(r * r2, fmaf(r2, fmaf(r2, fmaf(r2, 2.75573192e-06f, -1.98412698e-04f),
                                            8.33333333e-03f), -1.66666667e-01f), r);
  const float cr = fmaf(r2, fmaf(r2, fmaf(r2, fmaf(r2, fmaf(r2, -2.75573192e-07f, 2.48015873e-05f),
                                                  -1.38888889e-03f), 4.16666667e-02f), -0.5f), 1.0f);
  const int q = __float2int_rn(j);
  const float sv = (q & 1) ? cr : sr;
  const float cv = (q & 1) ? sr : cr;
  s = __int_as_float(__float_as_int(sv) ^ ((q & 2) << 30));
  c = __int_as_float(__float_as_int(cv) ^ (((q + 1) & 2) << 30));
}
__device__ __forceinline__ void sincos_cw(F2 x, F2& s, F2& c) {
  sincos_cw(x.v.x, s.v.x, c.v.x);
  sincos_cw(x.v.y, s.v.y, c.v.y);
}

// s(u) = sin(u)/u and cos(u) by their Taylor series in u^2: up to u^4 for
// |u| <= 0.1 (remainders < 2e-9; steps between neighbouring layers stay in
// this range), up to u^12 for |u| <= 1.25 (remainders < 2e-10), beyond that
// from sin and cos.  The series keep the straight-line limit kappa -> 0 exact.
template <class T>
__device__ __forceinline__ void sinc_series(T u2, T& s, T& cu, bool shortform) {
  if (shortform) {
    s = fma(u2, fma(u2, T(8.3333333e-03f), T(-1.6666667e-01f)), T(1.0f));
    cu = fma(u2, fma(u2, T(4.1666667e-02f), T(-0.5f)), T(1.0f));
  } else {
    s = fma(u2, fma(u2, fma(u2, fma(u2, fma(u2, fma(u2, T(1.6059044e-10f), T(-2.5052108e-08f)),
                                              T(2.7557319e-06f)), T(-1.9841270e-04f)),
                             T(8.3333333e-03f)), T(-1.6666667e-01f)), T(1.0f));
    cu = fma(u2, fma(u2, fma(u2, fma(u2, fma(u2, fma(u2, T(2.0876757e-09f), T(-2.7557319e-07f)),
                                               T(2.4801587e-05f)), T(-1.3888889e-03f)),
                              T(4.1666667e-02f)), T(-0.5f)), T(1.0f));
  }
}

__device__ __forceinline__ void sinc_c(float u, float& s, float& cu) {
  const float au = fabsf(u);
  if (au <= 1.25f) {
    sinc_series(u * u, s, cu, au <= 0.1f);
  } else {
    float sn;
    sincos_cw(u, sn, cu);
    s = fdiv(sn, u);
  }
}
__device__ __forceinline__ void sinc_c(F2 u, F2& s, F2& cu) {
  const F2 au = fabs_(u);
  if (all(le(au, F2(1.25f)))) {
    sinc_series(u * u, s, cu, all(le(au, F2(0.1f))));
  } else {
    sinc_c(u.v.x, s.v.x, cu.v.x);
    sinc_c(u.v.y, s.v.y, cu.v.y);
  }
}

// s'(u), the derivative of sin(u)/u, given s(u) and cos(u); series as above
// where (u cos u - sin u)/u^2 would cancel.
template <class T>
__device__ __forceinline__ T sinc_deriv_series(T u, bool shortform) {
  const T u2 = u * u;
  if (shortform) return u * fma(u2, fma(u2, T(-1.1904762e-03f), T(3.3333333e-02f)), T(-3.3333333e-01f));
  return u * fma(u2, fma(u2, fma(u2, fma(u2, fma(u2, T(1.9270853e-09f), T(-2.5052108e-07f)),
                                         T(2.2045855e-05f)), T(-1.1904762e-03f)),
                          T(3.3333333e-02f)), T(-3.3333333e-01f));
}
__device__ __forceinline__ float sinc_deriv(float u, float s, float cu) {
  const float au = fabsf(u);
  if (au <= 1.25f) return sinc_deriv_series(u, au <= 0.1f);
  return fdiv(cu - s, u);
}
__device__ __forceinline__ F2 sinc_deriv(F2 u, F2 s, F2 cu) {
  const F2 au = fabs_(u);
  if (all(le(au, F2(1.25f)))) return sinc_deriv_series(u, all(le(au, F2(0.1f))));
  return F2(sinc_deriv(u.v.x, s.v.x, cu.v.x), sinc_deriv(u.v.y, s.v.y, cu.v.y));
}

// sin(u)/u, cos(u) and the derivative of sin(u)/u with one range test.
__device__ __forceinline__ void sinc_cs(float u, float& s, float& cu, float& sp) {
  const float au = fabsf(u);
  if (au <= 1.25f) {
    const bool shortform = au <= 0.1f;
    sinc_series(u * u, s, cu, shortform);
    sp = sinc_deriv_series(u, shortform);
  } else {
    float sn;
    sincos_cw(u, sn, cu);
    s = fdiv(sn, u);
    sp = fdiv(cu - s, u);
  }
}
__device__ __forceinline__ void sinc_cs(F2 u, F2& s, F2& cu, F2& sp) {
  const F2 au = fabs_(u);
  if (all(le(au, F2(0.1f)))) {  // the common case first: one test
    sinc_series(u * u, s, cu, true);
    sp = sinc_deriv_series(u, true);
  } else if (all(le(au, F2(1.25f)))) {
    sinc_series(u * u, s, cu, false);
    sp = sinc_deriv_series(u, false);
  } else {
    sinc_cs(u.v.x, s.v.x, cu.v.x, sp.v.x);
    sinc_cs(u.v.y, s.v.y, cu.v.y, sp.v.y);
  }
}

// (c, s) <- (cos(a + d), sin(a + d)) from (c, s) = (cos a, sin a), given
// (cd, sd) = (cos d, sin d).
template <class T>
__device__ __forceinline__ void turn(T& c, T& s, T cd, T sd) {
  const T cn = fma(c, cd, -(s * sd));
  s = fma(s, cd, c * sd);
  c = cn;
}

// As turn(), for an angle d given by value: the change of an angle in one
// update is small, so the Taylor series of sin d and cos d (to d^5 and d^4,
// remainders < 2e-9 for |d| <= 0.1) replace a trigonometric call.
// turn_small: the series alone, for a caller that knows |d| <= 0.1.
template <class T>
__device__ __forceinline__ void turn_small(T& c, T& s, T d) {
  const T d2 = d * d;
  turn(c, s, fma(d2, fma(d2, T(4.1666667e-02f), T(-0.5f)), T(1.0f)),
       d * fma(d2, fma(d2, T(8.3333333e-03f), T(-1.6666667e-01f)), T(1.0f)));
}
template <class T>
__device__ __forceinline__ void turn_by(T& c, T& s, T d) {
  if (all(le(fabs_(d), T(0.1f)))) {
    turn_small(c, s, d);
  } else {
    T sd, cd;
    sincos_cw(d, sd, cd);
    turn(c, s, cd, sd);
  }
}

// FP64 variant: sin and cos from the CUDA math library; sin(u)/u and its
// derivative by their Taylor series (to u^8 and u^7, remainders below 1e-19
// relative for |u| < 1e-2) only where sin(u)/u and (cos u - sin(u)/u)/u
// would cancel.
__device__ __forceinline__ void sincos_cw(double x, double& s, double& c) { ::sincos(x, &s, &c); }
__device__ __forceinline__ void sinc_c(double u, double& s, double& cu) {
  double sn;
  ::sincos(u, &sn, &cu);
  if (::fabs(u) < 1e-2) {
    const double u2 = u * u;
    s = fma(u2, fma(u2, fma(u2, fma(u2, 1.0 / 362880.0, -1.0 / 5040.0), 1.0 / 120.0), -1.0 / 6.0),
            1.0);
  } else {
    s = sn / u;
  }
}
__device__ __forceinline__ double sinc_deriv(double u, double s, double cu) {
  if (::fabs(u) < 1e-2) {
    const double u2 = u * u;
    return u * fma(u2, fma(u2, fma(u2, 1.0 / 45360.0, -1.0 / 840.0), 1.0 / 30.0), -1.0 / 3.0);
  }
  return (cu - s) / u;
}
__device__ __forceinline__ void turn_by(double& c, double& s, double d) {
  double sd, cd;
  ::sincos(d, &sd, &cd);
  turn(c, s, cd, sd);
}
__device__ __forceinline__ void turn_small(double& c, double& s, double d) { turn_by(c, s, d); }
__device__ __forceinline__ void sinc_cs(double u, double& s, double& cu, double& sp) {
  sinc_c(u, s, cu);
  sp = sinc_deriv(u, s, cu);
}

// Two turns by small angles (as turn_by) with one range test.
template <class T>
__device__ __forceinline__ void turn_by2(T& c1, T& s1, T d1, T& c2, T& s2, T d2) {
  if (all(le(fmax_(fabs_(d1), fabs_(d2)), T(0.1f)))) {
    turn_small(c1, s1, d1);
    turn_small(c2, s2, d2);
  } else {
    turn_by(c1, s1, d1);
    turn_by(c2, s2, d2);
  }
}
__device__ __forceinline__ void turn_by2(double& c1, double& s1, double d1, double& c2, double& s2,
                                         double d2) {
  turn_by(c1, s1, d1);
  turn_by(c2, s2, d2);
}

// Nothing to overlap (the default of the propagations' ov argument).
struct NoOverlap {
  __device__ __forceinline__ void operator()() const {}
};

// Cosine and sine of phi and theta, carried with the track.
template <class T>
struct Trig {
  T cphi, sphi, cth, sth;
};

template <class T>
__device__ __forceinline__ Trig<T> trig_of(const T (&p)[6]) {
  Trig<T> t;
  sincos_cw(p[4], t.sphi, t.cphi);
  sincos_cw(p[5], t.sth, t.cth);
  return t;
}

// Transport Jacobian J = diag(unit rows) + E.  ROWS is the set of rows of J
// whose diagonal entry is 1 + E_ii (bit i); the other rows vanish.  EMASK
// marks the entries of E that can be non-zero (bit 6 i + k).  Rows and
// columns: x, y, z, w, phi, theta.
__host__ __device__ constexpr unsigned long long bit(int i, int k) { return 1ull << (6 * i + k); }
__host__ __device__ constexpr unsigned row(int i) { return 1u << i; }
// p2z: grad h = (0, 0, -tan, 0, 0, (Z - z)/cos^2); z' = Z, so the z row is 0.
constexpr unsigned kRowsZ = row(0) | row(1) | row(3) | row(4) | row(5);
constexpr unsigned long long kEZ =
    bit(0, 2) | bit(0, 3) | bit(0, 4) | bit(0, 5) |
    bit(1, 2) | bit(1, 3) | bit(1, 4) | bit(1, 5) |
    bit(4, 2) | bit(4, 3) | bit(4, 5);
// p2r: grad h has x, y, w, phi components.
constexpr unsigned kRowsR = row(0) | row(1) | row(2) | row(3) | row(4) | row(5);
constexpr unsigned long long kER =
    bit(0, 0) | bit(0, 1) | bit(0, 3) | bit(0, 4) |
    bit(1, 0) | bit(1, 1) | bit(1, 3) | bit(1, 4) |
    bit(2, 0) | bit(2, 1) | bit(2, 3) | bit(2, 4) | bit(2, 5) |
    bit(4, 0) | bit(4, 1) | bit(4, 3) | bit(4, 4);

// c <- J c J^T through the structure of the propagate-to-surface Jacobian,
// J = A + v g^T: A = I + E_h is the derivative of the helix at a fixed path
// length h, v = d p' / d h, and g = grad h, the dependence of h on the
// input state (the surface constraint).  With m = c g and s = g^T m,
//   J c J^T = A c A^T + n v^T + v n^T,   n = A m + (s / 2) v,
// so the dense product is replaced by a sparse similarity with A and a
// symmetric rank-2 update.  A's off-diagonal entries are those of E_h:
// row x: f03 (d x'/d w), f04 (d x'/d phi); row y: f13, f14; row z: f25
// (d z'/d theta, p2r only); row phi: g43 (d phi'/d w).  A factors as
// (I + G)(I + F), F holding rows x, y, z (which read only rows w, phi, theta,
// unchanged by F) and G the phi row, so both steps run in place.  VZ = false
// (p2z): the z row of J vanishes (z' = Z on the plane), so row and column z
// of the result are zero and v, g carry no z component in the result; GMASK
// and VMASK mark the components of g and v that can be non-zero.
template <bool P2R, unsigned GMASK, unsigned VMASK, class T>
__device__ __forceinline__ void similarity_rank1(T (&c)[21], T f03, T f04, T f13, T f14, T f25,
                                                 T g43, const T (&gr)[6], const T (&v)[6]) {
  // m = c g (with the input covariance), s = g^T m
  T m[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    T acc = T(0.f);
    bool first = true;
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (GMASK & (1u << k)) {
        acc = first ? c[sym(i, k)] * gr[k] : fma(c[sym(i, k)], gr[k], acc);
        first = false;
      }
    m[i] = acc;
  }
  T sg = T(0.f);
  {
    bool first = true;
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (GMASK & (1u << k)) {
        sg = first ? gr[k] * m[k] : fma(gr[k], m[k], sg);
        first = false;
      }
  }
  // F step: rows x, y (and z) from rows w, phi, theta.  Row i of F c F^T
  // (j <= i) needs the input cross block of rows j <= i and row i's new
  // cross block X_il = c_il + sum_k F_ik c_kl, so the rows run from the last
  // to the first and each overwrites its own cross block when it is done.
  constexpr int NF = P2R ? 3 : 2;
  const T F[3][3] = {{f03, f04, T(0.f)}, {f13, f14, T(0.f)}, {T(0.f), T(0.f), f25}};
  auto Fik = [&](int i, int k) -> T { return F[i][k - 3]; };
  auto Fnz = [](int i, int k) -> bool { return (i < 2 && k < 5) || (i == 2 && k == 5); };
#pragma unroll
  for (int i = NF - 1; i >= 0; --i) {
    T X[3];
#pragma unroll
    for (int l = 3; l < 6; ++l) {
      T acc = c[sym(i, l)];
#pragma unroll
      for (int k = 3; k < 6; ++k)
        if (Fnz(i, k)) acc = fma(Fik(i, k), c[sym(k, l)], acc);
      X[l - 3] = acc;
    }
    // c_ij <- c_ij + sum_k F_ik c_kj + sum_l X_il F_jl
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T acc = c[sym(i, j)];
#pragma unroll
      for (int k = 3; k < 6; ++k)
        if (Fnz(i, k)) acc = fma(Fik(i, k), c[sym(k, j)], acc);
#pragma unroll
      for (int l = 3; l < 6; ++l)
        if (Fnz(j, l)) acc = fma(X[l - 3], Fik(j, l), acc);
      c[sym(i, j)] = acc;
    }
#pragma unroll
    for (int l = 3; l < 6; ++l) c[sym(i, l)] = X[l - 3];
  }
  if constexpr (!P2R) {
#pragma unroll
    for (int j = 0; j < 6; ++j) c[sym(2, j)] = T(0.f);
  }
  // G step: row phi += g43 row w (and column phi likewise)
  {
    const T c43 = c[sym(4, 3)];
#pragma unroll
    for (int j = 0; j < 6; ++j)
      if (j != 3 && j != 4 && (P2R || j != 2)) c[sym(4, j)] = fma(g43, c[sym(3, j)], c[sym(4, j)]);
    const T c43n = fma(g43, c[sym(3, 3)], c43);
    c[sym(4, 3)] = c43n;
    c[sym(4, 4)] = fma(g43, c43 + c43n, c[sym(4, 4)]);
  }
  // n = A m + (s / 2) v, A = (I + G)(I + F)
  T n[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) n[i] = m[i];
#pragma unroll
  for (int i = 0; i < NF; ++i)
#pragma unroll
    for (int k = 3; k < 6; ++k)
      if (Fnz(i, k)) n[i] = fma(Fik(i, k), m[k], n[i]);
  if constexpr (!P2R) n[2] = T(0.f);
  n[4] = fma(g43, n[3], n[4]);
  const T hs = T(0.5f) * sg;
#pragma unroll
  for (int i = 0; i < 6; ++i)
    if (VMASK & (1u << i)) n[i] = fma(hs, v[i], n[i]);
  // c += n v^T + v n^T
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      if (!P2R && (i == 2 || j == 2)) continue;
      T acc = c[sym(i, j)];
      if (VMASK & (1u << j)) acc = fma(n[i], v[j], acc);
      if (VMASK & (1u << i)) acc = fma(v[i], n[j], acc);
      c[sym(i, j)] = acc;
    }
}

// p2r covariance in the cylinder's local coordinates.  A propagated
// covariance C' = J C J^T has the surface normal as a null vector: the
// constraint x'^2 + y'^2 = R^2 gives x' J_x + y' J_y = 0 for the position
// rows of J, and the Kalman update C - C H^T S^-1 H C keeps every null vector
// of C.  So from the first cylinder on, C = B c B^T exactly, with c the 5x5
// covariance of (l, z, w, phi, theta), l the position along the direction
// (-bs, bc) normal to the null vector (bc, bs), and B the 6x5 basis
// (-bs, bc) e_l + e_z ... e_theta.  The transport to the next cylinder is
// then c' = J_l c J_l^T with the 5x5 J_l = P' J B (P' = B'^T, the projection
// at the new point, whose null vector is its azimuth), and the update acts on
// c with the projected measurement: the same results as the 6x6 form in
// exact arithmetic, on 15 entries instead of 21.  to_local_r / to_global_r
// move between the two forms.
template <class T>
__device__ __forceinline__ void to_local_r(const T (&c)[21], T bc, T bs, T (&cl)[15]) {
  // l = -bs x + bc y
  cl[sym(0, 0)] = fma(bs * bs, c[sym(0, 0)],
                      fma(bc * bc, c[sym(1, 1)], T(-2.f) * (bs * bc) * c[sym(1, 0)]));
#pragma unroll
  for (int i = 1; i < 5; ++i) {
    cl[sym(i, 0)] = fma(bc, c[sym(i + 1, 1)], -(bs * c[sym(i + 1, 0)]));
#pragma unroll
    for (int j = 1; j <= i; ++j) cl[sym(i, j)] = c[sym(i + 1, j + 1)];
  }
}
template <class T>
__device__ __forceinline__ void to_global_r(const T (&cl)[15], T bc, T bs, T (&c)[21]) {
  const T l0 = cl[sym(0, 0)];
  c[sym(0, 0)] = (bs * bs) * l0;
  c[sym(1, 0)] = -(bs * bc) * l0;
  c[sym(1, 1)] = (bc * bc) * l0;
#pragma unroll
  for (int i = 1; i < 5; ++i) {
    c[sym(i + 1, 0)] = -(bs * cl[sym(i, 0)]);
    c[sym(i + 1, 1)] = bc * cl[sym(i, 0)];
#pragma unroll
    for (int j = 1; j <= i; ++j) c[sym(i + 1, j + 1)] = cl[sym(i, j)];
  }
}

// The start covariance in the loop form, for any start point.  The first
// propagation's J C J^T is unchanged if C is first carried to a surface
// through the start point itself: the map to the first surface passes that
// surface at path length 0, so by the chain rule J = J J_0 with J_0 the
// Jacobian of the zero-length propagation there, J_0 = I + v g^T
// (v = d p / d h = (cos phi, sin phi, cot theta, 0, kappa, 0), g = grad h).
// With y = C g and sigma = g^T y, J_0 C J_0^T = C + n v^T + v n^T,
// n = y + (sigma / 2) v.
//
// p2z: the plane z = z0, g = -tan(theta) e_z; the z row of J_0 vanishes
// (1 - cot tan = 0), which leaves the zero z row prop_z<true> needs.
template <class T>
__device__ __forceinline__ void enter_plane(T (&c)[21], const Trig<T>& g, T kappa) {
  const T tn = fdiv(g.sth, g.cth);
  const T sig = (tn * tn) * c[sym(2, 2)];
  const T v[6] = {g.cphi, g.sphi, T(0.f), T(0.f), kappa, T(0.f)};
  constexpr unsigned VM = (1u << 0) | (1u << 1) | (1u << 4);
  T n[6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
    n[i] = (VM & (1u << i)) ? fma(T(0.5f) * sig, v[i], -(tn * c[sym(i, 2)])) : -(tn * c[sym(i, 2)]);
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      if (i == 2 || j == 2) {
        c[sym(i, j)] = T(0.f);
        continue;
      }
      T acc = c[sym(i, j)];
      if (VM & (1u << j)) acc = fma(n[i], v[j], acc);
      if (VM & (1u << i)) acc = fma(v[i], n[j], acc);
      c[sym(i, j)] = acc;
    }
}

// p2r: the line through the start point across the transverse direction,
// (x - x0) cos phi + (y - y0) sin phi = 0, where g = -(cos phi, sin phi, 0,
// 0, 0, 0) (well conditioned for any start, unlike the cylinder through it).
// Its normal (cos phi, sin phi) is the null vector of the result, whose local
// form (to_local_r) is returned with (bc, bs) = (cos phi, sin phi):
// cl = B^T C B + n_l v_l^T + v_l n_l^T with v_l = B^T v = (0, cot, 0, kappa,
// 0) and n_l = B^T y + (sigma / 2) v_l.
template <class T>
__device__ __forceinline__ void enter_line(const T (&c)[21], const Trig<T>& g, T kappa,
                                           T (&cl)[15]) {
  const T bc = g.cphi, bs = g.sphi;
  const T cot = fdiv(g.cth, g.sth);
  T y[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] = -fma(bc, c[sym(i, 0)], bs * c[sym(i, 1)]);
  const T sig = -fma(bc, y[0], bs * y[1]);
  to_local_r(c, bc, bs, cl);
  const T hs = T(0.5f) * sig;
  const T n[5] = {fma(bc, y[1], -(bs * y[0])), fma(hs, cot, y[2]), y[3], fma(hs, kappa, y[4]),
                  y[5]};
  const T v[5] = {T(0.f), cot, T(0.f), kappa, T(0.f)};
  constexpr unsigned VM = (1u << 1) | (1u << 3);
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T acc = cl[sym(i, j)];
      if (VM & (1u << j)) acc = fma(n[i], v[j], acc);
      if (VM & (1u << i)) acc = fma(v[i], n[j], acc);
      cl[sym(i, j)] = acc;
    }
}

// c <- J_l c J_l^T in local coordinates.  With J = A + v g^T as for
// similarity_rank1, J_l = A_l + v_l g_l^T where g_l = B^T g = (gl0, 0, hw,
// hp, 0), v_l = P' v = (vl0, cot, 0, kappa, 0) and A_l = P' A B differs from
// the identity in the entries (l, l) = ctt (the cosine of the angle between
// the two l directions), (l, w) = a02, (l, phi) = a03, (z, theta) = f25 and
// (phi, w) = g43.  A_l = (I + G)(D + F) with D = diag(ctt, 1, ...), F the l
// and z rows (reading only rows w, phi, theta) and G the phi row, so both
// factors apply in place; then the rank-2 update as in similarity_rank1.
template <class T>
__device__ __forceinline__ void similarity_local_r(T (&c)[15], T ctt, T a02, T a03, T f25, T g43,
                                                   T gl0, T hw, T hp, T vl0, T cot, T kappa) {
  // m = c g_l, s = g_l^T m
  T m[5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
    m[i] = fma(c[sym(i, 3)], hp, fma(c[sym(i, 2)], hw, c[sym(i, 0)] * gl0));
  const T sg = fma(hp, m[3], fma(hw, m[2], gl0 * m[0]));
  // D + F.  Row z: R1 = e_z + f25 e_theta; row l: R0 = ctt e_l + a02 e_w + a03 e_phi.
  // X_il = (R_i c)_l for l in w, phi, theta are the new cross blocks.
  T X1[3], X0[3];
#pragma unroll
  for (int l = 2; l < 5; ++l) X1[l - 2] = fma(f25, c[sym(4, l)], c[sym(1, l)]);
  const T c11 = fma(f25, X1[2], fma(f25, c[sym(4, 1)], c[sym(1, 1)]));
  const T c10 = fma(a03, X1[1], fma(a02, X1[0], ctt * fma(f25, c[sym(4, 0)], c[sym(1, 0)])));
  const T y0 = fma(a03, c[sym(3, 0)], fma(a02, c[sym(2, 0)], ctt * c[sym(0, 0)]));
#pragma unroll
  for (int l = 2; l < 5; ++l)
    X0[l - 2] = fma(a03, c[sym(3, l)], fma(a02, c[sym(2, l)], ctt * c[sym(0, l)]));
  c[sym(0, 0)] = fma(a03, X0[1], fma(a02, X0[0], ctt * y0));
  c[sym(1, 0)] = c10;
  c[sym(1, 1)] = c11;
#pragma unroll
  for (int l = 2; l < 5; ++l) {
    c[sym(1, l)] = X1[l - 2];
    c[sym(0, l)] = X0[l - 2];
  }
  // G: row phi += g43 row w (and column phi likewise)
  {
    const T c32 = c[sym(3, 2)];
    c[sym(3, 0)] = fma(g43, c[sym(2, 0)], c[sym(3, 0)]);
    c[sym(3, 1)] = fma(g43, c[sym(2, 1)], c[sym(3, 1)]);
    c[sym(4, 3)] = fma(g43, c[sym(4, 2)], c[sym(4, 3)]);
    const T c32n = fma(g43, c[sym(2, 2)], c32);
    c[sym(3, 2)] = c32n;
    c[sym(3, 3)] = fma(g43, c32 + c32n, c[sym(3, 3)]);
  }
  // n = A_l m + (s / 2) v_l;  c += n v_l^T + v_l n^T
  const T hs = T(0.5f) * sg;
  const T n[5] = {fma(hs, vl0, fma(a03, m[3], fma(a02, m[2], ctt * m[0]))),
                  fma(hs, cot, fma(f25, m[4], m[1])), m[2], fma(hs, kappa, fma(g43, m[2], m[3])),
                  m[4]};
  const T v[5] = {vl0, cot, T(0.f), kappa, T(0.f)};
  constexpr unsigned VM = (1u << 0) | (1u << 1) | (1u << 3);
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T acc = c[sym(i, j)];
      if (VM & (1u << j)) acc = fma(n[i], v[j], acc);
      if (VM & (1u << i)) acc = fma(v[i], n[j], acc);
      c[sym(i, j)] = acc;
    }
}

// Propagation to the plane z = Z.  Returns the mask of lanes whose plane is
// behind them; if any lane fails nothing is modified.  ZFREE: the caller
// guarantees that row and column z of c are zero (true from the first plane
// on: z' = Z makes the z row of J vanish, and an update keeps a zero row
// zero), so the z component of grad h meets only zeros and is skipped.
template <bool ZFREE = false, class T, class Overlap = NoOverlap>
__device__ __forceinline__ typename Lanes<T>::M prop_z(T (&p)[6], T (&c)[21], Trig<T>& g, T dkdw,
                                                       float Z, const Overlap& ov = Overlap()) {
  ov();  // the caller's independent work, beside the path length's reciprocal
  const T dz = T(Z) - p[2];
  const T tanth = fdiv(g.sth, g.cth);
  const T h = dz * tanth;
  const auto fail = not_(lt(T(0.f), h));
  if (any(fail)) return fail;
  const T kappa = dkdw * p[3];
  const T u = T(0.5f) * kappa * h;
  T s, cu, sp;
  sinc_cs(u, s, cu, sp);
  const T su = u * s;  // sin(u)
  T cm = g.cphi, sm = g.sphi;
  turn(cm, sm, cu, su);  // phi + u
  const T hs = h * s;
  const T dx = hs * cm, dy = hs * sm;
  T c1 = cm, s1 = sm;
  turn(c1, s1, cu, su);  // phi + 2u = phi'
  const T hh = T(0.5f) * h * h * dkdw;
  const T hth = fdiv(dz, g.cth * g.cth);  // dh/dtheta
  // grad h = (0, 0, -tan(theta), 0, 0, dh/dtheta); d p'/d h = (cos phi',
  // sin phi', 0 on the plane, 0, kappa, 0)
  const T gr[6] = {T(0.f), T(0.f), -tanth, T(0.f), T(0.f), hth};
  const T v[6] = {c1, s1, T(0.f), T(0.f), kappa, T(0.f)};
  similarity_rank1<false, (ZFREE ? 0u : (1u << 2)) | (1u << 5), (1u << 0) | (1u << 1) | (1u << 4)>(
      c, hh * fma(sp, cm, -(s * sm)), -dy, hh * fma(sp, sm, s * cm), dx, T(0.f), h * dkdw, gr, v);
  p[0] += dx;
  p[1] += dy;
  p[2] = T(Z);
  p[4] = fma(T(2.f), u, p[4]);
  g.cphi = c1;
  g.sphi = s1;
  return fail;
}

// atan(t) / t: its Taylor series to t^12 (remainder below 2.5e-10 for
// |t| <= 1/4, the range crossing_start admits); in double atan itself.
template <class T>
__device__ __forceinline__ T atan_ratio(T t) {
  const T t2 = t * t;
  return fma(t2, fma(t2, fma(t2, fma(t2, fma(t2, fma(t2, T(1.f / 13.f), T(-1.f / 11.f)),
                                             T(1.f / 9.f)), T(-1.f / 7.f)), T(1.f / 5.f)),
                      T(-1.f / 3.f)), T(1.f));
}
__device__ __forceinline__ double atan_ratio(double t) { return t != 0.0 ? ::atan(t) / t : 1.0; }

// Where the helix of the propagation crosses the cylinder r = R, in closed
// form.  With b0 and t0 the start's components along and across the
// direction phi, c0 = r0^2 - R^2 and t = tan(kappa h / 2), the transverse
// displacement over h is the chord 2 sin(kappa h / 2) / kappa at angle
// phi + kappa h / 2, and r(h)^2 = R^2 multiplied by (1 + t^2) kappa^2 / 2 is
// the quadratic
//   2 F t^2 + 2 kappa b0 t + kappa^2 c0 / 2 = 0,  F = 1 + kappa (t0 + kappa c0 / 4).
// Its discriminant is kappa^2 X with X = b0^2 - c0 F: the circle misses the
// cylinder exactly when X < 0.  The roots are t = kappa hl / 2 with
// hl = -c0 / (b0 +- sqrt(X)); each gives h = 2 atan(t) / kappa modulo one
// turn, 2 pi / |kappa|, and the first forward crossing is the smaller h in
// (0, 2 pi / |kappa|].
//
// crossing_exact: that first forward crossing for one lane, from any start
// (atan2 for the angles); -1 when the cylinder is not reached.  A track
// with |kappa| R below 1e-9 is a straight line: the smaller positive root of
// h^2 + 2 b0 h + c0 = 0.
template <class S>
__device__ __noinline__ S crossing_exact(S x, S y, S cph, S sph, S kappa, S R) {
  const S b0 = fma(x, cph, y * sph);
  const S t0 = fma(y, cph, -(x * sph));
  const S c0 = fma(x, x, fma(y, y, -(R * R)));
  S best = S(-1);
  if (fabs(kappa) * R < S(1e-9)) {
    const S disc = fma(b0, b0, -c0);
    if (!(disc >= S(0))) return S(-1);
    const S qv = -(b0 + copysign(sqrt(disc), b0));
    const S r[2] = {qv, qv != S(0) ? c0 / qv : S(0)};
    for (int k = 0; k < 2; ++k)
      if (r[k] > S(0) && (best < S(0) || r[k] < best)) best = r[k];
  } else {
    const S F = fma(kappa, fma(S(0.25) * kappa, c0, t0), S(1));
    const S X = fma(b0, b0, -(c0 * F));
    if (!(X >= S(0))) return S(-1);
    const S sq = sqrt(X), num = S(-0.5) * kappa * c0;
    const S period = S(2) * pi_<S>() / fabs(kappa);
    for (int k = 0; k < 2; ++k) {
      S hk = S(2) * atan2(num, k ? b0 - sq : b0 + sq) / kappa;
      hk -= floor(hk / period) * period;
      if (!(hk > S(0))) hk += period;
      if (best < S(0) || hk < best) best = hk;
    }
  }
  return best > S(0) ? best : S(-1);
}

// crossing_start: the same for all lanes.  From inside the cylinder
// (c0 <= 0) with X >= 0, the root with b0 + sqrt(X) > 0 is the first forward
// crossing: for F >= 0 the two roots in t have opposite signs and it is the
// forward one; for F < 0 both lie on the same side, ahead of the track when
// b0 > 0 with this one the nearer, behind it when b0 < 0, where
// b0 + sqrt(X) < 0.  Within |t| <= 1/4 (a turn below 0.49 rad) atan(t) / t
// is its series and h = hl atan(t) / t costs one square root and one
// division.  Returns the lanes that cannot reach the cylinder.  Every other
// lane needs crossing_exact: with EXACT a one-lane type calls it here;
// otherwise, and always for packed lanes (F2), such a lane is returned as
// failing and its caller reruns the surface for it (the fused kernel
// propagates each track of the pair alone from there; a call inside the
// packed loop cost it registers on every layer).
template <class T, bool EXACT>
__device__ __forceinline__ typename Lanes<T>::M crossing_start(T x, T y, T cph, T sph, T kappa,
                                                               float R, T b0, T c0, T& h) {
  using M = typename Lanes<T>::M;
  const T t0 = fma(y, cph, -(x * sph));
  const T F = fma(kappa, fma(T(0.25f) * kappa, c0, t0), T(1.f));
  const T X = fma(b0, b0, -(c0 * F));
  const T den = b0 + fsqrt(X);
  const T hl = fdiv(-c0, den);
  const T t = T(0.5f) * kappa * hl;
  // X < 0 (the circle misses the cylinder) makes den NaN, which fails den > 0
  const M ok = and_(le(c0, T(0.f)), and_(lt(T(0.f), den), le(fabs_(t), T(0.25f))));
  h = hl * atan_ratio(t);
  if constexpr (Lanes<T>::n > 1 || !EXACT) {
    return not_(ok);
  } else {
    if (ok) return false;
    h = crossing_exact<T>(x, y, cph, sph, kappa, T(R));
    return !(h > T(0));
  }
}

// Where path_r starts when line_start is not set.  kAuto: the closed-form
// crossing (crossing_start), in its exact form where a one-lane type needs it.
// kFast: the series form only; a lane that needs the exact form is returned
// as failing, so that the caller can rerun the surface with kGiven from
// crossing_exact outside its hot loop (a call or the exact form's code inside
// that loop slowed the memory-bound finder by 20 %).  kGiven: h_given.
enum class Start { kAuto, kFast, kGiven };

// The helix quantities of path_r's last evaluation.
template <class T>
struct PathR {
  T h, d, u, s, cu, sp, cm, sm, px, py, c1, s1;
  T ib;  // 1 / b, b = (px, py) . (c1, s1)
};

// Path length to the cylinder r = R by straight-line steps along the current
// direction: from a start h, repeatedly the helix at h and a straight step
// along its direction to the circle, until a step is below tol_abs.  With
// line_start (and with SEEDED) the start is the straight-line distance from
// (x, y) along phi, and a lane whose straight line misses the circle, or that
// starts outside moving outwards, counts as not reaching it.  Otherwise the
// start is the closed-form crossing (crossing_start), which decides
// reachability exactly, and one evaluation confirms it.  Returns the mask of
// lanes that cannot reach the cylinder (the other outputs are then
// meaningless); with packed lanes, and with Start::kFast, also those that
// need the exact form of the crossing start.  On return h is the path length;
// the helix quantities (u, s, cu, cm, sm, px, py, c1, s1) are those of the
// last evaluation, at h - d.  iters[i] counts lane i's iterations; notconv
// marks lanes that reached max_iter.
//
// SEEDED: gseed is the learned seed's output g (mlp.cuh); the iteration starts
// at h_line + g kappa h_line^2 / 2 instead of the straight-line distance
// h_line when the start is inside the cylinder and that value is finite and
// within h_line / 4 of h_line.  The iteration, its tolerance and its result
// are otherwise unchanged.
template <class T, bool SEEDED = false, Start START = Start::kAuto, class Overlap = NoOverlap>
__device__ __forceinline__ typename Lanes<T>::M path_r(const T (&p)[6], const Trig<T>& g, T kappa,
                                                       float R, int max_iter, float tol_abs,
                                                       bool line_start,
                                                       unsigned (&iters)[Lanes<T>::n],
                                                       typename Lanes<T>::M& notconv, PathR<T>& w,
                                                       T gseed = T(0.f), T h_given = T(0.f),
                                                       const Overlap& ov = Overlap()) {
  using M = typename Lanes<T>::M;
  const T sph = g.sphi, cph = g.cphi;
  const T x = p[0], y = p[1];
  const T R2 = T(R) * T(R);
  const T hk = T(0.5f) * kappa;  // u = hk h
  const T b0 = fma(x, cph, y * sph);
  const T c0 = fma(x, x, fma(y, y, -R2));
  const M inside = le(c0, T(0.f));
  T h;
  M fail;
  // ov: independent work of the caller, run once, in the same straight-line
  // code as the start's serial chain so that the two can interleave
  if constexpr (START == Start::kGiven) {
    ov();
    h = h_given;
    fail = not_(lt(T(0.f), h));
    if (any(fail)) return fail;
  } else if (SEEDED || line_start) {
    ov();
    // The transverse circle (centre c, radius rho = 1/|kappa|) reaches radius
    // R only if |c| + rho >= R, which always holds when rho >= R.
    fail = lt(T(1.f), T(R) * fabs_(kappa));
    if (any(fail)) {
      const T irs = frcp(kappa);  // signed radius
      const T cx = fma(-sph, irs, x), cy = fma(cph, irs, y);
      fail = and_(fail, lt(fsqrt(fma(cx, cx, cy * cy)) + fabs_(irs), T(R)));
    }
    // First step: along the initial direction to the circle (forward root
    // from inside; from outside, the nearer forward root when moving inwards).
    const T disc0 = fma(b0, b0, -c0);
    const T sq0 = fsqrt(disc0);
    fail = or_(fail, or_(lt(disc0, T(0.f)), and_(not_(inside), not_(lt(b0, T(0.f))))));
    if (any(fail)) return fail;
    h = sel(inside, sel(lt(T(0.f), b0), fdiv(-c0, b0 + sq0), sq0 - b0), fdiv(c0, sq0 - b0));
    if constexpr (SEEDED) {
      const T hs = fma(gseed * T(0.5f) * kappa, h * h, h);
      h = sel(and_(and_(inside, finite_(hs)), le(fabs_(hs - h), T(0.25f) * h)), hs, h);
    }
  } else {
    ov();
    fail = crossing_start<T, START == Start::kAuto>(x, y, cph, sph, kappa, R, b0, c0, h);
    if (any(fail)) return fail;
  }
  // The directions phi + u and phi + 2u come from turning (cos phi, sin phi)
  // by u.  A lane that has converged keeps its h.  The first step is taken
  // outside the loop (from the closed-form crossing it is almost always the
  // only one, and peeled it is 3 % faster); max_iter >= 1.
  M conv = lt(T(1.f), T(0.f));  // all false
  T u = T(0.f), s = T(1.f), cu = T(1.f), sp = T(0.f), sm = sph, cm = cph, px = x, py = y, c1 = cph,
    s1 = sph, d = T(0.f), ib = T(0.f);
  auto step = [&]() {
#pragma unroll
    for (int i = 0; i < Lanes<T>::n; ++i) iters[i] += Lanes<T>::get(conv, i) ? 0u : 1u;
    u = hk * h;
    sinc_cs(u, s, cu, sp);
    const T su = u * s;
    cm = cph;
    sm = sph;
    turn(cm, sm, cu, su);  // phi + u
    const T hs = h * s;
    px = fma(hs, cm, x);
    py = fma(hs, sm, y);
    c1 = cm;
    s1 = sm;
    turn(c1, s1, cu, su);  // phi + 2u
    // Step along (c1, s1) to the circle: d^2 + 2 b d + c2 = 0, smaller root.
    const T b = fma(px, c1, py * s1);
    const T c2 = fma(px, px, fma(py, py, -R2));
    ib = frcp(b);
    if (all(le(fabs_(c2), T(1e-4f) * (b * b)))) {
      // Close to the circle the root is -c2 / (2 b) (1 + c2 / (4 b^2) + ...):
      // the dropped factor is below 2.5e-5 relative, on a step below
      // 5e-5 |b|; on a converged step (|d| <= tol) it moves h by less than
      // 1e-12 R^2 / |b|, far below FP32 resolution.
      d = T(-0.5f) * c2 * ib;
    } else {
      const T disc = fma(b, b, -c2);
      // where the line misses the circle (disc < 0) the Newton step -c2 / (2 b)
      d = fdiv(-c2, sel(le(T(0.f), disc), b + copysign_(fsqrt(disc), b), T(2.f) * b));
    }
    d = sel(conv, T(0.f), d);
    h += d;
    conv = or_(conv, le(fabs_(d), T(tol_abs)));
  };
  step();
  for (int it = 1; it < max_iter && !all(conv); ++it) step();
  notconv = not_(conv);
  w = {h, d, u, s, cu, sp, cm, sm, px, py, c1, s1, ib};
  return fail;
}

// Propagation to the cylinder r = R (path length from path_r).  Returns the
// mask of lanes that cannot reach the cylinder; if any lane fails nothing is
// modified.  LOCAL: c holds the local form (to_local_r) with the null
// direction (bc, bs), and leaves in the local form at the new point, whose
// azimuth replaces (bc, bs); otherwise c is the 6x6 packed covariance.
// LOCAL also leaves the direction (g.cphi, g.sphi) at the angle of the last
// evaluation, lag = kappa d short of p[4]: the caller turns it on with the
// update's change of phi (normalise), one turn instead of two.
template <class T, bool SEEDED, Start START, bool LOCAL, class Overlap = NoOverlap>
__device__ __forceinline__ typename Lanes<T>::M prop_r_impl(
    T (&p)[6], T (&c)[LOCAL ? 15 : 21], T& bc, T& bs, Trig<T>& g, T dkdw, float R, int max_iter,
    float tol_abs, bool line_start, unsigned (&iters)[Lanes<T>::n],
    typename Lanes<T>::M& notconv, T gseed, T h_given, T& lag, const Overlap& ov = Overlap()) {
  const T x = p[0], y = p[1];
  const T kappa = dkdw * p[3];
  PathR<T> w;
  const auto fail = path_r<T, SEEDED, START>(p, g, kappa, R, max_iter, tol_abs, line_start,
                                             iters, notconv, w, gseed, h_given, ov);
  if (any(fail)) return fail;
  const T h = w.h, d = w.d, s = w.s, sp = w.sp, cm = w.cm, sm = w.sm;
  T px = w.px, py = w.py, c1 = w.c1, s1 = w.s1;
  // The loop evaluated the helix at h - d; move along the tangent by d
  // (the neglected curvature term, kappa d^2 / 2, is below FP32 resolution
  // once |d| <= tol) and turn the direction by kappa d.
  px = fma(d, c1, px);
  py = fma(d, s1, py);
  const T isth = frcp(g.sth);
  const T cot = g.cth * isth;
  const T dx = px - x, dy = py - y;
  const T hh = T(0.5f) * h * h * dkdw;
  const T Xw = hh * fma(sp, cm, -(s * sm));
  const T Yw = hh * fma(sp, sm, s * cm);
  // grad h = -grad g / (dg/dh) with g = x'^2 + y'^2 - R^2.  dg/dh / 2 =
  // (px, py) . (c1, s1) = b + d with b the last evaluation's: on converged
  // lanes (|d| <= tol) 1 / (b + d) = ib (1 - d ib) to within (d ib)^2.
  T iD;
  if (!any(notconv))
    iD = fma(-(d * w.ib), w.ib, w.ib);
  else
    iD = frcp(fma(px, c1, py * s1));
  const T hw = -(fma(px, Xw, py * Yw) * iD);
  const T hp = fma(px, dy, -(py * dx)) * iD;
  if constexpr (LOCAL) {
    // the new null direction: the azimuth of the crossing
    const T ir = frsqrt(fma(px, px, py * py));
    const T c2 = px * ir, s2 = py * ir;
    // A_l = P' A B: (l, l) = t'.t, (l, w) = t'.(Xw, Yw), (l, phi) = t'.(-dy, dx)
    // with t = (-bs, bc), t' = (-s2, c2); g_l = B^T g; v_l = P' v
    similarity_local_r(c, fma(s2, bs, c2 * bc), fma(c2, Yw, -(s2 * Xw)), fma(c2, dx, s2 * dy),
                       -(h * isth * isth), h * dkdw, fma(bs, px, -(bc * py)) * iD, hw, hp,
                       fma(c2, s1, -(s2 * c1)), cot, kappa);
    bc = c2;
    bs = s2;
  } else {
    const T hx = -(px * iD), hy = -(py * iD);
    // d p'/d h = (cos phi', sin phi', cot theta, 0, kappa, 0)
    const T gr[6] = {hx, hy, T(0.f), hw, hp, T(0.f)};
    const T v[6] = {c1, s1, cot, T(0.f), kappa, T(0.f)};
    similarity_rank1<true, (1u << 0) | (1u << 1) | (1u << 3) | (1u << 4),
                     (1u << 0) | (1u << 1) | (1u << 2) | (1u << 4)>(
        c, Xw, -dy, Yw, dx, -(h * isth * isth), h * dkdw, gr, v);
  }
  p[0] = px;
  p[1] = py;
  p[2] = fma(h, cot, p[2]);
  p[4] = fma(kappa, h, p[4]);
  if constexpr (LOCAL) {
    lag = kappa * d;
  } else {
    // the last step d is below the tolerance on converged lanes, so kappa d
    // is far inside the series' range and needs no range test
    if (!any(notconv))
      turn_small(c1, s1, kappa * d);
    else
      turn_by(c1, s1, kappa * d);
  }
  g.cphi = c1;
  g.sphi = s1;
  return fail;
}

template <class T, bool SEEDED = false, Start START = Start::kAuto>
__device__ __forceinline__ typename Lanes<T>::M prop_r(T (&p)[6], T (&c)[21], Trig<T>& g, T dkdw,
                                                       float R, int max_iter, float tol_abs,
                                                       bool line_start,
                                                       unsigned (&iters)[Lanes<T>::n],
                                                       typename Lanes<T>::M& notconv,
                                                       T gseed = T(0.f), T h_given = T(0.f)) {
  T unused0, unused1, unused2;
  return prop_r_impl<T, SEEDED, START, false>(p, c, unused0, unused1, g, dkdw, R, max_iter,
                                              tol_abs, line_start, iters, notconv, gseed,
                                              h_given, unused2);
}

// As prop_r, on the local form (cl, bc, bs) of the covariance; the direction
// (g.cphi, g.sphi) is left lag short of p[4] (see prop_r_impl).  ov: work
// independent of the path length, overlapped with its start (path_r).
template <class T, Start START = Start::kAuto, class Overlap = NoOverlap>
__device__ __forceinline__ typename Lanes<T>::M prop_r_local(T (&p)[6], T (&cl)[15], T& bc, T& bs,
                                                             Trig<T>& g, T dkdw, float R,
                                                             int max_iter, float tol_abs,
                                                             bool line_start,
                                                             unsigned (&iters)[Lanes<T>::n],
                                                             typename Lanes<T>::M& notconv,
                                                             T& lag, T h_given = T(0.f),
                                                             const Overlap& ov = Overlap()) {
  return prop_r_impl<T, false, START, true>(p, cl, bc, bs, g, dkdw, R, max_iter, tol_abs,
                                            line_start, iters, notconv, T(0.f), h_given, lag, ov);
}

// Kalman update with a 2-D measurement: a and b are the columns of C H^T (the
// two measured directions), S = H C H^T + H V H^T, K = C H^T S^-1,
// p += K r, C -= K S K^T, chi2 = r^T S^-1 r.  Evaluated in square-root form:
// with the Cholesky factor S = L L^T, U = [a b] L^-T and z = L^-1 r give
// K S K^T = U U^T, K r = U z and chi2 = |z|^2, i.e. with
// w0 = 1/sqrt(S00) and w1 = 1/sqrt(S00 det S),
//   u0 = a w0,  u1 = (b S00 - a S01) w1,  z0 = r0 w0,  z1 = (r1 S00 - r0 S01) w1,
//   p += u0 z0 + u1 z1,  C -= u0 u0^T + u1 u1^T,  chi2 = z0^2 + z1^2.
// Only the two columns of U stay live through the covariance update (the
// gain form keeps a, b and both columns of K).
//
// FP32 note (COMPENSATED): with the p2z measurement (x, y) the columns a and
// b are strongly correlated and so is S, so b S00 - a S01 and det S cancel;
// both are then formed with the rounding error of the second product
// recovered by an FMA (Kahan's 2x2 determinant).  Without it the 1/pT
// variance loses up to ~1e-4 relative accuracy after 20 layers.  The p2r
// measurement directions (azimuthal, z) are nearly uncorrelated and need no
// compensation.
template <bool COMPENSATED, class T>
struct Sqrt2 {
  T S00, S01, w0, w1;
  __device__ __forceinline__ Sqrt2(T s00, T s01, T s11) : S00(s00), S01(s01) {
    T det;
    if (COMPENSATED) {
      const T w01 = S01 * S01;
      det = fma(S00, s11, -w01) - fma(S01, S01, -w01);
    } else {
      det = fma(S00, s11, -(S01 * S01));
    }
    w0 = frsqrt(S00);
    w1 = frsqrt(S00 * det);
  }
  // x S00 - y S01, with the rounding error of y S01 recovered when compensated
  __device__ __forceinline__ T cross(T x, T y) const {
    if (COMPENSATED) {
      const T t = y * S01;
      return fma(x, S00, -t) - fma(y, S01, -t);
    }
    return fma(x, S00, -(y * S01));
  }
  // chi2 = |z|^2 of the residual r
  __device__ __forceinline__ T chi2(T r0, T r1, T& z0, T& z1) const {
    z0 = r0 * w0;
    z1 = cross(r1, r0) * w1;
    return fma(z0, z0, z1 * z1);
  }
};

//
// SKIP marks rows whose a and b entries the caller knows to be zero (row z
// after a p2z propagation): their parameters and covariance rows and columns
// are left as they are, which is what the update would compute.
// c -= u0 u0^T + u1 u1^T on the 6x6 form, rows in SKIP left alone.
template <unsigned SKIP, class T>
__device__ __forceinline__ void downdate6(T (&c)[21], const T (&u0)[6], const T (&u1)[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      if ((SKIP & (1u << i)) || (SKIP & (1u << j))) continue;
      c[sym(i, j)] = fma(-u0[i], u0[j], fma(-u1[i], u1[j], c[sym(i, j)]));
    }
}

// DEFER: the covariance part is left to the caller (downdate6 with u0, u1).
template <bool COMPENSATED, unsigned SKIP = 0, bool DEFER = false, class T>
__device__ __forceinline__ T kalman_2d(T (&p)[6], T (&c)[21], const T (&a)[6], const T (&b)[6],
                                       T S00, T S01, T S11, T r0, T r1, T (&u0)[6], T (&u1)[6]) {
  const Sqrt2<COMPENSATED, T> q(S00, S01, S11);
  T z0, z1;
  const T chi2 = q.chi2(r0, r1, z0, z1);
  // uncompensated: u1 = b (S00 w1) - a (S01 w1)
  const T al = q.S00 * q.w1, be = q.S01 * q.w1;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (SKIP & (1u << i)) continue;
    u0[i] = a[i] * q.w0;
    u1[i] = COMPENSATED ? q.cross(b[i], a[i]) * q.w1 : fma(b[i], al, -(a[i] * be));
    p[i] = fma(u0[i], z0, fma(u1[i], z1, p[i]));
  }
  if constexpr (!DEFER) downdate6<SKIP>(c, u0, u1);
  return chi2;
}
template <bool COMPENSATED, unsigned SKIP = 0, class T>
__device__ __forceinline__ T kalman_2d(T (&p)[6], T (&c)[21], const T (&a)[6], const T (&b)[6],
                                       T S00, T S01, T S11, T r0, T r1) {
  T u0[6], u1[6];
  return kalman_2d<COMPENSATED, SKIP, false>(p, c, a, b, S00, S01, S11, r0, r1, u0, u1);
}

// c -= u0 u0^T + u1 u1^T on the local form.
template <class T>
__device__ __forceinline__ void downdate_local(T (&c)[15], const T (&u0)[5], const T (&u1)[5]) {
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) c[sym(i, j)] = fma(-u0[i], u0[j], fma(-u1[i], u1[j], c[sym(i, j)]));
}

// kalman_2d on the local form of a p2r covariance (to_local_r), whose first
// measured direction projects onto l with the factor chp: a = chp c_l (c_l
// the l column of c), b = c_z.  chp is folded into the scalars, and the l
// component of the parameter change moves the position along (-bs, bc).
// DEFER: the covariance part, c -= u0 u0^T + u1 u1^T, is left to the caller
// (downdate_local), which can then overlap it with the serial start of the
// next propagation; u0 and u1 are returned either way.
template <bool DEFER = false, class T>
__device__ __forceinline__ T kalman_2d_local(T (&p)[6], T (&c)[15], T bc, T bs, T chp, T S00,
                                             T S01, T S11, T r0, T r1, T (&u0)[5], T (&u1)[5]) {
  const Sqrt2<false, T> q(S00, S01, S11);
  T z0, z1;
  const T chi2 = q.chi2(r0, r1, z0, z1);
  const T w0 = chp * q.w0, al = q.S00 * q.w1, be = chp * (q.S01 * q.w1);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    u0[i] = c[sym(i, 0)] * w0;
    u1[i] = fma(c[sym(i, 1)], al, -(c[sym(i, 0)] * be));
  }
  const T dl = fma(u0[0], z0, u1[0] * z1);
  p[0] = fma(-bs, dl, p[0]);
  p[1] = fma(bc, dl, p[1]);
#pragma unroll
  for (int i = 1; i < 5; ++i) p[i + 1] = fma(u0[i], z0, fma(u1[i], z1, p[i + 1]));
  if constexpr (!DEFER) downdate_local(c, u0, u1);
  return chi2;
}

// After an update: carry cos/sin of phi and theta through the change of the
// angles (given their values before the update), wrap phi into (-pi, pi], and
// flip the charge (qf = +-1 per lane) where w became negative.  Returns the
// mask of flipped lanes.
// NC = 21: the 6x6 covariance; NC = 15: the p2r local form (w is its third
// coordinate).  lag: how far (g.cphi, g.sphi) was behind phi_before.
template <int NC, class T>
__device__ __forceinline__ typename Lanes<T>::M normalise(T (&p)[6], T (&c)[NC], T& qf,
                                                          Trig<T>& g, T phi_before, T th_before,
                                                          T lag = T(0.f)) {
  constexpr int D = NC == 21 ? 6 : 5, W = NC == 21 ? 3 : 2;
  turn_by2(g.cphi, g.sphi, (p[4] - phi_before) + lag, g.cth, g.sth, p[5] - th_before);
  const T k = floor_((pi_<T>() - p[4]) * inv_two_pi_<T>());
  p[4] = fma(k, two_pi_<T>(), p[4]);
  const auto flip = lt(p[3], T(0.f));
  if (any(flip)) {
    const T sgn = sel(flip, T(-1.f), T(1.f));
    p[3] = p[3] * sgn;
    qf = qf * sgn;
#pragma unroll
    for (int i = 0; i < D; ++i)
      if (i != W) c[sym(W, i)] = c[sym(W, i)] * sgn;
  }
  return flip;
}

// p2z update: H measures x and y.  ZFREE: row and column z of c are zero
// (every update follows a propagation to a plane).
template <bool ZFREE = false, class T>
__device__ __forceinline__ T update_z(T (&p)[6], T (&c)[21], const T (&m)[3], const T (&v)[6]) {
  T a[6], b[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    a[i] = c[sym(i, 0)];
    b[i] = c[sym(i, 1)];
  }
  return kalman_2d<true, ZFREE ? (1u << 2) : 0u>(p, c, a, b, a[0] + v[0], b[0] + v[1],
                                                 b[1] + v[2], m[0] - p[0], m[1] - p[1]);
}
// update_z<true> with the covariance part deferred to the caller
// (downdate6<1 << 2> with u0, u1).
template <class T>
__device__ __forceinline__ T update_z_deferred(T (&p)[6], T (&c)[21], const T (&m)[3],
                                               const T (&v)[6], T (&u0)[6], T (&u1)[6]) {
  T a[6], b[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    a[i] = c[sym(i, 0)];
    b[i] = c[sym(i, 1)];
  }
  return kalman_2d<true, (1u << 2), true>(p, c, a, b, a[0] + v[0], b[0] + v[1], b[1] + v[2],
                                          m[0] - p[0], m[1] - p[1], u0, u1);
}

// p2r update: H measures the position along the cylinder's azimuthal
// direction t = (-sin phi_h, cos phi_h, 0) at the hit azimuth, and z.
template <class T>
__device__ __forceinline__ T update_r(T (&p)[6], T (&c)[21], const T (&m)[3], const T (&v)[6]) {
  const T ir = frsqrt(fma(m[0], m[0], m[1] * m[1]));
  const T sh = m[1] * ir, ch = m[0] * ir;
  T a[6], b[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    a[i] = fma(ch, c[sym(i, 1)], -(sh * c[sym(i, 0)]));
    b[i] = c[sym(i, 2)];
  }
  const T vtt = fma(sh * sh, v[0], fma(ch * ch, v[2], T(-2.f) * sh * ch * v[1]));
  const T vtz = fma(ch, v[4], -(sh * v[3]));
  const T S00 = fma(ch, a[1], -(sh * a[0])) + vtt;
  const T S01 = a[2] + vtz;
  const T S11 = b[2] + v[5];
  const T r0 = fma(ch, m[1] - p[1], -(sh * (m[0] - p[0])));
  const T r1 = m[2] - p[2];
  return kalman_2d<false>(p, c, a, b, S00, S01, S11, r0, r1);
}

// The p2r measurement against the local form (cl, bc, bs): the azimuthal
// measurement direction t_h projects onto l with chp = t_h . (-bs, bc), the
// cosine of the angle between the hit's azimuth and the basis azimuth.
// Shared by update_r_local and chi2_r_local, so that the chi2 of a chosen
// candidate is the one its update returns.
template <class T>
struct MeasR {
  T chp, S00, S01, S11, r0, r1;
  __device__ __forceinline__ MeasR(const T (&p)[6], const T (&cl)[15], T bc, T bs,
                                   const T (&m)[3], const T (&v)[6]) {
    const T ir = frsqrt(fma(m[0], m[0], m[1] * m[1]));
    const T sh = m[1] * ir, ch = m[0] * ir;
    chp = fma(sh, bs, ch * bc);
    const T vtt = fma(sh * sh, v[0], fma(ch * ch, v[2], T(-2.f) * sh * ch * v[1]));
    const T vtz = fma(ch, v[4], -(sh * v[3]));
    S00 = fma(chp * chp, cl[sym(0, 0)], vtt);
    S01 = fma(chp, cl[sym(1, 0)], vtz);
    S11 = cl[sym(1, 1)] + v[5];
    r0 = fma(ch, m[1] - p[1], -(sh * (m[0] - p[0])));
    r1 = m[2] - p[2];
  }
};

// update_r on the local form (cl, bc, bs).
template <class T>
__device__ __forceinline__ T update_r_local(T (&p)[6], T (&cl)[15], T bc, T bs, const T (&m)[3],
                                            const T (&v)[6]) {
  const MeasR<T> h(p, cl, bc, bs, m, v);
  T u0[5], u1[5];
  return kalman_2d_local(p, cl, bc, bs, h.chp, h.S00, h.S01, h.S11, h.r0, h.r1, u0, u1);
}
// The same with the covariance part deferred: cl -= u0 u0^T + u1 u1^T is
// the caller's (downdate_local).
template <class T>
__device__ __forceinline__ T update_r_local_deferred(T (&p)[6], T (&cl)[15], T bc, T bs,
                                                     const T (&m)[3], const T (&v)[6],
                                                     T (&u0)[5], T (&u1)[5]) {
  const MeasR<T> h(p, cl, bc, bs, m, v);
  return kalman_2d_local<true>(p, cl, bc, bs, h.chp, h.S00, h.S01, h.S11, h.r0, h.r1, u0, u1);
}

// chi2 of a hit against the prediction in the local form, without the update.
template <class T>
__device__ __forceinline__ T chi2_r_local(const T (&p)[6], const T (&cl)[15], T bc, T bs,
                                          const T (&m)[3], const T (&v)[6]) {
  const MeasR<T> h(p, cl, bc, bs, m, v);
  T z0, z1;
  return Sqrt2<false, T>(h.S00, h.S01, h.S11).chi2(h.r0, h.r1, z0, z1);
}

// chi2 = r^T S^-1 r of a hit on a plane against the prediction, without the
// update (track finding tries every candidate; chi2_r_local on a cylinder).
// The same expressions as update_z and kalman_2d, so the chi2 of the chosen
// candidate is the one its update returns.
template <class T>
__device__ __forceinline__ T chi2_z(const T (&p)[6], const T (&c)[21], const T (&m)[3],
                                    const T (&v)[6]) {
  const T S00 = c[sym(0, 0)] + v[0], S01 = c[sym(1, 0)] + v[1], S11 = c[sym(1, 1)] + v[2];
  T z0, z1;
  return Sqrt2<true, T>(S00, S01, S11).chi2(m[0] - p[0], m[1] - p[1], z0, z1);
}

}  // namespace fitk
