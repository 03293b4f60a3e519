// Reverse-mode derivative (adjoint) of one layer of the fused fit, one track
// per thread, FP32.
//
// layer_bwd() recomputes the layer forward from its checkpoint (the state at
// the layer's entry) and then runs the forward program's statements backwards:
// given the adjoints of the layer's outputs (p_out, packed c_out) and the
// weight of the layer's chi2, it returns the adjoints of the layer's inputs
// (p_in, packed c_in) and of the hit position.  Every adjoint statement is the
// reverse of one forward statement of track_math.cuh (same formulas, written
// with one track per thread); the p2r path length h is the implicit function
// of the state whose gradient the forward Jacobian already holds (implicit
// function theorem), so the iteration that finds it is not differentiated.
#pragma once

#include "track_math.cuh"

namespace fitk {

// s''(u) of sin(u)/u: Taylor series (u^10 and below) for |u| <= 1.25, else
// from u s'' + 2 s' + u s = 0.
__device__ __forceinline__ float sinc_dd(float u, float s, float sp) {
  const float u2 = u * u;
  if (fabsf(u) <= 1.25f)
    return fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, 2.1198007e-08f, -2.2546898e-06f),
                                           1.5432099e-04f), -5.9523810e-03f), 0.1f),
                -3.3333333e-01f);
  return -s - fdiv(2.f * sp, u);
}

// Adjoint of c' = J c J^T (similarity<ROWS, EMASK>): accumulates into cb
// (packed) and Eb from the output adjoint cbo (packed).
template <unsigned ROWS, unsigned long long EMASK>
__device__ __forceinline__ void similarity_bwd(const float (&E)[6][6], const float (&c)[21],
                                               const float (&cbo)[21], float (&cb)[21],
                                               float (&Eb)[6][6]) {
  float JC[6][6], JCb[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float acc = (ROWS & row(i)) ? c[sym(i, j)] : 0.f;
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (EMASK & bit(i, k)) acc = fmaf(E[i][k], c[sym(k, j)], acc);
      JC[i][j] = acc;
      JCb[i][j] = 0.f;
    }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      if (!((ROWS & row(i)) && (ROWS & row(j)))) continue;
      const float g = cbo[sym(i, j)];
      JCb[i][j] += g;
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (EMASK & bit(j, k)) {
          JCb[i][k] = fmaf(g, E[j][k], JCb[i][k]);
          Eb[j][k] = fmaf(g, JC[i][k], Eb[j][k]);
        }
    }
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float g = JCb[i][j];
      if (ROWS & row(i)) cb[sym(i, j)] += g;
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (EMASK & bit(i, k)) {
          Eb[i][k] = fmaf(g, c[sym(k, j)], Eb[i][k]);
          cb[sym(k, j)] = fmaf(g, E[i][k], cb[sym(k, j)]);
        }
    }
}

// ---- propagation to a plane ---------------------------------------------
// Forward (recomputed): as prop_z.  Backward: pb, cb get the adjoints of the
// inputs from pbo, cbo (adjoints of the outputs).
__device__ __forceinline__ void prop_z_bwd(const float (&p)[6], const float (&c)[21], float dkdw,
                                           float Z, const float (&pbo)[6], const float (&cbo)[21],
                                           float (&pb)[6], float (&cb)[21]) {
  float sth, cth, sph, cph;
  sincos_cw(p[5], sth, cth);
  sincos_cw(p[4], sph, cph);
  const float dz = Z - p[2];
  const float tanth = fdiv(sth, cth);
  const float h = dz * tanth;
  const float kappa = dkdw * p[3];
  const float u = 0.5f * kappa * h;
  float s, cu;
  sinc_c(u, s, cu);
  const float sp = sinc_deriv(u, s, cu);
  const float su = u * s;
  const float cm = fmaf(cph, cu, -sph * su), sm = fmaf(sph, cu, cph * su);
  const float hs = h * s;
  const float c1 = fmaf(cm, cu, -sm * su), s1 = fmaf(sm, cu, cm * su);
  const float hh = 0.5f * h * h * dkdw;
  const float icth2 = fdiv(1.f, cth * cth);
  const float hth = dz * icth2;
  float E[6][6], Eb[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int k = 0; k < 6; ++k) Eb[i][k] = 0.f;
  E[0][2] = -c1 * tanth;
  E[0][3] = hh * fmaf(sp, cm, -s * sm);
  E[0][4] = -hs * sm;
  E[0][5] = c1 * hth;
  E[1][2] = -s1 * tanth;
  E[1][3] = hh * fmaf(sp, sm, s * cm);
  E[1][4] = hs * cm;
  E[1][5] = s1 * hth;
  E[4][2] = -kappa * tanth;
  E[4][3] = h * dkdw;
  E[4][5] = kappa * hth;
#pragma unroll
  for (int k = 0; k < 21; ++k) cb[k] = 0.f;
  similarity_bwd<kRowsZ, kEZ>(E, c, cbo, cb, Eb);
  // p' = (x + dx, y + dy, Z, w, phi + 2u, theta)
  float dxb = pbo[0], dyb = pbo[1], ub = 2.f * pbo[4];
  pb[0] = pbo[0];
  pb[1] = pbo[1];
  pb[2] = 0.f;
  pb[3] = pbo[3];
  pb[4] = pbo[4];
  pb[5] = pbo[5];
  float c1b = 0.f, s1b = 0.f, tanb = 0.f, hhb = 0.f, spb = 0.f, cmb = 0.f, smb = 0.f, sb = 0.f;
  float hthb = 0.f, kapb = 0.f, hb = 0.f;
  // E entries
  c1b -= tanth * Eb[0][2];
  tanb -= c1 * Eb[0][2];
  hhb += fmaf(sp, cm, -s * sm) * Eb[0][3];
  {
    const float t = hh * Eb[0][3];
    spb += t * cm;
    cmb += t * sp;
    sb -= t * sm;
    smb -= t * s;
  }
  dyb -= Eb[0][4];
  c1b += hth * Eb[0][5];
  hthb += c1 * Eb[0][5];
  s1b -= tanth * Eb[1][2];
  tanb -= s1 * Eb[1][2];
  hhb += fmaf(sp, sm, s * cm) * Eb[1][3];
  {
    const float t = hh * Eb[1][3];
    spb += t * sm;
    smb += t * sp;
    sb += t * cm;
    cmb += t * s;
  }
  dxb += Eb[1][4];
  s1b += hth * Eb[1][5];
  hthb += s1 * Eb[1][5];
  kapb -= tanth * Eb[4][2];
  tanb -= kappa * Eb[4][2];
  hb += dkdw * Eb[4][3];
  kapb += hth * Eb[4][5];
  hthb += kappa * Eb[4][5];
  // hth = dz / cth^2
  float dzb = hthb * icth2;
  float cthb = -2.f * hthb * hth * fdiv(1.f, cth);
  // hh = h^2 dkdw / 2
  hb += hhb * h * dkdw;
  // (c1, s1) = (cm, sm) turned by u
  float cub = fmaf(c1b, cm, s1b * sm), sub = fmaf(-c1b, sm, s1b * cm);
  cmb += fmaf(c1b, cu, s1b * su);
  smb += fmaf(-c1b, su, s1b * cu);
  // dx = hs cm, dy = hs sm
  const float hsb = fmaf(dxb, cm, dyb * sm);
  cmb += dxb * hs;
  smb += dyb * hs;
  hb += hsb * s;
  sb += hsb * h;
  // (cm, sm) = (cos phi, sin phi) turned by u
  const float cphb = fmaf(cmb, cu, smb * su), sphb = fmaf(-cmb, su, smb * cu);
  cub += fmaf(cmb, cph, smb * sph);
  sub += fmaf(-cmb, sph, smb * cph);
  // su = u s; s, cu, sp functions of u
  ub += sub * s;
  sb += sub * u;
  ub += sb * sp - cub * su + spb * sinc_dd(u, s, sp);
  // u = kappa h / 2
  kapb += 0.5f * ub * h;
  hb += 0.5f * ub * kappa;
  // kappa = dkdw w
  pb[3] += kapb * dkdw;
  // h = dz tan(theta)
  dzb += hb * tanth;
  tanb += hb * dz;
  // tan = sin / cos
  const float sthb = tanb * fdiv(1.f, cth);
  cthb -= tanb * tanth * fdiv(1.f, cth);
  pb[2] -= dzb;
  pb[4] += sphb * cph - cphb * sph;
  pb[5] += sthb * cth - cthb * sth;
}

// ---- propagation to a cylinder ------------------------------------------
// Returns false if the cylinder is not reached (nothing is written then).
__device__ __forceinline__ bool prop_r_bwd(const float (&p)[6], const float (&c)[21], float dkdw,
                                           float R, int max_iter, float tol_abs, bool line_start,
                                           const float (&pbo)[6], const float (&cbo)[21],
                                           float (&pb)[6], float (&cb)[21]) {
  Trig<float> g = trig_of(p);
  const float kappa = dkdw * p[3];
  unsigned iters[1] = {0u};
  bool notconv = false;
  PathR<float> w;
  if (path_r(p, g, kappa, R, max_iter, tol_abs, line_start, iters, notconv, w)) return false;
  // Everything below is an explicit function of (p, h) at the final h.
  const float h = w.h;
  const float sph = g.sphi, cph = g.cphi, sth = g.sth, cth = g.cth;
  const float u = 0.5f * kappa * h;
  float s, cu;
  sinc_c(u, s, cu);
  const float sp = sinc_deriv(u, s, cu);
  const float su = u * s;
  const float cm = fmaf(cph, cu, -sph * su), sm = fmaf(sph, cu, cph * su);
  const float hs = h * s;
  const float dx = hs * cm, dy = hs * sm;
  const float px = p[0] + dx, py = p[1] + dy;
  const float c1 = fmaf(cm, cu, -sm * su), s1 = fmaf(sm, cu, cm * su);
  const float isth = fdiv(1.f, sth);
  const float cot = cth * isth;
  const float hh = 0.5f * h * h * dkdw;
  const float Xw = hh * fmaf(sp, cm, -s * sm), Yw = hh * fmaf(sp, sm, s * cm);
  const float D = fmaf(px, c1, py * s1);
  const float iD = fdiv(1.f, D);
  const float hx = -px * iD, hy = -py * iD;
  const float hw = -fmaf(px, Xw, py * Yw) * iD;
  const float hp = fmaf(px, dy, -py * dx) * iD;
  float E[6][6], Eb[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int k = 0; k < 6; ++k) Eb[i][k] = 0.f;
  E[0][0] = c1 * hx;
  E[0][1] = c1 * hy;
  E[0][3] = fmaf(c1, hw, Xw);
  E[0][4] = fmaf(c1, hp, -dy);
  E[1][0] = s1 * hx;
  E[1][1] = s1 * hy;
  E[1][3] = fmaf(s1, hw, Yw);
  E[1][4] = fmaf(s1, hp, dx);
  E[2][0] = cot * hx;
  E[2][1] = cot * hy;
  E[2][3] = cot * hw;
  E[2][4] = cot * hp;
  E[2][5] = -h * isth * isth;
  E[4][0] = kappa * hx;
  E[4][1] = kappa * hy;
  E[4][3] = fmaf(kappa, hw, h * dkdw);
  E[4][4] = kappa * hp;
#pragma unroll
  for (int k = 0; k < 21; ++k) cb[k] = 0.f;
  similarity_bwd<kRowsR, kER>(E, c, cbo, cb, Eb);
  // p' = (px, py, z + h cot, w, phi + kappa h, theta)
  float pxb = pbo[0], pyb = pbo[1];
  float hb = fmaf(pbo[2], cot, pbo[4] * kappa);
  float cotb = pbo[2] * h;
  float kapb = pbo[4] * h;
  pb[0] = 0.f;
  pb[1] = 0.f;
  pb[2] = pbo[2];
  pb[3] = pbo[3];
  pb[4] = pbo[4];
  pb[5] = pbo[5];
  float c1b = 0.f, s1b = 0.f, hxb = 0.f, hyb = 0.f, hwb = 0.f, hpb = 0.f, Xwb = 0.f, Ywb = 0.f;
  float dxb = 0.f, dyb = 0.f, isthb = 0.f;
  // E entries
  c1b += Eb[0][0] * hx + Eb[0][1] * hy + Eb[0][3] * hw + Eb[0][4] * hp;
  hxb += Eb[0][0] * c1;
  hyb += Eb[0][1] * c1;
  hwb += Eb[0][3] * c1;
  Xwb += Eb[0][3];
  hpb += Eb[0][4] * c1;
  dyb -= Eb[0][4];
  s1b += Eb[1][0] * hx + Eb[1][1] * hy + Eb[1][3] * hw + Eb[1][4] * hp;
  hxb += Eb[1][0] * s1;
  hyb += Eb[1][1] * s1;
  hwb += Eb[1][3] * s1;
  Ywb += Eb[1][3];
  hpb += Eb[1][4] * s1;
  dxb += Eb[1][4];
  cotb += Eb[2][0] * hx + Eb[2][1] * hy + Eb[2][3] * hw + Eb[2][4] * hp;
  hxb += Eb[2][0] * cot;
  hyb += Eb[2][1] * cot;
  hwb += Eb[2][3] * cot;
  hpb += Eb[2][4] * cot;
  hb -= Eb[2][5] * isth * isth;
  isthb -= 2.f * Eb[2][5] * h * isth;
  kapb += Eb[4][0] * hx + Eb[4][1] * hy + Eb[4][3] * hw + Eb[4][4] * hp;
  hxb += Eb[4][0] * kappa;
  hyb += Eb[4][1] * kappa;
  hwb += Eb[4][3] * kappa;
  hpb += Eb[4][4] * kappa;
  hb += Eb[4][3] * dkdw;
  // hp = (px dy - py dx) iD
  float iDb = hpb * fmaf(px, dy, -py * dx);
  {
    const float t = hpb * iD;
    pxb += t * dy;
    dyb += t * px;
    pyb -= t * dx;
    dxb -= t * py;
  }
  // hw = -(px Xw + py Yw) iD
  iDb -= hwb * fmaf(px, Xw, py * Yw);
  {
    const float t = -hwb * iD;
    pxb += t * Xw;
    Xwb += t * px;
    pyb += t * Yw;
    Ywb += t * py;
  }
  // hx = -px iD, hy = -py iD
  pxb -= hxb * iD;
  pyb -= hyb * iD;
  iDb -= hxb * px + hyb * py;
  // iD = 1 / D, D = px c1 + py s1
  const float Db = -iDb * iD * iD;
  pxb += Db * c1;
  c1b += Db * px;
  pyb += Db * s1;
  s1b += Db * py;
  // Xw = hh (sp cm - s sm), Yw = hh (sp sm + s cm)
  const float hhb = Xwb * fmaf(sp, cm, -s * sm) + Ywb * fmaf(sp, sm, s * cm);
  float spb, cmb, smb, sb;
  {
    const float t1 = Xwb * hh, t2 = Ywb * hh;
    spb = fmaf(t1, cm, t2 * sm);
    cmb = fmaf(t1, sp, t2 * s);
    sb = fmaf(-t1, sm, t2 * cm);
    smb = fmaf(-t1, s, t2 * sp);
  }
  hb += hhb * h * dkdw;
  // cot = cth isth, isth = 1 / sth
  float cthb = cotb * isth;
  isthb += cotb * cth;
  float sthb = -isthb * isth * isth;
  // (c1, s1) = (cm, sm) turned by u
  float cub = fmaf(c1b, cm, s1b * sm), sub = fmaf(-c1b, sm, s1b * cm);
  cmb += fmaf(c1b, cu, s1b * su);
  smb += fmaf(-c1b, su, s1b * cu);
  // px = x + hs cm, py = y + hs sm (dx, dy the same products)
  pb[0] += pxb;
  pb[1] += pyb;
  const float gx = pxb + dxb, gy = pyb + dyb;
  const float hsb = fmaf(gx, cm, gy * sm);
  cmb += gx * hs;
  smb += gy * hs;
  hb += hsb * s;
  sb += hsb * h;
  // (cm, sm) = (cos phi, sin phi) turned by u
  const float cphb = fmaf(cmb, cu, smb * su), sphb = fmaf(-cmb, su, smb * cu);
  cub += fmaf(cmb, cph, smb * sph);
  sub += fmaf(-cmb, sph, smb * cph);
  // su = u s; s, cu, sp functions of u
  float ub = sub * s;
  sb += sub * u;
  ub += sb * sp - cub * su + spb * sinc_dd(u, s, sp);
  // u = kappa h / 2
  kapb += 0.5f * ub * h;
  hb += 0.5f * ub * kappa;
  // theta, phi through their sine and cosine
  pb[5] += sthb * cth - cthb * sth;
  pb[4] += sphb * cph - cphb * sph;
  // kappa = dkdw w
  pb[3] += kapb * dkdw;
  // h = h(p): grad h = (hx, hy, 0, hw, hp, 0)
  pb[0] = fmaf(hb, hx, pb[0]);
  pb[1] = fmaf(hb, hy, pb[1]);
  pb[3] = fmaf(hb, hw, pb[3]);
  pb[4] = fmaf(hb, hp, pb[4]);
  return true;
}

// ---- Kalman update --------------------------------------------------------
// Adjoint of kalman_2d: from the adjoints of p+ (pbo), c+ (cbo, packed) and
// chi2 (chib) to those of p (pb, set), the columns a, b, S and r
// (accumulated by the caller into c and the hit).
struct UpdAdj {
  float ab[6], bb[6], S00b, S01b, S11b, r0b, r1b;
};

template <bool COMPENSATED>
__device__ __forceinline__ void kalman_2d_bwd(const float (&a)[6], const float (&b)[6], float S00,
                                              float S01, float S11, float r0, float r1,
                                              const float (&pbo)[6], const float (&cbo)[21],
                                              float chib, float (&pb)[6], UpdAdj& A) {
  float k0[6], k1[6], id;
  if (COMPENSATED) {
    const float w01 = S01 * S01;
    id = fdiv(1.f, fmaf(S00, S11, -w01) - fmaf(S01, S01, -w01));
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float t0 = b[i] * S01, t1 = a[i] * S01;
      k0[i] = (fmaf(a[i], S11, -t0) - fmaf(b[i], S01, -t0)) * id;
      k1[i] = (fmaf(b[i], S00, -t1) - fmaf(a[i], S01, -t1)) * id;
    }
  } else {
    id = fdiv(1.f, fmaf(S00, S11, -S01 * S01));
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      k0[i] = fmaf(a[i], S11 * id, -b[i] * S01 * id);
      k1[i] = fmaf(-a[i], S01 * id, b[i] * S00 * id);
    }
  }
  const float i00 = S11 * id, i01 = -S01 * id, i11 = S00 * id;
  // chi2 = Q id, Q = S11 r0^2 - 2 S01 r0 r1 + S00 r1^2
  const float Q = fmaf(S11 * r0, r0, fmaf(S00 * r1, r1, -2.f * S01 * r0 * r1));
  const float Qb = chib * id;
  float idb = chib * Q;
  A.r0b = Qb * 2.f * fmaf(S11, r0, -S01 * r1);
  A.r1b = Qb * 2.f * fmaf(S00, r1, -S01 * r0);
  A.S11b = Qb * r0 * r0;
  A.S01b = -2.f * Qb * r0 * r1;
  A.S00b = Qb * r1 * r1;
  float k0b[6], k1b[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    pb[i] = pbo[i];
    k0b[i] = pbo[i] * r0;
    k1b[i] = pbo[i] * r1;
    A.r0b = fmaf(pbo[i], k0[i], A.r0b);
    A.r1b = fmaf(pbo[i], k1[i], A.r1b);
    A.ab[i] = 0.f;
    A.bb[i] = 0.f;
  }
  // c[i][j] -= k0[i] a[j] + k1[i] b[j] for i >= j
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const float g = cbo[sym(i, j)];
      k0b[i] = fmaf(-g, a[j], k0b[i]);
      A.ab[j] = fmaf(-g, k0[i], A.ab[j]);
      k1b[i] = fmaf(-g, b[j], k1b[i]);
      A.bb[j] = fmaf(-g, k1[i], A.bb[j]);
    }
  // k0 = a i00 + b i01, k1 = a i01 + b i11
  float i00b = 0.f, i01b = 0.f, i11b = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    A.ab[i] += fmaf(k0b[i], i00, k1b[i] * i01);
    A.bb[i] += fmaf(k0b[i], i01, k1b[i] * i11);
    i00b = fmaf(k0b[i], a[i], i00b);
    i01b += fmaf(k0b[i], b[i], k1b[i] * a[i]);
    i11b = fmaf(k1b[i], b[i], i11b);
  }
  // i00 = S11 id, i01 = -S01 id, i11 = S00 id
  A.S11b += i00b * id;
  A.S01b -= i01b * id;
  A.S00b += i11b * id;
  idb += i00b * S11 - i01b * S01 + i11b * S00;
  // id = 1 / det, det = S00 S11 - S01^2
  const float detb = -idb * id * id;
  A.S00b += detb * S11;
  A.S11b += detb * S00;
  A.S01b -= 2.f * detb * S01;
}

// p2z update adjoint: cb (packed) and the hit adjoint mb are accumulated.
__device__ __forceinline__ void update_z_bwd(const float (&p)[6], const float (&c)[21],
                                             const float (&m)[3], const float (&v)[6],
                                             const float (&pbo)[6], const float (&cbo)[21],
                                             float chib, float (&pb)[6], float (&cb)[21],
                                             float (&mb)[3]) {
  float a[6], b[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    a[i] = c[sym(i, 0)];
    b[i] = c[sym(i, 1)];
  }
  UpdAdj A;
  kalman_2d_bwd<true>(a, b, a[0] + v[0], b[0] + v[1], b[1] + v[2], m[0] - p[0], m[1] - p[1], pbo,
                      cbo, chib, pb, A);
#pragma unroll
  for (int k = 0; k < 21; ++k) cb[k] = cbo[k];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    cb[sym(i, 0)] += A.ab[i];
    cb[sym(i, 1)] += A.bb[i];
  }
  cb[sym(0, 0)] += A.S00b;
  cb[sym(1, 0)] += A.S01b;
  cb[sym(1, 1)] += A.S11b;
  mb[0] = A.r0b;
  mb[1] = A.r1b;
  mb[2] = 0.f;
  pb[0] -= A.r0b;
  pb[1] -= A.r1b;
}

// p2r update adjoint (the measurement directions depend on the hit).
__device__ __forceinline__ void update_r_bwd(const float (&p)[6], const float (&c)[21],
                                             const float (&m)[3], const float (&v)[6],
                                             const float (&pbo)[6], const float (&cbo)[21],
                                             float chib, float (&pb)[6], float (&cb)[21],
                                             float (&mb)[3]) {
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
  const float dmx = m[0] - p[0], dmy = m[1] - p[1];
  const float r0 = fmaf(ch, dmy, -sh * dmx);
  const float r1 = m[2] - p[2];
  UpdAdj A;
  kalman_2d_bwd<false>(a, b, S00, S01, S11, r0, r1, pbo, cbo, chib, pb, A);
  float chb = 0.f, shb = 0.f;
  // r0 = ch (my - y) - sh (mx - x); r1 = mz - z
  chb += A.r0b * dmy;
  shb -= A.r0b * dmx;
  mb[0] = -A.r0b * sh;
  mb[1] = A.r0b * ch;
  mb[2] = A.r1b;
  pb[0] += A.r0b * sh;
  pb[1] -= A.r0b * ch;
  pb[2] -= A.r1b;
  // S11 = b2 + v5; S01 = a2 + vtz; S00 = ch a1 - sh a0 + vtt
  A.bb[2] += A.S11b;
  A.ab[2] += A.S01b;
  const float vtzb = A.S01b;
  chb += A.S00b * a[1];
  A.ab[1] += A.S00b * ch;
  shb -= A.S00b * a[0];
  A.ab[0] -= A.S00b * sh;
  const float vttb = A.S00b;
  // vtz = ch v4 - sh v3; vtt = sh^2 v0 + ch^2 v2 - 2 sh ch v1
  chb += vtzb * v[4];
  shb -= vtzb * v[3];
  shb += vttb * 2.f * fmaf(sh, v[0], -ch * v[1]);
  chb += vttb * 2.f * fmaf(ch, v[2], -sh * v[1]);
  // a = ch c[.,1] - sh c[.,0]; b = c[.,2]
#pragma unroll
  for (int k = 0; k < 21; ++k) cb[k] = cbo[k];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    cb[sym(i, 2)] += A.bb[i];
    cb[sym(i, 1)] = fmaf(A.ab[i], ch, cb[sym(i, 1)]);
    cb[sym(i, 0)] = fmaf(-A.ab[i], sh, cb[sym(i, 0)]);
    chb = fmaf(A.ab[i], c[sym(i, 1)], chb);
    shb = fmaf(-A.ab[i], c[sym(i, 0)], shb);
  }
  // sh = my ir, ch = mx ir, ir = (mx^2 + my^2)^(-1/2)
  mb[1] = fmaf(shb, ir, mb[1]);
  mb[0] = fmaf(chb, ir, mb[0]);
  const float irb = fmaf(shb, m[1], chb * m[0]);
  const float ir3 = ir * ir * ir;
  mb[0] = fmaf(-irb * m[0], ir3, mb[0]);
  mb[1] = fmaf(-irb * m[1], ir3, mb[1]);
}

}  // namespace fitk
