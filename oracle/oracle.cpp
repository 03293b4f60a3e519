// FP64 CPU oracle of the fused track propagation + Kalman update.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// CPU-baseline leg of bench.py load this library.  It shares no code, header,
// table or constant with the GPU library under paper_2409_09228_gb300/csrc,
// and neither includes the other.
//
// What it computes (paper Sec. 3, "Description of algorithm"): for every
// track, layer by layer, (1) propagate the track state and its covariance
// along a helix in a uniform solenoidal field to the next detector surface,
// a cylinder r = R (p2r) or a plane z = Z (p2z); (2) update the state with the
// hit on that surface (three coordinates and a 3x3 covariance, Sec. 3.2).
// The paper prints no formula, so this file writes out the textbook
// definitions, with every reading it takes stated where it is taken:
//
//   state p = (x, y, z, w, phi, theta): position [cm], w = 1/pT [1/GeV],
//   azimuth and polar angle of the momentum; charge q = +-1 kept apart.
//   Field B [T] along +z.  Signed curvature kappa = -q * kA * B * w [1/cm]
//   (a positive charge turns clockwise seen from +z, from F = q v x B).
//   Helix by transverse path length h:
//     x(h) = x + [sin(phi + kappa h) - sin(phi)] / kappa
//     y(h) = y - [cos(phi + kappa h) - cos(phi)] / kappa
//     z(h) = z + h cot(theta),  phi(h) = phi + kappa h,  w, theta fixed.
//   p2z: h = (Z - z) tan(theta), closed form.
//   p2r: the exact first positive root of x(h)^2 + y(h)^2 = R^2, from the
//        circle-circle intersection, polished by Newton's method.  (The GPU
//        method iterates towards the same root; the oracle is the root.)
//   Transport Jacobian J = d p_out / d p_in of the propagate-to-surface map,
//   including the dependence of h on p_in; it is obtained by forward-mode
//   differentiation of the map itself (dual.hpp), which is the definition.
//   Covariance C_out = J C J^T.
//   Kalman update with the hit's 2-D position on the surface: H is 2x6 and
//   acts on the position only; p2z measures (x, y); p2r measures z and the
//   coordinate along the cylinder's azimuthal direction at the hit azimuth
//   phi_h = atan2(y_hit, x_hit).  r = H (m - x), S = H C H^T + H V H^T,
//   K = C H^T S^-1, p += K r, C -= K S K^T, chi2 = r^T S^-1 r.
//   After the update phi is wrapped to (-pi, pi]; if w < 0 the charge and the
//   sign of w (with row/column 3 of C) are flipped, which leaves kappa fixed.
//
// Everything is templated on the scalar type: double gives the oracle's
// values, Dual<double, K> gives gradients of the summed chi2 through the
// whole chain (including the Jacobian, via nested duals).
//
// Packed symmetric storage (inputs and outputs): lower triangle, row-major,
// (0,0),(1,0),(1,1),(2,0),... ; 21 entries for C, 6 for the hit covariance
// (xx, yx, yy, zx, zy, zz).
#include <algorithm>
#include <cstdint>
#include <thread>
#include <vector>

#include "dual.hpp"

namespace orc {

constexpr double kA = 0.00299792458;  // GeV / (T cm): pT = kA * B * radius
constexpr double kPi = 3.14159265358979323846;

enum Mode { MODE_R = 0, MODE_Z = 1 };
enum : unsigned {
  ST_NO_INTERSECTION = 1u,
  ST_NOT_CONVERGED = 2u,
  ST_NONFINITE = 4u,
  ST_CHARGE_FLIP = 8u,
};
enum { PX = 0, PY = 1, PZ = 2, PW = 3, PPHI = 4, PTHETA = 5 };

inline int packed_index(int i, int j) {
  if (j > i) std::swap(i, j);
  return i * (i + 1) / 2 + j;
}

template <class T>
struct Track {
  T p[6];
  T C[6][6];
  int q;
};

template <class T>
T curvature(const T& w, int q, double B) {
  return (-double(q) * kA * B) * w;
}

// sin(u)/u, with its Taylor series near 0 so that the straight-line limit
// (kappa -> 0) and its derivatives are exact.
template <class T>
T sinc(const T& u) {
  if (fabs(value(u)) < 1e-4) {
    T u2 = u * u;
    return 1.0 - u2 / 6.0 + u2 * u2 / 120.0;
  }
  return sin(u) / u;
}

// Helix at transverse path length h (paper Sec. 3: "Charged particles in a
// constant magnetic field will travel in a helix").  The x and y lines are
// the definitions above rewritten with sin a - sin b = 2 cos((a+b)/2)
// sin((a-b)/2) and cos a - cos b = -2 sin((a+b)/2) sin((a-b)/2).
template <class T>
void helix(const T p[6], int q, double B, const T& h, T out[6]) {
  T kappa = curvature(p[PW], q, B);
  T u = 0.5 * kappa * h;
  T chord = h * sinc(u);
  T phim = p[PPHI] + u;
  out[PX] = p[PX] + chord * cos(phim);
  out[PY] = p[PY] + chord * sin(phim);
  out[PZ] = p[PZ] + h * cos(p[PTHETA]) / sin(p[PTHETA]);
  out[PW] = p[PW];
  out[PPHI] = p[PPHI] + kappa * h;
  out[PTHETA] = p[PTHETA];
}

// p2z path length to the plane z = Z (paper Sec. 3.2, "propagation to z").
template <class T>
unsigned path_to_z(const T p[6], double Z, T& h) {
  h = (Z - p[PZ]) * tan(p[PTHETA]);
  return value(h) > 0.0 ? 0u : ST_NO_INTERSECTION;
}

// p2r path length: first positive root of x(h)^2 + y(h)^2 = R^2 (paper
// Sec. 3.2, "propagation to r").  The transverse track circle has centre
// c = (x - sin(phi)/kappa, y + cos(phi)/kappa) and radius 1/|kappa|; along
// it (x, y) = c + (sin psi, -cos psi)/kappa with psi = phi + kappa h.  Then
// |.|^2 = R^2 reads sin(psi - alpha) = (R^2 - |c|^2 - 1/kappa^2) kappa/(2|c|),
// alpha = atan2(c_y, c_x), which has two solution families psi; each gives
// h = (psi - phi)/kappa modulo the period 2 pi/|kappa|.
template <class T>
unsigned path_to_r(const T p[6], int q, double B, double R, T& h) {
  T kappa = curvature(p[PW], q, B);
  const double kv = value(kappa);
  if (fabs(kv) * R < 1e-9) {
    // Straight line P + h u with |u| = 1: h^2 + 2 b h + c = 0.
    T b = p[PX] * cos(p[PPHI]) + p[PY] * sin(p[PPHI]);
    T c = p[PX] * p[PX] + p[PY] * p[PY] - R * R;
    T disc = b * b - c;
    if (value(disc) < 0.0) return ST_NO_INTERSECTION;
    T sq = sqrt(disc);
    T h1 = -b - sq, h2 = -b + sq;
    if (value(h1) > 0.0)
      h = h1;
    else if (value(h2) > 0.0)
      h = h2;
    else
      return ST_NO_INTERSECTION;
  } else {
    T cx = p[PX] - sin(p[PPHI]) / kappa;
    T cy = p[PY] + cos(p[PPHI]) / kappa;
    T cn = sqrt(cx * cx + cy * cy);
    T sig = (R * R - cn * cn - 1.0 / (kappa * kappa)) * kappa / (2.0 * cn);
    if (fabs(value(sig)) > 1.0) return ST_NO_INTERSECTION;
    T alpha = atan2(cy, cx);
    T a1 = asin(sig);
    T period = (2.0 * kPi) / fabs(kappa);
    T best = 0.0;
    bool have = false;
    for (int k = 0; k < 2; ++k) {
      T psi = (k == 0) ? alpha + a1 : alpha + (kPi - a1);
      T hk = (psi - p[PPHI]) / kappa;
      double n = floor(value(hk) / value(period));
      hk = hk - n * period;  // into [0, period)
      if (value(hk) <= 0.0) hk = hk + period;
      if (!have || value(hk) < value(best)) {
        best = hk;
        have = true;
      }
    }
    h = best;
  }
  // Newton polish of g(h) = x(h)^2 + y(h)^2 - R^2, g'(h) = 2 (x cos + y sin).
  for (int it = 0; it < 6; ++it) {
    T o[6];
    helix(p, q, B, h, o);
    T g = o[PX] * o[PX] + o[PY] * o[PY] - R * R;
    T dg = 2.0 * (o[PX] * cos(o[PPHI]) + o[PY] * sin(o[PPHI]));
    h = h - g / dg;
  }
  return 0u;
}

template <class T>
unsigned path_length(int mode, const T p[6], int q, double B, double s, T& h) {
  return mode == MODE_Z ? path_to_z(p, s, h) : path_to_r(p, q, B, s, h);
}

// Propagate-to-surface map and its Jacobian (paper Sec. 3.2: propagation
// "involve[s] ... matrix multiplication of up to 6x6 matrices").  J is the
// derivative of the map, computed by seeding the six inputs as duals.
template <class T>
unsigned transport(int mode, const T p[6], int q, double B, double s, T pout[6],
                   T J[6][6], T* hout = nullptr) {
  using D = Dual<T, 6>;
  D pd[6];
  for (int i = 0; i < 6; ++i) {
    pd[i] = D(p[i]);
    pd[i].d[i] = T(1.0);
  }
  D h;
  unsigned st = path_length(mode, pd, q, B, s, h);
  if (st) return st;
  D od[6];
  helix(pd, q, B, h, od);
  // On the plane z = Z by definition: (Z - z) tan(theta) cot(theta) = Z - z.
  if (mode == MODE_Z) od[PZ] = D(s);
  for (int i = 0; i < 6; ++i) {
    pout[i] = od[i].v;
    for (int j = 0; j < 6; ++j) J[i][j] = od[i].d[j];
  }
  if (hout) *hout = h.v;
  return 0u;
}

template <class T>
void symmetrize_from_lower(T C[6][6]) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < i; ++j) C[j][i] = C[i][j];
}

// Track propagation step: p <- f(p), C <- J C J^T.
template <class T>
unsigned propagate(int mode, Track<T>& t, double B, double s) {
  T pout[6], J[6][6];
  unsigned st = transport(mode, t.p, t.q, B, s, pout, J);
  if (st) return st;
  T JC[6][6], Cn[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      T acc = 0.0;
      for (int k = 0; k < 6; ++k) acc = acc + J[i][k] * t.C[k][j];
      JC[i][j] = acc;
    }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      T acc = 0.0;
      for (int k = 0; k < 6; ++k) acc = acc + JC[i][k] * J[j][k];
      Cn[i][j] = acc;
    }
  for (int i = 0; i < 6; ++i) {
    t.p[i] = pout[i];
    for (int j = 0; j < 6; ++j) t.C[i][j] = Cn[i][j];
  }
  symmetrize_from_lower(t.C);
  return 0u;
}

// Kalman update with one hit (paper Sec. 3 step 2 and Sec. 3.2: "small
// matrix multiplication and matrix inverse operations as well as
// trigonometric functions").  m: hit position, V: its 3x3 covariance.
template <class T>
T kalman_update(int mode, Track<T>& t, const T m[3], const T V[3][3], unsigned& st) {
  T Hp[2][3];
  if (mode == MODE_Z) {
    Hp[0][0] = 1.0; Hp[0][1] = 0.0; Hp[0][2] = 0.0;
    Hp[1][0] = 0.0; Hp[1][1] = 1.0; Hp[1][2] = 0.0;
  } else {
    T phih = atan2(m[1], m[0]);
    Hp[0][0] = -sin(phih); Hp[0][1] = cos(phih); Hp[0][2] = 0.0;
    Hp[1][0] = 0.0;        Hp[1][1] = 0.0;       Hp[1][2] = 1.0;
  }
  T r[2];
  for (int a = 0; a < 2; ++a) {
    T acc = 0.0;
    for (int k = 0; k < 3; ++k) acc = acc + Hp[a][k] * (m[k] - t.p[k]);
    r[a] = acc;
  }
  T CHt[6][2];  // C H^T; H is zero outside the position block
  for (int i = 0; i < 6; ++i)
    for (int a = 0; a < 2; ++a) {
      T acc = 0.0;
      for (int k = 0; k < 3; ++k) acc = acc + t.C[i][k] * Hp[a][k];
      CHt[i][a] = acc;
    }
  T S[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      T acc = 0.0;
      for (int k = 0; k < 3; ++k) acc = acc + Hp[a][k] * CHt[k][b];
      T v = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) v = v + Hp[a][k] * V[k][l] * Hp[b][l];
      S[a][b] = acc + v;
    }
  T det = S[0][0] * S[1][1] - S[0][1] * S[1][0];
  T Si[2][2];
  Si[0][0] = S[1][1] / det;
  Si[1][1] = S[0][0] / det;
  Si[0][1] = -S[0][1] / det;
  Si[1][0] = -S[1][0] / det;
  T K[6][2];
  for (int i = 0; i < 6; ++i)
    for (int a = 0; a < 2; ++a) K[i][a] = CHt[i][0] * Si[0][a] + CHt[i][1] * Si[1][a];
  for (int i = 0; i < 6; ++i) t.p[i] = t.p[i] + K[i][0] * r[0] + K[i][1] * r[1];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      T acc = 0.0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) acc = acc + K[i][a] * S[a][b] * K[j][b];
      t.C[i][j] = t.C[i][j] - acc;
    }
  symmetrize_from_lower(t.C);
  T chi2 = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) chi2 = chi2 + r[a] * Si[a][b] * r[b];

  // Normalisation: phi into (-pi, pi].
  double k = floor((kPi - value(t.p[PPHI])) / (2.0 * kPi));
  t.p[PPHI] = t.p[PPHI] + k * (2.0 * kPi);
  // A negative 1/pT means the other charge with the same curvature.
  if (value(t.p[PW]) < 0.0) {
    t.p[PW] = -t.p[PW];
    t.q = -t.q;
    for (int i = 0; i < 6; ++i) {
      if (i == PW) continue;
      t.C[PW][i] = -t.C[PW][i];
      t.C[i][PW] = -t.C[i][PW];
    }
    st |= ST_CHARGE_FLIP;
  }
  return chi2;
}

template <class T>
bool all_finite(const Track<T>& t) {
  for (int i = 0; i < 6; ++i) {
    if (!std::isfinite(value(t.p[i]))) return false;
    for (int j = 0; j <= i; ++j)
      if (!std::isfinite(value(t.C[i][j]))) return false;
  }
  return true;
}

// The per-track layer loop (paper Sec. 3.1: "propagating ... to the next
// layer", one hit per layer; propagation and update are one kernel, Sec. 3.1).
// A track that fails (no intersection, non-finite state) stops at the last
// good state and later layers contribute nothing.
template <class T>
unsigned fit_track(int mode, double B, int nlayer, const double* surf, Track<T>& t,
                   const T (*hpos)[3], const T (*hcov)[3][3], T* chi2_layer, T& chi2) {
  unsigned st = 0u;
  chi2 = 0.0;
  for (int l = 0; l < nlayer; ++l) chi2_layer[l] = 0.0;
  for (int l = 0; l < nlayer; ++l) {
    Track<T> keep = t;
    unsigned s = propagate(mode, t, B, surf[l]);
    if (s) {
      st |= s;
      t = keep;
      break;
    }
    T c = kalman_update(mode, t, hpos[l], hcov[l], st);
    if (!all_finite(t) || !std::isfinite(value(c))) {
      st |= ST_NONFINITE;
      t = keep;
      break;
    }
    chi2_layer[l] = c;
    chi2 = chi2 + c;
  }
  return st;
}

// Track finding (paper Sec. 3: the tracks come from mkFit's pattern
// recognition, whose choice of hit per layer the test codes leave out; they
// take the one hit given).  On each layer the track is propagated and each of
// ncand candidate hits is tried with the Kalman update above on a copy of the
// prediction; the candidate with the smallest chi2 strictly below the gate
// (the lowest index among equal chi2) updates the track, or none does and the
// track keeps its prediction.  cpos/ccov: [nlayer * ncand] candidates, layer
// major; chosen[l] = the candidate taken on layer l or -1; cand_chi2
// [nlayer * ncand] receives every tried chi2 (NaN for layers not reached).
template <class T>
unsigned find_track(int mode, double B, int nlayer, const double* surf, Track<T>& t, int ncand,
                    const T (*cpos)[3], const T (*ccov)[3][3], double gate, T* chi2_layer,
                    int* chosen, T* cand_chi2, T& chi2) {
  unsigned st = 0u;
  chi2 = 0.0;
  for (int l = 0; l < nlayer; ++l) {
    chi2_layer[l] = 0.0;
    chosen[l] = -1;
    for (int k = 0; k < ncand; ++k) cand_chi2[l * ncand + k] = std::nan("");
  }
  for (int l = 0; l < nlayer; ++l) {
    Track<T> keep = t;
    unsigned s = propagate(mode, t, B, surf[l]);
    if (s) {
      st |= s;
      t = keep;
      break;
    }
    int best = -1;
    double best_chi2 = gate;
    for (int k = 0; k < ncand; ++k) {
      Track<T> trial = t;
      unsigned ignored = 0u;
      T c = kalman_update(mode, trial, cpos[l * ncand + k], ccov[l * ncand + k], ignored);
      cand_chi2[l * ncand + k] = c;
      if (value(c) < best_chi2) {
        best = k;
        best_chi2 = value(c);
      }
    }
    chosen[l] = best;
    if (best < 0) continue;
    T c = kalman_update(mode, t, cpos[l * ncand + best], ccov[l * ncand + best], st);
    if (!all_finite(t) || !std::isfinite(value(c))) {
      st |= ST_NONFINITE;
      t = keep;
      break;
    }
    chi2_layer[l] = c;
    chi2 = chi2 + c;
  }
  return st;
}

template <class F>
void parallel_for(int64_t n, int nthreads, F f) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (n < 2 * nthreads) nthreads = 1;
  if (nthreads == 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> pool;
  int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int th = 0; th < nthreads; ++th) {
    int64_t lo = th * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    pool.emplace_back([=] {
      for (int64_t i = lo; i < hi; ++i) f(i);
    });
  }
  for (auto& th : pool) th.join();
}

// Unpacks one track's inputs from the structure-of-arrays buffers
// (component-major, track index fastest, track stride n).
inline void load_inputs(int64_t i, int64_t n, int nlayer, const double* par0,
                        const double* cov0, const int* q0, const double* hpos,
                        const double* hcov, Track<double>& t,
                        std::vector<double>& m, std::vector<double>& V) {
  for (int k = 0; k < 6; ++k) t.p[k] = par0[k * n + i];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) t.C[a][b] = cov0[packed_index(a, b) * n + i];
  t.q = q0[i];
  m.resize(3 * nlayer);
  V.resize(9 * nlayer);
  for (int l = 0; l < nlayer; ++l) {
    for (int k = 0; k < 3; ++k) m[3 * l + k] = hpos[(3 * l + k) * n + i];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) V[9 * l + 3 * a + b] = hcov[(6 * l + packed_index(a, b)) * n + i];
  }
}

}  // namespace orc

using namespace orc;

extern "C" {

// Helix at transverse path h (no surface).
int orc_helix(double B, int q, const double* p, double h, double* out) {
  helix(p, q, B, h, out);
  return 0;
}

// Path length to surface s (radius for mode 0, z for mode 1).
int orc_path_length(int mode, double B, double s, int q, const double* p, double* h) {
  return (int)path_length(mode, p, q, B, s, *h);
}

// p_out and J (row-major 6x6) of the propagate-to-surface map.
int orc_transport(int mode, double B, double s, int q, const double* p, double* pout,
                  double* J, double* h) {
  double Jm[6][6];
  unsigned st = transport(mode, p, q, B, s, pout, Jm, h);
  if (st) return (int)st;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) J[6 * i + j] = Jm[i][j];
  return 0;
}

// One propagation of (p, C) with C packed (21).
int orc_propagate(int mode, double B, double s, int q, const double* p, const double* cov,
                  double* pout, double* covout) {
  Track<double> t;
  for (int i = 0; i < 6; ++i) t.p[i] = p[i];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) t.C[a][b] = cov[packed_index(a, b)];
  t.q = q;
  unsigned st = propagate(mode, t, B, s);
  if (st) return (int)st;
  for (int i = 0; i < 6; ++i) pout[i] = t.p[i];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b <= a; ++b) covout[packed_index(a, b)] = t.C[a][b];
  return 0;
}

// One Kalman update; hit covariance packed (6).  Returns status bits.
int orc_update(int mode, int q, const double* p, const double* cov, const double* m,
               const double* hcov, double* pout, double* covout, int* qout, double* chi2) {
  Track<double> t;
  for (int i = 0; i < 6; ++i) t.p[i] = p[i];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) t.C[a][b] = cov[packed_index(a, b)];
  t.q = q;
  double V[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) V[a][b] = hcov[packed_index(a, b)];
  unsigned st = 0u;
  *chi2 = kalman_update(mode, t, m, V, st);
  for (int i = 0; i < 6; ++i) pout[i] = t.p[i];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b <= a; ++b) covout[packed_index(a, b)] = t.C[a][b];
  *qout = t.q;
  return (int)st;
}

// Exact transverse path length of n independent states (p [6][n], charge
// q [n]) to their own surface s [n] (radius or z): h [n], status [n].
int orc_path_lengths(int mode, double B, int64_t n, const double* s, const int* q,
                     const double* p, double* h, unsigned char* status, int nthreads) {
  parallel_for(n, nthreads, [&](int64_t i) {
    double pi[6];
    for (int k = 0; k < 6; ++k) pi[k] = p[k * n + i];
    double hi = 0.0;
    status[i] = (unsigned char)path_length(mode, pi, q[i], B, s[i], hi);
    h[i] = hi;
  });
  return 0;
}

// Full fit of n tracks over nlayer surfaces.  Layouts (track index fastest,
// stride n): par0/par [6][n], cov0/cov [21][n], q0/q [n], hpos [nlayer][3][n],
// hcov [nlayer][6][n], chi2 [n], chi2_layer [nlayer][n] (may be NULL),
// status [n].  nthreads <= 0 uses every hardware thread.
int orc_fit(int mode, double B, int nlayer, const double* surf, int64_t n,
            const double* par0, const double* cov0, const int* q0, const double* hpos,
            const double* hcov, double* par, double* cov, int* q, double* chi2,
            double* chi2_layer, unsigned char* status, int nthreads) {
  parallel_for(n, nthreads, [&](int64_t i) {
    Track<double> t;
    std::vector<double> m, V;
    load_inputs(i, n, nlayer, par0, cov0, q0, hpos, hcov, t, m, V);
    std::vector<double> cl(nlayer);
    double c2 = 0.0;
    unsigned st = fit_track(mode, B, nlayer, surf, t,
                            reinterpret_cast<const double(*)[3]>(m.data()),
                            reinterpret_cast<const double(*)[3][3]>(V.data()), cl.data(), c2);
    for (int k = 0; k < 6; ++k) par[k * n + i] = t.p[k];
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b <= a; ++b) cov[packed_index(a, b) * n + i] = t.C[a][b];
    q[i] = t.q;
    chi2[i] = c2;
    if (chi2_layer)
      for (int l = 0; l < nlayer; ++l) chi2_layer[l * n + i] = cl[l];
    status[i] = (unsigned char)st;
  });
  return 0;
}

// Track finding over n tracks (find_track).  Candidates [nlayer][ncand][3][n]
// and [nlayer][ncand][6][n]; chosen [nlayer][n]; cand_chi2 [nlayer][ncand][n]
// (may be NULL); other layouts as orc_fit.
int orc_find(int mode, double B, int nlayer, const double* surf, int64_t n, const double* par0,
             const double* cov0, const int* q0, int ncand, const double* cpos,
             const double* ccov, double gate, double* par, double* cov, int* q, double* chi2,
             double* chi2_layer, int* chosen, double* cand_chi2, unsigned char* status,
             int nthreads) {
  parallel_for(n, nthreads, [&](int64_t i) {
    Track<double> t;
    for (int k = 0; k < 6; ++k) t.p[k] = par0[k * n + i];
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) t.C[a][b] = cov0[packed_index(a, b) * n + i];
    t.q = q0[i];
    const int nc = nlayer * ncand;
    std::vector<double> m(3 * nc), V(9 * nc), cl(nlayer), cc(nc);
    std::vector<int> ch(nlayer);
    for (int j = 0; j < nc; ++j) {
      for (int k = 0; k < 3; ++k) m[3 * j + k] = cpos[(3 * j + k) * n + i];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) V[9 * j + 3 * a + b] = ccov[(6 * j + packed_index(a, b)) * n + i];
    }
    double c2 = 0.0;
    unsigned st = find_track(mode, B, nlayer, surf, t, ncand,
                             reinterpret_cast<const double(*)[3]>(m.data()),
                             reinterpret_cast<const double(*)[3][3]>(V.data()), gate, cl.data(),
                             ch.data(), cc.data(), c2);
    for (int k = 0; k < 6; ++k) par[k * n + i] = t.p[k];
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b <= a; ++b) cov[packed_index(a, b) * n + i] = t.C[a][b];
    q[i] = t.q;
    chi2[i] = c2;
    for (int l = 0; l < nlayer; ++l) {
      if (chi2_layer) chi2_layer[l * n + i] = cl[l];
      chosen[l * n + i] = ch[l];
    }
    if (cand_chi2)
      for (int j = 0; j < nc; ++j) cand_chi2[j * n + i] = cc[j];
    status[i] = (unsigned char)st;
  });
  return 0;
}

// Gradient of the summed chi2 of each track with respect to its initial
// parameters (6) and its hit positions (3 per layer), by forward-mode duals
// through the whole chain (seeded in blocks of kBlock inputs).  Layouts as in
// orc_fit; g_par0 [6][n], g_hpos [nlayer][3][n].
int orc_chi2_grad(int mode, double B, int nlayer, const double* surf, int64_t n,
                  const double* par0, const double* cov0, const int* q0, const double* hpos,
                  const double* hcov, double* chi2, double* g_par0, double* g_hpos,
                  unsigned char* status, int nthreads) {
  constexpr int kBlock = 8;
  using G = Dual<double, kBlock>;
  const int nin = 6 + 3 * nlayer;
  parallel_for(n, nthreads, [&](int64_t i) {
    Track<double> t0;
    std::vector<double> m, V;
    load_inputs(i, n, nlayer, par0, cov0, q0, hpos, hcov, t0, m, V);
    std::vector<G> mg(3 * nlayer), cl(nlayer);
    std::vector<G> Vg(9 * nlayer);
    for (int k = 0; k < 9 * nlayer; ++k) Vg[k] = G(V[k]);
    unsigned st = 0u;
    for (int first = 0; first < nin; first += kBlock) {
      Track<G> t;
      for (int k = 0; k < 6; ++k) {
        t.p[k] = G(t0.p[k]);
        if (k >= first && k < first + kBlock) t.p[k].d[k - first] = 1.0;
      }
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) t.C[a][b] = G(t0.C[a][b]);
      t.q = t0.q;
      for (int k = 0; k < 3 * nlayer; ++k) {
        mg[k] = G(m[k]);
        int idx = 6 + k;
        if (idx >= first && idx < first + kBlock) mg[k].d[idx - first] = 1.0;
      }
      G c2 = 0.0;
      st = fit_track(mode, B, nlayer, surf, t, reinterpret_cast<const G(*)[3]>(mg.data()),
                     reinterpret_cast<const G(*)[3][3]>(Vg.data()), cl.data(), c2);
      chi2[i] = c2.v;
      for (int j = 0; j < kBlock && first + j < nin; ++j) {
        int idx = first + j;
        if (idx < 6)
          g_par0[idx * n + i] = c2.d[j];
        else
          g_hpos[(idx - 6) * n + i] = c2.d[j];
      }
    }
    status[i] = (unsigned char)st;
  });
  return 0;
}

}  // extern "C"
