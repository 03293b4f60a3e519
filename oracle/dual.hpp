// Forward-mode dual numbers for the FP64 oracle.
//
// TEST INFRASTRUCTURE ONLY.  This header belongs to the CPU oracle under
// oracle/; nothing in the GPU library includes it.
//
// A Dual<T, N> carries a value v and N directional derivatives d[0..N-1]
// (the truncated Taylor expansion f(x + e) = f(x) + f'(x) e with e^2 = 0).
// T may itself be a Dual, which gives second derivatives: the oracle uses
// Dual<T, 6> to obtain the 6x6 transport Jacobian as the exact derivative
// of the propagate-to-surface map, and an outer Dual<double, K> to obtain
// the gradient of the summed chi2 through that Jacobian.
//
// Every rule below is the textbook derivative of the elementary function.
#pragma once

#include <cmath>
#include <type_traits>

namespace orc {

template <class T, int N>
struct Dual;

inline double value(double x) { return x; }
template <class T, int N>
double value(const Dual<T, N>& x) { return value(x.v); }

template <class T, int N>
struct Dual {
  T v;
  T d[N];

  Dual() : v(0.0) {
    for (int i = 0; i < N; ++i) d[i] = T(0.0);
  }
  // A constant (zero derivative) from anything convertible to T.
  template <class S, class = std::enable_if_t<std::is_convertible_v<S, T>>>
  Dual(const S& x) : v(T(x)) {
    for (int i = 0; i < N; ++i) d[i] = T(0.0);
  }

  // Hidden friends: found by argument-dependent lookup and, being plain
  // functions, they accept a double or a T on either side by conversion.
  friend Dual operator+(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v + b.v;
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
  }
  friend Dual operator-(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v - b.v;
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
  }
  friend Dual operator-(const Dual& a) {
    Dual r;
    r.v = -a.v;
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
  }
  friend Dual operator*(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v * b.v;
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
  }
  friend Dual operator/(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v / b.v;
    T b2 = b.v * b.v;
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / b2;
    return r;
  }
  Dual& operator+=(const Dual& b) { return *this = *this + b; }
  Dual& operator-=(const Dual& b) { return *this = *this - b; }
  Dual& operator*=(const Dual& b) { return *this = *this * b; }
  Dual& operator/=(const Dual& b) { return *this = *this / b; }
};

using std::asin;
using std::atan2;
using std::cos;
using std::fabs;
using std::floor;
using std::sin;
using std::sqrt;
using std::tan;

// d sin(a) = cos(a) da
template <class T, int N>
Dual<T, N> sin(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = sin(a.v);
  T c = cos(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = c * a.d[i];
  return r;
}
// d cos(a) = -sin(a) da
template <class T, int N>
Dual<T, N> cos(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = cos(a.v);
  T s = -sin(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = s * a.d[i];
  return r;
}
// d tan(a) = (1 + tan^2 a) da
template <class T, int N>
Dual<T, N> tan(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = tan(a.v);
  T g = 1.0 + r.v * r.v;
  for (int i = 0; i < N; ++i) r.d[i] = g * a.d[i];
  return r;
}
// d sqrt(a) = da / (2 sqrt a)
template <class T, int N>
Dual<T, N> sqrt(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = sqrt(a.v);
  T g = 0.5 / r.v;
  for (int i = 0; i < N; ++i) r.d[i] = g * a.d[i];
  return r;
}
// d asin(a) = da / sqrt(1 - a^2)
template <class T, int N>
Dual<T, N> asin(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = asin(a.v);
  T g = 1.0 / sqrt(1.0 - a.v * a.v);
  for (int i = 0; i < N; ++i) r.d[i] = g * a.d[i];
  return r;
}
// d atan2(y, x) = (x dy - y dx) / (x^2 + y^2)
template <class T, int N>
Dual<T, N> atan2(const Dual<T, N>& y, const Dual<T, N>& x) {
  Dual<T, N> r;
  r.v = atan2(y.v, x.v);
  T n = x.v * x.v + y.v * y.v;
  for (int i = 0; i < N; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) / n;
  return r;
}
// |a|: derivative sign(a) da (the oracle never evaluates it at a = 0)
template <class T, int N>
Dual<T, N> fabs(const Dual<T, N>& a) {
  return value(a) < 0.0 ? -a : a;
}

}  // namespace orc
