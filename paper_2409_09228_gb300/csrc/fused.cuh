// Device side of the fused propagate + update fit: the per-track layer loop
// over one or two tracks per thread, shared by the kernels of fit.cu and
// batch.cu.
//
// One thread owns one or two tracks for all layers (paper Sec. 3.1:
// propagation and update in one kernel; Sec. 4.2: per-track intermediates
// kept in registers).  Track state and covariance are loaded once, stay in
// registers through every layer, and are stored once.  Consecutive threads
// read consecutive words of each hit component (structure of arrays, track
// index fastest).
#pragma once

#include "internal.h"
#include "track_math.cuh"

namespace fitimpl {

// 8-byte asynchronous copy global -> shared (cp.async, completion per thread
// through commit and wait groups).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void count_status(unsigned st, unsigned long long* counters) {
  if (st & FIT_ST_NO_INTERSECTION) atomicAdd(&counters[0], 1ull);
  if (st & FIT_ST_NOT_CONVERGED) atomicAdd(&counters[1], 1ull);
  if (st & FIT_ST_NONFINITE) atomicAdd(&counters[2], 1ull);
  if (st & FIT_ST_CHARGE_FLIP) atomicAdd(&counters[3], 1ull);
}

using fitk::F2;
using fitk::Lanes;

// One or two tracks (lane type T) in registers for the whole layer loop.
// The layer loop carries the covariance in a loop form (enter_loop_form):
// for p2r the cylinder's local form cl with the null direction (bc, bs)
// (fitk::to_local_r), for p2z c with a zero z row.  c holds the 6x6
// covariance at load and store.
template <class T>
struct State {
  T p[6], c[21];
  T cl[15], bc, bs;
  T qf;    // charge as +-1.f
  T chi2;  // sum over layers
  fitk::Trig<T> g;
};

// Offset of component k (of K per track) of track t: structure of arrays
// [K][ld] (layout 0), or tiles of 32 consecutive tracks [t / 32][K][32]
// (layout 1, the paper's Matriplex-style AoSoA with bsize 32, Sec. 3.2).
// Arrays with one component per track are the same in both.
template <int L>
__device__ __forceinline__ int64_t ix(int k, int64_t t, int64_t ld, int K) {
  if (L == 0) return k * ld + t;
  return (((t >> 5) * K + k) << 5) + (t & 31);
}

template <int L = 0>
__device__ __forceinline__ void load_state(const FitArgs& a, int64_t t, State<float>& s) {
#pragma unroll
  for (int k = 0; k < 6; ++k) fitk::ld(s.p[k], a.par_in + ix<L>(k, t, a.ld_in, 6));
#pragma unroll
  for (int k = 0; k < 21; ++k) fitk::ld(s.c[k], a.cov_in + ix<L>(k, t, a.ld_in, 21));
  s.qf = (float)__ldcs(a.q_in + t);
  s.chi2 = 0.f;
  s.g = fitk::trig_of(s.p);
}
template <int L = 0>
__device__ __forceinline__ void load_state(const FitArgs& a, int64_t t, State<F2>& s) {
#pragma unroll
  for (int k = 0; k < 6; ++k) fitk::ld(s.p[k], a.par_in + ix<L>(k, t, a.ld_in, 6));
#pragma unroll
  for (int k = 0; k < 21; ++k) fitk::ld(s.c[k], a.cov_in + ix<L>(k, t, a.ld_in, 21));
  const int2 q = __ldcs(reinterpret_cast<const int2*>(a.q_in + t));
  s.qf = F2((float)q.x, (float)q.y);
  s.chi2 = F2(0.f);
  s.g = fitk::trig_of(s.p);
}

// The covariance of s in the loop form, projected onto a surface through the
// start point (fitk::enter_plane, fitk::enter_line): every layer, the first
// included, then propagates from the loop form, and the fit's results are
// those of the 6x6 form.  leave_loop_form: back to the 6x6 covariance in c.
template <int MODE, class T>
__device__ __forceinline__ void enter_loop_form(State<T>& s, float kB) {
  const T kappa = s.qf * T(-kB) * s.p[3];
  if (MODE == FIT_MODE_Z) {
    fitk::enter_plane(s.c, s.g, kappa);
  } else {
    fitk::enter_line(s.c, s.g, kappa, s.cl);
    s.bc = s.g.cphi;
    s.bs = s.g.sphi;
  }
}
template <int MODE, class T>
__device__ __forceinline__ void leave_loop_form(State<T>& s) {
  if (MODE == FIT_MODE_R) fitk::to_global_r(s.cl, s.bc, s.bs, s.c);
}

// Lane i of a two-track state (in the loop form) as a one-track state.
template <int MODE>
__device__ __forceinline__ State<float> lane_of(const State<F2>& s, int i) {
  State<float> r;
#pragma unroll
  for (int k = 0; k < 6; ++k) r.p[k] = Lanes<F2>::get(s.p[k], i);
  if (MODE == FIT_MODE_Z) {
#pragma unroll
    for (int k = 0; k < 21; ++k) r.c[k] = Lanes<F2>::get(s.c[k], i);
  } else {
#pragma unroll
    for (int k = 0; k < 15; ++k) r.cl[k] = Lanes<F2>::get(s.cl[k], i);
    r.bc = Lanes<F2>::get(s.bc, i);
    r.bs = Lanes<F2>::get(s.bs, i);
  }
  r.qf = Lanes<F2>::get(s.qf, i);
  r.chi2 = Lanes<F2>::get(s.chi2, i);
  r.g = {Lanes<F2>::get(s.g.cphi, i), Lanes<F2>::get(s.g.sphi, i), Lanes<F2>::get(s.g.cth, i),
         Lanes<F2>::get(s.g.sth, i)};
  return r;
}

// Writes the outputs of the lanes of s (tracks t, t+1, ...), after the final
// finiteness check.
template <int L = 0, class T>
__device__ __forceinline__ void store_state(const FitArgs& a, int64_t t, const State<T>& s,
                                            unsigned (&st)[Lanes<T>::n]) {
  auto fin = fitk::finite_(s.chi2);
#pragma unroll
  for (int k = 0; k < 6; ++k) fin = fitk::and_(fin, fitk::finite_(s.p[k]));
#pragma unroll
  for (int k = 0; k < 21; ++k) fin = fitk::and_(fin, fitk::finite_(s.c[k]));
#pragma unroll
  for (int i = 0; i < Lanes<T>::n; ++i)
    if (!Lanes<T>::get(fin, i)) st[i] |= FIT_ST_NONFINITE;
#pragma unroll
  for (int k = 0; k < 6; ++k) fitk::st(a.par_out + ix<L>(k, t, a.ld_out, 6), s.p[k]);
#pragma unroll
  for (int k = 0; k < 21; ++k) fitk::st(a.cov_out + ix<L>(k, t, a.ld_out, 21), s.c[k]);
  fitk::st(a.chi2 + t, s.chi2);
#pragma unroll
  for (int i = 0; i < Lanes<T>::n; ++i) {
    a.q_out[t + i] = (int32_t)Lanes<T>::get(s.qf, i);
    if (a.status) a.status[t + i] = (uint8_t)st[i];
  }
}

// The fused layer loop (paper Sec. 3.1: propagate to the next layer, update
// with its hit) for the lanes of s (in the loop form), tracks t, t+1, ...,
// from layer l0.  MODE selects the surface type at compile time.  Returns the layer whose
// surface some live lane cannot reach (its propagation is not applied), the
// layer after one where a packed lane turned non-finite, or nlayer.  A lane
// whose update turns non-finite stops (alive false); its later per-layer
// chi2 entries are 0.
//
// STAGE (p2z, two tracks per thread, SoA, kBlock threads per block): the five
// hit values the p2z update reads are copied one layer ahead into shared
// memory with per-thread asynchronous copies, so that the short plane
// propagation does not wait on their DRAM latency; each thread reads back
// only what it copied itself, so no barrier is needed.
template <int MODE, class T, int L = 0, bool STAGE = false>
__device__ __forceinline__ int run_layers(const FitArgs& a, const Geo& geo, int64_t t, int l0,
                                          State<T>& s,
                                          unsigned (&st)[Lanes<T>::n],
                                          unsigned (&iters)[Lanes<T>::n],
                                          typename Lanes<T>::M& alive) {
  using M = typename Lanes<T>::M;
  const int64_t ldh = a.ld_hit;
  // lanes that hit max_iter or flipped charge on some layer; the status bits
  // (with non-finite for lanes no longer alive) are set once, on return
  M any_nc = fitk::lt(T(1.f), T(0.f)), any_flip = any_nc;
  // The last update's covariance part (c -= pu0 pu0^T + pu1 pu1^T),
  // applied while the next propagation starts (its path length, a serial
  // chain that leaves the FMA pipe idle), or on return.  p2r: the local
  // form's 5 rows; p2z: the 6x6 rows but z.
  constexpr int NU = MODE == FIT_MODE_R ? 5 : 6;
  T pu0[NU], pu1[NU];
#pragma unroll
  for (int k = 0; k < NU; ++k) pu0[k] = pu1[k] = T(0.f);
  auto settle = [&]() {
    if constexpr (MODE == FIT_MODE_R)
      fitk::downdate_local(s.cl, pu0, pu1);
    else
      fitk::downdate6<(1u << 2)>(s.c, pu0, pu1);
#pragma unroll
    for (int k = 0; k < NU; ++k) pu0[k] = pu1[k] = T(0.f);
  };
  auto done = [&](int r) {
    if constexpr (STAGE) cp_async_wait<0>();
    settle();
#pragma unroll
    for (int i = 0; i < Lanes<T>::n; ++i) {
      if (Lanes<T>::get(any_nc, i)) st[i] |= FIT_ST_NOT_CONVERGED;
      if (Lanes<T>::get(any_flip, i)) st[i] |= FIT_ST_CHARGE_FLIP;
      if (!Lanes<T>::get(alive, i)) st[i] |= FIT_ST_NONFINITE;
    }
    return r;
  };
  // The hit rows are walked with two pointers, one row stride per load (ld
  // in SoA, 32 in AoSoA, where a track's rows follow each other within its
  // tile): the 64-bit index products of the indexed form cost p2r 6 % more
  // instructions and 4 % of its time.
  const int64_t rs = L == 0 ? ldh : 32;
  const float* hpl = a.hpos + ix<L>(3 * l0, t, ldh, 3 * a.nlayer);
  const float* hcl = a.hcov + ix<L>(6 * l0, t, ldh, 6 * a.nlayer);
  // STAGE: [layer parity][x, y, cov xx, yx, yy][thread]
  static_assert(!STAGE || (MODE == FIT_MODE_Z && L == 0 && Lanes<T>::n == 2), "p2z pairs only");
  __shared__ float2 hstage[STAGE ? 2 : 1][5][STAGE ? kBlock : 1];
  auto stage = [&](int l) {
    const float* p0 = a.hpos + ix<L>(3 * l, t, ldh, 3 * a.nlayer);
    const float* c0 = a.hcov + ix<L>(6 * l, t, ldh, 6 * a.nlayer);
    const int b = l & 1, x = threadIdx.x;
    cp_async8(&hstage[b][0][x], p0);
    cp_async8(&hstage[b][1][x], p0 + ldh);
    cp_async8(&hstage[b][2][x], c0);
    cp_async8(&hstage[b][3][x], c0 + ldh);
    cp_async8(&hstage[b][4][x], c0 + 2 * ldh);
    cp_async_commit();
  };
  if constexpr (STAGE) {
    if (l0 < a.nlayer) stage(l0);
  }
  // (the layer l + 1 copy is issued before layer l's wait, so one copy is
  // always in flight behind the layer being fitted)
  for (int l = l0; l < a.nlayer; ++l) {
    T m[3], v[6];
    if constexpr (STAGE) {
      if (l + 1 < a.nlayer) {
        stage(l + 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      const int b = l & 1, x = threadIdx.x;
      m[0] = T(hstage[b][0][x]);
      m[1] = T(hstage[b][1][x]);
      m[2] = T(0.f);
      v[0] = T(hstage[b][2][x]);
      v[1] = T(hstage[b][3][x]);
      v[2] = T(hstage[b][4][x]);
      v[3] = v[4] = v[5] = T(0.f);
    } else {
      const float* q = hpl;
#pragma unroll
      for (int k = 0; k < 3; ++k, q += rs) fitk::ld(m[k], q);
      hpl = q;
      q = hcl;
#pragma unroll
      for (int k = 0; k < 6; ++k, q += rs) fitk::ld(v[k], q);
      hcl = q;
    }
    const float sf = geo.surf.s[l];
    const T dkdw = s.qf * T(-geo.kB);
    M fail, nc = fitk::lt(T(1.f), T(0.f));
    T lag = T(0.f);
    if (MODE == FIT_MODE_Z)
      fail = fitk::prop_z<true>(s.p, s.c, s.g, dkdw, sf, settle);
    else
      fail = fitk::prop_r_local(s.p, s.cl, s.bc, s.bs, s.g, dkdw, sf, geo.max_iter,
                                geo.tol * sf, geo.line_start, iters, nc, lag, T(0.f), settle);
    if (fitk::any(fitk::and_(fail, alive))) return done(l);
    const T phi_pred = s.p[4], th_pred = s.p[5];
    T x2;
    M flip;
    if constexpr (MODE == FIT_MODE_Z) {
      x2 = fitk::update_z_deferred(s.p, s.c, m, v, pu0, pu1);
      flip = fitk::normalise(s.p, s.c, s.qf, s.g, phi_pred, th_pred);
    } else {
      x2 = fitk::update_r_local_deferred(s.p, s.cl, s.bc, s.bs, m, v, pu0, pu1);
      flip = fitk::normalise(s.p, s.cl, s.qf, s.g, phi_pred, th_pred, lag);
    }
    if (fitk::any(flip)) {  // the flip negates row w of the pending part too
      constexpr int W = MODE == FIT_MODE_R ? 2 : 3;
      const T sgn = fitk::sel(flip, T(-1.f), T(1.f));
      pu0[W] = pu0[W] * sgn;
      pu1[W] = pu1[W] * sgn;
    }
    alive = fitk::and_(alive, fitk::finite_(x2));
    any_nc = fitk::or_(any_nc, nc);
    any_flip = fitk::or_(any_flip, flip);
    x2 = fitk::sel(alive, x2, T(0.f));
    s.chi2 += x2;
    if (a.chi2_layer) fitk::st(a.chi2_layer + ix<L>(l, t, a.ld_out, a.nlayer), x2);
    if (!fitk::any(alive)) {
      if (a.chi2_layer)
        for (int r = l + 1; r < a.nlayer; ++r)
          fitk::st(a.chi2_layer + ix<L>(r, t, a.ld_out, a.nlayer), T(0.f));
      return done(a.nlayer);
    }
    // A packed lane that turned non-finite would fail every later
    // propagation, and a propagation that fails for any lane is applied to
    // none: the pair splits at the next layer, where the live track goes on
    // alone and the dead one is only stored.
    if constexpr (Lanes<T>::n > 1) {
      if (!fitk::all(alive)) return done(l + 1);
    }
  }
  return done(a.nlayer);
}

// Outputs of a state that run_layers left at layer l: the loop form back to
// the 6x6 covariance, or, where nothing was applied (l = 0: no layers, or
// the first surface out of reach), the input covariance again -- read from
// memory, so that no lane keeps it in registers through the loop.
template <int MODE, int L, class T>
__device__ __forceinline__ void finish_state(const FitArgs& a, int64_t t, int l, State<T>& s) {
  if (l > 0) {
    leave_loop_form<MODE>(s);
  } else {
#pragma unroll
    for (int k = 0; k < 21; ++k) fitk::ld(s.c[k], a.cov_in + ix<L>(k, t, a.ld_in, 21));
  }
}

// A new track (or pair) from memory, in the loop form.
template <int MODE, int L, class T>
__device__ __forceinline__ void begin_state(const FitArgs& a, const Geo& geo, int64_t t,
                                            State<T>& s) {
  load_state<L>(a, t, s);
  enter_loop_form<MODE>(s, geo.kB);
}

// One track alone from layer l0 to the end (or to a surface it cannot
// reach), then its outputs; s is in the loop form.
template <int MODE, int L = 0>
__device__ __forceinline__ void finish_one(const FitArgs& a, const Geo& geo, int64_t t, int l0,
                                           State<float>& s, unsigned& st, unsigned& iters,
                                           bool alive) {
  unsigned st1[1] = {st}, it1[1] = {iters};
  int l = l0;
  if (alive) {
    l = run_layers<MODE, float, L>(a, geo, t, l0, s, st1, it1, alive);
    if (l < a.nlayer) {
      st1[0] |= FIT_ST_NO_INTERSECTION;
      if (a.chi2_layer)
        for (int r = l; r < a.nlayer; ++r) a.chi2_layer[ix<L>(r, t, a.ld_out, a.nlayer)] = 0.f;
    }
  } else if (a.chi2_layer) {  // stopped earlier: no later layer adds to chi2
    for (int r = l0; r < a.nlayer; ++r) a.chi2_layer[ix<L>(r, t, a.ld_out, a.nlayer)] = 0.f;
  }
  finish_state<MODE, L>(a, t, l, s);
  store_state<L>(a, t, s, st1);
  st = st1[0];
  iters = it1[0];
}

// Tracks t and t+1 of the range [t0, t1) (t even).  Both valid: the pair
// shares packed instructions until a surface that one of them cannot reach
// (or, for p2r, whose crossing needs the one-lane form of the closed-form
// start), from where each finishes alone.  One valid (the range starts or ends at an
// odd index): that one alone.
template <int MODE, int L = 0, bool STAGE = false>
__device__ __forceinline__ void run_pair(const FitArgs& a, const Geo& geo, int64_t t0, int64_t t1,
                                         int64_t t, unsigned (&st)[2], unsigned (&iters)[2]) {
  const bool v0 = t >= t0, v1 = t + 1 < t1;
  if (v0 && v1) {
    State<F2> s;
    begin_state<MODE, L>(a, geo, t, s);
    fitk::M2 alive = {true, true};
    const int l = run_layers<MODE, F2, L, STAGE>(a, geo, t, 0, s, st, iters, alive);
    if (l == a.nlayer) {
      finish_state<MODE, L>(a, t, l, s);
      store_state<L>(a, t, s, st);
      return;
    }
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
      State<float> one = lane_of<MODE>(s, i);
      finish_one<MODE, L>(a, geo, t + i, l, one, st[i], iters[i], Lanes<F2>::get(alive, i));
    }
  } else {
    const int i = v0 ? 0 : 1;
    State<float> one;
    begin_state<MODE, L>(a, geo, t + i, one);
    finish_one<MODE, L>(a, geo, t + i, 0, one, st[i], iters[i], true);
  }
}

// First track of the thread's pair: pairs start at even indices so that the
// packed loads and stores are 8-byte aligned.
__device__ __forceinline__ int64_t pair_track(const FitArgs& a) {
  return (a.t0 & ~int64_t(1)) + 2 * ((int64_t)blockIdx.x * kBlock + threadIdx.x);
}

__device__ __forceinline__ void count_iterations(unsigned iters, unsigned long long* counter) {
  const unsigned mask = __activemask();
  const unsigned warp_iters = __reduce_add_sync(mask, iters);
  if ((int)(threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(counter, (unsigned long long)warp_iters);
}

// Variant for fit_propagate_update_noalloc: the same per-track work, with the
// counters kept per event.  a.counters points at a [nevt][kEventSlots] table
// (slot 0, the track count, is filled on the host); evt_off holds the first
// track of events e0..e1 (and the end of e1 - 1), so a track finds its event
// by binary search.
constexpr int kEventSlots = 6;

__device__ __forceinline__ int event_of(int64_t t, const int64_t* __restrict__ evt_off, int e0,
                                        int e1) {
  int lo = e0, hi = e1 - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (evt_off[mid] <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

}  // namespace fitimpl
