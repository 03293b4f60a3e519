// Track finding: on each layer the track is propagated and every candidate
// hit is tried against the prediction; the candidate with the smallest chi2
// strictly below the gate (the lowest index among equal chi2) updates the
// track, or none does and the track keeps its prediction.  The hit choice of
// mkFit's pattern recognition that the paper's test codes leave out (they
// take the one hit given, Sec. 3); the per-track math is the fused fit's
// (track_math.cuh), in FP32 or FP64, one track per thread.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "fit.h"
#include "fused.cuh"
#include "internal.h"

using namespace fitimpl;

namespace {

constexpr int kMaxCand = 16;

template <class T>
struct FindArgs {
  const T* par_in;
  const T* cov_in;
  const int32_t* q_in;
  int64_t ld_in;
  T* par_out;
  T* cov_out;
  int32_t* q_out;
  T* chi2;
  T* chi2_layer;
  uint8_t* status;
  int64_t ld_out;
  const T* cpos;  // [nlayer][ncand][3][ld_cand]
  const T* ccov;  // [nlayer][ncand][6][ld_cand]
  int ncand;
  int64_t ld_cand;
  int8_t* chosen;  // [nlayer][ld_out]
  T gate;
  int64_t t0, t1;
  int nlayer;
  T kB;
  unsigned long long* counters;
  Geo geo;
};

template <int MODE, class T>
__global__ void __launch_bounds__(kBlock) fit_find_kernel(const __grid_constant__ FindArgs<T> a) {
  const int64_t t = a.t0 + (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (t >= a.t1) return;
  // The covariance in the fused fit's loop form (fused.cuh, enter_loop_form):
  // p2z c with a zero z row, p2r the local form cl with the null direction
  // (bc, bs).
  T p[6], c[21], cl[15], bc, bs;
#pragma unroll
  for (int k = 0; k < 6; ++k) fitk::ld(p[k], a.par_in + k * a.ld_in + t);
#pragma unroll
  for (int k = 0; k < 21; ++k) fitk::ld(c[k], a.cov_in + k * a.ld_in + t);
  T qf = (T)__ldcs(a.q_in + t);
  T chi2 = T(0.f);
  fitk::Trig<T> g = fitk::trig_of(p);
  {
    const T kappa = qf * -a.kB * p[3];
    if (MODE == FIT_MODE_Z) {
      fitk::enter_plane(c, g, kappa);
    } else {
      fitk::enter_line(c, g, kappa, cl);
      bc = g.cphi;
      bs = g.sphi;
    }
  }
  unsigned st = 0u, iters[1] = {0u};
  const Geo& geo = a.geo;
  const int64_t ldc = a.ld_cand;
  // The layer loop runs the p2r crossing start in its series form only
  // (Start::kFast).  A surface where that form does not apply ends the inner
  // loop; the outer one then propagates to it from crossing_exact's start and
  // resumes the inner loop at its candidates.  Kept out of the inner loop,
  // the exact form costs the loop nothing (inside it, 20 %).
  int l = 0;
  bool propagated = false;  // layer l's propagation is done
  T lag = T(0.f);           // p2r: how far (g.cphi, g.sphi) trails p[4] (prop_r_local)
  for (;;) {
    bool rerun = false;
    for (; l < a.nlayer; ++l) {
      const float sf = geo.surf.s[l];
      const T dkdw = qf * -a.kB;
      bool nc = false, failed = false;
      if (propagated)
        propagated = false;
      else if (MODE == FIT_MODE_Z)
        failed = fitk::prop_z<true>(p, c, g, dkdw, sf);
      else
        failed = fitk::prop_r_local<T, fitk::Start::kFast>(p, cl, bc, bs, g, dkdw, sf,
                                                           geo.max_iter, geo.tol * sf,
                                                           geo.line_start, iters, nc, lag);
      if (failed) {
        if (MODE == FIT_MODE_R && !geo.line_start)
          rerun = true;
        else
          st |= FIT_ST_NO_INTERSECTION;
        break;
      }
      if (nc) st |= FIT_ST_NOT_CONVERGED;
      const T* cp = a.cpos + (int64_t)l * a.ncand * 3 * ldc + t;
      const T* cc = a.ccov + (int64_t)l * a.ncand * 6 * ldc + t;
      int best = -1;
      T best_chi2 = a.gate;
      // p2z walks the candidate rows with pointers (13 % faster there); the
      // p2r loop measured 60 % slower that way and keeps the indexed form
      const T* qp = cp;
      const T* qc = cc;
      for (int k = 0; k < a.ncand; ++k) {
        T m[3], v[6];
        if constexpr (MODE == FIT_MODE_Z) {
#pragma unroll
          for (int j = 0; j < 3; ++j, qp += ldc) fitk::ld(m[j], qp);
#pragma unroll
          for (int j = 0; j < 6; ++j, qc += ldc) fitk::ld(v[j], qc);
        } else {
#pragma unroll
          for (int j = 0; j < 3; ++j) fitk::ld(m[j], cp + (3 * k + j) * ldc);
#pragma unroll
          for (int j = 0; j < 6; ++j) fitk::ld(v[j], cc + (6 * k + j) * ldc);
        }
        const T x = (MODE == FIT_MODE_Z) ? fitk::chi2_z(p, c, m, v)
                                         : fitk::chi2_r_local(p, cl, bc, bs, m, v);
        if (x < best_chi2) {
          best = k;
          best_chi2 = x;
        }
      }
      a.chosen[(int64_t)l * a.ld_out + t] = (int8_t)best;
      T x2 = T(0.f);
      if (best >= 0) {
        T m[3], v[6];
#pragma unroll
        for (int j = 0; j < 3; ++j) fitk::ld(m[j], cp + (3 * best + j) * ldc);
#pragma unroll
        for (int j = 0; j < 6; ++j) fitk::ld(v[j], cc + (6 * best + j) * ldc);
        const T phi_pred = p[4], th_pred = p[5];
        bool flip;
        if (MODE == FIT_MODE_Z) {
          x2 = fitk::update_z<true>(p, c, m, v);
          flip = fitk::normalise(p, c, qf, g, phi_pred, th_pred);
        } else {
          x2 = fitk::update_r_local(p, cl, bc, bs, m, v);
          flip = fitk::normalise(p, cl, qf, g, phi_pred, th_pred, lag);
        }
        if (flip) st |= FIT_ST_CHARGE_FLIP;
        if (!fitk::finite_(x2)) {
          st |= FIT_ST_NONFINITE;
          x2 = T(0.f);
          if (a.chi2_layer) a.chi2_layer[(int64_t)l * a.ld_out + t] = x2;
          ++l;
          break;
        }
      } else if (MODE == FIT_MODE_R) {
        fitk::turn_by(g.cphi, g.sphi, lag);  // no update: the propagation's own turn
      }
      chi2 += x2;
      if (a.chi2_layer) a.chi2_layer[(int64_t)l * a.ld_out + t] = x2;
    }
    if (!rerun) break;
    const float sf = geo.surf.s[l];
    const T dkdw = qf * -a.kB;
    const T h0 = fitk::crossing_exact<T>(p[0], p[1], g.cphi, g.sphi, dkdw * p[3], T(sf));
    bool nc = false;
    if (fitk::prop_r_local<T, fitk::Start::kGiven>(p, cl, bc, bs, g, dkdw, sf, geo.max_iter,
                                                   geo.tol * sf, false, iters, nc, lag, h0)) {
      st |= FIT_ST_NO_INTERSECTION;
      break;
    }
    if (nc) st |= FIT_ST_NOT_CONVERGED;
    propagated = true;
  }
  for (int r = l; r < a.nlayer; ++r) {  // layers not reached
    a.chosen[(int64_t)r * a.ld_out + t] = -1;
    if (a.chi2_layer) a.chi2_layer[(int64_t)r * a.ld_out + t] = T(0.f);
  }
  if (l == 0) {  // nothing applied: the input covariance
#pragma unroll
    for (int k = 0; k < 21; ++k) fitk::ld(c[k], a.cov_in + k * a.ld_in + t);
  } else if (MODE == FIT_MODE_R) {
    fitk::to_global_r(cl, bc, bs, c);
  }
  bool fin = fitk::finite_(chi2);
#pragma unroll
  for (int k = 0; k < 6; ++k) fin = fin && fitk::finite_(p[k]);
#pragma unroll
  for (int k = 0; k < 21; ++k) fin = fin && fitk::finite_(c[k]);
  if (!fin) st |= FIT_ST_NONFINITE;
#pragma unroll
  for (int k = 0; k < 6; ++k) a.par_out[k * a.ld_out + t] = p[k];
#pragma unroll
  for (int k = 0; k < 21; ++k) a.cov_out[k * a.ld_out + t] = c[k];
  a.chi2[t] = chi2;
  a.q_out[t] = (int32_t)qf;
  if (a.status) a.status[t] = (uint8_t)st;
  if (st) count_status(st, a.counters);
  if (MODE == FIT_MODE_R) count_iterations(iters[0], &a.counters[4]);
}

bool aligned(const void* p, unsigned a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

template <class T, class In, class Out, class Cand>
int find_tracks(fit_handle* h, const In* in, const Out* out, const Cand* cand, double gate,
                int8_t* chosen, int nevt, const int64_t* ntrk, int nlayer, const int32_t* mode,
                void* stream, const std::string& w) {
  g_last_error.clear();
  if (!h || !in || !out || !cand || !chosen) return fail(FIT_ERR_ARG, w + ": NULL argument");
  if (nevt < 0) return fail(FIT_ERR_ARG, w + ": nevt < 0");
  if (nevt > 0 && (!ntrk || !mode)) return fail(FIT_ERR_ARG, w + ": ntrk or mode is NULL");
  if (cand->ncand < 1 || cand->ncand > kMaxCand)
    return fail(FIT_ERR_ARG, w + ": ncand out of [1, 16]");
  if (!(gate > 0.0)) return fail(FIT_ERR_ARG, w + ": chi2_gate must be > 0");
  int64_t total = 0;
  for (int e = 0; e < nevt; ++e) {
    if (ntrk[e] < 0) return fail(FIT_ERR_ARG, w + ": ntrk[e] < 0");
    if (mode[e] != FIT_MODE_R && mode[e] != FIT_MODE_Z)
      return fail(FIT_ERR_ARG, w + ": mode[e] is not FIT_MODE_R or FIT_MODE_Z");
    if (!h->has[mode[e]]) return fail(FIT_ERR_ARG, w + ": mode not configured");
    if (h->nlayer[mode[e]] != nlayer)
      return fail(FIT_ERR_ARG, w + ": nlayer differs from the configured one");
    total += ntrk[e];
  }
  if (total == 0) return FIT_OK;
  if (!in->par || !in->cov || !in->q || !out->par || !out->cov || !out->q || !out->chi2 ||
      !cand->pos || !cand->cov)
    return fail(FIT_ERR_ARG, w + ": NULL data pointer");
  const void* ptrs[] = {in->par, in->cov, out->par, out->cov, out->chi2, cand->pos, cand->cov};
  for (const void* p : ptrs)
    if (!aligned(p, sizeof(T))) return fail(FIT_ERR_ARG, w + ": misaligned pointer");
  if (in->ld < total || out->ld < total || cand->ld < total)
    return fail(FIT_ERR_ARG, w + ": ld smaller than the number of tracks");
  DeviceGuard guard(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FindArgs<T> a{};
  a.par_in = in->par;
  a.cov_in = in->cov;
  a.q_in = in->q;
  a.ld_in = in->ld;
  a.par_out = out->par;
  a.cov_out = out->cov;
  a.q_out = out->q;
  a.chi2 = out->chi2;
  a.chi2_layer = out->chi2_layer;
  a.status = out->status;
  a.ld_out = out->ld;
  a.cpos = cand->pos;
  a.ccov = cand->cov;
  a.ncand = cand->ncand;
  a.ld_cand = cand->ld;
  a.chosen = chosen;
  a.gate = (T)gate;
  a.nlayer = nlayer;
  a.counters = h->d_counters;
  int64_t t = 0;
  int e = 0;
  while (e < nevt) {  // one launch per run of same-mode events
    const int m = mode[e];
    int64_t t1 = t;
    while (e < nevt && mode[e] == m) t1 += ntrk[e++];
    if (t1 > t) {
      a.t0 = t;
      a.t1 = t1;
      a.geo = h->geo[m];
      a.kB = sizeof(T) == 8 ? (T)(0.00299792458 * (double)h->B[m]) : (T)h->geo[m].kB;
      const int64_t nblk = (t1 - t + kBlock - 1) / kBlock;
      if (nblk > 0x7fffffff) return fail(FIT_ERR_ARG, w + ": too many tracks");
      if (m == FIT_MODE_Z)
        fit_find_kernel<FIT_MODE_Z, T><<<(unsigned)nblk, kBlock, 0, s>>>(a);
      else
        fit_find_kernel<FIT_MODE_R, T><<<(unsigned)nblk, kBlock, 0, s>>>(a);
      cudaError_t err = cudaGetLastError();
      if (err != cudaSuccess) return cuda_fail(err, (w + ": launch").c_str());
    }
    t = t1;
  }
  h->tracks += (uint64_t)total;
  return FIT_OK;
}

}  // namespace

extern "C" int fit_find_tracks(fit_handle* h, const fit_tracks_in* in, const fit_tracks_out* out,
                               const fit_candidates* cand, float chi2_gate, int8_t* chosen,
                               int nevt, const int64_t* ntrk, int nlayer, const int32_t* mode,
                               void* stream) {
  return find_tracks<float>(h, in, out, cand, chi2_gate, chosen, nevt, ntrk, nlayer, mode, stream,
                            "fit_find_tracks");
}

extern "C" int fit_find_tracks_f64(fit_handle* h, const fit_tracks_in_f64* in,
                                   const fit_tracks_out_f64* out, const fit_candidates_f64* cand,
                                   double chi2_gate, int8_t* chosen, int nevt, const int64_t* ntrk,
                                   int nlayer, const int32_t* mode, void* stream) {
  return find_tracks<double>(h, in, out, cand, chi2_gate, chosen, nevt, ntrk, nlayer, mode, stream,
                             "fit_find_tracks_f64");
}
