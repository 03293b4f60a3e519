// The FP64 variant of the fused fit: the per-track math of fit_fused_kernel
// (track_math.cuh) instantiated on double, one track per thread, on double
// structure-of-arrays buffers.  The paper's test codes ran in double by
// default (Sec. 5, the FP32 runs are the exception); this variant measures
// what GB300's reduced FP64 rate costs on the same path.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "fit.h"
#include "fused.cuh"
#include "internal.h"

using namespace fitimpl;

namespace {

struct Args64 {
  const double* par_in;
  const double* cov_in;
  const int32_t* q_in;
  int64_t ld_in;
  double* par_out;
  double* cov_out;
  int32_t* q_out;
  double* chi2;
  double* chi2_layer;
  uint8_t* status;
  int64_t ld_out;
  const double* hpos;
  const double* hcov;
  int64_t ld_hit;
  int64_t t0, t1;
  int nlayer;
  double kB;  // kA * B in double
  unsigned long long* counters;
  Geo geo;
};

// One track per thread over all layers; status bits, per-layer chi2 and
// counters as fit_fused_kernel, and the covariance in the same loop form
// (fused.cuh, enter_loop_form): p2z with its zero z row, p2r in the
// cylinder's local coordinates.
template <int MODE>
__global__ void __launch_bounds__(kBlock) fit_f64_kernel(const __grid_constant__ Args64 a) {
  const int64_t t = a.t0 + (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (t >= a.t1) return;
  double p[6], c[21], cl[15], bc = 0.0, bs = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) fitk::ld(p[k], a.par_in + k * a.ld_in + t);
#pragma unroll
  for (int k = 0; k < 21; ++k) fitk::ld(c[k], a.cov_in + k * a.ld_in + t);
  double qf = (double)__ldcs(a.q_in + t);
  double chi2 = 0.0;
  fitk::Trig<double> g = fitk::trig_of(p);
  {
    const double kappa = qf * -a.kB * p[3];
    if (MODE == FIT_MODE_Z) {
      fitk::enter_plane(c, g, kappa);
    } else {
      fitk::enter_line(c, g, kappa, cl);
      bc = g.cphi;
      bs = g.sphi;
    }
  }
  bool moved = false;  // some propagation was applied
  unsigned st = 0u, iters[1] = {0u};
  const Geo& geo = a.geo;
  const int64_t ldh = a.ld_hit;
  for (int l = 0; l < a.nlayer; ++l) {
    double m[3], v[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) fitk::ld(m[k], a.hpos + (3 * l + k) * ldh + t);
#pragma unroll
    for (int k = 0; k < 6; ++k) fitk::ld(v[k], a.hcov + (6 * l + k) * ldh + t);
    const float sf = geo.surf.s[l];
    const double dkdw = qf * -a.kB;
    bool nc = false, failed;
    double lag = 0.0;
    if (MODE == FIT_MODE_Z)
      failed = fitk::prop_z<true>(p, c, g, dkdw, sf);
    else
      failed = fitk::prop_r_local(p, cl, bc, bs, g, dkdw, sf, geo.max_iter, geo.tol * sf,
                                  geo.line_start, iters, nc, lag);
    if (failed) {
      st |= FIT_ST_NO_INTERSECTION;
      if (a.chi2_layer)
        for (int r = l; r < a.nlayer; ++r) a.chi2_layer[(int64_t)r * a.ld_out + t] = 0.0;
      break;
    }
    moved = true;
    const double phi_pred = p[4], th_pred = p[5];
    double x2;
    bool flip;
    if (MODE == FIT_MODE_Z) {
      x2 = fitk::update_z<true>(p, c, m, v);
      flip = fitk::normalise(p, c, qf, g, phi_pred, th_pred);
    } else {
      x2 = fitk::update_r_local(p, cl, bc, bs, m, v);
      flip = fitk::normalise(p, cl, qf, g, phi_pred, th_pred, lag);
    }
    const bool alive = fitk::finite_(x2);
    if (nc) st |= FIT_ST_NOT_CONVERGED;
    if (flip) st |= FIT_ST_CHARGE_FLIP;
    if (!alive) st |= FIT_ST_NONFINITE;
    x2 = alive ? x2 : 0.0;
    chi2 += x2;
    if (a.chi2_layer) a.chi2_layer[(int64_t)l * a.ld_out + t] = x2;
    if (!alive) {
      if (a.chi2_layer)
        for (int r = l + 1; r < a.nlayer; ++r) a.chi2_layer[(int64_t)r * a.ld_out + t] = 0.0;
      break;
    }
  }
  if (!moved) {  // nothing applied: the input covariance
#pragma unroll
    for (int k = 0; k < 21; ++k) fitk::ld(c[k], a.cov_in + k * a.ld_in + t);
  } else if (MODE == FIT_MODE_R) {
    fitk::to_global_r(cl, bc, bs, c);
  }
  bool fin = isfinite(chi2);
#pragma unroll
  for (int k = 0; k < 6; ++k) fin = fin && isfinite(p[k]);
#pragma unroll
  for (int k = 0; k < 21; ++k) fin = fin && isfinite(c[k]);
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

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

}  // namespace

extern "C" int fit_propagate_update_f64(fit_handle* h, const fit_tracks_in_f64* in,
                                        const fit_tracks_out_f64* out, const fit_hits_f64* hits,
                                        int nevt, const int64_t* ntrk, int nlayer,
                                        const int32_t* mode, void* stream) {
  static const std::string w = "fit_propagate_update_f64";
  g_last_error.clear();
  if (!h || !in || !out || !hits) return fail(FIT_ERR_ARG, w + ": NULL argument");
  if (nevt < 0) return fail(FIT_ERR_ARG, w + ": nevt < 0");
  if (nevt > 0 && (!ntrk || !mode)) return fail(FIT_ERR_ARG, w + ": ntrk or mode is NULL");
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
      !hits->pos || !hits->cov)
    return fail(FIT_ERR_ARG, w + ": NULL data pointer");
  const void* ptrs[] = {in->par, in->cov, out->par, out->cov, out->chi2, hits->pos, hits->cov};
  for (const void* p : ptrs)
    if (!aligned8(p)) return fail(FIT_ERR_ARG, w + ": pointer not 8-byte aligned");
  if (in->ld < total || out->ld < total || hits->ld < total)
    return fail(FIT_ERR_ARG, w + ": ld smaller than the number of tracks");
  DeviceGuard guard(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Args64 a{};
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
  a.hpos = hits->pos;
  a.hcov = hits->cov;
  a.ld_hit = hits->ld;
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
      a.kB = 0.00299792458 * (double)h->B[m];
      const int64_t nblk = (t1 - t + kBlock - 1) / kBlock;
      if (nblk > 0x7fffffff) return fail(FIT_ERR_ARG, w + ": too many tracks");
      if (m == FIT_MODE_Z)
        fit_f64_kernel<FIT_MODE_Z><<<(unsigned)nblk, kBlock, 0, s>>>(a);
      else
        fit_f64_kernel<FIT_MODE_R><<<(unsigned)nblk, kBlock, 0, s>>>(a);
      cudaError_t err = cudaGetLastError();
      if (err != cudaSuccess) return cuda_fail(err, "fit_propagate_update_f64: launch");
    }
    t = t1;
  }
  h->tracks += (uint64_t)total;
  return FIT_OK;
}
