// libfit: gradient of the summed chi2 of each track with respect to its hit
// positions and initial parameters (fit_adjoint_forward / _backward in
// fit.h), by a hand-written reverse sweep over the layers with per-layer
// checkpoints.
//
// Forward: the fused fit, one track per thread, that also writes the tape --
// the state (p, packed C, q) at the entry of every layer, and the number of
// layers each track completed.  Backward: for each track, layer by layer from
// the last, the layer is recomputed from its checkpoint and its adjoint
// (adjoint_math.cuh) carries d(weight * sum chi2)/d(state) back to the
// previous layer; the hit-position gradient of each layer falls out on the
// way, the initial-parameter (and initial-covariance) gradient at the end.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "adjoint_math.cuh"
#include "fit.h"
#include "fused.cuh"

namespace fitimpl {
namespace {

constexpr int kTapeRow = 29;  // p (6), packed C (21), q at entry, q after the update
constexpr int kAdjBlock = 128;

struct AdjArgs {
  const float* hpos;
  const float* hcov;
  int64_t ld;  // hits, tape, gradients and grad_chi2 share it
  const float* tape;
  const int32_t* ndone;
  const float* grad_chi2;
  float* g_hpos;
  float* g_par0;
  float* g_cov0;
  int64_t t0, t1;
  int nlayer;
  Geo geo;
};

template <int MODE>
__global__ void __launch_bounds__(kAdjBlock) fit_tape_kernel(const __grid_constant__ FitArgs a,
                                                             float* tape, int32_t* ndone) {
  const int64_t t = a.t0 + (int64_t)blockIdx.x * kAdjBlock + threadIdx.x;
  if (t >= a.t1) return;
  const int64_t ld = a.ld_out;
  State<float> s;
  load_state(a, t, s);
  unsigned st = 0u, iters[1] = {0u};
  int l = 0;
  for (; l < a.nlayer; ++l) {
    float* row = tape + (int64_t)l * kTapeRow * ld + t;
#pragma unroll
    for (int k = 0; k < 6; ++k) row[k * ld] = s.p[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) row[(6 + k) * ld] = s.c[k];
    row[27 * ld] = s.qf;
    float m[3], v[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) m[k] = __ldcs(a.hpos + (3 * l + k) * a.ld_hit + t);
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = __ldcs(a.hcov + (6 * l + k) * a.ld_hit + t);
    const float sf = a.geo.surf.s[l];
    const float dkdw = -s.qf * a.geo.kB;
    bool fail, nc = false;
    if (MODE == FIT_MODE_Z)
      fail = fitk::prop_z(s.p, s.c, s.g, dkdw, sf);
    else
      fail = fitk::prop_r(s.p, s.c, s.g, dkdw, sf, a.geo.max_iter, a.geo.tol * sf,
                          a.geo.line_start, iters, nc);
    if (fail) {
      st |= FIT_ST_NO_INTERSECTION;
      break;
    }
    if (nc) st |= FIT_ST_NOT_CONVERGED;
    const float phi_pred = s.p[4], th_pred = s.p[5];
    const float x2 = (MODE == FIT_MODE_Z) ? fitk::update_z(s.p, s.c, m, v) : fitk::update_r(s.p, s.c, m, v);
    if (fitk::normalise(s.p, s.c, s.qf, s.g, phi_pred, th_pred)) st |= FIT_ST_CHARGE_FLIP;
    row[28 * ld] = s.qf;
    if (!isfinite(x2)) {
      st |= FIT_ST_NONFINITE;
      break;
    }
    s.chi2 += x2;
    if (a.chi2_layer) a.chi2_layer[(int64_t)l * ld + t] = x2;
  }
  if (a.chi2_layer)
    for (int r = l; r < a.nlayer; ++r) a.chi2_layer[(int64_t)r * ld + t] = 0.f;
  ndone[t] = l;
  unsigned st1[1] = {st};
  store_state(a, t, s, st1);
  if (st1[0]) count_status(st1[0], a.counters);
}

template <int MODE>
__global__ void __launch_bounds__(kAdjBlock) fit_adjoint_kernel(const __grid_constant__ AdjArgs b) {
  const int64_t t = b.t0 + (int64_t)blockIdx.x * kAdjBlock + threadIdx.x;
  if (t >= b.t1) return;
  const int64_t ld = b.ld;
  const float wgt = b.grad_chi2[t];
  const int nl = b.ndone[t];
  float pb[6], cb[21];
#pragma unroll
  for (int k = 0; k < 6; ++k) pb[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 21; ++k) cb[k] = 0.f;
  for (int l = b.nlayer - 1; l >= nl; --l)
#pragma unroll
    for (int k = 0; k < 3; ++k) b.g_hpos[(3 * l + k) * ld + t] = 0.f;
  for (int l = nl - 1; l >= 0; --l) {
    const float* row = b.tape + (int64_t)l * kTapeRow * ld + t;
    float p[6], c[21], m[3], v[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k] = row[k * ld];
#pragma unroll
    for (int k = 0; k < 21; ++k) c[k] = row[(6 + k) * ld];
    const float qf = row[27 * ld];
#pragma unroll
    for (int k = 0; k < 3; ++k) m[k] = b.hpos[(3 * l + k) * ld + t];
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = b.hcov[(6 * l + k) * ld + t];
    // A charge flip in this layer's update (w < 0) negated w and row/column 3
    // of C: the same signs apply to their adjoints.
    if (row[28 * ld] != qf) {
      pb[3] = -pb[3];
#pragma unroll
      for (int i = 0; i < 6; ++i)
        if (i != 3) cb[fitk::sym(3, i)] = -cb[fitk::sym(3, i)];
    }
    const float sf = b.geo.surf.s[l];
    const float dkdw = -qf * b.geo.kB;
    // forward to the update's inputs
    float p1[6], c1[21];
#pragma unroll
    for (int k = 0; k < 6; ++k) p1[k] = p[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) c1[k] = c[k];
    fitk::Trig<float> g = fitk::trig_of(p1);
    unsigned iters[1] = {0u};
    bool nc = false;
    if (MODE == FIT_MODE_Z)
      fitk::prop_z(p1, c1, g, dkdw, sf);
    else
      fitk::prop_r(p1, c1, g, dkdw, sf, b.geo.max_iter, b.geo.tol * sf, b.geo.line_start, iters,
                   nc);
    float pb1[6], cb1[21], mb[3];
    if (MODE == FIT_MODE_Z)
      fitk::update_z_bwd(p1, c1, m, v, pb, cb, wgt, pb1, cb1, mb);
    else
      fitk::update_r_bwd(p1, c1, m, v, pb, cb, wgt, pb1, cb1, mb);
#pragma unroll
    for (int k = 0; k < 3; ++k) b.g_hpos[(3 * l + k) * ld + t] = mb[k];
    if (MODE == FIT_MODE_Z)
      fitk::prop_z_bwd(p, c, dkdw, sf, pb1, cb1, pb, cb);
    else
      fitk::prop_r_bwd(p, c, dkdw, sf, b.geo.max_iter, b.geo.tol * sf, b.geo.line_start, pb1, cb1,
                       pb, cb);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) b.g_par0[k * ld + t] = pb[k];
  if (b.g_cov0)
#pragma unroll
    for (int k = 0; k < 21; ++k) b.g_cov0[k * ld + t] = cb[k];
}

}  // namespace
}  // namespace fitimpl

using namespace fitimpl;

extern "C" {

size_t fit_tape_bytes(int nlayer, int64_t ld) {
  if (nlayer < 0 || ld < 0) return 0;
  return ((size_t)kTapeRow * (size_t)nlayer * (size_t)ld + (size_t)ld) * sizeof(float);
}

int fit_adjoint_forward(fit_handle* h, const fit_tracks_in* in, const fit_tracks_out* out,
                        const fit_hits* hits, int nevt, const int64_t* ntrk, int nlayer,
                        const int32_t* mode, void* tape, void* stream) {
  g_last_error.clear();
  if (!h) return fail(FIT_ERR_ARG, "fit_adjoint_forward: NULL argument");
  int64_t total = 0;
  int rc = check_call(h, in, out, hits, nevt, ntrk, nlayer, mode, &total, "fit_adjoint_forward");
  if (rc != FIT_OK || total == 0) return rc;
  if (!tape || !aligned16(tape)) return fail(FIT_ERR_ARG, "fit_adjoint_forward: tape NULL or misaligned");
  if (out->ld != hits->ld)
    return fail(FIT_ERR_ARG, "fit_adjoint_forward: outputs and hits must share ld");
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FitArgs a = base_args(in, out, hits, nlayer, h->d_counters);
  float* tp = static_cast<float*>(tape);
  int32_t* ndone = reinterpret_cast<int32_t*>(tp + (size_t)kTapeRow * nlayer * out->ld);
  int64_t t = 0;
  int e = 0;
  while (e < nevt) {
    const int m = mode[e];
    int64_t t1 = t;
    while (e < nevt && mode[e] == m) t1 += ntrk[e++];
    if (t1 > t) {
      a.t0 = t;
      a.t1 = t1;
      a.geo = h->geo[m];
      const unsigned nblk = (unsigned)((t1 - t + kAdjBlock - 1) / kAdjBlock);
      if (m == FIT_MODE_Z)
        fit_tape_kernel<FIT_MODE_Z><<<nblk, kAdjBlock, 0, s>>>(a, tp, ndone);
      else
        fit_tape_kernel<FIT_MODE_R><<<nblk, kAdjBlock, 0, s>>>(a, tp, ndone);
      cudaError_t err = cudaGetLastError();
      if (err != cudaSuccess) return cuda_fail(err, "fit_adjoint_forward: launch");
    }
    t = t1;
  }
  h->tracks += (uint64_t)total;
  return FIT_OK;
}

int fit_adjoint_backward(fit_handle* h, const fit_hits* hits, int nevt, const int64_t* ntrk,
                         int nlayer, const int32_t* mode, const void* tape, const float* grad_chi2,
                         float* grad_hpos, float* grad_par0, float* grad_cov0, void* stream) {
  g_last_error.clear();
  static const char* kWho = "fit_adjoint_backward";
  if (!h || !hits) return fail(FIT_ERR_ARG, std::string(kWho) + ": NULL argument");
  if (nevt < 0 || (nevt > 0 && (!ntrk || !mode)))
    return fail(FIT_ERR_ARG, std::string(kWho) + ": bad event arrays");
  int64_t total = 0;
  for (int e = 0; e < nevt; ++e) {
    if (ntrk[e] < 0 || (mode[e] != FIT_MODE_R && mode[e] != FIT_MODE_Z) || !h->has[mode[e]] ||
        h->nlayer[mode[e]] != nlayer)
      return fail(FIT_ERR_ARG, std::string(kWho) + ": bad event size, mode or nlayer");
    total += ntrk[e];
  }
  if (total == 0) return FIT_OK;
  const int64_t ld = hits->ld;
  if (ld < total || (ld & 3)) return fail(FIT_ERR_ARG, std::string(kWho) + ": bad ld");
  const void* ptrs[] = {hits->pos, hits->cov, tape, grad_chi2, grad_hpos, grad_par0};
  for (const void* p : ptrs)
    if (!p || !aligned16(p)) return fail(FIT_ERR_ARG, std::string(kWho) + ": NULL or misaligned pointer");
  if (grad_cov0 && !aligned16(grad_cov0))
    return fail(FIT_ERR_ARG, std::string(kWho) + ": grad_cov0 misaligned");
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  AdjArgs b{};
  b.hpos = hits->pos;
  b.hcov = hits->cov;
  b.ld = ld;
  b.tape = static_cast<const float*>(tape);
  b.ndone = reinterpret_cast<const int32_t*>(b.tape + (size_t)kTapeRow * nlayer * ld);
  b.grad_chi2 = grad_chi2;
  b.g_hpos = grad_hpos;
  b.g_par0 = grad_par0;
  b.g_cov0 = grad_cov0;
  b.nlayer = nlayer;
  int64_t t = 0;
  int e = 0;
  while (e < nevt) {
    const int m = mode[e];
    int64_t t1 = t;
    while (e < nevt && mode[e] == m) t1 += ntrk[e++];
    if (t1 > t) {
      b.t0 = t;
      b.t1 = t1;
      b.geo = h->geo[m];
      const unsigned nblk = (unsigned)((t1 - t + kAdjBlock - 1) / kAdjBlock);
      if (m == FIT_MODE_Z)
        fit_adjoint_kernel<FIT_MODE_Z><<<nblk, kAdjBlock, 0, s>>>(b);
      else
        fit_adjoint_kernel<FIT_MODE_R><<<nblk, kAdjBlock, 0, s>>>(b);
      cudaError_t err = cudaGetLastError();
      if (err != cudaSuccess) return cuda_fail(err, std::string(kWho + std::string(": launch")).c_str());
    }
    t = t1;
  }
  return FIT_OK;
}

}  // extern "C"
