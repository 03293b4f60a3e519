// libfit: the fused propagate + Kalman-update kernels and the C ABI of fit.h.
//
// One thread owns one track for all layers (paper Sec. 3.1: propagation and
// update in one kernel; Sec. 4.2: per-track intermediates kept in registers).
// Track state and covariance are loaded once, stay in registers through every
// layer, and are stored once.  The hits of layer l+1 are loaded while layer l
// is computed; consecutive threads read consecutive words of each hit
// component (structure of arrays, track index fastest), so every load of a
// warp is one 128-byte line.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>

#include "fit.h"
#include "track_math.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(FIT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr int kBlock = 128;
constexpr int kCounters = 5;  // no_intersection, not_converged, nonfinite, charge_flip,
                               // p2r path-length iterations

struct Surfaces {
  float s[FIT_MAX_LAYERS];
};

struct FitArgs {
  const float* par_in;
  const float* cov_in;
  const int32_t* q_in;
  int64_t ld_in;
  float* par_out;
  float* cov_out;
  int32_t* q_out;
  float* chi2;
  float* chi2_layer;
  uint8_t* status;
  int64_t ld_out;
  const float* hpos;
  const float* hcov;
  int64_t ld_hit;
  int64_t t0, t1;  // track range [t0, t1)
  int nlayer;
  float kB;        // kA * B
  int max_iter;
  float tol;
  unsigned long long* counters;
  Surfaces surf;
};

__device__ __forceinline__ void count_status(unsigned st, unsigned long long* counters) {
  if (st & FIT_ST_NO_INTERSECTION) atomicAdd(&counters[0], 1ull);
  if (st & FIT_ST_NOT_CONVERGED) atomicAdd(&counters[1], 1ull);
  if (st & FIT_ST_NONFINITE) atomicAdd(&counters[2], 1ull);
  if (st & FIT_ST_CHARGE_FLIP) atomicAdd(&counters[3], 1ull);
}

// The fused per-track layer loop.  MODE selects the surface type at compile
// time (no divergence between cylinder and plane code within a launch).
template <int MODE>
__global__ void __launch_bounds__(kBlock) fit_fused_kernel(const __grid_constant__ FitArgs a) {
  const int64_t t = a.t0 + (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (t >= a.t1) return;

  float p[6], c[21];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = __ldcs(a.par_in + k * a.ld_in + t);
#pragma unroll
  for (int k = 0; k < 21; ++k) c[k] = __ldcs(a.cov_in + k * a.ld_in + t);
  int q = __ldcs(a.q_in + t);
  float dkdw = -(float)q * a.kB;

  const float* hp = a.hpos + t;
  const float* hc = a.hcov + t;
  const int64_t ldh = a.ld_hit;
  float m[3], v[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) m[k] = __ldcs(hp + k * ldh);
#pragma unroll
  for (int k = 0; k < 6; ++k) v[k] = __ldcs(hc + k * ldh);

  float chi2 = 0.f;
  unsigned st = 0u;
  unsigned iters = 0u;
  int l = 0;
  for (; l < a.nlayer; ++l) {
    // Prefetch the next layer's hit while this one is processed.
    float mn[3], vn[6];
    const int ln = (l + 1 < a.nlayer) ? l + 1 : l;
#pragma unroll
    for (int k = 0; k < 3; ++k) mn[k] = __ldcs(hp + (3 * ln + k) * ldh);
#pragma unroll
    for (int k = 0; k < 6; ++k) vn[k] = __ldcs(hc + (6 * ln + k) * ldh);

    const float s = a.surf.s[l];
    unsigned sp;
    if (MODE == FIT_MODE_Z)
      sp = fitk::prop_z(p, c, dkdw, s);
    else
      sp = fitk::prop_r(p, c, dkdw, s, a.max_iter, a.tol * s, iters);
    st |= sp;
    if (sp & FIT_ST_NO_INTERSECTION) break;
    const float x2 = (MODE == FIT_MODE_Z) ? fitk::update_z(p, c, m, v) : fitk::update_r(p, c, m, v);
    const unsigned flip = fitk::normalise(p, c, q);
    if (flip) {
      st |= flip;
      dkdw = -(float)q * a.kB;
    }
    if (!isfinite(x2)) {
      st |= FIT_ST_NONFINITE;
      break;
    }
    chi2 += x2;
    if (a.chi2_layer) a.chi2_layer[(int64_t)l * a.ld_out + t] = x2;
#pragma unroll
    for (int k = 0; k < 3; ++k) m[k] = mn[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = vn[k];
  }
  if (a.chi2_layer)
    for (int r = (l < a.nlayer) ? l : a.nlayer; r < a.nlayer; ++r)
      a.chi2_layer[(int64_t)r * a.ld_out + t] = 0.f;

  bool finite = isfinite(chi2);
#pragma unroll
  for (int k = 0; k < 6; ++k) finite = finite && isfinite(p[k]);
#pragma unroll
  for (int k = 0; k < 21; ++k) finite = finite && isfinite(c[k]);
  if (!finite) st |= FIT_ST_NONFINITE;

#pragma unroll
  for (int k = 0; k < 6; ++k) a.par_out[k * a.ld_out + t] = p[k];
#pragma unroll
  for (int k = 0; k < 21; ++k) a.cov_out[k * a.ld_out + t] = c[k];
  a.q_out[t] = q;
  a.chi2[t] = chi2;
  if (a.status) a.status[t] = (uint8_t)st;
  if (st) count_status(st, a.counters);
  if (MODE == FIT_MODE_R) {
    const unsigned mask = __activemask();
    const unsigned warp_iters = __reduce_add_sync(mask, iters);
    if ((int)(threadIdx.x & 31) == __ffs(mask) - 1)
      atomicAdd(&a.counters[4], (unsigned long long)warp_iters);
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() { cudaSetDevice(prev_); }

 private:
  int prev_ = 0;
};

}  // namespace

struct fit_handle {
  int device = 0;
  bool has[2] = {false, false};
  int nlayer[2] = {0, 0};
  float kB[2] = {0.f, 0.f};
  int max_iter[2] = {10, 10};
  float tol[2] = {1e-6f, 1e-6f};
  Surfaces surf[2];
  unsigned long long* d_counters = nullptr;  // [kCounters]
  uint64_t tracks = 0;
};

extern "C" {

const char* fit_last_error(void) { return g_last_error.c_str(); }

int fit_init(fit_handle** out, const fit_config* cfg_r, const fit_config* cfg_z, int device) {
  g_last_error.clear();
  if (!out) return fail(FIT_ERR_ARG, "fit_init: handle pointer is NULL");
  *out = nullptr;
  if (!cfg_r && !cfg_z) return fail(FIT_ERR_ARG, "fit_init: no mode configured");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "fit_init: cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(FIT_ERR_ARG, "fit_init: no such device");
  fit_handle* h = new fit_handle();
  h->device = device;
  const fit_config* cfgs[2] = {cfg_r, cfg_z};
  for (int m = 0; m < 2; ++m) {
    const fit_config* c = cfgs[m];
    if (!c) continue;
    if (c->nlayer < 1 || c->nlayer > FIT_MAX_LAYERS || !c->surf) {
      delete h;
      return fail(FIT_ERR_ARG, "fit_init: nlayer out of range or surf is NULL");
    }
    for (int l = 0; l < c->nlayer; ++l) {
      if (!(c->surf[l] == c->surf[l]) || (m == FIT_MODE_R && !(c->surf[l] > 0.f))) {
        delete h;
        return fail(FIT_ERR_ARG, "fit_init: invalid surface position");
      }
      h->surf[m].s[l] = c->surf[l];
    }
    h->has[m] = true;
    h->nlayer[m] = c->nlayer;
    h->kB[m] = fitk::kA * c->B;
    h->max_iter[m] = c->max_iter > 0 ? c->max_iter : 10;
    h->tol[m] = c->tol > 0.f ? c->tol : 1e-6f;
  }
  DeviceGuard g(device);
  e = cudaMalloc(&h->d_counters, kCounters * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    delete h;
    return fail(FIT_ERR_NOMEM, std::string("fit_init: cudaMalloc: ") + cudaGetErrorString(e));
  }
  e = cudaMemset(h->d_counters, 0, kCounters * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaFree(h->d_counters);
    delete h;
    return cuda_fail(e, "fit_init: cudaMemset");
  }
  *out = h;
  return FIT_OK;
}

int fit_propagate_update(fit_handle* h, const fit_tracks_in* in, const fit_tracks_out* out,
                         const fit_hits* hits, int nevt, const int64_t* ntrk, int nlayer,
                         const int32_t* mode, void* stream) {
  g_last_error.clear();
  if (!h || !in || !out || !hits) return fail(FIT_ERR_ARG, "fit_propagate_update: NULL argument");
  if (nevt < 0) return fail(FIT_ERR_ARG, "fit_propagate_update: nevt < 0");
  if (nevt > 0 && (!ntrk || !mode))
    return fail(FIT_ERR_ARG, "fit_propagate_update: ntrk or mode is NULL");
  int64_t total = 0;
  for (int e = 0; e < nevt; ++e) {
    if (ntrk[e] < 0) return fail(FIT_ERR_ARG, "fit_propagate_update: ntrk[e] < 0");
    if (mode[e] != FIT_MODE_R && mode[e] != FIT_MODE_Z)
      return fail(FIT_ERR_ARG, "fit_propagate_update: mode[e] is not FIT_MODE_R or FIT_MODE_Z");
    if (!h->has[mode[e]]) return fail(FIT_ERR_ARG, "fit_propagate_update: mode not configured");
    if (h->nlayer[mode[e]] != nlayer)
      return fail(FIT_ERR_ARG, "fit_propagate_update: nlayer differs from the configured one");
    total += ntrk[e];
  }
  if (total == 0) return FIT_OK;
  if (nlayer < 1 || nlayer > FIT_MAX_LAYERS)
    return fail(FIT_ERR_ARG, "fit_propagate_update: nlayer out of range");
  if (!in->par || !in->cov || !in->q || !out->par || !out->cov || !out->q || !out->chi2 ||
      !hits->pos || !hits->cov)
    return fail(FIT_ERR_ARG, "fit_propagate_update: NULL data pointer");
  const void* ptrs[] = {in->par, in->cov, in->q, out->par, out->cov, out->q, out->chi2,
                        hits->pos, hits->cov};
  for (const void* p : ptrs)
    if (!aligned16(p)) return fail(FIT_ERR_ARG, "fit_propagate_update: pointer not 16-byte aligned");
  if (in->ld < total || out->ld < total || hits->ld < total)
    return fail(FIT_ERR_ARG, "fit_propagate_update: ld smaller than the number of tracks");
  if ((in->ld | out->ld | hits->ld) & 3)
    return fail(FIT_ERR_ARG, "fit_propagate_update: ld not a multiple of 4");

  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FitArgs a{};
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
  // Consecutive events of one mode form one launch.
  int64_t t = 0;
  int e = 0;
  while (e < nevt) {
    const int m = mode[e];
    int64_t t1 = t;
    while (e < nevt && mode[e] == m) t1 += ntrk[e++];
    if (t1 > t) {
      a.t0 = t;
      a.t1 = t1;
      a.kB = h->kB[m];
      a.max_iter = h->max_iter[m];
      a.tol = h->tol[m];
      a.surf = h->surf[m];
      const int64_t nblk = (t1 - t + kBlock - 1) / kBlock;
      if (nblk > 0x7fffffff) return fail(FIT_ERR_ARG, "fit_propagate_update: too many tracks");
      if (m == FIT_MODE_Z)
        fit_fused_kernel<FIT_MODE_Z><<<(unsigned)nblk, kBlock, 0, s>>>(a);
      else
        fit_fused_kernel<FIT_MODE_R><<<(unsigned)nblk, kBlock, 0, s>>>(a);
      cudaError_t err = cudaGetLastError();
      if (err != cudaSuccess) return cuda_fail(err, "fit_propagate_update: launch");
    }
    t = t1;
  }
  h->tracks += (uint64_t)total;
  return FIT_OK;
}

int fit_sync(fit_handle* h, void* stream, double timeout_s, fit_status* st) {
  g_last_error.clear();
  if (!h) return fail(FIT_ERR_ARG, "fit_sync: handle is NULL");
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (timeout_s > 0) {
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
      cudaError_t q = cudaStreamQuery(s);
      if (q == cudaSuccess) break;
      if (q != cudaErrorNotReady) return cuda_fail(q, "fit_sync: cudaStreamQuery");
      if (std::chrono::steady_clock::now() > deadline)
        return fail(FIT_ERR_TIMEOUT, "fit_sync: timed out waiting for the stream");
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
  unsigned long long c[kCounters] = {0, 0, 0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(c, h->d_counters, sizeof(c), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "fit_sync: counter copy");
  e = cudaMemsetAsync(h->d_counters, 0, sizeof(c), s);
  if (e != cudaSuccess) return cuda_fail(e, "fit_sync: counter reset");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "fit_sync: cudaStreamSynchronize");
  if (st) {
    st->tracks = h->tracks;
    st->no_intersection = c[0];
    st->not_converged = c[1];
    st->nonfinite = c[2];
    st->charge_flip = c[3];
    st->iterations = c[4];
  }
  h->tracks = 0;
  return FIT_OK;
}

void fit_destroy(fit_handle* h) {
  if (!h) return;
  {
    DeviceGuard g(h->device);
    if (h->d_counters) {
      cudaDeviceSynchronize();
      cudaFree(h->d_counters);
    }
  }
  delete h;
}

}  // extern "C"
