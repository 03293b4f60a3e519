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
#include <mutex>
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

// The fused per-track layer loop for track t.  MODE selects the surface type
// at compile time (no divergence between cylinder and plane code within a
// launch).  Returns the track's status bits and its p2r path-length
// iteration count.
template <int MODE>
__device__ __forceinline__ void run_track(const FitArgs& a, int64_t t, unsigned& st_out,
                                          unsigned& iters_out) {
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
  st_out = st;
  iters_out = iters;
}

__device__ __forceinline__ void count_iterations(unsigned iters, unsigned long long* counter) {
  const unsigned mask = __activemask();
  const unsigned warp_iters = __reduce_add_sync(mask, iters);
  if ((int)(threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(counter, (unsigned long long)warp_iters);
}

template <int MODE>
__global__ void __launch_bounds__(kBlock) fit_fused_kernel(const __grid_constant__ FitArgs a) {
  const int64_t t = a.t0 + (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (t >= a.t1) return;
  unsigned st, iters;
  run_track<MODE>(a, t, st, iters);
  if (st) count_status(st, a.counters);
  if (MODE == FIT_MODE_R) count_iterations(iters, &a.counters[4]);
}

// Variant for fit_propagate_update_noalloc: the same per-track work, with the
// counters kept per event.  a.counters points at a [nevt][kEventSlots] table
// (slot 0, the track count, is filled on the host); evt_off holds the first
// track of events e0..e1 (and the end of e1 - 1), so a track finds its event
// by binary search.
constexpr int kEventSlots = 6;

template <int MODE>
__global__ void __launch_bounds__(kBlock)
    fit_fused_kernel_noalloc(const __grid_constant__ FitArgs a, const int64_t* __restrict__ evt_off,
                             int e0, int e1) {
  const int64_t t = a.t0 + (int64_t)blockIdx.x * kBlock + threadIdx.x;
  if (t >= a.t1) return;
  unsigned st, iters;
  run_track<MODE>(a, t, st, iters);
  int lo = e0, hi = e1 - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (evt_off[mid] <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  unsigned long long* cnt = a.counters + (int64_t)lo * kEventSlots + 1;
  if (st) count_status(st, cnt);
  if (MODE == FIT_MODE_R) {
    const unsigned mask = __activemask();
    const int first = __shfl_sync(mask, lo, __ffs(mask) - 1);
    if (__all_sync(mask, lo == first))
      count_iterations(iters, &cnt[4]);
    else
      atomicAdd(&cnt[4], (unsigned long long)iters);
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

namespace {

// Copies the two modes' geometry and numerics into h (no allocation).
int configure_modes(fit_handle* h, const fit_config* cfg_r, const fit_config* cfg_z,
                    const char* who) {
  const fit_config* cfgs[2] = {cfg_r, cfg_z};
  for (int m = 0; m < 2; ++m) {
    const fit_config* c = cfgs[m];
    if (!c) continue;
    if (c->nlayer < 1 || c->nlayer > FIT_MAX_LAYERS || !c->surf)
      return fail(FIT_ERR_ARG, std::string(who) + ": nlayer out of range or surf is NULL");
    for (int l = 0; l < c->nlayer; ++l) {
      if (!(c->surf[l] == c->surf[l]) || (m == FIT_MODE_R && !(c->surf[l] > 0.f)))
        return fail(FIT_ERR_ARG, std::string(who) + ": invalid surface position");
      h->surf[m].s[l] = c->surf[l];
    }
    h->has[m] = true;
    h->nlayer[m] = c->nlayer;
    h->kB[m] = fitk::kA * c->B;
    h->max_iter[m] = c->max_iter > 0 ? c->max_iter : 10;
    h->tol[m] = c->tol > 0.f ? c->tol : 1e-6f;
  }
  return FIT_OK;
}

// Argument checks shared by the entry points that run the fused kernel.
int check_call(const fit_handle* h, const fit_tracks_in* in, const fit_tracks_out* out,
               const fit_hits* hits, int nevt, const int64_t* ntrk, int nlayer,
               const int32_t* mode, int64_t* total_out, const char* who) {
  const std::string w(who);
  if (!in || !out || !hits) return fail(FIT_ERR_ARG, w + ": NULL argument");
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
  *total_out = total;
  if (total == 0) return FIT_OK;
  if (nlayer < 1 || nlayer > FIT_MAX_LAYERS) return fail(FIT_ERR_ARG, w + ": nlayer out of range");
  if (!in->par || !in->cov || !in->q || !out->par || !out->cov || !out->q || !out->chi2 ||
      !hits->pos || !hits->cov)
    return fail(FIT_ERR_ARG, w + ": NULL data pointer");
  const void* ptrs[] = {in->par, in->cov, in->q, out->par, out->cov, out->q, out->chi2,
                        hits->pos, hits->cov};
  for (const void* p : ptrs)
    if (!aligned16(p)) return fail(FIT_ERR_ARG, w + ": pointer not 16-byte aligned");
  if (in->ld < total || out->ld < total || hits->ld < total)
    return fail(FIT_ERR_ARG, w + ": ld smaller than the number of tracks");
  if ((in->ld | out->ld | hits->ld) & 3) return fail(FIT_ERR_ARG, w + ": ld not a multiple of 4");
  return FIT_OK;
}

FitArgs base_args(const fit_tracks_in* in, const fit_tracks_out* out, const fit_hits* hits,
                  int nlayer, unsigned long long* counters) {
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
  a.counters = counters;
  return a;
}

// Runs consecutive events of one mode as one launch each.  launch(a, m, nblk,
// e0, e1) issues the kernel for tracks [a.t0, a.t1) = events [e0, e1).
template <class Launch>
int launch_segments(const fit_handle* h, FitArgs a, int nevt, const int64_t* ntrk,
                    const int32_t* mode, const char* who, Launch launch) {
  int64_t t = 0;
  int e = 0;
  while (e < nevt) {
    const int m = mode[e];
    const int e0 = e;
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
      if (nblk > 0x7fffffff) return fail(FIT_ERR_ARG, std::string(who) + ": too many tracks");
      launch(a, m, (unsigned)nblk, e0, e);
      cudaError_t err = cudaGetLastError();
      if (err != cudaSuccess) return cuda_fail(err, (std::string(who) + ": launch").c_str());
    }
    t = t1;
  }
  return FIT_OK;
}

// Scratch of fit_propagate_update_noalloc, in the library image instead of
// allocated memory: per-event counters [FIT_NOALLOC_MAX_EVENTS][kEventSlots]
// followed by the event offsets [FIT_NOALLOC_MAX_EVENTS + 1] (int64).  Every
// device that loads the library holds it (192 KiB) until the process exits.
constexpr size_t kNoallocCounterWords = (size_t)FIT_NOALLOC_MAX_EVENTS * kEventSlots;
static __device__ __align__(256)
    unsigned long long g_noalloc_scratch[kNoallocCounterWords + FIT_NOALLOC_MAX_EVENTS + 1];

// Device address of g_noalloc_scratch per device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device, with that device current, and cached.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned long long* g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(int device, unsigned long long** ptr) {
  if (device < 0 || device >= kMaxDevices)
    return fail(FIT_ERR_ARG, "fit_propagate_update_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "fit_propagate_update_noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[device] = static_cast<unsigned long long*>(p);
  }
  *ptr = g_noalloc_ptr[device];
  return FIT_OK;
}

}  // namespace

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
  int rc = configure_modes(h, cfg_r, cfg_z, "fit_init");
  if (rc != FIT_OK) {
    delete h;
    return rc;
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
  if (!h) return fail(FIT_ERR_ARG, "fit_propagate_update: NULL argument");
  int64_t total = 0;
  int rc = check_call(h, in, out, hits, nevt, ntrk, nlayer, mode, &total, "fit_propagate_update");
  if (rc != FIT_OK || total == 0) return rc;
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = launch_segments(h, base_args(in, out, hits, nlayer, h->d_counters), nevt, ntrk, mode,
                       "fit_propagate_update",
                       [s](const FitArgs& a, int m, unsigned nblk, int, int) {
                         if (m == FIT_MODE_Z)
                           fit_fused_kernel<FIT_MODE_Z><<<nblk, kBlock, 0, s>>>(a);
                         else
                           fit_fused_kernel<FIT_MODE_R><<<nblk, kBlock, 0, s>>>(a);
                       });
  if (rc != FIT_OK) return rc;
  h->tracks += (uint64_t)total;
  return FIT_OK;
}

int fit_propagate_update_noalloc(const fit_config* cfg_r, const fit_config* cfg_z,
                                 const fit_tracks_in* in, const fit_tracks_out* out,
                                 const fit_hits* hits, int nevt, const int64_t* ntrk, int nlayer,
                                 const int32_t* mode, void* stream, fit_status* per_event) {
  static const char* kWho = "fit_propagate_update_noalloc";
  g_last_error.clear();
  if (!cfg_r && !cfg_z) return fail(FIT_ERR_ARG, std::string(kWho) + ": no mode configured");
  if (nevt > FIT_NOALLOC_MAX_EVENTS)
    return fail(FIT_ERR_ARG, std::string(kWho) + ": nevt exceeds FIT_NOALLOC_MAX_EVENTS (" +
                                 std::to_string(FIT_NOALLOC_MAX_EVENTS) +
                                 "); split the events over several calls");
  fit_handle h;  // geometry only; nothing allocated
  int rc = configure_modes(&h, cfg_r, cfg_z, kWho);
  if (rc != FIT_OK) return rc;
  int64_t total = 0;
  rc = check_call(&h, in, out, hits, nevt, ntrk, nlayer, mode, &total, kWho);
  if (rc != FIT_OK) return rc;
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_fail(e, "fit_propagate_update_noalloc: cudaGetDevice");
  unsigned long long* scratch = nullptr;
  rc = noalloc_scratch(device, &scratch);
  if (rc != FIT_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (nevt > 0) {
    // The counters of this call's events start at zero; the event offsets
    // are staged from the stack.
    int64_t off[FIT_NOALLOC_MAX_EVENTS + 1];
    off[0] = 0;
    for (int i = 0; i < nevt; ++i) off[i + 1] = off[i] + ntrk[i];
    int64_t* d_off = reinterpret_cast<int64_t*>(scratch + kNoallocCounterWords);
    e = cudaMemsetAsync(scratch, 0, (size_t)nevt * kEventSlots * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "fit_propagate_update_noalloc: cudaMemsetAsync");
    e = cudaMemcpyAsync(d_off, off, (size_t)(nevt + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "fit_propagate_update_noalloc: offset copy");
    if (total > 0) {
      rc = launch_segments(&h, base_args(in, out, hits, nlayer, scratch), nevt, ntrk, mode, kWho,
                           [s, d_off](const FitArgs& a, int m, unsigned nblk, int e0, int e1) {
                             if (m == FIT_MODE_Z)
                               fit_fused_kernel_noalloc<FIT_MODE_Z>
                                   <<<nblk, kBlock, 0, s>>>(a, d_off, e0, e1);
                             else
                               fit_fused_kernel_noalloc<FIT_MODE_R>
                                   <<<nblk, kBlock, 0, s>>>(a, d_off, e0, e1);
                           });
      if (rc != FIT_OK) return rc;
    }
  }
  if (per_event && nevt > 0) {
    static_assert(sizeof(fit_status) == kEventSlots * sizeof(unsigned long long),
                  "fit_status mirrors one row of the per-event counter table");
    e = cudaMemcpyAsync(per_event, scratch, (size_t)nevt * sizeof(fit_status),
                        cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "fit_propagate_update_noalloc: counter copy");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "fit_propagate_update_noalloc: cudaStreamSynchronize");
    for (int i = 0; i < nevt; ++i) per_event[i].tracks = (uint64_t)ntrk[i];
  }
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
