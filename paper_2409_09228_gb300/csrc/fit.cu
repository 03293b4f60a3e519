// libfit: the fused propagate + Kalman-update kernels over runs of same-mode
// events, and the C ABI of fit.h (handle, fit_propagate_update,
// fit_propagate_update_noalloc, fit_sync).  The batched persistent form is in
// batch.cu.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>

#include "fit.h"
#include "fused.cuh"

namespace fitimpl {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(FIT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {

// 3 resident blocks per SM for p2r (156 registers, no spills; 2 blocks were
// 17 % slower); p2z fits 4 (128 registers, no spills).
template <int MODE, int L = 0>
__global__ void __launch_bounds__(kBlock, MODE == FIT_MODE_Z ? 4 : 3)
    fit_fused_kernel(const __grid_constant__ FitArgs a) {
  const int64_t t = pair_track(a);
  if (t >= a.t1) return;
  unsigned st[2] = {0u, 0u}, iters[2] = {0u, 0u};
  run_pair<MODE, L, MODE == FIT_MODE_Z && L == 0>(a, a.geo, a.t0, a.t1, t, st, iters);
  if (st[0]) count_status(st[0], a.counters);
  if (st[1]) count_status(st[1], a.counters);
  if (MODE == FIT_MODE_R) count_iterations(iters[0] + iters[1], &a.counters[4]);
}

template <int MODE>
__global__ void __launch_bounds__(kBlock, MODE == FIT_MODE_Z ? 4 : 3)
    fit_fused_kernel_noalloc(const __grid_constant__ FitArgs a, const int64_t* __restrict__ evt_off,
                             int e0, int e1) {
  const int64_t t = pair_track(a);
  if (t >= a.t1) return;
  unsigned st[2] = {0u, 0u}, iters[2] = {0u, 0u};
  run_pair<MODE>(a, a.geo, a.t0, a.t1, t, st, iters);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    if (t + i < a.t0 || t + i >= a.t1) continue;
    unsigned long long* cnt = a.counters + (int64_t)event_of(t + i, evt_off, e0, e1) * kEventSlots + 1;
    if (st[i]) count_status(st[i], cnt);
    if (MODE == FIT_MODE_R && iters[i]) atomicAdd(&cnt[4], (unsigned long long)iters[i]);
  }
}


}  // namespace

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
      h->geo[m].surf.s[l] = c->surf[l];
    }
    h->has[m] = true;
    h->nlayer[m] = c->nlayer;
    h->geo[m].kB = fitk::kA * c->B;
    h->B[m] = c->B;
    h->geo[m].max_iter = c->max_iter > 0 ? c->max_iter : 10;
    h->geo[m].tol = c->tol > 0.f ? c->tol : 1e-6f;
    if (c->start != FIT_START_CROSSING && c->start != FIT_START_LINE)
      return fail(FIT_ERR_ARG, std::string(who) + ": start is not a FIT_START_* value");
    h->geo[m].line_start = c->start == FIT_START_LINE;
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
      a.geo = h->geo[m];
      const int64_t npairs = (t1 - (t & ~int64_t(1)) + 1) / 2;  // two tracks per thread
      const int64_t nblk = (npairs + kBlock - 1) / kBlock;
      if (nblk > 0x7fffffff) return fail(FIT_ERR_ARG, std::string(who) + ": too many tracks");
      launch(a, m, (unsigned)nblk, e0, e);
      cudaError_t err = cudaGetLastError();
      if (err != cudaSuccess) return cuda_fail(err, (std::string(who) + ": launch").c_str());
    }
    t = t1;
  }
  return FIT_OK;
}

// The fused fit of events [0, nevt) on the tracks of a (a.t0, a.t1 set per
// run of same-mode events): the p2r runs on stream s, the p2z runs on sz.
int run_fit(const fit_handle* h, const FitArgs& a, int nevt, const int64_t* ntrk,
            const int32_t* mode, const char* who, cudaStream_t s, cudaStream_t sz) {
  return launch_segments(h, a, nevt, ntrk, mode, who,
                         [s, sz, h](const FitArgs& a1, int m, unsigned nblk, int, int) {
                           if (m == FIT_MODE_Z)
                             fit_fused_kernel<FIT_MODE_Z><<<nblk, kBlock, 0, sz>>>(a1);
                           else if (h->seeded)
                             launch_seeded_fit(a1, h->d_mlp, s);
                           else
                             fit_fused_kernel<FIT_MODE_R><<<nblk, kBlock, 0, s>>>(a1);
                         });
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

}  // namespace fitimpl

using namespace fitimpl;

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
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (h->join) cudaEventDestroy(h->join);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->side) cudaStreamDestroy(h->side);
    cudaFree(h->d_counters);
    delete h;
    return cuda_fail(e, "fit_init: counters, stream and events");
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
  static const char* kWho = "fit_propagate_update";
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const FitArgs a = base_args(in, out, hits, nlayer, h->d_counters);
  bool used[2] = {false, false};
  for (int e = 0; e < nevt; ++e)
    if (ntrk[e] > 0) used[mode[e] == FIT_MODE_Z] = true;
  if (!(used[0] && used[1])) {
    rc = run_fit(h, a, nevt, ntrk, mode, kWho, s, s);
  } else {
    // The two modes' events are independent: the p2z launches go to the
    // handle's second stream, so that they overlap the p2r launches (their
    // blocks fill the SMs a launch's last wave leaves idle).  The join is
    // recorded even after a failed launch, so that the caller's stream
    // still follows everything that was queued.
    std::lock_guard<std::mutex> lock(h->side_mu);
    cudaError_t e = cudaEventRecord(h->fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "fit_propagate_update: fork to the second stream");
    rc = run_fit(h, a, nevt, ntrk, mode, kWho, s, h->side);
    e = cudaEventRecord(h->join, h->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->join, 0);
    if (e != cudaSuccess && rc == FIT_OK)
      return cuda_fail(e, "fit_propagate_update: join from the second stream");
  }
  if (rc != FIT_OK) return rc;
  h->tracks += (uint64_t)total;
  return FIT_OK;
}

int fit_propagate_update_layout(fit_handle* h, const fit_tracks_in* in, const fit_tracks_out* out,
                                const fit_hits* hits, int nevt, const int64_t* ntrk, int nlayer,
                                const int32_t* mode, int layout, void* stream) {
  static const char* kWho = "fit_propagate_update_layout";
  g_last_error.clear();
  if (!h) return fail(FIT_ERR_ARG, std::string(kWho) + ": NULL argument");
  if (layout == FIT_LAYOUT_SOA)
    return fit_propagate_update(h, in, out, hits, nevt, ntrk, nlayer, mode, stream);
  if (layout != FIT_LAYOUT_AOSOA32) return fail(FIT_ERR_ARG, std::string(kWho) + ": unknown layout");
  int64_t total = 0;
  int rc = check_call(h, in, out, hits, nevt, ntrk, nlayer, mode, &total, kWho);
  if (rc != FIT_OK || total == 0) return rc;
  if ((in->ld | out->ld | hits->ld) & 31)
    return fail(FIT_ERR_ARG, std::string(kWho) + ": AoSoA slots (ld) must be a multiple of 32");
  if (h->seeded) return fail(FIT_ERR_ARG, std::string(kWho) + ": no learned seed in AoSoA");
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = launch_segments(h, base_args(in, out, hits, nlayer, h->d_counters), nevt, ntrk, mode, kWho,
                       [s](const FitArgs& a, int m, unsigned nblk, int, int) {
                         if (m == FIT_MODE_Z)
                           fit_fused_kernel<FIT_MODE_Z, 1><<<nblk, kBlock, 0, s>>>(a);
                         else
                           fit_fused_kernel<FIT_MODE_R, 1><<<nblk, kBlock, 0, s>>>(a);
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
    if (h->d_counters || h->d_mlp || h->host_stage) cudaDeviceSynchronize();
    if (h->d_counters) cudaFree(h->d_counters);
    if (h->d_mlp) cudaFree(h->d_mlp);
    if (h->join) cudaEventDestroy(h->join);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->side) cudaStreamDestroy(h->side);
    destroy_host_stage(h);
  }
  delete h;
}

}  // extern "C"
