// fit_propagate_update_host: the fused fit on HOST buffers.  The tracks are
// cut into chunks of at most kChunk; chunk i goes through device staging set
// i % kSets on internal stream i % kSets -- host-to-device copies, the fused
// kernels, device-to-host copies -- so the copies of one chunk overlap the fit
// and copies of the others (paper Sec. 3.1: inputs are copied to the device
// before the kernel and results back after it).  The caller's stream orders
// the whole call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "fit.h"
#include "internal.h"

using namespace fitimpl;

namespace {

constexpr int64_t kChunk = FIT_HOST_CHUNK;  // tracks per chunk (a multiple of 4)
static_assert(kChunk % 4 == 0, "chunks start at multiples of 4 tracks");
// Staging sets and streams.  On GB300 the host link moves ~211 GB/s H2D
// whatever the number of streams, but 2-D copies lose bandwidth with narrow
// rows (~0.3 us per row): 65536-, 131072- and 262144-track chunks move
// 144, 186 and 207 GB/s.  Measured end to end (bench step, both modes):
// 262144 tracks with 3 sets 8.14 ms, against 9.29 ms with 131072; larger
// chunks or a fourth set change nothing.
constexpr int kSets = 3;

struct HostStage {
  int64_t cap = 0;  // tracks per staging set
  int nlayer = 0;
  char* buf[kSets] = {};
  cudaStream_t st[kSets] = {};
  cudaEvent_t ev_start = nullptr, ev_done[kSets] = {};
};

// Staging set layout: par [6][cap], cov [21][cap], q [cap], chi2 [cap],
// hpos [3 nlayer][cap], hcov [6 nlayer][cap], chi2_layer [nlayer][cap] (all
// 4-byte elements), status [cap] bytes.  cap is a multiple of 4, so every row
// starts on a 16-byte boundary.
struct Set {
  float *par, *cov, *chi2, *hpos, *hcov, *chi2_layer;
  int32_t* q;
  uint8_t* status;
};

size_t set_bytes(int64_t cap, int nlayer) {
  return (size_t)cap * 4 * (6 + 21 + 1 + 1 + 9 * (size_t)nlayer + nlayer) + (size_t)cap;
}

Set carve(char* b, int64_t cap, int nlayer) {
  Set s;
  float* f = reinterpret_cast<float*>(b);
  s.par = f;
  s.cov = s.par + 6 * cap;
  s.q = reinterpret_cast<int32_t*>(s.cov + 21 * cap);
  s.chi2 = reinterpret_cast<float*>(s.q + cap);
  s.hpos = s.chi2 + cap;
  s.hcov = s.hpos + (int64_t)3 * nlayer * cap;
  s.chi2_layer = s.hcov + (int64_t)6 * nlayer * cap;
  s.status = reinterpret_cast<uint8_t*>(s.chi2_layer + (int64_t)nlayer * cap);
  return s;
}

void free_stage(HostStage* hs) {
  for (int i = 0; i < kSets; ++i) {
    if (hs->buf[i]) cudaFree(hs->buf[i]);
    if (hs->st[i]) cudaStreamDestroy(hs->st[i]);
    if (hs->ev_done[i]) cudaEventDestroy(hs->ev_done[i]);
  }
  if (hs->ev_start) cudaEventDestroy(hs->ev_start);
  delete hs;
}

// The handle's staging, (re)allocated for cap tracks and nlayer layers.
int stage_for(fit_handle* h, int64_t cap, int nlayer, HostStage** out) {
  HostStage* hs = static_cast<HostStage*>(h->host_stage);
  if (hs && hs->cap >= cap && hs->nlayer >= nlayer) {
    *out = hs;
    return FIT_OK;
  }
  if (hs) {
    cudaDeviceSynchronize();
    free_stage(hs);
    h->host_stage = nullptr;
  }
  hs = new HostStage();
  hs->cap = cap;
  hs->nlayer = nlayer;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < kSets && e == cudaSuccess; ++i) {
    e = cudaMalloc(&hs->buf[i], set_bytes(cap, nlayer));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hs->st[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hs->ev_done[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hs->ev_start, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_stage(hs);
    return fail(FIT_ERR_NOMEM, std::string("fit_propagate_update_host: staging: ") +
                                   cudaGetErrorString(e));
  }
  h->host_stage = hs;
  *out = hs;
  return FIT_OK;
}

// rows x width bytes between a host array of pitch hp and a staging array of
// pitch sp.
cudaError_t copy_rows(void* dst, size_t dp, const void* src, size_t sp, size_t width, size_t rows,
                      cudaMemcpyKind kind, cudaStream_t s) {
  return cudaMemcpy2DAsync(dst, dp, src, sp, width, rows, kind, s);
}

}  // namespace

namespace fitimpl {

void destroy_host_stage(fit_handle* h) {
  if (h->host_stage) free_stage(static_cast<HostStage*>(h->host_stage));
  h->host_stage = nullptr;
}

}  // namespace fitimpl

extern "C" int fit_propagate_update_host(fit_handle* h, const fit_tracks_in* in,
                                         const fit_tracks_out* out, const fit_hits* hits,
                                         int nevt, const int64_t* ntrk, int nlayer,
                                         const int32_t* mode, void* stream) {
  static const char* kWho = "fit_propagate_update_host";
  g_last_error.clear();
  if (!h) return fail(FIT_ERR_ARG, std::string(kWho) + ": NULL handle");
  int64_t total = 0;
  int rc = check_call(h, in, out, hits, nevt, ntrk, nlayer, mode, &total, kWho);
  if (rc != FIT_OK || total == 0) return rc;
  DeviceGuard guard(h->device);
  const int64_t cap = std::min<int64_t>(kChunk, (total + 3) & ~int64_t(3));
  HostStage* hs = nullptr;
  rc = stage_for(h, cap, nlayer, &hs);
  if (rc != FIT_OK) return rc;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaEventRecord(hs->ev_start, cs);
  for (int i = 0; i < kSets && e == cudaSuccess; ++i)
    e = cudaStreamWaitEvent(hs->st[i], hs->ev_start, 0);
  if (e != cudaSuccess) return cuda_fail(e, "fit_propagate_update_host: stream order");

  const size_t P = (size_t)hs->cap * 4;  // staging pitch
  const size_t pin = (size_t)in->ld * 4, pout = (size_t)out->ld * 4, phit = (size_t)hits->ld * 4;
  std::vector<int64_t> es(nevt + 1, 0);  // first track of each event
  for (int e2 = 0; e2 < nevt; ++e2) es[e2 + 1] = es[e2] + ntrk[e2];
  std::vector<int64_t> nt_local;
  std::vector<int32_t> md_local;
  int ev = 0;  // first event that ends after the chunk's start
  int k = 0;
  for (int64_t c0 = 0; c0 < total; c0 += hs->cap, ++k) {
    const int64_t c1 = std::min(total, c0 + hs->cap), nc = c1 - c0;
    const int b = k % kSets;
    cudaStream_t s = hs->st[b];
    const Set S = carve(hs->buf[b], hs->cap, hs->nlayer);
    // the events (or parts of events) of [c0, c1), in order
    nt_local.clear();
    md_local.clear();
    while (ev < nevt && es[ev + 1] <= c0) ++ev;
    for (int e2 = ev; e2 < nevt && es[e2] < c1; ++e2) {
      const int64_t lo = std::max(es[e2], c0), hi = std::min(es[e2 + 1], c1);
      if (hi > lo) {
        nt_local.push_back(hi - lo);
        md_local.push_back(mode[e2]);
      }
    }
    const size_t w = (size_t)nc * 4;
    e = copy_rows(S.par, P, in->par + c0, pin, w, 6, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = copy_rows(S.cov, P, in->cov + c0, pin, w, 21, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S.q, in->q + c0, w, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = copy_rows(S.hpos, P, hits->pos + c0, phit, w, 3 * (size_t)nlayer, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = copy_rows(S.hcov, P, hits->cov + c0, phit, w, 6 * (size_t)nlayer, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "fit_propagate_update_host: copy to device");
    fit_tracks_in sin{S.par, S.cov, S.q, hs->cap};
    fit_tracks_out sout{S.par, S.cov, S.q, S.chi2, out->chi2_layer ? S.chi2_layer : nullptr,
                        out->status ? S.status : nullptr, hs->cap};
    fit_hits shit{S.hpos, S.hcov, hs->cap};
    rc = run_fit(h, base_args(&sin, &sout, &shit, nlayer, h->d_counters), (int)nt_local.size(),
                 nt_local.data(), md_local.data(), kWho, s, s);
    if (rc != FIT_OK) return rc;
    e = copy_rows(out->par + c0, pout, S.par, P, w, 6, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = copy_rows(out->cov + c0, pout, S.cov, P, w, 21, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->q + c0, S.q, w, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->chi2 + c0, S.chi2, w, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && out->status)
      e = cudaMemcpyAsync(out->status + c0, S.status, (size_t)nc, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && out->chi2_layer)
      e = copy_rows(out->chi2_layer + c0, pout, S.chi2_layer, P, w, (size_t)nlayer,
                    cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "fit_propagate_update_host: copy to host");
  }
  for (int i = 0; i < kSets && e == cudaSuccess; ++i) {
    e = cudaEventRecord(hs->ev_done[i], hs->st[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, hs->ev_done[i], 0);
  }
  if (e != cudaSuccess) return cuda_fail(e, "fit_propagate_update_host: stream order");
  h->tracks += (uint64_t)total;
  return FIT_OK;
}

namespace {

// Whether p lies in page-locked host memory that the current device reaches
// under the same address (so a kernel may dereference it).
bool mapped_host(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error of a pointer CUDA does not know
    return false;
  }
  return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

}  // namespace

extern "C" int fit_propagate_update_mapped(fit_handle* h, const fit_tracks_in* in,
                                           const fit_tracks_out* out, const fit_hits* hits,
                                           int nevt, const int64_t* ntrk, int nlayer,
                                           const int32_t* mode, void* stream) {
  static const char* kWho = "fit_propagate_update_mapped";
  g_last_error.clear();
  if (!h) return fail(FIT_ERR_ARG, std::string(kWho) + ": NULL handle");
  int64_t total = 0;
  int rc = check_call(h, in, out, hits, nevt, ntrk, nlayer, mode, &total, kWho);
  if (rc != FIT_OK || total == 0) return rc;
  DeviceGuard guard(h->device);
  const void* ptrs[] = {in->par, in->cov, in->q, out->par, out->cov, out->q, out->chi2,
                        out->chi2_layer, out->status, hits->pos, hits->cov};
  for (const void* p : ptrs)
    if (p && !mapped_host(p))
      return fail(FIT_ERR_ARG, std::string(kWho) +
                                   ": a buffer is not page-locked host memory mapped into the "
                                   "device's address space");
  rc = run_fit(h, base_args(in, out, hits, nlayer, h->d_counters), nevt, ntrk, mode, kWho,
               static_cast<cudaStream_t>(stream), static_cast<cudaStream_t>(stream));
  if (rc != FIT_OK) return rc;
  h->tracks += (uint64_t)total;
  return FIT_OK;
}
