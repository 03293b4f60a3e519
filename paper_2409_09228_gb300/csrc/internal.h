// Internal declarations shared by the libfit translation units (not part of
// the C ABI).  Host-side helpers and the kernel argument blocks.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "fit.h"

namespace fitimpl {

// Error reporting: the message of the last failure on the calling thread.
extern thread_local std::string g_last_error;
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

constexpr int kBlock = 128;
constexpr int kCounters = 5;  // no_intersection, not_converged, nonfinite, charge_flip,
                               // p2r path-length iterations

struct Surfaces {
  float s[FIT_MAX_LAYERS];
};

// Geometry and numerics of one mode.
struct Geo {
  float kB;  // kA * B
  int max_iter;
  float tol;
  int line_start;  // p2r: start the path-length iteration at the straight-line step
  Surfaces surf;
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
  unsigned long long* counters;
  Geo geo;
};

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

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


}  // namespace fitimpl


struct fit_handle {
  int device = 0;
  bool has[2] = {false, false};
  int nlayer[2] = {0, 0};
  fitimpl::Geo geo[2];
  unsigned long long* d_counters = nullptr;  // [kCounters]
  uint64_t tracks = 0;
  void* d_mlp = nullptr;  // learned-seed weights (fit_mlp_attach), device
  bool seeded = false;    // p2r seeds from d_mlp
  void* host_stage = nullptr;  // staging of fit_propagate_update_host (host.cu)
  float B[2] = {0.f, 0.f};     // field of each mode's configuration
  // A call of fit_propagate_update with events of both modes runs its p2z
  // launches on `side`, forked from the caller's stream by `fork` and joined
  // back by `join`; side_mu keeps concurrent calls from interleaving them.
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  std::mutex side_mu;
};


namespace fitimpl {

// Argument checks shared by the entry points that run the fused kernel.
int check_call(const fit_handle* h, const fit_tracks_in* in, const fit_tracks_out* out,
               const fit_hits* hits, int nevt, const int64_t* ntrk, int nlayer,
               const int32_t* mode, int64_t* total_out, const char* who);
FitArgs base_args(const fit_tracks_in* in, const fit_tracks_out* out, const fit_hits* hits,
                  int nlayer, unsigned long long* counters);

// The p2r fit seeded by the learned path length (mlp.cu), one track per
// thread over a.t0 .. a.t1; img is the handle's d_mlp.
void launch_seeded_fit(const FitArgs& a, const void* img, cudaStream_t s);

// The fused fit of events [0, nevt) (fit.cu): one launch per run of
// same-mode events, the p2r runs on stream s and the p2z runs on sz.
int run_fit(const fit_handle* h, const FitArgs& a, int nevt, const int64_t* ntrk,
            const int32_t* mode, const char* who, cudaStream_t s, cudaStream_t sz);

// Frees the staging of fit_propagate_update_host (host.cu).
void destroy_host_stage(fit_handle* h);

}  // namespace fitimpl
