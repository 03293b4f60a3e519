// libfit: batched form of the fused fit -- many events of uneven size and
// mixed surface types (p2r / p2z) in one persistent launch, replayed from a
// CUDA graph, with a launch-shape autotuner (fit_plan_* in fit.h).
//
// Work items are tiles of one event: threads_per_block x tracks_per_thread
// consecutive tracks (two per thread in packed f32x2 instructions, or one),
// never crossing an event, so each item has one surface type and the branch
// on it is uniform across the block.  Blocks pull items
// from an atomic counter until none is left (dynamic load balance across
// uneven events and the cheaper p2z items).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fit.h"
#include "fused.cuh"

namespace fitimpl {
namespace {

struct WorkItem {
  int64_t first;       // the item's first track (even with two per thread)
  int64_t begin, end;  // the event's track range
  int32_t mode;
  int32_t event;
};

struct BatchArgs {
  FitArgs a;  // buffers, nlayer, counters (a.t0/a.t1/a.geo unused)
  Geo geo[2];
  const WorkItem* items;
  int nitems;
  unsigned* work_counter;
};

// TPT tracks per thread.  Two: at least 384 resident threads per SM (3
// blocks of 128, 6 of 64, 12 of 32), as for fit_fused_kernel's p2r: left
// free, the compiler takes ~190 registers and only 2 blocks of 128 fit.
// One: at least 512 (128 registers).  Blocks of 256: at least two per SM.
// L: the layout of the caller's track and hit arrays (FIT_LAYOUT_*).
constexpr int batched_min_blocks(int blk, int tpt) {
  return blk == 256 ? 2 : (tpt == 2 ? 384 : 512) / blk;
}

template <int BLK, int TPT, int L>
__global__ void __launch_bounds__(BLK, batched_min_blocks(BLK, TPT))
    fit_batched_kernel(const __grid_constant__ BatchArgs b) {
  __shared__ int s_item;
  for (;;) {
    __syncthreads();  // every thread has read the previous item index
    if (threadIdx.x == 0) s_item = (int)atomicAdd(b.work_counter, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= b.nitems) return;
    const WorkItem w = b.items[it];
    if constexpr (TPT == 1) {
      const int64_t t = w.first + (int64_t)threadIdx.x;
      if (t < w.end) {
        unsigned st = 0u, iters = 0u;
        State<float> s;
        if (w.mode == FIT_MODE_Z) {
          begin_state<FIT_MODE_Z, L>(b.a, b.geo[FIT_MODE_Z], t, s);
          finish_one<FIT_MODE_Z, L>(b.a, b.geo[FIT_MODE_Z], t, 0, s, st, iters, true);
        } else {
          begin_state<FIT_MODE_R, L>(b.a, b.geo[FIT_MODE_R], t, s);
          finish_one<FIT_MODE_R, L>(b.a, b.geo[FIT_MODE_R], t, 0, s, st, iters, true);
          count_iterations(iters, &b.a.counters[4]);
        }
        if (st) count_status(st, b.a.counters);
      }
      continue;
    }
    const int64_t t = w.first + 2 * (int64_t)threadIdx.x;
    if (t < w.end) {
      unsigned st[2] = {0u, 0u}, iters[2] = {0u, 0u};
      if (w.mode == FIT_MODE_Z) {
        run_pair<FIT_MODE_Z, L>(b.a, b.geo[FIT_MODE_Z], w.begin, w.end, t, st, iters);
      } else {
        run_pair<FIT_MODE_R, L>(b.a, b.geo[FIT_MODE_R], w.begin, w.end, t, st, iters);
        count_iterations(iters[0] + iters[1], &b.a.counters[4]);
      }
      if (st[0]) count_status(st[0], b.a.counters);
      if (st[1]) count_status(st[1], b.a.counters);
    }
  }
}

// Index of component k (of K) of track t in layout L, leading dimension ld.
__device__ __forceinline__ int64_t lay_ix(int L, int k, int64_t t, int64_t ld, int K) {
  return L == FIT_LAYOUT_SOA ? k * ld + t : (((t >> 5) * K + k) << 5) + (t & 31);
}

// dst[k, t] = src[k, t] for rows k < K and tracks t < n, 4-byte elements.
__global__ void relayout_kernel(const uint32_t* __restrict__ src, int64_t src_ld, int src_layout,
                                uint32_t* __restrict__ dst, int64_t dst_ld, int dst_layout, int K,
                                int64_t n) {
  const int64_t total = (int64_t)K * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i / n);
    const int64_t t = i - (int64_t)k * n;
    dst[lay_ix(dst_layout, k, t, dst_ld, K)] = src[lay_ix(src_layout, k, t, src_ld, K)];
  }
}

// Same-mode runs of events, one launch each (the fit_propagate_update path),
// kept as an autotuner candidate: for few, large events it can win.
template <int MODE, int L>
__global__ void __launch_bounds__(kBlock, MODE == FIT_MODE_Z ? 4 : 3)
    fit_segment_kernel(const __grid_constant__ FitArgs a) {
  const int64_t t = pair_track(a);
  if (t >= a.t1) return;
  unsigned st[2] = {0u, 0u}, iters[2] = {0u, 0u};
  run_pair<MODE, L>(a, a.geo, a.t0, a.t1, t, st, iters);
  if (st[0]) count_status(st[0], a.counters);
  if (st[1]) count_status(st[1], a.counters);
  if (MODE == FIT_MODE_R) count_iterations(iters[0] + iters[1], &a.counters[4]);
}

int tracks_per_thread(const fit_launch_config& c) { return c.tracks_per_thread == 1 ? 1 : 2; }

// The batched kernel of a launch shape and its launcher, or NULL for a
// shape not compiled: two tracks per thread with 32, 64, 128 or 256 threads
// per block, one with 64, 128 or 256; either layout.
using BatchedLaunch = void (*)(const BatchArgs&, unsigned, cudaStream_t);
template <int BLK, int TPT, int L>
void launch_batched(const BatchArgs& b, unsigned grid, cudaStream_t s) {
  fit_batched_kernel<BLK, TPT, L><<<grid, BLK, 0, s>>>(b);
}
struct BatchedShape {
  int tpb, tpt, layout;
  const void* kernel;
  BatchedLaunch launch;
};
#define FIT_BATCHED_SHAPE(BLK, TPT, L) \
  {BLK, TPT, L, (const void*)fit_batched_kernel<BLK, TPT, L>, launch_batched<BLK, TPT, L>}
const BatchedShape kBatchedShapes[] = {
    FIT_BATCHED_SHAPE(32, 2, 0),  FIT_BATCHED_SHAPE(64, 2, 0),  FIT_BATCHED_SHAPE(128, 2, 0),
    FIT_BATCHED_SHAPE(256, 2, 0), FIT_BATCHED_SHAPE(64, 1, 0),  FIT_BATCHED_SHAPE(128, 1, 0),
    FIT_BATCHED_SHAPE(256, 1, 0), FIT_BATCHED_SHAPE(32, 2, 1),  FIT_BATCHED_SHAPE(64, 2, 1),
    FIT_BATCHED_SHAPE(128, 2, 1), FIT_BATCHED_SHAPE(256, 2, 1), FIT_BATCHED_SHAPE(64, 1, 1),
    FIT_BATCHED_SHAPE(128, 1, 1), FIT_BATCHED_SHAPE(256, 1, 1)};
#undef FIT_BATCHED_SHAPE

const BatchedShape* batched_shape(int tpb, int tpt, int layout) {
  for (const BatchedShape& b : kBatchedShapes)
    if (b.tpb == tpb && b.tpt == tpt && b.layout == layout) return &b;
  return nullptr;
}
const void* batched_kernel(int tpb, int tpt, int layout) {
  const BatchedShape* b = batched_shape(tpb, tpt, layout);
  return b ? b->kernel : nullptr;
}

int max_blocks_per_sm(int tpb, int tpt, int layout) {
  const void* k = batched_kernel(tpb, tpt, layout);
  int n = 0;
  if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, tpb, 0) != cudaSuccess) return 0;
  return n;
}

std::string cache_key(int device, int nlayer, const std::vector<int64_t>& ntrk,
                      const std::vector<int32_t>& mode, int layout) {
  // Device, geometry depth, and the event-size histogram (powers of two) per
  // mode: plans with the same key have the same shape of work.
  cudaDeviceProp prop;
  std::string name = "gpu";
  if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) name = prop.name;
  for (char& ch : name)
    if (ch == ' ' || ch == '\t') ch = '_';
  int hist[2][64] = {};
  int64_t tracks[2] = {0, 0};
  for (size_t e = 0; e < ntrk.size(); ++e) {
    int b = 0;
    while ((int64_t(1) << b) < ntrk[e] && b < 63) ++b;
    hist[mode[e]][b]++;
    tracks[mode[e]] += ntrk[e];
  }
  std::string k = name + ";v3;layout=" + std::to_string(layout) + ";nlayer=" +
                  std::to_string(nlayer) + ";tracks=" +
                  std::to_string(tracks[0]) + "," + std::to_string(tracks[1]) + ";hist=";
  for (int m = 0; m < 2; ++m)
    for (int b = 0; b < 64; ++b)
      if (hist[m][b]) k += std::to_string(m) + ":" + std::to_string(b) + ":" + std::to_string(hist[m][b]) + ",";
  return k;
}

std::mutex g_tune_mu;
std::map<std::string, fit_launch_config> g_tune_memo;  // key -> tuned shape, this process

bool read_cache(const char* path, const std::string& key, fit_launch_config* cfg) {
  if (!path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[4096];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    char* tab = std::strchr(line, '\t');
    if (!tab) continue;
    *tab = 0;
    if (key != line) continue;
    fit_launch_config c{};
    if (std::sscanf(tab + 1, "%d %d %d %d %d", &c.threads_per_block, &c.blocks_per_sm,
                    &c.persistent, &c.tracks_per_thread, &c.layout) == 5) {
      *cfg = c;  // the last matching line wins
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void append_cache(const char* path, const std::string& key, const fit_launch_config& c, float ms) {
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s\t%d %d %d %d %d %.4f\n", key.c_str(), c.threads_per_block, c.blocks_per_sm,
               c.persistent, tracks_per_thread(c), c.layout, ms);
  std::fclose(f);
}

}  // namespace
}  // namespace fitimpl

using namespace fitimpl;

struct fit_plan {
  fit_handle* h = nullptr;
  int nlayer = 0;
  std::vector<int64_t> ntrk;
  std::vector<int32_t> mode;
  int64_t total = 0;
  fit_launch_config cfg{128, 0, 1, 2, FIT_LAYOUT_SOA};
  bool layout_free = false;  // created with FIT_LAYOUT_TUNE and not tuned yet
  int sms = 0;
  WorkItem* d_items = nullptr;
  int nitems = 0;
  int items_tile = 0;  // tracks per work item of the current table
  int items_tpt = 0;
  unsigned* d_work = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* key_ptrs[12] = {};
  unsigned long long* d_tune_counters = nullptr;  // counters of the tuning runs
  int64_t key_ld[3] = {};
  int tuned = 0;
  float best_ms = 0.f;
};

namespace {

// Work items of tpb x tpt tracks.  With two tracks per thread an item starts
// at an even track (packed loads are 8-byte aligned), so an event's first
// item may begin one track early; the kernel skips tracks outside the event.
int build_items(fit_plan* p, int tpb, int tpt) {
  if (p->items_tile == tpb * tpt && p->items_tpt == tpt && p->d_items) return FIT_OK;
  std::vector<WorkItem> items;
  int64_t start = 0;
  for (size_t e = 0; e < p->ntrk.size(); ++e) {
    const int64_t begin = start, end = start + p->ntrk[e];
    start = end;
    if (end == begin) continue;
    const int64_t first = tpt == 2 ? begin & ~int64_t(1) : begin;
    for (int64_t t = first; t < end; t += (int64_t)tpb * tpt)
      items.push_back({t, begin, end, p->mode[e], (int32_t)e});
  }
  if (items.size() > 0x7fffffff) return fail(FIT_ERR_ARG, "fit_plan: too many work items");
  DeviceGuard g(p->h->device);
  if (p->d_items) {  // a run of the old shape may still read them
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "fit_plan: synchronize");
    cudaFree(p->d_items);
  }
  p->d_items = nullptr;
  p->nitems = (int)items.size();
  p->items_tile = tpb * tpt;
  p->items_tpt = tpt;
  if (items.empty()) return FIT_OK;
  cudaError_t e = cudaMalloc(&p->d_items, items.size() * sizeof(WorkItem));
  if (e != cudaSuccess) return fail(FIT_ERR_NOMEM, "fit_plan: cudaMalloc of the work items");
  e = cudaMemcpy(p->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "fit_plan: work-item upload");
  return FIT_OK;
}

// Issues the plan's work for one shape on stream s (captured into a graph).
int issue(fit_plan* p, const FitArgs& base, cudaStream_t s) {
  if (p->total == 0) return FIT_OK;
  if (p->cfg.persistent) {
    BatchArgs b{};
    b.a = base;
    b.geo[0] = p->h->geo[0];
    b.geo[1] = p->h->geo[1];
    b.items = p->d_items;
    b.nitems = p->nitems;
    b.work_counter = p->d_work;
    cudaError_t e = cudaMemsetAsync(p->d_work, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_fail(e, "fit_plan: work counter reset");
    const unsigned grid = (unsigned)std::max(1, p->cfg.blocks_per_sm * p->sms);
    const BatchedShape* shape =
        batched_shape(p->cfg.threads_per_block, tracks_per_thread(p->cfg), p->cfg.layout);
    if (!shape) return fail(FIT_ERR_ARG, "fit_plan: launch shape not compiled");
    shape->launch(b, grid, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fit_plan: launch");
    return FIT_OK;
  }
  FitArgs a = base;
  int64_t t = 0;
  size_t e = 0;
  const size_t nevt = p->ntrk.size();
  while (e < nevt) {
    const int m = p->mode[e];
    int64_t t1 = t;
    while (e < nevt && p->mode[e] == m) t1 += p->ntrk[e++];
    if (t1 > t) {
      a.t0 = t;
      a.t1 = t1;
      a.geo = p->h->geo[m];
      const int64_t npairs = (t1 - (t & ~int64_t(1)) + 1) / 2;
      const unsigned nblk = (unsigned)((npairs + kBlock - 1) / kBlock);
      if (p->cfg.layout == FIT_LAYOUT_AOSOA32) {
        if (m == FIT_MODE_Z)
          fit_segment_kernel<FIT_MODE_Z, 1><<<nblk, kBlock, 0, s>>>(a);
        else
          fit_segment_kernel<FIT_MODE_R, 1><<<nblk, kBlock, 0, s>>>(a);
      } else if (m == FIT_MODE_Z) {
        fit_segment_kernel<FIT_MODE_Z, 0><<<nblk, kBlock, 0, s>>>(a);
      } else {
        fit_segment_kernel<FIT_MODE_R, 0><<<nblk, kBlock, 0, s>>>(a);
      }
      cudaError_t err = cudaGetLastError();
      if (err != cudaSuccess) return cuda_fail(err, "fit_plan: launch");
    }
    t = t1;
  }
  return FIT_OK;
}

void drop_graph(fit_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  p->exec = nullptr;
  std::memset(p->key_ptrs, 0, sizeof(p->key_ptrs));
}

// Captures the plan's work for these buffers into a graph (once per buffer
// set and shape) and launches it on s.
int run_graph(fit_plan* p, const fit_tracks_in* in, const fit_tracks_out* out,
              const fit_hits* hits, cudaStream_t s, unsigned long long* counters) {
  const void* ptrs[12] = {in->par, in->cov, in->q, out->par, out->cov, out->q,
                          out->chi2, out->chi2_layer, out->status, hits->pos, hits->cov,
                          counters};
  const int64_t lds[3] = {in->ld, out->ld, hits->ld};
  const bool same = p->exec && std::memcmp(ptrs, p->key_ptrs, sizeof(ptrs)) == 0 &&
                    std::memcmp(lds, p->key_ld, sizeof(lds)) == 0;
  if (!same) {
    drop_graph(p);
    int rc = build_items(p, p->cfg.threads_per_block, tracks_per_thread(p->cfg));
    if (rc != FIT_OK) return rc;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "fit_plan: cudaStreamBeginCapture");
    rc = issue(p, base_args(in, out, hits, p->nlayer, counters), p->cap);
    e = cudaStreamEndCapture(p->cap, &graph);
    if (rc != FIT_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "fit_plan: cudaStreamEndCapture");
    e = cudaGraphInstantiate(&p->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      p->exec = nullptr;
      return cuda_fail(e, "fit_plan: cudaGraphInstantiate");
    }
    std::memcpy(p->key_ptrs, ptrs, sizeof(ptrs));
    std::memcpy(p->key_ld, lds, sizeof(lds));
  }
  cudaError_t e = cudaGraphLaunch(p->exec, s);
  if (e != cudaSuccess) return cuda_fail(e, "fit_plan: cudaGraphLaunch");
  return FIT_OK;
}

int check_plan_buffers(fit_plan* p, const fit_tracks_in* in, const fit_tracks_out* out,
                       const fit_hits* hits, const char* who) {
  int64_t total = 0;
  int rc = check_call(p->h, in, out, hits, (int)p->ntrk.size(), p->ntrk.data(), p->nlayer,
                      p->mode.data(), &total, who);
  if (rc == FIT_OK && p->cfg.layout == FIT_LAYOUT_AOSOA32 && total > 0 &&
      ((in->ld | out->ld | hits->ld) & 31))
    return fail(FIT_ERR_ARG, std::string(who) + ": AoSoA slots (ld) must be a multiple of 32");
  return rc;
}

int relayout(const void* src, int64_t src_ld, int src_layout, void* dst, int64_t dst_ld,
             int dst_layout, int K, int64_t n, cudaStream_t s) {
  if (K <= 0 || n <= 0) return FIT_OK;
  const int64_t total = (int64_t)K * n;
  const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
  relayout_kernel<<<grid, 256, 0, s>>>(static_cast<const uint32_t*>(src), src_ld, src_layout,
                                       static_cast<uint32_t*>(dst), dst_ld, dst_layout, K, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FIT_OK : cuda_fail(e, "relayout: launch");
}

}  // namespace

extern "C" {

int fit_plan_create(fit_handle* h, int nevt, const int64_t* ntrk, const int32_t* mode, int nlayer,
                    const fit_launch_config* cfg, fit_plan** out) {
  if (!out) return fail(FIT_ERR_ARG, "fit_plan_create: plan pointer is NULL");
  *out = nullptr;
  if (!h) return fail(FIT_ERR_ARG, "fit_plan_create: handle is NULL");
  if (nevt < 0 || (nevt > 0 && (!ntrk || !mode)))
    return fail(FIT_ERR_ARG, "fit_plan_create: bad event arrays");
  int64_t total = 0;
  for (int e = 0; e < nevt; ++e) {
    if (ntrk[e] < 0) return fail(FIT_ERR_ARG, "fit_plan_create: ntrk[e] < 0");
    if (mode[e] != FIT_MODE_R && mode[e] != FIT_MODE_Z)
      return fail(FIT_ERR_ARG, "fit_plan_create: mode[e] is not FIT_MODE_R or FIT_MODE_Z");
    if (!h->has[mode[e]]) return fail(FIT_ERR_ARG, "fit_plan_create: mode not configured");
    if (h->nlayer[mode[e]] != nlayer)
      return fail(FIT_ERR_ARG, "fit_plan_create: nlayer differs from the configured one");
    total += ntrk[e];
  }
  if (cfg && cfg->layout != FIT_LAYOUT_SOA && cfg->layout != FIT_LAYOUT_AOSOA32 &&
      cfg->layout != FIT_LAYOUT_TUNE)
    return fail(FIT_ERR_ARG, "fit_plan_create: layout must be FIT_LAYOUT_SOA, "
                             "FIT_LAYOUT_AOSOA32 or FIT_LAYOUT_TUNE");
  const int run_layout = cfg && cfg->layout == FIT_LAYOUT_AOSOA32 ? 1 : 0;
  if (cfg && (cfg->tracks_per_thread < 0 || cfg->tracks_per_thread > 2 || cfg->blocks_per_sm < 0 ||
              !batched_kernel(cfg->threads_per_block, tracks_per_thread(*cfg), run_layout) ||
              (!cfg->persistent && tracks_per_thread(*cfg) != 2)))
    return fail(FIT_ERR_ARG, "fit_plan_create: threads_per_block must be 32, 64, 128 or 256 with "
                             "two tracks per thread, 64, 128 or 256 with one (persistent only)");
  DeviceGuard g(h->device);
  fit_plan* p = new fit_plan();
  p->h = h;
  p->nlayer = nlayer;
  p->ntrk.assign(ntrk, ntrk + nevt);
  p->mode.assign(mode, mode + nevt);
  p->total = total;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, h->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "fit_plan_create: cudaGetDeviceProperties");
  }
  p->sms = prop.multiProcessorCount;
  if (cfg) p->cfg = *cfg;
  p->layout_free = p->cfg.layout == FIT_LAYOUT_TUNE;
  p->cfg.layout = run_layout;
  p->cfg.tracks_per_thread = tracks_per_thread(p->cfg);
  if (p->cfg.blocks_per_sm == 0)
    p->cfg.blocks_per_sm =
        max_blocks_per_sm(p->cfg.threads_per_block, p->cfg.tracks_per_thread, p->cfg.layout);
  if (p->cfg.blocks_per_sm <= 0) p->cfg.blocks_per_sm = 1;
  e = cudaMalloc(&p->d_work, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_tune_counters, kCounters * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    fit_plan_destroy(p);
    return fail(FIT_ERR_NOMEM, std::string("fit_plan_create: ") + cudaGetErrorString(e));
  }
  int rc = build_items(p, p->cfg.threads_per_block, p->cfg.tracks_per_thread);
  if (rc != FIT_OK) {
    fit_plan_destroy(p);
    return rc;
  }
  *out = p;
  return FIT_OK;
}

int fit_plan_run(fit_plan* p, const fit_tracks_in* in, const fit_tracks_out* out,
                 const fit_hits* hits, void* stream) {
  g_last_error.clear();
  if (!p) return fail(FIT_ERR_ARG, "fit_plan_run: plan is NULL");
  int rc = check_plan_buffers(p, in, out, hits, "fit_plan_run");
  if (rc != FIT_OK) return rc;
  if (p->total == 0) return FIT_OK;
  DeviceGuard g(p->h->device);
  rc = run_graph(p, in, out, hits, static_cast<cudaStream_t>(stream), p->h->d_counters);
  if (rc == FIT_OK) p->h->tracks += (uint64_t)p->total;
  return rc;
}

int fit_plan_tune(fit_plan* p, const fit_tracks_in* in, const fit_tracks_out* out,
                  const fit_hits* hits, void* stream, const char* cache_path) {
  g_last_error.clear();
  if (!p) return fail(FIT_ERR_ARG, "fit_plan_tune: plan is NULL");
  int rc = check_plan_buffers(p, in, out, hits, "fit_plan_tune");
  if (rc != FIT_OK) return rc;
  if (p->total == 0) return FIT_OK;
  if (in->par == out->par || in->cov == out->cov || (const void*)in->q == (void*)out->q)
    return fail(FIT_ERR_ARG, "fit_plan_tune: the outputs must not alias the inputs");
  DeviceGuard g(p->h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int in_layout = p->cfg.layout;  // the layout of the caller's buffers
  const std::string key = cache_key(p->h->device, p->nlayer, p->ntrk, p->mode,
                                    p->layout_free ? FIT_LAYOUT_TUNE : in_layout);
  fit_launch_config found{};
  bool have = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_memo.find(key);
    if (it != g_tune_memo.end()) {
      found = it->second;
      have = true;
    }
  }
  if (!have && read_cache(cache_path, key, &found)) have = true;
  if (have && batched_kernel(found.threads_per_block, tracks_per_thread(found), found.layout)) {
    drop_graph(p);
    p->cfg = found;
    p->layout_free = false;
    p->tuned = 2;
    p->best_ms = 0.f;
    return FIT_OK;
  }
  // Candidates: persistent with two tracks per thread and 32, 64, 128 or 256
  // threads per block, or one track per thread and 64, 128 or 256, each at
  // every resident-block count; and the one-launch-per-segment form.  With
  // the layout left to the tuner, each in both layouts: the other layout's
  // runs read a converted copy of the inputs (scratch, freed on return).
  std::vector<int> layouts = {in_layout};
  if (p->layout_free) layouts.push_back(1 - in_layout);
  std::vector<fit_launch_config> cands;
  for (int L : layouts) {
    for (int tpt : {2, 1})
      for (int tpb : {32, 64, 128, 256}) {
        if (!batched_kernel(tpb, tpt, L)) continue;
        const int maxb = max_blocks_per_sm(tpb, tpt, L);
        for (int b = 1; b <= maxb; ++b) cands.push_back({tpb, b, 1, tpt, L});
      }
    cands.push_back({128, 0, 0, 2, L});
  }
  // the other layout's copies: par, cov and hit arrays converted, outputs
  // written to scratch (per-track arrays -- q, chi2, status -- are laid out
  // alike in both layouts and used as they are)
  void* scratch = nullptr;
  fit_tracks_in in2 = *in;
  fit_tracks_out out2 = *out;
  fit_hits hits2 = *hits;
  if (layouts.size() > 1) {
    const int L2 = layouts[1];
    const int64_t ld2 = L2 == FIT_LAYOUT_AOSOA32 ? (p->total + 31) & ~int64_t(31)
                                                 : (p->total + 3) & ~int64_t(3);
    const int nl = p->nlayer;
    const size_t rows = 27 + 27 + 9 * (size_t)nl + (out->chi2_layer ? nl : 0);
    cudaError_t e = cudaMalloc(&scratch, rows * (size_t)ld2 * 4);
    if (e != cudaSuccess) return fail(FIT_ERR_NOMEM, "fit_plan_tune: scratch of the layout search");
    float* f = static_cast<float*>(scratch);
    in2.par = f;
    in2.cov = f + 6 * ld2;
    in2.ld = ld2;
    out2.par = f + 27 * ld2;
    out2.cov = f + 33 * ld2;
    out2.ld = ld2;
    hits2.pos = f + 54 * ld2;
    hits2.cov = f + (54 + 3 * (int64_t)nl) * ld2;
    hits2.ld = ld2;
    out2.chi2_layer = out->chi2_layer ? f + (54 + 9 * (int64_t)nl) * ld2 : nullptr;
    rc = relayout(in->par, in->ld, in_layout, (void*)in2.par, ld2, L2, 6, p->total, s);
    if (rc == FIT_OK) rc = relayout(in->cov, in->ld, in_layout, (void*)in2.cov, ld2, L2, 21, p->total, s);
    if (rc == FIT_OK)
      rc = relayout(hits->pos, hits->ld, in_layout, (void*)hits2.pos, ld2, L2, 3 * nl, p->total, s);
    if (rc == FIT_OK)
      rc = relayout(hits->cov, hits->ld, in_layout, (void*)hits2.cov, ld2, L2, 6 * nl, p->total, s);
    if (rc != FIT_OK) {
      cudaFree(scratch);
      return rc;
    }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (scratch) cudaFree(scratch);
    return fail(FIT_ERR_CUDA, "fit_plan_tune: cudaEventCreate");
  }
  float best = 1e30f;
  fit_launch_config best_cfg = p->cfg;
  for (const fit_launch_config& c : cands) {
    const bool own = c.layout == in_layout;
    const fit_tracks_in* ci = own ? in : &in2;
    const fit_tracks_out* co = own ? out : &out2;
    const fit_hits* ch = own ? hits : &hits2;
    drop_graph(p);
    p->cfg = c;
    rc = run_graph(p, ci, co, ch, s, p->d_tune_counters);  // warm-up (and capture)
    if (rc != FIT_OK) break;
    float t[3];
    for (int r = 0; r < 3 && rc == FIT_OK; ++r) {
      cudaEventRecord(e0, s);
      rc = run_graph(p, ci, co, ch, s, p->d_tune_counters);
      cudaEventRecord(e1, s);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) rc = cuda_fail(e, "fit_plan_tune: cudaEventSynchronize");
      cudaEventElapsedTime(&t[r], e0, e1);
    }
    if (rc != FIT_OK) break;
    std::sort(t, t + 3);
    if (t[1] < best) {
      best = t[1];
      best_cfg = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graph(p);
  if (scratch) {
    cudaStreamSynchronize(s);
    cudaFree(scratch);
  }
  if (rc != FIT_OK) return rc;
  p->cfg = best_cfg;
  p->layout_free = false;
  p->tuned = 1;
  p->best_ms = best;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_memo[key] = best_cfg;
  }
  append_cache(cache_path, key, best_cfg, best);
  return FIT_OK;
}

int fit_plan_get_info(const fit_plan* p, fit_plan_info* info) {
  if (!p || !info) return fail(FIT_ERR_ARG, "fit_plan_get_info: NULL argument");
  info->config = p->cfg;
  info->tracks = p->total;
  int64_t items = 0, start = 0;
  const int tpt = tracks_per_thread(p->cfg);
  const int64_t tile = (int64_t)p->cfg.threads_per_block * tpt;
  for (size_t e = 0; e < p->ntrk.size(); ++e) {
    const int64_t end = start + p->ntrk[e];
    const int64_t first = tpt == 2 ? start & ~int64_t(1) : start;
    if (end > start) items += (end - first + tile - 1) / tile;
    start = end;
  }
  info->items = (int32_t)items;
  info->tuned = p->tuned;
  info->best_ms = p->best_ms;
  return FIT_OK;
}

int fit_relayout(const void* src, int64_t src_ld, int src_layout, void* dst, int64_t dst_ld,
                 int dst_layout, int rows, int64_t n, void* stream) {
  g_last_error.clear();
  auto ok_layout = [](int L) { return L == FIT_LAYOUT_SOA || L == FIT_LAYOUT_AOSOA32; };
  if (!src || !dst || rows < 0 || n < 0 || !ok_layout(src_layout) || !ok_layout(dst_layout))
    return fail(FIT_ERR_ARG, "fit_relayout: bad argument");
  if (src == dst) return fail(FIT_ERR_ARG, "fit_relayout: src and dst must not be the same array");
  auto ld_ok = [n](int L, int64_t ld) {
    return ld >= n && (L == FIT_LAYOUT_SOA || (ld & 31) == 0);
  };
  if (!ld_ok(src_layout, src_ld) || !ld_ok(dst_layout, dst_ld))
    return fail(FIT_ERR_ARG, "fit_relayout: ld smaller than n, or not a multiple of 32 for "
                             "FIT_LAYOUT_AOSOA32");
  return relayout(src, src_ld, src_layout, dst, dst_ld, dst_layout, rows, n,
                  static_cast<cudaStream_t>(stream));
}

void fit_plan_destroy(fit_plan* p) {
  if (!p) return;
  {
    DeviceGuard g(p->h->device);
    if (p->cap) cudaStreamSynchronize(p->cap);
    drop_graph(p);
    if (p->d_items) cudaFree(p->d_items);
    if (p->d_work) cudaFree(p->d_work);
    if (p->d_tune_counters) cudaFree(p->d_tune_counters);
    if (p->cap) cudaStreamDestroy(p->cap);
  }
  delete p;
}

}  // extern "C"
