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
// One: at least 512 (128 registers).
template <int BLK, int TPT>
__global__ void __launch_bounds__(BLK, (TPT == 2 ? 384 : 512) / BLK)
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
        load_state(b.a, t, s);
        if (w.mode == FIT_MODE_Z) {
          finish_one<FIT_MODE_Z>(b.a, b.geo[FIT_MODE_Z], t, 0, s, st, iters, true);
        } else {
          finish_one<FIT_MODE_R>(b.a, b.geo[FIT_MODE_R], t, 0, s, st, iters, true);
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
        run_pair<FIT_MODE_Z>(b.a, b.geo[FIT_MODE_Z], w.begin, w.end, t, st, iters);
      } else {
        run_pair<FIT_MODE_R>(b.a, b.geo[FIT_MODE_R], w.begin, w.end, t, st, iters);
        count_iterations(iters[0] + iters[1], &b.a.counters[4]);
      }
      if (st[0]) count_status(st[0], b.a.counters);
      if (st[1]) count_status(st[1], b.a.counters);
    }
  }
}

// Same-mode runs of events, one launch each (the fit_propagate_update path),
// kept as an autotuner candidate: for few, large events it can win.
template <int MODE>
__global__ void __launch_bounds__(kBlock, MODE == FIT_MODE_Z ? 4 : 3)
    fit_segment_kernel(const __grid_constant__ FitArgs a) {
  const int64_t t = pair_track(a);
  if (t >= a.t1) return;
  unsigned st[2] = {0u, 0u}, iters[2] = {0u, 0u};
  run_pair<MODE>(a, a.geo, a.t0, a.t1, t, st, iters);
  if (st[0]) count_status(st[0], a.counters);
  if (st[1]) count_status(st[1], a.counters);
  if (MODE == FIT_MODE_R) count_iterations(iters[0] + iters[1], &a.counters[4]);
}

int tracks_per_thread(const fit_launch_config& c) { return c.tracks_per_thread == 1 ? 1 : 2; }

// The batched kernel for a launch shape, or NULL for a shape not compiled.
const void* batched_kernel(int tpb, int tpt) {
  if (tpt == 2) {
    if (tpb == 32) return (const void*)fit_batched_kernel<32, 2>;
    if (tpb == 64) return (const void*)fit_batched_kernel<64, 2>;
    if (tpb == 128) return (const void*)fit_batched_kernel<128, 2>;
  } else {
    if (tpb == 64) return (const void*)fit_batched_kernel<64, 1>;
    if (tpb == 128) return (const void*)fit_batched_kernel<128, 1>;
  }
  return nullptr;
}

int max_blocks_per_sm(int tpb, int tpt) {
  const void* k = batched_kernel(tpb, tpt);
  int n = 0;
  if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, tpb, 0) != cudaSuccess) return 0;
  return n;
}

std::string cache_key(int device, int nlayer, const std::vector<int64_t>& ntrk,
                      const std::vector<int32_t>& mode) {
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
  std::string k = name + ";v2;nlayer=" + std::to_string(nlayer) + ";tracks=" +
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
    if (std::sscanf(tab + 1, "%d %d %d %d", &c.threads_per_block, &c.blocks_per_sm, &c.persistent,
                    &c.tracks_per_thread) == 4) {
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
  std::fprintf(f, "%s\t%d %d %d %d %.4f\n", key.c_str(), c.threads_per_block, c.blocks_per_sm,
               c.persistent, tracks_per_thread(c), ms);
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
  fit_launch_config cfg{128, 0, 1, 2};
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
    const int tpb = p->cfg.threads_per_block;
    if (tracks_per_thread(p->cfg) == 1) {
      if (tpb == 64)
        fit_batched_kernel<64, 1><<<grid, 64, 0, s>>>(b);
      else
        fit_batched_kernel<128, 1><<<grid, 128, 0, s>>>(b);
    } else if (tpb == 32) {
      fit_batched_kernel<32, 2><<<grid, 32, 0, s>>>(b);
    } else if (tpb == 64) {
      fit_batched_kernel<64, 2><<<grid, 64, 0, s>>>(b);
    } else {
      fit_batched_kernel<128, 2><<<grid, 128, 0, s>>>(b);
    }
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
      if (m == FIT_MODE_Z)
        fit_segment_kernel<FIT_MODE_Z><<<nblk, kBlock, 0, s>>>(a);
      else
        fit_segment_kernel<FIT_MODE_R><<<nblk, kBlock, 0, s>>>(a);
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
  return check_call(p->h, in, out, hits, (int)p->ntrk.size(), p->ntrk.data(), p->nlayer,
                    p->mode.data(), &total, who);
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
  if (cfg && (cfg->tracks_per_thread < 0 || cfg->tracks_per_thread > 2 || cfg->blocks_per_sm < 0 ||
              !batched_kernel(cfg->threads_per_block, tracks_per_thread(*cfg)) ||
              (!cfg->persistent && tracks_per_thread(*cfg) != 2)))
    return fail(FIT_ERR_ARG, "fit_plan_create: threads_per_block must be 32, 64 or 128 with two "
                             "tracks per thread, 64 or 128 with one (persistent only)");
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
  p->cfg.tracks_per_thread = tracks_per_thread(p->cfg);
  if (p->cfg.blocks_per_sm == 0)
    p->cfg.blocks_per_sm = max_blocks_per_sm(p->cfg.threads_per_block, p->cfg.tracks_per_thread);
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
  const std::string key = cache_key(p->h->device, p->nlayer, p->ntrk, p->mode);
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
  if (have) {
    drop_graph(p);
    p->cfg = found;
    p->tuned = 2;
    p->best_ms = 0.f;
    return FIT_OK;
  }
  // Candidates: persistent with two tracks per thread and 32, 64 or 128
  // threads per block, or one track per thread and 64 or 128, each at every
  // resident-block count; and the one-launch-per-segment form.
  std::vector<fit_launch_config> cands;
  for (int tpt : {2, 1})
    for (int tpb : {32, 64, 128}) {
      if (!batched_kernel(tpb, tpt)) continue;
      const int maxb = max_blocks_per_sm(tpb, tpt);
      for (int b = 1; b <= maxb; ++b) cands.push_back({tpb, b, 1, tpt});
    }
  cands.push_back({128, 0, 0, 2});
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(FIT_ERR_CUDA, "fit_plan_tune: cudaEventCreate");
  float best = 1e30f;
  fit_launch_config best_cfg = p->cfg;
  for (const fit_launch_config& c : cands) {
    drop_graph(p);
    p->cfg = c;
    rc = run_graph(p, in, out, hits, s, p->d_tune_counters);  // warm-up (and capture)
    if (rc != FIT_OK) break;
    float t[3];
    for (int r = 0; r < 3 && rc == FIT_OK; ++r) {
      cudaEventRecord(e0, s);
      rc = run_graph(p, in, out, hits, s, p->d_tune_counters);
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
  if (rc != FIT_OK) return rc;
  p->cfg = best_cfg;
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
