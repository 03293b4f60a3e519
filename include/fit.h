/*
 * fit.h -- C ABI of libfit, the GB300 (sm_103a) fused track propagation +
 * Kalman update library.
 *
 * The operation (paper Sec. 3, "Description of algorithm"; Sec. 3.1 "Input
 * data"; Sec. 3.2 "Computations and data structure"): for every track, layer
 * by layer, propagate the track state and its covariance along a helix in a
 * uniform solenoidal field to the next detector surface -- a cylinder r = R
 * ("p2r") or a plane z = Z ("p2z") -- and update the state with the one hit on
 * that surface (three coordinates and a 3x3 covariance).  Propagation and
 * update run as one fused GPU kernel over all tracks (Sec. 3.1).
 *
 * Conventions shared by every entry point
 *   - Units: cm, GeV, T.  Field along +z.
 *   - Track parameters p = (x, y, z, w, phi, theta): position, w = 1/pT > 0,
 *     azimuth and polar angle of the momentum.  Charge q = +1 or -1, int32.
 *     A positive charge bends clockwise seen from +z.
 *   - Symmetric matrices are stored as their lower triangle, row-major:
 *     (0,0),(1,0),(1,1),(2,0),(2,1),(2,2),...  A 6x6 covariance has 21
 *     entries; a 3x3 hit covariance has 6: (xx, yx, yy, zx, zy, zz).
 *   - Structure of arrays, track index fastest: component k of track t sits at
 *     base[k * ld + t].  ld (the leading dimension, in elements) is >= the
 *     number of tracks; pointers must be 16-byte aligned and ld a multiple of 4.
 *   - Every data pointer is a DEVICE pointer owned by the caller, except where
 *     an entry point says "host".  The library never frees caller memory.
 *   - Calls are asynchronous on the caller's CUDA stream (a cudaStream_t passed
 *     as void*, NULL = legacy default stream).  fit_sync waits and reports.
 *   - Return value: FIT_OK (0) or a negative FIT_ERR_* code.  No exception or
 *     abort crosses the ABI.  fit_last_error() describes the last failure on
 *     the calling thread.
 *   - Per-track problems never abort a call: they set a bit in the optional
 *     per-track status byte and count into the handle's counters.
 */
#ifndef FIT_H_
#define FIT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FIT_MAX_LAYERS 64

/* Return codes. */
#define FIT_OK 0
#define FIT_ERR_ARG (-1)     /* invalid argument (pointer, size, alignment) */
#define FIT_ERR_CUDA (-2)    /* a CUDA runtime call failed */
#define FIT_ERR_TIMEOUT (-3) /* fit_sync gave up waiting */
#define FIT_ERR_NOMEM (-4)   /* the library could not allocate its scratch */

/* Per-track status bits. */
#define FIT_ST_NO_INTERSECTION 1u /* the surface is not reached; the track stops
                                     at its last good state */
#define FIT_ST_NOT_CONVERGED 2u   /* p2r path-length iteration hit max_iter */
#define FIT_ST_NONFINITE 4u       /* a non-finite value appeared; the track stops
                                     and its outputs are unspecified */
#define FIT_ST_CHARGE_FLIP 8u     /* an update made w negative: q and the sign of
                                     w (and row/column 3 of C) were flipped */

typedef enum { FIT_MODE_R = 0, FIT_MODE_Z = 1 } fit_mode;

/* Geometry and numerics of one mode (p2r or p2z). */
typedef struct {
  float B;           /* field along +z [T] */
  int nlayer;        /* number of surfaces, 1..FIT_MAX_LAYERS */
  const float* surf; /* HOST pointer: nlayer radii (p2r) or z positions (p2z)
                        [cm], in the order the tracks cross them; copied */
  int max_iter;      /* p2r: maximum path-length iterations (<= 0: 10) */
  float tol;         /* p2r: stop when a step is <= tol * R (<= 0: 1e-6) */
  int start;         /* p2r: where the path-length iteration starts, a FIT_START_*
                        value; 0 (a zeroed struct) is FIT_START_CROSSING */
} fit_config;

/* Start of the p2r path-length iteration (Sec. 3.2: the iteration advances
 * the track in straight-line steps to the cylinder).  Both converge to the
 * same crossing under the same tolerance; they differ in the steps taken.
 *   FIT_START_CROSSING: the crossing of the track's transverse circle with the
 *     cylinder in closed form (a quadratic in tan of half the turning angle),
 *     where the start is inside the cylinder and the track turns by less than
 *     0.49 rad on the way; the first step then confirms it.  Elsewhere, the
 *     straight-line start.
 *   FIT_START_LINE: the straight-line distance along the initial direction. */
#define FIT_START_CROSSING 0
#define FIT_START_LINE 1

typedef struct fit_handle fit_handle;

/* Input tracks (read only). */
typedef struct {
  const float* par; /* [6][ld]  */
  const float* cov; /* [21][ld] */
  const int32_t* q; /* [ld]     */
  int64_t ld;
} fit_tracks_in;

/* Output tracks.  par/cov/q may alias the inputs (in-place fit). */
typedef struct {
  float* par;        /* [6][ld]  fitted state after the last layer */
  float* cov;        /* [21][ld] */
  int32_t* q;        /* [ld]     */
  float* chi2;       /* [ld]     sum over layers of the update chi2 */
  float* chi2_layer; /* [nlayer][ld] per-layer chi2, or NULL */
  uint8_t* status;   /* [ld]     FIT_ST_* bits, or NULL */
  int64_t ld;
} fit_tracks_out;

/* Hits: one per track and layer (paper Sec. 3.1). */
typedef struct {
  const float* pos; /* [nlayer][3][ld]  x, y, z */
  const float* cov; /* [nlayer][6][ld]  packed 3x3 */
  int64_t ld;
} fit_hits;

/* What fit_sync reports: counters accumulated since the previous fit_sync. */
typedef struct {
  uint64_t tracks;          /* tracks processed */
  uint64_t no_intersection; /* tracks with FIT_ST_NO_INTERSECTION */
  uint64_t not_converged;   /* ... FIT_ST_NOT_CONVERGED */
  uint64_t nonfinite;       /* ... FIT_ST_NONFINITE */
  uint64_t charge_flip;     /* ... FIT_ST_CHARGE_FLIP */
  uint64_t iterations;      /* p2r path-length iterations, summed over tracks
                               and layers */
} fit_status;

/*
 * fit_init: creates a handle on CUDA device `device` for the two modes.
 * cfg_r / cfg_z describe the p2r cylinders and the p2z planes; either may be
 * NULL if that mode is never used.  The handle allocates its own small device
 * scratch (status counters) and creates a second CUDA stream with two events
 * (see fit_propagate_update); fit_destroy frees them.
 * Errors: FIT_ERR_ARG (bad config), FIT_ERR_CUDA, FIT_ERR_NOMEM.
 */
int fit_init(fit_handle** h, const fit_config* cfg_r, const fit_config* cfg_z, int device);

/*
 * fit_propagate_update: the fused hot path (paper Sec. 3.1-3.2).  The tracks
 * are nevt events stored one after another: event e holds ntrk[e] tracks
 * (HOST array) and uses mode[e] (HOST array of fit_mode).  For every track
 * and for l = 0..nlayer-1: propagate (p, C) to surface l of its mode, then
 * update with hit l.  Track t of the concatenation reads in.par[k*in.ld + t],
 * hits.pos[(l*3 + k)*hits.ld + t], ... and writes out.par[k*out.ld + t], ...
 * nlayer must equal the configured nlayer of every mode used.
 * Consecutive events of the same mode run as one kernel launch.  A call with
 * events of both modes runs its p2z launches on the handle's second stream,
 * forked from `stream` before them and joined back after them, so that they
 * overlap the p2r launches; `stream` follows the whole call as before.  Calls
 * on one handle from several host threads take turns for that stream.
 * Errors: FIT_ERR_ARG (NULL pointer, misaligned pointer or ld, sizes out of
 * range, unconfigured mode), FIT_ERR_CUDA (launch failure).
 */
int fit_propagate_update(fit_handle* h, const fit_tracks_in* in, const fit_tracks_out* out,
                         const fit_hits* hits, int nevt, const int64_t* ntrk, int nlayer,
                         const int32_t* mode, void* stream);

/*
 * fit_sync: waits for the work queued by this handle on `stream`, then reads
 * and clears the handle's counters into *st (st may be NULL).  timeout_s <= 0
 * waits without limit; otherwise the wait polls and returns FIT_ERR_TIMEOUT
 * after timeout_s seconds (the work is still queued; call again).
 */
int fit_sync(fit_handle* h, void* stream, double timeout_s, fit_status* st);

/*
 * fit_propagate_update_noalloc: the same fused fit as fit_propagate_update,
 * for callers that cannot allocate device memory.  (The paper has no
 * counterpart; it is an addition of this library.)
 *
 * Who needs it: a process that reserves all of its GPU memory when it starts
 * and must not allocate while it processes events -- an online trigger farm,
 * for example -- or a plug-in running inside a host framework that owns the
 * device memory.  fit_init allocates a counter block with cudaMalloc, so such
 * callers cannot create a handle.  This entry point takes the geometry
 * directly, allocates nothing (no cudaMalloc, no cudaFree, no allocating
 * library call), and keeps its scratch -- per-event status counters and the
 * event offsets -- in a fixed array compiled into the library: 192 KiB that
 * every GPU which loads the library holds until the process exits.
 *
 * Arguments as fit_propagate_update, except:
 *   cfg_r, cfg_z  geometry of the modes used (either may be NULL), as for
 *                 fit_init; validated on every call.
 *   nevt          at most FIT_NOALLOC_MAX_EVENTS; a larger value returns
 *                 FIT_ERR_ARG without touching the GPU (split the events over
 *                 several calls).
 *   per_event     HOST array of nevt fit_status, or NULL.  If given, the call
 *                 waits for its work on `stream` and fills entry e with the
 *                 counts of event e (tracks = ntrk[e]).  If NULL the call
 *                 does not wait for its kernels; but the event offsets are
 *                 copied to the device from a local (pageable) host array,
 *                 and for such a copy the CUDA driver may wait for the work
 *                 queued earlier on `stream` before the call returns.
 * The work runs on the current CUDA device.  The first call on a device looks
 * up the device address of the fixed array (once per device).  That first
 * call may also be where CUDA loads the library's kernels onto the device
 * (with lazy module loading, CUDA's default), which allocates device memory
 * for their code and for the fixed array: make the first call while the
 * process may still allocate (at start-up), or set CUDA_MODULE_LOADING=EAGER
 * so that loading happens when the library is loaded.  Later calls allocate nothing.  Every call shares the one
 * array and each call clears the counters of its own events before its
 * kernels run, so calls whose work overlaps on the GPU (other streams, other
 * host threads) race on it: serialise them.
 */
#define FIT_NOALLOC_MAX_EVENTS 4096

int fit_propagate_update_noalloc(const fit_config* cfg_r, const fit_config* cfg_z,
                                 const fit_tracks_in* in, const fit_tracks_out* out,
                                 const fit_hits* hits, int nevt, const int64_t* ntrk, int nlayer,
                                 const int32_t* mode, void* stream, fit_status* per_event);

/*
 * Batched form (many events of uneven size and mixed modes in one launch).
 *
 * A plan fixes the event structure (ntrk[], mode[], nlayer) once.  Its work is
 * cut into items -- tiles of one event, 2 x threads_per_block tracks -- that a
 * persistent kernel's blocks pull from a counter until none is left, so the
 * uneven events and the two surface types share one launch.  fit_plan_run
 * captures that launch (and the counter reset) in a CUDA graph the first time
 * it sees a set of buffers and replays the graph afterwards.  The results are
 * those of fit_propagate_update on the same events.
 */
typedef struct {
  int threads_per_block; /* 32, 64, 128 or 256 (64, 128 or 256 with one track per thread) */
  int blocks_per_sm;     /* grid = blocks_per_sm x SM count; 0 = as many as fit */
  int persistent;        /* 1: one persistent launch; 0: one launch per run of
                            same-mode events (fit_propagate_update's form) */
  int tracks_per_thread; /* 2 (or 0, a zeroed struct): two tracks per thread in
                            packed f32x2 instructions; 1: one track per thread
                            (persistent form only) */
  int layout;            /* how the plan reads the caller's track and hit arrays:
                            FIT_LAYOUT_SOA (0, a zeroed struct) or
                            FIT_LAYOUT_AOSOA32 (see fit_propagate_update_layout);
                            at fit_plan_create also FIT_LAYOUT_TUNE: run as SoA
                            until fit_plan_tune picks one of the two */
} fit_launch_config;

typedef struct {
  fit_launch_config config; /* the launch shape the plan runs with */
  int64_t tracks;           /* tracks in the plan */
  int32_t items;            /* work items of the persistent form */
  int32_t tuned;            /* 0: default or given; 1: measured by fit_plan_tune;
                               2: taken from the tuning cache */
  float best_ms;            /* fit_plan_tune: time of the chosen shape, else 0 */
} fit_plan_info;

typedef struct fit_plan fit_plan;

/*
 * fit_plan_create: a plan for nevt events (ntrk, mode: HOST arrays, copied).
 * cfg may be NULL (persistent, 128 threads per block, two tracks per thread,
 * as many blocks per SM as fit).  The plan allocates its work-item table and a counter on the
 * handle's device.  Errors: FIT_ERR_ARG, FIT_ERR_NOMEM, FIT_ERR_CUDA.
 */
int fit_plan_create(fit_handle* h, int nevt, const int64_t* ntrk, const int32_t* mode, int nlayer,
                    const fit_launch_config* cfg, fit_plan** plan);

/*
 * fit_plan_run: the fused fit of the plan's events on these buffers (layouts
 * as fit_propagate_update), asynchronous on `stream`; counts into the handle's
 * counters (fit_sync).
 */
int fit_plan_run(fit_plan* plan, const fit_tracks_in* in, const fit_tracks_out* out,
                 const fit_hits* hits, void* stream);

/*
 * fit_plan_tune: the autotuner (paper Sec. 5: hand-set launch parameters were
 * worth ~30 %, registers per thread ~10 %).  Times every candidate launch
 * shape -- persistent with two tracks per thread and 32, 64, 128 or 256 threads
 * per block, or one track per thread and 64, 128 or 256 threads per block,
 * each at every resident-block count, and the per-segment form -- on these
 * buffers (out must not alias in; it is written) and keeps the fastest.  The
 * buffers are in the plan's layout.  A plan created with FIT_LAYOUT_TUNE
 * passes SoA buffers and has every shape timed in both layouts (the AoSoA runs
 * read a converted copy of the inputs in scratch device memory, about 4 bytes
 * x (54 + 10 nlayer) per track, allocated and freed by the call); afterwards
 * the plan runs in the layout chosen (fit_plan_get_info) and fit_plan_run
 * takes buffers in that layout (fit_relayout converts).  A shape found before
 * for the same device, layout choice, depth and event-size histogram (in this
 * process, or in the text file cache_path if not NULL) is reused without
 * measuring; new results are appended to cache_path.  Waits for the stream.
 * The tuning runs do not count into the handle.
 */
int fit_plan_tune(fit_plan* plan, const fit_tracks_in* in, const fit_tracks_out* out,
                  const fit_hits* hits, void* stream, const char* cache_path);

/* fit_plan_get_info: the plan's launch shape and sizes. */
int fit_plan_get_info(const fit_plan* plan, fit_plan_info* info);

/* fit_plan_destroy: frees the plan (after its pending work ends). */
void fit_plan_destroy(fit_plan* plan);

/*
 * fit_relayout: copies rows x n 4-byte elements (float or int32; component k
 * of track t) from the DEVICE array src in layout src_layout (FIT_LAYOUT_SOA
 * or FIT_LAYOUT_AOSOA32, leading dimension src_ld) into the DEVICE array dst
 * in dst_layout (dst_ld); src and dst must not overlap.  For the track and
 * hit arrays of a plan whose tuner chose AoSoA: par (rows 6), cov (21), hit
 * positions (3 x nlayer), hit covariances (6 x nlayer), per-layer chi2
 * (nlayer); arrays of one component per track (q, chi2, status) are the same
 * in both layouts.  ld >= n, and a multiple of 32 in FIT_LAYOUT_AOSOA32.
 * Asynchronous on `stream`.  Errors: FIT_ERR_ARG, FIT_ERR_CUDA.
 */
int fit_relayout(const void* src, int64_t src_ld, int src_layout, void* dst, int64_t dst_ld,
                 int dst_layout, int rows, int64_t n, void* stream);

/*
 * Gradient of each track's summed chi2 with respect to its hit positions and
 * its initial parameters (and covariance): a reverse sweep over the layers,
 * written by hand, from per-layer checkpoints.
 *
 * fit_tape_bytes: size of the tape for nlayer layers and leading dimension ld
 * (per track and layer the state at the layer's entry -- 6 parameters, 21
 * covariance entries, the charge before and after the update, as floats --
 * then one int32 per track, the number of layers it completed).
 *
 * fit_adjoint_forward: as fit_propagate_update (same arguments and outputs;
 * out->ld must equal hits->ld), one track per thread, and writes the tape
 * (DEVICE, caller-owned, fit_tape_bytes(nlayer, out->ld) bytes, 16-byte
 * aligned).  Counts into the handle like fit_propagate_update.
 *
 * fit_adjoint_backward: for every track t of the events, with weight
 * grad_chi2[t] (the derivative of the caller's loss with respect to the
 * track's summed chi2), writes
 *   grad_hpos[(l*3 + k)*ld + t] = grad_chi2[t] * d chi2_t / d hit_pos[l][k]
 *   grad_par0[k*ld + t]        = grad_chi2[t] * d chi2_t / d par_in[k]
 *   grad_cov0[k*ld + t]        = grad_chi2[t] * d chi2_t / d cov_in[k]
 *                                (packed entry k; grad_cov0 may be NULL)
 * from the tape of a fit_adjoint_forward on the same inputs (ld = hits->ld).
 * Layers a track did not complete contribute nothing.  All pointers DEVICE.
 */
size_t fit_tape_bytes(int nlayer, int64_t ld);
int fit_adjoint_forward(fit_handle* h, const fit_tracks_in* in, const fit_tracks_out* out,
                        const fit_hits* hits, int nevt, const int64_t* ntrk, int nlayer,
                        const int32_t* mode, void* tape, void* stream);
int fit_adjoint_backward(fit_handle* h, const fit_hits* hits, int nevt, const int64_t* ntrk,
                         int nlayer, const int32_t* mode, const void* tape, const float* grad_chi2,
                         float* grad_hpos, float* grad_par0, float* grad_cov0, void* stream);

/*
 * fit_propagate_update_layout: fit_propagate_update with the track and hit
 * arrays in one of two layouts (paper Sec. 3.2 describes the test codes'
 * Matriplex-style layout: tracks in blocks of bsize, each component of a
 * block contiguous):
 *   FIT_LAYOUT_SOA     structure of arrays, component k of track t at
 *                      base[k * ld + t] (what every other entry point takes);
 *   FIT_LAYOUT_AOSOA32 tiles of 32 consecutive tracks (of the events laid end
 *                      to end): component k of track t at
 *                      base[((t / 32) * K + k) * 32 + t % 32], K the number of
 *                      components per track of that array (6 for par, 21 for
 *                      cov, 3 nlayer for hit positions with k = 3 l + j,
 *                      6 nlayer for hit covariances, nlayer for chi2_layer, 1
 *                      for q, chi2 and status, which are then plain arrays).
 *                      ld is the number of track slots, a multiple of 32.
 * The arithmetic is the same; the results are bit-identical.  Not with the
 * learned seed attached (FIT_ERR_ARG).
 */
#define FIT_LAYOUT_SOA 0
#define FIT_LAYOUT_AOSOA32 1
#define FIT_LAYOUT_TUNE 2 /* fit_plan_create only: let fit_plan_tune choose */
int fit_propagate_update_layout(fit_handle* h, const fit_tracks_in* in, const fit_tracks_out* out,
                                const fit_hits* hits, int nevt, const int64_t* ntrk, int nlayer,
                                const int32_t* mode, int layout, void* stream);

/*
 * FP64 variant.  The paper's test codes computed in double unless told
 * otherwise (Sec. 5 runs p2r in FP32 only where double is emulated); this is
 * the same fused fit with every floating-point operation in IEEE double, one
 * track per thread, on double buffers of the same layouts (track index
 * fastest, ld >= tracks; pointers 8-byte aligned).  Geometry, iteration limit
 * and tolerance are the handle's; the field enters as kA * B in double.
 * The p2r Jacobian is taken at the iteration's last iterate, one step (at most
 * tol * R) short of the root, a relative error of ~kappa * tol * R: configure
 * p2r with tol ~1e-12 for a double fit (the FP32 default 1e-6 limits it to
 * ~1e-6).  Outputs, status bits and counters as fit_propagate_update.
 */
typedef struct {
  const double* par;  /* [6][ld] */
  const double* cov;  /* [21][ld] */
  const int32_t* q;   /* [ld] */
  int64_t ld;
} fit_tracks_in_f64;

typedef struct {
  double* par;        /* [6][ld] */
  double* cov;        /* [21][ld] */
  int32_t* q;         /* [ld] */
  double* chi2;       /* [ld] */
  double* chi2_layer; /* [nlayer][ld] or NULL */
  uint8_t* status;    /* [ld] or NULL */
  int64_t ld;
} fit_tracks_out_f64;

typedef struct {
  const double* pos;  /* [nlayer][3][ld] */
  const double* cov;  /* [nlayer][6][ld] */
  int64_t ld;
} fit_hits_f64;

int fit_propagate_update_f64(fit_handle* h, const fit_tracks_in_f64* in,
                             const fit_tracks_out_f64* out, const fit_hits_f64* hits, int nevt,
                             const int64_t* ntrk, int nlayer, const int32_t* mode, void* stream);

/*
 * Track finding.  The paper's test codes take the one hit given on each layer;
 * the pattern recognition around them (mkFit, Sec. 3) chooses it among
 * several.  fit_find_tracks does that choice inside the fused fit: on each
 * layer the track is propagated, every candidate hit is tried against the
 * prediction (chi2 = r^T S^-1 r of the update it would make), and the
 * candidate with the smallest chi2 strictly below chi2_gate (the lowest
 * index among equal chi2) updates the track; if none qualifies the track keeps
 * its prediction and the layer adds nothing to chi2.  chosen [nlayer][ld_out]
 * (DEVICE int8) receives the candidate taken on each layer, or -1 (also for
 * layers a stopped track did not reach).  Candidates: positions
 * [nlayer][ncand][3][ld] and covariances [nlayer][ncand][6][ld], track
 * fastest, 1 <= ncand <= 16.  One track per thread; outputs, status bits and
 * counters as fit_propagate_update.  fit_find_tracks_f64: the same in double.
 */
typedef struct {
  const float* pos;
  const float* cov;
  int32_t ncand;
  int64_t ld;
} fit_candidates;

typedef struct {
  const double* pos;
  const double* cov;
  int32_t ncand;
  int64_t ld;
} fit_candidates_f64;

int fit_find_tracks(fit_handle* h, const fit_tracks_in* in, const fit_tracks_out* out,
                    const fit_candidates* cand, float chi2_gate, int8_t* chosen, int nevt,
                    const int64_t* ntrk, int nlayer, const int32_t* mode, void* stream);
int fit_find_tracks_f64(fit_handle* h, const fit_tracks_in_f64* in, const fit_tracks_out_f64* out,
                        const fit_candidates_f64* cand, double chi2_gate, int8_t* chosen,
                        int nevt, const int64_t* ntrk, int nlayer, const int32_t* mode,
                        void* stream);

/*
 * fit_propagate_update_host: fit_propagate_update on HOST buffers (same
 * structs, layouts and checks; every data pointer in in, out and hits is a
 * host pointer, page-locked for the copies to overlap the kernels -- pageable
 * memory works but serialises).  The library cuts the tracks into chunks of
 * up to FIT_HOST_CHUNK and moves each through one of three device staging
 * sets on one of three internal streams: copy in, fit, copy out, so that one
 * chunk's copies overlap the others' fits (the paper's transfers of Sec. 3.1
 * and its measurement with them included).  A chunk's rows are 2-D copies of
 * FIT_HOST_CHUNK x 4 bytes per row; narrower rows cost the copy engine
 * bandwidth (512 KiB rows moved 186 GB/s where 1 MiB rows move 207).  Asynchronous on `stream` like
 * fit_propagate_update: the host buffers must stay valid and unchanged until
 * the stream passes the call (fit_sync).  The staging (about 1 KiB per track
 * of a chunk and per 20 layers, three times) is allocated on first use and
 * kept by the handle.  Per-chunk results are bit-identical to fit_propagate_update.
 */
#define FIT_HOST_CHUNK 262144
int fit_propagate_update_host(fit_handle* h, const fit_tracks_in* in, const fit_tracks_out* out,
                              const fit_hits* hits, int nevt, const int64_t* ntrk, int nlayer,
                              const int32_t* mode, void* stream);

/*
 * fit_propagate_update_mapped: fit_propagate_update on page-locked HOST
 * buffers that the fused kernel reads and writes in place, over the host
 * link, without staging copies (zero-copy; on a Grace host the NVLink-C2C
 * link).  Same structs, layouts, checks and results as fit_propagate_update
 * (bit-identical: the same kernels run on the same values).  Every data
 * pointer must lie in page-locked host memory (cudaHostAlloc, or
 * cudaHostRegister'ed) that the handle's device reaches under the same
 * address; each is checked with cudaPointerGetAttributes and a pointer that
 * is not returns FIT_ERR_ARG before anything runs.  Asynchronous on `stream`:
 * the host buffers must stay valid, and the outputs unread, until the stream
 * passes the call (fit_sync).  Allocates nothing.  This is the host-path
 * counterpart of the paper's transfer measurement (Sec. 3.1, Sec. 5) for a
 * device that shares a coherent link with its host.
 */
int fit_propagate_update_mapped(fit_handle* h, const fit_tracks_in* in, const fit_tracks_out* out,
                                const fit_hits* hits, int nevt, const int64_t* ntrk, int nlayer,
                                const int32_t* mode, void* stream);

/*
 * Learned path-length seed for p2r.  The paper's p2r finds the path length to
 * the cylinder by discrete straight-line steps (Sec. 3.2); these entry points
 * add a small network, 8 -> 64 -> 64 -> 1 with ReLU, BF16 weights and FP32
 * accumulation on the tensor cores, whose output starts that iteration closer
 * to the root.  The iteration then runs exactly as without it (same
 * tolerance, same result within it): the network only changes where it
 * starts, and a seed that is not finite or further than a quarter of the
 * straight-line distance from it is replaced by the straight-line seed.  The
 * paper has no network; this is an addition.
 *
 * Inputs of one sample (a track state p, charge q, target radius R), in the
 * frame whose x axis points along the track's transverse position:
 *   x[0] = r0 / R, x[1] = z / R, x[2] = kA B w R / 2, x[3] = cos psi,
 *   x[4] = sin psi, x[5] = cos theta, x[6] = q, x[7] = R / 100 cm,
 * with r0 = sqrt(x^2 + y^2), psi = phi - atan2(y, x), kA = 0.00299792458.
 * Target: g = (h - h_line) / (kappa h_line^2 / 2), h the exact transverse path
 * length, h_line the straight-line distance along the momentum to the
 * cylinder, kappa = -q kA B w; the seed is h_line + g kappa h_line^2 / 2.
 *
 * Parameters: FIT_MLP_PARAMS floats, W1[64][8], b1[64], W2[64][64], b2[64],
 * W3[64], b3 (W[out][in]); the master copy is FP32, the forward pass rounds
 * weights and activations to BF16 (round to nearest even) and each input to a
 * pair of BF16 numbers hi = bf16(x), lo = bf16(x - hi).
 */
#define FIT_MLP_INPUTS 8
#define FIT_MLP_HIDDEN 64
#define FIT_MLP_PARAMS 4801

typedef struct fit_mlp fit_mlp;

typedef struct {
  int epochs;      /* passes over the samples */
  int batch;       /* samples per Adam step, 64..65536 */
  float lr;        /* learning rate of the first step ... */
  float lr_final;  /* ... decayed along a half cosine to this at the last */
  float beta1, beta2, eps; /* Adam (Kingma and Ba, 2015) */
  uint64_t seed;   /* order of the batches */
} fit_mlp_train_config;

/*
 * fit_mlp_create: a network on `device` with He-uniform weights drawn from
 * `seed` and zero biases; Adam state zero.  fit_mlp_destroy frees it.
 */
int fit_mlp_create(fit_mlp** m, int device, uint64_t seed);
void fit_mlp_destroy(fit_mlp* m);

/* fit_mlp_set_params / get_params: the FP32 master parameters, HOST arrays of
 * FIT_MLP_PARAMS floats.  set_params also resets the Adam state. */
int fit_mlp_set_params(fit_mlp* m, const float* params);
int fit_mlp_get_params(const fit_mlp* m, float* params);

/*
 * fit_mlp_prepare: the inputs x (DEVICE, [n][8] row-major) of n samples --
 * states par ([6][ld], track fastest), charges q [n], target radii R [n] --
 * for field B; with h_exact (DEVICE [n], the exact path lengths) also the
 * targets (DEVICE [n]); a sample with no straight-line crossing from inside
 * the cylinder, or kappa = 0, gets a NaN target, which training skips.
 */
int fit_mlp_prepare(float B, const float* par, int64_t ld, const int32_t* q, const float* R,
                    const float* h_exact, int64_t n, float* x, float* target, void* stream);

/* fit_mlp_forward: the network's output y [n] (DEVICE) for inputs x [n][8]. */
int fit_mlp_forward(const fit_mlp* m, const float* x, int64_t n, float* y, void* stream);

/*
 * fit_mlp_gradient: the gradient (DEVICE [FIT_MLP_PARAMS]) of the mean squared
 * error L = (1/n) sum_i (y_i - target_i)^2 over the n samples with finite
 * targets (the rounding to BF16 passes gradients through unchanged), and L
 * itself (DEVICE [1]).  1 <= n <= 65536.
 */
int fit_mlp_gradient(fit_mlp* m, const float* x, const float* target, int64_t n, float* grad,
                     float* loss, void* stream);

/* fit_mlp_adam_step: one Adam update of the master parameters with the
 * gradient grad (DEVICE), learning rate lr and the network's Adam settings
 * (beta1 0.9, beta2 0.999, eps 1e-8 unless fit_mlp_train set others). */
int fit_mlp_adam_step(fit_mlp* m, const float* grad, float lr, void* stream);

/*
 * fit_mlp_train: minimises the mean squared error of the network's output
 * against the targets by Adam over `epochs` passes of batches of cfg->batch
 * consecutive samples (from a per-epoch offset drawn from cfg->seed; n must
 * be >= cfg->batch).  Each step is one forward+backward kernel, one Adam
 * kernel and one kernel that rebuilds the BF16 weights, on `stream`.  loss_per_epoch (HOST [epochs], may be NULL) receives the
 * mean training loss of each epoch; the call then waits for the stream.
 */
int fit_mlp_train(fit_mlp* m, const float* x, const float* target, int64_t n,
                  const fit_mlp_train_config* cfg, float* loss_per_epoch, void* stream);

/*
 * fit_mlp_attach: the handle's p2r fits (fit_propagate_update) and
 * fit_path_lengths seed from the network's current weights (a copy taken on
 * `stream`); m = NULL detaches.  An attached handle runs p2r with one track
 * per thread so that each warp evaluates the network on its 32 tracks
 * together; fit_plan_*, fit_adjoint_* and fit_propagate_update_noalloc do
 * not use the seed.
 */
int fit_mlp_attach(fit_handle* h, const fit_mlp* m, void* stream);

/*
 * fit_path_lengths: the p2r path-length iteration alone, for n independent
 * states par ([6][ld]) with charges q [n] to their own radii R [n], with the
 * handle's p2r tolerance and iteration limit: h_out [n] the path length
 * (NaN when the cylinder is not reached), iters_out [n] (may be NULL) the
 * iterations taken.  seeded = 1 starts from the attached network (FIT_ERR_ARG
 * if none), 0 from the handle's p2r start (fit_config.start).  All DEVICE.
 */
int fit_path_lengths(fit_handle* h, const float* par, int64_t ld, const int32_t* q,
                     const float* R, int64_t n, float* h_out, int32_t* iters_out, int seeded,
                     void* stream);

/* fit_destroy: frees the handle and its scratch (after pending work ends). */
void fit_destroy(fit_handle* h);

/* fit_last_error: text of the last error on the calling thread ("" if none). */
const char* fit_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FIT_H_ */
