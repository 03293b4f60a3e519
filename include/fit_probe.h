/*
 * fit_probe.h -- measurement probes of libfit (C ABI).
 *
 * Not part of the fit.  The fused kernel's roofline is its FP32 rate against
 * the GPU's FP32 ceiling; the ceiling is derived from unit counts (SMs x 128
 * FP32 lanes x 2 flops x clock), and this probe measures it on the device the
 * fit runs on, with scalar and with packed (two-lane) fused multiply-adds, so
 * that the derived figure is checked rather than assumed.  The paper has no
 * counterpart (it reports throughput, not a roofline).
 */
#ifndef FIT_PROBE_H
#define FIT_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Threads per block of the probe. */
#define FIT_PROBE_THREADS 256

/*
 * fit_probe_fp32: launches an FP32 throughput kernel on the CURRENT device,
 * on `stream` (a cudaStream_t; NULL = the default stream), and returns at
 * once; time it with events on the same stream.
 *
 *   packed  0: every thread runs 16 independent chains of scalar fused
 *           multiply-adds (fma.rn.f32); 1: 16 chains of packed two-lane
 *           fused multiply-adds (fma.rn.f32x2), i.e. 32 FP32 FMAs per round.
 *   blocks  grid size (>= 1), FIT_PROBE_THREADS threads each.
 *   iters   rounds per thread (>= 1).
 *   out     DEVICE buffer of at least blocks x FIT_PROBE_THREADS floats
 *           (caller-owned); each thread writes the sum of its chains there
 *           so that no chain can be optimised away.
 *   flops   HOST pointer; receives the FP32 flops the launch performs
 *           (an FMA counts as 2): blocks x threads x iters x 16 x 2
 *           (x 2 again when packed).
 *
 * Returns FIT_OK (0), FIT_ERR_ARG (-1) on a bad argument, FIT_ERR_CUDA (-2)
 * if the launch fails (message in fit_last_error()).
 */
int fit_probe_fp32(int packed, int blocks, int iters, float* out, void* stream, double* flops);

#ifdef __cplusplus
}
#endif

#endif /* FIT_PROBE_H */
