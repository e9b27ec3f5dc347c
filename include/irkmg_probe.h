/*
 * Arithmetic-peak probe shipped beside the irkmg library (libirkmg_probe.so):
 * the measured rates behind the ALU-bound rooflines that the benchmark
 * reports.  The paper has no counterpart; it is measurement support, not part
 * of the solver.
 */
#ifndef IRKMG_PROBE_H
#define IRKMG_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One timed launch (after one short warm-up launch) of 8 CTAs of 256 threads
 * per SM, each thread running eight independent chains of `iters` dependent
 * multiply-adds, on cuda_stream (a cudaStream_t; NULL = legacy default stream).
 * kind 0: FP64 FMA, kind 1: FP32 FMA (*ops_per_s in flop/s, 2 per FMA);
 * kind 2: mad.wide.s32, 32 × 32 → 64-bit integer multiply-add with a 64-bit
 * addend (*ops_per_s in multiply-adds per second).  The device is the current
 * one; a 64-byte buffer is allocated and freed.  Returns 0, or 1 (bad
 * arguments), 2 (allocation failed), 3 (a CUDA call failed). */
int irkmg_probe_peak(int kind, int64_t iters, void *cuda_stream, double *ops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* IRKMG_PROBE_H */
