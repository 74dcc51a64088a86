/*
 * pond_checks.h -- measurement and self-check entry points of the GB300
 * Particles-on-Demand library.  None of them is a step of the method
 * (arXiv:2302.00310 has no counterpart): they measure this GPU and check the
 * step kernels' own arithmetic helpers against CUDA's correctly rounded
 * operations, so that tests and benchmarks can state both.
 *
 * Conventions as in pond.h: every call returns a pond_status; device arrays
 * are caller-owned CUDA device pointers on the current device; nothing is
 * allocated on the device except by pond_measure_fma_peak (a stream and two
 * events, released before it returns).
 */
#ifndef POND_CHECKS_H
#define POND_CHECKS_H

#include <stdint.h>

#include "pond.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Peak multiply-add throughput of the current device in TFLOP/s (a fused
 * multiply-add counting 2 flops): a kernel of independent fma chains in FP64
 * (precision POND_FP64) or FP32 (POND_FP32_MIXED), as many resident CTAs as
 * every SM holds, the loop lengthened until one launch lasts min_seconds/5;
 * the best of five launches of that length, and its duration in ms.  The
 * denominator of the step kernels' arithmetic roofline.  Synchronous; takes
 * about min_seconds.  Errors: POND_E_INVAL (precision, min_seconds outside
 * (0, 60]), POND_E_CUDA. */
pond_status pond_measure_fma_peak(int32_t precision, double min_seconds, double *tflops, double *ms);

/* The FP64 reciprocal the step kernels use in the van Leer limiter (the
 * hardware approximation refined by one Newton-Raphson step) beside CUDA's
 * correctly rounded __drcp_rn, for n device values y: r[i], r_ref[i].
 * Runs on `stream` (a cudaStream_t, NULL = legacy default stream) and
 * synchronises it.  Errors: POND_E_INVAL (n < 0 or above 2^31, NULL arrays),
 * POND_E_CUDA. */
pond_status pond_check_reciprocal(const double *y, double *r, double *r_ref, int64_t n, void *stream);

/* The step kernels' FP64 van Leer limiter (half the harmonic mean x y/(x+y)
 * when x y > 0, else 0: the limited slope of Sec. IV.A.2 without its factor 2)
 * beside the same expression with CUDA's correctly rounded division, for n
 * device pairs (x, y): l[i], l_ref[i].  Stream, synchronisation and errors as
 * pond_check_reciprocal. */
pond_status pond_check_vanleer(const double *x, const double *y, double *l, double *l_ref, int64_t n,
                               void *stream);

#ifdef __cplusplus
}
#endif

#endif /* POND_CHECKS_H */
