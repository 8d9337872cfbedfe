/*
 * arkcos_peaks.h -- measured arithmetic peaks of the current device (part of libarkcos.so).
 *
 * Roofline denominators for the kernels of the library that are bound by arithmetic rather
 * than by memory traffic: the FP32 FMA rate (ring FFT butterflies, the band contraction, the
 * coefficient generation on the CUDA cores), the FP64 FMA rate (the kernel-sample distances)
 * and the tcgen05 kind::tf32 product rate (the 3xTF32 coefficient generation and knot
 * projection, which issue three TF32 products per FP32 product).  The paper has no counterpart;
 * it reports no roofline.
 */
#ifndef ARKCOS_PEAKS_H
#define ARKCOS_PEAKS_H

#include "arkcos.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Runs a short isolated kernel on the current device and reports its arithmetic rate.
 * unit: 0 = FP32 FMA (fmaf, 2 flop each), 1 = packed two-lane FP32 FMA (2 x 2 flop per
 * instruction), 2 = FP64 FMA, 3 = tcgen05.mma kind::tf32 of M = 128, N = 256, K = 8 issued by
 * one thread per SM from shared memory into tensor memory (2 M N K flop each).  The kernel is
 * launched six times on `stream` (a cudaStream_t, NULL = legacy default stream) and timed with
 * CUDA events; the first launch warms up and *ms receives the best of the other five, *tflops
 * the flop of one launch over it.  Synchronises the stream and allocates a few bytes of device
 * memory for the duration of the call.  The tf32 kernel's completion wait is bounded (about a
 * second).  Errors: EINVAL (unit out of range, NULL outputs), ETIMEOUT (the wait gave up),
 * ECUDA. */
arkcos_status arkcos_measure_peak(int unit, double *tflops, double *ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ARKCOS_PEAKS_H */
