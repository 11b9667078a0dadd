/*
 * carbox_peaks.h - measurement utility of the library (not part of the
 * method; the paper has no counterpart).
 *
 * The solver's kernels are bound by the FP64 (and, in the mixed mode, FP32)
 * FMA pipes, so their roofline fractions divide by a measured FMA peak rather
 * than a nominal one. This probe provides it: a kernel whose threads run 8
 * independent chains of dependent FMAs.
 */
#ifndef CARBOX_PEAKS_H
#define CARBOX_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Launch the probe on `stream` (cudaStream_t as void*; asynchronous): `grid`
 * CTAs of `block` threads (a multiple of 32, <= 1024), `iters` iterations of 8
 * FMAs per thread, in FP64 (fp64 != 0) or FP32. sink: device buffer of at
 * least grid values of that type (never written for these constants, but it
 * keeps the result live). The caller times the launch (CUDA events on the
 * stream) and divides cbx_peak_fma_flops(grid, block, iters) by the time.
 * Returns 0, -1 for a bad argument, -2 if the launch failed.
 */
int cbx_peak_fma(int fp64, int grid, int block, int iters, void* stream, void* sink);

/* Flops of one probe launch: 2 * 8 * grid * block * iters. */
double cbx_peak_fma_flops(int grid, int block, int iters);

#ifdef __cplusplus
}
#endif

#endif /* CARBOX_PEAKS_H */
