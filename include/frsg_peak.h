/*
 * frsg_peak.h - FMA throughput microbenchmark (libfrsg_peak.so).
 *
 * Not part of the FR-SG scheme: it measures the compute denominators that the stage
 * kernels' roofline fractions use (the FP64 form of the scheme is bound by the FP64 pipe).
 * It changes no clock or other GPU setting.
 */
#ifndef FRSG_PEAK_H
#define FRSG_PEAK_H

#ifdef __cplusplus
extern "C" {
#endif

/* Dense fused multiply-add throughput of the current device in TFLOP/s (2 flops per FMA),
 * FP64 (fp64 = 1) or FP32 (fp64 = 0): independent FMA chains in every thread of 8 CTAs of 256
 * threads per SM, iters rounds of 128 FMAs per thread, best of reps timed launches (CUDA
 * events) after one warm-up launch.  Allocates and frees one small device buffer.  Returns 0,
 * or 1 on a CUDA error or a bad argument (tflops unchanged). */
int frsg_peak_fma(int fp64, int iters, int reps, double* tflops);

#ifdef __cplusplus
}
#endif

#endif /* FRSG_PEAK_H */
