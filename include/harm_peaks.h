/*
 * harm_peaks.h -- arithmetic-pipe microbenchmarks (libharm_peaks.so).
 *
 * The echo kernels are bound by FP32 arithmetic and instruction issue, not by
 * memory (the paper's method has no counterpart to this: it only fixes what the
 * echo path computes). Their roofline denominators are measured on the GPU that
 * runs them with these kernels: independent chains of FP32 FMA, packed FP32x2
 * FMA, FP64 FMA and __sinf (the special-function unit) per thread, on a grid of
 * `blocks` CTAs of 256 threads.
 */
#ifndef HARM_PEAKS_H
#define HARM_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HARM_PEAK_FFMA = 0,   /* fmaf chains: 2 flops per FMA */
    HARM_PEAK_FFMA2 = 1,  /* __ffma2_rn chains: 4 flops per instruction */
    HARM_PEAK_DFMA = 2,   /* fma (double) chains: 2 flops per FMA */
    HARM_PEAK_SINF = 3    /* __sinf chains: 1 evaluation each */
};

/* Launch benchmark `kind` on `stream` (a cudaStream_t, NULL = default stream):
   `blocks` CTAs of 256 threads, `iters` iterations of 8 chains per thread. Each
   thread writes one float to out_dev, which must hold blocks x 256 floats of
   device memory. Asynchronous; the caller times it (CUDA events on the stream).
   Returns 0, 1 for a bad argument, 2 for a launch error. */
int harm_peak_launch(int kind, int blocks, int iters, void *out_dev, void *stream);

/* Operations one such launch performs (flops, or __sinf evaluations). */
long long harm_peak_ops(int kind, int blocks, int iters);

#ifdef __cplusplus
}
#endif

#endif /* HARM_PEAKS_H */
