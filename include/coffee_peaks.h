/* Throughput microbenchmarks of the current CUDA device (libcoffee.so).
 *
 * The rooflines of the library's kernels divide achieved work by a measured peak. The copy
 * bandwidth and the dense bf16 GEMM rate are measured outside the library; these entry points
 * measure the two rates that are not: the FP64 FMA rate (bound of the FP64 kernels) and the
 * tcgen05 MMA rate of one issuing thread per SM on shared-memory operands (bound of the
 * tensor-core kernels, per operand kind). They are measurement tools: no assembly path calls
 * them. Each call allocates a few bytes of device memory, launches a kernel twice on the legacy
 * default stream (the second launch is timed with CUDA events), synchronises and frees.
 * Errors: COFFEE_ERR_INVALID_ARG for a NULL result or an unsupported option,
 * COFFEE_ERR_CUDA / COFFEE_ERR_NOMEM from the runtime, COFFEE_ERR_TIMEOUT if the MMA loop's
 * bounded wait gave up; the message is in coffee_last_error(). */
#ifndef COFFEE_PEAKS_H
#define COFFEE_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* FP64 FMA rate: 8 blocks per SM x 256 threads, 8 independent FMA chains per thread.
 *   tflops  host, out: 2 flops per FMA / time, in TFLOP/s. */
int coffee_peak_fp64(double* tflops);

/* tcgen05.mma rate, cta_group::1, M = 128, N = n (128 or 256), one 32-byte K-step per
 * instruction (K = 8 for tf32, 16 for bf16), back-to-back into one TMEM accumulator, one CTA
 * per SM.
 *   precision  COFFEE_TF32 (kind::tf32) or COFFEE_BF16 (kind::f16 with bf16 operands)
 *   tflops     host, out: 2 M N K per instruction / time, in TFLOP/s. */
int coffee_peak_mma(int precision, int n, double* tflops);

#ifdef __cplusplus
}
#endif

#endif /* COFFEE_PEAKS_H */
