/*
 * mg_diag.h -- diagnostics of libmg.so used for roofline denominators.
 *
 * The paper reports throughput only (Tables 1-4); the ALU peaks that bound the
 * FP64 and FP32 matrix-element kernels are not in MEASURED_PEAKS-style copy or
 * GEMM measurements, so the library measures them itself with an FMA loop.
 */
#ifndef MG_DIAG_H
#define MG_DIAG_H

#ifdef __cplusplus
extern "C" {
#endif

#define MG_DIAG_FP32 0
#define MG_DIAG_FP64 1

/* Peak FMA throughput of the current device: a kernel of independent FMA
 * chains on every SM (grid = 8 CTAs x SM count), timed with CUDA events on a
 * private stream after one warm-up launch.  kind: MG_DIAG_FP32 or MG_DIAG_FP64.
 * *gflops receives 2 * FMAs / second / 1e9.  Synchronous.  Returns MG_OK,
 * MG_ERR_ARG or MG_ERR_CUDA (codes of mg.h). */
int mg_diag_fma_peak(int kind, double* gflops);

#ifdef __cplusplus
}
#endif

#endif /* MG_DIAG_H */
