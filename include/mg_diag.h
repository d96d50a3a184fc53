/*
 * mg_diag.h -- diagnostics of libmg.so used for roofline denominators.
 *
 * The paper reports throughput only (Tables 1-4); the ALU peaks that bound the
 * FP64 and FP32 matrix-element kernels are not among the copy and GEMM peak
 * measurements of the hardware, so the library measures them itself with an
 * FMA loop.  The kernels of a multi-kernel ME call are timed one by one.
 */
#ifndef MG_DIAG_H
#define MG_DIAG_H

#include <stdint.h>

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

/* Dense FP16 tensor-core throughput of the current device, as the colour
 * kernels use it: one CTA per SM issues 16384 tcgen05.mma kind::f16 of
 * M = N = 128, K = 16 (FP16 operands in shared memory, FP32 accumulation in
 * tensor memory) back to back, timed with CUDA events on a private stream
 * after one shorter warm-up launch.  *tflops receives 2 M N K MMAs / second /
 * 1e12.  Synchronous.  Returns MG_OK, MG_ERR_ARG, MG_ERR_CUDA or
 * MG_ERR_TIMEOUT (the bounded wait for the MMAs ran out). */
int mg_diag_mma_peak(double* tflops);

typedef struct mg_process mg_process;

/* One mg_sigma call (same arguments, same kernels) with CUDA events recorded
 * on the stream before the first kernel and after every kernel, for
 * processes whose ME call launches two kernels per slice of the good
 * helicities (the two-phase mixed g g > t t~ g g g path: colour flows to a
 * workspace, then the tensor-core colour form).  Waits for the stream.
 * *ms_first / *ms_second receive the summed durations of the first and
 * second kernel of every slice, *slices the number of slices.  Any output may
 * be NULL.  MG_ERR_ARG for a handle without such a path or bad arguments. */
int mg_diag_sigma_phases(mg_process* h, const double* momenta_dev, int64_t nevt, double* me_out_dev, void* stream,
                         float* ms_first, float* ms_second, int* slices);

/* Bound of the first wait on every device barrier of this handle's kernels
 * (the bulk copy of the momenta tile, each tensor-core MMA): polls of
 * mbarrier.try_wait before the kernel gives up, sets a status bit (read with
 * mg_process_status: MG_ERR_TIMEOUT) and returns without writing its outputs.
 * The default, MG_DIAG_WAIT_POLLS, is never reached by a healthy launch; a
 * bound of 0 makes every such wait give up at once, so that a test can take
 * the timeout path on a healthy case.  After giving up, a kernel still waits
 * with the full default bound for the copy or MMA it started, so nothing is
 * left in flight.  Launches queued (and CUDA graphs captured) before the call
 * keep the bound they had.  Errors: MG_ERR_ARG (NULL handle). */
#define MG_DIAG_WAIT_POLLS (1u << 22)
int mg_diag_set_wait_polls(mg_process* h, uint32_t polls);

#ifdef __cplusplus
}
#endif

#endif /* MG_DIAG_H */
