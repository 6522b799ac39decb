/*
 * dg_probe.h -- measurement aid of the GB300 DG library: the sustained
 * fused multiply-add rate of this GPU's FP64 or FP32 pipe.
 *
 * The paper has no counterpart (it reports CPU wall-clock times only).  The
 * FP64 DG kernels of this library are bound by the FP64 pipe rather than by
 * HBM, so their roofline needs the pipe's peak on the GPU at hand; this call
 * measures it with independent FMA chains instead of relying on a nominal
 * figure.
 */
#ifndef DG_PROBE_H
#define DG_PROBE_H

#include "dg_swe.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Times a kernel of independent fused multiply-add chains (8 chains per
 * thread, 8 blocks of 256 threads per SM of the current device) on `stream`
 * (a cudaStream_t, NULL for the legacy default stream): five untimed launches,
 * then `repeats` launches timed together with CUDA events on that stream.
 *  precision: DG_PREC_FP64 or DG_PREC_FP32.
 *  repeats:   1 .. 1000.
 *  out_flops_per_second: receives 2 x FMAs / elapsed seconds (host pointer).
 * The kernel stores one value per thread (so that no chain is dead code)
 * into `scratch`, a device buffer of at least dg_probe_scratch_bytes() bytes
 * that the caller provides (the library allocates nothing) and that the call
 * overwrites.  Synchronizes the stream.
 * Returns DG_ERR_ARG for a bad precision, repeat count, or null pointers,
 * DG_ERR_CUDA if a CUDA call fails. */
dg_status dg_probe_fma_rate(int precision, int repeats, void *scratch, void *stream,
                            double *out_flops_per_second);

/* Bytes of device scratch dg_probe_fma_rate needs on the current device. */
size_t dg_probe_scratch_bytes(void);

#ifdef __cplusplus
}
#endif
#endif /* DG_PROBE_H */
