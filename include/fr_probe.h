/*
 * fr_probe.h — device throughput probe used to state the ALU roofline of the FP64 path.
 *
 * Not part of the FR method (the paper measures FLOP/s against its own machine's peak; this
 * probe measures this GPU's fused multiply-add throughput so the FP64 kernels can be reported
 * as a fraction of it).
 */
#ifndef FR_PROBE_H
#define FR_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * fr_probe_fma — run independent FMA chains on every SM of the current device and return the
 * measured rate in FLOP/s (2 per FMA) in *flops.  precision: 0 = FP64 (DFMA), 1 = FP32 (FFMA).
 * `iters` FMAs per chain (>= 1).  Synchronous; allocates and frees a small device buffer.
 * Returns 0 on success, non-zero on a CUDA error or bad argument.
 */
int32_t fr_probe_fma(int32_t precision, int32_t iters, double *flops);

#ifdef __cplusplus
}
#endif

#endif /* FR_PROBE_H */
