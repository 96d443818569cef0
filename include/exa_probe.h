/*
 * exa_probe.h -- measurement probe of the GB300 derivative-evaluation library.
 *
 * Not a callback of the paper's interface: this call measures a hardware rate that bounds the
 * library's FP64 kernels, so that their roofline is stated against a measured peak rather than a
 * derived one.  The generated FP64 evaluation kernels issue DFMA, DMUL and DADD instructions, all
 * on the FP64 pipe; on GB300 that pipe, not memory bandwidth, is their binding unit.
 */
#ifndef EXA_PROBE_H
#define EXA_PROBE_H

#include <stdint.h>

#include "exa.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Measures the FP64 fused multiply-add rate of `device`: a kernel of independent dependent-FMA
 * chains on every SM (resident CTAs x SM count, 256 threads each) is run once to warm up and size
 * the work, then timed with CUDA events over about target_ms milliseconds (clamped to 10..2000).
 * Outputs (host pointers, any may be NULL): *inst_per_s = thread-level DFMA instructions per
 * second (an FMA counts as one instruction and two flops), *ms = the timed kernel's duration,
 * *sms = the SM count used.  Synchronizes the device; allocates and frees one 8-byte device buffer.
 * Errors: EXA_E_INVALID (bad device ordinal), EXA_E_CUDA (a launch, allocation or timing call
 * failed); the outputs are then left untouched. */
exa_status exa_probe_fp64_fma(int32_t device, double target_ms, double *inst_per_s, double *ms,
                              int32_t *sms);

#ifdef __cplusplus
}
#endif
#endif /* EXA_PROBE_H */
