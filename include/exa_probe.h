/*
 * exa_probe.h -- measurement probe of the GB300 derivative-evaluation library.
 *
 * Not callbacks of the paper's interface: these calls measure hardware rates that bound the
 * library's work, so that it is stated against measured peaks rather than derived ones.  The
 * generated FP64 evaluation kernels issue DFMA, DMUL and DADD instructions, all on the FP64 pipe;
 * on GB300 that pipe, not memory bandwidth, is their binding unit.  The end-to-end call with host
 * buffers is bound by the host link.
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

/* Measures the host link of `device`: cudaMemcpyAsync between a page-locked host buffer and a
 * device buffer of `bytes` bytes each (clamped to 64 MiB..4 GiB), one warm-up copy each way, then
 * the best of three timed copies per direction (CUDA events).  Outputs (host pointers, any may be
 * NULL): host-to-device and device-to-host bytes per second.  The end-to-end calls of this library
 * (exa_eval_all_host) move their inputs and outputs over this link.  Allocates and frees both
 * buffers; synchronizes the device.  Errors: EXA_E_INVALID (bad device ordinal), EXA_E_OOM (an
 * allocation failed), EXA_E_CUDA (a copy or timing call failed); the outputs are then left
 * untouched. */
exa_status exa_probe_host_link(int32_t device, int64_t bytes, double *h2d_bytes_per_s,
                               double *d2h_bytes_per_s);

#ifdef __cplusplus
}
#endif
#endif /* EXA_PROBE_H */
