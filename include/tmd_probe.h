/*
 * tmd_probe.h -- measurement support of the hard-to-round search library:
 * the issue-rate probe behind the integer-pipe roofline.  Not part of the
 * search path (the paper has no counterpart): it lives in its own shared
 * library, libtmd_probe.so, next to libtmd.so.
 */
#ifndef TMD_PROBE_H
#define TMD_PROBE_H

#include "tmd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Measured issue rates of the pipes the search runs on (no counterpart in the
 * paper: the measured denominator of the integer-pipe roofline).  Long
 * independent chains of one instruction kind per thread, 8 CTAs of 256
 * threads on every SM of `device`, timed by the SM cycle counter:
 * out[0..3] = lane-operations per SM per clock of 32-bit add, 3-input
 * logic, 32-bit multiply-add and FP32 fused multiply-add; out[4] (if
 * n_out > 4) = the SM clock in MHz during the add run.  Writes
 * min(n_out, 5) values.  Synchronises the device; allocates and frees
 * about 1.3 MB of device memory. */
tmd_status tmd_pipe_rates(int device, double* out, int n_out);

#ifdef __cplusplus
}
#endif

#endif /* TMD_PROBE_H */
