/*
 * msa_probe.h -- measurement aid of libmsa.so.  The paper has no counterpart:
 * this call times the integer instructions the Smith-Waterman cell update is
 * made of, so that the roofline of the DP kernels can be stated from a
 * measured issue rate rather than assumed.
 */
#ifndef MSA_PROBE_H
#define MSA_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSA_PROBE_VIADDMAX_S16X2 0   /* max(a+b, c) on two int16 lanes (DPX) */
#define MSA_PROBE_VIMAX3_S16X2   1   /* max(a, b, c) on two int16 lanes (DPX) */
#define MSA_PROBE_VIADDMAX_S32   2   /* max(a+b, c) on int32 (DPX) */
#define MSA_PROBE_PRMT           3   /* byte permute (profile unpacking) */

/* Run a throughput kernel of `op` on the current device (every SM, 2048
 * threads each, 8 independent dependency chains per thread) and report
 * instructions per second and per clock per SM (using the device's maximum
 * SM clock).  Outputs are host doubles.  Returns 0, MSA_EINVAL for an unknown
 * op, or MSA_ECUDA. */
int msa_probe_int_rate(int op, double *ops_per_sec_out, double *ops_per_clk_sm_out);

#ifdef __cplusplus
}
#endif

#endif /* MSA_PROBE_H */
